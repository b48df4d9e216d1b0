"""Seeded synthetic Hermitian matrices in CSR form.

These are the inputs of the solver and of the oracle.  The module builds
matrices only; it holds none of the filter or eigensolver arithmetic.

Every generator returns a :class:`CSR` whose row pointer is int64, column
indices int32 (sorted within each row, both triangles stored) and values
float64 or complex128.  Lattice site (x, y[, z]) has index x + L*y (+ L*L*z).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import rng


@dataclass
class CSR:
    n: int
    rowptr: np.ndarray   # int64, n + 1
    colidx: np.ndarray   # int32, nnz
    vals: np.ndarray     # float64 or complex128, nnz
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.colidx.shape[0])

    @property
    def is_complex(self) -> bool:
        return np.iscomplexobj(self.vals)

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.vals, self.colidx.astype(np.int64), self.rowptr),
                             shape=(self.n, self.n))

    def to_dense(self) -> np.ndarray:
        return self.to_scipy().toarray()


def csr_from_coo(n: int, rows, cols, vals, meta=None) -> CSR:
    """Sort (row, col) entries and sum duplicates into CSR."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    key = rows * n + cols
    uniq, start = np.unique(key, return_index=True)
    summed = np.add.reduceat(vals, start) if vals.size else vals
    urow = uniq // n
    ucol = uniq % n
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, urow + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSR(n=n, rowptr=rowptr, colidx=ucol.astype(np.int32), vals=summed,
               meta=dict(meta or {}))


def _site_coords(L: int, dim: int):
    idx = np.arange(L ** dim, dtype=np.int64)
    coords = []
    for _ in range(dim):
        coords.append(idx % L)
        idx = idx // L
    return coords


def _site_index(coords, L: int) -> np.ndarray:
    out = np.zeros_like(coords[0])
    mult = 1
    for c in coords:
        out = out + c * mult
        mult *= L
    return out


def laplacian2d_dirichlet(L: int, seed: int, pot_halfwidth: float = 0.5) -> CSR:
    """2D 5-point Laplacian on an L x L grid with Dirichlet boundary plus a
    diagonal potential uniform in [-pot_halfwidth, pot_halfwidth].

    Diagonal 4 + V_i, off-diagonals -1 between grid neighbours.
    """
    n = L * L
    x, y = _site_coords(L, 2)
    site = np.arange(n, dtype=np.int64)
    pot = pot_halfwidth * (2.0 * rng.uniform(seed, rng.STREAM_POTENTIAL, site) - 1.0)
    rows = [site]
    cols = [site]
    vals = [4.0 + pot]
    for dx, dy in ((1, 0), (0, 1)):
        ok = (x + dx < L) & (y + dy < L)
        i = site[ok]
        j = _site_index([x[ok] + dx, y[ok] + dy], L)
        rows += [i, j]
        cols += [j, i]
        vals += [-np.ones(i.size), -np.ones(i.size)]
    return csr_from_coo(n, np.concatenate(rows), np.concatenate(cols),
                        np.concatenate(vals),
                        meta=dict(kind="laplacian2d_dirichlet", L=L, seed=seed,
                                  pot_halfwidth=pot_halfwidth))


def anderson(L: int, dim: int, W: float, seed: int, complex_phases: bool,
             t: float = 1.0) -> CSR:
    """Anderson model on a periodic L^dim lattice.

    On-site energy uniform in [-W/2, W/2]; nearest-neighbour hopping -t on each
    bond, times a Peierls phase e^{i theta}, theta ~ U[0, 2 pi), when
    ``complex_phases``.  Bond from site i to its +e_d neighbour j stores
    H[i, j] = -t e^{i theta} and H[j, i] = conj(H[i, j]).  Requires L >= 3.
    """
    if L < 3:
        raise ValueError("periodic lattice needs L >= 3")
    n = L ** dim
    coords = _site_coords(L, dim)
    site = np.arange(n, dtype=np.int64)
    eps = W * (rng.uniform(seed, rng.STREAM_POTENTIAL, site) - 0.5)
    rows = [site]
    cols = [site]
    vals = [eps.astype(np.complex128) if complex_phases else eps]
    for d in range(dim):
        nb = list(coords)
        nb[d] = (coords[d] + 1) % L
        j = _site_index(nb, L)
        if complex_phases:
            theta = 2.0 * np.pi * rng.uniform(seed, rng.STREAM_PHASE, site * dim + d)
            h = -t * np.exp(1j * theta)
        else:
            h = -t * np.ones(n)
        rows += [site, j]
        cols += [j, site]
        vals += [h, np.conj(h)]
    return csr_from_coo(n, np.concatenate(rows), np.concatenate(cols),
                        np.concatenate(vals),
                        meta=dict(kind="anderson", L=L, dim=dim, W=W, seed=seed,
                                  complex=bool(complex_phases), t=t))


# Central-difference weights of the second derivative, eighth order
# (Fornberg, Math. Comp. 51, 1988, table 1): offsets 0, +-1, +-2, +-3, +-4.
FD8_WEIGHTS = (-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0)


def ks_like_3d(L: int, seed: int, n_wells: int = 64, sigma: float = 1.5,
               depth: float = 1.0) -> CSR:
    """Real symmetric Kohn-Sham-like Hamiltonian on a periodic L^3 grid.

    -1/2 times the eighth-order finite-difference Laplacian (25 nonzeros per
    row, grid spacing 1) plus a local potential equal to a sum of n_wells
    negative Gaussians of width sigma at seeded centres (minimum-image
    distance).  Requires L >= 9.
    """
    if L < 9:
        raise ValueError("eighth-order periodic stencil needs L >= 9")
    n = L ** 3
    x, y, z = _site_coords(L, 3)
    site = np.arange(n, dtype=np.int64)
    centres = L * rng.uniform(seed, rng.STREAM_CENTRES,
                              np.arange(3 * n_wells, dtype=np.uint64)).reshape(n_wells, 3)
    pot = np.zeros(n)
    pos = np.stack([x, y, z], axis=1).astype(np.float64)
    for g in range(n_wells):
        d = pos - centres[g]
        d = d - L * np.round(d / L)
        pot -= depth * np.exp(-np.sum(d * d, axis=1) / (2.0 * sigma * sigma))
    rows = [site]
    cols = [site]
    vals = [-0.5 * 3.0 * FD8_WEIGHTS[0] + pot]
    coords = [x, y, z]
    for d in range(3):
        for off in range(1, 5):
            for sgn in (1, -1):
                nb = list(coords)
                nb[d] = (coords[d] + sgn * off) % L
                rows.append(site)
                cols.append(_site_index(nb, L))
                vals.append(np.full(n, -0.5 * FD8_WEIGHTS[off]))
    return csr_from_coo(n, np.concatenate(rows), np.concatenate(cols),
                        np.concatenate(vals),
                        meta=dict(kind="ks_like_3d", L=L, seed=seed, n_wells=n_wells,
                                  sigma=sigma, depth=depth))


def random_sparse_hermitian(n: int, nnz_per_row: int, seed: int, is_complex: bool) -> CSR:
    """Unstructured sparse Hermitian test matrix with a ragged row length mix.

    Each row i draws up to ``nnz_per_row`` random partner columns; entries are
    symmetrised (A + A^H)/2 so both triangles are stored.  Used to exercise the
    kernels on rows of uneven length and on a non-banded pattern.
    """
    rows_i = np.repeat(np.arange(n, dtype=np.int64), nnz_per_row)
    u = rng.uniform(seed, rng.STREAM_TEST, np.arange(rows_i.size * 3, dtype=np.uint64))
    cols_i = np.minimum((u[0::3] * n).astype(np.int64), n - 1)
    re = 2.0 * u[1::3] - 1.0
    im = 2.0 * u[2::3] - 1.0 if is_complex else 0.0
    v = re + 1j * im if is_complex else re
    diag = np.arange(n, dtype=np.int64)
    dval = 2.0 * rng.uniform(seed, rng.STREAM_POTENTIAL, diag) - 1.0
    rows = np.concatenate([rows_i, cols_i, diag])
    cols = np.concatenate([cols_i, rows_i, diag])
    vals = np.concatenate([0.5 * v, 0.5 * np.conj(v), dval.astype(v.dtype if is_complex else np.float64)])
    return csr_from_coo(n, rows, cols, vals,
                        meta=dict(kind="random_sparse", n=n, seed=seed, complex=is_complex))


def csr_to_sell(A: CSR, C: int, sigma: int):
    """Convert CSR to SELL-C-sigma (Kreutzer et al., SIAM J. Sci. Comput. 2014).

    Rows are sorted by decreasing length inside windows of ``sigma`` rows,
    grouped into chunks of C rows, and each chunk is stored column-major with
    its length padded to the longest row of the chunk (padding: column 0,
    value 0).  Returns (perm, chunk_ptr, chunk_len, colidx, vals): ``perm[r]``
    is the original row stored at sorted position r.
    """
    n = A.n
    lens = np.diff(A.rowptr)
    perm = np.arange(n, dtype=np.int64)
    for w0 in range(0, n, sigma):
        w1 = min(n, w0 + sigma)
        seg = perm[w0:w1]
        perm[w0:w1] = seg[np.argsort(-lens[seg], kind="stable")]
    nchunks = (n + C - 1) // C
    chunk_len = np.zeros(nchunks, dtype=np.int32)
    for c in range(nchunks):
        rs = perm[c * C:min(n, (c + 1) * C)]
        chunk_len[c] = lens[rs].max() if rs.size else 0
    chunk_ptr = np.zeros(nchunks + 1, dtype=np.int64)
    chunk_ptr[1:] = np.cumsum(chunk_len.astype(np.int64) * C)
    colidx = np.zeros(int(chunk_ptr[-1]), dtype=np.int32)
    vals = np.zeros(int(chunk_ptr[-1]), dtype=A.vals.dtype)
    for c in range(nchunks):
        for r in range(C):
            pos = c * C + r
            if pos >= n:
                continue
            row = perm[pos]
            s, e = A.rowptr[row], A.rowptr[row + 1]
            for t in range(e - s):
                colidx[chunk_ptr[c] + t * C + r] = A.colidx[s + t]
                vals[chunk_ptr[c] + t * C + r] = A.vals[s + t]
    return perm, chunk_ptr, chunk_len, colidx, vals
