/*
 * apf.h -- adaptive polynomial filtering for Hermitian interior eigenproblems
 * on one NVIDIA GB300 (sm_103a).  C ABI.
 *
 * The library computes every eigenpair (lambda, v) of a sparse Hermitian
 * matrix A with lambda in a given interval [a, b] (Sec. 1, Eq. (ori_problem)
 * of Xu, Ni, Li and Zhang, "Adaptive Polynomial Filtering for Hermitian
 * Interior Eigenproblems").  It runs filtered subspace iteration with the
 * adaptive, damped Chebyshev expansion of the step function as the filter
 * (Alg. 4, "AdaPolySI"): each outer step applies the filter by Clenshaw's
 * recurrence (Alg. 2), orthonormalises with Cholesky QR, performs
 * Rayleigh-Ritz, tests residuals, rejects spurious Ritz values (Eq. (tau_s))
 * and locks converged pairs.  Every step runs in this library's CUDA kernels.
 *
 * Conventions
 *  - Every function returns an apf_status; APF_OK (0) means success.
 *    apf_status_string() names a status.  On error, output arguments are
 *    left unchanged unless stated otherwise.
 *  - Dense blocks are row-major: element (i, c) of an n x p block with
 *    leading dimension ld sits at offset i*ld + c.  Complex values are
 *    interleaved (re, im) pairs of the real type.
 *  - "device" pointers are CUDA global-memory pointers on the context's
 *    device; "host" pointers are ordinary CPU memory.  The library never
 *    keeps a caller pointer beyond the call that received it.
 *  - All device work is ordered on the context's stream; calls that return
 *    host data synchronise that stream.
 *  - A context is not thread-safe: use one context per host thread.
 */
#ifndef APF_H
#define APF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  APF_OK = 0,
  APF_ERR_ARG = 1,             /* invalid argument (sizes, a > b, interval outside spectrum, ...) */
  APF_ERR_OOM = 2,             /* device allocation failed */
  APF_ERR_CUDA = 3,            /* a CUDA runtime call failed */
  APF_ERR_NOT_HERMITIAN = 4,   /* ingest found A != A^H beyond tolerance */
  APF_ERR_CHOL = 5,            /* Cholesky QR broke down even with the shifted retry */
  APF_ERR_NO_CONVERGENCE = 6,  /* max_iter reached; the result holds the pairs locked so far */
  APF_ERR_EIGH = 7,            /* the small dense eigensolver did not converge */
  APF_ERR_TIMEOUT = 8,         /* a device-side wait exceeded its time limit */
  APF_ERR_NOT_READY = 9        /* the object has no data of the requested kind */
} apf_status;

typedef enum {
  APF_R64 = 0,    /* real double */
  APF_C128 = 1    /* complex double (re, im) */
} apf_dtype;

typedef enum {
  APF_DAMP_LANCZOS_M = 0,  /* exponent-m Lanczos factors, Eq. (m_Lanczos_damping) (paper default) */
  APF_DAMP_JACKSON = 1,    /* Jackson factors, Sec. 2.2 */
  APF_DAMP_NONE = 2        /* no damping */
} apf_damping;

typedef enum {
  /* Filter recurrence in FP64 (complex FP64 for Hermitian A). */
  APF_FILTER_F64 = 0,
  /* Filter recurrence in FP32 with FP32 accumulation.  Accurate to about
   * 1e-7 relative: the residual stalls there (kept for comparison). */
  APF_FILTER_F32 = 1,
  /* FP32 recurrence on the defect: rho(A)V = V rho(Lambda) + D, where D
   * obeys the Clenshaw recurrence driven by the Ritz residual
   * R = A V - V Lambda.  The FP64 part is exact; the FP32 error scales with
   * ||R||, so the iteration converges to FP64 accuracy.  First outer step
   * (no Ritz values yet) uses APF_FILTER_F32. */
  APF_FILTER_F32_DEFECT = 2
} apf_filter_precision;

typedef struct apf_ctx apf_ctx;
typedef struct apf_matrix apf_matrix;
typedef struct apf_result apf_result;

/* Solver parameters.  apf_params_default() fills the paper's defaults
 * (Sec. 4): m = 0.5, tau_a = 1e-3, C = 1.4, k = ceil(2.5 k^(1)), tau_c = 1e-10. */
typedef struct {
  double a, b;              /* interval of interest, a < b */
  int64_t p;                /* subspace size (<= APF_MAX_P, <= n); 0: estimated, p = ceil(mu e~) (Sec. 3.4) */
  int32_t k_fixed;          /* 0: adaptive degree (Eq. (compute_k_1), Alg. 3); > 0: fixed degree */
  int32_t damping;          /* apf_damping */
  double C;                 /* Eq. (compute_k_1) constant, 1.4 */
  double k_ratio;           /* maximum degree k = ceil(k_ratio * k^(1)), 2.5 */
  double m_d;               /* damping exponent m of Eq. (m_Lanczos_damping), 0.5 */
  double tau_a;             /* adaptive threshold of Alg. 3, 1e-3 */
  double tau_c;             /* convergence threshold: lock when ||r|| <= tau_c ||A||, 1e-10 (||A||: apf_stats.norm_a) */
  int32_t max_iter;         /* outer iteration cap, 50 */
  int32_t lanczos_steps;    /* Lanczos steps for the spectrum bounds (Sec. 3.4), 40 */
  double bound_pad;         /* outward padding of the bounds, fraction of the Ritz spread, 0.01 */
  int32_t filter_precision; /* apf_filter_precision, APF_FILTER_F64 */
  int32_t spurious_rule;    /* 1: spurious-eigenvalue test of Alg. 4 (Sec. 3.3.2) on (default); 0: off */
  uint64_t seed;            /* seed of the initial block and Lanczos start vector */
  const void* init_block;   /* optional n x p initial block (row-major, ld = p); NULL: seeded */
  int32_t init_on_device;   /* 1 if init_block is a device pointer */
  int32_t max_degree_cap;   /* safety cap on the maximum degree k, 100000 */
  double mu;                /* p = ceil(mu e~) when p = 0 (Sec. 3.4), 1.8 */
  int32_t trace_probes;     /* probe vectors m of the count estimate e~, 32 */
  int32_t filter_graphs;    /* 1: replay recurring filter applications as CUDA graphs (default); 0: plain launches */
  int32_t gram_tensor_cores; /* 1: Gram products of CholQR / Rayleigh-Ritz on the tensor cores (apf_gram_tc, default); 0: FP64 cores */
} apf_params;

/* Statistics of one solve (the metrics of Table 2 plus per-stage times). */
typedef struct {
  int32_t iterations;        /* outer iterations run */
  int32_t k1, k_max;         /* initial degree k^(1) and maximum degree k */
  double avg_degree;         /* mean filter degree over the iterations */
  int64_t spmv_columns;      /* sparse matrix times vector products (columns), Table 2 "SpMVs" */
  int64_t filter_launches;   /* Clenshaw step kernels launched */
  int64_t gpu_launches;      /* all kernels launched by this solve */
  double lambda_min, lambda_max;  /* estimated spectrum bounds */
  double norm_a;             /* ||A|| of the convergence test: max |theta| over the Lanczos Ritz values (<= the spectral radius) */
  double ms_total, ms_setup, ms_filter, ms_orth, ms_rr, ms_check;  /* stage wall times */
  double filter_kernel_ms;   /* summed device time of the Clenshaw SpMM launches (CUDA events) */
  double filter_bytes;       /* algorithmic bytes of those launches */
  double max_residual;       /* max ||A v - lambda v|| / ||A|| over the returned pairs */
  int64_t filter_steps;      /* Clenshaw steps (a two-step launch counts 2) */
  double filter_step_bytes;  /* algorithmic bytes of the same steps run one per launch */
  double trace_estimate;     /* estimated eigenvalue count e~ (sum over slices), 0 if p was given */
  int64_t p_used;            /* subspace size used (sum over slices) */
  int32_t filter_kind;       /* FP32 Clenshaw step kernel of the first filter application (kinds as in
                                apf_matrix_set_filter_kernel, CSR reported as 3); -1 for the FP64 filter
                                and for a served request whose steps all ran in the batched launch */
  int32_t filter_g, filter_vpt;  /* its shape: lanes per row, 16-byte vectors per lane */
  int64_t filter_graph_replays;  /* filter applications replayed from a captured CUDA graph */
} apf_stats;

#define APF_MAX_P 1024
/* largest total subspace size of a batched solve (apf_solve_slices) */
#define APF_MAX_SUM_P 8192

/* ---- context --------------------------------------------------------- */

/* Create a context on CUDA device `device`: the state that the paper's
 * solver keeps across the outer iterations of Alg. 4 (device buffers, the
 * stream, device error word, workspace) lives here.  `cuda_stream` is a
 * cudaStream_t to order all work on (not owned), or NULL for a stream owned
 * by the context.  *out is released by apf_destroy.  APF_ERR_ARG for a bad
 * device or null out; APF_ERR_CUDA when the device cannot be used. */
apf_status apf_create(apf_ctx** out, int device, void* cuda_stream);
/* Destroy a context.  Destroy its matrices and results first: they refer to it. */
apf_status apf_destroy(apf_ctx* ctx);
const char* apf_status_string(int status);
/* Text of the last error recorded on this context ("" if none). */
const char* apf_last_error_message(const apf_ctx* ctx);
/* Kernels launched on this context since creation (a counter). */
int64_t apf_launch_count(const apf_ctx* ctx);

/* Time limit of every device-side wait of this context's kernels: the filter
 * kernels' shared-memory barrier and two-step dependency waits, and the small
 * eigensolver's grid barrier.  A wait that runs out makes the kernel record a
 * timeout, let its own copies land and return; the call then fails with
 * APF_ERR_TIMEOUT and the context stays usable.  ns = 0 restores the defaults
 * (1 s for the filter waits, 2 s for the grid barrier); at most 60 s, else
 * APF_ERR_ARG.  The paper has no counterpart: its CPU code has no device
 * waits. */
apf_status apf_set_wait_limit(apf_ctx* ctx, int64_t ns);
/* Failure-path check, with no counterpart in the paper: launch a kernel whose
 * device-side wait nothing will satisfy and return the status the library
 * makes of it (APF_ERR_TIMEOUT when the wait gave up as it should).
 * which = 0: the two-step filter pass (Alg. 2, two Clenshaw steps per pass)
 * over A's SELL copy, with every second step waiting for dependency counts
 * that are never reached (A needs a SELL copy and n > 32, else APF_ERR_ARG);
 * which = 1: the eigensolver's grid barrier, waiting for one block more than
 * the launch has (A unused, may be NULL).  Each waiting block gives up after
 * the limit of apf_set_wait_limit: set a short one first. */
apf_status apf_wait_probe(apf_ctx* ctx, const apf_matrix* A, int32_t which);

/* ---- matrices ---------------------------------------------------------- */

/* Copy a sparse Hermitian matrix, given in CSR with both triangles stored,
 * into the library's device layout (Sec. 3.3.1: CSR storage of A).
 * rowptr: n + 1 int64 offsets, monotone, rowptr[0] = 0, rowptr[n] = nnz.
 * colidx: nnz int32 column indices in [0, n).  vals: nnz values of `dtype`.
 * `on_device` = 1 if the three arrays are device pointers, 0 if host.
 * Missing diagonal entries are stored as explicit zeros.  The matrix is
 * checked for A = A^H (relative tolerance 1e-12): APF_ERR_NOT_HERMITIAN. */
apf_status apf_matrix_create_csr(apf_ctx* ctx, int64_t n, int64_t nnz,
                                 const int64_t* rowptr, const int32_t* colidx,
                                 const void* vals, int32_t dtype, int32_t on_device,
                                 apf_matrix** out);

/* Same, from SELL-C-sigma (Kreutzer et al. 2014): rows permuted by `perm`
 * (perm[r] = original row stored at sorted position r), grouped in chunks of C
 * rows stored column-major; chunk c holds chunk_len[c] * C entries starting at
 * chunk_ptr[c]; padding entries have value 0.  Host pointers only.  The
 * matrix is converted to CSR on ingest (same device layout as above). */
apf_status apf_matrix_create_sell(apf_ctx* ctx, int64_t n, int32_t C, int32_t sigma,
                                  const int64_t* perm, const int64_t* chunk_ptr,
                                  const int32_t* chunk_len, const int32_t* colidx,
                                  const void* vals, int32_t dtype, apf_matrix** out);
apf_status apf_matrix_destroy(apf_matrix* A);
/* The Clenshaw step kernel of the FP32 filter (Alg. 2) for this matrix.  By
 * default (kind 0) an autotuner times the compiled variants on the first
 * filter application at each block width and keeps the fastest.  Every
 * variant does the same operations in the same order, so the choice changes
 * the time, never the result.  Pin one instead: kind 1 = SELL-8, one step per
 * launch; 2 = SELL-8, two steps per pass over a banded (reverse Cuthill-McKee)
 * copy; 3 = CSR; 4 = SELL-8 with the block cut into column tiles of G x VPT
 * vectors, one tile per CTA, swept tile after tile (any width; the tile width
 * is what keeps the far neighbours' rows of W in L2); 5 = as 4, with the rows
 * of W within H rows of a CTA's own staged in shared memory (H, up to 16, is
 * chosen at ingest from the entries near the diagonal: 4 for the 25-point
 * stencil of an eighth-order 3D Laplacian).  (G, VPT) = lanes per row x
 * 16-byte vectors per lane, (0, 0) for the shape with the fewest idle lanes.
 * Where a pinned kind does not apply (matrix, width) it falls back
 * 5 -> 4 -> 1, 2 -> 1 -> 3.  APF_ERR_ARG for a kind outside 0..5. */
apf_status apf_matrix_set_filter_kernel(apf_matrix* A, int32_t kind, int32_t G, int32_t VPT);
apf_status apf_matrix_info(const apf_matrix* A, int64_t* n, int64_t* nnz, int32_t* dtype);

/* ---- solve -------------------------------------------------------------- */

void apf_params_default(apf_params* p);

/* Alg. 4: all eigenpairs of A in [a, b].  On APF_OK or APF_ERR_NO_CONVERGENCE
 * *out receives a result (to be freed with apf_result_destroy) holding the
 * locked pairs in ascending order of eigenvalue. */
apf_status apf_solve(apf_ctx* ctx, const apf_matrix* A, const apf_params* params,
                     apf_result** out);
/* Spectrum slicing (Sec. 1: the spectrum cut into slices whose eigenpairs are
 * computed in parallel): Alg. 4 for `nslices` intervals [a[s], b[s]] of the
 * same matrix with subspace sizes p[s] (host arrays), advanced together.  One
 * filter launch per Clenshaw step serves every slice: each slice's columns of
 * the combined block carry that slice's coefficients (zero above its current
 * degree), so a slice of lower degree simply joins the recurrence later.
 * Orthogonalisation, Rayleigh-Ritz, locking and Alg. 3 run per slice.
 * `params` supplies every other setting (its a, b and p are ignored; its
 * init_block must be NULL: slice s starts from the seeded random block of
 * stream 1 + s).  The intervals must be pairwise disjoint, 1 <= p[s], and
 * p[s] <= APF_MAX_P and sum(p) <= min(n, APF_MAX_SUM_P); else APF_ERR_ARG.
 * The result holds the union
 * of the slices' pairs in ascending order of eigenvalue;
 * apf_result_slice_counts gives the count per slice (in input order).
 * APF_ERR_NO_CONVERGENCE if any slice reaches max_iter (partial result). */
apf_status apf_solve_slices(apf_ctx* ctx, const apf_matrix* A, int32_t nslices, const double* a,
                            const double* b, const int64_t* p, const apf_params* params,
                            apf_result** out);
/* counts[s] = pairs found in slice s (host array of nslices); nslices must be
 * the number the result was solved with (APF_ERR_ARG otherwise, also for a
 * result of apf_solve). */
apf_status apf_result_slice_counts(const apf_result* r, int32_t nslices, int64_t* counts);
/* The result of Alg. 4: the locked set L of eigenpairs inside [a, b] at
 * exit.  The accessors below read it; none transfers ownership, and every one
 * returns APF_ERR_ARG for a null argument.  e = |L|, the count of eigenvalues
 * in [a, b] (Alg. 4 output). */
apf_status apf_result_count(const apf_result* r, int64_t* e);
/* e eigenvalues, ascending, to host memory (host_out: e doubles, caller-owned). */
apf_status apf_result_eigvals(const apf_result* r, double* host_out);
/* n x e eigenvectors, column-major with leading dimension ld >= n (column j
 * belongs to eigenvalue j), of the matrix dtype; `out_on_device` selects
 * where `out` lives. */
apf_status apf_result_eigvecs(const apf_result* r, void* out, int64_t ld, int32_t out_on_device);
/* e relative residuals ||A v - lambda v|| / norm_a to host memory (norm_a
 * never exceeds the spectral radius, so these bound the residuals relative to
 * the true ||A|| from above). */
apf_status apf_result_residuals(const apf_result* r, double* host_out);
/* The counters of Table 2 (iterations, SpMV columns, degrees) and stage times. */
apf_status apf_result_stats(const apf_result* r, apf_stats* out);
/* Per-iteration history, up to `cap` records of 6 doubles each:
 * (degree, active width, e, locked this iteration, n_lock before, max in-interval residual / ||A||).
 * Returns the number of records in *count. */
apf_status apf_result_history(const apf_result* r, double* host_out, int32_t cap, int32_t* count);
/* Free a result (and, for a served request, the request's own context). */
apf_status apf_result_destroy(apf_result* r);

/* ---- serving: many solves on one GPU -------------------------------------- */
/* The paper solves one problem at a time; this loop serves independent
 * requests (Sec. 1: slices and problems need no communication) with
 * continuous batching on one device.  One engine thread runs every admitted
 * request's Alg. 4; each launch of the batched Clenshaw step carries the next
 * step (Alg. 2) of every request in the filter phase of its current outer
 * iteration (one launch for the real and one for the complex problems), so
 * the filter steps of requests of different sizes, widths and degrees share
 * launches.  A request whose recurrence ends runs its orthogonalisation,
 * Rayleigh-Ritz and residual steps on its own CUDA stream, overlapping the
 * others, and rejoins the launches with its next iteration.  Requests are
 * admitted in arrival order between launches, when a slot is free and their
 * estimated device footprint fits in the budget left by the running ones (or
 * when none runs).  Each request's subspace and filter state stays on the
 * device from admission to completion.  A request's arithmetic does not
 * depend on the other requests: its result is the same alone and in a mix,
 * and the same as apf_solve's.  Requests large enough to fill the GPU with
 * their own steps (at least eight 32-row tiles of the step per SM), with an
 * FP64 filter, or whose matrix has no SELL copy filter on their own stream,
 * concurrently with the batched launches. */
typedef struct apf_server apf_server;

typedef struct {
  int32_t status;          /* the solve's apf_status */
  int32_t worker;          /* worker slot that ran it */
  double queue_ms;         /* submit -> admission */
  double run_ms;           /* admission -> done (ingest + solve) */
  double latency_ms;       /* submit -> done */
  int64_t footprint_bytes; /* device bytes reserved at admission (estimate) */
} apf_request_info;

typedef struct {
  int32_t queued, running, peak_running, workers;  /* workers: most requests in flight at once */
  int64_t in_flight_bytes, peak_in_flight_bytes, budget_bytes, completed;
  int64_t batched_launches;  /* Clenshaw-step launches that served the running requests together */
  int32_t widest_batch;      /* most requests in one such launch */
  int32_t reserved;
} apf_server_info;

/* Start the serving engine on `device` with at most `max_concurrent` (1..64;
 * more than 32 counts as 32) requests in flight.  hbm_budget_bytes: device
 * bytes the running requests may reserve; 0 means 90 % of the memory free at
 * creation. */
apf_status apf_server_create(apf_server** out, int32_t device, int32_t max_concurrent,
                             int64_t hbm_budget_bytes);
/* Queue one solve of the n x n Hermitian matrix (host CSR, both triangles,
 * dtype APF_R64 or APF_C128; the arrays are copied) with `params` (p = 0
 * estimates the subspace size; init_block must be NULL).  *ticket identifies
 * the request.  APF_ERR_OOM when its footprint estimate alone exceeds the
 * budget. */
apf_status apf_server_submit(apf_server* s, int64_t n, int64_t nnz, const int64_t* rowptr,
                             const int32_t* colidx, const void* vals, int32_t dtype,
                             const apf_params* params, int64_t* ticket);
/* Block until the request is done; return its status.  *out receives its
 * result (as apf_solve gives it; NULL when the solve failed), which owns the
 * request's context: apf_result_destroy releases both.  `info` (nullable)
 * receives the request's times.  A ticket can be waited for once: a second
 * wait, also from another thread while the first blocks, gives APF_ERR_ARG. */
apf_status apf_server_wait(apf_server* s, int64_t ticket, apf_result** out, apf_request_info* info);
apf_status apf_server_state(apf_server* s, apf_server_info* out);
/* Finish every queued request, stop the workers, free the results nobody
 * waited for.  Results already handed out stay valid. */
apf_status apf_server_destroy(apf_server* s);

/* ---- the steps of the path, callable one by one (device buffers) ---------- */

/* Set-up of Alg. 4 (Sec. 2.2, Eq. (c_j), Eq. (m_Lanczos_damping)): the
 * coefficients a_j = c_j d_{j,k}, j = 0..k, for the mapped interval
 * [am, bm] inside (-1, 1), to host memory (k + 1 doubles). */
apf_status apf_filter_coefficients(double am, double bm, int32_t k, int32_t damping,
                                   double m_d, double* host_out);

/* Alg. 3: the degree for the next iteration from p Ritz values (host),
 * in-interval count e and coefficients a_0..a_k (host). */
apf_status apf_degree_select(const double* ritz, int32_t p, int32_t e, const double* coef,
                             int32_t k, double l1, double l2, double tau_a, int32_t* degree);

/* Sec. 3.4: spectrum bounds by `steps` Lanczos steps (full
 * reorthogonalisation) from the seeded start vector, padded outward by
 * |beta_m s_m| + pad (theta_max - theta_min) and clipped to the Gershgorin
 * interval.  host_out[6] = {lmin, lmax, theta_min, theta_max, gersh_lo, gersh_hi}. */
apf_status apf_spectrum_bounds(apf_ctx* ctx, const apf_matrix* A, int32_t steps,
                               uint64_t seed, double pad, double* host_out);

/* Alg. 2: Y = rho(l(A)) X with rho = sum_{j=0}^{degree} coef[j] T_j and
 * l(x) = l1 x + l2.  X, Y: device n x p blocks of the matrix dtype (X and Y
 * may not overlap).  coef: host, degree + 1 doubles.  precision:
 * APF_FILTER_F64 or APF_FILTER_F32. */
apf_status apf_filter_apply(apf_ctx* ctx, const apf_matrix* A, const double* coef,
                            int32_t degree, double l1, double l2, int32_t precision,
                            const void* X, int64_t ldx, int64_t p, void* Y, int64_t ldy);

/* Alg. 2 in the defect form of APF_FILTER_F32_DEFECT: Y = rho(l(A)) V using
 * the FP64 identity rho(l(A)) V = V diag(rho(l(lam))) + D and an FP32
 * recurrence for D driven by R = A V - V diag(lam).  V, AV: device n x p
 * blocks (ld), lam: device p doubles. */
apf_status apf_filter_apply_defect(apf_ctx* ctx, const apf_matrix* A, const double* coef,
                                   int32_t degree, double l1, double l2, const void* V,
                                   const void* AV, const double* lam, int64_t ld, int64_t p,
                                   void* Y, int64_t ldy);

/* Sec. 3.4: the eigenvalue count estimate e~ = (1/m) sum_c z_c^H rho(l(A)) z_c,
 * the trace of the filter rho = sum_{j=0}^{degree} coef[j] T_j (host
 * coefficients) estimated with m real probe vectors of +-1 (Hutchinson 1989):
 * z_c[i] = -1 when the uniform draw of counter i m + c of SplitMix64 keyed by
 * (seed, stream 3) is below 1/2, else +1.  precision: APF_FILTER_F64 or
 * APF_FILTER_F32 (as apf_filter_apply); 1 <= m <= 8 APF_MAX_P.  *host_out
 * receives e~.  Allocates (and frees) n x m blocks on the device. */
apf_status apf_count_estimate(apf_ctx* ctx, const apf_matrix* A, const double* coef,
                              int32_t degree, double l1, double l2, int32_t precision,
                              int32_t m, uint64_t seed, double* host_out);

/* Y = A X (FP64 sparse times dense block), device blocks. */
apf_status apf_spmm(apf_ctx* ctx, const apf_matrix* A, const void* X, int64_t ldx,
                    int64_t p, void* Y, int64_t ldy);

/* G = X^H Y: the tall-skinny Gram product of the Cholesky QR and
 * Rayleigh-Ritz steps of Alg. 4.  X: n x pa, Y: n x pb,
 * G: pa x pb row-major (ldg >= pb), all device, of `dtype`.  apf_gram_tc
 * below computes the same product on the tensor cores. */
apf_status apf_gram(apf_ctx* ctx, int32_t dtype, int64_t n, int64_t pa, int64_t pb,
                    const void* X, int64_t ldx, const void* Y, int64_t ldy,
                    void* G, int64_t ldg);

/* The same G = X^H Y as apf_gram, to FP64 accuracy, on the tcgen05 tensor
 * cores (bf16 in, FP32 accumulate): each column is split into seven balanced
 * 8-bit digits of round(x 2^(55 - e_a)) under a per-column power of two 2^e_a
 * (the Ozaki scheme); the digit products of each diagonal s + t = d <= 6
 * accumulate exactly in FP32 over 32-row chunks and are carried exactly in
 * 64-bit integers.  The error is at most about n 2^(e_a + e_b - 55), where
 * 2^e_a (< twice column a's largest entry) bounds column a: within a small
 * factor of an FP64 product's worst case.  Same arguments and errors as
 * apf_gram (APF_ERR_TIMEOUT if a device wait gave up); pa, pb <= APF_MAX_P.
 * The digits (7 x n x pa bf16, twice for complex) live in a workspace of the
 * context that grows to the largest call and is kept until apf_destroy. */
apf_status apf_gram_tc(apf_ctx* ctx, int32_t dtype, int64_t n, int64_t pa, int64_t pb,
                       const void* X, int64_t ldx, const void* Y, int64_t ldy,
                       void* G, int64_t ldg);

/* Z = beta Z + alpha X M: the tall block products of Alg. 4 (X R^{-1} in
 * Cholesky QR, the Ritz vectors Q U of Rayleigh-Ritz, the projection
 * X - V (V^H X) against the locked vectors).  X: n x pa, M: pa x pb, Z: n x pb,
 * all device, row-major, of `dtype`; Z must not overlap X or M.
 * tensor_cores = 0: FP64 cores; 1: the tcgen05 tensor cores with the same
 * digit slicing as apf_gram_tc (each row of X and each column of M under its
 * own power of two, seven 8-bit digits, exact integer carry), to FP64
 * accuracy relative to the row and column maxima.  pa, pb <= APF_MAX_P. */
apf_status apf_block_update(apf_ctx* ctx, int32_t dtype, int64_t n, int64_t pa, int64_t pb, const void* X,
                            int64_t ldx, const void* M, int64_t ldm, void* Z, int64_t ldz, double alpha,
                            double beta, int32_t tensor_cores);

/* Orthogonalisation of Alg. 4: X (device n x p) is replaced by Q with X = Q R, by CholQR2
 * (shifted CholQR3 when the first factorisation breaks down). */
apf_status apf_cholqr2(apf_ctx* ctx, int32_t dtype, int64_t n, int64_t p, void* X, int64_t ld);

/* Hermitian eigendecomposition B = U diag(w) U^H of a small p x p device
 * matrix (p <= APF_MAX_P): w ascending (device), U row-major (ldu).
 * One-sided Jacobi on B + s I, s = 2 ||B||_inf. */
apf_status apf_eigh_small(apf_ctx* ctx, int32_t dtype, int64_t p, const void* B, int64_t ldb,
                          double* w, void* U, int64_t ldu);

/* Alg. 1 Rayleigh-Ritz: Q (device n x p, orthonormal columns) ->
 * Ritz values w (device, ascending) and Ritz vectors V = Q U (device n x p). */
apf_status apf_rayleigh_ritz(apf_ctx* ctx, const apf_matrix* A, const void* Q, int64_t ld,
                             int64_t p, double* w, void* V, int64_t ldv);

/* ||A v_j - w_j v_j||_2 for the p columns of V (device) into host_out[p]. */
apf_status apf_residual_norms(apf_ctx* ctx, const apf_matrix* A, const void* V, int64_t ld,
                              int64_t p, const double* w, double* host_out);

/* G = X^H Y as apf_gram computes it, to the same FP64 tolerance (not bit for
 * bit: the array below caps the number of row splits, so the summation order
 * can differ), for callers that cannot allocate device memory (code inside a CUDA graph being captured, an allocator's own
 * callbacks, a host with a fixed memory budget).  The paper has no
 * counterpart: this is a deployment variant of the Gram step.
 * It takes no context and allocates nothing: the partial sums of its row
 * splits live in one file-scope device array of 8 MiB that every GPU loading
 * the library holds until the process exits.  Limits: pa * pb elements of
 * `dtype` must fit in 8 MiB (pa = pb <= 1024 real, <= 724 complex), else
 * APF_ERR_ARG.  X, Y, G: device pointers on the current device; work is
 * ordered on `cuda_stream` (a cudaStream_t, NULL for the legacy default
 * stream).  The first call on each device looks up the array's device address
 * with cudaGetSymbolAddress while that device is current: make that first
 * call before any stream capture.  A device reset (cudaDeviceReset) makes a
 * new context: the first call after it looks the address up again, so it too
 * belongs before any capture.  All calls on a device share the array and
 * it keeps the last call's contents (no call needs it cleared); calls whose
 * work overlaps on the GPU (different streams, no ordering) race on it. */
apf_status apf_gram_noalloc(int32_t dtype, int64_t n, int64_t pa, int64_t pb, const void* X,
                            int64_t ldx, const void* Y, int64_t ldy, void* G, int64_t ldg,
                            void* cuda_stream);

/* The seeded initial block: entry (i, c) uniform in [-1, 1) from counter-based
 * SplitMix64 (Steele, Lea and Flood 2014) keyed by (seed, stream); real entry
 * uses counter i*p + c, complex entry counters 2(i*p + c) and 2(i*p + c) + 1. */
apf_status apf_random_block(apf_ctx* ctx, int32_t dtype, uint64_t seed, uint32_t stream,
                            int64_t n, int64_t p, void* X, int64_t ld);

#ifdef __cplusplus
}
#endif

#endif /* APF_H */
