#!/usr/bin/env python3
"""Benchmark: converged eigenpairs per second of AdaPolySI (Alg. 4) on GB300.

A step is one complete solve (Lanczos bounds, coefficients, and every outer
iteration: filter, CholQR2, Rayleigh-Ritz, residuals, spurious test, locking,
degree selection) of the workload's interior eigenproblem, with the matrix
already resident in HBM.  Default workload: the complex Hermitian 3D Anderson
model on a 64^3 periodic grid (n = 262,144, random Peierls phases, disorder
U[-2, 2]), interval [-0.0017, 0.0017] (about 100 eigenvalues), p = 160, FP32
defect-corrected filter with FP64 orthogonalisation and Rayleigh-Ritz.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torch.distributed (one process per GPU): the ranks solve
independent replicas (one interval: the path has no exchange step), time is
the maximum over ranks and the value counts the eigenpairs of all ranks.
The reference arm times the FP64 CPU oracle on a bounded sample (see
``cpu_sample``).  One JSON line is printed by rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "converged eigenpairs/s at residual 1e-10"
UNIT = "eigenpairs/s"

# Work of one solve of the default workload, as measured on a GB300 (iterations
# and the sum over iterations of filter degree x active block width).  Used only
# to scale the CPU oracle's bounded sample to a whole solve in the reference arm,
# which runs without a GPU; the main arm uses the profile of its own solves.
WORK_PROFILE = {"anderson3d_c_64": {"iterations": 30, "degree_width": 22.1e6, "eigenpairs": 99}}

# dram__bytes_read.sum + dram__bytes_write.sum per launch of the FP32
# Clenshaw step at full width (both V and Y terms), mean of three launches of
# one ncu capture of the kernel (profiles/clenshaw_sell_traffic_<workload>.md),
# keyed by workload and step kernel kind: a line whose solve picked another
# kernel reports no traffic.
TRAFFIC_BYTES = {("anderson3d_c_64", 1): 1.3486e9}

# the FP32 step kernels (apf_matrix_set_filter_kernel kinds)
KERNEL_NAMES = {1: "SELL-8", 2: "SELL-8 two-step", 3: "CSR", 4: "SELL-8 column-tiled",
                5: "SELL-8 column-tiled, near rows staged"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="anderson3d_c_64")
    ap.add_argument("--precision", default="f32_defect", choices=["f64", "f32", "f32_defect"])
    ap.add_argument("--max-iter", type=int, default=100)
    ap.add_argument("--filter-graphs", type=int, default=1,
                    help="1: recurring filter applications replayed as CUDA graphs; 0: plain launches")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=1,
                    help="end-to-end solves through the C ABI from host buffers (after the timed ones)")
    ap.add_argument("--p", type=int, default=-1, help="subspace size override (0: estimated, Sec. 3.4)")
    ap.add_argument("--f64-compare", default="anderson3d_c_40",
                    help="workload on which one plain FP64 solve is timed against the FP32 defect form "
                         "('' to skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--filter-only", type=int, default=0,
                    help="time only N applications of the filter kernel (degree --degree) instead of solves")
    ap.add_argument("--degree", type=int, default=20)
    ap.add_argument("--dense-only", type=int, default=0,
                    help="time N tensor-core Gram products X^H X and N block updates X M on the workload's "
                         "n x p block instead of solves")
    ap.add_argument("--shape", default="0,0",
                    help="with --kernel: step kernel shape 'G,VPT' (lanes per row, vectors per lane; 0,0 = default)")
    ap.add_argument("--kernel", type=int, default=0,
                    help="pin the FP32 step kernel (0 autotune, 1 SELL, 2 SELL two-step, 3 CSR, 4 SELL column "
                         "tiles, 5 column tiles with near rows staged)")
    ap.add_argument("--requests", type=int, default=24, help="serving workload: number of requests")
    ap.add_argument("--compare-single", action="store_true",
                    help="slice workloads: also solve the slices one after another")
    ap.add_argument("--concurrency", type=int, default=4, help="serving workload: requests in flight")
    ap.add_argument("--n-hi", type=float, default=1e5, help="serving workload: largest matrix size")
    ap.add_argument("--count-hi", type=int, default=64, help="serving workload: largest target count")
    ap.add_argument("--burst-concurrency", type=int, default=16,
                    help="serving workload: requests in flight in the saturated (all at once) run; 0 skips it")
    return ap.parse_args()


# ---- distributed plumbing ---------------------------------------------------------------

class Dist:
    """Rank bookkeeping and the two reductions the timing needs (max of the
    ranks' times, sum of their eigenpairs).  NCCL on GPUs, gloo on the CPU."""

    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.on = self.world > 1
        self.device = "cpu"
        if self.on:
            import torch
            import torch.distributed as dist
            if torch.cuda.is_available():
                torch.cuda.set_device(self.local)
                self.device = "cuda"
            dist.init_process_group("nccl" if self.device == "cuda" else "gloo")
            self.dist = dist

    def barrier(self):
        if self.on:
            self.dist.barrier()

    def reduce(self, x, op):
        if not self.on:
            return x
        import torch
        t = torch.tensor([float(x)], device=self.device, dtype=torch.float64)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        return self.reduce(x, self.dist.ReduceOp.MAX) if self.on else x

    def sum(self, x):
        return self.reduce(x, self.dist.ReduceOp.SUM) if self.on else x

    def close(self):
        if self.on:
            self.dist.destroy_process_group()


# ---- clocks during the timed region ------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        power = [num(r[3]) for r in rows if num(r[3]) is not None]
        loaded = [s for s, p in zip(sm, power) if p is not None and p > 250.0] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": num(rows[0][2]), "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---- the CPU oracle's bounded sample -----------------------------------------------------

def cpu_sample(workload: str, steps: int = 4):
    """Time the oracle on a bounded sample of one solve of `workload`: `steps`
    Clenshaw steps (Alg. 2) at the full block width and one orthogonalisation
    + Rayleigh-Ritz + residual pass (CholQR2, Alg. 1).  Returns per-unit times."""
    import numpy as np
    from oracle import chebyshev as cb
    from oracle import fsi
    from oracle.filter import clenshaw_apply
    from synth import rng, workloads
    w = workloads.WORKLOADS[workload]()
    A = w.matrix()
    As = A.to_scipy()
    V = rng.uniform_block(w.seed, rng.STREAM_INIT_BLOCK, A.n, w.p, A.is_complex)
    coef = cb.filter_coefficients(-0.001, 0.001, steps)
    t0 = time.perf_counter()
    X = clenshaw_apply(As, coef, 0.18, 0.0, V)
    t1 = time.perf_counter()
    Q = fsi.cholqr2(X)
    lam, Vr = fsi.rayleigh_ritz(As, Q)
    fsi.residual_norms(As, Vr, lam)
    t2 = time.perf_counter()
    return dict(step_s=(t1 - t0) / steps, width=w.p, iter_s=t2 - t1, n=A.n,
                cores=os.cpu_count(),
                sample=f"{steps} Clenshaw steps (n={A.n}, width {w.p}) + 1 CholQR2/Rayleigh-Ritz/residual pass "
                       f"of the oracle on the full {workload} matrix, scaled to one solve by its work profile")


def cpu_eigenpairs_per_s(sample, profile):
    t = (sample["step_s"] * profile["degree_width"] / sample["width"]
         + sample["iter_s"] * profile["iterations"])
    return profile["eigenpairs"] / t


# ---- arms ----------------------------------------------------------------------------------

def reference_arm(args, dist):
    if dist.rank != 0:
        return
    prof = WORK_PROFILE[args.workload]
    vals = []
    sample = None
    for i in range(args.warmup + args.steps):
        sample = cpu_sample(args.workload, steps=2)
        if i >= args.warmup:
            vals.append(cpu_eigenpairs_per_s(sample, prof))
    v = statistics.median(vals)
    # a step is one whole solve of the workload, at the sampled rate
    ms_solve = 1e3 * prof["eigenpairs"] / v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_solve,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": sample["cores"], "kind": "oracle",
                             "sample": sample["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def ours_arm(args, dist):
    import numpy as np
    import torch
    from paper_2604_00914_gb300 import binding as B
    from synth import workloads

    torch.cuda.set_device(dist.local)
    # a stream of its own (not the legacy default stream): the library launches
    # on it and the timing events below are recorded on it
    stream = torch.cuda.Stream()
    w = workloads.WORKLOADS[args.workload]()
    A = w.matrix()
    ctx = B.Context(dist.local, stream=stream.cuda_stream)
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    if args.kernel and not args.filter_only:  # a pinned step kernel instead of the autotuner's pick
        M.set_filter_kernel(args.kernel, *(int(t) for t in args.shape.split(",")))
    prec = {"f64": B.APF_FILTER_F64, "f32": B.APF_FILTER_F32, "f32_defect": B.APF_FILTER_F32_DEFECT}[args.precision]
    p_used = w.p if args.p < 0 else args.p
    prm = B.default_params(a=w.a, b=w.b, p=p_used, seed=w.seed + 1000 * dist.rank, filter_precision=prec,
                           max_iter=args.max_iter, filter_graphs=args.filter_graphs)
    peak, peak_kind = measured_peaks()

    def one_solve():
        r = B.solve(ctx, M, prm)
        out = (r.count(), r.stats(), r.history())
        r.close()
        return out

    if args.filter_only:
        return filter_only(args, dist, B, ctx, M, A, w, peak, peak_kind)
    if args.dense_only:
        return dense_only(args, dist, B, ctx, A, w, stream)

    for _ in range(args.warmup):
        one_solve()
    sampler = ClockSampler(dist.local)
    dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = ctx.launch_count()
    ev0.record(stream)
    eig = 0
    fbytes = fms = fstep_bytes = 0.0
    flaunch = fsteps = 0
    deg_width = 0.0
    iters = 0
    maxres = 0.0
    p_stat = deg_seq = None
    step_kernel = (-1, 0, 0)
    stage = {"setup": 0.0, "filter": 0.0, "orth_rr": 0.0, "check": 0.0, "total": 0.0}
    for _ in range(args.steps):
        e, st, hist = one_solve()
        p_stat = st["p_used"]
        for k_, s_ in (("setup", "ms_setup"), ("filter", "ms_filter"), ("orth_rr", "ms_rr"), ("check", "ms_check"),
                       ("total", "ms_total")):
            stage[k_] += st[s_] / args.steps
        deg_seq = [int(h["degree"]) for h in hist]
        eig += e
        fbytes += st["filter_bytes"]
        fstep_bytes += st["filter_step_bytes"]
        fms += st["filter_kernel_ms"]
        flaunch += st["filter_launches"]
        fsteps += st["filter_steps"]
        deg_width += sum(h["degree"] * h["width"] for h in hist)
        iters += st["iterations"]
        maxres = max(maxres, st["max_residual"])
        step_kernel = (st["filter_kind"], st["filter_g"], st["filter_vpt"])
    ev1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clocks = sampler.stop()
    launches = ctx.launch_count() - launches0
    ms_local = ev0.elapsed_time(ev1)
    ms = dist.max(ms_local)
    eig_all = dist.sum(eig)
    value = eig_all / (ms / 1e3)

    # end to end through the C ABI: host CSR in pinned memory -> solve -> eigenpairs to host
    e2e = None
    if not args.no_e2e and args.e2e_steps > 0:
        rp = torch.from_numpy(A.rowptr).pin_memory()
        ci = torch.from_numpy(A.colidx).pin_memory()
        vv = torch.from_numpy(A.vals).pin_memory()
        h2d = rp.numel() * 8 + ci.numel() * 4 + vv.numel() * vv.element_size()
        dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e_tot = 0
        d2h = 0
        for _ in range(args.e2e_steps):
            M2 = B.Matrix.from_csr(ctx, A.n, rp.numpy(), ci.numpy(), vv.numpy())
            r = B.solve(ctx, M2, prm)
            e = r.count()
            lam = r.eigvals()
            vecs = torch.empty((e, A.n), dtype=torch.complex128 if A.is_complex else torch.float64).pin_memory()
            ctx.lib.check(ctx.lib.apf_result_eigvecs(r.h, vecs.data_ptr(), A.n, 0), ctx.h)
            d2h = lam.nbytes + vecs.numel() * vecs.element_size()
            e_tot += e
            r.close()
            M2.close()
        torch.cuda.synchronize()
        dt = dist.max(time.perf_counter() - t0)
        e2e = {"value": dist.sum(e_tot) / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "solves": args.e2e_steps}

    plain = None
    if args.f64_compare and dist.rank == 0:
        plain = f64_compare(args, dist, B, stream)

    cpu = None
    if dist.rank == 0 and args.gpus == 1 and not args.no_cpu_baseline:
        s = cpu_sample(args.workload, steps=4)
        prof = {"iterations": iters / args.steps, "degree_width": deg_width / args.steps,
                "eigenpairs": eig / args.steps}
        cpu = {"value": cpu_eigenpairs_per_s(s, prof), "unit": UNIT, "cores": s["cores"], "kind": "oracle",
               "sample": s["sample"].replace("its work profile", "the work profile of the timed GPU solves")}

    achieved = fbytes / (fms * 1e-3) / 1e9 if fms > 0 else None
    per_step = fstep_bytes / (fms * 1e-3) / 1e9 if fms > 0 else None
    kind = "complex" if A.is_complex else "real"
    bits = {"f64": "FP64", "f32": "FP32", "f32_defect": "FP32"}[args.precision]
    blk_mb = A.n * w.p * (8 if A.is_complex else 4) / 1e6
    traffic = (TRAFFIC_BYTES.get((args.workload, step_kernel[0]))
               if args.precision != "f64" and args.p < 0 else None)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": (({"f64": "c128", "f32": "c64", "f32_defect": "c64+c128"} if A.is_complex else
                   {"f64": "f64", "f32": "f32", "f32_defect": "f32+f64"})[args.precision]),
        "data": "synthetic",
        "config": {"workload": args.workload, "n": A.n, "nnz": A.nnz, "p": p_used, "interval": [w.a, w.b],
                   "precision": args.precision, "eigenpairs_per_solve": eig / args.steps,
                   "iterations_per_solve": iters / args.steps, "max_residual": maxres,
                   "p_used": p_stat, "degree_sequence": deg_seq,
                   "stage_ms_per_solve": {k_: round(v_, 1) for k_, v_ in stage.items()},
                   "l2": f"inputs larger than L2 (FP32 block {blk_mb:.0f} MB, FP64 block {2 * blk_mb:.0f} MB)",
                   "parallelism": f"replicas{args.gpus}"},
        "roofline": {"kernel": f"Clenshaw filter step ({bits} {kind}, {KERNEL_NAMES.get(step_kernel[0], 'FP64 CSR')})",
                     "step_kernel": {"kind": step_kernel[0], "G": step_kernel[1], "VPT": step_kernel[2]},
                     "bound": "hbm",
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None,
                     "traffic": traffic,
                     "avg_launch_us": 1e3 * fms / flaunch if flaunch else None,
                     "launches": flaunch, "steps": fsteps,
                     "us_per_step": 1e3 * fms / fsteps if fsteps else None,
                     "one_step_equivalent_gbs": per_step},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "plain_f64": plain,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    M.close()
    ctx.close()


def f64_compare(args, dist, B, stream):
    """The spec ratio: one solve with the plain FP64 filter against one
    with the FP32 defect-corrected filter (after a warm-up solve that tunes its
    kernel) on `--f64-compare`'s workload, both to ||r|| <= 1e-10 ||A||.
    Reports both rates, the speed-up, and per result the eigenvalue difference
    between the two forms and each form's relative residual (for Hermitian A a
    residual bounds the distance of the Ritz value to the spectrum)."""
    import numpy as np
    import torch
    from synth import workloads
    w = workloads.WORKLOADS[args.f64_compare]()
    A = w.matrix()
    ctx = B.Context(dist.local, stream=stream.cuda_stream)
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(prec):
        prm = B.default_params(a=w.a, b=w.b, p=w.p, seed=w.seed, filter_precision=prec, max_iter=args.max_iter)
        torch.cuda.synchronize()
        ev0.record(stream)
        r = B.solve(ctx, M, prm, allow_no_convergence=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        out = dict(ms=ev0.elapsed_time(ev1), status=r.status, lam=r.eigvals(), res=r.residuals(),
                   st=r.stats())
        r.close()
        return out

    timed(B.APF_FILTER_F32_DEFECT)  # warm-up: kernel tuning of this matrix
    f32 = timed(B.APF_FILTER_F32_DEFECT)
    f64 = timed(B.APF_FILTER_F64)
    M.close()
    ctx.close()

    def arm(o):
        e = int(o["lam"].size)
        return {"value": e / (o["ms"] / 1e3), "unit": UNIT, "seconds": o["ms"] / 1e3, "eigenpairs": e,
                "status": o["status"], "iterations": o["st"]["iterations"],
                "max_residual": float(o["res"].max()) if e else None}

    same = f32["lam"].size == f64["lam"].size
    norm_a = f64["st"]["norm_a"]
    dl = (np.abs(f32["lam"] - f64["lam"]) / norm_a) if same else None
    a32, a64 = arm(f32), arm(f64)
    return {"workload": args.f64_compare, "n": A.n, "p": w.p, "interval": [w.a, w.b],
            "f32_defect": a32, "f64": a64,
            "speedup_vs_plain_f64": a32["value"] / a64["value"] if a64["value"] else None,
            "same_count": bool(same),
            "max_dlambda_over_normA": float(dl.max()) if dl is not None and dl.size else None,
            "per_result": {"dlambda_over_normA": [float(f"{x:.3g}") for x in dl] if dl is not None else None,
                           "residual_f32_defect": [float(f"{x:.3g}") for x in f32["res"]],
                           "residual_f64": [float(f"{x:.3g}") for x in f64["res"]]}}


def serving_arm(args, dist):
    """Independent requests (synth.workloads.serving_requests) through the
    serving loop: first every request once, one at a time (the serial
    capacity), then all of them again with Poisson arrivals at 0.8 x that
    capacity and `--concurrency` worker slots; p50/p99 latency, throughput and
    whether each result equals its serial run.  Rank 0 only (one GPU)."""
    import math
    import numpy as np
    import torch
    from paper_2604_00914_gb300 import binding as B
    from synth import rng, workloads

    if dist.rank != 0:
        return
    torch.cuda.set_device(dist.local)
    reqs = workloads.serving_requests(args.requests, n_hi=args.n_hi, count_hi=args.count_hi)
    mats = [r.matrix() for r in reqs]
    prms = [B.default_params(a=r.a, b=r.b, p=0, seed=r.seed, filter_precision=B.APF_FILTER_F32_DEFECT,
                             max_iter=args.max_iter) for r in reqs]
    # serial capacity: every request one at a time (after one warm-up)
    srv = B.Server(dist.local, max_concurrent=1)
    res, _ = srv.wait(srv.submit(mats[0].n, mats[0].rowptr, mats[0].colidx, mats[0].vals, prms[0]),
                      allow_no_convergence=True)
    if res is not None:
        res.close()
    serial_lam, serial_lat = [], []
    t0 = time.perf_counter()
    for i, A in enumerate(mats):
        res, info = srv.wait(srv.submit(A.n, A.rowptr, A.colidx, A.vals, prms[i]), allow_no_convergence=True)
        serial_lat.append(info["latency_ms"])
        serial_lam.append(res.eigvals() if res is not None else None)
        if res is not None:
            res.close()
    serial_s = (time.perf_counter() - t0) / len(mats)
    srv.close()
    rate = 0.8 / serial_s
    u = rng.uniform(BASE_ARRIVALS, rng.STREAM_TEST, np.arange(len(reqs), dtype=np.uint64))
    gaps = -np.log1p(-u) / rate
    srv = B.Server(dist.local, max_concurrent=args.concurrency)
    sampler = ClockSampler(dist.local)
    sampler.start()
    t0 = time.perf_counter()
    tickets = []
    due = 0.0
    for i, A in enumerate(mats):
        due += gaps[i]
        delay = t0 + due - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        tickets.append(srv.submit(A.n, A.rowptr, A.colidx, A.vals, prms[i]))
    lat, eig, ok, same = [], 0, 0, 0
    for i, t in enumerate(tickets):
        res, info = srv.wait(t, allow_no_convergence=True)
        lat.append(info["latency_ms"])
        if res is not None:
            eig += res.count()
            same += int(serial_lam[i] is not None and np.array_equal(serial_lam[i], res.eigvals()))
            res.close()
        ok += info["status"] == 0
    wall = time.perf_counter() - t0
    state = srv.state()
    srv.close()
    # saturated: every request submitted at once, the makespan against the serial total
    burst = None
    if args.burst_concurrency > 0:
        srv = B.Server(dist.local, max_concurrent=args.burst_concurrency)
        tb = time.perf_counter()
        tks = [srv.submit(A.n, A.rowptr, A.colidx, A.vals, prms[i]) for i, A in enumerate(mats)]
        blat, bsame = [], 0
        for i, t in enumerate(tks):
            res, info = srv.wait(t, allow_no_convergence=True)
            blat.append(info["latency_ms"])
            if res is not None:
                bsame += int(serial_lam[i] is not None and np.array_equal(serial_lam[i], res.eigvals()))
                res.close()
        makespan = time.perf_counter() - tb
        bst = srv.state()
        srv.close()
        burst = {"concurrency": args.burst_concurrency, "makespan_s": makespan,
                 "serial_total_s": serial_s * len(mats), "speedup_vs_serial": serial_s * len(mats) / makespan,
                 "throughput_requests_per_s": len(mats) / makespan, "p50_ms": float(np.percentile(blat, 50)),
                 "p99_ms": float(np.percentile(blat, 99)), "same_as_serial": bsame,
                 "batched_launches": bst["batched_launches"], "widest_batch": bst["widest_batch"],
                 "peak_running": bst["peak_running"]}
    clocks = sampler.stop()
    lat = np.array(lat)
    print(json.dumps({
        "metric": "serving latency (p50/p99)", "mode": "serving", "requests": len(reqs), "converged": ok,
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()), "serial_ms_per_request": 1e3 * serial_s,
        "serial_p50_ms": float(np.percentile(serial_lat, 50)), "serial_p99_ms": float(np.percentile(serial_lat, 99)),
        "same_as_serial": same,
        "arrival_rate_per_s": rate, "throughput_requests_per_s": len(reqs) / wall,
        "eigenpairs_per_s": eig / wall, "concurrency": args.concurrency,
        "peak_running": state["peak_running"], "peak_in_flight_bytes": state["peak_in_flight_bytes"],
        "batched_launches": state["batched_launches"], "widest_batch": state["widest_batch"],
        "saturated": burst,
        "data": "synthetic", "clocks": clocks,
        "config": {"workload": "serving", "n_range": [1e4, args.n_hi], "target_counts": [8, args.count_hi],
                   "p": "estimated (Sec. 3.4)", "precision": "f32_defect"}}), flush=True)


def slices_arm(args, dist):
    """A spectrum-slice workload (synth.workloads.SLICE_WORKLOADS) through
    apf_solve_slices: every slice's filter in one launch per Clenshaw step.
    A step is one whole batched solve; with --compare-single the same slices
    are also solved one after another with apf_solve."""
    import numpy as np
    import torch
    from paper_2604_00914_gb300 import binding as B
    from synth import workloads

    torch.cuda.set_device(dist.local)
    stream = torch.cuda.Stream()  # the library's stream and the timing events' stream
    w = workloads.SLICE_WORKLOADS[args.workload]()
    A = w.matrix()
    ctx = B.Context(dist.local, stream=stream.cuda_stream)
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    prec = {"f64": B.APF_FILTER_F64, "f32": B.APF_FILTER_F32, "f32_defect": B.APF_FILTER_F32_DEFECT}[args.precision]
    prm = B.default_params(seed=w.seed + 1000 * dist.rank, filter_precision=prec, max_iter=args.max_iter)
    peak, peak_kind = measured_peaks()

    def one():
        r = B.solve_slices(ctx, M, w.a, w.b, w.p, prm, allow_no_convergence=True)
        out = (r.status, r.count(), r.slice_counts(len(w.a)), r.stats())
        r.close()
        return out

    for _ in range(args.warmup):
        one()
    sampler = ClockSampler(dist.local)
    dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = ctx.launch_count()
    ev0.record(stream)
    eig, fbytes, fms, flaunch, statuses, counts, st = 0, 0.0, 0.0, 0, [], None, None
    for _ in range(args.steps):
        status, e, counts, st = one()
        statuses.append(status)
        eig += e
        fbytes += st["filter_bytes"]
        fms += st["filter_kernel_ms"]
        flaunch += st["filter_launches"]
    ev1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clocks = sampler.stop()
    launches = ctx.launch_count() - launches0
    ms = dist.max(ev0.elapsed_time(ev1))
    value = dist.sum(eig) / (ms / 1e3)
    single = None
    if args.compare_single:
        t0 = time.perf_counter()
        e_single = 0
        for s in range(len(w.a)):
            p_s = int(w.p[s])
            r = B.solve(ctx, M, B.default_params(a=w.a[s], b=w.b[s], p=p_s, seed=prm.seed, filter_precision=prec,
                                                 max_iter=args.max_iter), allow_no_convergence=True)
            e_single += r.count()
            r.close()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        single = {"value": e_single / dt, "unit": UNIT, "seconds": dt, "eigenpairs": e_single}
    achieved = fbytes / (fms * 1e-3) / 1e9 if fms > 0 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"f64": "f64", "f32": "f32", "f32_defect": "f32+f64"}[args.precision],
        "data": "synthetic", "mode": "slices",
        "config": {"workload": args.workload, "n": A.n, "nnz": A.nnz, "slices": len(w.a),
                   "intervals": [[x, y] for x, y in zip(w.a, w.b)],
                   "p": "estimated (Sec. 3.4)" if not any(w.p) else [int(q) for q in w.p],
                   "p_total": st["p_used"], "count_estimate": st["trace_estimate"],
                   "slice_counts": [int(c) for c in counts], "status": statuses,
                   "iterations": st["iterations"], "max_residual": st["max_residual"],
                   "graph_replays": st["filter_graph_replays"],
                   "step_kernel": {"kind": st["filter_kind"], "G": st["filter_g"], "VPT": st["filter_vpt"]},
                   "precision": args.precision, "parallelism": f"replicas{args.gpus}"},
        "roofline": {"kernel": "Clenshaw filter step (FP32 real, all slices per launch)", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None, "traffic": None,
                     "avg_launch_us": 1e3 * fms / flaunch if flaunch else None, "launches": flaunch},
        "single_solves": single,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    M.close()
    ctx.close()


def sweep_arm(args, dist):
    """Parameter sensitivity of Sec. 4 on a synthetic matrix: the damping
    exponent m in [0, 3] (step 0.1), the adaptive threshold tau_a in
    [1e-4, 0.5], and C_r = C / (alpha - beta) over 13 values spanning a factor
    12 (the paper's [10, 120] span) around the default C = 1.4 of this
    interval, with the adaptive filter and with the fixed degree
    k = ceil(2.5 k^(1)).  Each point is one solve; the line reports
    iterations, mean degree, SpMV columns and time per point.  Rank 0 only."""
    import math
    import numpy as np
    import torch
    from paper_2604_00914_gb300 import binding as B
    from synth import matrices

    if dist.rank != 0:
        return
    torch.cuda.set_device(dist.local)
    A = matrices.anderson(24, 3, 4.0, SWEEP_SEED, complex_phases=True)
    a, b = -0.012, 0.012
    ctx = B.Context(dist.local)
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    base = dict(a=a, b=b, p=0, seed=SWEEP_SEED, filter_precision=B.APF_FILTER_F32_DEFECT, max_iter=args.max_iter)

    def run(**kw):
        prm = B.default_params(**{**base, **kw})
        r = B.solve(ctx, M, prm, allow_no_convergence=True)
        st = r.stats()
        out = {"status": r.status, "e": r.count(), "iterations": st["iterations"],
               "avg_degree": round(st["avg_degree"], 1), "spmv_columns": st["spmv_columns"],
               "ms": round(st["ms_total"], 1), "k1": st["k1"], "k_max": st["k_max"]}
        r.close()
        return out

    ref = run()  # warm-up and the default point
    st = B.default_params(**base)
    r = B.solve(ctx, M, st, allow_no_convergence=True)
    s = r.stats()
    r.close()
    l1 = 2.0 / (s["lambda_max"] - s["lambda_min"])
    l2 = -(s["lambda_max"] + s["lambda_min"]) / (s["lambda_max"] - s["lambda_min"])
    width = math.acos(l1 * a + l2) - math.acos(l1 * b + l2)  # alpha - beta
    out = {"mode": "sweep", "data": "synthetic",
           "config": {"workload": "anderson3d_c_24 sweep", "n": A.n, "interval": [a, b], "p": "estimated",
                      "precision": "f32_defect"},
           "default": ref, "m": [], "tau_a": [], "C_r_adaptive": [], "C_r_fixed": []}
    for m in np.round(np.arange(0.0, 3.0001, 0.1), 1):
        out["m"].append({"m": float(m), **run(m_d=float(m))})
    for ta in [1e-4, 3e-4, 1e-3, 3e-3, 1e-2, 3e-2, 1e-1, 0.5]:
        out["tau_a"].append({"tau_a": ta, **run(tau_a=ta)})
    cr0 = 1.4 / width
    for cr in cr0 * np.linspace(0.3, 3.6, 13):
        C = float(cr) * width
        k1 = int(math.ceil(cr)) - 1
        out["C_r_adaptive"].append({"C_r": float(cr), **run(C=C)})
        out["C_r_fixed"].append({"C_r": float(cr), **run(k_fixed=int(math.ceil(2.5 * k1)))})
    print(json.dumps(out), flush=True)
    M.close()
    ctx.close()


SWEEP_SEED = 20260407

# seed of the serving workload's arrival times
BASE_ARRIVALS = 20260406


def filter_only(args, dist, B, ctx, M, A, w, peak, peak_kind):
    """Time N applications of the FP32 filter recurrence of degree `--degree` on
    the workload's matrix and block width (the dominant kernel alone)."""
    import numpy as np
    import torch
    from synth import rng
    n, p = A.n, w.p
    g_, v_ = (int(t) for t in args.shape.split(","))
    M.set_filter_kernel(args.kernel, g_, v_)
    X = torch.from_numpy(rng.uniform_block(w.seed, rng.STREAM_INIT_BLOCK, n, p, A.is_complex)).cuda()
    Y = torch.empty_like(X)
    coef = np.linspace(1.0, 0.1, args.degree + 1)
    for _ in range(args.warmup):
        B.filter_apply(ctx, M, coef, 0.18, 0.0, X, Y, B.APF_FILTER_F32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.filter_only):
        B.filter_apply(ctx, M, coef, 0.18, 0.0, X, Y, B.APF_FILTER_F32)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    if dist.rank == 0:
        print(json.dumps({"mode": "filter-only", "workload": args.workload, "degree": args.degree,
                          "applications": args.filter_only, "seconds": dt}), flush=True)


def dense_only(args, dist, B, ctx, A, w, stream):
    """Time the dense products of one outer iteration on the tensor cores:
    G = X^H X (apf_gram_tc) and Z = X M (apf_block_update) on the workload's
    n x p block, and the p x p eigensolve of Rayleigh-Ritz (apf_eigh_small),
    with CUDA events on the library's stream.  The tensor-pipe
    rate counts the bf16 MMAs the digit scheme issues: 28 digit pairs x
    2 x 128 x 32 x 32 flops per 32-row chunk of each 128 x 32 output tile."""
    import math
    import numpy as np
    import torch
    from synth import rng
    n, p, cplx = A.n, w.p, A.is_complex
    C = 2 if cplx else 1
    X = torch.from_numpy(rng.uniform_block(w.seed, rng.STREAM_INIT_BLOCK, n, p, cplx)).cuda()
    Mt = torch.from_numpy(rng.uniform_block(w.seed, rng.STREAM_TEST, p, p, cplx)).cuda()
    G = torch.empty((p, p), dtype=X.dtype, device="cuda")
    Z = torch.empty_like(X)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for _ in range(max(1, args.warmup)):
        B.gram_tc(ctx, X, X, G)
        B.block_update(ctx, X, Mt, Z)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(args.dense_only):
        B.gram_tc(ctx, X, X, G)
    ev[1].record(stream)
    for _ in range(args.dense_only):
        B.block_update(ctx, X, Mt, Z)
    ev[2].record(stream)
    torch.cuda.synchronize()
    gram_ms = ev[0].elapsed_time(ev[1]) / args.dense_only
    upd_ms = ev[1].elapsed_time(ev[2]) / args.dense_only
    # the p x p Hermitian eigensolve of Rayleigh-Ritz (one-sided Jacobi) on a
    # Gram-like matrix of the same size
    Hm = torch.from_numpy(rng.uniform_block(w.seed, rng.STREAM_TEST, p, p, cplx)).cuda()
    Hm = (Hm + Hm.conj().T).contiguous()
    wv = torch.empty(p, dtype=torch.float64, device="cuda")
    Um = torch.empty_like(Hm)
    torch.cuda.synchronize()  # Hm is written on torch's stream, read on the library's
    B.eigh_small(ctx, Hm, wv, Um)
    torch.cuda.synchronize()
    ev[2].record(stream)
    for _ in range(args.dense_only):
        B.eigh_small(ctx, Hm, wv, Um)
    ev[3].record(stream)
    torch.cuda.synchronize()
    eigh_ms = ev[2].elapsed_time(ev[3]) / args.dense_only
    chunk_flops = 28 * 2 * 128 * 32 * 32  # 28 pairs x (2 flops x M 128 x N 32 x K 32)
    pP, nP = 128 * math.ceil(p / 128), 32 * math.ceil(p / 32)
    gram_tiles = (pP // 128) * (C * nP // 32)
    gram_mma = gram_tiles * (C * 32 * math.ceil(n / 32) // 32) * chunk_flops
    upd_tiles = math.ceil(n / 128) * math.ceil(C * p / 32)
    upd_mma = upd_tiles * math.ceil(C * p / 32) * chunk_flops
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16 = float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        bf16 = 1900.0
    fp64_flops = (8 if cplx else 2) * n * p * p
    if dist.rank == 0:
        print(json.dumps({
            "mode": "dense-only", "workload": args.workload, "n": n, "p": p, "dtype": "c128" if cplx else "f64",
            "gram_ms": gram_ms, "gram_tensor_tflops": gram_mma / gram_ms / 1e9,
            "gram_tensor_frac_of_bf16_peak": gram_mma / gram_ms / 1e9 / bf16,
            "gram_fp64_equivalent_tflops": fp64_flops / gram_ms / 1e9,
            "update_ms": upd_ms, "update_tensor_tflops": upd_mma / upd_ms / 1e9,
            "update_tensor_frac_of_bf16_peak": upd_mma / upd_ms / 1e9 / bf16,
            "update_fp64_equivalent_tflops": fp64_flops / upd_ms / 1e9,
            "eigh_small_ms": eigh_ms,
            "bf16_peak_tflops": bf16, "calls": args.dense_only}), flush=True)


def main():
    args = parse()
    dist = Dist()
    try:
        if args.impl == "reference":
            reference_arm(args, dist)
        elif args.workload == "serving":
            serving_arm(args, dist)
        elif args.workload.endswith("_slices"):
            slices_arm(args, dist)
        elif args.workload == "sweep":
            sweep_arm(args, dist)
        else:
            ours_arm(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
