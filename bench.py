#!/usr/bin/env python
"""Benchmark: time to a 1e-10 relative residual on the 3D convection-diffusion
workload (128^3, 7-point first-order upwind, n = 2,097,152, nnz = 14,581,760),
FP64, p-BiCGSafe (Alg. 4) with the FP64 true-residual check; plain
ssBiCGSafe2 (Alg. 3) and the mixed-precision pipelined solve are measured
beside it on the same system.

One step = one complete solve from x_0 = 0 to ||b - A x|| <= 1e-10 ||b||
(one persistent kernel launch).  `value` = solves/s over all ranks with
inputs resident in HBM; `e2e` = the same through bcs_solve_host (host b, x;
copies inside the timed region).  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-10 rel. residual, pipelined vs plain; HBM GB/s per iter; solves/s"
HBM_PEAK_FALLBACK = 6800.0
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 rate (nominal; the FP64 units also bound the FP64 kernel)
GOLDEN = os.path.join(ROOT, "tests", "golden", "cd3d128_full_solves.json")
# the oracle's complete FP64 solves of the side workloads (tests/golden/make_*_solves.py)
SIDE_GOLDEN = {"powerlaw_4m": "powerlaw_4m_full_solves.json", "cd3d27_192": "cd3d27_192_full_solves.json",
               "cd3d_128_pc": "cd3d128_full_solves.json", "batch_cd2d_512": "batch_cd2d_512_solves.json"}


# DRAM traffic of the solve kernel from ncu (dram__bytes_read.sum + dram__bytes_write.sum) on this
# workload, p-BiCGSafe, CSR: captures of 10- and 20-iteration solves, differenced for the bytes of one
# iteration; the intercept is the set-up and final true-residual work of an outer step.  Valid only
# for the kernel sources they were taken on (KERNEL_SHA); otherwise the bench reports null.
TRAFFIC = {"fp64": {"per_iter": 914.4e6, "per_outer": 1021.8e6},
           "fp32": {"per_iter": 381.3e6, "per_outer": 867.4e6}}
KERNEL_SHA = "37789c66f04d6fdc"


# The measured kernel's sources and its launch path.  Other translation units
# (batched solves, preconditioner set-up, the standalone inner products, tuning
# helpers) do not change the measured kernel.  Comments are stripped before
# hashing: editing a comment changes no compiled code.
KERNEL_FILES = ["solver.cuh", "device.cuh", "xacc.cuh", "internal.h", "api.cu", "matrix.cu",
                "solver_f64_0.cu", "solver_f64_1.cu", "solver_f64_2.cu",
                "solver_f32_0.cu", "solver_f32_1.cu", "solver_f32_2.cu",
                "solver_bf16_0.cu", "solver_bf16_1.cu", "solver_bf16_2.cu"]


def _code_only(text):
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def kernel_sources_sha():
    h = hashlib.sha256()
    files = [os.path.join(ROOT, "paper_2108_10591_gb300", "csrc", f) for f in KERNEL_FILES]
    files.append(os.path.join(ROOT, "include", "bcs.h"))
    for f in files:
        with open(f) as fh:
            h.update(os.path.basename(f).encode())
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


# Side workloads (the other synthetic configurations): one JSON line each, not the benchmark line.
SIDE_WORKLOADS = {
    "powerlaw_4m": "random nonsymmetric, n=4,194,304, power-law rows (exponent 2.1, mean 16, max 512), 90% of columns "
                   "within n/100 of the diagonal, N(0,1) values, diagonal 1.2 x row abs-sum",
    "cd3d27_192": "3D 27-point convection-diffusion, 192^3 (n=7,077,888), beta=100 on the face couplings",
    "batch_cd2d_512": "512 independent 2D 5-point convection-diffusion systems, side U{32..256}, beta U[0,50]",
    "cd3d_128_pc": "the benchmark's 128^3 upwind system as a side workload (preconditioned runs)",
}


def shard_systems(nsys, rank, world):
    """Systems of a batch taken by one rank (weak scaling, no collective): every world-th system
    of the list in decreasing size, so that the ranks' shares have about equal work."""
    return list(range(rank, nsys, world))


def max_over_ranks(value, dist=None, device=None):
    """Largest value over the ranks (the slowest rank's time); the value itself on one rank."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": HBM_PEAK_FALLBACK}, "fallback"


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kind", default="p-BiCGSafe")
    ap.add_argument("--tpr", type=int, default=0, help="CSR lanes per row (0 = library default)")
    ap.add_argument("--layout", default="csr")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--no-extras", action="store_true", help="skip the plain / mixed side measurements")
    ap.add_argument("--cpu-iters", type=int, default=30, help="oracle iterations in the CPU sample")
    ap.add_argument("--size", type=int, default=128, help="grid side k of the k^3 system (128 = the benchmark)")
    ap.add_argument("--maxit", type=int, default=10000, help="iteration limit (smaller for profiling runs)")
    ap.add_argument("--workload", default="cd3d_128", choices=list(SIDE_WORKLOADS) + ["cd3d_128"],
                    help="cd3d_128 (the benchmark line); the others print a side measurement line")
    ap.add_argument("--tune", action="store_true", help="side workloads: autotune the layout / lanes per row first")
    ap.add_argument("--precond", default="none", choices=["none", "jacobi", "block-jacobi"],
                    help="side workloads: preconditioner")
    ap.add_argument("--block-size", type=int, default=8, help="block-jacobi: rows per diagonal block")
    ap.add_argument("--matrix", default=None,
                    help="side measurement on a Matrix Market file (a supplied SuiteSparse matrix): b = A*1, x0 = 0")
    ap.add_argument("--big-ctas", type=int, default=-1,
                    help="batch: CTAs per cluster of the second lane for the largest systems (0 = one lane; "
                         "default: 8 with FP32/BF16 inner solves, where it was measured 10 %% faster, 0 in FP64, "
                         "where the batch is throughput-bound and it was slower)")
    ap.add_argument("--big-systems", type=int, default=0, help="batch: systems in the second lane (0 = automatic)")
    ap.add_argument("--profile", action="store_true",
                    help="only the timed solves (no end-to-end, side-by-side or CPU legs): the command profiled by ncu")
    return ap.parse_args()


def bench_config(a, n, nnz, world=1):
    """The `config` of the benchmark line (the same for both arms)."""
    return {"workload": "cd3d_%d: 3D -Lap u + 50(u_x+u_y+u_z), %d^3, 7-point upwind, n=%d, nnz=%d, "
                        "b=A*1, x0=0" % (a.size, a.size, n, nnz),
            "kind": a.kind, "precision": a.precision, "layout": a.layout, "tol": 1e-10,
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "no flush: matrix (183 MB) and vectors (16 x 16.8 MB) exceed the 129 MB L2"}


def make_workload(k=128):
    import workloads as W
    A = W.cd3d_upwind(k, 50.0)
    b = W.rhs_ones(A)
    return A, b


def oracle_golden():
    """The oracle's complete FP64 solves of the 128^3 system (iterations, outer runs, x digest and
    x at sampled rows), written by tests/golden/make_cd3d128_full_solves.py from oracle/ alone."""
    with open(GOLDEN) as fh:
        return json.load(fh)


def x_sha256(x):
    return hashlib.sha256(np.ascontiguousarray(x, dtype="<f8").tobytes()).hexdigest()


def error_vs_oracle(x, kind, gold):
    """Error of a returned x against the FP64 oracle's x for the same method: max |x - x_oracle|
    over the golden file's 4096 sampled rows, and whether the whole vector is bit-identical."""
    g = gold["solves"].get(kind)
    if g is None:
        return None
    rows = np.asarray(gold["sample_rows"])
    ref = np.array([float.fromhex(v) for v in g["x_sample"]])
    return {"oracle_kind": kind, "max_abs_err_sampled": float(np.max(np.abs(x[rows] - ref))),
            "sampled_rows": len(rows), "bit_identical": x_sha256(x) == g["x_sha256"],
            "oracle_iterations": g["iterations"], "oracle_outer_steps": g["outer_steps"]}


def error_vs_oracle_side(x, kind, n, gold):
    """error_vs_oracle for a side workload's returned x against the golden file's oracle solve of
    this system: by the same method when the file holds it, else by the first of p-BiCGSafe-rr,
    ssBiCGSafe2 and p-BiCGSafe that it holds (every one solved the system to 1e-10; oracle_kind
    says which)."""
    if gold is None or gold.get("n") != n:
        return None
    solves = gold.get("solves", {})
    ref = kind if kind in solves else next((k for k in ("p-BiCGSafe-rr", "ssBiCGSafe2", "p-BiCGSafe")
                                            if k in solves), None)
    return None if ref is None else error_vs_oracle(x, ref, gold)


def side_golden(workload):
    """The golden file of a side workload (the oracle's solves), or None."""
    f = SIDE_GOLDEN.get(workload)
    path = os.path.join(ROOT, "tests", "golden", f) if f else None
    if not path or not os.path.exists(path):
        return None
    with open(path) as fh:
        return json.load(fh)


def batch_sample_rows(n, k):
    """k evenly spaced rows of an n-row system, the first and the last included (the rows whose
    x values the batch golden file records)."""
    return np.unique(np.linspace(0, n - 1, k).round().astype(np.int64))


def batch_error_vs_oracle(xs, which, gold):
    """Error of the returned x of batched systems against the FP64 oracle's x of the same system
    (the golden file's method, named in oracle_kind): max |x - x_oracle| over the file's sampled
    rows of every system, and how many systems are bit-identical.  xs[j] is system which[j] of the
    batch (host arrays)."""
    if gold is None:
        return None
    err, same = 0.0, 0
    k = gold["samples_per_system"]
    for x, s in zip(xs, which):
        g = gold["systems"][s]
        ref = np.array([float.fromhex(v) for v in g["x_sample"]])
        err = max(err, float(np.max(np.abs(x[batch_sample_rows(len(x), k)] - ref))))
        same += x_sha256(x) == g["x_sha256"]
    return {"oracle_kind": gold["kind"], "systems_checked": len(which), "bit_identical_systems": same,
            "max_abs_err_sampled": err, "sampled_rows_per_system": k}


def oracle_check_small(bcs, torch):
    """Every method and precision on the 64x64 convection-diffusion system (4096 rows) against the
    FP64 oracle's solve of the same method: max |x - x_oracle| over the whole vector, and whether x
    is bit-identical (outside every timed region)."""
    import oracle
    import workloads as W
    A = W.cd2d(64, 20.0)
    b = W.rhs_ones(A)
    M = bcs.csr_upload(A, stores=bcs.STORE_F32 | bcs.STORE_BF16)
    bd = torch.from_numpy(b).cuda()
    out = {}
    for kind in ["ssBiCGSafe2", "p-BiCGSafe", "p-BiCGSafe-rr"]:
        ref = oracle.solve(A, b, kind=kind, tol=1e-10, maxit=10000, max_restarts=29)
        for prec in ["fp64", "fp32", "bf16"]:
            S = bcs.solver_create(M, kind, tol=1e-10, maxit=10000, precision=prec, max_outer=30)
            x = torch.zeros_like(bd)
            res = bcs.solve(S, bd, x)
            xh = x.cpu().numpy()
            out["%s_%s" % (kind, prec)] = {"status": res["status_name"], "iterations": res["iterations"],
                                           "oracle_iterations": ref["iterations"],
                                           "max_abs_err_vs_oracle": float(np.max(np.abs(xh - ref["x"]))),
                                           "bit_identical": bool(np.array_equal(xh, ref["x"]))}
    return out


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


# ---- algorithmic work per solve ---------------------------------------------------------

def flops_per_iter(kind, n, nnz):
    """FP64 flops of one iteration from Table 1: two SpMVs (2 flops per nonzero each) and the
    alpha*x and x+y counts per row (26 + 22 for p-BiCGSafe, 16 + 14 for ssBiCGSafe2).  The nine
    inner products run exactly on the integer units and are not counted against the FP64 peak."""
    ax, xy = (16, 14) if kind == "ssBiCGSafe2" else (26, 22)
    return 2 * 2 * nnz + (ax + xy) * n


def bytes_per_iter(kind, n, nnz, vbytes=8, mbytes=8):
    """Algorithmic HBM bytes of one iteration: two passes over the CSR matrix
    (values, int32 columns and row pointers) plus V + 2 vector passes (the two
    SpMV inputs read once each), V = 25 (p-BiCGSafe: 11 state vectors read and
    written, r* read, As written and re-read... lower bound) or 20 (ssBiCGSafe2)."""
    V = 20 if kind == "ssBiCGSafe2" else 25
    matrix = nnz * (mbytes + 4) + 4 * (n + 1)
    return 2 * matrix + (V + 2) * n * vbytes


def solve_work(kind, n, nnz, iters, outer, vbytes=8, mbytes=8):
    f = iters * flops_per_iter(kind, n, nnz) + outer * (2 * nnz + 4 * n)
    b = iters * bytes_per_iter(kind, n, nnz, vbytes, mbytes) + outer * (nnz * 12 + 4 * n * 8)
    if kind != "ssBiCGSafe2":
        f += outer * 2 * nnz
        b += outer * (nnz * (mbytes + 4) + 2 * n * vbytes)
    return f, b


# ---- clocks ---------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons)}


# ---- the CPU oracle baseline ---------------------------------------------------------------

def cpu_sample(A, b, kind, iters, parallel=False):
    """Time `iters` iterations of the CPU oracle on the full system: the single-threaded parity
    build, or (parallel) the same source built with OpenMP on every host core."""
    import oracle
    oracle.lib(parallel)
    t0 = time.perf_counter()
    o = oracle.solve(A, b, kind=kind, tol=0.0, maxit=iters, parallel=parallel)
    dt = time.perf_counter() - t0
    return dt, o


def reference_arm(a):
    """The oracle (all host cores) on the benchmark's workload: each step times a bounded sample of
    iterations, scaled to one solve by the oracle's own iteration count for that method (the
    golden file of its complete solves)."""
    A, b = make_workload(a.size)
    kind = a.kind
    gold = oracle_golden()
    cores = host_cores()
    times = []
    if a.size == 128 and kind in gold["solves"]:
        iters_full = gold["solves"][kind]["iterations"]
        per = max(2, min(a.cpu_iters, 20))
        for s in range(a.warmup + a.steps):
            dt, _ = cpu_sample(A, b, kind, per, parallel=True)
            if s >= a.warmup:
                times.append(dt)
        solve_s = sum(times) / (len(times) * per) * iters_full
        sample = ("each step: %d iterations of the FP64 oracle (OpenMP build of the same source, bit-identical, "
                  "%d threads) on the full system, scaled to one solve by the oracle's complete-solve count of "
                  "%d iterations" % (per, cores, iters_full))
    else:
        # a system outside the golden file: every step is one complete oracle solve (small grids only)
        import oracle
        oracle.lib(True)
        for s in range(a.warmup + a.steps):
            t0 = time.perf_counter()
            oracle.solve(A, b, kind=kind, tol=1e-10, maxit=a.maxit, max_restarts=29, parallel=True)
            if s >= a.warmup:
                times.append(time.perf_counter() - t0)
        solve_s = sum(times) / len(times)
        sample = ("each step: one complete solve to 1e-10 by the FP64 oracle (OpenMP build of the same source, "
                  "%d threads)" % cores)
    val = 1.0 / solve_s
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "solves/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": solve_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(a, A.n, A.nnz),
            "cpu_baseline": {"value": val, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- side workloads --------------------------------------------------------------------------

def side_single(a, bcs, torch, dist, world, rank):
    import workloads as W
    if a.matrix:
        A = W.read_matrix_market(a.matrix)
    else:
        A = (W.powerlaw() if a.workload == "powerlaw_4m" else W.cd3d_upwind(128, 50.0) if a.workload == "cd3d_128_pc"
             else W.cd3d27(192, 100.0))
    b = W.rhs_ones(A)
    layouts = bcs.LAYOUT_CSR | bcs.LAYOUT_SELL
    M = bcs.csr_upload(A, layouts=layouts, stores=bcs.STORE_F32 | bcs.STORE_BF16)
    tune = None
    if a.tune:
        best, cands = bcs.autotune(M, a.kind, precision=a.precision, iters=20)
        tune = {"best": best, "candidates": cands}
        layout, tpr = "auto", 0
    else:
        layout, tpr = a.layout, a.tpr
    pc = dict(precond=a.precond, block_size=a.block_size) if a.precond == "block-jacobi" else dict(precond=a.precond)
    S = bcs.solver_create(M, a.kind, tol=1e-10, maxit=a.maxit, precision=a.precision, layout=layout,
                          threads_per_row=tpr, max_outer=30, **pc)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    for _ in range(a.warmup):
        xd.zero_()
        bcs.solve(S, bd, xd)
    if a.profile:
        # only the solves (the command that ncu captures)
        for _ in range(a.steps):
            xd.zero_()
            r = bcs.solve(S, bd, xd)
        return {"profile_run": True, "workload": a.workload, "kind": a.kind, "precision": a.precision,
                "iterations": r["iterations"], "kernel_ms": r["seconds"] * 1e3}
    times, res = [], None
    for _ in range(a.steps):
        xd.zero_()
        res = bcs.solve(S, bd, xd)
        times.append(res["seconds"])
    t = max_over_ranks(statistics.mean(times), dist, "cuda")
    lo = a.precision != "fp64"
    vb, mb = (4, 4 if a.precision == "fp32" else 2) if lo else (8, 8)
    _, by = solve_work(a.kind, A.n, A.nnz, res["iterations"], res["outer_steps"], vb, mb)
    if a.precond == "block-jacobi":
        # two M^-1 applications per iteration: each reads bs entries of M^-1 per row and writes one copy
        by += 2.0 * res["iterations"] * A.n * (a.block_size + 1) * vb
    peaks, src = measured_peaks()
    gbs = by / t / 1e9
    hp = float(peaks.get("hbm_gbs", HBM_PEAK_FALLBACK))
    return {"metric": "time to 1e-10 rel. residual", "value": world / t, "unit": "solves/s", "n_gpus": world,
            "ms_per_solve": t * 1e3, "iterations": res["iterations"], "outer_steps": res["outer_steps"],
            "us_per_iter": t * 1e6 / max(1, res["iterations"]), "status": res["status_name"],
            "rel_res_true": res["rel_res_true"],
            "error_vs_oracle": None if a.matrix else error_vs_oracle_side(xd.cpu().numpy(), a.kind, A.n,
                                                                         side_golden(a.workload)),
            "config": {"workload": ("Matrix Market file %s" % os.path.basename(a.matrix)) if a.matrix else
                       "%s: %s" % (a.workload, SIDE_WORKLOADS[a.workload]), "n": A.n, "nnz": A.nnz,
                       "kind": a.kind, "precision": a.precision, "layout": layout, "threads_per_row": tpr,
                       "precond": a.precond,
                       "block_size": a.block_size if a.precond == "block-jacobi" else None},
            "hbm": {"achieved": gbs, "peak": hp, "unit": "GB/s", "frac": gbs / hp, "peak_source": src},
            "tune": tune}


def side_batch(a, bcs, torch, dist, world, rank):
    import workloads as W
    mats, sides, betas = W.batch_cd2d(512)
    order = sorted(range(len(mats)), key=lambda k: -(mats[k].nnz + mats[k].n))
    mine = [order[k] for k in shard_systems(len(order), rank, world)]
    mats = [mats[k] for k in mine]
    Ms = [bcs.csr_upload(A, stores=bcs.STORE_F32 | bcs.STORE_BF16) for A in mats]
    big = a.big_ctas if a.big_ctas >= 0 else (0 if a.precision == "fp64" else 8)
    kw = dict(precision=a.precision, max_outer=30, big_ctas=big, big_systems=a.big_systems)
    if a.kind == "p-BiCGSafe-rr":
        kw["rr_m"] = 20
    tune = None
    if a.tune:
        kw, cands = bcs.batch_autotune(Ms, kind=a.kind, iters=20, **kw)
        tune = {"options": {"threads_per_row": kw["threads_per_row"], "ctas_per_sm": kw["ctas_per_sm"]},
                "candidates": cands}
    bt = bcs.Batch(Ms, kind=a.kind, tol=1e-10, maxit=a.maxit, **kw)
    offs = np.cumsum([0] + [A.n for A in mats])
    bflat = torch.from_numpy(np.concatenate([W.rhs_ones(A) for A in mats])).cuda()
    xflat = torch.zeros_like(bflat)
    bs = [bflat[offs[k]:offs[k + 1]] for k in range(len(mats))]
    xs = [xflat[offs[k]:offs[k + 1]] for k in range(len(mats))]
    for _ in range(a.warmup):
        xflat.zero_()
        bt.solve(bs, xs)
    times, res, code = [], None, 0
    for _ in range(a.steps):
        xflat.zero_()
        code, res = bt.solve(bs, xs)
        times.append(res[0]["seconds"])
    t = max_over_ranks(statistics.mean(times), dist, "cuda")
    its = [r["iterations"] for r in res]
    ok = sum(1 for r in res if r["status"] == 0)
    t0 = min(r["t_start"] for r in res)
    spans = sorted(((r["t_end"] - r["t_start"]) * 1e-6, A.n) for r, A in zip(res, mats))
    ends = sorted((r["t_end"] - t0) * 1e-6 for r in res)
    return {"metric": "solves/s", "value": 512 / t, "unit": "solves/s", "n_gpus": world, "ms_per_batch": t * 1e3,
            "systems": 512, "systems_this_rank": len(mats), "converged_this_rank": ok, "worst_status": code,
            "iterations": {"min": min(its), "median": float(np.median(its)), "max": max(its)},
            "max_rel_res_true": max(r["rel_res_true"] for r in res),
            "error_vs_oracle": batch_error_vs_oracle([x.cpu().numpy() for x in xs], mine, side_golden(a.workload)),
            "per_system_ms": {"median": spans[len(spans) // 2][0], "max": spans[-1][0], "max_n": spans[-1][1],
                              "last_finish": ends[-1], "p90_finish": ends[int(0.9 * (len(ends) - 1))]},
            "config": {"workload": "%s: %s" % (a.workload, SIDE_WORKLOADS[a.workload]), "kind": a.kind,
                       "precision": a.precision, "batch_options": {k: kw[k] for k in kw
                                                                    if k in ("threads_per_row", "ctas_per_sm",
                                                                             "big_ctas", "big_systems")},
                       "parallelism": "systems sharded over ranks" if world > 1 else "single GPU"},
            "tune": tune}


# ---- our arm ---------------------------------------------------------------------------------

def main():
    a = args_parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        if rank == 0:
            reference_arm(a)
        return
    import torch
    torch.cuda.set_device(local)   # before the process group: NCCL binds this rank to its GPU
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    import paper_2108_10591_gb300 as bcs

    if a.workload != "cd3d_128" or a.matrix:
        fn = side_batch if (a.workload == "batch_cd2d_512" and not a.matrix) else side_single
        line = fn(a, bcs, torch, dist, world, rank)
        if rank == 0:
            line["data"] = "matrix file" if a.matrix else "synthetic"
            line["side_measurement"] = True
            print(json.dumps(line), flush=True)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    A, b = make_workload(a.size)
    n, nnz = A.n, A.nnz
    gold = oracle_golden() if a.size == 128 else None
    layouts = bcs.LAYOUT_CSR | (bcs.LAYOUT_SELL if a.layout == "sell" else 0)
    M = bcs.csr_upload(A, layouts=layouts, stores=bcs.STORE_F32 | bcs.STORE_BF16)
    stream = torch.cuda.current_stream()
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    solvers = {}

    def get_solver(kind, precision="fp64"):
        key = (kind, precision)
        if key not in solvers:
            solvers[key] = bcs.solver_create(M, kind, tol=1e-10, maxit=a.maxit, precision=precision,
                                             threads_per_row=a.tpr, layout=a.layout, max_outer=30)
        return solvers[key]

    def run(kind, precision, steps, warmup, clocks=None):
        S = get_solver(kind, precision)
        for _ in range(warmup):
            xd.zero_()
            bcs.solve(S, bd, xd, stream=stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * steps)]
        results = []
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(steps):
            xd.zero_()
            ev[2 * k].record(stream)
            results.append(bcs.solve(S, bd, xd, stream=stream))
            ev[2 * k + 1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        total_ms = t0.elapsed_time(t1)
        per = [ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(steps)]
        # accuracy of the last solve against the exact solution of A x = A 1 and against the FP64
        # oracle's x for the same method (outside the timed region)
        results[-1]["max_abs_err_vs_ones"] = float((xd - 1.0).abs().max().item())
        if gold is not None:
            results[-1]["error_vs_oracle"] = error_vs_oracle(xd.cpu().numpy(), kind, gold)
        return total_ms, per, results

    if a.profile:
        total_ms, per, results = run(a.kind, a.precision, a.steps, a.warmup)
        r0 = results[-1]
        if rank == 0:
            print(json.dumps({"profile_run": True, "kind": a.kind, "precision": a.precision, "layout": a.layout,
                              "size": a.size, "iterations": r0["iterations"], "status": r0["status_name"],
                              "kernel_ms": statistics.mean(per)}), flush=True)
        return
    with Clocks(local) as ck:
        total_ms, per, results = run(a.kind, a.precision, a.steps, a.warmup)
    clocks = ck.summary()
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / a.steps
    r0 = results[-1]
    ok = all(r["status"] == 0 and r["rel_res_true"] <= 1e-10 for r in results)
    iters, outer = r0["iterations"], r0["outer_steps"]
    kernel_ms = statistics.mean(per)

    # roofline of the solve kernel (the only kernel in the step): HBM, on the algorithmic bytes of
    # the solve (two matrix passes and V + 2 vector passes per iteration, plus each outer step's
    # set-up), against the measured copy bandwidth; the FP64 units' share beside it
    peaks, peak_src = measured_peaks()
    lo = a.precision != "fp64"
    vb, mb = (4, 4 if a.precision == "fp32" else 2) if lo else (8, 8)
    f, by = solve_work(a.kind, n, nnz, iters, outer, vb, mb)
    achieved_tf = f / (kernel_ms * 1e-3) / 1e12
    achieved_gbs = by / (kernel_ms * 1e-3) / 1e9
    hbm_peak = float(peaks.get("hbm_gbs", HBM_PEAK_FALLBACK))
    traffic = None
    tr = TRAFFIC.get(a.precision)
    if (tr and a.kind == "p-BiCGSafe" and a.layout == "csr" and a.size == 128 and a.tpr in (0, 1)
            and kernel_sources_sha() == KERNEL_SHA):
        traffic = tr["per_iter"] * iters + tr["per_outer"] * outer
    kname = "solve_kernel<%s,%s,%s,1,static>" % ("float" if lo else "double",
                                        {"fp64": "double", "fp32": "float", "bf16": "bf16"}[a.precision],
                                        a.layout.upper())
    roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved_gbs / hbm_peak, "traffic": traffic, "kernel": kname,
                "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_src if peak_src == "measured"
                else "fallback 6800 GB/s",
                "algorithmic_bytes": by, "traffic_vs_algorithmic": None if traffic is None else traffic / by}
    if not lo:
        roofline["fp64_units"] = {"achieved": achieved_tf, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                                  "frac": achieved_tf / FP64_NOMINAL_TFLOPS,
                                  "peak_source": "nominal GB300 FP64 rate (Table 1 flops: 2 SpMVs + 48 "
                                                 "vector flops per row per iteration)"}

    # end to end through the public API with host buffers
    bh = torch.from_numpy(b).pin_memory().numpy()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory().numpy()
    S = get_solver(a.kind, "fp64")
    for _ in range(max(1, a.warmup)):
        xh[:] = 0.0
        bcs.solve_host(S, bh, xh, stream=stream)
    torch.cuda.synchronize()
    t = time.perf_counter()
    e2e_steps = max(3, a.steps // 2)
    for _ in range(e2e_steps):
        xh[:] = 0.0
        bcs.solve_host(S, bh, xh, stream=stream)
    e2e_s = (time.perf_counter() - t) / e2e_steps
    if dist:
        tt = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_s = float(tt.item())

    extras = {}
    if not a.no_extras:
        for kind, prec in [("ssBiCGSafe2", "fp64"), ("p-BiCGSafe", "fp32"), ("ssBiCGSafe2", "fp32"),
                           ("p-BiCGSafe-rr", "fp64")]:
            tm, pr, rs = run(kind, prec, 3, 1)
            rr = rs[-1]
            e = {"ms_per_solve": tm / 3, "iterations": rr["iterations"], "outer_steps": rr["outer_steps"],
                 "rel_res_true": rr["rel_res_true"], "max_abs_err_vs_ones": rr["max_abs_err_vs_ones"],
                 "error_vs_oracle": rr.get("error_vs_oracle"), "status": rr["status_name"],
                 "us_per_iter": 1e3 * tm / 3 / max(1, rr["iterations"])}
            pvb, pmb = (8, 8) if prec == "fp64" else (4, 4 if prec == "fp32" else 2)
            _, pby = solve_work(kind, n, nnz, rr["iterations"], rr["outer_steps"], pvb, pmb)
            pgbs = pby / (statistics.mean(pr) * 1e-3) / 1e9
            e["hbm"] = {"achieved": pgbs, "peak": hbm_peak, "unit": "GB/s", "frac": pgbs / hbm_peak}
            extras["%s_%s" % (kind, prec)] = e

    small = oracle_check_small(bcs, torch) if rank == 0 else None
    line = None
    if rank == 0:
        cpu = None
        if world == 1:
            # the oracle's own complete-solve iteration count scales the samples (the GPU's when the
            # golden file does not cover this configuration)
            g_it = gold["solves"][a.kind]["iterations"] if gold and a.kind in gold["solves"] else iters
            cores = host_cores()
            dtp, _ = cpu_sample(A, b, a.kind, a.cpu_iters, parallel=True)
            dt1, _ = cpu_sample(A, b, a.kind, a.cpu_iters)
            cpu = {"value": a.cpu_iters / (dtp * g_it), "unit": "solves/s", "cores": cores, "kind": "oracle",
                   "sample": "%d iterations of the FP64 oracle (%s; OpenMP build of the same source, bit-identical, "
                             "%d threads) on the full system in %.2f s, scaled to one solve by the oracle's %d "
                             "iterations" % (a.cpu_iters, a.kind, cores, dtp, g_it),
                   "single_thread": {"value": a.cpu_iters / (dt1 * g_it), "unit": "solves/s", "cores": 1,
                                     "sample": "the same %d iterations with the single-threaded parity build in "
                                               "%.1f s" % (a.cpu_iters, dt1)}}
        line = {"metric": METRIC, "value": world * 1e3 / ms_per_step, "unit": "solves/s", "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "fp32": "f32", "bf16": "bf16"}[a.precision], "data": "synthetic",
                "config": bench_config(a, n, nnz, world),
                "iterations": iters, "outer_steps": outer, "converged_all_steps": ok,
                "rel_res_true": r0["rel_res_true"], "max_abs_err_vs_ones": r0["max_abs_err_vs_ones"],
                "error_vs_oracle": r0.get("error_vs_oracle"),
                "kernel_ms": kernel_ms,
                "us_per_iter": 1e3 * kernel_ms / max(1, iters),
                "gb_per_s_per_iter": achieved_gbs,
                "roofline": roofline,
                "e2e": {"value": world / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": 2 * n * 8,
                        "d2h_bytes_per_step": n * 8 + 16 * 8},
                "gpu_launches": a.steps,
                "clocks": clocks,
                "cpu_baseline": cpu,
                "side_by_side": extras,
                "oracle_check_cd2d_64": small}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
