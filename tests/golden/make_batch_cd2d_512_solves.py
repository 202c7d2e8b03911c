"""Writes batch_cd2d_512_solves.json: the oracle's complete FP64 solves of the
512 independent 2D 5-point convection-diffusion systems of the batched
workload (grid side k ~ U{32..256}, beta ~ U[0, 50], b = A*1, x_0 = 0), each
to a 1e-10 relative true residual with p-BiCGSafe-rr (Algorithm 5, m = 20),
with the true-residual restarts of the exit check (at most 30 runs, 10,000
iterations in all).

Only oracle/ and the input generator are called; nothing here touches the
CUDA library.  The systems are solved by a pool of worker processes, one
system per task, with the oracle's single-threaded parity build:

    python tests/golden/make_batch_cd2d_512_solves.py

Recorded per system: side, n, status, iterations (summed over the runs), outer
runs, replacement steps, the relative true residual, SHA-256 digests of b and
of the returned x (little-endian FP64 bytes), and x at 16 evenly spaced rows
(hex floats; the rows are sample_rows(n)).
"""
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "batch_cd2d_512_solves.json")
KIND = "p-BiCGSafe-rr"
OPTIONS = {"tol": 1e-10, "maxit": 10000, "max_runs": 30, "rr_m": 20, "rr_M": 10001}


NSAMPLE = 16


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<f8").tobytes()).hexdigest()


def sample_rows(n, k=NSAMPLE):
    """k evenly spaced rows of an n-row system, the first and the last included."""
    return np.unique(np.linspace(0, n - 1, k).round().astype(np.int64))


_BATCH = {}


def solve_one(k):
    sys.path.insert(0, ROOT)
    import oracle
    import workloads as W
    if not _BATCH:   # the systems, generated once per worker process
        _BATCH["mats"], _BATCH["sides"], _ = W.batch_cd2d(512)
    mats, sides = _BATCH["mats"], _BATCH["sides"]
    A = mats[k]
    b = W.rhs_ones(A)
    r = oracle.solve(A, b, kind=KIND, tol=OPTIONS["tol"], maxit=OPTIONS["maxit"], rr_m=OPTIONS["rr_m"],
                     rr_M=OPTIONS["rr_M"], max_restarts=OPTIONS["max_runs"] - 1, hist_cap=16)
    return {"side": int(sides[k]), "n": int(A.n), "status": r["status_name"], "iterations": r["iterations"],
            "outer_steps": r["restarts"] + 1, "rr_steps": r["rr_steps"],
            "rel_res_true": float(r["rel_res_true"]).hex(), "b_sha256": digest(b), "x_sha256": digest(r["x"]),
            "x_sample": [float(v).hex() for v in r["x"][sample_rows(A.n)]]}


def main():
    t0 = time.time()
    with mp.get_context("spawn").Pool(os.cpu_count() or 4) as pool:
        systems = pool.map(solve_one, range(512), chunksize=4)
    out = {"workload": "batch_cd2d_512: 512 cd2d systems, side U{32..256}, beta U[0,50], b=A*1, x0=0",
           "kind": KIND, "options": OPTIONS, "samples_per_system": NSAMPLE, "systems": systems,
           "oracle_seconds": round(time.time() - t0, 1)}
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=0)
        fh.write("\n")
    its = [s["iterations"] for s in systems]
    print("systems %d, statuses %s, iterations %d..%d, %.1f s" % (
        len(systems), sorted(set(s["status"] for s in systems)), min(its), max(its), time.time() - t0))


if __name__ == "__main__":
    main()
