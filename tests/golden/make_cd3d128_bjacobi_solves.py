"""Writes cd3d128_bjacobi_solves.json: the oracle's complete FP64 solves of the
128^3 convection-diffusion system (n = 2,097,152, 7-point first-order upwind,
beta = 50, b = A*1, x_0 = 0) with block-Jacobi right preconditioning, to a
1e-10 relative true residual, with the true-residual restarts of the exit
check (at most 30 runs, 10,000 iterations in all): p-BiCGSafe with blocks of 4
rows, p-BiCGSafe-rr (m = 100) with blocks of 2 and ssBiCGSafe2 with blocks of 8.

Only oracle/ and the input generator are called; nothing here touches the
CUDA library.  The oracle's all-cores build is used for speed; it gives the
parity build's bits (tests/test_oracle_pins.py pins that):

    python tests/golden/make_cd3d128_bjacobi_solves.py

Recorded per solve: iterations (summed over the runs), outer runs, replacement
steps, status, the relative true residual, the SHA-256 digest of the returned
x (little-endian FP64 bytes), max |x_i - 1|, and x at 4096 evenly spaced rows.
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "cd3d128_bjacobi_solves.json")
SOLVES = [("p-BiCGSafe", 4), ("p-BiCGSafe-rr", 2), ("ssBiCGSafe2", 8)]
OPTIONS = {"tol": 1e-10, "maxit": 10000, "max_runs": 30, "rr_m": 100, "rr_M": 10001}
NSAMPLE = 4096


def sample_rows(n, k=NSAMPLE):
    """k evenly spaced rows, the first and the last included."""
    return np.unique(np.linspace(0, n - 1, k).round().astype(np.int64))


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<f8").tobytes()).hexdigest()


def main():
    A = W.cd3d_upwind(128, 50.0)
    b = W.rhs_ones(A)
    rows = sample_rows(A.n)
    out = {"workload": "cd3d_128: -Lap u + 50(u_x+u_y+u_z), 128^3, h=1/129, 7-point first-order upwind, "
                       "b=A*1, x0=0; block-Jacobi right preconditioning",
           "n": A.n, "nnz": A.nnz, "options": OPTIONS, "b_sha256": digest(b),
           "sample_rows": rows.tolist(), "solves": {}}
    for kind, bs in SOLVES:
        t0 = time.time()
        r = oracle.solve_bjacobi(A, b, bs, kind=kind, tol=OPTIONS["tol"], maxit=OPTIONS["maxit"],
                                 rr_m=OPTIONS["rr_m"], rr_M=OPTIONS["rr_M"], max_restarts=OPTIONS["max_runs"] - 1,
                                 hist_cap=16, parallel=True)
        x = r["x"]
        out["solves"]["%s/%d" % (kind, bs)] = {
            "kind": kind, "block_size": bs,
            "status": r["status_name"], "iterations": r["iterations"], "outer_steps": r["restarts"] + 1,
            "rr_steps": r["rr_steps"], "rel_res_true": float(r["rel_res_true"]).hex(),
            "x_sha256": digest(x), "max_abs_err_vs_ones": float(np.max(np.abs(x - 1.0))),
            "x_sample": [float(v).hex() for v in x[rows]], "oracle_seconds": round(time.time() - t0, 1)}
        print(kind, bs, {k: v for k, v in out["solves"]["%s/%d" % (kind, bs)].items() if k != "x_sample"},
              flush=True)
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
