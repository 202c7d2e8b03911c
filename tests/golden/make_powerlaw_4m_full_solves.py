"""Writes powerlaw_4m_full_solves.json: the oracle's complete FP64 solves of the
random power-law system (n = 4,194,304; row lengths from a truncated power law,
exponent 2.1, mean 16, max 512; 90 % of the columns within n/100 of the
diagonal; N(0,1) values; diagonal 1.2 x the row's absolute sum; b = A*1,
x_0 = 0) to a 1e-10 relative true residual, for ssBiCGSafe2 (Algorithm 3),
p-BiCGSafe (Algorithm 4) and p-BiCGSafe-rr (Algorithm 5, m = 100), with the
true-residual restarts of the exit check (at most 30 runs, 20,000 iterations
in all).

Only oracle/ and the input generator are called; nothing here touches the
CUDA library.  The oracle's all-cores build is used for speed; it gives the
parity build's bits (tests/test_oracle_pins.py pins that):

    python tests/golden/make_powerlaw_4m_full_solves.py

Recorded per method: iterations (summed over the runs), outer runs,
replacement steps, status, the relative true residual, SHA-256 digests of
b and of the returned x (little-endian FP64 bytes), max |x_i - 1|, and x at
4096 evenly spaced rows (hex floats).
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

OUT = os.path.join(HERE, "powerlaw_4m_full_solves.json")
KINDS = ["ssBiCGSafe2", "p-BiCGSafe", "p-BiCGSafe-rr"]
OPTIONS = {"tol": 1e-10, "maxit": 20000, "max_runs": 30, "rr_m": 100, "rr_M": 20001}
NSAMPLE = 4096


def sample_rows(n, k=NSAMPLE):
    """k evenly spaced rows, the first and the last included."""
    return np.unique(np.linspace(0, n - 1, k).round().astype(np.int64))


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<f8").tobytes()).hexdigest()


def main():
    A = W.powerlaw()
    b = W.rhs_ones(A)
    rows = sample_rows(A.n)
    out = {"workload": "powerlaw_4m: random nonsymmetric, power-law rows (exponent 2.1, mean 16, max 512), "
                       "90% of columns within n/100 of the diagonal, N(0,1) values, diagonal 1.2 x row abs-sum, "
                       "b=A*1, x0=0",
           "n": A.n, "nnz": A.nnz, "options": OPTIONS, "b_sha256": digest(b),
           "sample_rows": rows.tolist(), "solves": {}}
    for kind in KINDS:
        t0 = time.time()
        r = oracle.solve(A, b, kind=kind, tol=OPTIONS["tol"], maxit=OPTIONS["maxit"], rr_m=OPTIONS["rr_m"],
                         rr_M=OPTIONS["rr_M"], max_restarts=OPTIONS["max_runs"] - 1, hist_cap=16, parallel=True)
        x = r["x"]
        out["solves"][kind] = {
            "status": r["status_name"], "iterations": r["iterations"], "outer_steps": r["restarts"] + 1,
            "rr_steps": r["rr_steps"], "rel_res_true": float(r["rel_res_true"]).hex(),
            "x_sha256": digest(x), "max_abs_err_vs_ones": float(np.max(np.abs(x - 1.0))),
            "x_sample": [float(v).hex() for v in x[rows]], "oracle_seconds": round(time.time() - t0, 1)}
        print(kind, {k: v for k, v in out["solves"][kind].items() if k != "x_sample"}, flush=True)
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
