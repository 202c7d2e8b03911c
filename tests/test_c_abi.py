"""The C ABI used from plain C (tests/c_abi_solve.c: include/bcs.h and
libbcs.so, no Python or PyTorch in the process).  On the CPU: the program
compiles with gcc as C99 against the header, links against the library, and
the calls that need no device behave as declared.  On the GPU: a complete FP64
solve of each method from host buffers (bcs_csr_upload of host CSR arrays,
bcs_solve_host) returns the oracle's iterations, outer runs, replacement steps
and x, bit for bit."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIBDIR = os.path.join(ROOT, "paper_2108_10591_gb300")
CUDA_LIB = "/usr/local/cuda/lib64"


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    if not os.path.exists(os.path.join(LIBDIR, "libbcs.so")):
        pytest.skip("libbcs.so is not built")
    exe = str(tmp_path_factory.mktemp("cabi") / "c_abi_solve")
    cmd = [cc, "-std=c99", "-O1", "-Wall", "-Werror", "-I" + os.path.join(ROOT, "include"),
           os.path.join(HERE, "c_abi_solve.c"), "-o", exe, "-L" + LIBDIR, "-lbcs",
           "-Wl,-rpath," + LIBDIR]
    if os.path.isdir(CUDA_LIB):
        cmd += ["-Wl,-rpath-link," + CUDA_LIB]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_program_builds_and_checks_arguments_without_a_device(prog):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([prog, "--no-gpu"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, (r.stdout, r.stderr)
    assert "no-gpu checks ok" in r.stdout


def _write_system(path, A, b):
    with open(path, "wb") as fh:
        np.array([A.n, A.nnz], dtype=np.int64).tofile(fh)
        np.asarray(A.rowptr, dtype=np.int64).tofile(fh)
        np.asarray(A.col, dtype=np.int32).tofile(fh)
        np.asarray(A.val, dtype=np.float64).tofile(fh)
        np.asarray(b, dtype=np.float64).tofile(fh)


@pytest.mark.gpu
@pytest.mark.parametrize("kind", [0, 1, 2])
def test_c_program_solve_matches_oracle(prog, orc, tmp_path, kind):
    A = W.powerlaw(n=20001, seed=9)   # irregular rows, n not a multiple of 32
    b = W.rhs_ones(A)
    src, out = str(tmp_path / "sys.bin"), str(tmp_path / "x.bin")
    _write_system(src, A, b)
    r = subprocess.run([prog, src, out, str(kind)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.stdout, r.stderr)
    status, iters, outer, rr, rel = r.stdout.split()
    x = np.fromfile(out, dtype=np.float64)
    name = ["ssBiCGSafe2", "p-BiCGSafe", "p-BiCGSafe-rr"][kind]
    ref = orc.solve(A, b, kind=name, tol=1e-10, maxit=10000, rr_m=100, max_restarts=29)
    assert int(status) == 0 and ref["status_name"] == "ok"
    assert int(iters) == ref["iterations"] and int(outer) == ref["restarts"] + 1 and int(rr) == ref["rr_steps"]
    assert float.fromhex(rel) == ref["rel_res_true"]
    assert np.array_equal(x, ref["x"])
