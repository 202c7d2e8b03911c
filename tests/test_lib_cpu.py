"""CPU-only checks of the C ABI library: it loads, exports every entry point
that include/bcs.h declares, and its host-side argument checks return the
documented codes without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bcs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2108_10591_gb300 as m
    return m


def declared_symbols():
    """Every bcs_* function that a header under include/ declares."""
    syms = set()
    for name in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if name.endswith(".h"):
            src = open(os.path.join(ROOT, "include", name)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            syms.update(re.findall(r"\b(bcs_[a-z_0-9]+)\s*\(", src))
    return sorted(syms)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ["bcs_csr_upload", "bcs_solver_create", "bcs_solve", "bcs_solve_batched"]:
        assert s in syms


def test_library_exports_every_declared_symbol(bcs):
    lib = ctypes.CDLL(bcs.LIB_PATH)
    for s in declared_symbols():
        assert hasattr(lib, s), s
    assert sorted(declared_symbols()) == sorted(bcs.EXPORTED)


def test_status_strings(bcs):
    for code in [0, 1, -1, -2, -3, -4, -5, -6]:
        assert bcs.status_string(code) not in ("", "unknown status")
    assert bcs.status_string(12345) == "unknown status"


def test_options_default(bcs):
    o = bcs.options()
    assert o.rr_m == 100 and o.precision == bcs.FP64 and o.max_outer == 30 and o.inner_tol == 1e-2 and o.inner_stall == 20
    assert o.layout == bcs.LAYOUT_AUTO and o.threads_per_row == 0 and o.spin_budget_ms > 0


def test_argument_checks_without_gpu(bcs):
    lib = bcs.lib
    h = ctypes.c_void_p()
    rp = np.array([0, 1], dtype=np.int64)
    ci = np.array([0], dtype=np.int32)
    va = np.array([1.0])
    # negative sizes, bad layouts, bad SELL parameters, null output
    assert lib.bcs_csr_upload(-1, 0, rp.ctypes.data, None, None, 1, 32, 256, 1, None, ctypes.byref(h)) == bcs.ERR_ARG
    assert lib.bcs_csr_upload(1, 1, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, 0, 32, 256, 1, None,
                              ctypes.byref(h)) == bcs.ERR_ARG
    assert lib.bcs_csr_upload(1, 1, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, 2, 16, 256, 1, None,
                              ctypes.byref(h)) == bcs.ERR_ARG
    assert lib.bcs_csr_upload(1, 1, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, 2, 32, 100, 1, None,
                              ctypes.byref(h)) == bcs.ERR_ARG
    assert lib.bcs_csr_upload(1, 1, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, 1, 32, 256, 1, None,
                              None) == bcs.ERR_ARG
    assert lib.bcs_csr_upload(1, 1, rp.ctypes.data, None, None, 1, 32, 256, 1, None, ctypes.byref(h)) == bcs.ERR_ARG
    o = bcs.options()
    assert lib.bcs_solver_create(None, 0, 1e-8, 10, ctypes.byref(o), ctypes.byref(h)) == bcs.ERR_ARG
    assert lib.bcs_solve(None, None, None, None, None) == bcs.ERR_ARG
    assert lib.bcs_solve_host(None, None, None, None, None) == bcs.ERR_ARG
    assert lib.bcs_get_history(None, None, 0, None) == bcs.ERR_ARG
    assert lib.bcs_spmv(None, 1, 1, None, None, 0, 0, None) == bcs.ERR_ARG
    assert lib.bcs_solve_batched(-1, None, 0, 1e-8, 10, None, None, None, None, None) == bcs.ERR_ARG
    assert lib.bcs_solve_batched(0, None, 0, 1e-8, 10, None, None, None, None, None) == bcs.OK
    assert lib.bcs_solve_batched(1, None, 7, 1e-8, 10, None, None, None, None, None) == bcs.ERR_ARG
    sig = (ctypes.c_int * 2)(32, 256)
    best = ctypes.c_int()
    assert lib.bcs_autotune_sell_sigma(None, 1, 0, 10, sig, 2, None, ctypes.byref(best), None, None) == bcs.ERR_ARG
    lib.bcs_matrix_free(None)
    lib.bcs_solver_destroy(None)


def test_host_tensors_are_refused_before_the_library(bcs):
    """A CPU tensor passed where the library expects device memory is refused by the binding
    (its pointer would otherwise be read by a kernel as a device address)."""
    torch = pytest.importorskip("torch")
    x = torch.ones(8, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA tensor"):
        bcs.dot(x, x)
    with pytest.raises(ValueError, match="CUDA tensor"):
        bcs.dot_noalloc(x, x, torch.zeros(1, dtype=torch.float64))


def test_import_fails_loudly_without_the_library(tmp_path):
    """The binding has no CPU fallback: a package directory without libbcs.so refuses to
    import, naming the missing library."""
    import shutil
    import subprocess
    import sys
    pkg = tmp_path / "paper_2108_10591_gb300"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "paper_2108_10591_gb300", "__init__.py"), pkg / "__init__.py")
    r = subprocess.run([sys.executable, "-c", "import paper_2108_10591_gb300"], cwd=str(tmp_path),
                       capture_output=True, text=True, env=dict(os.environ, PYTHONPATH=str(tmp_path)))
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "libbcs.so is not built" in r.stderr
