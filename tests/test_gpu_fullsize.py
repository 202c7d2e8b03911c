"""Parity at the full sizes of the synthetic configurations, in the launch
configuration bench.py times (default options: one 24-warp CTA per SM, CSR one
lane per row).  The oracle cannot finish these solves in seconds, so the checks
are (a) the first 20 iterations, which the oracle can run, and (b) properties
that hold at any size, measured by the oracle on the GPU's output: the FP64
true residual ||b - A x|| / ||b|| <= 1e-10 at exit.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_10591_gb300 as bcs
    return bcs, torch, orc


@pytest.fixture(scope="module")
def cd3d(env):
    bcs, torch, orc = env
    A = W.cd3d_upwind(128, 50.0)
    b = W.rhs_ones(A)
    M = bcs.csr_upload(A, stores=bcs.STORE_F32)
    return A, b, M


@pytest.mark.parametrize("kind", ["ssBiCGSafe2", "p-BiCGSafe"])
def test_cd3d_128_first_20_iterations(env, cd3d, kind):
    """n = 2,097,152: residual history and scalars of the first 20 iterations against the
    oracle's; bound 1e-8 relative (the FP64 path is in fact bit-identical)."""
    bcs, torch, orc = env
    A, b, M = cd3d
    S = bcs.solver_create(M, kind, tol=0.0, maxit=20, max_outer=1)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    res = bcs.solve(S, bd, x)
    h, sc = bcs.get_history(S), bcs.get_scalars(S)
    ref = orc.solve(A, b, kind=kind, tol=0.0, maxit=20)
    assert res["iterations"] == ref["iterations"] == 20
    n = min(len(h), len(ref["hist"]))
    assert n >= 20
    assert np.all(np.abs(h[:n] - ref["hist"][:n]) <= 1e-8 * np.abs(ref["hist"][:n]))
    assert np.array_equal(h[:n], ref["hist"][:n])
    assert np.array_equal(sc[:20], ref["scalars"][:20])
    assert np.array_equal(x.cpu().numpy(), ref["x"])


@pytest.mark.parametrize("kind,prec", [("ssBiCGSafe2", "fp64"), ("p-BiCGSafe", "fp64"), ("p-BiCGSafe", "fp32"),
                                       ("p-BiCGSafe-rr", "fp32"), ("p-BiCGSafe-rr", "bf16")])
def test_cd3d_128_full_solve_true_residual(env, cd3d, kind, prec):
    """Full solves of the benchmark system to 1e-10: the FP64 true residual of the
    returned x, recomputed by the oracle, meets the tolerance."""
    bcs, torch, orc = env
    A, b, M = cd3d
    if prec == "bf16":
        M = bcs.csr_upload(A, stores=bcs.STORE_BF16)
    S = bcs.solver_create(M, kind, tol=1e-10, maxit=20000, precision=prec, max_outer=60)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    res = bcs.solve(S, bd, x)
    assert res["status"] == 0
    xh = x.cpu().numpy()
    rel = orc.true_residual(A, b, xh) / np.linalg.norm(b)
    assert rel <= 1e-10
    assert abs(rel - res["rel_res_true"]) <= 1e-3 * rel + 1e-16


def test_powerlaw_4m_fp32_refinement(env):
    """The irregular 4M-row configuration (power-law rows up to 512): FP32 values and vectors
    with FP64 refinement reach the FP64 tolerance, checked by the oracle's true residual."""
    bcs, torch, orc = env
    A = W.powerlaw()
    b = W.rhs_ones(A)
    M = bcs.csr_upload(A, stores=bcs.STORE_F32)
    for prec in ["fp32", "fp64"]:
        S = bcs.solver_create(M, "p-BiCGSafe-rr", tol=1e-10, maxit=20000, precision=prec, max_outer=30)
        bd = torch.from_numpy(b).cuda()
        x = torch.zeros_like(bd)
        res = bcs.solve(S, bd, x)
        assert res["status"] == 0
        assert orc.true_residual(A, b, x.cpu().numpy()) / np.linalg.norm(b) <= 1e-10
