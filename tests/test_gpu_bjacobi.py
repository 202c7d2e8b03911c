"""GPU parity of block-Jacobi right preconditioning (bcs.h, BCS_PRECOND_BLOCK_JACOBI)
against the oracle's orc_solve_bjacobi on the same seeded inputs:
  - the diagonal blocks and their Gauss-Jordan inverses: bit-exact (the same
    operations per element on both sides);
  - FP64 solves: every product gathers M^-1 v formed with the oracle's fma
    order, the inner products are correctly rounded on both sides, so the
    residual histories, scalars, iteration counts and x are bit-identical;
  - refinement modes: FP64 true residual of the original system <= 1e-10 and x
    within 1e-7 of the FP64 oracle's.
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


def _pivoting_matrix(n, seed):
    """Random nonsymmetric matrix whose diagonal blocks need row swaps (small diagonal)."""
    rng = np.random.default_rng(seed)
    Ad = np.where(rng.random((n, n)) < 0.2, rng.standard_normal((n, n)), 0.0)
    Ad += np.diag(rng.uniform(0.05, 0.5, n))
    for i in range(n):   # strong couplings inside the 8-row blocks keep the matrix well conditioned
        j = (i // 8) * 8 + (i + 3) % 8
        if j < n:
            Ad[i, j] += 4.0
    return W.dense_to_csr(Ad)


MATS = {
    "cd2d_64": lambda: W.cd2d(64, 20.0),
    "powerlaw_20001": lambda: W.powerlaw(n=20001, seed=9),
    "pivoting_203": lambda: _pivoting_matrix(203, 4),
}


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("bs", [1, 2, 4, 8, 16, 32])
def test_bjacobi_blocks_bit_exact(env, name, bs):
    """D and E = D^-1 (Gauss-Jordan, partial pivoting) equal the oracle's bit for bit, ragged
    last blocks included."""
    bcs, torch, orc = env
    A = MATS[name]()
    try:
        D0, E0 = orc.bjacobi_blocks(A, bs)
    except ValueError:
        pytest.skip("singular block for this size")
    M = bcs.csr_upload(A)
    S = bcs.solver_create(M, "p-BiCGSafe", precond="block-jacobi", block_size=bs)
    D, E = bcs.precond_blocks(S)
    assert np.array_equal(D, D0)
    assert np.array_equal(E, E0)


def _gpu_solve(bcs, torch, A, b, kind, x0=None, **kw):
    M = bcs.csr_upload(A, stores=bcs.STORE_F32 | bcs.STORE_BF16)
    S = bcs.solver_create(M, kind, tol=kw.pop("tol", 1e-10), maxit=kw.pop("maxit", 5000), precond="block-jacobi",
                          **kw)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd) if x0 is None else torch.from_numpy(x0.copy()).cuda()
    res = bcs.solve(S, bd, xd)
    return res, xd.cpu().numpy(), bcs.get_history(S), bcs.get_scalars(S)


@pytest.mark.parametrize("kind", ["ssBiCGSafe2", "p-BiCGSafe", "p-BiCGSafe-rr"])
@pytest.mark.parametrize("name,bs,cfg", [("cd2d_64", 8, {}), ("cd2d_64", 1, {}), ("cd2d_64", 32, dict(max_ctas=3)),
                                         ("powerlaw_20001", 4, dict(max_ctas=16)),
                                         ("pivoting_203", 8, dict(max_ctas=1))])
def test_bjacobi_solve_bit_identical(env, kind, name, bs, cfg):
    """FP64: histories, scalars, iteration, outer-step and replacement counts and x
    bit-identical to the oracle's preconditioned runs (several grid sizes, ragged n; a
    replacement every 10 iterations for p-BiCGSafe-rr)."""
    bcs, torch, orc = env
    A = MATS[name]()
    b = W.rhs_ones(A)
    res, x, h, sc = _gpu_solve(bcs, torch, A, b, kind, block_size=bs, rr_m=10, **cfg)
    ref = orc.solve_bjacobi(A, b, bs, kind=kind, tol=1e-10, maxit=5000, rr_m=10, max_restarts=29)
    assert res["status"] == 0 and ref["status"] == 0, (res, ref["status_name"])
    assert res["iterations"] == ref["iterations"]
    assert res["rr_steps"] == ref["rr_steps"]
    if kind == "p-BiCGSafe-rr":
        assert res["rr_steps"] >= 1
    assert res["outer_steps"] == ref["restarts"] + 1
    assert np.array_equal(h, ref["hist"])
    assert np.array_equal(sc[:len(ref["scalars"])], ref["scalars"][:len(sc)])
    assert np.array_equal(x, ref["x"])
    assert orc.true_residual(A, b, x) / np.linalg.norm(b) <= 1e-10


@pytest.mark.parametrize("n,bs", [(1, 8), (5, 8), (33, 4), (37, 32)])
def test_bjacobi_tiny_and_ragged(env, n, bs):
    """Systems smaller than one block or one tile, and a last block of one row: bit-identical to
    the oracle (a single ragged block is the whole matrix: its M^-1 is the inverse)."""
    bcs, torch, orc = env
    A = W.tiny_random(n, seed=n, density=0.5) if n > 1 else W.dense_to_csr(np.array([[3.0]]))
    b = W.rhs_ones(A)
    res, x, h, sc = _gpu_solve(bcs, torch, A, b, "p-BiCGSafe", block_size=bs, maxit=500)
    ref = orc.solve_bjacobi(A, b, bs, kind="p-BiCGSafe", tol=1e-10, maxit=500, max_restarts=29)
    assert res["status"] == ref["status"] == 0, (res, ref["status_name"])
    assert res["iterations"] == ref["iterations"]
    assert np.array_equal(h, ref["hist"]) and np.array_equal(x, ref["x"])


def test_bjacobi_start_vector(env):
    """A non-zero x_0 enters as y_0 = M x_0 on both sides: bit-identical runs."""
    bcs, torch, orc = env
    A = W.cd2d(48, 30.0)
    b = W.rhs_ones(A)
    x0 = np.random.default_rng(2).standard_normal(A.n)
    res, x, h, _ = _gpu_solve(bcs, torch, A, b, "p-BiCGSafe", x0=x0, block_size=4)
    ref = orc.solve_bjacobi(A, b, 4, x0=x0, kind="p-BiCGSafe", tol=1e-10, maxit=5000, max_restarts=29)
    assert res["iterations"] == ref["iterations"]
    assert np.array_equal(h, ref["hist"]) and np.array_equal(x, ref["x"])


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("kind", ["ssBiCGSafe2", "p-BiCGSafe"])
def test_bjacobi_refinement_modes(env, prec, kind):
    """FP32/BF16 inner solves on A M^-1 (M^-1 rounded to FP32) inside FP64 refinement: the FP64
    true residual of the original system reaches 1e-10 and x is within 1e-7 of the FP64
    oracle's."""
    bcs, torch, orc = env
    A = W.cd2d(64, 20.0)
    b = W.rhs_ones(A)
    res, x, _, _ = _gpu_solve(bcs, torch, A, b, kind, precision=prec, block_size=8)
    ref = orc.solve_bjacobi(A, b, 8, kind=kind, tol=1e-10, maxit=5000, max_restarts=29)
    assert res["status"] == 0, res
    assert orc.true_residual(A, b, x) / np.linalg.norm(b) <= 1e-10
    assert np.max(np.abs(x - ref["x"])) <= 1e-7
    assert res["outer_steps"] >= 2


def test_bjacobi_refusals(env):
    """Combinations the preconditioned kernel is not built for, block sizes that do not divide
    a tile and singular blocks are refused at bcs_solver_create; the library's defaults are
    adjusted instead of refused."""
    bcs, torch, orc = env
    A = W.cd2d(20, 20.0)
    M = bcs.csr_upload(A, layouts=bcs.LAYOUT_CSR | bcs.LAYOUT_SELL)
    bad = [dict(layout="sell"), dict(threads_per_row=8), dict(tile_order=2), dict(block_size=3), dict(block_size=64)]
    for kw in bad:
        kind = kw.pop("kind", "p-BiCGSafe")
        with pytest.raises(bcs.BcsError):
            bcs.solver_create(M, kind, precond="block-jacobi", **kw)
    S = bcs.solver_create(M, "p-BiCGSafe", precond="block-jacobi", threads_per_row=1, tile_order=1)
    assert bcs.precond_blocks(S)[0].shape == (A.n, 8)   # default block size 8
    # after autotuning (which may record SELL for the matrix) the default layout still gives a
    # block-Jacobi solver on CSR
    bcs.autotune(M, "p-BiCGSafe", precision="fp64", iters=5)
    S = bcs.solver_create(M, "p-BiCGSafe", precond="block-jacobi", layout="auto")
    assert bcs.precond_blocks(S)[0].shape == (A.n, 8)
    Ad = np.eye(16)
    Ad[2:4, 2:4] = [[1.0, 2.0], [2.0, 4.0]]
    Ad[3, 9] = 1.0
    with pytest.raises(bcs.BcsError):
        bcs.solver_create(bcs.csr_upload(W.dense_to_csr(Ad)), "p-BiCGSafe", precond="block-jacobi", block_size=2)
    S0 = bcs.solver_create(M, "p-BiCGSafe")
    with pytest.raises(bcs.BcsError):
        bcs.precond_blocks(S0)


def test_bjacobi_rr_reaches_tolerance_where_pipelined_stalls(env):
    """Blocks of 2 rows on the 128^3 system: p-BiCGSafe's recursive residual stalls above 1e-10
    (the residual gap of Section 4); with replacement steps every 100 iterations p-BiCGSafe-rr
    reaches the FP64 true residual of 1e-10."""
    bcs, torch, orc = env
    A = W.cd3d_upwind(128, 50.0)
    b = W.rhs_ones(A)
    M = bcs.csr_upload(A)
    S = bcs.solver_create(M, "p-BiCGSafe-rr", tol=1e-10, maxit=10000, precond="block-jacobi", block_size=2)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    res = bcs.solve(S, bd, x)
    assert res["status"] == 0 and res["rr_steps"] >= 1, res
    assert orc.true_residual(A, b, x.cpu().numpy()) / np.linalg.norm(b) <= 1e-10


@pytest.mark.parametrize("bs", [2, 8])
def test_bjacobi_cd3d_128_first_iterations(env, bs):
    """n = 2,097,152 in the default launch configuration: the first 30 preconditioned
    p-BiCGSafe iterations' histories and scalars bit-identical to the oracle's."""
    bcs, torch, orc = env
    A = W.cd3d_upwind(128, 50.0)
    b = W.rhs_ones(A)
    M = bcs.csr_upload(A)
    S = bcs.solver_create(M, "p-BiCGSafe", tol=0.0, maxit=30, max_outer=1, precond="block-jacobi", block_size=bs)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    res = bcs.solve(S, bd, x)
    h, sc = bcs.get_history(S), bcs.get_scalars(S)
    ref = orc.solve_bjacobi(A, b, bs, kind="p-BiCGSafe", tol=0.0, maxit=30, parallel=True)
    assert res["iterations"] == ref["iterations"] == 30
    assert len(h) == len(ref["hist"]) >= 30
    assert np.array_equal(h, ref["hist"])
    assert np.array_equal(sc[:30], ref["scalars"][:30])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_bjacobi_cd3d_128(env, prec):
    """The 128^3 upwind system (n = 2,097,152) with blocks of 8 rows along x: the FP64 true
    residual of the original system reaches 1e-10."""
    bcs, torch, orc = env
    A = W.cd3d_upwind(128, 50.0)
    b = W.rhs_ones(A)
    M = bcs.csr_upload(A, stores=bcs.STORE_F32)
    S = bcs.solver_create(M, "p-BiCGSafe", tol=1e-10, maxit=10000, precision=prec, precond="block-jacobi",
                          block_size=8)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    res = bcs.solve(S, bd, xd)
    x = xd.cpu().numpy()
    assert res["status"] == 0, res
    assert orc.true_residual(A, b, x) / np.linalg.norm(b) <= 1e-10


def _golden_bjacobi():
    import json
    import os
    p = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cd3d128_bjacobi_solves.json")
    with open(p) as fh:
        return json.load(fh)


@pytest.mark.parametrize("key", ["p-BiCGSafe/4", "p-BiCGSafe-rr/2", "ssBiCGSafe2/8"])
def test_bjacobi_cd3d_128_full_solve_matches_oracle(env, key):
    """The complete preconditioned FP64 solves of the 128^3 system in the default launch
    configuration against the oracle's (tests/golden/cd3d128_bjacobi_solves.json, written by
    make_cd3d128_bjacobi_solves.py from oracle/ alone): the same iterations, outer runs and
    replacement steps, the same true residual and the same x, bit for bit."""
    import hashlib
    bcs, torch, orc = env
    gold = _golden_bjacobi()
    g = gold["solves"][key]
    o = gold["options"]
    A = W.cd3d_upwind(128, 50.0)
    b = W.rhs_ones(A)
    assert hashlib.sha256(np.ascontiguousarray(b, dtype="<f8").tobytes()).hexdigest() == gold["b_sha256"]
    M = bcs.csr_upload(A)
    S = bcs.solver_create(M, g["kind"], tol=o["tol"], maxit=o["maxit"], max_outer=o["max_runs"], rr_m=o["rr_m"],
                          rr_M=o["rr_M"], precond="block-jacobi", block_size=g["block_size"])
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    res = bcs.solve(S, bd, x)
    assert g["status"] == "ok" and res["status"] == bcs.OK
    assert res["iterations"] == g["iterations"]
    assert res["outer_steps"] == g["outer_steps"] and res["rr_steps"] == g["rr_steps"]
    xh = x.cpu().numpy()
    rows = np.asarray(gold["sample_rows"])
    assert np.array_equal(xh[rows], np.array([float.fromhex(v) for v in g["x_sample"]]))
    assert hashlib.sha256(np.ascontiguousarray(xh, dtype="<f8").tobytes()).hexdigest() == g["x_sha256"]
    assert res["rel_res_true"] == float.fromhex(g["rel_res_true"])
