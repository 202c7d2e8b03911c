"""The row-partitioned solve (bcs_dist: Section 3's setting, every rank a block of
rows with its own Krylov vectors and halo, the nine inner products reduced over
all ranks) against the single-process oracle.  In FP64 the inner products are
exact and every row is summed in CSR order, so the partitioned histories,
scalars, iteration counts and x are bit-identical to the oracle's for any
number of ranks; this is checked on a small stencil, a ragged power-law matrix
whose columns reach every rank, and the 128^3 benchmark system."""
import hashlib
import json
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cd3d128_full_solves.json")


@pytest.fixture(scope="module")
def env(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_10591_gb300 as bcs
    return bcs, torch, orc


def _solve(bcs, torch, A, b, nparts, kind, **kw):
    D = bcs.Dist(A, nparts, kind=kind, **kw)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    res = D.solve(bd, x)
    return D, res, x.cpu().numpy()


@pytest.mark.parametrize("nparts", [1, 2, 3, 5])
@pytest.mark.parametrize("kind", ["ssBiCGSafe2", "p-BiCGSafe", "p-BiCGSafe-rr"])
def test_dist_bit_identical_cd2d_64(env, nparts, kind):
    bcs, torch, orc = env
    A = W.cd2d(64, 20.0)
    b = W.rhs_ones(A)
    D, res, x = _solve(bcs, torch, A, b, nparts, kind, tol=1e-10, maxit=2000, rr_m=25, max_outer=30)
    ref = orc.solve(A, b, kind=kind, tol=1e-10, maxit=2000, rr_m=25, max_restarts=29)
    assert res["status"] == 0 and ref["status"] == 0
    assert res["iterations"] == ref["iterations"]
    assert res["outer_steps"] == ref["restarts"] + 1
    assert res["rr_steps"] == ref["rr_steps"]
    h = D.history()
    assert np.array_equal(h, ref["hist"][:len(h)]) and len(h) == len(ref["hist"])
    sc = D.scalars()
    k = min(len(sc), len(ref["scalars"]))
    assert np.array_equal(sc[:k], ref["scalars"][:k])
    assert np.array_equal(x, ref["x"])
    # every rank got a block and CTAs; the middle ranks exchange with both neighbours
    infos = [D.info(r) for r in range(nparts)]
    assert sum(i["nloc"] for i in infos) == A.n and all(i["ctas"] >= 1 for i in infos)
    if nparts > 2:
        assert infos[1]["nleft"] > 0 and infos[1]["nright"] > 0


def test_dist_ragged_powerlaw_many_ranks(env):
    """Power-law rows (n mod 32 != 0) with 10 % of the columns anywhere: every rank's halo draws
    from every other rank."""
    bcs, torch, orc = env
    A = W.powerlaw(n=20011, seed=7)
    b = W.rhs_ones(A)
    for nparts in [4, 7]:
        D, res, x = _solve(bcs, torch, A, b, nparts, "p-BiCGSafe-rr", tol=1e-10, maxit=3000, rr_m=50)
        ref = orc.solve(A, b, kind="p-BiCGSafe-rr", tol=1e-10, maxit=3000, rr_m=50, max_restarts=29)
        assert res["iterations"] == ref["iterations"]
        assert np.array_equal(D.history(), ref["hist"][:len(D.history())])
        assert np.array_equal(x, ref["x"])
        assert all(D.info(r)["nleft"] + D.info(r)["nright"] > 0 for r in range(nparts))


def test_dist_given_bounds_and_uneven_blocks(env):
    """Caller-given blocks, one of them a single row and one not a multiple of 32."""
    bcs, torch, orc = env
    A = W.cd2d(40, 5.0)
    b = W.rhs_ones(A)
    bounds = np.array([0, 1, 700, 1337, A.n], dtype=np.int64)
    D, res, x = _solve(bcs, torch, A, b, 4, "p-BiCGSafe", tol=1e-10, maxit=2000, bounds=bounds)
    ref = orc.solve(A, b, kind="p-BiCGSafe", tol=1e-10, maxit=2000, max_restarts=29)
    assert res["iterations"] == ref["iterations"]
    assert np.array_equal(x, ref["x"])
    assert D.info(0)["nloc"] == 1


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_dist_refinement_modes(env, prec):
    """FP32 / BF16 inner solves with FP64 refinement across ranks reach the FP64 tolerance (the
    per-lane FP64 sums depend on which rows a lane visits, so only the tolerance is shared)."""
    bcs, torch, orc = env
    A = W.cd2d(64, 20.0)
    b = W.rhs_ones(A)
    D, res, x = _solve(bcs, torch, A, b, 3, "p-BiCGSafe", tol=1e-10, maxit=5000, precision=prec, max_outer=40)
    assert res["status"] == 0
    assert orc.true_residual(A, b, x) / np.linalg.norm(b) <= 1e-10


def test_dist_rejects_unsupported_options(env):
    bcs, torch, orc = env
    A = W.cd2d(16, 1.0)
    with pytest.raises(bcs.BcsError):
        bcs.Dist(A, 2, layout="sell")
    with pytest.raises(bcs.BcsError):
        bcs.Dist(A, 2, threads_per_row=8)
    with pytest.raises(bcs.BcsError):
        bcs.Dist(A, 17)


@pytest.mark.parametrize("nparts", [2, 4])
def test_dist_cd3d_128_matches_oracle_full_solve(env, nparts):
    """The 128^3 benchmark system split over 2 and 4 ranks: the complete p-BiCGSafe FP64 solve
    has the oracle's iteration count and outer runs and its x, bit for bit."""
    bcs, torch, orc = env
    with open(GOLDEN) as fh:
        gold = json.load(fh)
    A = W.cd3d_upwind(128, 50.0)
    b = W.rhs_ones(A)
    o = gold["options"]
    g = gold["solves"]["p-BiCGSafe"]
    D, res, x = _solve(bcs, torch, A, b, nparts, "p-BiCGSafe", tol=o["tol"], maxit=o["maxit"],
                       max_outer=o["max_runs"])
    assert res["status"] == 0
    assert res["iterations"] == g["iterations"] and res["outer_steps"] == g["outer_steps"]
    assert hashlib.sha256(np.ascontiguousarray(x, dtype="<f8").tobytes()).hexdigest() == g["x_sha256"]


def test_one_process_per_gpu_form_with_one_rank(env):
    """The multi-GPU form (bcs_dist_rank_*: one process per GPU, peers' arenas opened by CUDA IPC,
    a system-scope barrier on rank 0's counter that is not reset between solves) with the one
    rank this machine allows: export, connect, two solves in a row, each bit-identical to the
    oracle; a solve before connect and a rank outside the partition are refused."""
    bcs, torch, orc = env
    A = W.cd2d(48, 10.0)
    b = W.rhs_ones(A)
    ref = orc.solve(A, b, kind="p-BiCGSafe", tol=1e-10, maxit=2000, max_restarts=29)
    D = bcs.DistRank(A, 1, 0, kind="p-BiCGSafe", tol=1e-10, maxit=2000)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    with pytest.raises(bcs.BcsError):
        D.solve(bd, x)
    h = D.export_handle()
    assert len(h) == bcs.DIST_HANDLE_BYTES
    D.connect([h])
    for _ in range(2):
        x.zero_()
        res = D.solve(bd, x)
        assert res["status"] == 0 and res["iterations"] == ref["iterations"]
        assert np.array_equal(x.cpu().numpy(), ref["x"])
        assert np.array_equal(D.history(), ref["hist"])
    assert D.info(0)["nloc"] == A.n
    with pytest.raises(bcs.BcsError):
        bcs.DistRank(A, 2, 2)
