"""Parity at the full sizes of the synthetic configurations, in the launch
configuration bench.py times (default options: one 24-warp CTA per SM, CSR one
lane per row).  The oracle cannot finish these solves in seconds, so the checks
are (a) the first 20 iterations, which the oracle can run; (b) the complete
FP64 solves against golden files that scripts beside them wrote from oracle/
alone (tests/golden/make_*_full_solves.py): the same iterations, outer runs,
replacement steps, true residual and x, bit for bit; and (c) properties that
hold at any size, measured by the oracle on the GPU's output: the FP64 true
residual ||b - A x|| / ||b|| <= 1e-10 at exit.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cd3d128_full_solves.json")


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<f8").tobytes()).hexdigest()


# Any two solutions of one system to a 1e-10 relative residual differ by at most 2e-10 ||A^-1|| ||b||
# in the 2-norm; on these systems the refinement modes' x differ from the oracle's by at most 6e-8 over
# the sampled rows (bench.py error_vs_oracle), and the bound below leaves a wide margin.
X_VS_ORACLE = 1e-6


def _x_err_vs_golden(x, gold, kind):
    """max |x - x_oracle| over the golden file's sampled rows; x_oracle is the file's solve by the
    same method, else by p-BiCGSafe-rr or ssBiCGSafe2 (every one solved the system to 1e-10)."""
    solves = gold["solves"]
    ref = kind if kind in solves else ("p-BiCGSafe-rr" if "p-BiCGSafe-rr" in solves else "ssBiCGSafe2")
    rows = np.asarray(gold["sample_rows"])
    return float(np.max(np.abs(x[rows] - np.array([float.fromhex(v) for v in solves[ref]["x_sample"]]))))

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


@pytest.mark.parametrize("kind", ["ssBiCGSafe2", "p-BiCGSafe", "p-BiCGSafe-rr"])
def test_cd3d_128_full_solve_matches_oracle(env, cd3d, kind):
    """The complete FP64 solve of the benchmark system, in the benchmark's launch configuration
    and options, against the oracle's complete solve (tests/golden/cd3d128_full_solves.json,
    written by make_cd3d128_full_solves.py from oracle/ alone): the iteration count within 5 %
    of the oracle's -- and in fact the same iterations, outer runs and replacement steps, and
    the same x, bit for bit."""
    bcs, torch, orc = env
    A, b, M = cd3d
    with open(GOLDEN) as fh:
        gold = json.load(fh)
    assert _sha(b) == gold["b_sha256"], "the input generator gives a different b than the golden run"
    o = gold["options"]
    g = gold["solves"][kind]
    S = bcs.solver_create(M, kind, tol=o["tol"], maxit=o["maxit"], max_outer=o["max_runs"], rr_m=o["rr_m"],
                          rr_M=o["rr_M"])
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    res = bcs.solve(S, bd, x)
    assert g["status"] == "ok" and res["status"] == bcs.OK
    assert abs(res["iterations"] - g["iterations"]) <= 0.05 * g["iterations"]
    assert res["iterations"] == g["iterations"]
    assert res["outer_steps"] == g["outer_steps"]
    assert res["rr_steps"] == g["rr_steps"]
    xh = x.cpu().numpy()
    rows = np.asarray(gold["sample_rows"])
    assert np.array_equal(xh[rows], np.array([float.fromhex(v) for v in g["x_sample"]]))
    assert _sha(xh) == g["x_sha256"]
    assert res["rel_res_true"] == float.fromhex(g["rel_res_true"])


@pytest.mark.parametrize("kind,prec", [("ssBiCGSafe2", "fp64"), ("p-BiCGSafe", "fp64"), ("p-BiCGSafe", "fp32"),
                                       ("p-BiCGSafe-rr", "fp32"), ("p-BiCGSafe-rr", "bf16")])
def test_cd3d_128_full_solve_true_residual(env, cd3d, kind, prec):
    """Full solves of the benchmark system to 1e-10: the FP64 true residual of the
    returned x, recomputed by the oracle, meets the tolerance, and x agrees with the oracle's
    complete solve (tests/golden/cd3d128_full_solves.json) within X_VS_ORACLE at its sampled rows."""
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
    with open(GOLDEN) as fh:
        assert _x_err_vs_golden(xh, json.load(fh), kind) <= X_VS_ORACLE


@pytest.fixture(scope="module")
def powerlaw(env):
    bcs, torch, orc = env
    A = W.powerlaw()
    M = bcs.csr_upload(A, stores=bcs.STORE_F32)
    return A, M


GOLDENPL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "powerlaw_4m_full_solves.json")
PL_KINDS = ["ssBiCGSafe2", "p-BiCGSafe", "p-BiCGSafe-rr"]


@pytest.mark.parametrize("tile_order", ["library", "static"])
@pytest.mark.parametrize("kind", PL_KINDS)
def test_powerlaw_4m_full_solve_matches_oracle(env, powerlaw, kind, tile_order):
    """The complete FP64 solves of the irregular 4M-row system against the oracle's
    (tests/golden/powerlaw_4m_full_solves.json, written by make_powerlaw_4m_full_solves.py
    from oracle/ alone), CSR with one lane per row: in the library's tile order for this
    matrix (warps claim tiles, as bench.py runs it) and in the static order, the same
    iterations, outer runs and replacement steps, the same true residual and x, bit for bit."""
    bcs, torch, orc = env
    A, M = powerlaw
    b = W.rhs_ones(A)
    with open(GOLDENPL) as fh:
        gold = json.load(fh)
    assert _sha(b) == gold["b_sha256"]
    o = gold["options"]
    g = gold["solves"][kind]
    S = bcs.solver_create(M, kind, tol=o["tol"], maxit=o["maxit"], max_outer=o["max_runs"], rr_m=o["rr_m"],
                          rr_M=o["rr_M"], layout="csr", threads_per_row=1,
                          tile_order=0 if tile_order == "library" else 1)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    res = bcs.solve(S, bd, x)
    assert g["status"] == "ok" and res["status"] == bcs.OK
    assert res["iterations"] == g["iterations"]
    assert res["outer_steps"] == g["outer_steps"] and res["rr_steps"] == g["rr_steps"]
    xh = x.cpu().numpy()
    rows = np.asarray(gold["sample_rows"])
    assert np.array_equal(xh[rows], np.array([float.fromhex(v) for v in g["x_sample"]]))
    assert _sha(xh) == g["x_sha256"]
    assert res["rel_res_true"] == float.fromhex(g["rel_res_true"])


def test_powerlaw_4m_fp32_refinement(env, powerlaw):
    """The irregular 4M-row configuration (power-law rows up to 512): FP32 values and vectors
    with FP64 refinement reach the FP64 tolerance, checked by the oracle's true residual, and x
    agrees with the oracle's complete solve within X_VS_ORACLE at its sampled rows."""
    bcs, torch, orc = env
    A, M = powerlaw
    b = W.rhs_ones(A)
    for prec in ["fp32", "fp64"]:
        S = bcs.solver_create(M, "p-BiCGSafe-rr", tol=1e-10, maxit=20000, precision=prec, max_outer=30)
        bd = torch.from_numpy(b).cuda()
        x = torch.zeros_like(bd)
        res = bcs.solve(S, bd, x)
        assert res["status"] == 0
        xh = x.cpu().numpy()
        assert orc.true_residual(A, b, xh) / np.linalg.norm(b) <= 1e-10
        with open(GOLDENPL) as fh:
            assert _x_err_vs_golden(xh, json.load(fh), "p-BiCGSafe-rr") <= X_VS_ORACLE


# ---- 27-point 192^3 stencil (n = 7,077,888, nnz = 189,119,224): CSR and SELL-C-sigma ----------

@pytest.fixture(scope="module")
def cd3d27(env):
    bcs, torch, orc = env
    A = W.cd3d27(192, 100.0)
    M = bcs.csr_upload(A, layouts=bcs.LAYOUT_CSR | bcs.LAYOUT_SELL, sell_sigma=256,
                       stores=bcs.STORE_F32 | bcs.STORE_BF16)
    return A, M


def _row_abs_sums(orc, A, x):
    """sum_j |a_ij x_j| per row, by the oracle's SpMV on |A| and |x|."""
    return orc.spmv(W.CSR(A.n, A.rowptr, A.col, np.abs(A.val)), np.abs(x))


def test_cd3d27_192_format_build_bit_exact(env, cd3d27):
    """The full-size CSR copy, its FP32 / BF16 roundings and the SELL-32-256 arrays equal
    the oracle's, bit for bit."""
    bcs, torch, orc = env
    A, M = cd3d27
    E = bcs.matrix_export(M, csr=True, f32=True, bf16=True, sell=True)
    assert np.array_equal(E["rowptr"], A.rowptr.astype(np.int32))
    assert np.array_equal(E["col"], A.col)
    assert np.array_equal(E["val64"].view(np.uint64), A.val.view(np.uint64))
    assert np.array_equal(E["val32"].view(np.uint32), A.val.astype(np.float32).view(np.uint32))
    assert np.array_equal(E["valbf16"], orc.to_bf16_bits(A.val))
    del E["val32"], E["valbf16"], E["val64"], E["col"]
    S = orc.sell_build(A, 32, 256)
    assert np.array_equal(E["perm"], S["perm"])
    assert np.array_equal(E["slice_ptr"], S["slice_ptr"])
    assert np.array_equal(E["scol"], S["col"])
    assert np.array_equal(E["sval64"].view(np.uint64), S["val"].view(np.uint64))


def test_cd3d27_192_spmv_all_stores(env, cd3d27):
    """y = A x at full size: FP64 with one lane per row and SELL bit-identical to the oracle's
    sequential row sums; FP32 and BF16 value copies within the FP32 accumulation bound of the
    exact product of the stored values."""
    bcs, torch, orc = env
    A, M = cd3d27
    x = np.random.default_rng(5).standard_normal(A.n)
    want = orc.spmv(A, x)
    xd = torch.from_numpy(x).cuda()
    for lay, tpr in [(bcs.LAYOUT_CSR, 1), (bcs.LAYOUT_SELL, 0)]:
        yd = torch.full_like(xd, np.nan)
        bcs.spmv(M, xd, yd, layout=lay, threads_per_row=tpr)
        assert np.array_equal(yd.cpu().numpy(), want), (lay, tpr)
    del xd, yd
    x32 = x.astype(np.float32)
    xd = torch.from_numpy(x32).cuda()
    lens = np.diff(A.rowptr)
    for store in [bcs.STORE_F32, bcs.STORE_BF16]:
        if store == bcs.STORE_F32:
            vals = A.val.astype(np.float32).astype(np.float64)
        else:
            vals = (orc.to_bf16_bits(A.val).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        Ar = W.CSR(A.n, A.rowptr, A.col, vals)
        exact = orc.spmv(Ar, x32.astype(np.float64))
        bound = _row_abs_sums(orc, Ar, x32.astype(np.float64)) * (lens + 1) * 2.0 ** -24
        for lay, tpr in [(bcs.LAYOUT_CSR, 1), (bcs.LAYOUT_SELL, 0)]:
            yd = torch.zeros_like(xd)
            bcs.spmv(M, xd, yd, layout=lay, store=store, threads_per_row=tpr)
            y = yd.cpu().numpy().astype(np.float64)
            assert np.all(np.abs(y - exact) <= bound + 1e-30), (store, lay, tpr)


GOLDEN27 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cd3d27_192_full_solves.json")


@pytest.mark.parametrize("kind,layout", [("ssBiCGSafe2", "csr"), ("p-BiCGSafe-rr", "csr"), ("ssBiCGSafe2", "sell")])
def test_cd3d27_192_full_solve_matches_oracle(env, cd3d27, kind, layout):
    """The complete FP64 solves of the 27-point system (n = 7,077,888) against the oracle's
    (tests/golden/cd3d27_192_full_solves.json, written by make_cd3d27_192_full_solves.py from
    oracle/ alone), CSR with one lane per row and SELL-32-256: the same iterations, outer runs
    and replacement steps, the same true residual and x, bit for bit."""
    bcs, torch, orc = env
    A, M = cd3d27
    b = W.rhs_ones(A)
    with open(GOLDEN27) as fh:
        gold = json.load(fh)
    assert _sha(b) == gold["b_sha256"]
    o = gold["options"]
    g = gold["solves"][kind]
    S = bcs.solver_create(M, kind, tol=o["tol"], maxit=o["maxit"], max_outer=o["max_runs"], rr_m=o["rr_m"],
                          rr_M=o["rr_M"], layout=layout, threads_per_row=1 if layout == "csr" else 0)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    res = bcs.solve(S, bd, x)
    assert g["status"] == "ok" and res["status"] == bcs.OK
    assert res["iterations"] == g["iterations"]
    assert res["outer_steps"] == g["outer_steps"] and res["rr_steps"] == g["rr_steps"]
    xh = x.cpu().numpy()
    rows = np.asarray(gold["sample_rows"])
    assert np.array_equal(xh[rows], np.array([float.fromhex(v) for v in g["x_sample"]]))
    assert _sha(xh) == g["x_sha256"]
    assert res["rel_res_true"] == float.fromhex(g["rel_res_true"])


@pytest.mark.parametrize("kind,prec,layout", [("p-BiCGSafe", "fp32", "csr"), ("p-BiCGSafe", "fp32", "sell"),
                                              ("p-BiCGSafe-rr", "fp64", "csr"), ("ssBiCGSafe2", "fp64", "sell")])
def test_cd3d27_192_full_solve_true_residual(env, cd3d27, kind, prec, layout):
    """Full solves of the 27-point system to 1e-10, the true residual of the returned x
    recomputed by the oracle, and x against the oracle's complete solve
    (tests/golden/cd3d27_192_full_solves.json) within X_VS_ORACLE at its sampled rows."""
    bcs, torch, orc = env
    A, M = cd3d27
    b = W.rhs_ones(A)
    S = bcs.solver_create(M, kind, tol=1e-10, maxit=20000, precision=prec, layout=layout, max_outer=60)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    res = bcs.solve(S, bd, x)
    assert res["status"] == 0
    xh = x.cpu().numpy()
    rel = orc.true_residual(A, b, xh) / np.linalg.norm(b)
    assert rel <= 1e-10
    assert abs(rel - res["rel_res_true"]) <= 1e-3 * rel + 1e-16
    with open(GOLDEN27) as fh:
        assert _x_err_vs_golden(xh, json.load(fh), kind) <= X_VS_ORACLE


# ---- 512 independent 2D systems, sides 32..256, in one persistent launch -------------------------

GOLDENB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch_cd2d_512_solves.json")


def test_batch_cd2d_512_fp64_matches_oracle(env):
    """The full 512-system FP64 batch in the configuration bench.py times (one launch, one lane
    per row, clusters of two CTAs, replacement every 20 iterations) against the oracle's solve of
    every system (tests/golden/batch_cd2d_512_solves.json, written by
    make_batch_cd2d_512_solves.py from oracle/ alone): for each system the same iterations,
    outer runs and replacement steps, the same true residual and x, bit for bit."""
    bcs, torch, orc = env
    with open(GOLDENB) as fh:
        gold = json.load(fh)
    o = gold["options"]
    mats, sides, betas = W.batch_cd2d()
    Ms = [bcs.csr_upload(A) for A in mats]
    bs = [W.rhs_ones(A) for A in mats]
    assert [_sha(b) for b in bs] == [g["b_sha256"] for g in gold["systems"]]
    bd = [torch.from_numpy(b).cuda() for b in bs]
    xd = [torch.zeros_like(b) for b in bd]
    worst, res = bcs.solve_batched(Ms, bd, xd, kind=gold["kind"], tol=o["tol"], maxit=o["maxit"], precision="fp64",
                                   max_outer=o["max_runs"], rr_m=o["rr_m"], rr_M=o["rr_M"])
    assert worst == 0
    bad = []
    for k, (g, r, x) in enumerate(zip(gold["systems"], res, xd)):
        same = (g["status"] == "ok" and r["status"] == bcs.OK and r["iterations"] == g["iterations"] and
                r["outer_steps"] == g["outer_steps"] and r["rr_steps"] == g["rr_steps"] and
                r["rel_res_true"] == float.fromhex(g["rel_res_true"]) and _sha(x.cpu().numpy()) == g["x_sha256"])
        if not same:
            bad.append((k, g["n"], g["iterations"], r["iterations"]))
    assert not bad, bad


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_cd2d_512_true_residuals(env, prec):
    """The full 512-system batch in the configuration bench.py times (default batched options,
    replacement every 20 iterations): every system converges, its true residual, recomputed by
    the oracle, meets 1e-10, and its x agrees with the oracle's solve of the same system
    (tests/golden/batch_cd2d_512_solves.json) within X_VS_ORACLE at the file's sampled rows."""
    bcs, torch, orc = env
    mats, sides, betas = W.batch_cd2d()
    Ms = [bcs.csr_upload(A, stores=bcs.STORE_F32) for A in mats]
    bs = [W.rhs_ones(A) for A in mats]
    bd = [torch.from_numpy(b).cuda() for b in bs]
    xd = [torch.zeros_like(b) for b in bd]
    worst, res = bcs.solve_batched(Ms, bd, xd, kind="p-BiCGSafe-rr", tol=1e-10, maxit=10000, precision=prec,
                                   max_outer=30, rr_m=20)
    assert worst == 0
    assert all(r["status"] == 0 for r in res)
    with open(GOLDENB) as fh:
        gold = json.load(fh)
    k = gold["samples_per_system"]
    for A, b, x, g in zip(mats, bs, xd, gold["systems"]):
        xh = x.cpu().numpy()
        assert orc.true_residual(A, b, xh) / np.linalg.norm(b) <= 1e-10
        rows = np.unique(np.linspace(0, A.n - 1, k).round().astype(np.int64))
        assert np.max(np.abs(xh[rows] - np.array([float.fromhex(v) for v in g["x_sample"]]))) <= X_VS_ORACLE
