"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(no GPU).  Each test names what it pins; together they are chosen so that a
dropped term, a wrong sign, a wrong index or a swapped operand in any
statement of Algorithms 3-5 fails at least one of them."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import workloads as W
from oracle import exact

KINDS = ["ssBiCGSafe2", "p-BiCGSafe", "p-BiCGSafe-rr"]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def fma(a, b, c):
    """Correctly rounded a*b + c (CPython's int/int true division rounds correctly)."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _exact_dot(x, y):
    return sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, y)), Fraction(0))


# ---------------------------------------------------------------- primitives

def test_dot_correctly_rounded(orc):
    """(x, y) is the exact sum of exact products rounded once to nearest even: equal, bit
    for bit, to the exact rational sum converted to float (CPython rounds int/int
    correctly), over wide exponent ranges, cancellation, subnormal results and ties."""
    rng = np.random.default_rng(1)
    for n in [0, 1, 2, 7, 100, 3000]:
        for scale in [1e-300, 1e-160, 1.0, 1e150]:
            x = rng.standard_normal(n) * scale * 10.0 ** rng.integers(-20, 20, n)
            y = rng.standard_normal(n) * 10.0 ** rng.integers(-20, 20, n)
            assert orc.dot(x, y) == float(_exact_dot(x, y))
    # heavy cancellation: x.y = tiny while the terms are huge
    x = np.array([1e300, 1.0, -1e300, 3e-300])
    y = np.array([1.0, 1e-300, 1.0, 1.0])
    assert orc.dot(x, y) == float(_exact_dot(x, y)) == 4e-300
    # an exact tie between two doubles rounds to even
    x = np.array([1.0, 2.0 ** -53])
    y = np.array([1.0, 1.0])
    assert orc.dot(x, y) == 1.0
    x = np.array([1.0 + 2.0 ** -52, 2.0 ** -53])
    assert orc.dot(x, y) == 1.0 + 2.0 ** -51
    # order independence
    x, y = rng.standard_normal(1001), rng.standard_normal(1001)
    p = rng.permutation(1001)
    assert orc.dot(x, y) == orc.dot(x[p], y[p])
    assert np.isnan(orc.dot(np.array([1.0, np.nan]), np.array([1.0, 1.0])))


def test_spmv_exact_on_integers(orc):
    """With small-integer values every product and sum is exact: y must equal A x exactly."""
    M = W.tiny_integer(30, seed=3)
    A = W.dense_to_csr(M.astype(float))
    x = np.arange(30, dtype=float) - 7.0
    assert np.array_equal(orc.spmv(A, x), M @ x)


def test_spmv_row_order_and_empty_rows(orc):
    """Rows with no entries give 0; a row is summed in storage order with fma."""
    D = np.zeros((5, 5))
    D[1, 0], D[1, 3], D[3, 4] = 0.1, 0.2, 0.3
    A = W.dense_to_csr(D)
    x = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    y = orc.spmv(A, x)
    assert y[0] == 0.0 and y[2] == 0.0 and y[4] == 0.0
    assert y[1] == fma(0.2, 4.0, fma(0.1, 1.0, 0.0))
    assert y[3] == fma(0.3, 5.0, 0.0)


def test_stencil_shapes():
    """Closed-form nonzero counts of the synthetic workloads: 5n-4k (2D), 7n-6k^2 (3D), (3k-2)^3 (27-point)."""
    A = W.cd2d(64, 20.0)
    assert A.n == 4096 and A.nnz == 5 * 4096 - 4 * 64 == 20224
    A3 = W.cd3d_upwind(12, 50.0)
    assert A3.nnz == 7 * 12 ** 3 - 6 * 12 ** 2
    A27 = W.cd3d27(10, 100.0)
    assert A27.nnz == (3 * 10 - 2) ** 3
    # b = A*1 is the row sum; consistency of -Lap: the 27-point stencil annihilates constants
    # in the interior (row sum = 3*beta/h - 3*beta/h = 0 for beta-upwind too)
    b = W.rhs_ones(A27)
    k = 10
    interior = (k // 2) + k * (k // 2) + k * k * (k // 2)
    assert abs(b[interior]) < 1e-9 * abs(A27.val).max()
    # the 27-point Laplacian is second-order consistent: applied to x^2 it gives -2
    Ap = W.cd3d27(10, 0.0)
    h = 1.0 / 11
    g = np.arange(1, 11) * h
    X = np.tile(g, 100)
    D = Ap.to_dense()
    assert abs((D @ X ** 2)[interior] + 2.0) < 1e-8


# ---------------------------------------------------------------- whole solve

@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("seed", [11, 12, 13])
def test_lu_tiny(orc, kind, seed):
    """Dense LU (LAPACK) solution of tiny well-conditioned nonsymmetric systems."""
    A = W.tiny_random(24, seed)
    D = A.to_dense()
    b = np.random.default_rng(seed).standard_normal(24)
    o = orc.solve(A, b, kind=kind, tol=1e-13, maxit=200, rr_m=5, max_restarts=3)
    x_lu = np.linalg.solve(D, b)
    assert o["status_name"] == "ok"
    assert np.max(np.abs(o["x"] - x_lu)) <= 1e-10 * np.max(np.abs(x_lu))
    assert o["rel_res_true"] <= 1e-12


@pytest.mark.parametrize("kind", KINDS)
def test_cd2d_64_reaches_tolerance(orc, kind):
    """The paper's setting (Section 5): b = A*1, x_0 = 0; the FP64 true residual at exit is <= tol."""
    A = W.cd2d(64, 20.0)
    b = W.rhs_ones(A)
    o = orc.solve(A, b, kind=kind, tol=1e-10, maxit=2000, rr_m=100, max_restarts=5)
    assert o["status_name"] == "ok"
    assert o["rel_res_true"] <= 1e-10
    assert np.max(np.abs(o["x"] - 1.0)) < 1e-7
    assert 100 <= o["iterations"] <= 160


# ---------------------------------------------------------------- exact arithmetic

def _frac_system(n, seed):
    M = W.tiny_integer(n, seed)
    A = [[Fraction(int(v)) for v in row] for row in M]
    b = [sum(row, Fraction(0)) for row in A]
    return M, A, b


@pytest.mark.parametrize("n,seed", [(4, 1), (5, 2), (6, 3)])
@pytest.mark.parametrize("kind", KINDS)
def test_exact_finite_termination(n, seed, kind):
    """BiCG-type finite termination: in exact arithmetic r_i = 0 at some i <= n and x = A^-1 b = ones."""
    _, A, b = _frac_system(n, seed)
    res = exact.solve(A, b, kind=kind, maxit=3 * n, rr_m=2)
    assert res["terminated"] and res["iterations"] <= n
    assert all(v == 1 for v in res["x"])


@pytest.mark.parametrize("n,seed", [(5, 2), (6, 3), (6, 5)])
def test_exact_plain_equals_pipelined(n, seed):
    """Section 3: Alg. 4 (and Alg. 5) are equivalent rewrites of Alg. 3 -- identical
    (r_i, r_i) and scalars in exact arithmetic."""
    _, A, b = _frac_system(n, seed)
    ref = exact.solve(A, b, kind="ssBiCGSafe2", maxit=3 * n)
    for kind in ["p-BiCGSafe", "p-BiCGSafe-rr"]:
        got = exact.solve(A, b, kind=kind, maxit=3 * n, rr_m=2)
        assert got["rr"] == ref["rr"]
        assert got["scalars"] == ref["scalars"]


@pytest.mark.parametrize("kind", KINDS)
def test_fp64_oracle_tracks_exact(orc, kind):
    """The FP64 oracle's first iterations agree with the exact-arithmetic run."""
    n, seed = 6, 5
    M, A, b = _frac_system(n, seed)
    ref = exact.solve(A, b, kind=kind, maxit=3 * n, rr_m=2)
    Acsr = W.dense_to_csr(M.astype(float))
    bf = np.array([float(v) for v in b])
    o = orc.solve(Acsr, bf, kind=kind, tol=0.0, maxit=ref["iterations"] - 1, rr_m=2)
    r0 = math.sqrt(float(ref["rr"][0]))
    for i in range(ref["iterations"] - 1):
        want = math.sqrt(float(ref["rr"][i])) / r0
        assert abs(o["hist"][i] - want) <= 1e-9 * max(want, 1e-3)
        for k in range(4):
            assert abs(o["scalars"][i][k] - float(ref["scalars"][i][k])) <= 1e-9 * max(1.0, abs(float(ref["scalars"][i][k])))


def test_golden_i0_branch(orc):
    """Hand-derived i = 0 values (tests/golden/i0_branch_2x2.txt, Alg. 3/4 i = 0 branch)."""
    vals = {}
    with open(os.path.join(GOLDEN, "i0_branch_2x2.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            vals[k] = [Fraction(t) for t in v]
    D = np.array([float(v) for v in vals["matrix"]]).reshape(2, 2)
    A = W.dense_to_csr(D)
    b = np.array([float(v) for v in vals["b"]])
    for kind in ["ssBiCGSafe2", "p-BiCGSafe"]:
        o = orc.solve(A, b, kind=kind, tol=0.0, maxit=5, dump_iter=0, dump_phase=0)
        S = o["dump_scalars"]
        for key in ["a", "d", "f", "g"]:
            assert S[key] == float(vals[key][0])
        assert S["r"] == float(vals["rr"][0])
        assert abs(S["alpha"] - float(vals["alpha0"][0])) <= 1e-16
        assert abs(S["zeta"] - float(vals["zeta0"][0])) <= 1e-16
        assert S["beta"] == 0.0 and S["eta"] == 0.0
        o1 = orc.solve(A, b, kind=kind, tol=0.0, maxit=5, dump_iter=0, dump_phase=1)
        x1 = [float(v) for v in vals["x1"]]
        assert np.max(np.abs(o1["state"]["x"] - x1)) <= 4e-16
    # the exact mini-oracle agrees exactly
    Af = [[Fraction(3), Fraction(1)], [Fraction(1), Fraction(2)]]
    res = exact.solve(Af, [Fraction(4), Fraction(3)], kind="ssBiCGSafe2", maxit=0)
    assert res["scalars"][0] == (vals["alpha0"][0], 0, vals["zeta0"][0], 0)


# ---------------------------------------------------------------- definitions the recurrences maintain

def _dump(orc, A, b, kind, it, phase):
    return orc.solve(A, b, kind=kind, tol=0.0, maxit=it + 5, rr_m=3, dump_iter=it, dump_phase=phase)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("it", [1, 3, 4, 6])
def test_recurrence_definitions(orc, kind, it):
    """After the scalars of iteration i (dump phase 0):
    r_i = b - A x_i; y_i = A z_{i-1}; t_{i-1} = A (p_{i-1} - u_{i-1});
    plain: s_i = A r_i and w_{i-1} = A u_{i-1}; pipelined (Eqs. (s),(w),(l),(g)):
    s_i = A r_i, g_i = A y_i, l_{i-1} = A t_{i-1}, w_{i-1} = A u_{i-1}, As_i = A s_i."""
    A = W.tiny_random(40, 21, density=0.2)
    D = A.to_dense()
    b = np.random.default_rng(5).standard_normal(40)
    st = _dump(orc, A, b, kind, it, 0)["state"]
    nrm = lambda v: np.linalg.norm(v)
    scale = np.linalg.norm(D, 2)

    def close(lhs, rhs, ref):
        # rounding in the recurrences accumulates relative to the earlier, larger
        # iterates (~u*||b||); a wrong term would be of the size of the vector itself
        tol = 1e-11 * scale * ref + 1e-13 * scale * nrm(b)
        assert nrm(lhs - rhs) <= tol, (nrm(lhs - rhs), ref)

    close(st["r"], b - D @ st["x"], nrm(b))
    close(st["y"], D @ st["z"], nrm(st["z"]))
    close(st["t"], D @ (st["p"] - st["u"]), nrm(st["p"]) + nrm(st["u"]))
    close(st["s"], D @ st["r"], nrm(st["r"]))
    close(st["w"], D @ st["u"], nrm(st["u"]))
    if kind != "ssBiCGSafe2":
        close(st["g"], D @ st["y"], nrm(st["y"]))
        close(st["l"], D @ st["t"], nrm(st["t"]))
        close(st["As"], D @ st["s"], nrm(st["s"]))


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("it", [1, 2, 5])
def test_zeta_eta_minimise_associate_residual(orc, kind, it):
    """Eq. (eta&zeta_ssBiCGSafe2): zeta_i, eta_i minimise ||r_i - zeta A r_i - eta y_i||_2."""
    A = W.tiny_random(40, 22, density=0.2)
    b = np.random.default_rng(6).standard_normal(40)
    o = _dump(orc, A, b, kind, it, 0)
    st, S = o["state"], o["dump_scalars"]
    M = np.stack([st["s"], st["y"]], axis=1)
    (zeta, eta), *_ = np.linalg.lstsq(M, st["r"], rcond=None)
    assert abs(S["zeta"] - zeta) <= 1e-9 * abs(zeta)
    assert abs(S["eta"] - eta) <= 1e-9 * max(abs(eta), 1e-3 * abs(zeta))


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("it", [0, 1, 4])
def test_alpha_is_bicg_alpha(orc, kind, it):
    """alpha_i = (r0*, r_i) / (r0*, A p_i) (BiCG's alpha; g_i + beta_i h_i = (r0*, A p_i))."""
    A = W.tiny_random(40, 23, density=0.2)
    D = A.to_dense()
    b = np.random.default_rng(7).standard_normal(40)
    o0 = _dump(orc, A, b, kind, it, 0)
    o1 = _dump(orc, A, b, kind, it, 1)
    S = o0["dump_scalars"]
    p = o1["state"]["p"]
    rs = o0["state"]["rs"]
    want = S["f"] / float(rs @ (D @ p))
    assert abs(S["alpha"] - want) <= 1e-10 * abs(want)
    # o_i = A p_i (the vector the alpha denominator uses)
    assert np.linalg.norm(o1["state"]["o"] - D @ p) <= 1e-11 * np.linalg.norm(D, 2) * np.linalg.norm(p)


def test_beta_definition(orc):
    """beta_i = (alpha_{i-1} / zeta_{i-1}) (f_i / f_{i-1}) (Alg. 3/4)."""
    A = W.tiny_random(40, 24, density=0.2)
    b = np.random.default_rng(8).standard_normal(40)
    o = orc.solve(A, b, kind="p-BiCGSafe", tol=0.0, maxit=8)
    f = [_dump(orc, A, b, "p-BiCGSafe", i, 0)["dump_scalars"]["f"] for i in range(6)]
    sc = o["scalars"]
    for i in range(1, 6):
        want = (sc[i - 1][0] / sc[i - 1][2]) * (f[i] / f[i - 1])
        assert abs(sc[i][1] - want) <= 1e-12 * abs(want)


def test_residual_replacement_step(orc):
    """Alg. 5: at i mod m = 0, 0 < i < M the vectors are replaced by their definitions:
    after the step r = b - A x exactly as computed, s = A r, g = A y, l = A t, w = A u."""
    A = W.tiny_random(40, 25, density=0.2)
    b = np.random.default_rng(9).standard_normal(40)
    o = orc.solve(A, b, kind="p-BiCGSafe-rr", tol=0.0, maxit=12, rr_m=3, dump_iter=3, dump_phase=1)
    st = o["state"]
    assert o["dump_scalars"]["rr"] == 1.0
    assert np.array_equal(st["r"], b - orc.spmv(A, st["x"]))
    assert np.array_equal(st["s"], orc.spmv(A, st["r"]))
    assert np.array_equal(st["g"], orc.spmv(A, st["y"]))
    assert np.array_equal(st["l"], orc.spmv(A, st["t"]))
    assert np.array_equal(st["w"], orc.spmv(A, st["u"]))
    # rr count: replacements at i = 3, 6, 9 only (m = 3), none at i = 0
    full = orc.solve(A, b, kind="p-BiCGSafe-rr", tol=0.0, maxit=10, rr_m=3)
    assert full["rr_steps"] == 3
    lim = orc.solve(A, b, kind="p-BiCGSafe-rr", tol=0.0, maxit=10, rr_m=3, rr_M=6)
    assert lim["rr_steps"] == 1


def test_fp64_plain_vs_pipelined_early_agreement(orc):
    """Section 5.1: plain and pipelined histories are nearly identical early on
    (agree to 1e-9 over the first 15 iterations)."""
    A = W.cd2d(64, 20.0)
    b = W.rhs_ones(A)
    p = orc.solve(A, b, kind="ssBiCGSafe2", tol=0.0, maxit=16)["hist"]
    q = orc.solve(A, b, kind="p-BiCGSafe", tol=0.0, maxit=16)["hist"]
    assert np.max(np.abs(p[:16] - q[:16]) / p[:16]) <= 1e-9


def test_stop_test_position(orc):
    """Alg. 3/4: the stop test follows the inner products; x returned is x_i and
    iterations = i.  With b = 0 the first test stops at i = 0 with x = x_0."""
    A = W.tiny_random(10, 3)
    o = orc.solve(A, np.zeros(10), kind="p-BiCGSafe", tol=1e-10, maxit=50)
    assert o["iterations"] == 0 and np.all(o["x"] == 0) and o["status_name"] == "ok"
    A = W.cd2d(16, 5.0)
    b = W.rhs_ones(A)
    o = orc.solve(A, b, kind="ssBiCGSafe2", tol=1e-6, maxit=500)
    h = o["hist"]
    assert h[o["iterations"]] <= 1e-6 and np.all(h[:o["iterations"]] > 1e-6)


def test_restart_policy_reaches_true_tolerance(orc):
    """Build addition (true-residual check with restarts): the exit true residual is <= tol
    whenever the run reports success."""
    A = W.cd3d_upwind(20, 50.0)
    b = W.rhs_ones(A)
    for kind in KINDS:
        o = orc.solve(A, b, kind=kind, tol=1e-12, maxit=3000, max_restarts=5)
        assert o["status_name"] == "ok" and o["rel_res_true"] <= 1e-12


# ---------------------------------------------------------------- formats

def test_sell_invariants(orc):
    """SELL-C-sigma: perm is a permutation; lengths non-increasing inside each
    sigma window with ties in original order; slices padded to their longest
    row; the SELL product equals the CSR product exactly (same per-row order)."""
    A = W.powerlaw(n=3000, seed=7)
    C, sigma = 32, 256
    S = orc.sell_build(A, C, sigma)
    perm = S["perm"]
    assert np.array_equal(np.sort(perm), np.arange(A.n))
    lens = np.diff(A.rowptr)
    for w0 in range(0, A.n, sigma):
        seg = perm[w0:w0 + sigma]
        L = lens[seg]
        assert np.all(L[:-1] >= L[1:])
        for a, bb, la, lb in zip(seg[:-1], seg[1:], L[:-1], L[1:]):
            if la == lb:
                assert a < bb
        assert set(seg.tolist()) == set(range(w0, min(w0 + sigma, A.n)))
    inv = np.empty(A.n, dtype=np.int64)
    inv[perm] = np.arange(A.n)
    x = np.random.default_rng(1).standard_normal(A.n)
    xp = x[perm]
    yp = np.zeros(A.n)
    ns = (A.n + C - 1) // C
    for s in range(ns):
        width = (S["slice_ptr"][s + 1] - S["slice_ptr"][s]) // C
        rows = np.arange(s * C, min((s + 1) * C, A.n))
        assert width == lens[perm[rows]].max()
        acc = np.zeros(len(rows))
        for k in range(width):
            idx = S["slice_ptr"][s] + k * C + (rows - s * C)
            acc = np.array([fma(v, xp[c], a) for v, c, a in zip(S["val"][idx], S["col"][idx], acc)])
        yp[rows] = acc
    assert np.array_equal(yp, orc.spmv(A, x)[perm])


def test_bf16_round_to_nearest_even(orc):
    """BF16 conversion returns the nearest BF16 value, ties to even mantissa."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    v = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-30, 30, 5000),
                        [0.0, -0.0, 1.0, -1.0, 3.0e38, 1e-40, 65504.0]])
    bits = orc.to_bf16_bits(v)
    dec = torch.from_numpy(bits.view(np.int16).copy()).view(torch.bfloat16).double().numpy()
    nxt_up = torch.from_numpy((bits.astype(np.int32) + 1).astype(np.uint16).view(np.int16)).view(torch.bfloat16).double().numpy()
    nxt_dn = torch.from_numpy((bits.astype(np.int32) - 1).clip(0).astype(np.uint16).view(np.int16)).view(torch.bfloat16).double().numpy()
    err = np.abs(dec - v)
    fin = np.isfinite(nxt_up) & np.isfinite(nxt_dn) & (bits & 0x7FFF != 0)
    assert np.all(err[fin] <= np.abs(nxt_up - v)[fin])
    assert np.all(err[fin] <= np.abs(nxt_dn - v)[fin])
    # exact ties: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 -> even (1.0)
    t = orc.to_bf16_bits(np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8]))
    assert t[0] == 0x3F80 and t[1] == 0x3F82
    # values exactly representable in FP32 agree with torch's FP32 -> BF16 (RNE)
    f = rng.standard_normal(1000).astype(np.float32)
    tb = torch.from_numpy(f).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(orc.to_bf16_bits(f.astype(np.float64)), tb)


def test_all_cores_build_is_bit_identical(orc):
    """The OpenMP build of the same source (the all-cores CPU baseline) gives the single-threaded
    oracle's bits: SpMV rows, the vector recurrences and the correctly rounded inner products
    (exact per-thread partial sums merged exactly; checked on sums that cancel heavily and on a
    non-finite operand), and whole solves of all three methods with a restart."""
    rng = np.random.default_rng(11)
    n = 100003
    x = rng.standard_normal(n) * 10.0 ** rng.integers(-30, 30, n)
    y = rng.standard_normal(n)
    for a, b in [(x, y), (x, -x[::-1].copy()), (np.concatenate([x, -x]), np.concatenate([y, y]))]:
        assert orc.dot(a, b, parallel=True) == orc.dot(a, b)
    bad = y.copy()
    bad[n // 2] = np.inf
    assert np.isnan(orc.dot(x * 0, bad, parallel=True)) == np.isnan(orc.dot(x * 0, bad))
    A = W.cd2d(24, 20.0)
    b = W.rhs_ones(A)
    xs = rng.standard_normal(A.n)
    assert np.array_equal(orc.spmv(A, xs, parallel=True), orc.spmv(A, xs))
    for kind in ["ssBiCGSafe2", "p-BiCGSafe", "p-BiCGSafe-rr"]:
        r1 = orc.solve(A, b, kind=kind, tol=1e-12, maxit=400, rr_m=25, max_restarts=3)
        r8 = orc.solve(A, b, kind=kind, tol=1e-12, maxit=400, rr_m=25, max_restarts=3, parallel=True)
        assert r1["iterations"] == r8["iterations"] and r1["restarts"] == r8["restarts"]
        assert np.array_equal(r1["hist"], r8["hist"])
        assert np.array_equal(r1["x"], r8["x"])
