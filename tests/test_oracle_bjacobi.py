"""Pins of the oracle's block-Jacobi preconditioning (no GPU): the diagonal
blocks and their inverses against exact rational inverses, numpy's
independent inversion and the dense block product; the preconditioned runs
against the plain oracle on the explicitly formed operator A M^-1, against
dense solves of block-diagonal systems, and against the true residual of the
original system.  A transposed block, a wrong block offset, a lost pivot swap
or an inverse applied on the wrong side fails at least one of them."""
from fractions import Fraction

import numpy as np
import pytest

import workloads as W

KINDS = ["ssBiCGSafe2", "p-BiCGSafe", "p-BiCGSafe-rr"]


def _dense_blocks(A, bs):
    """Diagonal blocks of A taken from its dense form (independent of the oracle)."""
    Ad = A.to_dense()
    out = []
    for b0 in range(0, A.n, bs):
        m = min(bs, A.n - b0)
        out.append((b0, Ad[b0:b0 + m, b0:b0 + m]))
    return out


def _as_dense_operator(M, n, bs):
    """The block-diagonal matrix whose rows are stored in M ([n, bs], block columns)."""
    out = np.zeros((n, n))
    for i in range(n):
        b0 = i - i % bs
        m = min(bs, n - b0)
        out[i, b0:b0 + m] = M[i, :m]
    return out


def test_bjacobi_bs1_is_the_reciprocal_diagonal(orc):
    """Blocks of one row: D is diag(A) and E its IEEE reciprocal, bit for bit."""
    A = W.cd2d(12, 20.0)
    D, E = orc.bjacobi_blocks(A, 1)
    d = np.diag(A.to_dense())
    assert np.array_equal(D[:, 0], d)
    assert np.array_equal(E[:, 0], 1.0 / d)


def test_bjacobi_inverse_exact_on_dyadic_blocks(orc):
    """Blocks whose elimination stays exact (dyadic entries, power-of-two pivots, one block
    that needs a row swap): E equals the exact rational inverse bit for bit.  The blocks are
    not symmetric, so a transposed inverse fails."""
    blocks = [
        np.array([[2.0, 0.0, 0.0], [1.0, 4.0, 0.0], [-0.5, 2.0, 8.0]]),       # lower triangular
        np.array([[0.0, 2.0, 0.0], [4.0, 0.0, 0.0], [0.0, 0.0, 0.5]]),        # needs the row swap
        np.array([[1.0, 0.5, 0.25], [0.0, 2.0, 1.0], [0.0, 0.0, 4.0]]),       # upper triangular
    ]
    n = 3 * len(blocks)
    Ad = np.zeros((n, n))
    for k, B in enumerate(blocks):
        Ad[3 * k:3 * k + 3, 3 * k:3 * k + 3] = B
    Ad[0, 5] = 3.0      # couplings outside the blocks must be ignored
    Ad[7, 1] = -7.0
    A = W.dense_to_csr(Ad)
    D, E = orc.bjacobi_blocks(A, 3)
    for k, B in enumerate(blocks):
        F = [[Fraction(float(v)) for v in row] for row in B]
        # exact inverse by Fraction Gauss-Jordan
        m = 3
        aug = [F[r] + [Fraction(int(r == c)) for c in range(m)] for r in range(m)]
        for p in range(m):
            piv = max(range(p, m), key=lambda r: abs(aug[r][p]))
            aug[p], aug[piv] = aug[piv], aug[p]
            d = aug[p][p]
            aug[p] = [v / d for v in aug[p]]
            for r in range(m):
                if r != p:
                    f = aug[r][p]
                    aug[r] = [a - f * b for a, b in zip(aug[r], aug[p])]
        exact = np.array([[float(aug[r][m + c]) for c in range(m)] for r in range(m)])
        assert np.array_equal(E[3 * k:3 * k + 3, :3], exact), k
        assert np.array_equal(D[3 * k:3 * k + 3, :3], B)


@pytest.mark.parametrize("n,bs,seed", [(37, 8, 1), (64, 4, 2), (100, 32, 3), (45, 2, 4), (33, 16, 5)])
def test_bjacobi_inverse_matches_numpy(orc, n, bs, seed):
    """Random nonsymmetric matrices (ragged last block when bs does not divide n): D is the
    dense diagonal block exactly, E agrees with numpy's inverse of it, and entries beyond a
    ragged block are zero."""
    rng = np.random.default_rng(seed)
    Ad = np.where(rng.random((n, n)) < 0.5, rng.standard_normal((n, n)), 0.0)
    Ad += np.diag(rng.uniform(0.1, 3.0, n) * rng.choice([-1.0, 1.0], n))   # not dominant: pivoting happens
    A = W.dense_to_csr(Ad)
    D, E = orc.bjacobi_blocks(A, bs)
    for b0, B in _dense_blocks(A, bs):
        m = B.shape[0]
        assert np.array_equal(D[b0:b0 + m, :m], B)
        assert not D[b0:b0 + m, m:].any() and not E[b0:b0 + m, m:].any()
        ref = np.linalg.inv(B)
        scale = np.abs(ref).max() * np.linalg.cond(B)
        assert np.abs(E[b0:b0 + m, :m] - ref).max() <= 1e-13 * scale


def test_bjacobi_singular_block_refused(orc):
    Ad = np.eye(8)
    Ad[4:6, 4:6] = [[1.0, 2.0], [2.0, 4.0]]     # singular 2x2 block, the matrix is not
    Ad[4, 0] = 1.0
    with pytest.raises(ValueError):
        orc.bjacobi_blocks(W.dense_to_csr(Ad), 2)
    Ad[4:6, 4:6] = [[0.0, 0.0], [0.0, 1.0]]     # zero column in the block
    with pytest.raises(ValueError):
        orc.bjacobi_blocks(W.dense_to_csr(Ad), 2)


@pytest.mark.parametrize("bs", [1, 2, 8, 32])
def test_bjacobi_apply_is_the_block_product(orc, bs):
    """z = M v agrees with the dense block-diagonal product (numpy), bit for bit at bs = 1."""
    A = W.tiny_random(70, seed=11, density=0.3)
    D, E = orc.bjacobi_blocks(A, bs)
    v = np.random.default_rng(3).standard_normal(A.n)
    for M in (D, E):
        z = orc.bjacobi_apply(M, v, bs)
        ref = _as_dense_operator(M, A.n, bs) @ v
        assert np.allclose(z, ref, rtol=1e-14, atol=1e-14 * np.abs(ref).max())
        if bs == 1:
            assert np.array_equal(z, M[:, 0] * v)
    # E (D x) returns x
    x = np.random.default_rng(4).standard_normal(A.n)
    assert np.allclose(orc.bjacobi_apply(E, orc.bjacobi_apply(D, x, bs), bs), x, rtol=0, atol=1e-13)


@pytest.mark.parametrize("kind", KINDS)
def test_bjacobi_solves_block_diagonal_system_at_once(orc, kind):
    """A block-diagonal A with the same blocks: A M^-1 is the identity up to rounding, so the
    preconditioned run stops after at most two iterations at numpy's solution."""
    rng = np.random.default_rng(7)
    n, bs = 96, 8
    Ad = np.zeros((n, n))
    for b0 in range(0, n, bs):
        Ad[b0:b0 + bs, b0:b0 + bs] = rng.standard_normal((bs, bs)) + 4.0 * np.eye(bs)
    A = W.dense_to_csr(Ad)
    b = rng.standard_normal(n)
    r = orc.solve_bjacobi(A, b, bs, kind=kind, tol=1e-10, maxit=50)
    assert r["status"] == 0 and r["iterations"] <= 2, r
    assert np.allclose(r["x"], np.linalg.solve(Ad, b), rtol=0, atol=1e-10)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("bs", [2, 8])
def test_bjacobi_runs_on_the_explicit_operator(orc, kind, bs):
    """The preconditioned run follows the plain oracle run on A M^-1 formed densely by numpy
    (histories within 1e-9 over the first 15 iterations; 1e-7 for p-BiCGSafe-rr, whose
    replacement steps recompute b - A x from an unconverged x, where the two operators'
    different rounding is amplified by cancellation); its x solves the original system (true
    residual of A, computed without the preconditioner, within the tolerance)."""
    A = W.cd2d(16, 20.0)
    b = W.rhs_ones(A)
    D, E = orc.bjacobi_blocks(A, bs)
    Ahat = W.dense_to_csr(A.to_dense() @ _as_dense_operator(E, A.n, bs))
    r = orc.solve_bjacobi(A, b, bs, kind=kind, tol=1e-10, maxit=500, rr_m=7, max_restarts=5)
    ref = orc.solve(Ahat, b, kind=kind, tol=1e-10, maxit=500, rr_m=7, max_restarts=5)
    k = min(15, len(r["hist"]), len(ref["hist"]))
    assert k >= 10
    assert np.allclose(r["hist"][:k], ref["hist"][:k], rtol=1e-7 if kind == "p-BiCGSafe-rr" else 1e-9, atol=0)
    assert r["status"] == 0
    assert orc.true_residual(A, b, r["x"]) <= 1e-10 * np.linalg.norm(b) * 1.0000001


def test_bjacobi_pipelined_follows_plain(orc):
    """Section 3's equivalence carried to A M^-1: p-BiCGSafe and p-BiCGSafe-rr (a replacement
    every 7 iterations) follow ssBiCGSafe2, histories within 1e-9 over the first 15
    iterations, all still above 1e-6."""
    A = W.cd2d(24, 50.0)
    b = np.random.default_rng(5).standard_normal(A.n)
    runs = {kind: orc.solve_bjacobi(A, b, 4, kind=kind, tol=1e-12, maxit=300, rr_m=7) for kind in KINDS}
    h0 = runs["ssBiCGSafe2"]["hist"][:15]
    assert len(h0) == 15 and h0.min() >= 1e-6
    assert runs["p-BiCGSafe-rr"]["rr_steps"] >= 2
    for kind in KINDS[1:]:
        assert np.allclose(runs[kind]["hist"][:15], h0, rtol=1e-9, atol=0), kind


def test_bjacobi_start_vector(orc):
    """A non-zero x_0 enters as y_0 = M x_0: starting from the solution of a block-diagonal
    system, the first true residual is at rounding level."""
    rng = np.random.default_rng(9)
    n, bs = 40, 4
    Ad = np.zeros((n, n))
    for b0 in range(0, n, bs):
        Ad[b0:b0 + bs, b0:b0 + bs] = rng.standard_normal((bs, bs)) + 3.0 * np.eye(bs)
    A = W.dense_to_csr(Ad)
    xs = rng.standard_normal(n)
    b = Ad @ xs
    r = orc.solve_bjacobi(A, b, bs, x0=xs, tol=1e-10, maxit=20)
    assert r["r0_norm"] <= 1e-12 * np.linalg.norm(b)
    assert np.allclose(r["x"], xs, rtol=0, atol=1e-12)
