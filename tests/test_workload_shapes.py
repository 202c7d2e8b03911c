"""The synthetic inputs have the sizes and structure stated for them (CPU):
nonzero counts equal the closed forms of the stencils, and the random
generators' statistics are those of their recipe."""
import numpy as np

import workloads as W


def _check_csr(A):
    assert A.rowptr[0] == 0 and A.rowptr[-1] == A.nnz and np.all(np.diff(A.rowptr) >= 0)
    for i in range(0, A.n, max(1, A.n // 97)):
        c = A.col[A.rowptr[i]:A.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0) and c.min() >= 0 and c.max() < A.n


def test_cd2d_closed_form():
    for k in [1, 2, 7, 64]:
        A = W.cd2d(k, 20.0)
        assert A.n == k * k and A.nnz == 5 * k * k - 4 * k
        _check_csr(A)
    assert W.cd2d(64, 20.0).nnz == 20224


def test_cd3d_upwind_closed_form():
    for k in [1, 3, 16]:
        A = W.cd3d_upwind(k, 50.0)
        assert A.n == k ** 3 and A.nnz == 7 * k ** 3 - 6 * k ** 2
        _check_csr(A)
    assert 7 * 128 ** 3 - 6 * 128 ** 2 == 14581760


def test_cd3d27_closed_form():
    for k in [1, 2, 5]:
        A = W.cd3d27(k, 100.0)
        assert A.n == k ** 3 and A.nnz == (3 * k - 2) ** 3
        _check_csr(A)
    assert (3 * 192 - 2) ** 3 == 189119224


def test_powerlaw_statistics():
    A = W.powerlaw(n=200000, seed=7)
    lens = np.diff(A.rowptr)
    assert abs(lens.mean() - 16.0) < 0.5 and lens.max() <= 512 and lens.min() >= 1
    # heavy tail: a few rows far above the mean
    assert np.percentile(lens, 99.9) > 100
    rows = np.repeat(np.arange(A.n), lens)
    off = A.col != rows
    dist = np.abs(A.col[off] - rows[off])
    dist = np.minimum(dist, A.n - dist)  # local band wraps around
    local = np.mean(dist <= A.n // 100)
    assert 0.88 < local < 0.93  # 90 % local + the uniform ones that happen to land in the band
    # diagonal = 1.2 x off-diagonal absolute row sum
    i = 12345
    seg = slice(A.rowptr[i], A.rowptr[i + 1])
    c, v = A.col[seg], A.val[seg]
    d = v[c == i][0]
    assert np.isclose(d, 1.2 * np.abs(v[c != i]).sum())
    _check_csr(A)


def test_batch_ranges():
    mats, sides, betas = W.batch_cd2d(count=512)
    assert len(mats) == 512 and sides.min() >= 32 and sides.max() <= 256
    assert betas.min() >= 0.0 and betas.max() <= 50.0
    assert all(A.n == k * k for A, k in zip(mats[:20], sides[:20]))
