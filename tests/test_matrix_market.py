"""The Matrix Market reader (workloads.read_matrix_market): general, symmetric,
skew-symmetric and pattern files, repeated entries, comments, and refusals, each
checked against the dense matrix written into the file (no GPU)."""
import numpy as np
import pytest

import workloads as W


def _write(path, header, size, entries, comments=("% a comment",)):
    with open(path, "w") as fh:
        fh.write(header + "\n")
        for c in comments:
            fh.write(c + "\n")
        fh.write(size + "\n")
        for e in entries:
            fh.write(" ".join(str(t) for t in e) + "\n")


def test_general_real_with_repeats(tmp_path):
    p = tmp_path / "g.mtx"
    _write(p, "%%MatrixMarket matrix coordinate real general", "3 3 5",
           [(1, 1, 2.5), (3, 1, -1.0), (2, 3, 4.0), (1, 1, 0.5), (3, 3, 1e-3)])
    A = W.read_matrix_market(str(p))
    D = np.array([[3.0, 0, 0], [0, 0, 4.0], [-1.0, 0, 1e-3]])
    assert A.n == 3 and A.nnz == 4
    assert np.array_equal(A.to_dense(), D)
    for i in range(A.n):   # canonical CSR: columns ascending
        assert np.all(np.diff(A.col[A.rowptr[i]:A.rowptr[i + 1]]) > 0)
    assert np.array_equal(W.rhs_ones(A), D.sum(axis=1))


def test_symmetric_skew_and_pattern(tmp_path):
    p = tmp_path / "s.mtx"
    _write(p, "%%MatrixMarket matrix coordinate real symmetric", "3 3 3", [(1, 1, 1.0), (3, 1, 2.0), (3, 2, -5.0)])
    assert np.array_equal(W.read_matrix_market(str(p)).to_dense(),
                          np.array([[1.0, 0, 2.0], [0, 0, -5.0], [2.0, -5.0, 0]]))
    p = tmp_path / "k.mtx"
    _write(p, "%%MatrixMarket matrix coordinate real skew-symmetric", "2 2 1", [(2, 1, 3.0)])
    assert np.array_equal(W.read_matrix_market(str(p)).to_dense(), np.array([[0, -3.0], [3.0, 0]]))
    p = tmp_path / "p.mtx"
    _write(p, "%%MatrixMarket matrix coordinate pattern general", "2 2 3", [(1, 1), (1, 2), (2, 2)])
    assert np.array_equal(W.read_matrix_market(str(p)).to_dense(), np.array([[1.0, 1.0], [0, 1.0]]))
    p = tmp_path / "i.mtx"
    _write(p, "%%MatrixMarket matrix coordinate integer general", "2 2 2", [(1, 1, 7), (2, 2, -2)])
    assert np.array_equal(W.read_matrix_market(str(p)).to_dense(), np.array([[7.0, 0], [0, -2.0]]))


def test_round_trip_of_a_workload(tmp_path):
    """A generated system written out and read back is the same CSR, bit for bit."""
    A = W.powerlaw(n=500, seed=3)
    p = tmp_path / "pl.mtx"
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    _write(p, "%%MatrixMarket matrix coordinate real general", "%d %d %d" % (A.n, A.n, A.nnz),
           [(r + 1, c + 1, repr(float(v))) for r, c, v in zip(rows, A.col, A.val)])
    B = W.read_matrix_market(str(p))
    assert B.n == A.n and np.array_equal(B.rowptr, A.rowptr)
    assert np.array_equal(B.col, A.col) and np.array_equal(B.val, A.val)


def test_refusals(tmp_path):
    cases = [("%%MatrixMarket matrix array real general", "2 2", []),
             ("%%MatrixMarket matrix coordinate complex general", "2 2 1", [(1, 1, 1.0, 0.0)]),
             ("%%MatrixMarket matrix coordinate real general", "2 3 1", [(1, 1, 1.0)]),
             ("%%MatrixMarket matrix coordinate real general", "2 2 2", [(1, 1, 1.0)]),
             ("%%MatrixMarket matrix coordinate real general", "2 2 1", [(3, 1, 1.0)]),
             ("%%NotMatrixMarket", "2 2 1", [(1, 1, 1.0)])]
    for k, (h, size, entries) in enumerate(cases):
        p = tmp_path / ("bad%d.mtx" % k)
        _write(p, h, size, entries)
        with pytest.raises(ValueError):
            W.read_matrix_market(str(p))


@pytest.mark.gpu
def test_solve_from_a_matrix_market_file(tmp_path):
    """A system read from a Matrix Market file solves on the GPU bit-identically to the oracle
    (FP64 p-BiCGSafe): the reader's CSR is what both sides take."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    import paper_2108_10591_gb300 as bcs
    A0 = W.cd2d(40, 30.0)
    rows = np.repeat(np.arange(A0.n), np.diff(A0.rowptr))
    p = tmp_path / "cd2d40.mtx"
    _write(p, "%%MatrixMarket matrix coordinate real general", "%d %d %d" % (A0.n, A0.n, A0.nnz),
           [(r + 1, c + 1, repr(float(v))) for r, c, v in zip(rows, A0.col, A0.val)])
    A = W.read_matrix_market(str(p))
    b = W.rhs_ones(A)
    S = bcs.solver_create(bcs.csr_upload(A), "p-BiCGSafe", tol=1e-10, maxit=2000, threads_per_row=1)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    res = bcs.solve(S, bd, xd)
    ref = oracle.solve(A, b, kind="p-BiCGSafe", tol=1e-10, maxit=2000, max_restarts=29)
    assert res["status"] == 0 and res["iterations"] == ref["iterations"]
    assert np.array_equal(xd.cpu().numpy(), ref["x"])
