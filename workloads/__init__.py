"""Seeded synthetic inputs shaped like the paper's workloads.

Shared by the CUDA path's tests/benchmark and the CPU oracle; this module
holds none of the solver's arithmetic -- only matrix assembly and the
right-hand side b = A*1 (row sums), so that the exact solution is the all-ones
vector as in the paper's experiments (Section 5: "the solution is the unit
vector", x_0 = 0).

The paper's SuiteSparse matrices (Table 2) are not available; these stand in
for their shapes:
  cd2d      2D convection-diffusion, 5-point central differences (~ sherman3,
            tmt_unsym: 4-5 nonzeros per row)
  cd3d      3D convection-diffusion, 7-point first-order upwind (~ atmosmodd,
            6.9 per row, fluid dynamics)
  cd3d27    3D 27-point Laplacian + first-order upwind (~ poisson3Db, 27.7 per row)
  powerlaw  random nonsymmetric matrix with power-law row lengths, mostly
            near-diagonal columns (~ the irregular structural matrices)
  batch     hundreds of independent cd2d systems of uneven size
All assemblies list a row's columns in ascending order (canonical CSR).
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    n: int
    rowptr: np.ndarray  # int64[n+1]
    col: np.ndarray     # int32[nnz]
    val: np.ndarray     # float64[nnz]

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        D = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        np.add.at(D, (rows, self.col), self.val)
        return D


def rhs_ones(A: CSR) -> np.ndarray:
    """b = A * ones, i.e. the row sums (each row summed left to right)."""
    lens = np.diff(A.rowptr)
    b = np.zeros(A.n)
    nz = lens > 0
    if A.nnz:
        sums = np.add.reduceat(A.val, A.rowptr[:-1][nz])
        b[nz] = sums
    return b


def read_matrix_market(path: str) -> CSR:
    """A square real matrix from a Matrix Market file (coordinate format; real, integer or
    pattern; general, symmetric or skew-symmetric), as canonical CSR: columns ascending in
    every row, repeated (row, column) entries summed.  Symmetric files list one triangle: the
    mirrored entries are added (negated for skew-symmetric).  Pattern entries are 1.  This is
    how a supplied SuiteSparse matrix (the paper's Table 2) enters the solvers; none ships with
    this repository."""
    with open(path) as fh:
        header = fh.readline().split()
        if len(header) < 5 or header[0] != "%%MatrixMarket" or header[1].lower() != "matrix":
            raise ValueError("not a Matrix Market matrix file: %s" % path)
        fmt, field, sym = header[2].lower(), header[3].lower(), header[4].lower()
        if fmt != "coordinate":
            raise ValueError("only the coordinate format is read (got %s)" % fmt)
        if field not in ("real", "integer", "pattern"):
            raise ValueError("only real, integer or pattern entries are read (got %s)" % field)
        if sym not in ("general", "symmetric", "skew-symmetric"):
            raise ValueError("only general, symmetric or skew-symmetric matrices are read (got %s)" % sym)
        line = fh.readline()
        while line.startswith("%") or not line.strip():
            line = fh.readline()
        m, ncols, nz = (int(t) for t in line.split()[:3])
        if m != ncols:
            raise ValueError("the solvers take square matrices (got %d x %d)" % (m, ncols))
        ncolumns = 2 if field == "pattern" else 3
        data = np.loadtxt(fh, ndmin=2, comments="%", usecols=range(ncolumns)) if nz else np.zeros((0, ncolumns))
    if data.shape[0] != nz:
        raise ValueError("expected %d entries, read %d" % (nz, data.shape[0]))
    rows = data[:, 0].astype(np.int64) - 1
    cols = data[:, 1].astype(np.int64) - 1
    vals = np.ones(nz) if field == "pattern" else data[:, 2].astype(np.float64)
    if nz and (rows.min() < 0 or cols.min() < 0 or rows.max() >= m or cols.max() >= m):
        raise ValueError("entry index out of range")
    if sym != "general":
        off = rows != cols
        sign = -1.0 if sym == "skew-symmetric" else 1.0
        rows, cols, vals = (np.concatenate([rows, cols[off]]), np.concatenate([cols, rows[off]]),
                            np.concatenate([vals, sign * vals[off]]))
    key = rows * m + cols
    uk, inv = np.unique(key, return_inverse=True)
    summed = np.zeros(len(uk))
    np.add.at(summed, inv, vals)
    r, c = uk // m, uk % m
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    np.cumsum(rowptr, out=rowptr)
    return CSR(m, rowptr, c.astype(np.int32), summed)


def _stencil(dims, offsets):
    """Assemble a stencil matrix on a lexicographic grid (x fastest).
    dims: (kx, ky[, kz]); offsets: list of (offset tuple, coefficient)."""
    dims = tuple(int(d) for d in dims)
    nd = len(dims)
    n = int(np.prod(dims))
    strides = [1]
    for d in dims[:-1]:
        strides.append(strides[-1] * d)
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for d in dims:
        coords.append((rem % d).astype(np.int32))
        rem //= d
    del rem
    offs = sorted(offsets, key=lambda oc: sum(o * s for o, s in zip(oc[0], strides)))
    masks = []
    counts = np.zeros(n, dtype=np.int64)
    for off, _ in offs:
        m = np.ones(n, dtype=bool)
        for a in range(nd):
            if off[a] < 0:
                m &= coords[a] >= -off[a]
            elif off[a] > 0:
                m &= coords[a] < dims[a] - off[a]
        masks.append(m)
        counts += m
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    nnz = int(rowptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    fill = rowptr[:-1].copy()
    for (off, coef), m in zip(offs, masks):
        rows = np.nonzero(m)[0]
        lin = sum(o * s for o, s in zip(off, strides))
        pos = fill[rows]
        col[pos] = (rows + lin).astype(np.int32)
        val[pos] = coef
        fill[rows] += 1
    return CSR(n, rowptr, col, val)


def cd2d(k: int, beta: float) -> CSR:
    """-Lap(u) + beta (u_x + u_y) on a k x k interior grid, h = 1/(k+1),
    5-point central differences: centre 4/h^2, W,S -1/h^2 - beta/(2h),
    E,N -1/h^2 + beta/(2h)."""
    h = 1.0 / (k + 1)
    c, m1, p1 = 4.0 / h**2, -1.0 / h**2 - beta / (2 * h), -1.0 / h**2 + beta / (2 * h)
    return _stencil((k, k), [((0, 0), c), ((-1, 0), m1), ((1, 0), p1), ((0, -1), m1), ((0, 1), p1)])


def cd3d_upwind(k: int, beta: float) -> CSR:
    """-Lap(u) + beta (u_x + u_y + u_z) on k^3, h = 1/(k+1), 7-point Laplacian
    plus first-order upwind (backward) differences for the positive
    convection: centre 6/h^2 + 3 beta/h, minus-neighbours -1/h^2 - beta/h,
    plus-neighbours -1/h^2."""
    h = 1.0 / (k + 1)
    c = 6.0 / h**2 + 3.0 * beta / h
    m1, p1 = -1.0 / h**2 - beta / h, -1.0 / h**2
    offs = [((0, 0, 0), c)]
    for a in range(3):
        e = [0, 0, 0]
        e[a] = -1
        offs.append((tuple(e), m1))
        e[a] = 1
        offs.append((tuple(e), p1))
    return _stencil((k, k, k), offs)


def cd3d27(k: int, beta: float) -> CSR:
    """27-point Laplacian (centre 26, all 26 neighbours -1, scaled 1/(9 h^2) so
    that it is consistent with -Lap) plus beta-upwind on the 6 face neighbours
    as in cd3d_upwind; h = 1/(k+1)."""
    h = 1.0 / (k + 1)
    s = 1.0 / (9.0 * h**2)
    offs = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                off = (dx, dy, dz)
                nzc = sum(1 for v in off if v != 0)
                if nzc == 0:
                    coef = 26.0 * s + 3.0 * beta / h
                else:
                    coef = -s
                    if nzc == 1 and min(off) == -1:
                        coef -= beta / h
                offs.append((off, coef))
    return _stencil((k, k, k), offs)


def _powerlaw_xmin(a=2.1, hi=512.0, mean=16.0):
    """x_min of a continuous power law with density ~ x^-a on [x_min, hi] and the given mean."""
    def m(lo):
        num = (hi ** (2 - a) - lo ** (2 - a)) / (2 - a)
        den = (hi ** (1 - a) - lo ** (1 - a)) / (1 - a)
        return num / den
    lo, up = 1.0, hi
    for _ in range(200):
        mid = 0.5 * (lo + up)
        if m(mid) < mean:
            lo = mid
        else:
            up = mid
    return 0.5 * (lo + up)


def powerlaw(n: int = 4194304, seed: int = 210810591, exponent: float = 2.1, mean: float = 16.0,
             max_len: int = 512, p_local: float = 0.9) -> CSR:
    """Random nonsymmetric sparse matrix.  Row length L (diagonal included) is
    the rounded draw of a continuous power law (density ~ x^-exponent,
    truncated to [x_min, max_len], x_min chosen so the mean is `mean`),
    clipped to [1, max_len].  Each of the L-1 off-diagonal columns is, with
    probability p_local, uniform within +-n/100 of the row (wrapping around),
    otherwise uniform over [0, n); repeats and the diagonal are redrawn.
    Off-diagonal values are N(0,1); the diagonal is 1.2 x the row's absolute
    off-diagonal sum."""
    rng = np.random.default_rng(seed)
    a = exponent
    lo = _powerlaw_xmin(a, float(max_len), mean)
    u = rng.random(n)
    c0, c1 = lo ** (1 - a), float(max_len) ** (1 - a)
    xs = (c0 - u * (c0 - c1)) ** (1.0 / (1 - a))
    L = np.clip(np.rint(xs), 1, min(max_len, n)).astype(np.int64)
    noff = L - 1
    m = int(noff.sum())
    rows = np.repeat(np.arange(n, dtype=np.int64), noff)
    half = max(1, n // 100)

    def draw(r):
        k = len(r)
        loc = rng.random(k) < p_local
        c = np.empty(k, dtype=np.int64)
        nl = int(loc.sum())
        c[loc] = (r[loc] + rng.integers(-half, half + 1, size=nl)) % n
        c[~loc] = rng.integers(0, n, size=k - nl)
        return c

    cols = draw(rows)
    while True:
        key = rows * n + cols
        order = np.argsort(key, kind="stable")
        ks = key[order]
        bad_sorted = np.zeros(m, dtype=bool)
        if m > 1:
            bad_sorted[1:] = ks[1:] == ks[:-1]
        bad = np.zeros(m, dtype=bool)
        bad[order[bad_sorted]] = True
        bad |= cols == rows
        nb = int(bad.sum())
        if nb == 0:
            break
        cols[bad] = draw(rows[bad])
    offval = rng.standard_normal(m)
    # assemble with the diagonal, columns ascending
    absum = np.zeros(n)
    np.add.at(absum, rows, np.abs(offval))
    all_rows = np.concatenate([rows, np.arange(n, dtype=np.int64)])
    all_cols = np.concatenate([cols, np.arange(n, dtype=np.int64)])
    all_vals = np.concatenate([offval, 1.2 * absum])
    order = np.argsort(all_rows * n + all_cols, kind="stable")
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(L, out=rowptr[1:])
    return CSR(n, rowptr, all_cols[order].astype(np.int32), all_vals[order])


def batch_cd2d(count: int = 512, seed: int = 210810592, kmin: int = 32, kmax: int = 256):
    """`count` independent cd2d systems: side k ~ U{kmin..kmax}, beta ~ U[0, 50].
    Returns (list of CSR, sides, betas)."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(kmin, kmax + 1, size=count)
    betas = rng.uniform(0.0, 50.0, size=count)
    return [cd2d(int(k), float(bt)) for k, bt in zip(sides, betas)], sides, betas


def tiny_random(n: int, seed: int, density: float = 0.4, dominance: float = 1.5) -> CSR:
    """Small random nonsymmetric sparse matrix with N(0,1) off-diagonals and a
    diagonal of dominance x (row absolute sum) + 1."""
    rng = np.random.default_rng(seed)
    D = np.where(rng.random((n, n)) < density, rng.standard_normal((n, n)), 0.0)
    np.fill_diagonal(D, 0.0)
    np.fill_diagonal(D, dominance * np.abs(D).sum(axis=1) + 1.0)
    return dense_to_csr(D)


def tiny_integer(n: int, seed: int, lo: int = -3, hi: int = 3, shift: int = 9) -> np.ndarray:
    """Small dense integer matrix (entries in [lo, hi], about half zero) plus shift*I."""
    rng = np.random.default_rng(seed)
    M = rng.integers(lo, hi + 1, size=(n, n))
    M[rng.random((n, n)) < 0.5] = 0
    return M + shift * np.eye(n, dtype=np.int64)


def dense_to_csr(D: np.ndarray) -> CSR:
    n = D.shape[0]
    rows, cols = np.nonzero(D)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    np.cumsum(rowptr, out=rowptr)
    return CSR(n, rowptr, cols.astype(np.int32), D[rows, cols].astype(np.float64))


# Named workloads (the benchmark's and the tests' configurations).
WORKLOADS = {
    "cd2d_64": dict(desc="2D -Lap u + 20(u_x+u_y), 64x64 interior, central differences, FP64",
                    make=lambda: cd2d(64, 20.0)),
    "cd3d_128": dict(desc="3D -Lap u + 50(u_x+u_y+u_z), 128^3, 7-point first-order upwind, FP64",
                     make=lambda: cd3d_upwind(128, 50.0)),
    "powerlaw_4m": dict(desc="random nonsymmetric n=4194304, power-law rows (2.1, mean 16, max 512)",
                        make=lambda: powerlaw()),
    "cd3d27_192": dict(desc="3D 27-point Laplacian + 100-upwind, 192^3", make=lambda: cd3d27(192, 100.0)),
}
