"""bench.py's algorithmic-work model (CPU): the per-iteration bytes and flops
that the roofline numbers divide by, on the 128^3 benchmark system."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

N, NNZ = 2097152, 14581760   # 128^3 interior grid, 7-point stencil: 7 n - 6 * 128^2


def test_bytes_per_iteration_fp64():
    # two CSR passes (8-byte values, 4-byte columns, 4-byte row pointers) + 27 vector passes
    b = bench.bytes_per_iter("p-BiCGSafe", N, NNZ)
    assert b == 2 * (NNZ * 12 + 4 * (N + 1)) + 27 * N * 8
    assert b == pytest.approx(819.7e6, rel=1e-4)
    # ssBiCGSafe2 carries fewer vectors: 22 passes
    assert bench.bytes_per_iter("ssBiCGSafe2", N, NNZ) == 2 * (NNZ * 12 + 4 * (N + 1)) + 22 * N * 8


def test_bytes_per_iteration_fp32():
    b = bench.bytes_per_iter("p-BiCGSafe", N, NNZ, vbytes=4, mbytes=4)
    assert b == pytest.approx(476.6e6, rel=1e-4)


def test_flops_per_iteration_table1():
    # Table 1: 2 MV (2 flops per nonzero) + 26 alpha*x + 22 x+y per row for p-BiCGSafe
    assert bench.flops_per_iter("p-BiCGSafe", N, NNZ) == 4 * NNZ + 48 * N
    assert bench.flops_per_iter("ssBiCGSafe2", N, NNZ) == 4 * NNZ + 30 * N


def test_solve_work_adds_outer_step_set_up():
    f1, b1 = bench.solve_work("p-BiCGSafe", N, NNZ, 100, 1)
    f2, b2 = bench.solve_work("p-BiCGSafe", N, NNZ, 100, 2)
    assert f2 > f1 and b2 > b1
    assert f1 >= 100 * bench.flops_per_iter("p-BiCGSafe", N, NNZ)
    assert b1 >= 100 * bench.bytes_per_iter("p-BiCGSafe", N, NNZ)
