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


def test_reference_arm_json_line():
    """`bench.py --impl reference` (the oracle on the host cores) prints the contract's JSON line;
    run here on a 16^3 grid so that it takes a second."""
    import json
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--size", "16",
                          "--steps", "1", "--warmup", "0", "--cpu-iters", "5"],
                         capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["unit"] == "solves/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == bench.host_cores()
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("cd3d_16:")
