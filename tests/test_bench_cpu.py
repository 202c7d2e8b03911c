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


def _load(path):
    import importlib.util
    spec = importlib.util.spec_from_file_location("_golden_maker", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_side_lines_state_error_against_the_oracle_golden_files():
    """The side lines' error_vs_oracle reads the oracle's golden solves: the sampled rows of the
    batch file are the ones its generator recorded, an x that carries the oracle's values at the
    sampled rows has zero sampled error (but is not bit-identical), a method that the file lacks is
    compared with the file's p-BiCGSafe-rr solve, and another system size gives no comparison."""
    import numpy as np
    here = os.path.dirname(os.path.abspath(__file__))
    maker = _load(os.path.join(here, "golden", "make_batch_cd2d_512_solves.py"))
    for n in (1024, 4096, 30625, 65536):
        assert np.array_equal(bench.batch_sample_rows(n, maker.NSAMPLE), maker.sample_rows(n))

    gold = bench.side_golden("batch_cd2d_512")
    which = [0, 7, 511]
    xs = []
    for s in which:
        g = gold["systems"][s]
        x = np.zeros(g["n"])
        x[bench.batch_sample_rows(g["n"], gold["samples_per_system"])] = [float.fromhex(v) for v in g["x_sample"]]
        xs.append(x)
    e = bench.batch_error_vs_oracle(xs, which, gold)
    assert e["max_abs_err_sampled"] == 0.0 and e["bit_identical_systems"] == 0 and e["systems_checked"] == 3
    xs[1][bench.batch_sample_rows(len(xs[1]), gold["samples_per_system"])[3]] += 0.5
    assert bench.batch_error_vs_oracle(xs, which, gold)["max_abs_err_sampled"] == pytest.approx(0.5, abs=1e-12)

    pl = bench.side_golden("powerlaw_4m")
    rows = np.asarray(pl["sample_rows"])
    x = np.zeros(pl["n"])
    x[rows] = [float.fromhex(v) for v in pl["solves"]["ssBiCGSafe2"]["x_sample"]]
    e = bench.error_vs_oracle_side(x, "ssBiCGSafe2", pl["n"], pl)
    assert e["max_abs_err_sampled"] == 0.0 and not e["bit_identical"]
    assert bench.error_vs_oracle_side(x, "ssBiCGSafe2", pl["n"] - 1, pl) is None
    e = bench.error_vs_oracle_side(x, "GPBiCG", pl["n"], pl)   # a method the file lacks: its first solve
    assert e["oracle_kind"] == "p-BiCGSafe-rr" and e["max_abs_err_sampled"] > 0.0
    assert bench.side_golden("no_such_workload") is None
