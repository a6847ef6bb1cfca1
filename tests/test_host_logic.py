"""Host-side logic on CPU: seeded inputs, the learned workload's set-up
helpers, and the benchmark's command line (no GPU, no library calls)."""
import importlib.util
import os

import numpy as np

from paper_2505_00384_gb300 import inputs
from paper_2505_00384_gb300 import learned as LP

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_splitmix64_known_values():
    """splitmix64 from seed 0: the first outputs of the published generator."""
    z = inputs.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_normal_deviates_are_standard():
    x = inputs.normal(inputs.DEFAULT_SEED, 200000)
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1.0) < 0.01
    assert np.array_equal(x, inputs.normal(inputs.DEFAULT_SEED, 200000))


def test_hill_heights_are_seeded_and_in_range():
    h = LP.hill_heights(16)
    assert h.shape == (16,) and h.min() >= 200.0 and h.max() <= 800.0
    assert np.array_equal(h, LP.hill_heights(16)) and not np.array_equal(h, LP.hill_heights(16, seed=7))


def test_box_mesh_description():
    d = LP.box_mesh(450.0)
    assert (d.nx, d.ny, d.nz, d.degree) == (4, 4, 4, 2)
    assert d.terrain == 1 and d.bc_lateral == 2 and d.h_c == 450.0
    assert d.x_c == d.y_c == 500.0 and d.Lx == d.Ly == d.Lz == 1000.0


def test_bench_defaults():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    import sys
    argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        a = bench.parse()
    finally:
        sys.argv = argv
    assert a.gpus == 1 and a.warmup >= 3 and a.workload == "hill" and a.impl == "ours"
    w = bench.workload(a)
    assert (w["nx"], w["ny"], w["nz"], w["r"]) == (64, 64, 32, 4) and w["bc_lateral"] == 1  # far field


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    return bench


def test_bench_hbm_fractions():
    bench = _bench()
    gbs, src = bench.measured_hbm_gbs()
    assert gbs > 1000.0 and isinstance(src, str)
    a, f = bench.hbm_fractions(2e9, 0.5, 8000.0)
    assert abs(a - 4.0) < 1e-12 and abs(f - 0.0005) < 1e-15
    assert bench.hbm_fractions(None, 0.5, 8000.0) == (None, None)
    assert bench.hbm_fractions(1e9, 0.0, 8000.0) == (None, None)


def test_bench_oracle_baseline_on_one_core():
    """The CPU-baseline leg on a bounded sample: all cores, then one thread
    (restored afterwards), both positive and scaled to a step."""
    import oracle as O
    bench = _bench()
    w = dict(bench.SMALL)
    w.update(bench.COMMON)
    before = O.max_threads()
    v, sample, threads = bench.oracle_step_cost(w, budget_s=0.5)
    v1, sample1, threads1 = bench.oracle_step_cost(w, budget_s=0.5, threads=1)
    assert v > 0 and v1 > 0 and threads == before and threads1 == 1 and O.max_threads() == before
    assert "random cells" in sample and "random cells" in sample1


def _default_args(bench):
    import sys
    argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        return bench.parse()
    finally:
        sys.argv = argv


def _reference_line(bench, monkeypatch, capsys, rank):
    """Run the reference arm's driver with the oracle timing replaced by a
    fixed cost (the arm's JSON line, not the oracle, is under test here)."""
    import sys
    calls = []

    def fake_cost(work, budget_s=15.0, threads=None):
        calls.append(budget_s)
        return 123.0 + len(calls), "fixed sample", 4

    monkeypatch.setattr(bench, "oracle_step_cost", fake_cost)
    monkeypatch.setenv("RANK", str(rank))
    monkeypatch.setenv("LOCAL_RANK", str(rank))
    monkeypatch.setenv("WORLD_SIZE", "2" if rank else "1")
    argv = sys.argv
    try:
        sys.argv = ["bench.py", "--impl", "reference", "--steps", "3", "--warmup", "2"]
        assert bench.main() == 0
    finally:
        sys.argv = argv
    return calls, capsys.readouterr().out


def test_bench_reference_arm_line(monkeypatch, capsys):
    """Rank 0 prints one JSON line with the contract's keys; the value is the
    median of the timed steps only (warm-up steps excluded)."""
    import json
    bench = _bench()
    calls, out = _reference_line(bench, monkeypatch, capsys, 0)
    lines = [l for l in out.splitlines() if l.strip()]
    assert len(calls) == 5 and len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["higher_is_better"] is False and d["steps"] == 3 and d["warmup"] == 2
    assert d["value"] == 127.0 and abs(d["ms_per_step"] - 127000.0) < 1e-9  # median of 126, 127, 128
    assert d["config"] == {"workload": bench.workload(_default_args(bench))["name"]}
    cb = d["cpu_baseline"]
    assert cb["value"] == d["value"] and cb["cores"] == 4 and cb["kind"] == "oracle" and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_bench_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    bench = _bench()
    calls, out = _reference_line(bench, monkeypatch, capsys, 1)
    assert calls == [] and out.strip() == ""
