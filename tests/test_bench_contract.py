"""The benchmark's reference arm on the CPU: the oracle timed on a bounded
sample, and the JSON line it prints (the keys and units the GPU arm uses, an
end-to-end figure with no host-device traffic)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_oracle_sample_times_a_bounded_number_of_steps():
    rate, steps, secs, threads = bench.oracle_sample(0.2)
    assert 1 <= steps <= 400
    assert secs > 0 and threads >= 1
    dof = bench.NX * bench.NX * (bench.P + 1) ** 2
    assert rate == dof * 3 * steps / secs


def test_reference_arm_prints_one_contract_line(monkeypatch, capsys):
    calls = []

    def fake_sample(target_s):
        calls.append(target_s)
        return 1.0e8, 10, 0.5, 16

    monkeypatch.setattr(bench, "oracle_sample", fake_sample)

    class Args:
        steps, warmup, gpus = 3, 2, 1

    bench.run_reference(Args, 1, 0)
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert len(calls) == Args.steps + Args.warmup
    # each sample stays bounded so that the whole arm ends within minutes
    assert all(2.0 <= t <= 150.0 for t in calls)
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["steps"] == 3 and d["warmup"] == 2 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "euler_vortex_128x128_p3_t10"
    dof = bench.NX * bench.NX * (bench.P + 1) ** 2
    assert d["value"] == dof * 3 * 30 / 1.5
    assert d["ms_per_step"] == 500.0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 16 and cb["value"] == d["value"]
    assert cb["unit"] == d["unit"] and "sample" in cb
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_is_silent_off_rank_zero(monkeypatch, capsys):
    monkeypatch.setattr(bench, "oracle_sample", lambda t: (_ for _ in ()).throw(AssertionError("ran")))

    class Args:
        steps, warmup, gpus = 1, 0, 2

    assert bench.run_reference(Args, 2, 1) is None
    assert capsys.readouterr().out == ""
