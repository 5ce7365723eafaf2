"""The benchmark's reference arm on the CPU: the oracle timed on a bounded
sample of the headline workload, and the JSON line it prints (the keys and
units the GPU arm uses, an end-to-end figure with no host-device traffic),
plus the host-side helpers of the GPU arm's line."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_headline_workload_is_the_seeded_batch():
    specs = bench.batch_specs()
    assert len(specs) == 64
    assert all(32 <= s["N"] <= 256 and s["p"] in (2, 3, 4) and 1.0 <= s["eps"] <= 5.0 for s in specs)
    assert bench.batch_dof(specs) == sum(s["N"] ** 2 * (s["p"] + 1) ** 2 for s in specs)
    # larger than L2 (129 MB) per FP32 state array, as the line's config says
    assert bench.batch_dof(specs) * 16 > 3 * 129e6


def test_oracle_batch_sample_times_the_given_instances(monkeypatch):
    tiny = [{"N": 4, "p": 2, "eps": 3.0}, {"N": 5, "p": 3, "eps": 2.0}]
    monkeypatch.setattr(bench, "batch_specs", lambda: tiny)
    states = bench.oracle_batch_states()
    assert [o.nx for o, _ in states] == [4, 5]
    rate, work, secs, threads = bench.oracle_batch_sample(2, states=states, threads=1)
    assert work == (16 * 9 + 25 * 16) * 3 * 2
    assert secs > 0 and threads == 1 and rate == work / secs


def test_reference_arm_prints_one_contract_line(monkeypatch, capsys):
    calls = []
    monkeypatch.setattr(bench, "oracle_batch_states", lambda every=1: ["s"])

    def fake_sample(steps=1, every=1, threads=None, states=None):
        calls.append((steps, states))
        return 1.0e8, 5.0e7, 0.5, 16

    monkeypatch.setattr(bench, "oracle_batch_sample", fake_sample)

    class Args:
        steps, warmup, gpus = 3, 2, 1

    bench.run_reference(Args, 1, 0)
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert len(calls) == Args.steps + Args.warmup
    assert all(s == 1 and st == ["s"] for s, st in calls)  # one bounded RK3 step per sample
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["steps"] == 3 and d["warmup"] == 2 and d["n_gpus"] == 1
    assert d["config"]["workload"] == bench.WORKLOAD
    assert d["value"] == 1.0e8  # 3 x 5e7 DOF-stages in 3 x 0.5 s
    assert d["ms_per_step"] == 500.0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 16 and cb["value"] == d["value"]
    assert cb["unit"] == d["unit"] and "sample" in cb and cb["cpu"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_is_silent_off_rank_zero(monkeypatch, capsys):
    monkeypatch.setattr(bench, "oracle_batch_states", lambda every=1: (_ for _ in ()).throw(AssertionError("ran")))

    class Args:
        steps, warmup, gpus = 1, 0, 2

    assert bench.run_reference(Args, 2, 1) is None
    assert capsys.readouterr().out == ""


def test_compact_rounds_floats_only():
    x = {"a": 1.23456789, "b": [2.0000001, 3], "c": "s", "d": None, "e": 0.0}
    assert bench.compact(x) == {"a": 1.235, "b": [2.0, 3], "c": "s", "d": None, "e": 0.0}


def test_loglog_interpolates_a_power_law():
    errs = [1e-2, 1e-3, 1e-4]
    times = [1.0, 10.0, 100.0]  # t ~ err^-1
    assert abs(bench.loglog(errs, times, 10 ** -3.5) - 10 ** 1.5) < 1e-9
    assert bench.loglog(errs, times, 1e-6) is None


def test_time_to_error_follows_the_frontier():
    rows = [{"ms": 10.0, "err": 1e-3}, {"ms": 20.0, "err": 1e-4}, {"ms": 40.0, "err": 2e-4},
            {"ms": 80.0, "err": 1e-5}]
    # the 40 ms run is beaten by the cheaper 20 ms one and is not on the frontier
    assert bench.time_to_error(rows, 1e-3) == 10.0
    assert abs(bench.time_to_error(rows, 10 ** -3.5) - 10 * 2 ** 0.5) < 1e-9
    assert abs(bench.time_to_error(rows, 10 ** -4.5) - 20 * 2 ** 1.0) < 1e-9
    assert bench.time_to_error(rows, 1e-6) is None
    assert bench.time_to_error(rows, 1.0) == 10.0
