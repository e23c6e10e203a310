"""The reference arm of the benchmark on CPU: `bench.py --impl reference` times the oracle
as it stands on a bounded sample of the benchmark workload and prints one JSON line with the
same metric, unit and config as the GPU arm, plus the CPU-baseline and end-to-end records."""
import json

import bench


def test_reference_arm_line(monkeypatch):
    real = bench.cpu_baseline
    monkeypatch.setattr(bench, "cpu_baseline", lambda prob, delta, budget_s=15.0: real(prob, delta, budget_s=0.1))
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)

    class Args:
        steps, warmup = 2, 1
    res = bench.run_reference(Args())
    line = json.loads(json.dumps(res))
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["config"] == {"workload": bench.WORKLOAD} and line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0 and line["higher_is_better"] is True and line["vs_baseline"] is None
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and "patches" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    # one step is one forward map of the workload, extrapolated from the sample
    n = bench.problem().n
    assert abs(line["ms_per_step"] - 1e3 * 4 * n / line["value"]) < 1e-9 * line["ms_per_step"]
