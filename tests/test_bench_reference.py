"""The reference arm of the benchmark on CPU: `bench.py --impl reference` times the oracle
as it stands (its forward map restricted to sampled whole patches whose kernel rows are built
beforehand) and prints one JSON line with the same metric, unit and config as the GPU arm,
plus the CPU-baseline and end-to-end records.  Run here on the 9,600-node sphere to stay
short; the benchmark's default workload is the 153,600-node sphere."""
import json

import bench


def test_reference_arm_line(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)

    class Args:
        steps, warmup, workload = 2, 1, "sphere9600"
    res = bench.run_reference(Args())
    line = json.loads(json.dumps(res))
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["config"] == {"workload": bench.WORKLOADS["sphere9600"]}
    assert line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0 and line["higher_is_better"] is True and line["vs_baseline"] is None
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and "patches" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    # a step processes the sampled rows: value = 4 x rows per step / step time
    rows = 2 * bench.problem("sphere9600").nc ** 2
    assert abs(line["value"] - 4 * rows / (line["ms_per_step"] / 1e3)) < 1e-9 * line["value"]


def test_oracle_matvec_rows_match_the_full_oracle_map():
    """The sampled oracle matvec gives the oracle's full forward map on its rows."""
    import numpy as np
    from inputs import CONFIG_SPHERE_SMALL, random_densities
    from oracle import cbie
    prob = CONFIG_SPHERE_SMALL(8)
    delta = bench.delta_of(prob)
    om = bench.OracleMatvec(prob, delta, [1, 4])
    y = random_densities(prob.n, 3)
    op = cbie.build_operator(prob, cbie.QuadParams(delta=delta, n_beta=48, cov_d=4.0))
    full = cbie.apply(op, y)
    assert np.abs(om(y) - full[:, om.rows]).max() < 1e-12 * np.abs(full).max()
