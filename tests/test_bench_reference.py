"""The benchmark's reference arm (the CPU oracle timed on the host cores)
runs without a GPU and prints one JSON line with the keys the benchmark
contract asks of it: the same metric, unit and direction as the GPU arm, an
`e2e` object with no host/device copies, and a `cpu_baseline` object that
describes the run itself (kind, cores, the bounded sample)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "5", "--warmup", "3"]
    env = dict(os.environ)
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout[-3000:]
    line = json.loads(lines[0])

    import bench
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC
    assert line["unit"] == "solves/s" and line["higher_is_better"] is True
    assert line["n_gpus"] == 1 and line["steps"] == 5 and line["warmup"] == 3
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["config"]["workload"] == bench.WORKLOAD_DESC
    assert line["vs_baseline"] is None and line["extrapolated"] is True

    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["value"] == line["value"] and cpu["unit"] == line["unit"]
    assert cpu["cores"] >= 1 and isinstance(cpu["sample"], str) and cpu["sample"]
    # the median sample time, extrapolated to a whole solve, is what `value` inverts
    assert abs(1.0 / (cpu["full_product_s_median"] * bench.PRODUCTS_PER_SOLVE_FP64) - line["value"]) \
        <= 1e-12 * line["value"]

    e2e = line["e2e"]
    assert e2e == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
