"""The benchmark's command-line contract.  On the CPU: the reference arm (the oracle on the
host cores) prints one JSON line with the keys the contract names, and too few warm-up steps
are refused.  On the GPU: the GPU arm's line carries its roofline, e2e, clocks and launch
count."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _bench("--impl", "reference", "--workload", "small", "--steps", "2", "--warmup", "3")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "vehicle-steps/s" and d["unit"] == "vehicle-steps/s"
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["config"]["workload"] == "small" and d["data"] == "synthetic"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_too_few_warmup_steps_are_refused():
    r = _bench("--impl", "reference", "--workload", "small", "--steps", "2", "--warmup", "2")
    assert r.returncode != 0 and "--warmup must be >= 3" in (r.stdout + r.stderr)


@pytest.mark.gpu
def test_gpu_arm_line_carries_roofline_e2e_clocks_and_launches():
    """The GPU arm on the 1M-vehicle grid (a few steps): the keys the contract adds to the
    line -- roofline of the dominant kernel against the measured peak, e2e through the C ABI
    with its copy sizes, clocks sampled during the timed region, the count of launches."""
    r = _bench("--workload", "grid1m", "--steps", "3", "--warmup", "3", "--no-cpu-baseline")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["metric"] == "vehicle-steps/s" and d["value"] > 0 and d["dtype"] == "f32"
    assert d["gpu_launches"] == 5 * d["steps"]
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and rf["kernel"] in rf["kernel_ms"]
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-9 and 0 < rf["frac"] < 1.5
    assert set(rf["kernel_frac"]) == set(rf["kernel_ms"])
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] > 0
    c = d["clocks"]
    assert c["sm_mhz"] > 0 and c["sm_max_mhz"] > 0 and isinstance(c["reasons"], list)
