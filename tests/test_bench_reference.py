"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps
the one-JSON-line contract of the main arm: same metric and unit, its own
cpu_baseline and e2e entries, the warm-up rule.  It runs the oracle only, so
it needs no GPU; the tube workload keeps it to a second."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=300)


def test_reference_arm_prints_one_contract_line():
    import bench

    r = _run("--impl", "reference", "--workload", "tube", "--steps", "3", "--warmup", "3")
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "MSUPS"
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == "tube" and d["config"]["fluid_sites"] == 12608
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "MSUPS", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_fewer_than_three_warmup_steps_are_refused():
    r = _run("--impl", "reference", "--workload", "tube", "--steps", "3", "--warmup", "2")
    assert r.returncode != 0 and "--warmup must be >= 3" in r.stderr
