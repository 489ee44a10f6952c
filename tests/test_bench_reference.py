"""The benchmark's reference arm (the oracle timed on the host cores) keeps
the one-JSON-line contract on a machine without a GPU, and under a multi-rank
launch only rank 0 runs and prints."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env, *args):
    env = dict(os.environ, **extra_env)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--n", "4096", *args], cwd=ROOT, env=env, capture_output=True,
                          text=True, timeout=300)


def test_reference_line_contract():
    r = _run({}, "--steps", "2", "--warmup", "1", "--gpus", "1")
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["unit"] == "Gpair-interactions/s"
    assert d["higher_is_better"] is True
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 2, 1)
    assert d["config"]["n"] == 4096 and d["data"] == "synthetic"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_other_ranks_exit_quietly():
    env = {"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"}
    r = _run(env, "--steps", "1", "--warmup", "0", "--gpus", "2")
    assert r.returncode == 0, r.stderr
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


@pytest.mark.parametrize("workload", ["c1", "c3", "c4", "paper", "plunge", "sym"])
def test_reference_arm_of_each_workload(workload):
    """The secondary workloads' reference arm times the oracle on the same
    workload's metric, on the host cores only."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", workload, "--steps", "1", "--warmup", "0"], cwd=ROOT,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["higher_is_better"] is (workload != "c1")
    assert d["unit"] == ("us/step" if workload == "c1" else "Gpair-interactions/s")
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["config"]["workload"] == d["workload"]


def test_serving_workload_has_no_reference():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "c5"], cwd=ROOT, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr
    d = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][0])
    assert d["impl"] == "reference" and "unavailable" in d
