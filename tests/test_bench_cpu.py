"""bench.py's reference arm (the CPU oracle) and its JSON line, on the host.

The reference arm needs no GPU: it times the oracle on a bounded sample of
the workload.  Its line must carry the contract's keys; under several ranks
only rank 0 prints.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True, text=True,
                       timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    return [l for l in r.stdout.splitlines() if l.strip()]


@pytest.mark.parametrize("workload", ["config1", "hwea300"])
def test_reference_arm_line(workload):
    lines = _run(["--impl", "reference", "--workload", workload, "--steps", "1", "--warmup", "0"])
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "variant-shots/s" and d["steps"] == 1 and d["warmup"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("config1" if workload == "config1" else "hwea300")
    assert d["vs_baseline"] is None


def test_reference_arm_other_ranks_are_silent():
    lines = _run(["--impl", "reference", "--workload", "config1", "--steps", "1", "--warmup", "0"],
                 {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert lines == []


def test_cpu_baseline_single_and_threaded():
    """The GPU arm's cpu_baseline: the oracle single-threaded and over all
    host cores (spawned processes)."""
    sys.path.insert(0, ROOT)
    import bench
    from workloads import config1
    b = bench.oracle_baseline([config1()], threaded_budget_s=1.0)
    assert b["kind"] == "oracle" and b["cores"] == 1 and b["value"] > 0
    t = b["threaded"]
    assert t["cores"] == bench.host_cores() and t["value"] > 0 and t["unit"] == b["unit"]
