"""bench.py's reference arm (the oracle timed on the host cores) keeps the
benchmark's one-line JSON contract: the same metric and unit as the GPU
arm, impl "reference", a cpu_baseline describing the run, an e2e object
with no host-device bytes, and no output on ranks other than 0. Also the
failure path of the GPU arm's fresh-process end-to-end run."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "12",
                           "--steps", "2", "--warmup", "1"], capture_output=True, text=True, env=env, timeout=600,
                          cwd=ROOT)


def test_reference_line():
    import bench
    r = _run()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["n_qubits"] == 12 and "12 qubits" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_other_ranks_are_silent():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_e2e_child_failure_is_reported_not_raised():
    """Where the fresh-process end-to-end run cannot run (here: no GPU), the
    benchmark gets an error record instead of an exception, and keeps its
    in-process measurement."""
    import pytest
    import torch
    if torch.cuda.is_available():
        pytest.skip("the child run succeeds where a GPU is present")
    import bench
    out = bench.e2e_child(12, "beam", 9, 0, True, 0, 0, 3)
    assert set(out) == {"error"} and out["error"].startswith("e2e child exited")
