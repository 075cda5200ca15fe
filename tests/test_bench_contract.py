"""The benchmark's reference arm (the oracle, timed on the host cores) keeps
the JSON-line contract, and under a multi-rank launch only rank 0 works and
prints.  CPU only: the arm never touches a GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env):
    env = dict(os.environ)
    env.update(extra_env)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                           "--warmup", "1", "--T", "10"], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_json_line():
    r = _run({})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in d, key
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["higher_is_better"] is False and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_reference_arm_other_ranks_exit_quietly():
    r = _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_benchmark_partition_is_the_library_default():
    """The benchmark's supernode partition (used by its GPU workloads and
    by the oracle baselines' analysis) is the library's default one, so the
    IPM workload (library defaults) and the KKT / batch workloads (explicit
    options) run the same partition."""
    sys.path.insert(0, ROOT)
    import ctypes
    import bench
    from paper_2403_15913_gb300 import _native as nat
    o = nat.Options()
    nat.lib().kkt_default_options(ctypes.byref(o))
    for key, val in bench.PARTITION.items():
        assert getattr(o, key) == val, key
    assert o.subtree_cols == bench.SUBTREE_COLS
