"""The benchmark's reference arm (the oracle on the host cores) keeps the
JSON contract of the benchmark line: one line on rank 0 with the metric of
the GPU arm, its own CPU-baseline record and an end-to-end record with no
host-device traffic; other ranks print nothing and exit 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra, steps=1, warmup=3):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", str(steps),
                        "--warmup", str(warmup)], capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)
    return r


def test_reference_arm_line():
    r = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == "Msegments/s fwd+adjoint" and d["unit"] == "Msegments/s"
    assert d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"] is True and d["value"] > 0
    assert d["config"]["workload"].startswith("procedural office")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_do_nothing():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.strip().startswith("{")]


def test_cpu_baseline_record():
    """The GPU arm's cpu_baseline record: the oracle timed on the host cores
    over a bounded sample, with a single-thread figure beside it."""
    sys.path.insert(0, ROOT)
    import bench
    sc, lights, truth = bench.workload()
    r = bench.cpu_baseline(sc, lights, truth, budget_s=1.0)
    assert r["kind"] == "oracle" and r["unit"] == "Msegments/s" and r["cores"] == (os.cpu_count() or 1)
    assert r["value"] > 0 and r["sample"].startswith("photons [0, ")
    st = r["single_thread"]
    assert st["unit"] == "Msegments/s" and 0 < st["value"] and "one thread" in st["sample"]
