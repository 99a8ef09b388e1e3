"""The benchmark's reference arm (the FP64 CPU oracle) keeps the JSON-line
contract: one line on rank 0 with the metric, unit, timing, the CPU baseline
description and a zero-copy e2e block; other ranks exit 0 silently."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env):
    env = dict(os.environ)
    env.update(extra_env)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run({"RANK": "0"})
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["unit"] == "pair-interactions/s" and d["value"] > 0
    assert d["ms_per_step"] > 0
    assert d["config"]["workload"] and d["config"]["n_points"] == 138830
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == d["value"] and cb["unit"] == d["unit"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_silently():
    r = _run({"RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_near_fraction_sample_matches_the_full_count():
    """The roofline's far/near flop weighting uses a sampled near-pair
    fraction; on the h = 1/16 sphere it agrees with the count over all
    ordered pairs."""
    sys.path.insert(0, ROOT)
    import bench
    from oracle import quadrature as Q
    h = 1 / 16
    xyz = Q.sphere_points(1.0, h)["xyz"]
    n = xyz.shape[1]
    r2 = (bench.RHO_FAR * 3 * h) ** 2
    full = sum(int((((xyz[:, i:i + 512, None] - xyz[:, None, :]) ** 2).sum(0) < r2).sum())
               for i in range(0, n, 512)) / n / n
    assert abs(bench.near_fraction(xyz, 3 * h) - full) < 0.1 * full
