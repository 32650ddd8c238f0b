"""The benchmark's contract on the CPU: the reference arm (the FP64 oracle on a
bounded triple sample) prints one JSON line with the keys the driver reads, the
non-zero ranks of a multi-rank reference run print nothing, and the seeded
serving stream is reproducible."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=600)
    return r


def test_reference_arm_prints_one_contract_line():
    pytest.importorskip("oracle")
    import oracle
    oracle.build()
    r = _run(["--impl", "reference", "--no", "3", "--nv", "8", "--steps", "1", "--warmup", "3"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC  # the same metric as the native arm
    assert d["unit"] == "TFLOP/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "no=3 nv=8" in cb["sample"]
    assert isinstance(cb["cpu"], str) and cb["cpu"]
    assert d["e2e"] == {"value": d["value"], "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_are_silent():
    r = _run(["--impl", "reference", "--no", "3", "--nv", "8", "--steps", "1", "--warmup", "3"],
             {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_bench_rejects_short_warmup():
    r = _run(["--impl", "reference", "--no", "3", "--nv", "8", "--steps", "1", "--warmup", "2"])
    assert r.returncode != 0


def test_serve_stream_is_seeded():
    sys.path.insert(0, ROOT)
    import bench
    a = bench.serve_stream(6, 4.0, 3, 5, seed=3)
    b = bench.serve_stream(6, 4.0, 3, 5, seed=3)
    assert len(a) == len(b) == 6
    for x, y in zip(a, b):
        assert all(x[k] == y[k] for k in ("t", "kind", "no", "nv", "nvec", "flop", "bytes"))
        assert np.array_equal(x["inp"].t2, y["inp"].t2)
        assert 3 <= x["no"] <= 5 and 6 * x["no"] - 1 <= x["nv"] <= 10 * x["no"] + 1
        mult = 1 if x["kind"] == "omega" else 2 * x["nvec"]
        assert x["flop"] == 4.0 * x["nv"] ** 4 * (x["no"] ** 3 - x["no"]) * mult
    times = [x["t"] for x in a]
    assert times[0] == 0.0 and np.all(np.diff(times) >= 0)


def test_serving_stream_is_the_mixed_workload():
    # 256 requests, Poisson 4/s, no ~ U{4..24}, nv = round(no * U[6, 10]),
    # residual or Jacobian with 1-6 vectors: the sizes are drawn without inputs
    sys.path.insert(0, ROOT)
    import bench
    plan = bench.serve_plan(256, 4.0, 4, 24)
    assert len(plan) == 256
    nos = [q["no"] for q in plan]
    assert min(nos) >= 4 and max(nos) <= 24 and len(set(nos)) > 15
    kinds = [q["kind"] for q in plan]
    assert 80 < kinds.count("omega") < 176
    assert all(1 <= q["nvec"] <= 6 for q in plan)
    rate = len(plan) / plan[-1]["t"]
    assert 3.0 < rate < 5.0


def test_blas_baseline_times_a_bounded_sample():
    """The BLAS-backed CPU baseline times the oracle's matrix form on a seeded
    sample; at a size where the sample is the whole loop its rate is positive."""
    import bench
    from cc3_inputs import make_inputs
    inp = make_inputs(3, 8, seed=2)
    r = bench.blas_sample(inp, seconds_target=30.0)
    assert r["value"] > 0 and r["cores"] >= 1 and r["unit"] == "TFLOP/s"
    assert r["sample"].startswith("7 of 7 triples (weight 24 of 24)")
