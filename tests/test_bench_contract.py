"""The benchmark's JSON line, on the host: the reference arm (the FP64 oracle
on the host cores) on a tiny sample prints one line with the keys the
measurement contract asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--ref-galaxies", "2",
           "--steps", "1", "--warmup", "0", "--n-warmup", "10", "--n-samples", "10", "--leapfrog", "4"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["impl"] == "reference"
    for k in ("value", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling", "vs_baseline",
              "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_gpus_2_starts_two_ranks_and_rank_0_prints_one_line():
    """--gpus 2 outside a launcher starts two ranks on this node (the driver's
    torchrun form); for the reference arm rank 0 alone measures and prints,
    reporting two GPUs, and the other rank exits 0."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--impl", "reference",
           "--ref-galaxies", "2", "--steps", "1", "--warmup", "0", "--n-warmup", "10", "--n-samples", "10",
           "--leapfrog", "4"]
    env = dict(os.environ)
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
        env.pop(k, None)
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["n_gpus"] == 2 and d["impl"] == "reference" and d["value"] > 0


def test_captured_traffic_applies_only_to_the_captured_source_and_settings():
    """The roofline's traffic is a captured figure per unit: it is reported for
    the kernel source and sampler settings it was captured on, and null once
    either differs."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    saved = dict(bench.CAPTURED_TRAFFIC)
    try:
        for kind, (path, _, per_unit, fixed) in saved.items():
            with open(os.path.join(ROOT, path), "rb") as fh:
                now = hashlib.sha256(fh.read()).hexdigest()
            bench.CAPTURED_TRAFFIC[kind] = (path, now, per_unit, fixed)
            assert bench.captured_traffic(kind, 300, dict(fixed)) == per_unit * 300
            for k, v in fixed.items():
                assert bench.captured_traffic(kind, 300, dict(fixed, **{k: v + 1})) is None
            bench.CAPTURED_TRAFFIC[kind] = (path, "0" * 64, per_unit, fixed)
            assert bench.captured_traffic(kind, 300, dict(fixed)) is None
    finally:
        bench.CAPTURED_TRAFFIC.clear()
        bench.CAPTURED_TRAFFIC.update(saved)
