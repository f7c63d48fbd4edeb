"""bench.py's reference arm (the FP64 oracle on the host cores) under torchrun
with two ranks, as the multi-GPU runs launch it: rank 0 alone works and prints
one JSON line on the GPU arm's workload config; the other rank exits 0
without work.  Needs no GPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_under_torchrun():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    from paper_2503_18118_gb300 import inputs
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(free_port()), os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--gpus", "2", "--steps", "2", "--warmup", "1", "--ref-seconds", "1.5"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["steps"] == 2 and out["warmup"] == 1
    assert out["metric"] == "mc_beamforming_trials_per_s" and out["unit"] == "trials/s" and out["higher_is_better"]
    assert out["config"] == bench.workload_config(inputs.HEADLINE)
    assert out["value"] > 0 and out["e2e"]["value"] == out["value"]
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["e2e"]["d2h_bytes_per_step"] == 0
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == out["value"] and cb["cores"] >= 1
    assert out["sample_trials_per_step"] >= 8 and str(out["sample_trials_per_step"]) in cb["sample"]
