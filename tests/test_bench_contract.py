"""bench.py's reference arm (the FP64 oracle on the host cores) prints one
JSON line with the contract's keys (CPU only, a tiny sample)."""
import json
import os
import subprocess
import sys

from tests.conftest import ROOT


def test_reference_arm_prints_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--sample-steps", "5"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_step_counters_are_used_only_for_the_captured_source(tmp_path, monkeypatch):
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "k.cuh"
    src.write_text("__global__ void k() {}\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    prof = tmp_path / "p.md"
    prof.write_text("# summary\n\ncounters: " + json.dumps({"source_sha256": sha, "dram_bytes_per_step": 1.5e6,
                                                            "l1tex_throughput_frac": 0.4,
                                                            "issue_active_frac": 0.45}) + "\n")
    monkeypatch.setattr(bench, "STEP_PROFILE", str(prof))
    monkeypatch.setattr(bench, "STEP_SOURCE", str(src))
    c = bench.step_kernel_counters()
    assert c["dram_bytes_per_step"] == 1.5e6
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.step_kernel_counters() is None
    monkeypatch.setattr(bench, "STEP_PROFILE", str(tmp_path / "missing.md"))
    assert bench.step_kernel_counters() is None


def test_reference_arm_runs_on_rank_zero_only():
    # under torchrun every rank starts bench.py; the reference arm (the host
    # oracle) runs and prints on rank 0 alone, the other ranks exit 0 at once
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "0", "--sample-steps", "5"], capture_output=True, text=True,
                         timeout=300, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == ""
