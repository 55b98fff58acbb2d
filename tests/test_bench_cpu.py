"""bench.py's reference arm (the FP64 oracle timed on the host cores) needs no GPU: it runs
here, honours --steps / --warmup and prints the one JSON line of the bench contract."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
           "--warmup", "1", "--oracle-seconds", "0.5", "--n", "1500"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, check=True)
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference"
    assert rec["unit"] == "submatrices/s" and rec["higher_is_better"] is True
    assert rec["steps"] == 2 and rec["warmup"] == 1 and rec["n_gpus"] == 1
    assert rec["value"] > 0 and rec["ms_per_step"] > 0
    cb = rec["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == rec["value"] and cb["cores"] >= 1
    assert "2 timed step(s) after 1 untimed" in cb["sample"]
    e2e = rec["e2e"]
    assert e2e["value"] == rec["value"] and e2e["unit"] == rec["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert rec["config"]["workload"].startswith("overlap_uniform(n=1500,")


def test_reference_arm_reports_the_paper_lu_route_for_p1():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
           "--warmup", "0", "--oracle-seconds", "0.3", "--n", "800", "--p", "1"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, check=True)
    rec = json.loads(out.stdout.strip().splitlines()[-1])
    lu = rec["paper_lu_p1"]
    assert lu["value"] > 0 and lu["unit"] == rec["unit"] and lu["cores"] >= 1
    assert "p=1" in rec["config"]["workload"]


def test_reference_arm_under_torchrun_two_ranks():
    """Launched like the multi-GPU bench (torchrun, two ranks): rank 0 alone prints one line,
    the other rank exits 0 without work."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0", "--oracle-seconds", "0.3", "--rows", "500"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, check=True)
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2
    assert rec["config"]["workload"].startswith("overlap_uniform(n=1000,")   # weak scaling
