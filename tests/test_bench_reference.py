"""The benchmark's reference arm (the FP64 oracle timed on the host cores)
keeps the JSON-line contract, alone and under a two-rank launch where only
rank 0 runs and prints (CPU only, no GPU)."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload_config():
    # the configuration keys the main arm reports for the 16x16 workload
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_main", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    from paper_2504_12037_gb300 import workloads as wl

    w = wl.workload(b.CONFIG)
    return b.headline_config(w, w.batch)


def _check_line(d, n_gpus):
    assert d["impl"] == "reference" and d["n_gpus"] == n_gpus
    # the same workload configuration as the main arm (its bounded sample in cpu_baseline)
    cfg = _workload_config()
    assert {k: d["config"][k] for k in cfg} == cfg
    assert d["config"]["batch_per_beta"] == 16384 and d["config"]["instances"] == 5
    assert d["value"] > 0 and d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["unit"] == d["e2e"]["unit"] == d["cpu_baseline"]["unit"]


def test_reference_arm_single_process():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    _check_line(json.loads(lines[0]), 1)


def test_reference_arm_two_ranks_rank0_prints():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    _check_line(json.loads(lines[0]), 2)
