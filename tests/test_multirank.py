"""The N > 1 path of bench.py on the CPU: world size 2 with the gloo backend
(the GPU machine has one GPU, so the ranks' host logic is tested here).  The step
of one domain does not shard: ranks are independent replicas, and the only
cross-rank operations are the max over ranks of the step time and rank 0's
report."""
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


def torchrun(args, timeout):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={free_port()}"] + args
    env = dict(os.environ, OMP_NUM_THREADS="1")
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def json_lines(text):
    out = []
    for line in text.splitlines():
        line = line.strip()
        if line.startswith("{"):
            out.append(json.loads(line))
    return out


def test_slowest_rank_and_aggregate_throughput_gloo():
    pytest.importorskip("torch")
    r = torchrun([os.path.join("tests", "multirank_worker.py")], timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = sorted(json_lines(r.stdout), key=lambda d: d["rank"])
    assert [d["rank"] for d in lines] == [0, 1]
    for d in lines:
        assert d["world"] == 2
        assert d["slowest_ms"] == 15.0                  # max over ranks, seen by every rank
        assert d["value"] == pytest.approx(2 * 1e6 / 15e-3 / 1e6)
    assert lines[0]["seed"] != lines[1]["seed"]          # replicas step different cities


def test_reference_arm_two_ranks_rank0_reports():
    """--impl reference under torchrun: rank 0 alone times the oracle and prints
    one line; the other rank exits 0 without work."""
    pytest.importorskip("torch")
    r = torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "3",
                  "--ref-workload", "small"], timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["nproc"] >= 1 and d["cpu_baseline"]["cpu_model"]
    assert 1 <= d["steps"] <= 2 and len(d["sweeps_per_step"]) == d["steps"]
    assert all(s > 0 for s in d["sweeps_per_step"])
    assert d["e2e"]["h2d_bytes_per_step"] == 0
