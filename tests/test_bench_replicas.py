"""The benchmark's multi-GPU path is independent replicas: every rank solves its own copy,
the step time is the maximum over ranks and the value counts the work of all ranks.  These
CPU tests run that host logic with world size 2 over gloo (127.0.0.1), and check that the
reference arm (the CPU oracle) prints its single JSON line on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SNIPPET = r"""
import json, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world, _ = bench.dist_env()
t = bench.max_over_ranks(1.5 * (rank + 1), world)
bench.barrier(world)
print(json.dumps({{"rank": rank, "world": world, "t_max": t}}))
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _env(rank, world, port):
    return dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))


def test_max_over_ranks_and_barrier_with_two_gloo_ranks():
    port = _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", SNIPPET.format(root=ROOT)], env=_env(r, 2, port),
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = [p.communicate(timeout=180) for p in procs]
    for p, (out, err) in zip(procs, outs):
        assert p.returncode == 0, err
    rows = [json.loads(out.strip().splitlines()[-1]) for out, _ in outs]
    assert sorted(r["rank"] for r in rows) == [0, 1]
    assert all(r["world"] == 2 and r["t_max"] == 3.0 for r in rows)


def test_reference_arm_prints_on_rank_zero_only():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "1",
           "--cpu-sample", "6"]
    other = subprocess.run(cmd, env=_env(1, 2, 29555), capture_output=True, text=True, timeout=300)
    assert other.returncode == 0 and other.stdout.strip() == ""
    zero = subprocess.run(cmd, env=_env(0, 1, 29555), capture_output=True, text=True, timeout=300)
    assert zero.returncode == 0, zero.stderr
    lines = zero.stdout.strip().splitlines()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "DOF/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
