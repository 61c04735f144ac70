"""The N > 1 path of bench.py on CPU: world size 2 over gloo.

Every rank of a multi-GPU run executes its own replica of the workload (the
transforms shard by job; no data-path collective); the timing is a barrier
plus the maximum over ranks, and only rank 0 prints.  Here two CPU processes
check those helpers, and that a non-zero rank of the reference arm exits
without doing any work.
"""

from __future__ import annotations

import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys
sys.path.insert(0, {root!r})
import torch
import bench
world, rank, local = bench.dist_setup()
assert world == 2
bench.dist_init(world, "gloo")
bench.dist_barrier(world)
m = bench.dist_max(1.5 + rank, world, torch.device("cpu"))
assert m == 2.5, m
bench.dist_barrier(world)
import argparse
args = argparse.Namespace(steps=1, warmup=3, gpus=2)
if rank == 1:
    bench.run_reference(args)   # returns at once on rank 1
print("rank", rank, "ok", flush=True)
import torch.distributed as dist
dist.destroy_process_group()
"""


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_timing_helpers_over_gloo(tmp_path):
    pytest.importorskip("torch.distributed")
    script = tmp_path / "worker.py"
    script.write_text(WORKER.format(root=ROOT))
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True))
    outs = []
    for p in procs:
        out, _ = p.communicate(timeout=180)
        outs.append(out)
        assert p.returncode == 0, out
    assert "rank 0 ok" in outs[0] and "rank 1 ok" in outs[1]
