"""Host logic of the window-sharded MSM on CPU: world size 2 over gloo.

Algorithm 2 shards its windows over devices; ``paper_2604_17808_gb300.msm_shard``
gives each rank a contiguous range of windows, all-gathers the per-rank
parts and adds them.  Here the GPU calls are replaced by the oracle (the part
of a window range is sum_{k in range} 2^(k c) W_k with Algorithm 2's window
sums), so two CPU processes check the range assignment, the gather and the
final sum against the MSM definition.
"""

from __future__ import annotations

import os
import socket
import subprocess
import sys

import pytest

from paper_2604_17808_gb300.msm_shard import window_range

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_window_ranges_partition_the_windows():
    for K in range(0, 41):
        for world in range(1, 7):
            ranges = [window_range(K, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == K
            for (b0, e0), (b1, e1) in zip(ranges, ranges[1:]):
                assert e0 == b1
            sizes = [e - b for b, e in ranges]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0
    with pytest.raises(ValueError):
        window_range(10, 2, 2)


WORKER = r"""
import os, sys
sys.path.insert(0, {root!r})
import numpy as np
import torch
import torch.distributed as dist
import ntt_synth
from oracle import limbs_to_ints
from oracle import msm_oracle as mo
from paper_2604_17808_gb300.msm_shard import sharded_msm

world = int(os.environ["WORLD_SIZE"])
rank = int(os.environ["RANK"])
dist.init_process_group("gloo", rank=rank, world_size=world)

curve = mo.BN254_G1
c = 4
K = mo.num_windows(mo.BN254_SCALAR_BITS, c)
n = 20
ss = limbs_to_ints(ntt_synth.uniform_elements("bn254_fr", n, 0x5A00))
pts = mo.fixed_base_points(limbs_to_ints(ntt_synth.uniform_elements("bn254_fr", n, 0x5A01)))

class Plan:  # the one plan property the host logic reads
    def info(self):
        return {{"num_windows": K}}

def encode(P):
    return torch.from_numpy(mo.points_to_words([P]).view(np.int64)[0].copy())

def decode(t):
    return mo.words_to_points(t.numpy().view(np.uint64))

def partial(begin, end):
    acc = None
    for k in range(begin, end):
        W = mo.bucket_reduce_tree(mo.bucket_accumulate(mo.bucketize(ss, pts, k, c)))
        acc = curve.add(acc, mo.scalar_mul(curve, 1 << (k * c), W))
    return encode(acc)

def add_all(stacked):
    acc = None
    for P in decode(stacked):
        acc = curve.add(acc, P)
    return encode(acc)

scalars = torch.zeros((n, 4), dtype=torch.int64)
got = decode(sharded_msm(Plan(), scalars, None, partial_fn=partial, sum_fn=add_all))[0]
assert got == mo.msm(ss, pts), "sharded MSM differs from the definition"
print("rank", rank, "ok", flush=True)
dist.destroy_process_group()
"""


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_sharded_msm_over_gloo(tmp_path):
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
        try:
            out, _ = p.communicate(timeout=300)
        except subprocess.TimeoutExpired:
            p.kill()
            out, _ = p.communicate()
        outs.append((p.returncode, out))
    for rank, (rc, out) in enumerate(outs):
        assert rc == 0, f"rank {rank} failed:\n{out}"
        assert f"rank {rank} ok" in out
