"""The benchmark's N > 1 host logic on the CPU with two gloo ranks: the job
time is the slowest rank's (max over ranks), the library is compiled by local
rank 0 before the other ranks look at it, and the reference arm runs on rank
0 alone (the path does not shard: each rank is an independent replica)."""

import json
import os
import socket
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CHILD = r"""
import argparse, json, os, sys, time
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
import bench
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:" + os.environ["PORT"], rank=rank,
                        world_size=world)
m = bench.max_over_ranks(1.5 + rank, world, "cpu")
log = os.environ["LOG"]

def fake_build():
    with open(log, "a") as f:
        f.write(f"start {rank}\n")
    if rank == 0:
        time.sleep(0.5)
    with open(log, "a") as f:
        f.write(f"end {rank}\n")

bench.build_in_rank_order(rank, world, fake_build, dist.barrier)
ref = None
if rank == 1:
    ref = bench.run_reference(argparse.Namespace(walls="beam", ref_sample=10, warmup=3, steps=1, gpus=2), rank, world)
dist.destroy_process_group()
print(json.dumps({"rank": rank, "max": m, "ref": ref}))
"""


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks(tmp_path):
    log = tmp_path / "build.log"
    port = str(_port())
    procs = []
    for r in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), PORT=port,
                   LOG=str(log), MASTER_ADDR="127.0.0.1")
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=240)
        assert p.returncode == 0, e
        lines = [line for line in o.splitlines() if line.strip()]
        assert len(lines) == 1  # rank 1's reference arm printed nothing
        outs.append(json.loads(lines[0]))
    assert [o["max"] for o in outs] == [2.5, 2.5]
    assert all(o["ref"] is None for o in outs)
    events = log.read_text().split("\n")[:4]
    assert events == ["start 0", "end 0", "start 1", "end 1"]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    calls = []
    assert bench.max_over_ranks(3.25, 1) == 3.25
    bench.build_in_rank_order(0, 1, lambda: calls.append("build"), lambda: calls.append("barrier"))
    assert calls == ["build"]
