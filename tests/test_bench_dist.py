"""Multi-process host logic of bench.py on CPU (gloo, world size 2).

With N GPUs the bench runs N independent replicas (every view is an
independent function of the frame and the camera): each rank times its own
steps, the slowest rank's time is taken, and the rate counts the units of
all ranks.  These tests run that logic with two gloo ranks on 127.0.0.1.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r'''
import os, sys, json
sys.path.insert(0, {root!r})
import torch, torch.distributed as dist
import bench
dist.init_process_group("gloo", rank=int(os.environ["RANK"]), world_size=int(os.environ["WORLD_SIZE"]))
rank = dist.get_rank()
ms = [12.5, 20.0][rank]
m = bench.max_over_ranks(ms, torch.device("cpu"))
rate = bench.whole_job_rate(50, dist.get_world_size(), m)
seeds = bench.make_scene("tiny", rank).views[0].opacity.sum()
out = [None, None]
dist.all_gather_object(out, float(seeds))
print(json.dumps({{"rank": rank, "max": m, "rate": rate, "scene_sums": out}}))
dist.destroy_process_group()
'''


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_timing_and_replicas():
    port = _free_port()
    code = WORKER.format(root=ROOT)
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=240)
        assert p.returncode == 0, e[-2000:]
        outs.append(o.strip().splitlines()[-1])
    import json
    res = [json.loads(o) for o in outs]
    for r in res:
        assert r["max"] == 20.0                      # the slowest rank's time
        assert abs(r["rate"] - 2 * 50 / 0.020) < 1e-6  # units of both ranks over that time
        a, b = r["scene_sums"]
        assert a != b                                # each replica renders its own frame


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", CUDA_VISIBLE_DEVICES="")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=240)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""
