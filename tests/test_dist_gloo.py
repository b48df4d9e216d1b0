"""The multi-rank plumbing of bench.py on the CPU: two gloo ranks launched the
way torchrun launches them (RANK / WORLD_SIZE / MASTER_* in the environment).
The timing rule: the job's time is the maximum over ranks and its value the
sum of the ranks' eigenpairs divided by that time; the reference arm runs on
rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, os, sys
sys.path.insert(0, sys.argv[1])
import bench
d = bench.Dist()
rank = d.rank
t = d.max(1.5 + rank)          # per-rank times 1.5 and 2.5
e = d.sum(10 * (rank + 1))     # per-rank eigenpairs 10 and 20
d.barrier()
class A:  # the reference arm's arguments; rank 1 must return without work
    workload = "no-such-workload"
    warmup = 0
    steps = 1
    gpus = 2
out = {"rank": rank, "world": d.world, "max": t, "sum": e, "value": e / t}
if rank != 0:
    bench.reference_arm(A(), d)
    out["reference_returned"] = True
d.close()
print(json.dumps(out))
'''


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_gloo_ranks_reduce_like_the_bench():
    pytest.importorskip("torch.distributed")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        so, se = p.communicate(timeout=240)
        assert p.returncode == 0, se[-2000:]
        outs.append(json.loads(so.strip().splitlines()[-1]))
    outs.sort(key=lambda o: o["rank"])
    for o in outs:
        assert o["world"] == 2
        assert o["max"] == 2.5 and o["sum"] == 30.0 and o["value"] == 12.0
    assert outs[1]["reference_returned"]
