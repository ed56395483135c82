"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2).

The hot path shards over cells, but every box in this setting has one GPU, so several GPUs
run independent replicas: the only cross-rank operations are the barrier and the max of the
timed region over ranks.  These tests run that logic, and the reference arm's rank-0-only rule,
with two gloo processes on 127.0.0.1.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


WORKER = r"""
import os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, ws = dist.get_rank(), dist.get_world_size()
t = bench.max_over_ranks(1.0 + rank, ws)
bench.barrier(ws)
print(f"rank{{rank}} max={{t}}", flush=True)
dist.destroy_process_group()
"""


def run_ranks(code, nranks=2, extra_env=None, timeout=120):
    port = free_port()
    procs = []
    for r in range(nranks):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(nranks),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1")
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=timeout)
        assert p.returncode == 0, e
        outs.append(o)
    return outs


def test_max_over_ranks_and_barrier_gloo():
    outs = run_ranks(WORKER.format(root=ROOT))
    assert "rank0 max=2.0" in outs[0]
    assert "rank1 max=2.0" in outs[1]


def test_reference_arm_prints_on_rank0_only():
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); sys.argv=['bench.py','--impl','reference',"
            "'--gpus','2','--steps','1','--warmup','0','--ref-cells','2']; import bench; bench.main()")
    outs = run_ranks(code, timeout=300)
    import json

    line = json.loads(outs[0].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    assert outs[1].strip() == ""
