"""The benchmark's multi-rank host logic on CPU (one process per rank, gloo):
rendezvous from the launcher's environment, the barrier, the slowest rank's
time (max over ranks), the units of all ranks (sum over ranks) and one
seeded instance per rank (weak scaling, no collective on the data path).  The
GPU path of the same helpers differs only in the backend (NCCL) and the device
of the reduced scalar.  Also: the reference arm does no work on ranks other
than 0.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, sys
sys.path.insert(0, %r)
import torch.distributed as dist
import bench
rank, world, local = bench.dist_setup("gloo")
bench.barrier(world)
mx = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
sm = bench.sum_over_ranks(100.0 + rank, world, "cpu")
bench.barrier(world)
print(json.dumps({"rank": rank, "world": world, "local": local, "max": mx, "sum": sm,
                  "seed": bench.rank_seed(rank)}))
dist.destroy_process_group()
""" % ROOT


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reduce_and_seed():
    pytest.importorskip("torch")
    import json
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=240)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    outs.sort(key=lambda d: d["rank"])
    assert [d["rank"] for d in outs] == [0, 1]
    for d in outs:
        assert d["world"] == 2 and d["local"] == d["rank"]
        assert d["max"] == 15.0  # the slowest rank's time, seen by every rank
        assert d["sum"] == 201.0  # the units of both ranks
    assert outs[0]["seed"] != outs[1]["seed"]  # each rank its own instance


def test_single_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.sum_over_ranks(7.0, 1, "cpu") == 7.0
    bench.barrier(1)


def test_reference_arm_is_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    # returns at once: no instance is generated and nothing is printed
    assert bench.run_reference(None) is None
