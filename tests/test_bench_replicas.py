"""The multi-GPU path of bench.py on CPU: two gloo ranks run the same
cross-rank reduction and throughput formula the NCCL run uses (replicas, no
collective on the data path; the job is timed by its slowest rank)."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) * 100 ms for its replica of 1e9 updates
        ms = (rank + 1) * 100.0
        t_max = bench.max_over_ranks(ms, world, "cpu")
        value = bench.replicas_throughput(1e9, world, t_max / 1e3)
        dist.barrier()
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"t_max": t_max, "value": value}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_and_aggregate(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for r in res:
        assert r["t_max"] == 200.0                 # the slowest rank's time on every rank
        assert r["value"] == pytest.approx(2e9 / 0.2)   # both ranks' work over that time


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.replicas_throughput(3e6, 1, 0.5) == 6e6


def test_reference_arm_silent_on_other_ranks(monkeypatch):
    """Under torchrun only rank 0 times the oracle and prints; the other
    ranks return at once without work."""
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(gpus=2, steps=1, warmup=0)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, {"name": "unused", "mol": None, "model": None})
    assert buf.getvalue() == ""
