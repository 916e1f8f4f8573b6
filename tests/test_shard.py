"""Host logic of the direction-sharded 3D iteration (Sect. 2.2: the
directions of one radiation-field simulation are independent, so each rank
marches a share of them and the per-cell sums are added over the ranks
before the solve), on CPU with two gloo ranks.

A stand-in model keeps a fixed contribution per direction to each
accumulator array; its march sums the contributions of the directions it is
given, and its solve records the sums it sees.  With the directions split
over the ranks and the arrays all-reduced, every rank's solve must see the
sums over all directions -- the single-device result -- in every iteration.
"""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2009_12609_gb300 import shard  # noqa: E402

N_DIR, N_CELL = 48, 37


def test_direction_ranges_cover_every_direction_once():
    for n_dir in (1, 2, 12, 47, 48):
        for world in range(1, n_dir + 1):
            seen = np.zeros(n_dir, int)
            prev_end = 0
            for r in range(world):
                b, e = shard.direction_range(n_dir, r, world)
                assert b == prev_end and e > b
                assert e - b in (n_dir // world, n_dir // world + 1)
                seen[b:e] += 1
                prev_end = e
            assert prev_end == n_dir and (seen == 1).all()
    with pytest.raises(ValueError):
        shard.direction_range(4, 0, 5)
    with pytest.raises(ValueError):
        shard.direction_range(8, 2, 2)


class _StandIn:
    """Per-direction contributions d -> 4 arrays (float32 like the library's
    {SIJ, ESC}, compensation, NORM, compensation), seeded; iteration k adds
    k to every contribution so each iteration's sums differ."""

    def __init__(self):
        import torch
        rng = np.random.default_rng(7)
        self.contrib = [rng.random((N_DIR, 2 * N_CELL)), rng.random((N_DIR, 2 * N_CELL)) * 1e-7,
                        rng.random((N_DIR, N_CELL)), rng.random((N_DIR, N_CELL)) * 1e-7]
        self.bufs = [torch.zeros(c.shape[1], dtype=torch.float64) for c in self.contrib]
        self.it = 0
        self.seen = []

    def n_dir(self):
        return N_DIR

    def march(self, dir_range, **opts):
        b, e = dir_range
        for buf, c in zip(self.bufs, self.contrib):
            buf.copy_(__import__("torch").from_numpy((c[b:e] + self.it).sum(axis=0)))

    def solve(self, **opts):
        self.seen.append([buf.numpy().copy() for buf in self.bufs])
        self.it += 1
        return {"iterations": 1}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = _StandIn()
        reps = shard.iterate_sharded(m, 3, rank, world, tensors=lambda model, prec: model.bufs,
                                     precision="fp32")
        assert len(reps) == 3
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump([[a.tolist() for a in s] for s in m.seen], f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_to_the_single_device_accumulators(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    ref = _StandIn()
    for k in range(3):
        ref.march((0, N_DIR))
        ref.solve()
    for r in range(world):
        seen = json.load(open(tmp_path / f"r{r}.json"))
        assert len(seen) == 3
        for k in range(3):
            for a, b in zip(seen[k], ref.seen[k]):
                np.testing.assert_allclose(np.array(a), b, rtol=1e-12)
