"""Two-rank (gloo, CPU) tests of the multi-GPU host logic: beam sharding, the final dose sum
and the max-over-ranks timing. The per-beam deposits are stand-ins with known sums."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2508_04484_gb300 import multigpu as MG


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _beam_dose(i, n=64):
    rng = np.random.default_rng(100 + i)
    return rng.random(n)


def _worker(rank, world, port, n_beams, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = MG.shard_indices(n_beams, rank, world)
        dose = torch.zeros(64, dtype=torch.float64)
        for i in mine:
            dose += torch.from_numpy(_beam_dose(i))
        MG.reduce_dose(dose)
        t = MG.max_over_ranks(1.0 + rank)
        out[rank] = (dose.numpy().copy(), t, mine)
    finally:
        dist.destroy_process_group()


def test_sharding_covers_every_beam_once():
    beams = list(range(11))
    parts = [MG.shard_beams(beams, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == beams
    assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1
    with pytest.raises(ValueError):
        MG.shard_beams(beams, 3, 3)


def test_two_ranks_sum_the_dose_and_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    n_beams = 7
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n_beams, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    total = sum(_beam_dose(i) for i in range(n_beams))
    for r in range(2):
        dose, t, mine = out[r]
        assert np.allclose(dose, total, rtol=0, atol=1e-12)
        assert t == 2.0
    assert sorted(out[0][2] + out[1][2]) == list(range(n_beams))
