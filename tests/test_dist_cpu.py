"""Multi-rank host logic on CPU: two gloo ranks (world size 2)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2507_09772_gb300 import dist as jdist
from paper_2507_09772_gb300 import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, units = jdist.reduce_step_timing(dist, 10.0 + rank, 100.0 * (rank + 1))
        # partial J from each rank: rank r owns rows r::world of a symmetric matrix
        rng = np.random.default_rng(0)
        full = rng.standard_normal((6, 6))
        full = full + full.T
        part = np.zeros_like(full)
        part[rank::world] = full[rank::world]
        t = torch.tensor(part)
        jdist.sum_partials(dist, [t, None])
        opts = jdist.partition_options(rank, world)
        q.put((rank, ms, units, float(np.abs(t.numpy() - full).max()), opts,
               jdist.batch_seed_base(rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_work_and_partials():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, ms, units, err, opts, seed in out:
        assert ms == 11.0                       # max over ranks
        assert units == 300.0                   # sum over ranks
        assert err == 0.0                       # partials summed to the full matrix
        assert opts == {"part_count": 2, "part_index": rank}
    assert out[0][5] != out[1][5]               # each rank builds its own batch


def test_rank_batches_differ():
    a = synth.batched_molecule(0, seed_base=jdist.batch_seed_base(0))
    b = synth.batched_molecule(0, seed_base=jdist.batch_seed_base(1))
    assert not np.array_equal(a.coords[:3], b.coords[:3])
