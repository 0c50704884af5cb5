"""Multi-process host logic of the sharded sampler (paper_2509_04336_gb300.shard) on CPU:
two gloo ranks, as torchrun would start them on two GPUs.  Each rank gets its own events
(no overlap of injections or noise seeds) and the measurement reductions are max / sum."""
import os
import socket

import numpy as np
import pytest

from paper_2509_04336_gb300 import shard

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, wsz, local = shard.rank_info()
        ws = shard.rank_population(8, r)
        seeds = torch.tensor([w.seed for w in ws], dtype=torch.int64)
        inj = torch.tensor(np.stack([w.injection for w in ws]), dtype=torch.float64)
        all_seeds = [torch.zeros_like(seeds) for _ in range(wsz)]
        all_inj = [torch.zeros_like(inj) for _ in range(wsz)]
        dist.all_gather(all_seeds, seeds)
        dist.all_gather(all_inj, inj)
        t, work = shard.reduce_max_sum(10.0 * (r + 1), 100.0 + r)
        if r == 0:
            out.put((wsz, local, [s.tolist() for s in all_seeds], [i.numpy() for i in all_inj], t, work))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_events_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    wsz, local, seeds, inj, t, work = q.get(timeout=10)
    assert wsz == 2 and local == 0
    assert seeds[0] == [100 + e for e in range(8)]          # rank 0 keeps the single-GPU population
    assert not set(seeds[0]) & set(seeds[1])                 # no event shared between ranks
    assert not np.any(np.all(np.isclose(inj[0][:, None, :], inj[1][None, :, :]), axis=2))
    assert t == 20.0 and work == 201.0                       # max of times, sum of work


def test_single_process_defaults():
    assert shard.rank_info({}) == (0, 1, 0)
    assert shard.reduce_max_sum(3.0, 4.0) == (3.0, 4.0)
    assert shard.single_event_seed_offset(0) == 0 and shard.batched_base_seed(100, 0) == 100
