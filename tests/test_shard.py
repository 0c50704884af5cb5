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


class _Handle:
    """A stand-in for a library handle in the walker-sharding protocol: per event the walk outputs
    of its k walkers, which ns_batch_walk fills for its range with values fixed by (batch, event,
    walker) -- as the library's are by the walkers' Philox counters -- and ns_batch_end checks."""

    def __init__(self, ks, dims):
        self.ks, self.dims, self.batch, self.open = ks, dims, 0, False
        self.out = None

    def expected(self, ev, j):
        d = self.dims[ev]
        base = 1000.0 * self.batch + 100.0 * ev + j
        return (base + np.arange(d) / 10.0, -base, int(j % 7), int(j % 11 + 1), int(3 * j), int(5 * j))


class _FakeLib:
    """The ns_batch_* calls of the binding, on _Handle (host only)."""

    @staticmethod
    def ns_batch_begin(h):
        assert not h.open
        h.open = True
        h.out = [(np.full((k, d), np.nan), np.full(k, np.nan), np.full(k, -1, np.int32), np.full(k, -1, np.int32),
                  np.full(k, -1, np.int64), np.full(k, -1, np.int64)) for k, d in zip(h.ks, h.dims)]

    @staticmethod
    def ns_batch_walk(h, b, e):
        for ev, k in enumerate(h.ks):
            for j in range(b, min(e, k)):
                for a, v in zip(h.out[ev], h.expected(ev, j)):
                    a[j] = v

    @staticmethod
    def ns_batch_walk_io(h, ev, b, u, lnl, na, nl, nb, ns, write):
        n = lnl.shape[0]
        for a, x in zip(h.out[ev], (u, lnl, na, nl, nb, ns)):
            if write:
                a[b:b + n] = x
            else:
                x[...] = a[b:b + n]

    @staticmethod
    def ns_batch_end(h, n_events):
        for ev, k in enumerate(h.ks):
            for j in range(k):
                for a, v in zip(h.out[ev], h.expected(ev, j)):
                    assert np.all(a[j] == v), (ev, j)
        h.open = False
        h.batch += 1
        return 0, [{"iterations": h.batch}] * n_events


def _shard_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ks, dims = [50, 23, 7], [11, 4, 11]   # uneven events, one with fewer walkers than ranks' share
        h = _Handle(ks, dims)
        for _ in range(3):
            code, prog = shard.sharded_batch(_FakeLib, h, ks, dims, rank, world)
        out.put((rank, code, prog[0]["iterations"]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_walker_sharding_exchange_over_gloo(world):
    # Every rank walks its own range and, after the exchange, holds every walker's outputs in
    # place before the insertion (_FakeLib.ns_batch_end checks each against its fixed value).
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=10) for _ in range(world))
    assert got == [(r, 0, 3) for r in range(world)]


def test_walker_ranges_partition():
    for k in (1, 7, 50, 500, 2000):
        for world in (1, 2, 3, 8):
            rs = shard.walker_ranges(k, world)
            assert rs[0][0] == 0 and rs[-1][1] == k
            assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
            assert max(e - b for b, e in rs) - min(e - b for b, e in rs) <= 1
