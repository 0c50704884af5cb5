"""Multi-GPU sharding of the sampler: one process per GPU, independent events per rank.

Events are independent inference problems, so every rank samples its own (weak scaling)
and nothing on the data path crosses ranks.  The only collectives are the reductions of a
measurement: the maximum of the per-rank times and the sum of the per-rank work.
"""
from __future__ import annotations

import os

from . import synth


def rank_info(env=None):
    """(rank, world size, local rank) from the torchrun environment (single process: 0, 1, 0)."""
    env = os.environ if env is None else env
    return int(env.get("RANK", 0)), int(env.get("WORLD_SIZE", 1)), int(env.get("LOCAL_RANK", 0))


def single_event_seed_offset(rank: int) -> int:
    """Noise-seed offset of a single-event workload on `rank` (rank 0 keeps the base seed)."""
    return rank


def batched_base_seed(base: int, rank: int) -> int:
    """Base seed of a rank's population of batched events (the populations never overlap:
    event e of rank r has seed base + 1000 r + e, and a population has at most 256 events)."""
    return base + 1000 * rank


def rank_population(n_events: int, rank: int, base: int = 100, **kw) -> list:
    """The batched-event workloads that `rank` samples."""
    return synth.batched_workloads(n_events, seed=batched_base_seed(base, rank), **kw)


def reduce_max_sum(t_ms: float, work: float, device=None):
    """(max over ranks of t_ms, sum over ranks of work) through torch.distributed (any
    backend: pass device="cuda" for NCCL); without an initialised process group, the inputs."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(t_ms), float(work)
    t = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    w = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


# ---------------------------------------------------------------- walker sharding of one event
def walker_ranges(k: int, world: int) -> list:
    """Contiguous walker ranges [begin, end) of the ranks: k walkers split as evenly as possible."""
    return [(k * r // world, k * (r + 1) // world) for r in range(world)]


def dist_exchange(local):
    """All ranks' copies of `local` (a tuple of numpy arrays), in rank order, through
    torch.distributed (any backend)."""
    import torch.distributed as dist
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, local)
    return out


def sharded_batch(lib, h, ks, dims, rank: int, world: int, exchange=dist_exchange):
    """One sampler batch with its walkers spread over `world` processes that hold identical
    handles: every rank runs the deletion (ns_batch_begin) and the insertion (ns_batch_end)
    itself, walks its own walker range of every event, and the ranks exchange the walk outputs
    (k x (D + 1) doubles and four counters per walker) in between.  ks, dims: num_delete and the
    sampled dimension of each event; lib: the binding (ns_batch_* calls).  Returns ns_batch_end's
    (code, progress)."""
    import numpy as np
    lib.ns_batch_begin(h)
    kmax = max(ks)
    b, e = walker_ranges(kmax, world)[rank]
    lib.ns_batch_walk(h, b, e)
    for ev, (k, d) in enumerate(zip(ks, dims)):
        ranges = [(min(rb, k), min(re_, k)) for rb, re_ in walker_ranges(kmax, world)]
        lb, le = ranges[rank]
        n = le - lb
        local = (np.zeros((n, d)), np.zeros(n), np.zeros(n, np.int32), np.zeros(n, np.int32),
                 np.zeros(n, np.int64), np.zeros(n, np.int64))
        if n > 0:
            lib.ns_batch_walk_io(h, ev, lb, *local, write=False)
        parts = exchange(local)
        for r, (rb, re_) in enumerate(ranges):
            if r != rank and re_ > rb:
                lib.ns_batch_walk_io(h, ev, rb, *[np.ascontiguousarray(a) for a in parts[r]], write=True)
    return lib.ns_batch_end(h, len(ks))
