"""Walker sharding of one event (the batch in phases: ns_batch_begin / ns_batch_walk /
ns_batch_walk_io / ns_batch_end) on one GPU: ranks emulated by host threads, each with its own
handle of the same events, exchanging the walk outputs through the host between the phases
(no kernel waits on another rank).  Every rank's run equals the unsharded ns_step run bit for bit."""
import threading

import numpy as np
import pytest

from oracle import likelihood as L
from paper_2509_04336_gb300 import gwns, shard, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2509_04336_gb300 import build
    build.build()


class ThreadExchange:
    """The ranks' exchange of shard.sharded_batch among host threads of one process."""

    def __init__(self, world):
        self.world, self.slots = world, [None] * world
        self.barrier = threading.Barrier(world)

    def for_rank(self, rank):
        def exchange(local):
            self.slots[rank] = local
            self.barrier.wait()
            got = list(self.slots)
            self.barrier.wait()
            return got
        return exchange


def _events(name, precision, n_live):
    w = synth.shrink(synth.workload(name), f_max=128.0, n_live=n_live)
    ev = synth.make_event(w, lambda e, d, th: L.project(e, d, th, w.waveform), L.inner)
    # a fixed speculation depth: ns_step's autotuner would otherwise change it (the chain is the
    # same at any depth, the count of speculative evaluations is not)
    return w, ev, gwns.make_config(w, synth.priors_with_injection(w, ev), precision=precision, spec_depth=8)


@pytest.mark.parametrize("name,precision,world", [("four_param_2det_taylorf2", synth.PREC_FP64, 2),
                                                  ("bbh11_3det_4s_taylorf2", synth.PREC_MIXED_FF, 3)])
def test_sharded_batches_equal_ns_step(name, precision, world):
    w, ev, cfg = _events(name, precision, 60)
    batches = 6
    ref = gwns.ns_init([cfg], [ev])
    hs = [gwns.ns_init([cfg], [ev]) for _ in range(world)]
    try:
        _, pref = gwns.ns_step(ref, batches)
        ex = ThreadExchange(world)
        results = [None] * world
        errors = []

        def rank_main(r):
            try:
                for _ in range(batches):
                    results[r] = shard.sharded_batch(gwns, hs[r], [w.num_delete], [w.n_dim], r, world, ex.for_rank(r))
            except Exception as e:   # reported below
                errors.append(e)
                ex.barrier.abort()

        ts = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
        for t in ts:
            t.start()
        for t in ts:
            t.join(300)
        assert not errors, errors
        th_ref, lw_ref = gwns.ns_posterior(ref, 0)
        for r in range(world):
            code, prog = results[r]
            for key in ("iterations", "n_like", "log_z", "log_x", "lnl_star", "n_steps", "n_bins", "n_spec"):
                assert prog[0][key] == pref[0][key], (r, key)
            th, lw = gwns.ns_posterior(hs[r], 0)
            assert np.array_equal(th, th_ref) and np.array_equal(lw, lw_ref)
    finally:
        gwns.ns_free(ref)
        for h in hs:
            gwns.ns_free(h)


def test_batch_phase_order_is_enforced():
    w, ev, cfg = _events("four_param_2det_taylorf2", synth.PREC_FP64, 30)
    h = gwns.ns_init([cfg], [ev])
    try:
        for call in (lambda: gwns.ns_batch_walk(h, 0, 5), lambda: gwns.ns_batch_end(h)):
            with pytest.raises(gwns.GwnsError) as e:
                call()
            assert e.value.code == gwns.NS_ESTATE
        gwns.ns_batch_begin(h)
        with pytest.raises(gwns.GwnsError) as e:
            gwns.ns_step(h, 1)
        assert e.value.code == gwns.NS_ESTATE
        with pytest.raises(gwns.GwnsError) as e:
            gwns.ns_batch_walk_io(h, 0, w.num_delete - 2, np.zeros((4, w.n_dim)), np.zeros(4), np.zeros(4, np.int32),
                                  np.zeros(4, np.int32), np.zeros(4, np.int64), np.zeros(4, np.int64), write=False)
        assert e.value.code == gwns.NS_EINVAL
        gwns.ns_batch_walk(h, 0, w.num_delete)
        code, prog = gwns.ns_batch_end(h)
        assert prog[0]["iterations"] == 1
        gwns.ns_step(h, 1)
    finally:
        gwns.ns_free(h)
