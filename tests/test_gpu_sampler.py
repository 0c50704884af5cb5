"""The sampler driven end to end against the oracle: the sequential case k = 1, both stopping
rules to termination, the posterior export and checkpoint / resume.

All runs are FP64 on identical Philox streams, so iteration counts, likelihood-call counts
and every dead point agree with the oracle's own run; a resumed run replays the run that was
never interrupted bit for bit (flow proposal included)."""
import math
import os
from dataclasses import replace

import numpy as np
import pytest

from oracle import likelihood as L, nested, prior as P
from paper_2509_04336_gb300 import gwns, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2509_04336_gb300 import build
    build.build()


def tiny(num_delete=None, **kw):
    """The 4-parameter zero-noise event at 20-64 Hz (177 bins), 30 live points, naccept 8."""
    w = synth.shrink(synth.workload("four_param_2det_taylorf2"), f_max=64.0, n_live=30,
                     num_delete=num_delete, naccept=8)
    w = replace(w, maxmcmc=400, **kw)
    ev = synth.make_event(w, lambda e, i, th: L.project(e, i, th, w.waveform), L.inner)
    pri = synth.priors_with_injection(w, ev)
    ll = lambda u: L.log_likelihood(ev, P.transform(u, pri), w.waveform, w.use_ratio)
    return w, ev, pri, ll


def oracle_run(w, pri, ll, **kw):
    return nested.run_nested(ll, w.n_dim, w.n_live, w.num_delete, w.naccept, w.maxmcmc,
                             P.periodic_mask(pri), (w.seed, 0), term_kind=w.term_kind,
                             term_value=w.term_value, n_replay=2, **kw)


def test_sequential_mode_matches_oracle():
    # k = 1: one deletion and one single-walker walk per iteration (the classical sampler,
    # Sec. 2), 60 iterations through the batch graph.
    w, ev, pri, ll = tiny(num_delete=1)
    iters = 60
    ref = oracle_run(w, pri, ll, max_iter=iters)
    h = gwns.ns_init([gwns.make_config(w, pri, precision=synth.PREC_FP64, max_iter=iters)], [ev])
    try:
        code, prog = gwns.ns_step(h, iters)
        th, lw = gwns.ns_posterior(h, 0)
    finally:
        gwns.ns_free(h)
    p = prog[0]
    assert p["iterations"] == iters and p["done"] == 1
    assert p["n_like"] == ref.n_like
    assert ref.dead_u.shape[0] == iters
    dead = np.stack([P.transform(u, pri) for u in ref.dead_u])
    assert np.allclose(th[:iters], dead, rtol=1e-12, atol=1e-12)
    assert abs(p["log_z"] - np.logaddexp.reduce(ref.dead_logw)) < 1e-9
    # the walk length followed the same retuning sequence (Eq. 16 with k = 1)
    assert p["n_steps"] == nested.retune(ref.stats[-1][1], ref.stats[-1][2], w.naccept,
                                         nested.batch_delay(w.naccept - 1, 1), w.maxmcmc)


def test_largest_live_set_matches_oracle():
    # n_live at its limit (4096, sorted by one CTA in shared memory) with k = 2048 walkers: two
    # whole batches against the oracle's run -- the deleted points in order, the likelihood calls
    # and the evidence (naccept 2 keeps the oracle's ~36k calls to seconds).
    w, ev, pri, ll = tiny()
    w = replace(w, n_live=4096, num_delete=2048, naccept=2)
    iters = 2
    ref = oracle_run(w, pri, ll, max_iter=iters)
    h = gwns.ns_init([gwns.make_config(w, pri, precision=synth.PREC_FP64, max_iter=iters)], [ev])
    try:
        code, prog = gwns.ns_step(h, iters)
        th, lw = gwns.ns_posterior(h, 0)
    finally:
        gwns.ns_free(h)
    p = prog[0]
    nd = iters * w.num_delete
    assert p["iterations"] == iters and p["n_like"] == ref.n_like
    assert ref.dead_u.shape[0] == nd and th.shape[0] == nd + w.n_live
    dead = np.stack([P.transform(u, pri) for u in ref.dead_u])
    assert np.allclose(th[:nd], dead, rtol=1e-12, atol=1e-12)
    assert abs(p["log_z"] - np.logaddexp.reduce(ref.dead_logw)) < 1e-9


def test_batches_with_likelihood_ratio_match_oracle():
    # use_ratio (Sec. 4.1.1): the sampler runs on ln Lambda = ln L + <d|d>/2; eight batches
    # follow the oracle's own run (same deletions, walks and evidence, which differs from the
    # ln L run's by the constant <d|d>/2).
    w, ev, pri, ll = tiny(use_ratio=True)
    iters = 8
    ref = oracle_run(w, pri, ll, max_iter=iters)
    h = gwns.ns_init([gwns.make_config(w, pri, precision=synth.PREC_FP64, max_iter=iters)], [ev])
    try:
        code, prog = gwns.ns_step(h, iters)
        th, lw = gwns.ns_posterior(h, 0)
    finally:
        gwns.ns_free(h)
    p = prog[0]
    assert p["iterations"] == iters and p["n_like"] == ref.n_like
    nd = ref.dead_u.shape[0]
    dead = np.stack([P.transform(u, pri) for u in ref.dead_u])
    assert np.allclose(th[:nd], dead, rtol=1e-12, atol=1e-12)
    assert abs(p["log_z"] - np.logaddexp.reduce(ref.dead_logw)) < 1e-9 * max(1.0, abs(p["log_z"]))


@pytest.mark.parametrize("term_kind,term_value", [(synth.TERM_FRAC_REMAINING, 0.05),
                                                  (synth.TERM_DLOGZ, 0.3)])
def test_run_to_termination_matches_oracle(term_kind, term_value):
    # Both stopping rules stop at the oracle's iteration; the evidence with the final live
    # points, the information and the posterior export (dead then live, normalised
    # weights, Eq. 1) agree.
    w, ev, pri, ll = tiny(term_kind=term_kind, term_value=term_value)
    ref = oracle_run(w, pri, ll)
    n_it = ref.n_iter
    h = gwns.ns_init([gwns.make_config(w, pri, precision=synth.PREC_FP64)], [ev])
    try:
        code, prog = gwns.ns_step(h, 4 * n_it)
        lz, lz_err, info, n_like = gwns.ns_evidence(h, 0)
        th, lw = gwns.ns_posterior(h, 0)
    finally:
        gwns.ns_free(h)
    p = prog[0]
    assert p["done"] == 1 and p["iterations"] == n_it
    assert n_like == ref.n_like
    assert abs(lz - ref.log_z) < 1e-9
    assert abs(info - ref.info_h) < 1e-8
    assert lz_err > 0
    n_dead = ref.dead_u.shape[0]
    assert th.shape[0] == n_dead + w.n_live
    dead = np.stack([P.transform(u, pri) for u in ref.dead_u])
    assert np.allclose(th[:n_dead], dead, rtol=1e-12, atol=1e-12)
    assert np.allclose(lw[:n_dead], ref.dead_logw - ref.log_z, rtol=0, atol=1e-9)
    # the final live points, in any slot order
    live = np.stack([P.transform(u, pri) for u in ref.live_u])
    lw_live = ref.live_lnl + ref.log_x - math.log(w.n_live) - ref.log_z
    o_ref, o_gpu = np.argsort(lw_live), np.argsort(lw[n_dead:])
    assert np.allclose(lw[n_dead:][o_gpu], lw_live[o_ref], rtol=0, atol=1e-9)
    assert np.allclose(th[n_dead:][o_gpu], live[o_ref], rtol=1e-12, atol=1e-12)
    assert abs(np.logaddexp.reduce(lw)) < 1e-12


@pytest.mark.parametrize("flow", [False, True])
def test_resume_replays_the_uninterrupted_run(tmp_path, flow):
    # Save after 3 batches, load into a fresh handle, run 3 more: the same dead points,
    # evidence, call counts, walk length and flow parameters as 6 batches in one go.
    w, ev, pri, ll = tiny()
    kw = dict(p_flow=0.5, flow_layers=2, flow_epochs=4) if flow else {}
    prec = synth.PREC_MIXED_FF if flow else synth.PREC_FP64
    cfg = lambda: gwns.make_config(w, pri, precision=prec, max_iter=6, **kw)
    path = os.path.join(tmp_path, "state.bin")

    def finish(h):
        code, prog = gwns.ns_step(h, 3)
        th, lw = gwns.ns_posterior(h, 0)
        out = dict(prog=prog[0], th=th, lw=lw, ev=gwns.ns_evidence(h, 0))
        if flow:
            out["flow"] = gwns.ns_flow_get(h, 0, w.n_dim)
        return out

    h = gwns.ns_init([cfg()], [ev])
    try:
        gwns.ns_step(h, 3)
        gwns.ns_state_save(h, path)
        straight = finish(h)
    finally:
        gwns.ns_free(h)
    h = gwns.ns_init([cfg()], [ev])
    try:
        gwns.ns_step(h, 1)          # a different history, overwritten by the load
        gwns.ns_state_load(h, path)
        resumed = finish(h)
    finally:
        gwns.ns_free(h)
    a, b = straight["prog"], resumed["prog"]
    for key in ("iterations", "done", "n_like", "n_steps", "log_z"):
        assert a[key] == b[key], key
    assert a["iterations"] == 6
    assert np.array_equal(straight["th"], resumed["th"])
    assert np.array_equal(straight["lw"], resumed["lw"])
    assert straight["ev"][0] == resumed["ev"][0] and straight["ev"][3] == resumed["ev"][3]
    if flow:
        for x, y in zip(straight["flow"], resumed["flow"]):
            assert np.array_equal(x, y)


def test_truncated_state_leaves_the_handle_untouched(tmp_path):
    # A checkpoint is read and checked in full before anything is applied.
    w, ev, pri, ll = tiny()
    path = os.path.join(tmp_path, "state.bin")
    cut = os.path.join(tmp_path, "cut.bin")
    cfg = lambda: gwns.make_config(w, pri, precision=synth.PREC_FP64, max_iter=6)
    h = gwns.ns_init([cfg()], [ev])
    try:
        gwns.ns_step(h, 3)
        gwns.ns_state_save(h, path)
    finally:
        gwns.ns_free(h)
    with open(path, "rb") as fh:
        blob = fh.read()
    with open(cut, "wb") as fh:
        fh.write(blob[: len(blob) - 100])
    h = gwns.ns_init([cfg()], [ev])
    try:
        _, before = gwns.ns_step(h, 1)
        th0, lw0 = gwns.ns_posterior(h, 0)
        with pytest.raises(gwns.GwnsError) as e:
            gwns.ns_state_load(h, cut)
        assert e.value.code == gwns.NS_EIO
        th1, lw1 = gwns.ns_posterior(h, 0)
        assert np.array_equal(th0, th1) and np.array_equal(lw0, lw1)
        _, after = gwns.ns_step(h, 1)
        assert after[0]["iterations"] == before[0]["iterations"] + 1
    finally:
        gwns.ns_free(h)


def test_state_load_rejects_a_mismatched_handle(tmp_path):
    w, ev, pri, ll = tiny()
    path = os.path.join(tmp_path, "state.bin")
    h = gwns.ns_init([gwns.make_config(w, pri, precision=synth.PREC_FP64, max_iter=2)], [ev])
    try:
        gwns.ns_step(h, 1)
        gwns.ns_state_save(h, path)
    finally:
        gwns.ns_free(h)
    w2 = replace(w, n_live=32, num_delete=16)
    h = gwns.ns_init([gwns.make_config(w2, pri, precision=synth.PREC_FP64, max_iter=2)], [ev])
    try:
        with pytest.raises(gwns.GwnsError) as e:
            gwns.ns_state_load(h, path)
        assert e.value.code == gwns.NS_EIO
        with pytest.raises(gwns.GwnsError):
            gwns.ns_state_load(h, os.path.join(tmp_path, "missing.bin"))
        # the handle still runs after the failed loads
        code, prog = gwns.ns_step(h, 1)
        assert prog[0]["iterations"] == 1
    finally:
        gwns.ns_free(h)
