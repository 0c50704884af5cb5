"""CUDA hit-and-run slice sampling vs the oracle (oracle/hrss.py) on the same Philox streams:
ns_hrss_batch in FP64 (move and likelihood-call counts bit-exact, positions to rounding) and in
the mixed precisions (the same, for walkers whose decisions all lie farther from ln L* than the
mixed likelihood's tolerance), and the sampler with HRSS as its inner kernel (ns_step with
NS_PROPOSAL_HRSS) against the oracle sampler's own HRSS run."""
import math

import numpy as np
import pytest

from oracle import hrss, prior as P
from paper_2509_04336_gb300 import gwns, synth

from _util import event, priors
from test_gpu_walk import walk_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2509_04336_gb300 import build
    build.build()


@pytest.mark.parametrize("name", ["four_param_2det_taylorf2", "bbh11_3det_4s_taylorf2"])
def test_hrss_chain_matches_oracle(name):
    w, ev = event(name)
    ll, surv, u0, l0, lnl_star = walk_inputs(w, ev, 60, 16, 5)
    n_steps, it, off = 4, 2, 9
    periodic = P.periodic_mask(priors(w, ev))
    ou, ol, om, on = hrss.hrss_walk(ll, u0, l0, lnl_star, surv, n_steps, periodic, (w.seed, 0), it,
                                    walker_ids=np.arange(16) + off)
    h = gwns.ns_init([gwns.make_config(w, priors(w, ev), precision=synth.PREC_FP64)], [ev])
    try:
        gu, gl, gm, gn = gwns.ns_hrss_batch(h, 0, surv, u0, l0, lnl_star, n_steps, it, off)
    finally:
        gwns.ns_free(h)
    assert np.array_equal(gm, om) and np.array_equal(gn, on)
    assert np.allclose(gu, ou, rtol=0, atol=1e-12)
    assert np.all(np.abs(gl - ol) <= 1e-11 * np.maximum(np.abs(ol), 1.0))
    assert np.all(gl > lnl_star) and np.all((gu >= 0) & (gu <= 1))
    assert np.all(gm == n_steps)


@pytest.mark.parametrize("precision", [synth.PREC_MIXED, synth.PREC_MIXED_FF])
def test_hrss_chain_mixed_precision(precision):
    # the mixed likelihoods are within 1e-6 of |ln L|; a walker whose every decision lies
    # farther than that from ln L* follows the oracle's chain exactly
    w, ev = event("bbh11_3det_4s_taylorf2")
    ll, surv, u0, l0, lnl_star = walk_inputs(w, ev, 60, 24, 7)
    n_steps, it, off = 3, 4, 0
    periodic = P.periodic_mask(priors(w, ev))
    ou, ol, om, on, margin = hrss.hrss_walk(ll, u0, l0, lnl_star, surv, n_steps, periodic, (w.seed, 0), it,
                                            walker_ids=np.arange(24) + off, return_margin=True)
    h = gwns.ns_init([gwns.make_config(w, priors(w, ev), precision=precision)], [ev])
    try:
        gu, gl, gm, gn = gwns.ns_hrss_batch(h, 0, surv, u0, l0, lnl_star, n_steps, it, off)
    finally:
        gwns.ns_free(h)
    same = margin > 4e-6 * max(abs(lnl_star), 1.0)
    assert same.sum() >= 20
    assert np.array_equal(gm[same], om[same]) and np.array_equal(gn[same], on[same])
    assert np.allclose(gu[same], ou[same], rtol=0, atol=1e-12)
    assert np.all(np.abs(gl[same] - ol[same]) <= 1e-6 * np.abs(ol[same]))
    assert np.all(gl > lnl_star)


@pytest.mark.parametrize("name", ["bbh11_3det_4s_taylorf2", "bbh11_3det_8s_phenomd"])
def test_hrss_float_float_rounds_give_the_same_chain(name):
    # the float-float HRSS kernel evaluates up to spec candidates of a move per round and replays
    # the sequential move over them: any round size gives the same chain, bit for bit (the calls
    # after the replay's stopping point are speculative and not counted)
    w, ev = event(name)
    ll, surv, u0, l0, lnl_star = walk_inputs(w, ev, 60, 10, 8)
    outs = []
    for spec in (1, 2, 5, 16):
        h = gwns.ns_init([gwns.make_config(w, priors(w, ev), precision=synth.PREC_MIXED_FF, spec_depth=spec)], [ev])
        try:
            outs.append(gwns.ns_hrss_batch(h, 0, surv, u0, l0, lnl_star, 3, 6, 2))
        finally:
            gwns.ns_free(h)
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)
    gu, gl, gm, gn = outs[0]
    assert np.all(gl > lnl_star) and np.all(gm > 0) and np.all(gn >= gm)


def tiny_hrss():
    """The 4-parameter zero-noise event at 20-64 Hz (177 bins), 30 live points, k = 15."""
    from dataclasses import replace
    from oracle import likelihood as L
    w = synth.shrink(synth.workload("four_param_2det_taylorf2"), f_max=64.0, n_live=30, naccept=8)
    w = replace(w, maxmcmc=400)
    ev = synth.make_event(w, lambda e, i, th: L.project(e, i, th, w.waveform), L.inner)
    pri = synth.priors_with_injection(w, ev)
    ll = lambda u: L.log_likelihood(ev, P.transform(u, pri), w.waveform, w.use_ratio)
    return w, ev, pri, ll


def test_sampler_with_hrss_matches_oracle():
    # ns_step with HRSS as the inner kernel: survivors' Cholesky factor on the device, 3 moves a
    # walker and batch, 10 batches through the batch graph, against the oracle sampler's
    # run_nested(inner="hrss") on the same seed: every dead point, the likelihood-call count
    # and the evidence agree
    from oracle import nested
    w, ev, pri, ll = tiny_hrss()
    iters, moves = 10, 3
    ref = nested.run_nested(ll, w.n_dim, w.n_live, w.num_delete, w.naccept, w.maxmcmc, P.periodic_mask(pri),
                            (w.seed, 0), term_kind=w.term_kind, term_value=w.term_value, n_replay=2,
                            max_iter=iters, inner="hrss", hrss_steps=moves)
    h = gwns.ns_init([gwns.make_config(w, pri, precision=synth.PREC_FP64, max_iter=iters, hrss_moves=moves)], [ev])
    try:
        code, prog = gwns.ns_step(h, iters)
        th, lw = gwns.ns_posterior(h, 0)
    finally:
        gwns.ns_free(h)
    p = prog[0]
    assert p["iterations"] == ref.n_iter == iters
    assert p["n_like"] == ref.n_like
    assert p["n_steps"] == moves
    nd = ref.dead_u.shape[0]
    dead = np.stack([P.transform(u, pri) for u in ref.dead_u])
    assert np.allclose(th[:nd], dead, rtol=1e-12, atol=1e-12)
    assert abs(p["log_z"] - np.logaddexp.reduce(ref.dead_logw)) < 1e-9 * max(1.0, abs(p["log_z"]))
    assert abs(p["mean_accept"] - ref.stats[-1][2]) < 1e-12


def test_sampler_hrss_float_float_evidence():
    # the float-float HRSS sampler to termination: ln Z within the runs' errors of the oracle's
    # FP64 HRSS run on the same seed
    from oracle import nested
    w, ev, pri, ll = tiny_hrss()
    ref = nested.run_nested(ll, w.n_dim, w.n_live, w.num_delete, w.naccept, w.maxmcmc, P.periodic_mask(pri),
                            (w.seed, 0), term_kind=w.term_kind, term_value=w.term_value, n_replay=50,
                            inner="hrss", hrss_steps=8)
    h = gwns.ns_init([gwns.make_config(w, pri, precision=synth.PREC_MIXED_FF, hrss_moves=8)], [ev])
    try:
        done = False
        for _ in range(50):
            _, prog = gwns.ns_step(h, 8)
            if prog[0]["done"]:
                done = True
                break
        lz, lz_err, info, n_like = gwns.ns_evidence(h, 0)
    finally:
        gwns.ns_free(h)
    assert done
    assert abs(lz - ref.log_z) < 3.0 * math.hypot(lz_err, ref.log_z_err) + 1e-9


def test_hrss_errors():
    w, ev = event("four_param_2det_taylorf2")
    ll, surv, u0, l0, lnl_star = walk_inputs(w, ev, 20, 2, 6)
    h = gwns.ns_init([gwns.make_config(w, priors(w, ev), precision=synth.PREC_FP64)], [ev])
    try:
        # two survivors span one direction: the covariance is singular
        with pytest.raises(gwns.GwnsError) as e:
            gwns.ns_hrss_batch(h, 0, surv[:2], u0, l0, lnl_star, 1)
        assert e.value.code == gwns.NS_EINVAL
        gu, gl, gm, gn = gwns.ns_hrss_batch(h, 0, surv, u0, l0, lnl_star, 0)
        assert np.array_equal(gu, u0) and np.array_equal(gl, l0) and np.all(gm == 0) and np.all(gn == 0)
    finally:
        gwns.ns_free(h)
    # HRSS in the sampler needs more survivors than dimensions; all events or none
    from dataclasses import replace
    w2 = replace(synth.shrink(w, n_live=8), num_delete=4)
    with pytest.raises(gwns.GwnsError) as e:
        gwns.ns_init([gwns.make_config(w2, priors(w2, ev), hrss_moves=2)], [ev])
    assert e.value.code == gwns.NS_EINVAL
    with pytest.raises(gwns.GwnsError) as e:
        gwns.ns_init([gwns.make_config(w, priors(w, ev), hrss_moves=2), gwns.make_config(w, priors(w, ev))], [ev, ev])
    assert e.value.code == gwns.NS_EINVAL
