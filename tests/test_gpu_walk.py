"""CUDA acceptance walk and batched nested sampling vs the oracle on the same Philox streams.

FP64 path: trajectories are compared exactly (positions to rounding, integer counts
bit-exact).  Mixed path: a walker whose oracle trajectory met a proposal with
|ln L' - ln L*| below the mixed tolerance may legitimately take the other branch; such
walkers are excluded from the exact comparison and only checked for validity."""
import math

import numpy as np
import pytest

from oracle import likelihood as L, nested, prior as P, walk
from paper_2509_04336_gb300 import gwns, synth

from _util import event, priors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2509_04336_gb300 import build
    build.build()


def oracle_loglike(w, ev):
    pri = priors(w, ev)
    return lambda u: L.log_likelihood(ev, P.transform(u, pri), w.waveform, w.use_ratio)


def walk_inputs(w, ev, n_surv, n_walk, seed):
    ll = oracle_loglike(w, ev)
    rng = np.random.default_rng(seed)
    surv = rng.random((n_surv, w.n_dim))
    lnl_s = np.array([ll(x) for x in surv])
    lnl_star = float(np.quantile(lnl_s, 0.3))
    ok = np.where(lnl_s > lnl_star)[0]
    starts = ok[rng.integers(0, ok.shape[0], n_walk)]
    return ll, surv, np.ascontiguousarray(surv[starts]), np.ascontiguousarray(lnl_s[starts]), lnl_star


@pytest.mark.parametrize("name,precision,spec", [
    ("four_param_2det_taylorf2", synth.PREC_FP64, 1),
    ("four_param_2det_taylorf2", synth.PREC_FP64, 3),
    ("bbh11_3det_4s_taylorf2", synth.PREC_FP64, 8),
    ("bbh11_3det_4s_taylorf2", synth.PREC_MIXED, 32),
    ("bbh11_3det_4s_taylorf2", synth.PREC_MIXED_FF, 2),
    ("bbh11_3det_4s_taylorf2", synth.PREC_MIXED_FF, 3),    # padded to 4: one proposal per warp
    ("bbh11_3det_4s_taylorf2", synth.PREC_MIXED_FF, 5),    # padded to 8
    ("bbh11_3det_4s_taylorf2", synth.PREC_MIXED_FF, 32),
    ("bbh11_3det_8s_phenomd", synth.PREC_FP64, 8),
    ("bbh11_3det_8s_phenomd", synth.PREC_MIXED_FF, 1),
    ("bbh11_3det_8s_phenomd", synth.PREC_MIXED_FF, 2),
    ("bbh11_3det_8s_phenomd", synth.PREC_MIXED_FF, 16),
])
def test_walk_parity(name, precision, spec):
    # Any speculation depth gives the chain of the one-step-at-a-time walk.
    w, ev = event(name, f_max=512.0) if "phenomd" in name else event(name)
    ll, surv, u0, l0, lnl_star = walk_inputs(w, ev, 60, 24, 4)
    n_steps, it, off = 12, 3, 7
    periodic = P.periodic_mask(priors(w, ev))
    key = (w.seed, 0)
    ou, ol, oa, on, margin = walk.acceptance_walk(ll, u0, l0, lnl_star, surv, n_steps, periodic, key, it,
                                                  walker_ids=np.arange(24) + off)
    cfg = gwns.make_config(w, priors(w, ev), precision=precision, spec_depth=spec)
    h = gwns.ns_init([cfg], [ev])
    try:
        gu, gl = np.zeros_like(u0), np.zeros(24)
        ga, gn = np.zeros(24, np.int32), np.zeros(24, np.int32)
        gwns.ns_walk_batch(h, 0, np.ascontiguousarray(surv), u0, l0, lnl_star, n_steps, it, off, gu, gl, ga, gn)
    finally:
        gwns.ns_free(h)
    if precision == synth.PREC_FP64:
        same = np.ones(24, bool)
        tol = 1e-11
    else:
        same = margin > 1e-6 * np.maximum(np.abs(lnl_star), 1.0) * 4
        tol = 1e-6
    assert same.sum() >= 20
    assert np.array_equal(ga[same], oa[same]) and np.array_equal(gn[same], on[same])
    assert np.allclose(gu[same], ou[same], rtol=0, atol=1e-12)
    assert np.all(np.abs(gl[same] - ol[same]) <= tol * np.maximum(np.abs(ol[same]), 1.0))
    # every walker, matched or not, ends inside the constraint and the cube
    assert np.all(gl > lnl_star)
    assert np.all((gu >= 0) & (gu <= 1))


def test_walk_device_pointers_and_zero_steps():
    import torch
    w, ev = event("four_param_2det_taylorf2")
    ll, surv, u0, l0, lnl_star = walk_inputs(w, ev, 30, 8, 2)
    cfg = gwns.make_config(w, priors(w, ev), precision=synth.PREC_FP64)
    h = gwns.ns_init([cfg], [ev])
    try:
        T = lambda a, dt=torch.float64: torch.tensor(a, device="cuda", dtype=dt)
        gu, gl = T(np.zeros_like(u0)), T(np.zeros(8))
        ga, gn = T(np.zeros(8), torch.int32), T(np.zeros(8), torch.int32)
        code = gwns.ns_walk_batch(h, 0, T(surv), T(u0), T(l0), lnl_star, 0, 0, 0, gu, gl, ga, gn)
        torch.cuda.synchronize()
        assert code == gwns.NS_OK
        assert np.array_equal(gu.cpu().numpy(), u0) and np.array_equal(gl.cpu().numpy(), l0)
        assert ga.sum().item() == 0 and gn.sum().item() == 0
    finally:
        gwns.ns_free(h)


@pytest.mark.parametrize("name,spec", [("four_param_2det_taylorf2", 0), ("four_param_2det_taylorf2", 1),
                                       ("four_param_2det_taylorf2", 32), ("bbh11_3det_8s_phenomd", 0)])
def test_batches_match_oracle_fp64(name, spec):
    # The whole batch pipeline (sort, deletion, evidence, starts, walk, insertion, retune)
    # on identical Philox streams: dead points and evidence agree after three batches.
    w, ev = event(name) if "four" in name else event(name, f_max=300.0, n_live=40)
    pri = priors(w, ev)
    ll = oracle_loglike(w, ev)
    batches = 3
    ref = nested.run_nested(ll, w.n_dim, w.n_live, w.num_delete, w.naccept, w.maxmcmc,
                            P.periodic_mask(pri), (w.seed, 0), max_iter=batches, n_replay=2)
    cfg = gwns.make_config(w, pri, precision=synth.PREC_FP64, max_iter=batches, spec_depth=spec)
    h = gwns.ns_init([cfg], [ev])
    try:
        code, prog = gwns.ns_step(h, batches)
        th, lw = gwns.ns_posterior(h, 0)
        lz, err, info, n_like = gwns.ns_evidence(h, 0)
    finally:
        gwns.ns_free(h)
    p = prog[0]
    assert p["iterations"] == batches and p["done"] == 1
    n_dead = ref.dead_lnl.shape[0]
    dead_theta = np.stack([P.transform(u, pri) for u in ref.dead_u])
    assert np.allclose(th[:n_dead], dead_theta, rtol=1e-12, atol=1e-12)
    assert abs(p["log_z"] - np.logaddexp.reduce(ref.dead_logw)) < 1e-9
    assert n_like == ref.n_like
    assert p["n_steps"] == nested.retune(ref.stats[-1][1], ref.stats[-1][2], w.naccept,
                                         nested.batch_delay(w.naccept - 1, w.num_delete), w.maxmcmc)
    assert abs(lz - ref.log_z) < 1e-9


def test_handles_in_sequence_and_step_statistics():
    # A second handle after a first one has run graph-replayed batches and been freed.
    w, ev = event("four_param_2det_taylorf2")
    pri = priors(w, ev)
    for rep in range(2):
        cfg = gwns.make_config(w, pri, precision=synth.PREC_MIXED, max_iter=2)
        h = gwns.ns_init([cfg], [ev])
        try:
            code, prog = gwns.ns_step(h, 2)
            p = prog[0]
            assert p["iterations"] == 2 and p["kernel_launches"] == 6
            assert p["walk_ms"] > 0 and p["n_bins"] > 0
            assert p["n_spec"] >= p["n_like"] - w.n_live and 1 <= p["spec_depth"] <= 32
            assert p["n_bins"] <= (p["n_like"] - w.n_live) * ev.n_bins
        finally:
            gwns.ns_free(h)
