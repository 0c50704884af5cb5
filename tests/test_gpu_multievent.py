"""Several independent events sampled in one handle (one walk grid over all their walkers,
uneven bin counts, live counts and walk lengths): every event follows its own oracle run."""
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


def small_events(precision):
    ws = synth.batched_workloads(8, seed=7, precision=precision)
    picks = [ws[0], ws[1], ws[2], ws[5]]
    out = []
    for i, w in enumerate(picks):
        n_live = (30, 44, 36, 50)[i]
        w = replace(w, f_max=w.f_min + 40.0, n_live=n_live, num_delete=n_live // 2, naccept=6, maxmcmc=200)
        ev = synth.make_event(w, lambda e, d, th, ww=w: L.project(e, d, th, ww.waveform), L.inner)
        out.append((w, ev))
    return out


def test_events_in_one_handle_follow_their_oracle_runs():
    evs = small_events(synth.PREC_FP64)
    assert len({ev.n_bins for _, ev in evs}) >= 2
    batches = 3
    cfgs = [gwns.make_config(w, synth.priors_with_injection(w, ev), max_iter=batches) for w, ev in evs]
    h = gwns.ns_init(cfgs, [ev for _, ev in evs])
    try:
        code, prog = gwns.ns_step(h, batches + 2, n_events=len(evs))
        for e, (w, ev) in enumerate(evs):
            pri = synth.priors_with_injection(w, ev)
            ll = lambda u, ev=ev, pri=pri, w=w: L.log_likelihood(ev, P.transform(u, pri), w.waveform)
            ref = nested.run_nested(ll, w.n_dim, w.n_live, w.num_delete, w.naccept, w.maxmcmc,
                                    P.periodic_mask(pri), (w.seed, e), max_iter=batches, n_replay=2)
            assert prog[e]["iterations"] == batches and prog[e]["done"] == 1
            assert prog[e]["n_like"] == ref.n_like
            assert abs(prog[e]["log_z"] - np.logaddexp.reduce(ref.dead_logw)) < 1e-9
            th, lw = gwns.ns_posterior(h, e)
            dead = np.stack([P.transform(u, pri) for u in ref.dead_u])
            assert np.allclose(th[:dead.shape[0]], dead, rtol=1e-12, atol=1e-12)
    finally:
        gwns.ns_free(h)


def test_mixed_precision_events_run_to_termination():
    evs = small_events(synth.PREC_MIXED_FF)
    cfgs = [gwns.make_config(w, synth.priors_with_injection(w, ev), max_iter=60) for w, ev in evs]
    h = gwns.ns_init(cfgs, [ev for _, ev in evs])
    try:
        code, prog = gwns.ns_step(h, 60, n_events=len(evs))
        for e, p in enumerate(prog):
            assert p["done"] == 1 and np.isfinite(p["log_z"])
            lz, err, info, n_like = gwns.ns_evidence(h, e)
            assert np.isfinite(lz) and err > 0 and info > 0 and n_like == p["n_like"]
    finally:
        gwns.ns_free(h)


def test_speculation_autotuner_choice_and_chain():
    # The speculation-depth autotuner (automatic depth): after the first batch the cap follows
    # the cost structure (FP64, short likelihoods of < 1k active bins: 8); from iteration 64 a
    # tuning pass tries every FP64 candidate cap {1, 2, 4, 8} in mirrored order and keeps one of
    # them; the depth in force never exceeds the cap.  Any depth gives the chain of the one-step
    # walk, so the tuned run equals a run at a fixed depth bit for bit.
    evs = small_events(synth.PREC_FP64)
    iters = 80
    def run(spec):
        cfgs = [replace_cfg(gwns.make_config(w, synth.priors_with_injection(w, ev), max_iter=iters, spec_depth=spec))
                for w, ev in evs]
        h = gwns.ns_init(cfgs, [ev for _, ev in evs])
        caps, depths = [], []
        try:
            for b in range(iters):
                _, prog = gwns.ns_step(h, 1, n_events=len(evs))
                caps.append(prog[0]["spec_cap"])
                depths.append([p["spec_depth"] for p in prog])
            post = [gwns.ns_posterior(h, e) for e in range(len(evs))]
        finally:
            gwns.ns_free(h)
        return prog, caps, depths, post

    prog_a, caps, depths, post_a = run(0)
    prog_f, _, _, post_f = run(3)
    assert caps[1] == 8                                   # the cost-structure guess after batch 1
    assert all(c in (1, 2, 4, 8) for c in caps[1:])
    assert caps[-1] in (1, 2, 4, 8)
    assert caps[64:72] == [1, 2, 4, 8, 8, 4, 2, 1]       # the tuning pass, one batch a candidate
    assert len(set(caps[72:])) == 1                       # then its choice, kept
    for c, ds in zip(caps[1:], depths[1:]):
        assert all(1 <= d <= c for d in ds)
    for e in range(len(evs)):
        assert prog_a[e]["iterations"] == prog_f[e]["iterations"] == iters
        assert prog_a[e]["n_like"] == prog_f[e]["n_like"]
        assert prog_a[e]["log_z"] == prog_f[e]["log_z"]
        assert np.array_equal(post_a[e][0], post_f[e][0]) and np.array_equal(post_a[e][1], post_f[e][1])


@pytest.mark.parametrize("precision", [synth.PREC_FP64, synth.PREC_MIXED, synth.PREC_MIXED_FF])
def test_chain_does_not_depend_on_the_speculation_depth(precision):
    # A proposal's ln L is summed in one order whether its round ran it on one warp (rounds of
    # four proposals or more) or on the whole CTA, so every depth runs the chain of the one-step
    # walk bit for bit, to the end of a run of 80 batches.  The live sets hold copies of points
    # (walkers that never moved); a DE difference of two copies proposes the current point again,
    # and its ln L must equal its copy's for the tie to break the same way at every depth.
    evs = small_events(precision)
    iters = 80
    def run(spec):
        cfgs = [replace_cfg(gwns.make_config(w, synth.priors_with_injection(w, ev), max_iter=iters, spec_depth=spec))
                for w, ev in evs]
        h = gwns.ns_init(cfgs, [ev for _, ev in evs])
        try:
            _, prog = gwns.ns_step(h, iters, n_events=len(evs))
            return prog, [gwns.ns_posterior(h, e) for e in range(len(evs))]
        finally:
            gwns.ns_free(h)

    prog1, post1 = run(1)
    for spec in (3, 8, 13):
        prog, post = run(spec)
        for e in range(len(evs)):
            assert prog[e]["iterations"] == iters and prog[e]["n_like"] == prog1[e]["n_like"]
            assert prog[e]["log_z"] == prog1[e]["log_z"], (spec, e)
            assert np.array_equal(post[e][0], post1[e][0]) and np.array_equal(post[e][1], post1[e][1]), (spec, e)


def replace_cfg(c):
    # run every event to the batch cap: a stopping threshold nothing reaches.  The remaining-
    # fraction rule compares ln(L_max X_live / Z) with ln(threshold) directly; the Delta ln Z rule
    # would not do (ln Z + the live term rounds to ln Z once that term is below half an ulp of
    # ln Z, ~1e-13 here, and then meets any positive threshold)
    c.term_kind = synth.TERM_FRAC_REMAINING
    c.term_value = 1e-300
    return c
