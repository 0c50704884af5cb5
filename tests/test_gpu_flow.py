"""The flow proposal on the GPU (tensor-core forward, inverse and gradient kernels, the
flow steps of the walk, training inside the sampler) against the oracle's flow.

Tolerances.  Both sides round the matrix-product operands to bfloat16 (the oracle with
bf16=True); they differ in accumulation (FP32 on the tensor cores, FP64 in the oracle) and
in FP32 elementwise functions.  An FP32 accumulation error (~1e-6 relative) occasionally
moves an activation across a bfloat16 rounding boundary (probability ~1e-6 / 2^-9 per
activation, ~0.5 flips over the ~2000 activations of one point); one flip shifts ln q by
about |w| 2^-9 ~ 1e-3 at most.  Hence: most points agree to 1e-4 in ln q, every point to
2e-2; gradients (means over 300 points) element by element within the bound of gradient_bound."""
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import flow as F, likelihood as L, nested, prior as P, walk
from paper_2509_04336_gb300 import gwns, synth

from _util import event, priors

pytestmark = pytest.mark.gpu

LOGQ_MOST, LOGQ_ALL = 1e-4, 2e-2


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2509_04336_gb300 import build
    build.build()


def flow_handle(name="four_param_2det_taylorf2", p_flow=0.5, layers=8, **kw):
    w, ev = event(name)
    cfg = gwns.make_config(w, priors(w, ev), p_flow=p_flow, flow_layers=layers, **kw)
    return w, ev, gwns.ns_init([cfg], [ev])


def random_params(D, L, seed, scale=0.05, zero_out=False):
    """float32-representable random parameters (so both sides start from the same weights).
    At scale 0.05 every layer is a mild map (hidden gains ~0.6, |s| ~ 0.3), as a trained flow
    near the data is; much larger random weights make the 8-layer map chaotic and amplify
    any rounding difference without bound."""
    f = F.Flow(D, 128, L)
    p = np.random.default_rng(seed).normal(0.0, scale, f.n_params()).astype(np.float32)
    if zero_out:   # W3 = b3 = 0: every coupling is the identity
        f.set_flat(p.astype(np.float64))
        for l in range(L):
            f.W3[l][...] = 0.0
            f.b3[l][...] = 0.0
        p = f.flat().astype(np.float32)
    f.set_flat(p.astype(np.float64))
    return f, p


def set_both(h, f, p, D, seed):
    rng = np.random.default_rng(seed)
    f.mu = rng.normal(0.0, 0.5, D)
    f.sigma = rng.uniform(0.5, 1.5, D)
    f.mu = f.mu.astype(np.float32).astype(np.float64)
    f.sigma = f.sigma.astype(np.float32).astype(np.float64)
    gwns.ns_flow_set(h, 0, p, f.mu, f.sigma)


@pytest.mark.parametrize("D_name,n", [("four_param_2det_taylorf2", 300), ("bbh11_3det_4s_taylorf2", 257)])
def test_logq_parity(D_name, n):
    w, ev, h = flow_handle(D_name)
    try:
        D = w.n_dim
        f, p = random_params(D, 8, 1)
        set_both(h, f, p, D, 2)
        u = np.random.default_rng(3).uniform(0.01, 0.99, (n, D))
        g = np.zeros(n)
        gwns.ns_flow_logq(h, 0, u, g)
    finally:
        gwns.ns_free(h)
    _, o = F.forward(f, u, bf16=True)
    d = np.abs(g - o)
    assert np.quantile(d, 0.9) < LOGQ_MOST, np.quantile(d, [0.5, 0.9, 1.0])
    assert d.max() < LOGQ_ALL
    # and the bf16 rounding itself is visible against the plain FP64 flow
    _, o64 = F.forward(f, u, bf16=False)
    assert np.abs(o64 - o).max() > 10 * LOGQ_MOST


def test_flow_layers_and_round_trip():
    """Forward then inverse with the GPU's own kernels returns the points (bf16 effects and
    all, the map is still a bijection up to FP32 rounding)."""
    w, ev, h = flow_handle("bbh11_3det_4s_taylorf2", layers=4)
    try:
        D = w.n_dim
        f, p = random_params(D, 4, 4)
        set_both(h, f, p, D, 5)
        n_w, n_s = 3, 70
        tu = np.zeros((n_w, n_s, D))
        tl = np.zeros((n_w, n_s))
        gwns.ns_flow_sample(h, 0, 9, 11, tu, tl)
        lq = np.zeros(n_w * n_s)
        gwns.ns_flow_logq(h, 0, np.ascontiguousarray(tu.reshape(-1, D)), lq)
    finally:
        gwns.ns_free(h)
    key = (w.seed, 0)
    for wk in range(n_w):
        x = np.stack([F.base_normals(t, np.array([11 + wk]), 9, D, key)[0] for t in range(n_s)])
        ou, ol = F.inverse(f, x, bf16=True)
        np.testing.assert_allclose(tu[wk], ou, rtol=0, atol=2e-5)
        dl = np.abs(tl[wk] - ol)
        assert np.quantile(dl, 0.9) < LOGQ_MOST and dl.max() < LOGQ_ALL
    # the sampler's ln q and the forward kernel's ln q at the sample agree (two code paths)
    d = np.abs(lq - tl.reshape(-1))
    assert np.quantile(d, 0.9) < 1e-3 and d.max() < LOGQ_ALL


def gradient_bound(f, u, og):
    """Per-parameter tolerance of the GPU gradient (mean of -ln q over the points) against the
    oracle's bf16 gradient og.  Both sides round the same operands to bfloat16; where an FP32
    accumulation difference moves an operand across a bf16 rounding boundary, that operand
    changes by one bf16 ulp (at most 2^-7 of its size), and the point's contribution c_ij to
    parameter j by about as much relative to itself.  Bound: 2^-7 times the mean over points of
    |c_ij| -- as if every point's contribution had moved by one ulp, which the flip rate (~0.5
    flips among ~2000 operands of a point) makes far from tight -- plus 2^-10 |og_j| for the
    FP32 accumulation and elementwise functions, plus a floor of 1e-9 of the largest |og|.  (The
    unrounded FP64 gradient already leaves this bound at some parameters.)"""
    C = np.stack([F.loss_and_grad(f, u[i:i + 1], bf16=True)[1] for i in range(u.shape[0])])
    assert np.allclose(C.mean(axis=0), og, rtol=1e-9, atol=1e-12 * np.abs(og).max())
    return 2.0 ** -7 * np.abs(C).mean(axis=0) + 2.0 ** -10 * np.abs(og) + 1e-9 * np.abs(og).max()


def block_edges(D, L):
    return np.cumsum([128 * D, 128, 128 * 128, 128, 2 * D * 128, 2 * D] * L)[:-1]


def test_gradient_parity():
    w, ev, h = flow_handle("bbh11_3det_4s_taylorf2", layers=3)
    try:
        D = w.n_dim
        f, p = random_params(D, 3, 6)
        set_both(h, f, p, D, 7)
        u = np.random.default_rng(8).uniform(0.02, 0.98, (300, D))
        gl, gg = gwns.ns_flow_grad(h, 0, u)
    finally:
        gwns.ns_free(h)
    ol, og = F.loss_and_grad(f, u, bf16=True)
    assert abs(gl - ol) < 1e-4 * max(1.0, abs(ol))
    # element by element, every parameter
    tol = gradient_bound(f, u, og)
    d = np.abs(gg.astype(np.float64) - og)
    bad = np.where(d > tol)[0]
    assert bad.size == 0, f"{bad.size} parameters outside the bound, worst d/tol {np.max(d / tol):.2f} at {bad[:8]}"
    # the bound is tight enough to catch a sign error: 2 |og_j| exceeds the tolerance of most
    # parameters, and of at least 40 % in every block (the output layer's entries are means
    # of contributions that largely cancel)
    catch = 2.0 * np.abs(og) > tol
    assert catch.mean() > 0.8
    for cb in np.split(catch, block_edges(D, 3)):
        assert cb.mean() > 0.4


def test_training_matches_oracle_and_fits_gaussian():
    rng = np.random.default_rng(51)
    cov = np.array([[1.0, 0.8], [0.8, 1.0]]) * 0.25
    mean = np.array([0.5, -0.7])
    # a 4-dimensional target: two correlated logit-normal dimensions, two uniform ones
    z = rng.multivariate_normal(mean, cov, size=2000)
    u = np.concatenate([1.0 / (1.0 + np.exp(-z)), rng.uniform(0.01, 0.99, (2000, 2))], axis=1)
    w, ev, h = flow_handle("four_param_2det_taylorf2", layers=4, flow_lr=3e-3)
    try:
        p0, _, _ = gwns.ns_flow_get(h, 0, 4)
        losses = gwns.ns_flow_train(h, 0, u, 150)
    finally:
        gwns.ns_free(h)
    of = F.init_flow(4, 128, 4, (w.seed, 0))
    np.testing.assert_allclose(p0, of.flat(), rtol=0, atol=1e-7)    # same seeded initial weights
    ol = F.train(of, u, 150, F.Adam(of.flat().size, lr=3e-3), bf16=True)
    assert abs(losses[0] - ol[0]) < 1e-3
    assert np.all(np.abs(np.array(losses) - np.array(ol)) < 0.02 + 0.02 * np.abs(ol))
    assert losses[-1] < losses[0] - 0.3


def test_walk_with_identity_flow_matches_oracle():
    """Flow steps with W3 = b3 = 0 (q = the standardised logit-normal, no bf16 effects):
    the GPU chain equals the oracle's flow + DE chain away from near-ties."""
    name = "four_param_2det_taylorf2"
    w, ev, h = flow_handle(name, p_flow=0.5)
    try:
        D = w.n_dim
        f, p = random_params(D, 8, 9, zero_out=True)
        f.mu = np.zeros(D)
        f.sigma = np.ones(D)
        pri = priors(w, ev)
        ll = lambda x: L.log_likelihood(ev, P.transform(x, pri), w.waveform, w.use_ratio)
        rng = np.random.default_rng(10)
        surv = rng.random((60, D))
        lnl_s = np.array([ll(x) for x in surv])
        lnl_star = float(np.quantile(lnl_s, 0.3))
        ok = np.where(lnl_s > lnl_star)[0]
        starts = ok[rng.integers(0, ok.shape[0], 24)]
        u0, l0 = np.ascontiguousarray(surv[starts]), np.ascontiguousarray(lnl_s[starts])
        # standardisation of the sampler's own choosing: fit to the survivors
        lg = np.log(surv) - np.log1p(-surv)
        f.mu = lg.mean(0).astype(np.float32).astype(np.float64)
        f.sigma = lg.std(0).astype(np.float32).astype(np.float64)
        gwns.ns_flow_set(h, 0, p, f.mu, f.sigma)
        n_steps, it, off = 16, 2, 5
        gu, gl = np.zeros_like(u0), np.zeros(24)
        ga, gn = np.zeros(24, np.int32), np.zeros(24, np.int32)
        gwns.ns_walk_batch(h, 0, np.ascontiguousarray(surv), u0, l0, lnl_star, n_steps, it, off, gu, gl, ga, gn)
    finally:
        gwns.ns_free(h)
    periodic = P.periodic_mask(pri)
    ou, ol, oa, on, margin = walk.acceptance_walk(ll, u0, l0, lnl_star, surv, n_steps, periodic, (w.seed, 0), it,
                                                  walker_ids=np.arange(24) + off, flow=f, p_flow=0.5,
                                                  flow_bf16=True)
    # decisions within 1e-3 of their threshold (an ln L or an ln q ratio; the GPU's proposals
    # and ln q are FP32, ~1e-7 relative, moving ln L by ~1e-4 at most here) may go either way
    same = margin > 1e-3
    assert same.sum() >= 16
    assert np.array_equal(ga[same], oa[same]) and np.array_equal(gn[same], on[same])
    assert np.allclose(gu[same], ou[same], rtol=0, atol=1e-6)
    assert np.all(gl > lnl_star)
    assert oa.sum() > 0 and on.sum() > 0


def test_mixed_walk_keeps_constrained_prior_uniform():
    """L* = -inf: the DE + flow walk, with a strongly non-uniform trained-looking flow, must
    leave the uniform prior invariant (a wrong q ratio, table index or carried ln q would
    pull the walkers towards q)."""
    w, ev, h = flow_handle("four_param_2det_taylorf2", p_flow=0.6)
    try:
        D = w.n_dim
        f, p = random_params(D, 8, 12, scale=0.12)
        rng = np.random.default_rng(13)
        gwns.ns_flow_set(h, 0, p, rng.normal(0.0, 0.5, D), np.full(D, 0.4))   # narrow q
        n = 3000
        rng = np.random.default_rng(14)
        surv = np.ascontiguousarray(rng.random((400, D)))
        u0 = np.ascontiguousarray(rng.random((n, D)))
        l0 = np.zeros(n)
        gu, gl = np.zeros_like(u0), np.zeros(n)
        ga, gn = np.zeros(n, np.int32), np.zeros(n, np.int32)
        gwns.ns_walk_batch(h, 0, surv, u0, l0, -np.inf, 10, 0, 0, gu, gl, ga, gn)
        # samples of q itself are far from uniform (so the test has power)
        tu = np.zeros((1, 2000, D))
        tl = np.zeros((1, 2000))
        gwns.ns_flow_sample(h, 0, 0, 0, tu, tl)
    finally:
        gwns.ns_free(h)
    for d in range(D):
        assert stats.kstest(gu[:, d], "uniform").pvalue > 1e-3, d
    assert min(stats.kstest(tu[0, :, d], "uniform").pvalue for d in range(D)) < 1e-6
    assert 0 < gn.sum() < 10 * n


def test_sampler_with_flow_runs_and_agrees_on_evidence():
    """The whole sampler with flow training inside the batch graph: ln Z within errors of the
    oracle's DE-only run on the zero-noise 4-parameter event."""
    w, ev = event("four_param_2det_taylorf2")
    cfg = gwns.make_config(w, priors(w, ev), p_flow=0.5, flow_layers=4, flow_epochs=10, flow_every=2)
    h = gwns.ns_init([cfg], [ev])
    try:
        for _ in range(200):
            _, pr = gwns.ns_step(h, 8)
            if pr[0]["done"]:
                break
        lz, lz_err, _, n_like = gwns.ns_evidence(h, 0)
        p1, mu, sg = gwns.ns_flow_get(h, 0, w.n_dim)
    finally:
        gwns.ns_free(h)
    assert pr[0]["done"]
    # the oracle's own run (DE walk), stored by tests/golden/make_logz_golden.py
    with open(os.path.join(os.path.dirname(__file__), "golden", "logz_oracle.json")) as fh:
        ref = json.load(fh)["four_param_2det_taylorf2"]
    assert abs(lz - ref["log_z"]) < 4 * math.hypot(max(lz_err, 0.05), max(ref["log_z_err"], 0.05))
    assert np.all(np.isfinite(p1)) and np.all(sg > 0)
    assert n_like > 0


def test_flow_raises_accepted_steps_per_likelihood_call():
    """What the trained flow gains over the DE walk alone, on the learned-proposal configuration
    (8 s IMRPhenomD form, 4000 live points, 2000 survivors to train on each batch): accepted
    walk steps per likelihood call in batches 21-25, DE only against p_flow = 0.9 on the same
    data and seed.  (On smaller live sets -- a few hundred survivors -- the flow fits less well
    and does not gain; the gain is a property of this configuration.)"""
    w = synth.workload("bbh11_3det_8s_phenomd_flow")
    ev = synth.make_event(w, lambda e, i, th: L.project(e, i, th, w.waveform), L.inner)
    rate = {}
    for pf in (0.0, 0.9):
        kw = {} if pf == 0.0 else {"p_flow": pf, "flow_layers": 8}
        cfg = gwns.make_config(w, synth.priors_with_injection(w, ev), precision=synth.PREC_MIXED_FF, **kw)
        h = gwns.ns_init([cfg], [ev])
        try:
            _, p0 = gwns.ns_step(h, 20)
            acc = 0.0
            for _ in range(5):
                _, p = gwns.ns_step(h, 1)
                acc += p[0]["mean_accept"] * w.num_delete
            rate[pf] = acc / (p[0]["n_like"] - p0[0]["n_like"])
        finally:
            gwns.ns_free(h)
    print("accepted steps per likelihood call:", rate)
    assert rate[0.9] > 1.3 * rate[0.0], rate


def test_flow_accept_weight_shortens_walks_by_its_rule():
    """flow_accept_weight w: after every batch the next walk length is the retune of the
    weighted count (accepted DE steps + w x accepted flow steps, per walker), the flow
    acceptances are part of the accepted steps, and the weighted run needs fewer likelihood
    calls than w = 1; on this small 4-parameter event its ln Z stays within errors of the
    oracle's (on the 11-parameter learned-proposal configuration it does not: the weight is an
    experiment).  The batch-phase calls, which do not carry flow acceptance counts, refuse such
    a handle."""
    w, ev = event("four_param_2det_taylorf2")
    k, N, wt = w.num_delete, w.naccept, 10.0
    delay_k = nested.batch_delay(float(N - 1), k)
    runs = {}
    for weight in (0.0, wt):
        cfg = gwns.make_config(w, priors(w, ev), p_flow=0.5, flow_layers=4, flow_epochs=10, flow_every=2,
                               flow_accept_weight=weight)
        h = gwns.ns_init([cfg], [ev])
        try:
            if weight == wt:
                with pytest.raises(gwns.GwnsError) as e:
                    gwns.ns_batch_begin(h)
                assert e.value.code == gwns.NS_EINVAL
            n_used = int(math.ceil(N / 0.25))
            seen_flow = 0.0
            for _ in range(400):
                _, pr = gwns.ns_step(h, 1)
                p = pr[0]
                a, af = p["mean_accept"], p["mean_accept_flow"]
                assert 0.0 <= af <= a
                seen_flow += af
                if not p["done"]:
                    acc, accf = round(a * k), round(af * k)
                    eff = (acc + ((weight if weight > 0 else 1.0) - 1.0) * accf) / k
                    assert p["n_steps"] == nested.retune(n_used, eff, N, delay_k, w.maxmcmc)
                n_used = p["n_steps"]
                if p["done"]:
                    break
            lz, lz_err, _, n_like = gwns.ns_evidence(h, 0)
        finally:
            gwns.ns_free(h)
        assert p["done"] and seen_flow > 0
        runs[weight] = (lz, lz_err, n_like)
    with open(os.path.join(os.path.dirname(__file__), "golden", "logz_oracle.json")) as fh:
        ref = json.load(fh)["four_param_2det_taylorf2"]
    lz, lz_err, n_like = runs[wt]
    assert abs(lz - ref["log_z"]) < 4 * math.hypot(max(lz_err, 0.05), max(ref["log_z_err"], 0.05))
    assert n_like < runs[0.0][2]
