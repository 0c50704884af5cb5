"""CUDA path vs the oracle: waveform element by element, ln L per parameter vector."""
import numpy as np
import pytest

from oracle import likelihood as L
from paper_2509_04336_gb300 import gwns, synth

from _util import event, priors, prior_draws, oracle_lnl

pytestmark = pytest.mark.gpu

# FP64 path: same arithmetic up to rounding order (phase regrouped by powers of f).
TOL_FP64 = 1e-11
# Mixed path: ln L within 1e-6 of |ln L| (FP32 sums; FP64 phase reduced before an FP32 sincos).
TOL_MIXED = 1e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2509_04336_gb300 import build
    build.build()


def handle(w, ev, precision):
    cfg = gwns.make_config(w, priors(w, ev), precision=precision)
    return gwns.ns_init([cfg], [ev])


@pytest.mark.parametrize("name", ["four_param_2det_taylorf2", "bbh11_3det_4s_taylorf2", "bbh11_3det_8s_phenomd"])
def test_waveform_elementwise(name):
    w, ev = event(name)
    h = handle(w, ev, synth.PREC_FP64)
    try:
        _, th = prior_draws(w, ev, 6, 11)
        th = np.vstack([ev.theta_inj, th])
        nd = len(ev.detectors)
        hr = np.zeros((th.shape[0], nd, ev.n_bins))
        hi = np.zeros_like(hr)
        gwns.ns_waveform(h, 0, np.ascontiguousarray(th), hr, hi)
        for i in range(th.shape[0]):
            for d in range(nd):
                want = L.project(ev, d, th[i], w.waveform)
                got = hr[i, d] + 1j * hi[i, d]
                scale = np.max(np.abs(want))
                assert np.all((want == 0) == (got == 0)), "cutoff bin differs"
                assert np.max(np.abs(got - want)) <= 1e-10 * scale
    finally:
        gwns.ns_free(h)


@pytest.mark.parametrize("name,precision,tol", [
    ("four_param_2det_taylorf2", synth.PREC_FP64, TOL_FP64),
    ("four_param_2det_taylorf2", synth.PREC_MIXED, TOL_MIXED),
    ("bbh11_3det_4s_taylorf2", synth.PREC_FP64, TOL_FP64),
    ("bbh11_3det_4s_taylorf2", synth.PREC_MIXED, TOL_MIXED),
    ("four_param_2det_taylorf2", synth.PREC_MIXED_FF, TOL_MIXED),
    ("bbh11_3det_4s_taylorf2", synth.PREC_MIXED_FF, TOL_MIXED),
    ("bbh11_3det_8s_phenomd", synth.PREC_FP64, TOL_FP64),
    ("bbh11_3det_8s_phenomd", synth.PREC_MIXED, TOL_MIXED),
    ("bbh11_3det_8s_phenomd", synth.PREC_MIXED_FF, TOL_MIXED),
])
def test_likelihood_parity(name, precision, tol):
    w, ev = event(name)
    h = handle(w, ev, precision)
    try:
        _, th = prior_draws(w, ev, 96, 5)
        th = np.ascontiguousarray(np.vstack([ev.theta_inj, th]))
        got = np.zeros(th.shape[0])
        gwns.ns_likelihood_batch(h, 0, th, got)
        want = oracle_lnl(w, ev, th)
        err = np.abs(got - want)
        # zero-noise truth has ln L = 0: an absolute floor of tol * SNR^2 / 2 there
        scale = np.maximum(np.abs(want), 0.5 * w.snr ** 2)
        print(f"\nLNL_ERR {name} precision {precision}: max |err| / scale {np.max(err / scale):.3e}, "
              f"max |err| {np.max(err):.3e}, points {th.shape[0]}")
        assert np.all(err <= tol * scale), f"max rel err {np.max(err / scale):.3e}"
    finally:
        gwns.ns_free(h)


def test_likelihood_device_pointers_and_edge_cases():
    import torch
    w, ev = event("bbh11_3det_4s_taylorf2")
    h = handle(w, ev, synth.PREC_MIXED)
    try:
        _, th = prior_draws(w, ev, 5, 9)
        # masses giving a cutoff below f_min: no active bin, h = 0, ln L = -<d|d>/2
        heavy = ev.theta_inj.copy(); heavy[0] = 400.0
        th = np.vstack([th, heavy])
        t = torch.tensor(th, device="cuda", dtype=torch.float64)
        out = torch.zeros(th.shape[0], device="cuda", dtype=torch.float64)
        gwns.ns_likelihood_batch(h, 0, t, out)
        torch.cuda.synchronize()
        want = oracle_lnl(w, ev, th)
        assert np.allclose(out.cpu().numpy(), want, rtol=TOL_MIXED, atol=0)
        # empty batch is a no-op
        gwns.ns_likelihood_batch(h, 0, np.zeros((0, 11)), np.zeros(0))
        # non-finite theta is reported, not evaluated
        bad = th[:2].copy(); bad[1, 3] = np.nan
        with pytest.raises(gwns.GwnsError) as e:
            gwns.ns_likelihood_batch(h, 0, np.ascontiguousarray(bad), np.zeros(2))
        assert e.value.code == gwns.NS_ENONFINITE
    finally:
        gwns.ns_free(h)


def test_likelihood_ragged_bins_small_event():
    # 23 bins: fewer than one CTA's threads, and a ragged tail.
    w, ev = event("bbh11_3det_4s_taylorf2", f_max=25.5)
    assert ev.n_bins == 23
    for prec, tol in ((synth.PREC_FP64, TOL_FP64), (synth.PREC_MIXED, TOL_MIXED), (synth.PREC_MIXED_FF, TOL_MIXED)):
        h = handle(w, ev, prec)
        try:
            _, th = prior_draws(w, ev, 17, 3)
            th = np.ascontiguousarray(th)
            got = np.zeros(17)
            gwns.ns_likelihood_batch(h, 0, th, got)
            want = oracle_lnl(w, ev, th)
            assert np.all(np.abs(got - want) <= tol * np.maximum(np.abs(want), 1.0))
        finally:
            gwns.ns_free(h)


def test_largest_batched_event_full_size():
    # The 64-event population's 16 s events have 32,449 bins (20-2048 Hz at 1/16 Hz), the
    # largest event the sampler is run on: ln L of sampled points against the oracle in the
    # FP64 and float-float modes at full size, and a short float-float walk.
    from oracle import prior as P, walk
    w = synth.batched_workloads(8, seed=100)[2]
    assert w.n_bins == 32449 and w.waveform == synth.PHENOMD_FORM
    ev = synth.make_event(w, lambda e, d, th: L.project(e, d, th, w.waveform), L.inner)
    pri = synth.priors_with_injection(w, ev)
    u = synth.uniform_unit_cube(12, w.n_dim, 31)
    th = np.ascontiguousarray(np.vstack([ev.theta_inj] + [P.transform(x, pri) for x in u]))
    want = np.array([L.log_likelihood(ev, t, w.waveform, w.use_ratio) for t in th])
    for prec, tol in ((synth.PREC_FP64, TOL_FP64), (synth.PREC_MIXED, TOL_MIXED), (synth.PREC_MIXED_FF, TOL_MIXED)):
        h = gwns.ns_init([gwns.make_config(w, pri, precision=prec)], [ev])
        try:
            got = np.zeros(th.shape[0])
            gwns.ns_likelihood_batch(h, 0, th, got)
            scale = np.maximum(np.abs(want), 0.5 * w.snr ** 2)
            print(f"\nLNL_ERR batched64_16s precision {prec}: max |err| / scale "
                  f"{np.max(np.abs(got - want) / scale):.3e}, max |err| {np.max(np.abs(got - want)):.3e}")
            assert np.all(np.abs(got - want) <= tol * scale), (prec, np.max(np.abs(got - want) / scale))
        finally:
            gwns.ns_free(h)
    # walk: 6 walkers, 8 steps, from survivors above the 40 % quantile of 40 prior points
    ll = lambda x: L.log_likelihood(ev, P.transform(x, pri), w.waveform, w.use_ratio)
    surv = synth.uniform_unit_cube(40, w.n_dim, 32)
    ls = np.array([ll(x) for x in surv])
    star = float(np.quantile(ls, 0.4))
    idx = np.where(ls > star)[0][:6]
    u0, l0 = np.ascontiguousarray(surv[idx]), np.ascontiguousarray(ls[idx])
    ou, ol, oa, on, margin = walk.acceptance_walk(ll, u0, l0, star, surv, 8, P.periodic_mask(pri), (w.seed, 0), 1)
    h = gwns.ns_init([gwns.make_config(w, pri, precision=synth.PREC_MIXED_FF, spec_depth=4)], [ev])
    try:
        gu, gl = np.zeros_like(u0), np.zeros(6)
        ga, gn = np.zeros(6, np.int32), np.zeros(6, np.int32)
        gwns.ns_walk_batch(h, 0, np.ascontiguousarray(surv), u0, l0, star, 8, 1, 0, gu, gl, ga, gn)
    finally:
        gwns.ns_free(h)
    same = margin > 4e-6 * max(abs(star), 1.0)
    assert same.sum() >= 4
    assert np.array_equal(ga[same], oa[same]) and np.array_equal(gn[same], on[same])
    assert np.allclose(gu[same], ou[same], rtol=0, atol=1e-12)
    assert np.all(gl > star)


@pytest.mark.parametrize("precision", [synth.PREC_FP64, synth.PREC_MIXED, synth.PREC_MIXED_FF])
def test_likelihood_ratio_parity(precision):
    # use_ratio (Sec. 4.1.1): ln Lambda = ln L + <d|d>/2 per detector sum, on the 11-parameter
    # 3-detector event, in every precision; the kernels form it from <d|h> - <h|h>/2 directly.
    from dataclasses import replace
    w, ev = event("bbh11_3det_4s_taylorf2")
    w = replace(w, use_ratio=True)
    h = handle(w, ev, precision)
    try:
        _, th = prior_draws(w, ev, 64, 17)
        th = np.ascontiguousarray(np.vstack([ev.theta_inj, th]))
        got = np.zeros(th.shape[0])
        gwns.ns_likelihood_batch(h, 0, th, got)
        want = oracle_lnl(w, ev, th)
        tol = TOL_FP64 if precision == synth.PREC_FP64 else TOL_MIXED
        scale = np.maximum(np.abs(want), 0.5 * w.snr ** 2)
        assert np.all(np.abs(got - want) <= tol * scale), f"max rel err {np.max(np.abs(got - want) / scale):.3e}"
        # ln Lambda - ln L is the data term <d|d>/2, the same for every theta
        plain = oracle_lnl(replace(w, use_ratio=False), ev, th[:3])
        dd = 0.5 * sum(L.inner(d.data, d.data, d.psd, ev.df) for d in ev.detectors)
        assert np.allclose(want[:3] - plain, dd, rtol=1e-12)
        assert want[0] > 0.4 * w.snr ** 2   # the injection: ln Lambda near SNR^2 / 2
    finally:
        gwns.ns_free(h)
