"""Relative-binning likelihood (ns_relbin_set) of the float-float mode against the oracle's
relative-binning likelihood (oracle/relbin.py) on the same edges and fiducial."""
import numpy as np
import pytest

from oracle import likelihood as L, relbin
from paper_2509_04336_gb300 import gwns, synth

from _util import event, priors, prior_draws

pytestmark = pytest.mark.gpu

# The summary data are FP64 sums stored in FP32 (relative 6e-8 each) and the ratio at the
# edges carries the float-float phase (~1e-7 cycles, ~7e-7 rad) through an FP32 sincos, so
# <d|h> - <h|h>/2 is good to ~1e-6 of max(|<d|h> - <h|h>/2|, SNR^2/2) even if the per-bin
# errors added up coherently; the bound is 1e-5 of that scale (the <d|d> term is FP64 on both
# sides and is left out of the scale).
TOL_RB = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2509_04336_gb300 import build
    build.build()


def bulk_points(w, ev, n, seed):
    """Points around the injection whose full ln L is within 30 of its value there."""
    rng = np.random.default_rng(seed)
    l0 = L.log_likelihood(ev, ev.theta_inj, w.waveform)
    scale = np.array([1e-2 * ev.theta_inj[0], 0.02, 0.02, 0.02, 50.0, 0.05, 0.05, 0.05, 2e-4, 0.02, 0.02])
    out = []
    for _ in range(n):
        step = scale * rng.normal(size=11)
        for _ in range(12):
            if L.log_likelihood(ev, ev.theta_inj + step, w.waveform) > l0 - 30.0:
                break
            step *= 0.5
        out.append(ev.theta_inj + step)
    return np.stack(out)


def check(w, ev, edges, theta):
    h = gwns.ns_init([gwns.make_config(w, priors(w, ev), precision=synth.PREC_MIXED_FF)], [ev])
    try:
        full = np.zeros(theta.shape[0])
        gwns.ns_likelihood_batch(h, 0, theta, full)
        gwns.ns_relbin_set(h, 0, edges, ev.theta_inj)
        got = np.zeros(theta.shape[0])
        gwns.ns_likelihood_batch(h, 0, theta, got)
        # back to the full likelihood: the same values as before, bit for bit
        gwns.ns_relbin_set(h, 0, None)
        again = np.zeros(theta.shape[0])
        gwns.ns_likelihood_batch(h, 0, theta, again)
    finally:
        gwns.ns_free(h)
    assert np.array_equal(full, again)
    sd = relbin.summary_data(ev, ev.theta_inj, edges, w.waveform)
    want = np.array([relbin.log_likelihood(ev, th, sd, w.waveform, w.use_ratio) for th in theta])
    base = 0.0 if w.use_ratio else -0.5 * sd["dd"]
    scale = np.maximum(np.abs(want - base), 0.5 * w.snr ** 2)
    err = np.abs(got - want) / scale
    print(f"{len(edges) - 1} coarse bins: max err {np.max(err):.2e} of the scale, "
          f"max |got - want| {np.max(np.abs(got - want)):.2e}")
    assert np.all(err <= TOL_RB), f"max rel err {np.max(err):.3e}"
    return got, want, full


@pytest.mark.parametrize("name,eps", [("four_param_2det_taylorf2", 0.25), ("bbh11_3det_4s_taylorf2", 0.25),
                                      ("bbh11_3det_4s_taylorf2", 3.0), ("bbh11_3det_8s_phenomd", 0.25)])
def test_relbin_likelihood_parity(name, eps):
    # The injection (r = 1 at every edge), points in the posterior bulk, and prior draws whose
    # cutoffs fall anywhere on the grid (the exact range then holds a different coarse bin).
    w, ev = event(name)
    edges = relbin.default_edges(ev.f_min, ev.df, ev.n_bins, eps)
    _, far = prior_draws(w, ev, 12, 21)
    theta = np.ascontiguousarray(np.vstack([ev.theta_inj, bulk_points(w, ev, 8, 5), far]))
    got, want, full = check(w, ev, edges, theta)
    if eps <= 0.25:
        # in the bulk the compressed ln L follows the full one (the oracle's own pin: 0.05)
        assert np.max(np.abs(got[:9] - full[:9])) < 0.1


def test_relbin_one_grid_bin_per_coarse_bin_is_the_full_likelihood():
    # Every coarse bin one grid bin wide except the last (no expansion is made across the
    # last bin): the expansion is exact and the GPU's compressed ln L is the full one.
    w, ev = event("four_param_2det_taylorf2", f_max=64.0)
    edges = np.arange(ev.n_bins + 1)
    _, th = prior_draws(w, ev, 8, 9)
    theta = np.ascontiguousarray(np.vstack([ev.theta_inj, th]))
    got, want, full = check(w, ev, edges, theta)
    scale = np.maximum(np.abs(full), 0.5 * w.snr ** 2)
    assert np.all(np.abs(got - full) <= TOL_RB * scale)


def test_relbin_edge_cases_and_errors():
    w, ev = event("four_param_2det_taylorf2", f_max=64.0)
    n = ev.n_bins
    h = gwns.ns_init([gwns.make_config(w, priors(w, ev), precision=synth.PREC_FP64)], [ev])
    try:
        with pytest.raises(gwns.GwnsError) as e:
            gwns.ns_relbin_set(h, 0, [0, n], ev.theta_inj)
        assert e.value.code == gwns.NS_EINVAL
    finally:
        gwns.ns_free(h)
    h = gwns.ns_init([gwns.make_config(w, priors(w, ev), precision=synth.PREC_MIXED_FF)], [ev])
    try:
        for bad in ([1, n], [0, n - 1], [0, 5, 5, n], [0]):
            with pytest.raises(gwns.GwnsError) as e:
                gwns.ns_relbin_set(h, 0, bad, ev.theta_inj)
            assert e.value.code == gwns.NS_EINVAL
        with pytest.raises(gwns.GwnsError):
            gwns.ns_relbin_set(h, 0, [0, n], np.full(11, np.nan))
        # a single coarse bin (the last one: summed exactly) is the full likelihood
        gwns.ns_relbin_set(h, 0, [0, n], ev.theta_inj)
        th = np.ascontiguousarray(np.vstack([ev.theta_inj, prior_draws(w, ev, 4, 2)[1]]))
        got = np.zeros(th.shape[0])
        gwns.ns_likelihood_batch(h, 0, th, got)
        want = np.array([L.log_likelihood(ev, t, w.waveform, w.use_ratio) for t in th])
        assert np.all(np.abs(got - want) <= 1e-6 * np.maximum(np.abs(want), 0.5 * w.snr ** 2))
        gwns.ns_step(h, 1)
        with pytest.raises(gwns.GwnsError) as e:
            gwns.ns_relbin_set(h, 0, [0, n], ev.theta_inj)
        assert e.value.code == gwns.NS_EINVAL
    finally:
        gwns.ns_free(h)


def test_relbin_sampler_evidence_matches_the_full_likelihood():
    # The sampler end to end on the compressed likelihood (the initial live points re-evaluated
    # by ns_relbin_set, the walks on the relative-binning kernel path): ln Z within the two
    # runs' sampling errors of the full-likelihood run on the same data and seed.
    w, ev = event("bbh11_3det_4s_taylorf2")
    from dataclasses import replace
    w = replace(w, n_live=400, num_delete=200)
    edges = relbin.default_edges(ev.f_min, ev.df, ev.n_bins, 0.25)
    res = {}
    for tag in ("full", "relbin"):
        h = gwns.ns_init([gwns.make_config(w, priors(w, ev), precision=synth.PREC_MIXED_FF)], [ev])
        try:
            if tag == "relbin":
                gwns.ns_relbin_set(h, 0, edges, ev.theta_inj)
            done, b = False, 0
            while not done and b < 2000:
                _, prog = gwns.ns_step(h, 8)
                b += 8
                done = bool(prog[0]["done"])
            assert done
            res[tag] = gwns.ns_evidence(h, 0)
        finally:
            gwns.ns_free(h)
    (lz_f, err_f, _, _), (lz_r, err_r, _, _) = res["full"], res["relbin"]
    print("ln Z full", lz_f, "+-", err_f, "relbin", lz_r, "+-", err_r)
    assert abs(lz_f - lz_r) < 4.0 * np.hypot(err_f, err_r)


def test_sampler_walks_take_the_relative_binning_path():
    # The sampler's batch graph chooses its walk kernel by whether an event uses the
    # relative-binning likelihood (a TaylorF2 float-float walk without flow or relative binning
    # runs a kernel compiled without those paths).  With ns_relbin_set before the first batch
    # the walks must evaluate the relative-binning likelihood: a call touches the ~35 coarse-bin
    # edges below the cutoff and one coarse bin's grid bins, where the full likelihood touches
    # every active bin (~190 on this event).  After a batch has run the call is refused.
    w, ev = event("four_param_2det_taylorf2")
    edges = relbin.default_edges(ev.f_min, ev.df, ev.n_bins, 0.25)
    per_call = {}
    for tag in ("full", "relbin"):
        h = gwns.ns_init([gwns.make_config(w, priors(w, ev), precision=synth.PREC_MIXED_FF)], [ev])
        try:
            if tag == "relbin":
                gwns.ns_relbin_set(h, 0, edges, ev.theta_inj)
            _, p0 = gwns.ns_step(h, 1)
            _, p1 = gwns.ns_step(h, 3)
            per_call[tag] = (p1[0]["n_bins"] - p0[0]["n_bins"]) / (p1[0]["n_like"] - p0[0]["n_like"])
            with pytest.raises(gwns.GwnsError) as e:
                gwns.ns_relbin_set(h, 0, None if tag == "relbin" else edges, ev.theta_inj)
            assert e.value.code == gwns.NS_EINVAL
        finally:
            gwns.ns_free(h)
    print("bins per call", per_call)
    assert per_call["relbin"] < 0.6 * per_call["full"]
