"""Pins of the relative-binning oracle (oracle/relbin.py) against the full likelihood."""
import numpy as np
import pytest

from oracle import likelihood as L, prior as P, relbin
from paper_2509_04336_gb300 import synth

from _util import event, priors


def _draws(w, ev, n, seed):
    pri = priors(w, ev)
    return [P.transform(x, pri) for x in synth.uniform_unit_cube(n, w.n_dim, seed)]


def test_edges_cover_the_grid_and_scale_with_eps():
    w, ev = event("bbh11_3det_4s_taylorf2")
    e1 = relbin.default_edges(ev.f_min, ev.df, ev.n_bins, eps=0.25)
    e2 = relbin.default_edges(ev.f_min, ev.df, ev.n_bins, eps=2.0)
    for e in (e1, e2):
        assert e[0] == 0 and e[-1] == ev.n_bins and np.all(np.diff(e) >= 1)
    assert 10 < len(e2) < len(e1) < ev.n_bins // 20


@pytest.mark.parametrize("name", ["bbh11_3det_4s_taylorf2", "bbh11_3det_8s_phenomd"])
def test_one_grid_bin_per_coarse_bin_is_the_full_likelihood(name):
    # With every coarse bin one grid bin wide, the linear term vanishes and the expansion is
    # exact: the relative-binning ln L equals the full one for any parameters.
    w, ev = event(name, f_max=200.0) if "phenomd" in name else event(name)
    edges = np.arange(ev.n_bins + 1)
    sd = relbin.summary_data(ev, ev.theta_inj, edges, w.waveform)
    for th in _draws(w, ev, 4, 3):
        want = L.log_likelihood(ev, th, w.waveform)
        assert abs(relbin.log_likelihood(ev, th, sd, w.waveform) - want) <= 1e-9 * abs(want)


@pytest.mark.parametrize("name", ["bbh11_3det_4s_taylorf2", "bbh11_3det_8s_phenomd"])
def test_fiducial_point_is_exact(name):
    # At theta0 the ratio is 1 at every edge: the summary data sum the full likelihood.
    w, ev = event(name)
    edges = relbin.default_edges(ev.f_min, ev.df, ev.n_bins)
    sd = relbin.summary_data(ev, ev.theta_inj, edges, w.waveform)
    want = L.log_likelihood(ev, ev.theta_inj, w.waveform)
    assert abs(relbin.log_likelihood(ev, ev.theta_inj, sd, w.waveform) - want) <= 1e-9 * abs(want)
    assert abs(relbin.log_likelihood(ev, ev.theta_inj, sd, w.waveform, use_ratio=True)
               - L.log_likelihood(ev, ev.theta_inj, w.waveform, use_ratio=True)) <= 1e-6


def test_frequency_independent_ratio_is_exact():
    # Distance and inclination change only the constant factor of h / h0 (the cutoff stays
    # put), so the linear expansion is exact whatever the bins.
    w, ev = event("bbh11_3det_4s_taylorf2")
    edges = relbin.default_edges(ev.f_min, ev.df, ev.n_bins, eps=3.0)
    sd = relbin.summary_data(ev, ev.theta_inj, edges, w.waveform)
    th = ev.theta_inj.copy()
    th[4] *= 1.7
    th[5] = 1.1
    want = L.log_likelihood(ev, th, w.waveform)
    assert abs(relbin.log_likelihood(ev, th, sd, w.waveform) - want) <= 1e-9 * abs(want)


@pytest.mark.parametrize("name", ["bbh11_3det_4s_taylorf2", "bbh11_3det_8s_phenomd"])
def test_close_to_the_full_likelihood_in_the_posterior_bulk(name):
    # Random points around theta0, shrunk until the full ln L is within 30 of its value at
    # theta0 (the bulk of the posterior): the compressed ln L stays within 0.05 of the full one.
    w, ev = event(name)
    edges = relbin.default_edges(ev.f_min, ev.df, ev.n_bins)
    sd = relbin.summary_data(ev, ev.theta_inj, edges, w.waveform)
    l0 = L.log_likelihood(ev, ev.theta_inj, w.waveform)
    rng = np.random.default_rng(4)
    scale = np.array([1e-2 * ev.theta_inj[0], 0.02, 0.02, 0.02, 50.0, 0.05, 0.05, 0.05, 2e-4, 0.02, 0.02])
    worst = 0.0
    for _ in range(6):
        step = scale * rng.normal(size=11)
        while True:
            th = ev.theta_inj + step
            want = L.log_likelihood(ev, th, w.waveform)
            if want > l0 - 30.0:
                break
            step *= 0.5
        got = relbin.log_likelihood(ev, th, sd, w.waveform)
        worst = max(worst, abs(got - want))
    assert worst < 0.05, worst


@pytest.mark.parametrize("name", ["four_param_2det_taylorf2", "bbh11_3det_4s_taylorf2", "bbh11_3det_8s_phenomd"])
def test_library_edges_follow_the_same_rule(name):
    # The library's edge rule (ns_relbin_edges, host code of libgwns, written separately) gives
    # the oracle's edges; the call does no device work, so it runs without a GPU.
    from paper_2509_04336_gb300 import build, gwns
    build.build()
    gwns.load()
    w = synth.workload(name)
    for eps in (0.1, 0.25, 1.0, 3.0):
        assert np.array_equal(gwns.ns_relbin_edges(w.f_min, w.df, w.n_bins, eps),
                              relbin.default_edges(w.f_min, w.df, w.n_bins, eps))
    assert np.array_equal(gwns.ns_relbin_edges(w.f_min, w.df, 1, 0.25), [0, 1])


@pytest.mark.parametrize("name", ["bbh11_3det_4s_taylorf2", "bbh11_3det_8s_phenomd"])
def test_summary_data_are_exact_for_a_linear_ratio(name):
    # For any ratio linear in f, r(f) = alpha + beta f (complex), the summary data reproduce
    # <d|h0 r> and <h0 r|h0 r> exactly: sum_b Re(A0 r_b + A1 beta) and
    # sum_b B0 |r_b|^2 + 2 B1 Re(conj(r_b) beta) + B2 |beta|^2, with r_b = r(f at edge b).
    # Every summary coefficient enters (a dropped term, a sign or a wrong offset fails).
    from paper_2509_04336_gb300.synth import frequencies
    w, ev = event(name)
    edges = relbin.default_edges(ev.f_min, ev.df, ev.n_bins, eps=1.0)
    sd = relbin.summary_data(ev, ev.theta_inj, edges, w.waveform)
    f = frequencies(ev.f_min, ev.df, ev.n_bins)
    alpha, beta = 0.7 - 0.4j, (2.0 + 1.5j) / (f[-1] - f[0])
    r_f = alpha + beta * f
    r_e = alpha + beta * sd["fe"][:-1]
    for i, d in enumerate(ev.detectors):
        h0 = L.project(ev, i, ev.theta_inj, w.waveform, cutoff=False)
        wgt = 4.0 * ev.df / d.psd
        dh_direct = float(np.sum((np.conj(d.data) * h0 * r_f).real * wgt))
        hh_direct = float(np.sum(np.abs(h0 * r_f) ** 2 * wgt))
        dh_sd = float(np.sum((sd["A0"][i] * r_e + sd["A1"][i] * beta).real))
        hh_sd = float(np.sum(sd["B0"][i] * np.abs(r_e) ** 2 + 2.0 * sd["B1"][i] * (np.conj(r_e) * beta).real
                             + sd["B2"][i] * abs(beta) ** 2))
        assert abs(dh_sd - dh_direct) <= 1e-9 * max(abs(dh_direct), hh_direct)
        assert abs(hh_sd - hh_direct) <= 1e-9 * hh_direct


@pytest.mark.parametrize("name", ["bbh11_3det_4s_taylorf2", "bbh11_3det_8s_phenomd"])
def test_coarse_bin_holding_the_cutoff_is_summed_exactly(name):
    # One grid bin per coarse bin except a wide one around the proposal's cutoff: the narrow
    # bins are exact, the wide one is the exact range (summed bin by bin up to the cutoff) and
    # the bins above contribute nothing, so the compressed ln L is the full one.
    w, ev = event(name)
    th = ev.theta_inj.copy()
    k_end = relbin.active_bins(ev, th, w.waveform)
    assert 40 < k_end < ev.n_bins - 40
    lo, hi = k_end - 20, k_end + 30
    edges = np.concatenate([np.arange(0, lo + 1), np.arange(hi, ev.n_bins + 1)])
    sd = relbin.summary_data(ev, ev.theta_inj, edges, w.waveform)
    assert relbin.n_expanded(edges, k_end, ev.n_bins) == lo
    for t in (th, th + np.array([0, 0, 0, 0, 30.0, 0.1, 0.1, 0.2, 1e-4, 0.01, 0.01])):
        assert relbin.active_bins(ev, t, w.waveform) == k_end
        want = L.log_likelihood(ev, t, w.waveform)
        assert abs(relbin.log_likelihood(ev, t, sd, w.waveform) - want) <= 1e-9 * abs(want)
