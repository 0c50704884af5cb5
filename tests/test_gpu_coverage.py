"""Percentile-percentile coverage of a seeded injection study (the paper's Sec. 4.2 test on a
synthetic set): 96 noisy 4-parameter events, true values drawn from the sampler's prior, all
sampled in one handle to their stopping rule.  The posterior percentiles of the true values
must be uniform (Kolmogorov-Smirnov) for every sampled parameter."""
import numpy as np
import pytest

from oracle import likelihood as L
from paper_2509_04336_gb300 import injection, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2509_04336_gb300 import build
    build.build()


def test_pp_coverage_of_injection_study():
    stats = pytest.importorskip("scipy.stats")
    ws = synth.injection_set(96, seed=500)
    evs = [synth.make_event(w, L.project, L.inner) for w in ws]
    pri = [synth.priors_with_injection(w, e) for w, e in zip(ws, evs)]
    res = injection.run(ws, evs, pri)
    assert res["done"]
    pct = res["percentiles"]
    assert pct.shape == (96, 4) and np.all((pct >= 0) & (pct <= 1))
    pvals = [stats.kstest(pct[:, j], "uniform").pvalue for j in range(pct.shape[1])]
    print("KS p-values (Mc, q, chi1, chi2):", np.round(pvals, 4), "wall", round(res["wall_s"], 2), "s")
    assert min(pvals) > 1e-3, pvals
    # 90 % credible intervals (5 %..95 % percentiles) hold the truth in ~90 % of the events
    inside = np.mean((pct > 0.05) & (pct < 0.95))
    assert 0.8 < inside < 0.97, inside
    assert np.all(np.isfinite(res["log_z"])) and np.all(res["log_z_err"] > 0)


def test_pp_coverage_eleven_parameters_paper_setting():
    # The paper's injection-study setting (Sec. 4.2) on synthetic data: 100 signals with all
    # 11 parameters drawn from the priors (Mc [20, 50], q [0.5, 1], spins [-0.8, 0.8], the rest
    # as Table 1; no SNR rescaling, so the SNR spans ~1 to ~13), three detectors, seeded noise,
    # 1400 live points, num_delete 700, naccept 60, stop when the live points hold < 0.1 % of
    # the evidence.  Every parameter's percentiles must be uniform.
    from dataclasses import replace
    from oracle import prior as P
    stats = pytest.importorskip("scipy.stats")
    base = synth.workload("bbh11_3det_4s_taylorf2")
    pri = synth._standard_priors((20.0, 50.0), (0.5, 1.0), (-0.8, 0.8))
    rng = np.random.Generator(np.random.Philox(key=np.array([700, 6666], dtype=np.uint64)))
    ws, evs, pris = [], [], []
    for e in range(100):
        theta = P.transform(rng.random(11), pri)
        w = replace(base, name=f"pp11_{e}", priors=pri, injection=theta, noise=True, seed=700 + e, n_live=1400,
                    num_delete=700, naccept=60, maxmcmc=5000, term_kind=synth.TERM_FRAC_REMAINING,
                    term_value=0.001, precision=synth.PREC_MIXED_FF)
        ev = synth.make_event(w, L.project, L.inner, rescale=False)
        ws.append(w)
        evs.append(ev)
        pris.append(synth.priors_with_injection(w, ev))
    res = injection.run(ws, evs, pris, max_batches=4000)
    assert res["done"]
    pct = res["percentiles"]
    assert pct.shape == (100, 11)
    pvals = [stats.kstest(pct[:, j], "uniform").pvalue for j in range(11)]
    print("KS p-values:", np.round(pvals, 4), "wall", round(res["wall_s"], 2), "s")
    assert min(pvals) > 1e-3, pvals
    inside = np.mean((pct > 0.05) & (pct < 0.95))
    assert 0.85 < inside < 0.95, inside
