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
