"""Host logic of the injection study (no GPU): the posterior percentile of a true value."""
import numpy as np

from paper_2509_04336_gb300 import injection, synth


def test_percentile_of_weighted_samples():
    # equal weights: the fraction of samples below the truth
    th = np.zeros((5, 11))
    th[:, 0] = [1.0, 2.0, 3.0, 4.0, 5.0]
    truth = np.zeros(11)
    truth[0] = 3.5
    assert np.isclose(injection.percentiles(th, np.zeros(5), truth, [0])[0], 0.6)
    # log weights of any normalisation: weights 1, 1, 1, 1, 6 (of 10)
    lw = np.log([1, 1, 1, 1, 6]) + 123.0
    assert np.isclose(injection.percentiles(th, lw, truth, [0])[0], 0.3)


def test_percentiles_of_prior_draws_are_uniform():
    # truth and samples from the same distribution: the percentile is uniform
    rng = np.random.default_rng(3)
    pct = []
    for _ in range(400):
        th = np.zeros((200, 11))
        th[:, 2] = rng.normal(size=200)
        truth = np.zeros(11)
        truth[2] = rng.normal()
        pct.append(injection.percentiles(th, np.zeros(200), truth, [2])[0])
    pct = np.array(pct)
    assert abs(pct.mean() - 0.5) < 0.05 and abs(np.mean(pct < 0.1) - 0.1) < 0.04


def test_injection_set_draws_the_sampled_parameters_from_their_priors():
    ws = synth.injection_set(200, seed=9)
    w0 = synth.workload("four_param_2det_taylorf2")
    inj = np.stack([w.injection for w in ws])
    for i, p in enumerate(w0.priors):
        if p.kind == synth.UNIFORM:
            assert np.all((inj[:, i] >= p.lo) & (inj[:, i] <= p.hi))
            assert abs(np.mean((inj[:, i] - p.lo) / (p.hi - p.lo)) - 0.5) < 0.06
        else:
            assert np.all(inj[:, i] == w0.injection[i])
    assert len({w.seed for w in ws}) == 200 and all(w.noise for w in ws)
