"""Pins of the oracle's counter-based RNG and unit-cube prior transforms."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import philox, prior, walk
from paper_2509_04336_gb300 import synth


@pytest.mark.parametrize("key,ctr", [((0, 0), (0, 0, 0, 0)), ((1, 2), (5, 0, 0, 0)),
                                     ((2**64 - 1, 7), (2**64 - 2, 3, 9, 2**63))])
def test_philox_matches_numpy(key, ctr):
    # numpy.random.Philox implements the same published Philox4x64-10 and increments
    # its counter (word 0, carrying) before producing each block.
    whole = sum(int(w) << (64 * i) for i, w in enumerate(ctr))
    whole = (whole - 1) % 2**256
    prev = [(whole >> (64 * i)) & (2**64 - 1) for i in range(4)]
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(prev, dtype=np.uint64))
    assert tuple(int(x) for x in bg.random_raw(4)) == philox.philox4x64(ctr, key)


def test_philox_vectorised_matches_scalar():
    rng = np.random.default_rng(3)
    c = rng.integers(0, 2**63, size=(50, 4), dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    key = (123456789012345, 2**63 + 5)
    vec = philox.philox4x64_vec(c[:, 0], c[:, 1], c[:, 2], c[:, 3], key)
    for i in range(50):
        assert tuple(int(v[i]) for v in vec) == philox.philox4x64(c[i], key)
    xs = rng.integers(0, 2**63, size=100, dtype=np.uint64)
    assert np.array_equal(philox.mulhi_vec(xs, 1000), [philox.mulhi(x, 1000) for x in xs])


def test_open_unit_range():
    assert philox.open_unit(0) > 0.0 and philox.open_unit(2**64 - 1) < 1.0


def test_de_scale_distribution():
    # Footnote of Sec. 3.1: with probability 1/2 the scale is 1, otherwise
    # 2.38/sqrt(2 D) * Gamma(shape 4, scale 0.25).
    D = 11
    ids = np.arange(20000)
    _, _, s = walk.de_step_draws(0, ids, 0, 100, D, (9, 9))
    unit = s == 1.0
    assert abs(unit.mean() - 0.5) < 0.02
    g = s[~unit] * math.sqrt(2 * D) / 2.38
    assert stats.kstest(g, stats.gamma(a=4, scale=0.25).cdf).pvalue > 1e-3


def test_de_pair_distinct_and_uniform():
    a, b, _ = walk.de_step_draws(3, np.arange(30000), 1, 7, 4, (1, 1))
    assert np.all(a != b) and a.min() >= 0 and b.max() <= 6
    counts = np.bincount(a, minlength=7)
    assert stats.chisquare(counts).pvalue > 1e-3
    counts = np.bincount(b, minlength=7)
    assert stats.chisquare(counts).pvalue > 1e-3


def _cdfs():
    two_pi = 2 * math.pi
    return [
        (synth.PriorEntry(synth.UNIFORM, 25.0, 50.0), lambda x: (x - 25.0) / 25.0),
        (synth.PriorEntry(synth.POWERLAW, 100.0, 5000.0, alpha=2.0),
         lambda x: (x ** 3 - 100.0 ** 3) / (5000.0 ** 3 - 100.0 ** 3)),
        (synth.PriorEntry(synth.SINE, 0.0, math.pi), lambda x: (1 - np.cos(x)) / 2),
        (synth.PriorEntry(synth.COSINE, -math.pi / 2, math.pi / 2), lambda x: (np.sin(x) + 1) / 2),
        (synth.PriorEntry(synth.UNIFORM, 0.0, two_pi, periodic=True), lambda x: x / two_pi),
    ]


@pytest.mark.parametrize("idx", range(5))
def test_prior_inverse_cdf(idx):
    # Table 1: each transform is the inverse of the prior's CDF, so CDF(T(u)) = u and
    # draws through T follow the prior (KS on 2e4 draws).
    entry, cdf = _cdfs()[idx]
    u = np.linspace(0.0, 1.0, 101)
    x = np.array([prior.transform_one(v, entry) for v in u])
    assert np.allclose(cdf(x), u, atol=1e-12)
    assert abs(x[0] - entry.lo) < 1e-9 and abs(x[-1] - entry.hi) < 1e-9
    draws = np.array([prior.transform_one(v, entry) for v in np.random.default_rng(idx).random(20000)])
    assert stats.kstest(draws, cdf).pvalue > 1e-3


def test_prior_density_matches_table1():
    # d_L power law 2 on [100, 5000] Mpc: density ~ d^2, normalised.
    e = synth.PriorEntry(synth.POWERLAW, 100.0, 5000.0, alpha=2.0)
    pri = [e]
    x = np.linspace(100, 5000, 200001)
    dens = np.exp([prior.log_prior_volume_density([v], pri) for v in x])
    assert abs(np.trapezoid(dens, x) - 1.0) < 1e-6


def test_fixed_parameters_pass_through():
    w = synth.workload("four_param_2det_taylorf2")
    th = prior.transform([0.5, 0.5, 0.5, 0.5], w.priors)
    assert th[0] == 30.0 and th[1] == 0.5625 and th[2] == 0.0
    assert np.allclose(th[5:], w.injection[5:])
    assert list(prior.periodic_mask(w.priors)) == [False] * 4
