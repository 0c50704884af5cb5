"""Pins of the oracle's flow proposal (oracle.flow) and of flow steps in the walk: bfloat16
rounding against torch, forward o inverse, log q against a finite-difference Jacobian,
gradients against central differences, the 2-D density integrating to one, Adam's first
step, recovery of a Gaussian's entropy, and invariance of the uniform constrained prior
under the mixed DE + flow walk."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import flow as F
from oracle import walk
from oracle.nested import run_nested

KEY = (7, 0)


def random_flow(D, H, L, seed, scale=0.3, mu=None, sigma=None):
    """A flow with every parameter random (W3 and biases too), so no layer is the identity."""
    f = F.Flow(D, H, L)
    rng = np.random.default_rng(seed)
    f.set_flat(rng.normal(0.0, scale, f.n_params()))
    f.mu = np.zeros(D) if mu is None else np.asarray(mu, float)
    f.sigma = np.ones(D) if sigma is None else np.asarray(sigma, float)
    return f


def interior(n, D, seed):
    return np.random.default_rng(seed).uniform(0.02, 0.98, size=(n, D))


# ------------------------------------------------------------------ bfloat16 rounding
def test_bf16_rounding_ties_and_torch():
    torch = pytest.importorskip("torch")
    one = 1.0
    assert F.round_bf16(one + 2.0 ** -8) == 1.0                  # tie -> even (mantissa 0)
    assert F.round_bf16(one + 3 * 2.0 ** -8) == one + 2.0 ** -6  # tie -> even (mantissa 2)
    assert F.round_bf16(one + 2.0 ** -8 + 2.0 ** -20) == one + 2.0 ** -7
    assert F.round_bf16(-(one + 3 * 2.0 ** -8)) == -(one + 2.0 ** -6)
    x = np.random.default_rng(1).normal(0.0, 3.0, 20000).astype(np.float32).astype(np.float64)
    x = np.concatenate([x, np.float32(np.linspace(-2, 2, 4097)).astype(np.float64)])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(F.round_bf16(x), ref)


# ------------------------------------------------------------------ bijection and density
@pytest.mark.parametrize("bf16", [False, True])
def test_forward_inverse_identity(bf16):
    f = random_flow(5, 16, 4, 3, mu=[0.1, -0.3, 0.0, 0.5, -1.0], sigma=[0.7, 1.3, 1.0, 0.4, 2.0])
    u = interior(200, 5, 4)
    x, lq = F.forward(f, u, bf16)
    u2, lq2 = F.inverse(f, x, bf16)
    np.testing.assert_allclose(u2, u, rtol=0, atol=1e-12)
    np.testing.assert_allclose(lq2, lq, rtol=0, atol=1e-10)


def test_logq_matches_finite_difference_jacobian():
    D = 4
    f = random_flow(D, 16, 4, 5, mu=[0.2, -0.1, 0.3, 0.0], sigma=[0.9, 1.1, 0.6, 1.4])
    u = interior(12, D, 6)
    _, lq = F.forward(f, u)
    h = 1e-6
    for i in range(u.shape[0]):
        J = np.empty((D, D))
        for d in range(D):
            up, um = u[i:i + 1].copy(), u[i:i + 1].copy()
            up[0, d] += h
            um[0, d] -= h
            J[:, d] = (F.forward(f, up)[0][0] - F.forward(f, um)[0][0]) / (2 * h)
        x = F.forward(f, u[i:i + 1])[0][0]
        ref = -0.5 * x @ x - 0.5 * D * math.log(2 * math.pi) + np.linalg.slogdet(J)[1]
        assert abs(lq[i] - ref) < 1e-6


def test_coupling_logdet_is_sum_of_scales():
    """One affine coupling layer: log|det| is the analytic sum of its log-scales."""
    D = 3
    f = random_flow(D, 8, 1, 8)
    z = np.random.default_rng(9).normal(size=(5, D))
    m = f.mask[0]
    s, t, _ = F._coupling_net(f, 0, m * z, False)
    out = lambda zz: m * zz + (1 - m) * (zz * np.exp(F._coupling_net(f, 0, m * zz, False)[0])
                                         + F._coupling_net(f, 0, m * zz, False)[1])
    h = 1e-6
    for i in range(z.shape[0]):
        J = np.empty((D, D))
        for d in range(D):
            zp, zm = z[i:i + 1].copy(), z[i:i + 1].copy()
            zp[0, d] += h
            zm[0, d] -= h
            J[:, d] = (out(zp)[0] - out(zm)[0]) / (2 * h)
        assert abs(np.linalg.slogdet(J)[1] - s[i].sum()) < 1e-7
        assert np.all(np.abs(s[i][m == 1]) == 0)        # conditioning dimensions are unscaled


def test_density_integrates_to_one_2d():
    f = random_flow(2, 16, 4, 11, scale=0.4, mu=[0.3, -0.2], sigma=[0.8, 1.2])
    n = 1200
    g = (np.arange(n) + 0.5) / n
    uu = np.stack(np.meshgrid(g, g, indexing="ij"), axis=-1).reshape(-1, 2)
    _, lq = F.forward(f, uu)
    total = np.exp(lq).sum() / n ** 2
    assert abs(total - 1.0) < 2e-3


def test_samples_follow_the_density_2d():
    f = random_flow(2, 16, 4, 12, scale=0.4, mu=[0.3, -0.2], sigma=[0.8, 1.2])
    n = 800
    g = (np.arange(n) + 0.5) / n
    uu = np.stack(np.meshgrid(g, g, indexing="ij"), axis=-1).reshape(-1, 2)
    p = np.exp(F.forward(f, uu)[1]) / n ** 2
    mean_grid = (p[:, None] * uu).sum(axis=0) / p.sum()
    x = np.random.default_rng(13).normal(size=(40000, 2))
    u, lq = F.inverse(f, x)
    se = u.std(axis=0) / math.sqrt(u.shape[0])
    assert np.all(np.abs(u.mean(axis=0) - mean_grid) < 5 * se)
    # the log-density the sampler reports is the density at the sample
    np.testing.assert_allclose(lq, F.forward(f, u)[1], atol=1e-9)


def test_base_normals_are_standard_normal():
    x = F.base_normals(3, np.arange(5000), 2, 11, KEY)
    assert x.shape == (5000, 11)
    for d in range(11):
        assert stats.kstest(x[:, d], "norm").pvalue > 1e-3
    assert abs(np.corrcoef(x[:, 0], x[:, 1])[0, 1]) < 0.05


# ------------------------------------------------------------------ gradients and training
def test_gradient_matches_central_differences():
    f = random_flow(3, 8, 3, 21, scale=0.5, mu=[0.1, 0.2, -0.3], sigma=[0.8, 1.1, 0.9])
    u = interior(25, 3, 22)
    loss, g = F.loss_and_grad(f, u)
    p0 = f.flat()
    rng = np.random.default_rng(23)
    idx = np.unique(np.concatenate([rng.choice(p0.size, 60, replace=False),
                                    [0, p0.size - 1, 3 * 8 + 8]]))
    h = 1e-6
    for i in idx:
        pp, pm = p0.copy(), p0.copy()
        pp[i] += h
        pm[i] -= h
        f.set_flat(pp)
        lp = F.loss_and_grad(f, u)[0]
        f.set_flat(pm)
        lm = F.loss_and_grad(f, u)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    f.set_flat(p0)
    assert abs(loss + F.forward(f, u)[1].mean()) < 1e-12


def test_bf16_gradient_close_to_fp64():
    f = random_flow(11, 32, 4, 31, scale=0.2)
    u = interior(64, 11, 32)
    _, g64 = F.loss_and_grad(f, u, False)
    _, g16 = F.loss_and_grad(f, u, True)
    assert np.linalg.norm(g16 - g64) < 3e-2 * np.linalg.norm(g64)


def test_adam_first_step_is_signed_learning_rate():
    a = F.Adam(5, lr=0.01)
    g = np.array([3.0, -2.0, 1e-3, -1e-5, 0.0])
    p = a.step(np.zeros(5), g)
    np.testing.assert_allclose(p, -0.01 * g / (np.abs(g) + F.ADAM_EPS), rtol=1e-12, atol=0)
    m0 = a.m.copy()
    p2 = a.step(p, np.array([np.nan, 0, 0, 0, 0]))   # a non-finite component is skipped
    assert p2[0] == p[0] and a.m[0] == m0[0] and a.t == 2
    # the others take an ordinary second step: m = 0.9 m1, v = 0.999 v1
    mh = 0.9 * m0[1:] / (1 - 0.9 ** 2)
    vh = 0.999 * (0.001 * g[1:] ** 2) / (1 - 0.999 ** 2)
    np.testing.assert_allclose(p2[1:], p[1:] - 0.01 * mh / (np.sqrt(vh) + F.ADAM_EPS), rtol=1e-12, atol=1e-15)


def test_initial_flow_is_standardised_identity():
    f = F.init_flow(4, 16, 3, KEY)
    u = interior(50, 4, 41)
    F.standardise(f, u)
    z, lq = F.forward(f, u)
    lg = np.log(u) - np.log1p(-u)
    np.testing.assert_allclose(z, (lg - lg.mean(0)) / lg.std(0), atol=1e-12)
    assert np.all(np.abs(f.W1[0]) <= 1 / 2 + 1e-15) and np.all(f.W3[0] == 0)
    assert np.std(f.W2[1]) > 0.5 / math.sqrt(3 * 16)


def test_training_recovers_gaussian_entropy():
    rng = np.random.default_rng(51)
    cov = np.array([[1.0, 0.8], [0.8, 1.0]]) * 0.25
    mean = np.array([0.5, -0.7])
    z = rng.multivariate_normal(mean, cov, size=2000)
    u = 1.0 / (1.0 + np.exp(-z))
    # exact mean negative log-density of the generating law in the unit square
    diff = z - mean
    logn = (-0.5 * np.einsum("ij,jk,ik->i", diff, np.linalg.inv(cov), diff)
            - 0.5 * np.linalg.slogdet(2 * math.pi * cov)[1])
    true_nll = -(logn - np.sum(np.log(u) + np.log1p(-u), axis=1)).mean()
    f = F.init_flow(2, 32, 4, KEY)
    adam = F.Adam(f.flat().size, lr=3e-3)
    losses = F.train(f, u, 300, adam)
    final = F.loss_and_grad(f, u)[0]
    assert losses[0] > true_nll + 0.3            # standardisation alone misses the correlation
    assert abs(final - true_nll) < 0.05


# ------------------------------------------------------------------ flow steps in the walk
def test_mixed_walk_preserves_uniform_prior():
    """ln L constant, L* = -inf: the DE + flow walk must leave U[0,1]^2 invariant even with a
    strongly non-uniform q (a wrong q-ratio would pull the points towards q)."""
    f = random_flow(2, 8, 2, 61, scale=0.3, mu=[0.8, -0.5], sigma=[0.5, 0.6])
    W = 3000
    u0 = np.random.default_rng(62).random((W, 2))
    surv = np.random.default_rng(63).random((500, 2))
    u, _, n_acc, n_like, _ = walk.acceptance_walk(lambda x: 0.0, u0, np.zeros(W), -np.inf, surv, 12,
                                                  np.array([False, True]), KEY, 0, flow=f, p_flow=0.6)
    for d in range(2):
        assert stats.kstest(u[:, d], "uniform").pvalue > 1e-3
    # the independence sampler accepts a fraction E[min(1, q(u)/q(u'))] < 1 of flow steps
    assert 0 < n_like.sum() < 12 * W


def test_mixed_walk_without_flow_is_the_de_walk():
    surv = np.random.default_rng(71).random((50, 3))
    u0 = surv[:4]
    ll = lambda x: -np.sum((x - 0.5) ** 2)
    lnl0 = np.array([ll(x) for x in u0])
    a = walk.acceptance_walk(ll, u0, lnl0, -0.3, surv, 20, np.zeros(3, bool), KEY, 1)
    b = walk.acceptance_walk(ll, u0, lnl0, -0.3, surv, 20, np.zeros(3, bool), KEY, 1,
                             flow=random_flow(3, 8, 2, 72), p_flow=0.0)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_nested_with_flow_gaussian_evidence():
    """Gaussian likelihood inside the unit square: ln Z = ln of the captured mass (~0)."""
    mu, sig = np.array([0.45, 0.55]), 0.05
    ll = lambda x: -0.5 * np.sum(((x - mu) / sig) ** 2) - 2 * math.log(sig) - math.log(2 * math.pi)
    r = run_nested(ll, 2, 100, 50, 10, 500, np.zeros(2, bool), (3, 0), max_iter=60,
                   p_flow=0.5, flow_epochs=10, flow_hidden=16, flow_layers=2)
    truth = sum(math.log(stats.norm.cdf((1 - m) / sig) - stats.norm.cdf(-m / sig)) for m in mu)
    assert abs(r.log_z - truth) < 4 * max(r.log_z_err, 0.05)
