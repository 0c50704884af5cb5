"""Pins of the oracle's acceptance walk and batched nested sampler."""
import math

import numpy as np
import pytest
from scipy import stats
from scipy.stats import norm

from oracle import nested, walk


def gaussian(mu, sig):
    mu = np.asarray(mu, dtype=np.float64)
    D = mu.shape[0]
    norm_c = D * math.log(sig * math.sqrt(2 * math.pi))

    def ll(u):
        return -0.5 * float(np.sum(((u - mu) / sig) ** 2)) - norm_c

    exact = float(np.sum(np.log(norm.cdf((1 - mu) / sig) - norm.cdf(-mu / sig))))
    return ll, exact


@pytest.mark.parametrize("D,mu,sig,n_live", [(2, 0.5, 0.05, 200), (4, 0.5, 0.08, 200), (4, 0.03, 0.05, 200)])
def test_gaussian_evidence_closed_form(D, mu, sig, n_live):
    # Z = prod_d [Phi((1-mu)/sig) - Phi(-mu/sig)] for a normalised Gaussian in U[0,1]^D;
    # the third case puts the peak next to a face of the cube (truncated Gaussian).
    ll, exact = gaussian(np.full(D, mu), sig)
    r = nested.run_nested(ll, D, n_live, n_live // 2, 20, 5000, np.zeros(D, bool), (11, D))
    assert abs(r.log_z - exact) < 3.5 * r.log_z_err + 0.05
    assert 0.02 < r.log_z_err < 1.0
    # Posterior mean from the weights recovers the truncated-Gaussian mean.
    u, lw = r.samples()
    mean = np.sum(np.exp(lw)[:, None] * u, axis=0)
    a, b = (0 - mu) / sig, (1 - mu) / sig
    tmean = mu + sig * (norm.pdf(a) - norm.pdf(b)) / (norm.cdf(b) - norm.cdf(a))
    assert np.all(np.abs(mean - tmean) < 5 * sig / math.sqrt(n_live))


@pytest.mark.slow
def test_gaussian_evidence_eleven_dims():
    ll, exact = gaussian(np.full(11, 0.5), 0.1)
    r = nested.run_nested(ll, 11, 300, 150, 30, 5000, np.zeros(11, bool), (5, 11))
    assert abs(r.log_z - exact) < 3.5 * r.log_z_err + 0.05


def test_shrinkage_after_one_batch():
    # After one batch of k deletions log X = -sum_{i<k} 1/(n - i) exactly (Sec. 3.2.1).
    ll, _ = gaussian([0.5, 0.5], 0.1)
    n, k = 60, 30
    r = nested.run_nested(ll, 2, n, k, 5, 50, np.zeros(2, bool), (1, 1), max_iter=1)
    assert abs(np.sum(-1.0 / r.dead_nlive) - (-sum(1.0 / (n - i) for i in range(k)))) < 1e-14
    assert list(r.dead_nlive) == list(range(n, n - k, -1))
    assert r.n_iter == 1


def test_n_gpu_rule():
    # Sec. 3.2.1: with k = n/2 the shrinkage per batch is ~ ln 2, so n_GPU = 2 ln2 n_CPU.
    n = 1400
    shrink = sum(1.0 / (n - i) for i in range(n // 2))
    assert abs(shrink - math.log(2)) < 1e-3
    assert abs(n / 2 / shrink - 1010) < 1.0


def test_walk_preserves_uniform_law():
    # With L* = -inf every in-bounds proposal is accepted; DE moves with a uniform
    # survivor set leave U[0,1]^D invariant (periodic dims wrap).
    D, W = 3, 400
    rng = np.random.default_rng(0)
    surv = rng.random((200, D))
    u0 = rng.random((W, D))
    u, lnl, n_acc, n_like, _ = walk.acceptance_walk(lambda x: 0.0, u0, np.zeros(W), -np.inf, surv, 25,
                                                    np.array([False, True, False]), (3, 4), 0)
    assert np.all(n_acc <= 25) and np.all(n_acc == n_like)
    for d in range(D):
        assert stats.kstest(u[:, d], "uniform").pvalue > 1e-3
    assert np.all((u >= 0) & (u <= 1))


def test_walk_stays_in_constrained_ball_and_is_uniform_there():
    # Constraint |u - c| < R: the walk targets the uniform law on the ball, so the
    # radius follows P(r < x) = (x/R)^D.
    D, W, R = 2, 300, 0.3
    c = np.full(D, 0.5)
    rng = np.random.default_rng(1)
    # survivors: uniform inside the ball (rejection)
    s = rng.random((20000, D))
    s = s[np.linalg.norm(s - c, axis=1) < R][:300]
    u0 = s[rng.integers(0, 300, W)]
    ll = lambda x: -float(np.linalg.norm(x - c))
    u, lnl, n_acc, _, _ = walk.acceptance_walk(ll, u0, np.array([ll(x) for x in u0]), -R, s, 40,
                                               np.zeros(D, bool), (2, 2), 0)
    r = np.linalg.norm(u - c, axis=1)
    assert np.all(r < R)
    assert stats.kstest(r, lambda x: np.clip(x / R, 0, 1) ** D).pvalue > 1e-3
    assert n_acc.mean() > 5


def test_walk_ties_reject_and_returns_start():
    # A flat likelihood equal to L*: every proposal ties and is rejected (strict >).
    u0 = np.full((5, 2), 0.5)
    u, lnl, n_acc, n_like, _ = walk.acceptance_walk(lambda x: 1.0, u0, np.ones(5), 1.0,
                                                    np.random.default_rng(0).random((10, 2)), 10,
                                                    np.zeros(2, bool), (0, 0), 0)
    assert np.all(n_acc == 0) and np.array_equal(u, u0) and np.all(n_like > 0)


def test_insertion_ranks_uniform():
    # Each new live point is an independent draw from the constrained prior, so its
    # rank among the survivors (by ln L) is uniform (Fowlie, Handley & Su 2020).
    ll, _ = gaussian([0.5, 0.5], 0.1)
    n, k = 100, 50
    key = (7, 7)
    ranks = []
    u = nested.initial_live_points(n, 2, key)
    lnl = np.array([ll(x) for x in u])
    n_steps = 60
    for it in range(12):
        order = np.lexsort((np.arange(n), lnl))
        dead, surv = order[:k], order[k:]
        starts = surv[nested.start_indices(k, it, n - k, key)]
        new_u, new_lnl, n_acc, _, _ = walk.acceptance_walk(ll, u[starts], lnl[starts], lnl[dead[-1]],
                                                           u[surv], n_steps, np.zeros(2, bool), key, it)
        if it >= 2:
            sl = np.sort(lnl[surv])
            ranks.extend(np.searchsorted(sl, new_lnl) / (n - k))
        u[dead], lnl[dead] = new_u, new_lnl
    assert stats.kstest(np.array(ranks), "uniform").pvalue > 1e-3


def test_sequential_and_batched_agree():
    # k = 1 with n live points and k = n/2 with n_GPU = 2 ln2 n agree within errors (Sec. 4.3).
    ll, exact = gaussian([0.4, 0.6], 0.07)
    seq = nested.run_nested(ll, 2, 70, 1, 10, 500, np.zeros(2, bool), (8, 1))
    bat = nested.run_nested(ll, 2, 100, 50, 10, 500, np.zeros(2, bool), (8, 2))
    tol = 3.5 * math.hypot(seq.log_z_err, bat.log_z_err)
    assert abs(seq.log_z - bat.log_z) < tol
    assert abs(seq.log_z - exact) < 3.5 * seq.log_z_err + 0.05


def test_retune_rule():
    assert nested.batch_delay(59.0, 1) == pytest.approx(59.0)
    assert nested.batch_delay(59.0, 500) < 1e-3
    assert nested.retune(100, 30.0, 60, 0.0, 5000) == 200
    assert nested.retune(100, 0.0, 60, 0.0, 5000) == 5000
    assert nested.retune(3, 60.0, 60, 0.0, 5000) == 3


def test_flow_accept_weight_is_a_rescaled_target_when_every_step_is_a_flow_step():
    # With p_flow = 1 every accepted step is a flow step, so the weighted count w a of the
    # retune equals a at the target naccept / w: weight 4 at naccept 12 runs the chain of
    # weight 1 at naccept 3 (same delay and first walk length; the batch means stay above 1/2,
    # where the clamp of the rule would tell the two apart).  A dropped or misplaced (w - 1)
    # term, or flow acceptances not counted, changes the walk lengths and the chain.
    ll, _ = gaussian([0.5, 0.5], 0.15)
    kw = dict(delay=2.0, n_steps0=24, max_iter=4, p_flow=1.0, flow_epochs=5, flow_hidden=16, flow_layers=2)
    a = nested.run_nested(ll, 2, 24, 12, 12, 500, np.zeros(2, bool), (3, 4), flow_accept_weight=4.0, **kw)
    b = nested.run_nested(ll, 2, 24, 12, 3, 500, np.zeros(2, bool), (3, 4), **kw)
    assert [s[2] for s in a.stats] == [s[2] for s in b.stats]
    assert min(s[2] for s in a.stats) >= 0.5
    assert [s[1] for s in a.stats] == [s[1] for s in b.stats]
    assert len({s[1] for s in a.stats}) > 1                     # the walk length did move
    assert a.log_z == b.log_z and np.array_equal(a.dead_u, b.dead_u)
    # and weight 1 at naccept 12 walks longer (its count is a quarter of the weighted one)
    c = nested.run_nested(ll, 2, 24, 12, 12, 500, np.zeros(2, bool), (3, 4), **kw)
    assert c.stats[1][1] > a.stats[1][1]
