"""Pins of the hit-and-run slice-sampling oracle (oracle/hrss.py).

The exact statements used: a slice-sampling move leaves the uniform distribution on the
constrained region invariant (Neal 2003, Sec. 4), so uniform starting points stay uniform
(checked through closed-form distributions of an interval, a ball and an ellipse); every
accepted point satisfies the constraint; the directions have covariance Sigma / D."""
import math

import numpy as np
import pytest

from oracle import hrss

KEY = (11, 0)


def _ks(x, cdf):
    stats = pytest.importorskip("scipy.stats")
    return stats.kstest(x, cdf).pvalue


def _ball_uniform(rng, n, d, c, r):
    g = rng.normal(size=(n, d))
    g /= np.linalg.norm(g, axis=1)[:, None]
    return c + r * g * rng.random(n)[:, None] ** (1.0 / d)


def test_interval_slice_keeps_uniform_points_uniform():
    # D = 1, ln L = -(x - c)^2, L* = -r^2: the region is (c - r, c + r); starts uniform there.
    rng = np.random.default_rng(1)
    c, r, n = 0.55, 0.2, 3000
    x0 = c - r + 2 * r * rng.random(n)
    like = lambda p: -float((p[0] - c) ** 2)
    u, l, moved, calls = hrss.hrss_walk(like, x0[:, None], [like([v]) for v in x0], -r * r, x0[:, None], 1,
                                        [False], KEY, 0)
    assert np.all(moved == 1)
    assert np.all(np.abs(u[:, 0] - c) < r) and np.all(l > -r * r)
    assert _ks(u[:, 0], lambda s: np.clip((s - (c - r)) / (2 * r), 0, 1)) > 1e-3


def test_cube_boundary_truncates_the_slice():
    # The region (c - r, c + r) reaches below 0: the slice is [0, c + r), and points outside
    # the cube cost no likelihood call.
    rng = np.random.default_rng(2)
    c, r, n = 0.05, 0.2, 3000
    hi = c + r
    x0 = hi * rng.random(n)
    count = {"n": 0}

    def like(p):
        count["n"] += 1
        assert 0.0 <= p[0] <= 1.0
        return -float((p[0] - c) ** 2)

    l0 = [-(v - c) ** 2 for v in x0]
    count["n"] = 0
    u, l, moved, calls = hrss.hrss_walk(like, x0[:, None], l0, -r * r, x0[:, None], 1, [False], KEY, 3)
    assert int(calls.sum()) == count["n"]
    assert np.all((u[:, 0] >= 0.0) & (u[:, 0] < hi))
    assert _ks(u[:, 0], lambda s: np.clip(s / hi, 0, 1)) > 1e-3


def test_ball_stays_uniform_in_three_dimensions():
    # Uniform points in a ball (|x - c| < R) after two moves: the radius has CDF (r / R)^3 and a
    # coordinate s = (x_1 - c_1) / R has CDF (3 s - s^3 + 2) / 4.
    rng = np.random.default_rng(3)
    D, R, n = 3, 0.3, 2000
    c = np.full(D, 0.5)
    x0 = _ball_uniform(rng, n, D, c, R)
    like = lambda p: -float(np.sum((p - c) ** 2))
    u, l, moved, _ = hrss.hrss_walk(like, x0, [like(p) for p in x0], -R * R, x0, 2, [False] * D, KEY, 1)
    assert np.all(moved == 2) and np.all(l > -R * R)
    rad = np.linalg.norm(u - c, axis=1) / R
    assert _ks(rad, lambda s: np.clip(s, 0, 1) ** 3) > 1e-3
    s = (u[:, 0] - c[0]) / R
    assert _ks(s, lambda v: (3 * np.clip(v, -1, 1) - np.clip(v, -1, 1) ** 3 + 2) / 4) > 1e-3
    # the walk moved the points: starts and ends are not the same sample
    assert np.mean(np.linalg.norm(u - x0, axis=1)) > 0.3 * R


def test_ellipse_with_covariance_directions():
    # A thin ellipse (semi-axes 0.3 and 0.03, rotated 30 degrees); the survivors' covariance
    # shapes the lines.  Mapped to the unit disc the points stay uniform: radius CDF r^2,
    # angle uniform.
    rng = np.random.default_rng(4)
    n = 2000
    c = np.array([0.5, 0.5])
    th = math.radians(30.0)
    Rot = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    M = Rot @ np.diag([0.3, 0.03])           # disc -> ellipse
    Minv = np.linalg.inv(M)
    x0 = c + _ball_uniform(rng, n, 2, np.zeros(2), 1.0) @ M.T
    like = lambda p: -float(np.sum((Minv @ (p - c)) ** 2))
    u, l, moved, calls = hrss.hrss_walk(like, x0, [like(p) for p in x0], -1.0, x0, 2, [False, False], KEY, 2)
    y = (u - c) @ Minv.T
    rad = np.linalg.norm(y, axis=1)
    ang = np.arctan2(y[:, 1], y[:, 0])
    assert np.all(rad < 1.0)
    assert _ks(rad, lambda s: np.clip(s, 0, 1) ** 2) > 1e-3
    assert _ks(ang, lambda a: (np.clip(a, -math.pi, math.pi) + math.pi) / (2 * math.pi)) > 1e-3
    # lines along the ellipse: a few likelihood calls per move, not dozens
    assert calls.mean() / 2 < 8.0


def test_directions_have_the_survivor_covariance():
    # d = C z / |z| with C C^T = Sigma: E[d d^T] = Sigma / D.
    rng = np.random.default_rng(5)
    A = rng.normal(size=(4, 4))
    surv = rng.normal(size=(5000, 4)) @ A.T * 0.01 + 0.5
    C = hrss.direction_factor(surv)
    sig = np.cov(surv, rowvar=False)
    assert np.allclose(C @ C.T, sig, rtol=1e-10, atol=1e-16)
    ds = []
    for w in range(6000):
        z = hrss.step_normals(0, w, 0, 4, KEY)
        ds.append(C @ z / np.linalg.norm(z))
    ds = np.array(ds)
    emp = ds.T @ ds / len(ds)
    assert np.allclose(emp, sig / 4, atol=0.06 * np.max(np.abs(sig)) / 4)
    assert np.allclose(ds.mean(axis=0), 0.0, atol=0.05 * math.sqrt(np.max(np.diag(sig))))


def test_step_normals_are_standard_normal():
    z = np.concatenate([hrss.step_normals(t, w, 7, 11, KEY) for t in range(3) for w in range(300)])
    stats = pytest.importorskip("scipy.stats")
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_bracket_contains_the_start_and_the_move():
    rng = np.random.default_rng(6)
    c, r = 0.5, 0.1
    like = lambda p: -float((p[0] - c) ** 2)
    for k in range(200):
        x = c - r + 2 * r * rng.random()
        d = np.array([0.03 + 0.3 * rng.random()]) * (1 if k % 2 else -1)
        uu, vv = rng.random(), rng.random()
        xs, l, calls, (lo, hi), t = hrss.slice_step(like, [x], -r * r, d, [False], uu, vv, iter(rng.random(100)))
        assert lo < 0.0 < hi and t is not None and lo < t < hi
        assert abs(xs[0] - c) < r and l == like(xs)
        assert abs(xs[0] - (x + t * d[0])) < 1e-15


def test_empty_slice_leaves_the_walker_in_place():
    # ln L* above the maximum: no point qualifies; the walker stays after max_shrink draws.
    x0 = np.array([[0.5, 0.5]])
    like = lambda p: -float(np.sum((p - 0.5) ** 2))
    surv = np.random.default_rng(7).random((50, 2))
    u, l, moved, calls = hrss.hrss_walk(like, x0, [0.0], 1.0, surv, 3, [False, False], KEY, 0, max_shrink=20)
    assert np.array_equal(u, x0) and moved[0] == 0 and l[0] == 0.0
    assert 3 * 20 <= calls[0] <= 3 * (20 + 9)


def test_periodic_coordinate_wraps():
    # A periodic coordinate with no constraint on it: moves wrap into [0, 1) and stay there.
    x0 = np.array([[0.95, 0.5]] * 200)
    like = lambda p: -float((p[1] - 0.5) ** 2)
    surv = np.random.default_rng(8).random((100, 2))
    u, l, moved, _ = hrss.hrss_walk(like, x0, [0.0] * 200, -0.04, surv, 2, [True, False], KEY, 0)
    assert np.all((u[:, 0] >= 0.0) & (u[:, 0] < 1.0)) and np.all(np.abs(u[:, 1] - 0.5) < 0.2)
    assert np.any(u[:, 0] < 0.5)   # some crossed the boundary at 1


def test_local_moves_keep_the_slice_edges_populated():
    # Lines much shorter than the region (survivor spread 0.01, at most 2 bracket widths): the
    # stepping-out budget runs out on most moves, where only the random split of the budget
    # between the two sides keeps the move reversible (Neal 2003, Sec. 4).  After 5 moves the
    # points within 0.02 of the region's ends must still hold 20 % of the mass.
    rng = np.random.default_rng(10)
    c, r, n = 0.5, 0.1, 4000
    x0 = c - r + 2 * r * rng.random(n)
    surv = (0.5 + 0.01 * rng.normal(size=200))[:, None]
    like = lambda p: -float((p[0] - c) ** 2)
    u, l, moved, calls = hrss.hrss_walk(like, x0[:, None], [like([v]) for v in x0], -r * r, surv, 5, [False],
                                        KEY, 0, max_out=2)
    edge = np.mean(np.abs(u[:, 0] - c) > r - 0.02)
    assert abs(edge - 0.2) < 4.0 * math.sqrt(0.2 * 0.8 / n), edge
    assert _ks(u[:, 0], lambda s: np.clip((s - (c - r)) / (2 * r), 0, 1)) > 1e-3


@pytest.mark.parametrize("D,mu,sig", [(2, 0.5, 0.05), (4, 0.03, 0.05)])
def test_sampler_with_hrss_gives_the_gaussian_evidence(D, mu, sig):
    # The batched sampler with HRSS as its inner kernel: Z of a normalised Gaussian in U[0,1]^D
    # is prod_d [Phi((1-mu)/sig) - Phi(-mu/sig)] (the second case truncated by a face).
    from scipy.stats import norm
    from oracle import nested
    c = D * math.log(sig * math.sqrt(2 * math.pi))
    ll = lambda u: -0.5 * float(np.sum(((u - mu) / sig) ** 2)) - c
    exact = D * math.log(norm.cdf((1 - mu) / sig) - norm.cdf(-mu / sig))
    r = nested.run_nested(ll, D, 200, 100, 20, 5000, np.zeros(D, bool), (13, D), inner="hrss", hrss_steps=2 * D)
    assert abs(r.log_z - exact) < 3.5 * r.log_z_err + 0.05, (r.log_z, exact, r.log_z_err)
    # every batch moved every walker
    assert all(st[2] == 2 * D for st in r.stats)


def test_hrss_insertion_ranks_uniform():
    # New points from HRSS moves are draws from the constrained prior: their ln L rank among
    # the survivors is uniform (Fowlie, Handley & Su 2020).
    from scipy import stats
    from oracle import nested
    c = math.log(0.1 * math.sqrt(2 * math.pi)) * 2
    ll = lambda u: -0.5 * float(np.sum(((u - 0.5) / 0.1) ** 2)) - c
    n, k, key = 100, 50, (7, 9)
    u = nested.initial_live_points(n, 2, key)
    lnl = np.array([ll(x) for x in u])
    ranks = []
    for it in range(12):
        order = np.lexsort((np.arange(n), lnl))
        dead, surv = order[:k], order[k:]
        starts = surv[nested.start_indices(k, it, n - k, key)]
        new_u, new_lnl, _, _ = hrss.hrss_walk(ll, u[starts], lnl[starts], lnl[dead[-1]], u[surv], 6,
                                              np.zeros(2, bool), key, it)
        if it >= 2:
            sl = np.sort(lnl[surv])
            ranks.extend(np.searchsorted(sl, new_lnl) / (n - k))
        u[dead], lnl[dead] = new_u, new_lnl
    assert stats.kstest(np.array(ranks), "uniform").pvalue > 1e-3


def test_margin_is_the_closest_decision():
    # The margin is the smallest |ln L - ln L*| over every evaluated candidate; it never exceeds
    # the distance of the accepted end point from the threshold.
    c = 0.5
    like = lambda p: -float(np.sum((p - c) ** 2))
    rng = np.random.default_rng(12)
    x0 = c + 0.1 * (rng.random((20, 2)) - 0.5)
    l0 = [like(p) for p in x0]
    star = -0.01
    u, l, moved, calls, margin = hrss.hrss_walk(like, x0, l0, star, x0, 2, [False, False], KEY, 0,
                                                return_margin=True)
    assert np.all(margin <= np.abs(l - star) + 1e-15)
    assert np.all(margin > 0.0) and np.all(np.isfinite(margin))
    u2, l2, m2, c2 = hrss.hrss_walk(like, x0, l0, star, x0, 2, [False, False], KEY, 0)
    assert np.array_equal(u, u2) and np.array_equal(calls, c2)
