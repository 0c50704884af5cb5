"""Hit-and-run slice sampling (HRSS) under the hard likelihood constraint -- the inner kernel
the paper names as the vectorised framework's original choice (Sec. 2.2) and as the direction
for GPU-native inner kernels (Sec. 5).  The oracle of that kernel, plain FP64 numpy, one
walker and one step at a time; test infrastructure (see the package header).

The method restated (Neal 2003, "Slice sampling", Sec. 4: stepping out and shrinkage; the
hit-and-run form draws a random line through the current point and slice-samples along it):
the target is the prior (uniform on the unit cube) restricted to ln L > ln L*, so the slice
along a line is S = {t : x + t d inside the cube (periodic coordinates wrapped), ln L > ln L*}.
Each step of walker w:
  1. direction d = C z / |z|, z ~ N(0, I_D), C the Cholesky factor of the covariance of the
     survivors of the batch deletion (unit-cube coordinates): lines follow the live points'
     shape, and d and -d are equally likely;
  2. bracket of width w0 placed at random around t = 0: lo = -w0 U, hi = lo + w0;
  3. stepping out with at most m widths: J = floor(m V) steps to the left and m - 1 - J to the
     right, each extending the bracket by w0 while its end is inside S;
  4. shrinkage: t ~ U(lo, hi); if x + t d is inside S it is the new point, otherwise the bracket
     shrinks to [t, hi] (t < 0) or [lo, t] (t > 0) and another t is drawn (at most
     max_shrink draws; after that the walker stays where it is).
A point outside the cube (non-periodic coordinates) is outside S without a likelihood call,
as in the DE walk.  Random numbers are Philox4x64-10 blocks (t, w, it, tag) under the key
(seed, event): tags 32 + c (c = 0, 1, 2) the normals z (Box-Muller, words (0, 1) and (2, 3)),
tag 40 the bracket draws (word 0: U, word 1: V), tags 48 + j // 4 word j % 4 the j-th shrinkage
draw.
"""
from __future__ import annotations

import math

import numpy as np

from .philox import philox4x64_vec, open_unit_vec

TAG_NORMAL = 32
TAG_BRACKET = 40
TAG_SHRINK = 48


def direction_factor(survivors) -> np.ndarray:
    """Lower Cholesky factor C of the survivors' sample covariance (unit-cube coordinates)."""
    s = np.asarray(survivors, dtype=np.float64)
    return np.linalg.cholesky(np.atleast_2d(np.cov(s, rowvar=False)))


def step_normals(t: int, walker: int, it: int, n_dim: int, key) -> np.ndarray:
    """z [n_dim] of step t of one walker (Box-Muller on blocks (t, w, it, 32 + c))."""
    out = []
    for c in range((n_dim + 3) // 4):
        blk = philox4x64_vec(np.uint64(t), np.array([walker], np.uint64), np.uint64(it),
                             np.uint64(TAG_NORMAL + c), key)
        for p in range(2):
            u1 = float(open_unit_vec(blk[2 * p])[0])
            u2 = float(open_unit_vec(blk[2 * p + 1])[0])
            r = math.sqrt(-2.0 * math.log(u1))
            out += [r * math.cos(2.0 * math.pi * u2), r * math.sin(2.0 * math.pi * u2)]
    return np.array(out[:n_dim])


def bracket_draws(t: int, walker: int, it: int, key):
    """(U, V) of step t: the bracket's placement and the split of the stepping-out budget."""
    blk = philox4x64_vec(np.uint64(t), np.array([walker], np.uint64), np.uint64(it), np.uint64(TAG_BRACKET), key)
    return float(open_unit_vec(blk[0])[0]), float(open_unit_vec(blk[1])[0])


def shrink_draw(t: int, walker: int, it: int, j: int, key) -> float:
    """The j-th shrinkage uniform of step t."""
    blk = philox4x64_vec(np.uint64(t), np.array([walker], np.uint64), np.uint64(it),
                         np.uint64(TAG_SHRINK + j // 4), key)
    return float(open_unit_vec(blk[j % 4])[0])


def slice_step(loglike, x, lnl_star, d, periodic, u, v, shrink_uniforms, width=1.0, max_out=10, margins=None):
    """One slice-sampling move of x along d.  shrink_uniforms: iterable of U(0, 1) draws.
    Returns (new x, its ln L or None if the walker stayed, likelihood calls, (lo, hi) of the
    final bracket, t of the move or None).  margins (a list, optional) receives |ln L - ln L*|
    of every evaluated point: how far each decision was from its threshold."""
    x = np.asarray(x, dtype=np.float64)
    periodic = np.asarray(periodic, dtype=bool)
    calls = 0

    def point(t):
        p = x + t * d
        return np.where(periodic, p - np.floor(p), p)

    def inside(t):
        """(in S, ln L) of the point at t; out-of-cube points cost no call."""
        nonlocal calls
        p = point(t)
        if np.any((p < 0.0) | (p > 1.0)):
            return False, None
        calls += 1
        lnl = loglike(p)
        if margins is not None:
            margins.append(abs(lnl - lnl_star))
        return lnl > lnl_star, lnl

    lo = -width * u
    hi = lo + width
    j_left = int(math.floor(max_out * v))
    k_right = (max_out - 1) - j_left
    while j_left > 0 and inside(lo)[0]:
        lo -= width
        j_left -= 1
    while k_right > 0 and inside(hi)[0]:
        hi += width
        k_right -= 1
    for s in shrink_uniforms:
        t = lo + (hi - lo) * s
        ok, lnl = inside(t)
        if ok:
            return point(t), lnl, calls, (lo, hi), t
        if t < 0.0:
            lo = t
        else:
            hi = t
    return x, None, calls, (lo, hi), None


def hrss_walk(loglike, u0, lnl0, lnl_star, survivors, n_steps, periodic, key, it, walker_ids=None,
              width=1.0, max_out=10, max_shrink=100, return_margin=False):
    """n_steps HRSS moves for every walker (rows of u0).  Returns (u, ln L, moves made,
    likelihood calls) per walker, and with return_margin the smallest |ln L - ln L*| of each
    walker's decisions (a walker whose margin is below another implementation's ln L error
    may legitimately take the other branch)."""
    u = np.array(u0, dtype=np.float64, copy=True)
    lnl = np.array(lnl0, dtype=np.float64, copy=True)
    W, D = u.shape
    ids = np.arange(W) if walker_ids is None else np.asarray(walker_ids)
    C = direction_factor(survivors)
    n_move = np.zeros(W, dtype=np.int64)
    n_like = np.zeros(W, dtype=np.int64)
    margin = np.full(W, np.inf)
    for w in range(W):
        wid = int(ids[w])
        ms = []
        for t in range(n_steps):
            z = step_normals(t, wid, it, D, key)
            d = C @ z / np.linalg.norm(z)
            uu, vv = bracket_draws(t, wid, it, key)
            draws = (shrink_draw(t, wid, it, j, key) for j in range(max_shrink))
            x, l, calls, _, tm = slice_step(loglike, u[w], lnl_star, d, periodic, uu, vv, draws, width, max_out, ms)
            n_like[w] += calls
            if tm is not None:
                u[w], lnl[w] = x, l
                n_move[w] += 1
        if ms:
            margin[w] = min(ms)
    if return_margin:
        return u, lnl, n_move, n_like, margin
    return u, lnl, n_move, n_like
