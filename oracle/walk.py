"""Differential-evolution acceptance walk under the hard likelihood constraint
(Sec. 3.1 and its footnote on the DE scale; batch form of Sec. 2.2.3).

Each of the W walkers runs n_steps steps in the unit hypercube.  At step t walker w:
  1. draws two distinct survivors a != b uniformly from the live points that remain
     after the batch deletion (Philox block (t, w, it, 0): words 0, 1);
  2. draws the scale: s = 1 with probability 1/2 (word 2, top bit set), otherwise
     s = 2.38 / sqrt(2 D) * g with g ~ Gamma(shape 4, scale 0.25), drawn exactly as
     g = -0.25 ln(U0 U1 U2 U3) from Philox block (t, w, it, 1);
  3. proposes u' = u + s (u_a - u_b); periodic dimensions are wrapped into [0, 1),
     a non-periodic coordinate outside [0, 1] rejects the step without a likelihood call;
  4. accepts iff ln L(u') > ln L*  (strict; ties reject).
The Philox key is (seed, event).  Returns the final positions, their ln L, the
accepted-step counts and the number of likelihood calls of each walker.

Flow steps (the paper only motivates flows, Sec. 5): with a flow q
(oracle.flow) and probability p_flow, step t is instead an independence proposal
u' = F^-1(x), x ~ N(0, I) (oracle.flow.base_normals, flow_step_draws).  It is accepted iff
ln U < ln q(u) - ln q(u') and ln L(u') > ln L*, a Metropolis-Hastings step for the uniform
prior restricted to L > L*.  The q-ratio test is taken first, so a rejected ratio costs no
likelihood call; ln q of the current point is carried along (re-evaluated after an
accepted DE move).
"""
import math

import numpy as np

from .philox import philox4x64_vec, mulhi_vec, open_unit_vec
from . import flow as flowmod

DE_SCALE = 2.38


def de_step_draws(t: int, walkers: np.ndarray, it: int, n_surv: int, n_dim: int, key):
    """Survivor indices a, b and the DE scale s of step t for the given walker ids."""
    w = np.asarray(walkers, dtype=np.uint64)
    A = philox4x64_vec(np.uint64(t), w, np.uint64(it), np.uint64(0), key)
    B = philox4x64_vec(np.uint64(t), w, np.uint64(it), np.uint64(1), key)
    a = mulhi_vec(A[0], n_surv)
    b = mulhi_vec(A[1], n_surv - 1)
    b = b + (b >= a)
    unit_scale = (A[2] >> np.uint64(63)) == np.uint64(1)
    prod = open_unit_vec(B[0]) * open_unit_vec(B[1]) * open_unit_vec(B[2]) * open_unit_vec(B[3])
    gamma = -0.25 * np.log(prod)
    s = np.where(unit_scale, 1.0, DE_SCALE / math.sqrt(2.0 * n_dim) * gamma)
    return a, b, s


def acceptance_walk(loglike, u0, lnl0, lnl_star, survivors, n_steps, periodic, key, it,
                    walker_ids=None, flow=None, p_flow=0.0, flow_bf16=False, flow_acc=None):
    """Run the walk for every walker.  loglike(u [D]) -> float; survivors [n_s, D].
    The returned margin is, per walker, the smallest distance of any accept decision from
    its threshold: |ln L(u') - ln L*| and, on flow steps, |ln U - (ln q(u) - ln q(u'))|.
    flow_acc (an integer array [W], if given) receives each walker's accepted flow steps,
    which n_acc includes."""
    u = np.array(u0, dtype=np.float64, copy=True)
    lnl = np.array(lnl0, dtype=np.float64, copy=True)
    W, D = u.shape
    survivors = np.asarray(survivors, dtype=np.float64)
    n_s = survivors.shape[0]
    periodic = np.asarray(periodic, dtype=bool)
    ids = np.arange(W) if walker_ids is None else np.asarray(walker_ids)
    n_acc = np.zeros(W, dtype=np.int64)
    n_like = np.zeros(W, dtype=np.int64)
    margin = np.full(W, np.inf)   # smallest distance of a decision from its threshold
    use_flow = flow is not None and p_flow > 0.0
    if use_flow:
        _, logq = flowmod.forward(flow, u, flow_bf16)
    for t in range(n_steps):
        a, b, s = de_step_draws(t, ids, it, n_s, D, key)
        prop = u + s[:, None] * (survivors[a] - survivors[b])
        prop = np.where(periodic[None, :], prop - np.floor(prop), prop)
        if use_flow:
            fstep, log_u = flowmod.flow_step_draws(t, ids, it, p_flow, key)
            fu, fq = flowmod.inverse(flow, flowmod.base_normals(t, ids, it, D, key), flow_bf16)
            prop = np.where(fstep[:, None], fu, prop)
        inside = np.all((prop >= 0.0) & (prop <= 1.0), axis=1)
        for w in range(W):
            if not inside[w]:
                continue
            if use_flow and fstep[w]:
                ratio = logq[w] - fq[w]
                margin[w] = min(margin[w], abs(log_u[w] - ratio))
                if not log_u[w] < ratio:
                    continue
            val = loglike(prop[w])
            n_like[w] += 1
            margin[w] = min(margin[w], abs(val - lnl_star))
            if val > lnl_star:
                u[w] = prop[w]
                lnl[w] = val
                n_acc[w] += 1
                if use_flow:
                    logq[w] = fq[w] if fstep[w] else flowmod.forward(flow, prop[w:w + 1], flow_bf16)[1][0]
                    if fstep[w] and flow_acc is not None:
                        flow_acc[w] += 1
    return u, lnl, n_acc, n_like, margin
