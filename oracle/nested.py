"""Batched nested sampling with the acceptance-walk inner kernel (Sec. 2.2.1, Sec. 2.2.3,
Sec. 3.1, Sec. 3.2, Sec. 3.2.1), expected-shrinkage evidence and posterior weights.

One batch (iteration `it`) of the sampler:
  1. order the live points by (ln L, index); the k = num_delete lowest die and
     ln L* is the largest ln L among them (Sec. 2.2.3);
  2. the dead points enter the evidence in ascending ln L with the live count falling
     n, n-1, ..., n-k+1 (the saw-tooth of Sec. 3.2): ln X_j = ln X_{j-1} - 1/(n - j)
     (expected shrinkage, Sec. 3.2.1), w_j = L_j (X_{j-1} - X_j), Z += w_j;
  3. each of the k walkers starts from a survivor drawn uniformly with replacement
     (Philox block (0, j, it, 2), word 0) and walks n_steps DE steps (oracle.walk);
  4. the k end points replace the dead slots; the walk length of the next batch is
     retuned from the batch mean accepted count a:
        n <- clamp(floor((delay_k n + n naccept / max(a, 1/2)) / (delay_k + 1) + 1/2), 1, maxmcmc)
     with delay_k / (delay_k + 1) = (delay / (delay + 1))^k, which equals the sequential
     smoothing at k = 1 (Sec. 3.2 makes delay a function of the batch size; the rule is
     not printed -- parity unpinned);
  5. stop when ln(Z + L_max X) - ln Z < dlogZ (Sec. 4.1.1), or, for the fractional rule,
     when the live evidence L_mean X is below the given fraction of Z (Sec. 4.2).
With a flow (p_flow > 0; the paper only motivates flows, Sec. 5): the flow starts from
oracle.flow.init_flow and, in every batch it % flow_every == 0, after the deletion, is
re-standardised and trained for flow_epochs full-batch Adam steps on the n_live - k
survivors, which sample the prior above the new L* that the walks target (warm start:
weights and Adam state persist); the walk then mixes flow steps with probability p_flow
(oracle.walk).  With flow_accept_weight w (a reading: the paper gives no walk-length rule for
flow steps), the retune of step 4 takes a = (sum of accepted steps + (w - 1) x sum of accepted
flow steps) / k: an accepted independence proposal counts as w DE acceptances; w = 1 is the
plain rule.
With inner="hrss" the walkers instead make hrss_steps hit-and-run slice-sampling moves each
(oracle.hrss; the inner kernel the paper names in Sec. 2.2 and Sec. 5) against the survivors,
with the same starts, deletion and evidence; the move count is fixed (no retuning).
The final live points each receive weight L_i X / n.  The logZ error is the standard
deviation over replays that draw every shrinkage factor t ~ Beta(n_j, 1).
Initial live points: u[i, d] from Philox block (i, d // 4, 0, 3), word d % 4.
A process pool (walk_pool) only spreads the DE walks of a batch over processes, in
contiguous walker ranges with their own walker ids; a walker's chain depends on its id
alone, so the result is the same as the one-process run's.
"""
import math
from dataclasses import dataclass, field

import numpy as np

from paper_2509_04336_gb300.synth import TERM_DLOGZ, TERM_FRAC_REMAINING

from .philox import philox4x64_vec, mulhi_vec, open_unit_vec
from .walk import acceptance_walk
from .hrss import hrss_walk
from . import flow as flowmod


def initial_live_points(n_live: int, n_dim: int, key) -> np.ndarray:
    i = np.arange(n_live, dtype=np.uint64)[:, None]
    d = np.arange(n_dim, dtype=np.uint64)[None, :]
    blk = philox4x64_vec(i, d // np.uint64(4), np.uint64(0), np.uint64(3), key)
    words = np.stack(blk, axis=-1)                      # [n, D, 4]
    pick = (np.arange(n_dim) % 4)[None, :, None]
    return open_unit_vec(np.take_along_axis(words, np.broadcast_to(pick, (n_live, n_dim, 1)), axis=2)[..., 0])


def start_indices(k: int, it: int, n_surv: int, key) -> np.ndarray:
    j = np.arange(k, dtype=np.uint64)
    blk = philox4x64_vec(np.uint64(0), j, np.uint64(it), np.uint64(2), key)
    return mulhi_vec(blk[0], n_surv)


def batch_delay(delay: float, k: int) -> float:
    if delay <= 0.0:
        return 0.0
    r = (delay / (delay + 1.0)) ** k
    return r / (1.0 - r)


def retune(n_steps: int, mean_accept: float, naccept: int, delay_k: float, maxmcmc: int) -> int:
    x = (delay_k * n_steps + n_steps * naccept / max(mean_accept, 0.5)) / (delay_k + 1.0)
    return int(min(max(math.floor(x + 0.5), 1), maxmcmc))


@dataclass
class NestedResult:
    log_z: float
    log_z_err: float
    info_h: float
    n_like: int
    n_iter: int
    dead_u: np.ndarray
    dead_lnl: np.ndarray
    dead_logw: np.ndarray
    dead_nlive: np.ndarray
    live_u: np.ndarray
    live_lnl: np.ndarray
    log_x: float
    stats: list = field(default_factory=list)

    def samples(self):
        """All points (dead then final live) with normalised log weights."""
        u = np.concatenate([self.dead_u, self.live_u])
        n = self.live_lnl.shape[0]
        logw = np.concatenate([self.dead_logw, self.live_lnl + self.log_x - math.log(n)])
        return u, logw - self.log_z


def log_z_replays(dead_lnl, dead_nlive, live_lnl, n_replay: int, rng) -> np.ndarray:
    """logZ under random shrinkage t_j ~ Beta(n_j, 1) (Skilling; Higson et al.)."""
    dead_lnl = np.asarray(dead_lnl)
    nl = np.asarray(dead_nlive, dtype=np.float64)
    n = live_lnl.shape[0]
    out = np.empty(n_replay)
    for r in range(n_replay):
        log_t = np.log(rng.random(nl.shape[0])) / nl
        log_x = np.cumsum(log_t)
        log_x_prev = np.concatenate([[0.0], log_x[:-1]])
        log_dx = log_x_prev + np.log1p(-np.exp(log_t))
        terms = np.concatenate([dead_lnl + log_dx, live_lnl + log_x[-1] - math.log(n)])
        m = terms.max()
        out[r] = m + math.log(np.sum(np.exp(terms - m)))
    return out


def _pooled_walk(pool, n_chunks, loglike, u0, lnl0, lnl_star, survivors, n_steps, periodic, key, it):
    """acceptance_walk over walker ranges in a process pool (same chains, same order)."""
    k = u0.shape[0]
    edges = np.linspace(0, k, max(1, n_chunks) + 1).astype(int)
    args = [(loglike, u0[a:b], lnl0[a:b], lnl_star, survivors, n_steps, periodic, key, it, np.arange(a, b))
            for a, b in zip(edges[:-1], edges[1:]) if b > a]
    parts = pool.starmap(acceptance_walk, args, chunksize=1)
    return tuple(np.concatenate([p[i] for p in parts]) for i in range(5))


def run_nested(loglike, n_dim: int, n_live: int, num_delete: int, naccept: int, maxmcmc: int,
               periodic, key, term_kind: int = TERM_DLOGZ, term_value: float = 0.1,
               delay: float | None = None, max_iter: int = 100000, n_replay: int = 200,
               initial_u=None, n_steps0: int | None = None, replay_seed: int = 12345,
               p_flow: float = 0.0, flow_every: int = 1, flow_epochs: int = 50, flow_lr: float = 3e-3,
               flow_hidden: int = 128, flow_layers: int = 8, flow_bf16: bool = False,
               flow_accept_weight: float = 1.0, inner: str = "de", hrss_steps: int = 0, walk_pool=None,
               walk_chunks: int = 1, progress=None) -> NestedResult:
    if inner not in ("de", "hrss"):
        raise ValueError("inner is 'de' or 'hrss'")
    k = num_delete
    if delay is None:
        delay = float(naccept - 1)
    delay_k = batch_delay(delay, k)
    u = initial_live_points(n_live, n_dim, key) if initial_u is None else np.array(initial_u, dtype=np.float64)
    lnl = np.array([loglike(x) for x in u])
    n_like = n_live
    n_steps = int(math.ceil(naccept / 0.25)) if n_steps0 is None else int(n_steps0)
    log_x, log_z = 0.0, -math.inf
    dead_u, dead_lnl, dead_logw, dead_nlive = [], [], [], []
    stats = []
    flow, adam = None, None
    if p_flow > 0.0:
        flow = flowmod.init_flow(n_dim, flow_hidden, flow_layers, key)
        adam = flowmod.Adam(flow.flat().size, flow_lr)
    it = 0
    while it < max_iter:
        order = np.lexsort((np.arange(n_live), lnl))
        dead, surv = order[:k], order[k:]
        lnl_star = lnl[dead[-1]]
        for j, idx in enumerate(dead):
            nj = n_live - j
            log_x_new = log_x - 1.0 / nj
            log_w = lnl[idx] + log_x_new + math.log(math.expm1(1.0 / nj))
            log_z = np.logaddexp(log_z, log_w)
            log_x = log_x_new
            dead_u.append(u[idx].copy())
            dead_lnl.append(lnl[idx])
            dead_logw.append(log_w)
            dead_nlive.append(nj)
        if flow is not None and it % flow_every == 0:
            flowmod.train(flow, u[surv], flow_epochs, adam, flow_bf16)
        starts = surv[start_indices(k, it, n_live - k, key)]
        n_accf = np.zeros(k, dtype=np.int64)   # accepted flow steps per walker
        if inner == "hrss":
            n_steps = hrss_steps
            new_u, new_lnl, n_acc, n_call = hrss_walk(loglike, u[starts], lnl[starts], lnl_star, u[surv],
                                                      n_steps, periodic, key, it)
        elif walk_pool is not None and flow is None:
            new_u, new_lnl, n_acc, n_call, _ = _pooled_walk(
                walk_pool, walk_chunks, loglike, u[starts], lnl[starts], lnl_star, u[surv], n_steps,
                periodic, key, it)
        else:
            new_u, new_lnl, n_acc, n_call, _ = acceptance_walk(
                loglike, u[starts], lnl[starts], lnl_star, u[surv], n_steps, periodic, key, it,
                flow=flow, p_flow=p_flow, flow_bf16=flow_bf16, flow_acc=n_accf)
        u[dead] = new_u
        lnl[dead] = new_lnl
        n_like += int(n_call.sum())
        mean_acc = float(n_acc.mean())
        stats.append((it, n_steps, mean_acc, int(n_call.sum()), lnl_star, log_z))
        if progress is not None:
            progress(stats[-1])
        eff = (float(n_acc.sum()) + (flow_accept_weight - 1.0) * float(n_accf.sum())) / k
        n_steps = retune(n_steps, eff, naccept, delay_k, maxmcmc)
        it += 1
        if term_kind == TERM_DLOGZ:
            if np.logaddexp(log_z, lnl.max() + log_x) - log_z < term_value:
                break
        elif term_kind == TERM_FRAC_REMAINING:
            m = lnl.max()
            log_live = m + math.log(np.mean(np.exp(lnl - m))) + log_x
            if log_live - log_z < math.log(term_value):
                break
    m = lnl.max()
    log_z_final = np.logaddexp(log_z, m + math.log(np.sum(np.exp(lnl - m))) + log_x - math.log(n_live))
    d_lnl = np.array(dead_lnl)
    d_logw = np.array(dead_logw)
    all_lnl = np.concatenate([d_lnl, lnl])
    all_logw = np.concatenate([d_logw, lnl + log_x - math.log(n_live)])
    p = np.exp(all_logw - log_z_final)
    info_h = float(np.sum(p * all_lnl) - log_z_final)
    reps = log_z_replays(d_lnl, dead_nlive, lnl, n_replay, np.random.default_rng(replay_seed))
    return NestedResult(float(log_z_final), float(np.std(reps)), info_h, n_like, it,
                        np.array(dead_u), d_lnl, d_logw, np.array(dead_nlive), u, lnl, log_x, stats)
