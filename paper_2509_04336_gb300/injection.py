"""Injection study: many synthetic events sampled together in one handle, and the posterior
percentiles of their true parameters.

If the sampler is calibrated, the percentile of a true value (drawn from the prior the sampler
uses) within its posterior is uniform on [0, 1] across injections -- the paper's
percentile-percentile coverage test (Sec. 4.2), here on a seeded synthetic set.  The events
are independent problems sharing one batched launch per batch; this module only drives the
library's calls and reduces the posteriors it returns.
"""
from __future__ import annotations

import time

import numpy as np

from . import gwns


def percentiles(theta, logw, truth, sampled) -> np.ndarray:
    """Posterior weight below the true value, per sampled parameter: theta [m][11] samples,
    logw [m] log weights (any normalisation), truth [11]."""
    wgt = np.exp(np.asarray(logw) - np.max(logw))
    wgt /= wgt.sum()
    theta = np.asarray(theta)
    return np.array([float(np.sum(wgt[theta[:, i] < truth[i]])) for i in sampled])


def run(workloads, events, priors, max_batches: int = 2000, chunk: int = 8) -> dict:
    """Sample every event to its stopping rule and return, per event, the posterior percentile
    of each sampled parameter's true value, the evidence and the run statistics.

    workloads: synth.Workload per event; events: synth.Event (with theta_inj); priors: the
    per-event prior lists the sampler uses (FIXED entries are not sampled).
    """
    n = len(events)
    cfgs = [gwns.make_config(w, p) for w, p in zip(workloads, priors)]
    sampled = [i for i, p in enumerate(priors[0]) if p.kind != 4]
    t0 = time.perf_counter()
    h = gwns.ns_init(cfgs, events)
    try:
        done = False
        batches = 0
        while not done and batches < max_batches:
            _, prog = gwns.ns_step(h, chunk, n)
            batches += chunk
            done = all(p["done"] for p in prog)
        pct = np.zeros((n, len(sampled)))
        log_z = np.zeros(n)
        log_z_err = np.zeros(n)
        n_like = np.zeros(n, dtype=np.int64)
        for e in range(n):
            th, lw = gwns.ns_posterior(h, e)
            pct[e] = percentiles(th, lw, events[e].theta_inj, sampled)
            log_z[e], log_z_err[e], _, n_like[e] = gwns.ns_evidence(h, e)
        iters = np.array([p["iterations"] for p in prog])
    finally:
        gwns.ns_free(h)
    return {"percentiles": pct, "sampled": sampled, "log_z": log_z, "log_z_err": log_z_err,
            "n_like": n_like, "iterations": iters, "done": done, "wall_s": time.perf_counter() - t0}
