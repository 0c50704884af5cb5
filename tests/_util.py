"""Shared helpers of the tests: oracle-made events and configs for the CUDA path."""
import functools

import numpy as np

from oracle import likelihood as L, prior as P
from paper_2509_04336_gb300 import synth


@functools.lru_cache(maxsize=None)
def event(name, f_max=None, n_live=None, precision=None, snr=None):
    w = synth.workload(name)
    if f_max is not None or n_live is not None:
        w = synth.shrink(w, f_max=f_max, n_live=n_live)
    if precision is not None:
        from dataclasses import replace
        w = replace(w, precision=precision)
    ev = synth.make_event(w, lambda e, i, th: L.project(e, i, th, w.waveform), L.inner, snr=snr)
    return w, ev


def priors(w, ev):
    return synth.priors_with_injection(w, ev)


def prior_draws(w, ev, n, seed):
    pri = priors(w, ev)
    u = synth.uniform_unit_cube(n, w.n_dim, seed)
    return u, np.stack([P.transform(x, pri) for x in u])


def oracle_lnl(w, ev, thetas):
    return np.array([L.log_likelihood(ev, th, w.waveform, w.use_ratio) for th in thetas])
