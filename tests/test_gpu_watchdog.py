"""Failure detection on the walk: the watchdog (ns_set_watchdog, ns_set_abort) ends walks on the
device without a fault, the handle reports NS_ETIMEOUT, keeps a consistent state and recovers.

The waits that run out here are the walks' own loops: a time budget far below one round, or an
abort flag set by the host (before a call, or from another thread while the call runs)."""
import threading
import time

import numpy as np
import pytest

from paper_2509_04336_gb300 import gwns, synth

from _util import event, priors
from test_gpu_walk import walk_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2509_04336_gb300 import build
    build.build()


def _walk(h, surv, u0, l0, star, n_steps):
    n = u0.shape[0]
    out = (np.zeros_like(u0), np.zeros(n), np.zeros(n, np.int32), np.zeros(n, np.int32))
    code = None
    try:
        gwns.ns_walk_batch(h, 0, surv, u0, l0, star, n_steps, 1, 0, *out)
    except gwns.GwnsError as e:
        code = e.code
    return code, out


@pytest.mark.parametrize("precision", [synth.PREC_FP64, synth.PREC_MIXED_FF])
def test_walk_budget_runs_out_and_the_handle_recovers(precision):
    w, ev = event("bbh11_3det_4s_taylorf2")
    ll, surv, u0, l0, star = walk_inputs(w, ev, 60, 16, 3)
    cfg = gwns.make_config(w, priors(w, ev), precision=precision, spec_depth=1)
    h = gwns.ns_init([cfg], [ev])
    ref = gwns.ns_init([cfg], [ev])
    try:
        gwns.ns_set_watchdog(h, 1e-6)
        code, (gu, gl, ga, gn) = _walk(h, surv, u0, l0, star, 2000)
        assert code == gwns.NS_ETIMEOUT
        # every walker stopped after its first round (one proposal; the float-float TaylorF2 round
        # is padded to four), at a point above L*
        per_round = 1 if precision == synth.PREC_FP64 else 4
        assert np.all(gl > star) and np.all(gn <= per_round) and np.all((gu >= 0) & (gu <= 1))
        # budget off: the same call runs the whole walk, as on a handle that never timed out
        gwns.ns_set_watchdog(h, 0.0)
        code, got = _walk(h, surv, u0, l0, star, 200)
        _, want = _walk(ref, surv, u0, l0, star, 200)
        assert code in (None, gwns.NS_WMAXMCMC)
        for a, b in zip(got, want):
            assert np.array_equal(a, b)
        assert got[3].sum() > gn.sum()
    finally:
        gwns.ns_free(h)
        gwns.ns_free(ref)


def test_sampler_timeout_and_abort_flag_then_recovery():
    w, ev = event("four_param_2det_taylorf2")
    h = gwns.ns_init([gwns.make_config(w, priors(w, ev), precision=synth.PREC_FP64)], [ev])
    try:
        gwns.ns_step(h, 2)
        _, p0 = gwns.ns_step(h, 0)
        # a budget below one round: the batches complete with truncated walks
        gwns.ns_set_watchdog(h, 1e-6)
        with pytest.raises(gwns.GwnsError) as e:
            gwns.ns_step(h, 2)
        assert e.value.code == gwns.NS_ETIMEOUT
        _, p1 = gwns.ns_step(h, 0)
        calls_timed_out = p1[0]["n_like"] - p0[0]["n_like"]
        assert p1[0]["iterations"] == p0[0]["iterations"] + 2
        assert calls_timed_out <= 2 * w.num_delete * 32     # at most one round (<= 32 proposals) a walker
        gwns.ns_set_watchdog(h, 0.0)
        # the abort flag, set by the host before the call
        gwns.ns_set_abort(h, True)
        with pytest.raises(gwns.GwnsError) as e:
            gwns.ns_step(h, 1)
        assert e.value.code == gwns.NS_ETIMEOUT
        gwns.ns_set_abort(h, False)
        # recovered: the run goes on and ends with a finite evidence
        code, p2 = gwns.ns_step(h, 200)
        assert code in (gwns.NS_OK, gwns.NS_WMAXMCMC) and p2[0]["done"] == 1
        lz, lz_err, info, n_like = gwns.ns_evidence(h, 0)
        assert np.isfinite(lz) and np.isfinite(lz_err) and n_like == p2[0]["n_like"]
    finally:
        gwns.ns_free(h)


def test_abort_from_another_thread_ends_a_running_walk():
    # a long FP64 walk (8 s IMRPhenomD-form event, one proposal per round) is stopped by
    # ns_set_abort called from another thread while ns_step waits for it
    w, ev = event("bbh11_3det_8s_phenomd", n_live=60)
    cfg = gwns.make_config(w, priors(w, ev), precision=synth.PREC_FP64, spec_depth=1, n_steps0=3000)
    full = gwns.ns_init([cfg], [ev])
    try:
        t0 = time.perf_counter()
        gwns.ns_step(full, 1)
        t_full = time.perf_counter() - t0
        _, pf = gwns.ns_step(full, 0)
    finally:
        gwns.ns_free(full)
    h = gwns.ns_init([cfg], [ev])
    try:
        delay = 0.1 * t_full
        th = threading.Timer(delay, lambda: gwns.ns_set_abort(h, True))
        th.start()
        t0 = time.perf_counter()
        with pytest.raises(gwns.GwnsError) as e:
            gwns.ns_step(h, 1)
        t_abort = time.perf_counter() - t0
        th.join()
        assert e.value.code == gwns.NS_ETIMEOUT
        _, pa = gwns.ns_step(h, 0)
        assert pa[0]["n_like"] < pf[0]["n_like"] and t_abort < 0.8 * t_full, (t_abort, t_full)
        gwns.ns_set_abort(h, False)
        code, _ = gwns.ns_step(h, 1)
        assert code in (gwns.NS_OK, gwns.NS_WMAXMCMC)
    finally:
        gwns.ns_free(h)


def test_hrss_budget_runs_out():
    w, ev = event("four_param_2det_taylorf2")
    ll, surv, u0, l0, star = walk_inputs(w, ev, 40, 8, 4)
    h = gwns.ns_init([gwns.make_config(w, priors(w, ev), precision=synth.PREC_FP64)], [ev])
    try:
        gwns.ns_set_watchdog(h, 1e-6)
        with pytest.raises(gwns.GwnsError) as e:
            gwns.ns_hrss_batch(h, 0, surv, u0, l0, star, 50)
        assert e.value.code == gwns.NS_ETIMEOUT
        gwns.ns_set_watchdog(h, 0.0)
        gu, gl, gm, gn = gwns.ns_hrss_batch(h, 0, surv, u0, l0, star, 5)
        assert np.all(gm == 5) and np.all(gl > star)
    finally:
        gwns.ns_free(h)
