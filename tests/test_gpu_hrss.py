"""CUDA hit-and-run slice sampling (ns_hrss_batch, FP64) vs the oracle (oracle/hrss.py) on the
same Philox streams: move and likelihood-call counts bit-exact, positions to rounding."""
import numpy as np
import pytest

from oracle import hrss, prior as P
from paper_2509_04336_gb300 import gwns, synth

from _util import event, priors
from test_gpu_walk import walk_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2509_04336_gb300 import build
    build.build()


@pytest.mark.parametrize("name", ["four_param_2det_taylorf2", "bbh11_3det_4s_taylorf2"])
def test_hrss_chain_matches_oracle(name):
    w, ev = event(name)
    ll, surv, u0, l0, lnl_star = walk_inputs(w, ev, 60, 16, 5)
    n_steps, it, off = 4, 2, 9
    periodic = P.periodic_mask(priors(w, ev))
    ou, ol, om, on = hrss.hrss_walk(ll, u0, l0, lnl_star, surv, n_steps, periodic, (w.seed, 0), it,
                                    walker_ids=np.arange(16) + off)
    h = gwns.ns_init([gwns.make_config(w, priors(w, ev), precision=synth.PREC_FP64)], [ev])
    try:
        gu, gl, gm, gn = gwns.ns_hrss_batch(h, 0, surv, u0, l0, lnl_star, n_steps, it, off)
    finally:
        gwns.ns_free(h)
    assert np.array_equal(gm, om) and np.array_equal(gn, on)
    assert np.allclose(gu, ou, rtol=0, atol=1e-12)
    assert np.all(np.abs(gl - ol) <= 1e-11 * np.maximum(np.abs(ol), 1.0))
    assert np.all(gl > lnl_star) and np.all((gu >= 0) & (gu <= 1))
    assert np.all(gm == n_steps)


def test_hrss_errors():
    w, ev = event("four_param_2det_taylorf2")
    ll, surv, u0, l0, lnl_star = walk_inputs(w, ev, 20, 2, 6)
    h = gwns.ns_init([gwns.make_config(w, priors(w, ev), precision=synth.PREC_MIXED_FF)], [ev])
    try:
        with pytest.raises(gwns.GwnsError) as e:
            gwns.ns_hrss_batch(h, 0, surv, u0, l0, lnl_star, 1)
        assert e.value.code == gwns.NS_EINVAL
    finally:
        gwns.ns_free(h)
    h = gwns.ns_init([gwns.make_config(w, priors(w, ev), precision=synth.PREC_FP64)], [ev])
    try:
        # two survivors span one direction: the covariance is singular
        with pytest.raises(gwns.GwnsError) as e:
            gwns.ns_hrss_batch(h, 0, surv[:2], u0, l0, lnl_star, 1)
        assert e.value.code == gwns.NS_EINVAL
        gu, gl, gm, gn = gwns.ns_hrss_batch(h, 0, surv, u0, l0, lnl_star, 0)
        assert np.array_equal(gu, u0) and np.array_equal(gl, l0) and np.all(gm == 0) and np.all(gn == 0)
    finally:
        gwns.ns_free(h)
