"""ns_walk_batch_noalloc against ns_walk_batch.

The no-allocation walk serves callers that cannot let the library call cudaMalloc after
start-up (a fixed device-memory budget, or a loop that cannot take cudaMalloc's device
synchronisation).  It must give the walk's results for the same arguments, on every call,
although all calls share one static scratch array.  This file is collected last so that a
failure here never hides the rest of the suite; it also passes when run on its own."""
import numpy as np
import pytest

from oracle import likelihood as L, prior as P
from paper_2509_04336_gb300 import gwns, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2509_04336_gb300 import build
    build.build()


def _setup():
    w = synth.shrink(synth.workload("bbh11_3det_4s_taylorf2"), f_max=200.0, n_live=60)
    ev = synth.make_event(w, L.project, L.inner)
    pri = synth.priors_with_injection(w, ev)
    rng = np.random.default_rng(21)
    surv = rng.random((40, w.n_dim))
    lnl_s = np.array([L.log_likelihood(ev, P.transform(x, pri)) for x in surv])
    star = float(np.quantile(lnl_s, 0.4))
    ok = np.where(lnl_s > star)[0]
    idx = ok[rng.integers(0, ok.shape[0], 12)]
    return w, ev, pri, surv, lnl_s[idx], surv[idx], star


def test_noalloc_walk_matches_walk_on_consecutive_calls():
    import torch
    w, ev, pri, surv, l0, u0, star = _setup()
    h = gwns.ns_init([gwns.make_config(w, pri, precision=synth.PREC_MIXED_FF)], [ev])
    try:
        T = lambda a, dt=torch.float64: torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=dt)
        for call, (it, off, steps) in enumerate([(3, 0, 15), (4, 12, 9)]):
            outs = []
            for fn in (gwns.ns_walk_batch, gwns.ns_walk_batch_noalloc):
                gu, gl = T(np.zeros_like(u0)), T(np.zeros(12))
                ga, gn = T(np.zeros(12), torch.int32), T(np.zeros(12), torch.int32)
                fn(h, 0, T(surv), T(u0), T(l0), star, steps, it, off, gu, gl, ga, gn)
                torch.cuda.synchronize()
                outs.append((gu.cpu().numpy(), gl.cpu().numpy(), ga.cpu().numpy(), gn.cpu().numpy()))
            (ru, rl, ra, rn), (nu, nl, na, nn) = outs
            assert np.array_equal(ra, na) and np.array_equal(rn, nn), f"call {call}"
            assert np.allclose(nu, ru, rtol=0, atol=1e-12), f"call {call}"
            assert np.all(np.abs(nl - rl) <= 1e-6 * np.abs(rl)), f"call {call}"
            assert ra.sum() > 0
    finally:
        gwns.ns_free(h)


def test_noalloc_rejects_too_many_walkers():
    import torch
    w, ev, pri, surv, l0, u0, star = _setup()
    h = gwns.ns_init([gwns.make_config(w, pri, precision=synth.PREC_MIXED)], [ev])
    try:
        n = 8193
        z = lambda *s, dt=torch.float64: torch.zeros(*s, device="cuda", dtype=dt)
        with pytest.raises(gwns.GwnsError) as e:
            gwns.ns_walk_batch_noalloc(h, 0, torch.tensor(surv, device="cuda"), z(n, w.n_dim), z(n), star, 3, 0, 0,
                                       z(n, w.n_dim), z(n), z(n, dt=torch.int32), z(n, dt=torch.int32))
        assert e.value.code == gwns.NS_EINVAL and "8192" in str(e.value)
    finally:
        gwns.ns_free(h)
