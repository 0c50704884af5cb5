"""ns_walk_batch_noalloc against ns_walk_batch.

The no-allocation walk serves callers that cannot let the library call cudaMalloc after
start-up (a fixed device-memory budget, or a loop that cannot take cudaMalloc's device
synchronisation).  Both calls launch the same walk kernel on the same task, so the results
must be identical, bit for bit, on every call, although all no-allocation calls share one
static scratch array.  This file is collected last so that a failure here never hides the
rest of the suite; it also passes when run on its own."""
import numpy as np
import pytest

from oracle import likelihood as L, prior as P
from paper_2509_04336_gb300 import gwns, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2509_04336_gb300 import build
    build.build()


def _setup(n_walk=12, seed=21):
    w = synth.shrink(synth.workload("bbh11_3det_4s_taylorf2"), f_max=200.0, n_live=60)
    ev = synth.make_event(w, L.project, L.inner)
    pri = synth.priors_with_injection(w, ev)
    rng = np.random.default_rng(seed)
    surv = rng.random((40, w.n_dim))
    lnl_s = np.array([L.log_likelihood(ev, P.transform(x, pri)) for x in surv])
    star = float(np.quantile(lnl_s, 0.4))
    ok = np.where(lnl_s > star)[0]
    idx = ok[rng.integers(0, ok.shape[0], n_walk)]
    return w, ev, pri, surv, lnl_s[idx], surv[idx], star


def _run(fn, h, surv, u0, l0, star, steps, it, off):
    import torch
    T = lambda a, dt=torch.float64: torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=dt)
    n = u0.shape[0]
    gu, gl = T(np.zeros_like(u0)), T(np.zeros(n))
    ga, gn = T(np.zeros(n), torch.int32), T(np.zeros(n), torch.int32)
    torch.cuda.synchronize()
    fn(h, 0, T(surv), T(u0), T(l0), star, steps, it, off, gu, gl, ga, gn)
    torch.cuda.synchronize()
    return gu.cpu().numpy(), gl.cpu().numpy(), ga.cpu().numpy(), gn.cpu().numpy()


def _same(a, b, what):
    for x, y, name in zip(a, b, ("u_out", "lnl_out", "n_accept", "n_like")):
        assert np.array_equal(x, y), f"{what}: {name} differs"


def test_noalloc_walk_matches_walk_on_consecutive_calls():
    import torch
    w, ev, pri, surv, l0, u0, star = _setup()
    # a throw-away handle runs the kernels once, so that loading their code is not counted below
    h0 = gwns.ns_init([gwns.make_config(w, pri, precision=synth.PREC_MIXED_FF)], [ev])
    try:
        _run(gwns.ns_walk_batch_noalloc, h0, surv, u0, l0, star, 2, 0, 0)
    finally:
        gwns.ns_free(h0)
    h = gwns.ns_init([gwns.make_config(w, pri, precision=synth.PREC_MIXED_FF)], [ev])
    try:
        # first call of the handle: the no-allocation walk, with device memory unchanged by it
        T = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
        args = [T(surv), T(u0), T(l0)]
        outs = [torch.zeros(12, w.n_dim, dtype=torch.float64, device="cuda"),
                torch.zeros(12, dtype=torch.float64, device="cuda"),
                torch.zeros(12, dtype=torch.int32, device="cuda"), torch.zeros(12, dtype=torch.int32, device="cuda")]
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        gwns.ns_walk_batch_noalloc(h, 0, *args, star, 15, 3, 0, *outs)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "the no-allocation walk changed free device memory"
        first = tuple(o.cpu().numpy() for o in outs)
        for call, (it, off, steps) in enumerate([(3, 0, 15), (4, 12, 9), (3, 0, 15)]):
            ref = _run(gwns.ns_walk_batch, h, surv, u0, l0, star, steps, it, off)
            got = _run(gwns.ns_walk_batch_noalloc, h, surv, u0, l0, star, steps, it, off)
            _same(ref, got, f"call {call}")
            assert ref[2].sum() > 0
            if call in (0, 2):
                _same(ref, first, "first call on a fresh handle")
    finally:
        gwns.ns_free(h)


def test_noalloc_walk_at_its_walker_limit():
    # 8192 walkers, the array's capacity: the block map's last entries are used.
    w, ev, pri, surv, l0, u0, star = _setup(n_walk=8192, seed=5)
    h = gwns.ns_init([gwns.make_config(w, pri, precision=synth.PREC_MIXED_FF)], [ev])
    try:
        ref = _run(gwns.ns_walk_batch, h, surv, u0, l0, star, 3, 7, 100)
        got = _run(gwns.ns_walk_batch_noalloc, h, surv, u0, l0, star, 3, 7, 100)
        _same(ref, got, "8192 walkers")
        assert ref[3][-64:].sum() > 0
    finally:
        gwns.ns_free(h)


def test_noalloc_walk_with_flow_proposals():
    # An event with flow steps: the call fills the handle's batch proposal table.
    w, ev, pri, surv, l0, u0, star = _setup(seed=9)
    h = gwns.ns_init([gwns.make_config(w, pri, precision=synth.PREC_MIXED_FF, p_flow=0.5)], [ev])
    try:
        for it, off, steps in [(2, 0, 12), (5, 30, 20)]:
            ref = _run(gwns.ns_walk_batch, h, surv, u0, l0, star, steps, it, off)
            got = _run(gwns.ns_walk_batch_noalloc, h, surv, u0, l0, star, steps, it, off)
            _same(ref, got, f"flow walk, iteration {it}")
    finally:
        gwns.ns_free(h)


def test_noalloc_walk_is_ordered_with_torch_default_stream():
    # Inputs made and outputs read by torch kernels on torch's default stream, with no
    # device-wide synchronisation around the call: the binding passes that stream, so the
    # walk runs after the fills and before the reads.
    import torch
    w, ev, pri, surv, l0, u0, star = _setup(seed=13)
    h = gwns.ns_init([gwns.make_config(w, pri, precision=synth.PREC_MIXED_FF)], [ev])
    try:
        ref = _run(gwns.ns_walk_batch, h, surv, u0, l0, star, 25, 1, 0)
        assert torch.cuda.current_stream().cuda_stream == 0
        big = torch.ones(1 << 24, dtype=torch.float64, device="cuda")
        dsurv = torch.tensor(surv, device="cuda") + big[:1] * 0.0   # made by a torch kernel
        du0 = torch.tensor(u0, device="cuda") + big[:1] * 0.0
        dl0 = torch.tensor(l0, device="cuda") + big[:1] * 0.0
        gu = torch.full((12, w.n_dim), float("nan"), dtype=torch.float64, device="cuda")
        gl = torch.full((12,), float("nan"), dtype=torch.float64, device="cuda")
        ga = torch.full((12,), -1, dtype=torch.int32, device="cuda")
        gn = torch.full((12,), -1, dtype=torch.int32, device="cuda")
        big.mul_(2.0)   # keep the default stream busy when the call is enqueued
        gwns.ns_walk_batch_noalloc(h, 0, dsurv, du0, dl0, star, 25, 1, 0, gu, gl, ga, gn)
        got = (gu.cpu().numpy(), gl.cpu().numpy(), ga.cpu().numpy(), gn.cpu().numpy())
        _same(ref, got, "default-stream ordering")
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
