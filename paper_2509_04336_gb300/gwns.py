"""Python binding of libgwns (include/gwns.h): argument marshalling only.

Every function has the name and argument order of its C counterpart.  Arrays may be
torch tensors (CUDA tensors are passed as device pointers on the current torch stream --
torch's default stream as cudaStreamLegacy, so the library's work is ordered with torch's --
CPU tensors as host pointers) or numpy arrays (host pointers).  Loading fails loudly when
the shared library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import synth

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgwns.so")

N_PARAMS = 11
MAX_DET = 4

NS_OK, NS_EINVAL, NS_ECUDA, NS_ENOMEM, NS_ENONFINITE, NS_ETIMEOUT, NS_ESTATE, NS_EIO = 0, -1, -2, -3, -4, -5, -6, -7
NS_WMAXMCMC = 1
NS_PTR_HOST, NS_PTR_DEVICE = 0, 1
NS_PREC_FP64, NS_PREC_MIXED, NS_PREC_MIXED_FF = 0, 1, 2
NS_PROPOSAL_DE, NS_PROPOSAL_DE_FLOW, NS_PROPOSAL_HRSS = 0, 1, 2
STATUS_NAMES = {0: "NS_OK", -1: "NS_EINVAL", -2: "NS_ECUDA", -3: "NS_ENOMEM", -4: "NS_ENONFINITE",
                -5: "NS_ETIMEOUT", -6: "NS_ESTATE", -7: "NS_EIO", 1: "NS_WMAXMCMC"}


class ns_prior(C.Structure):
    _fields_ = [("kind", C.c_int32), ("periodic", C.c_int32), ("lo", C.c_double), ("hi", C.c_double),
                ("alpha", C.c_double), ("value", C.c_double)]


class ns_config(C.Structure):
    _fields_ = [("prior", ns_prior * N_PARAMS), ("n_live", C.c_int32), ("num_delete", C.c_int32),
                ("naccept", C.c_int32), ("maxmcmc", C.c_int32), ("delay", C.c_double),
                ("use_ratio", C.c_int32), ("term_kind", C.c_int32), ("term_value", C.c_double),
                ("precision", C.c_int32), ("waveform", C.c_int32), ("max_iter", C.c_int32),
                ("n_steps0", C.c_int32), ("seed", C.c_uint64), ("spec_depth", C.c_int32), ("proposal", C.c_int32),
                ("p_flow", C.c_double), ("flow_layers", C.c_int32), ("flow_every", C.c_int32),
                ("flow_epochs", C.c_int32), ("hrss_moves", C.c_int32), ("flow_lr", C.c_double),
                ("flow_accept_weight", C.c_double)]


class ns_detector(C.Structure):
    _fields_ = [("vertex", C.c_double * 3), ("x_arm", C.c_double * 3), ("y_arm", C.c_double * 3),
                ("d_re", C.POINTER(C.c_double)), ("d_im", C.POINTER(C.c_double)), ("psd", C.POINTER(C.c_double))]


class ns_event(C.Structure):
    _fields_ = [("n_det", C.c_int32), ("n_bins", C.c_int32), ("f_min", C.c_double), ("df", C.c_double),
                ("gmst", C.c_double), ("det", ns_detector * MAX_DET)]


class ns_progress(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("n_like", C.c_int64), ("log_z", C.c_double), ("dlogz", C.c_double),
                ("log_x", C.c_double), ("lnl_star", C.c_double), ("mean_accept", C.c_double),
                ("n_steps", C.c_int32), ("done", C.c_int32), ("n_bins", C.c_int64), ("walk_ms", C.c_double),
                ("kernel_launches", C.c_int64), ("n_spec", C.c_int64), ("spec_depth", C.c_int32),
                ("spec_cap", C.c_int32), ("mean_accept_flow", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ("ns_init", "ns_waveform", "ns_likelihood_batch", "ns_walk_batch", "ns_step", "ns_evidence",
           "ns_posterior", "ns_state_save", "ns_state_load", "ns_walk_batch_noalloc", "ns_flow_num_params",
           "ns_flow_set", "ns_flow_get", "ns_flow_logq", "ns_flow_sample", "ns_flow_grad", "ns_flow_train",
           "ns_relbin_set", "ns_relbin_edges", "ns_hrss_batch", "ns_set_watchdog", "ns_set_abort",
           "ns_batch_begin", "ns_batch_walk", "ns_batch_walk_io", "ns_batch_end", "ns_free", "ns_last_error")

_lib = None


def load(path: str = LIB_PATH):
    """Load libgwns.so (once).  Raises if it is missing: build it with paper_2509_04336_gb300.build."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libgwns.so not found at {path}; run paper_2509_04336_gb300.build.build()")
    lib = C.CDLL(path)
    P, I, D, V = C.c_void_p, C.c_int, C.c_double, C.c_void_p
    lib.ns_init.argtypes = [C.POINTER(ns_config), C.POINTER(ns_event), I, I, C.POINTER(C.c_void_p)]
    lib.ns_waveform.argtypes = [P, I, P, I, P, P, I, V]
    lib.ns_likelihood_batch.argtypes = [P, I, P, I, P, I, V]
    lib.ns_walk_batch.argtypes = [P, I, P, I, P, P, D, I, I, C.c_int64, C.c_int64, P, P, P, P, I, V]
    lib.ns_step.argtypes = [P, I, C.POINTER(ns_progress)]
    lib.ns_evidence.argtypes = [P, I, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                C.POINTER(C.c_int64)]
    lib.ns_posterior.argtypes = [P, I, P, P, C.c_int64, C.POINTER(C.c_int64)]
    lib.ns_state_save.argtypes = [P, C.c_char_p]
    lib.ns_state_load.argtypes = [P, C.c_char_p]
    lib.ns_walk_batch_noalloc.argtypes = [P, I, P, I, P, P, D, I, I, C.c_int64, C.c_int64, P, P, P, P, V]
    lib.ns_flow_num_params.argtypes = [P, I, C.POINTER(C.c_int32)]
    lib.ns_flow_set.argtypes = [P, I, P, P, P]
    lib.ns_flow_get.argtypes = [P, I, P, P, P]
    lib.ns_flow_logq.argtypes = [P, I, P, I, P, I, V]
    lib.ns_flow_sample.argtypes = [P, I, C.c_int64, C.c_int64, I, I, P, P, I, V]
    lib.ns_flow_grad.argtypes = [P, I, P, I, P, C.POINTER(C.c_double)]
    lib.ns_flow_train.argtypes = [P, I, P, I, I, P]
    lib.ns_relbin_set.argtypes = [P, I, P, I, P]
    lib.ns_relbin_edges.argtypes = [D, D, I, D, P, I, C.POINTER(C.c_int32)]
    lib.ns_hrss_batch.argtypes = [P, I, P, I, P, P, D, I, I, C.c_int64, C.c_int64, P, P, P, P]
    lib.ns_set_watchdog.argtypes = [P, D]
    lib.ns_set_abort.argtypes = [P, I]
    lib.ns_batch_begin.argtypes = [P]
    lib.ns_batch_walk.argtypes = [P, C.c_int64, C.c_int64]
    lib.ns_batch_walk_io.argtypes = [P, I, C.c_int64, C.c_int64, P, P, P, P, P, P, I, I]
    lib.ns_batch_end.argtypes = [P, C.POINTER(ns_progress)]
    lib.ns_free.argtypes = [P]
    lib.ns_free.restype = None
    lib.ns_last_error.argtypes = [P]
    lib.ns_last_error.restype = C.c_char_p
    for name in EXPORTS[:-2]:
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


class GwnsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _check(code, handle, allow_warning=False):
    if code == NS_OK or (allow_warning and code == NS_WMAXMCMC):
        return code
    msg = _lib.ns_last_error(handle)
    raise GwnsError(code, msg.decode() if msg else "")


def _ptr(a):
    """(address, ptr_kind, stream) of a torch tensor or numpy array."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data, NS_PTR_HOST, None
    import torch
    if not a.is_contiguous():
        raise ValueError("tensors must be contiguous")
    if a.is_cuda:
        return a.data_ptr(), NS_PTR_DEVICE, _torch_stream(a.device)
    return a.data_ptr(), NS_PTR_HOST, None


# cudaStreamLegacy: the handle value that names the legacy default stream explicitly.
CUDA_STREAM_LEGACY = 0x1


def _torch_stream(device):
    """Stream handle of torch's current stream on `device`, never NULL: torch's default stream
    is the legacy default stream (handle 0), and a NULL stream means the handle's own stream to
    the library, which is not ordered with torch's work; it is passed as cudaStreamLegacy."""
    import torch
    st = torch.cuda.current_stream(device).cuda_stream
    return st if st != 0 else CUDA_STREAM_LEGACY


def _same_kind(*arrays):
    ptrs = [_ptr(a) for a in arrays]
    kinds = {p[1] for p in ptrs}
    if len(kinds) != 1:
        raise ValueError("all arrays of a call must be host or all device")
    return ptrs


# ---------------------------------------------------------------- marshalling helpers
def make_config(w: synth.Workload, priors=None, *, precision=None, max_iter=0, n_steps0=0, delay=-1.0,
                seed=None, spec_depth=0, p_flow=None, flow_layers=0, flow_every=0, flow_epochs=0,
                flow_lr=0.0, hrss_moves=None, flow_accept_weight=0.0) -> ns_config:
    """ns_config of a workload; p_flow (not None) selects NS_PROPOSAL_DE_FLOW, hrss_moves (not
    None; 0 means 2 D) NS_PROPOSAL_HRSS."""
    c = ns_config()
    pri = w.priors if priors is None else priors
    for i, p in enumerate(pri):
        c.prior[i] = ns_prior(p.kind, 1 if p.periodic else 0, p.lo, p.hi, p.alpha, p.value)
    c.n_live, c.num_delete, c.naccept, c.maxmcmc = w.n_live, w.num_delete, w.naccept, w.maxmcmc
    c.delay = delay
    c.use_ratio = 1 if w.use_ratio else 0
    c.term_kind, c.term_value = w.term_kind, w.term_value
    c.precision = w.precision if precision is None else precision
    c.waveform = w.waveform
    c.max_iter, c.n_steps0 = max_iter, n_steps0
    c.seed = w.seed if seed is None else seed
    c.spec_depth = spec_depth
    if p_flow is not None:
        c.proposal = NS_PROPOSAL_DE_FLOW
        c.p_flow = p_flow
        c.flow_layers, c.flow_every, c.flow_epochs, c.flow_lr = flow_layers, flow_every, flow_epochs, flow_lr
        c.flow_accept_weight = flow_accept_weight
    if hrss_moves is not None:
        c.proposal = NS_PROPOSAL_HRSS
        c.hrss_moves = hrss_moves
    return c


def make_event(ev: synth.Event):
    """ns_event for a synth.Event; returns (struct, keepalive) -- keep both alive until ns_init returns."""
    e = ns_event()
    e.n_det, e.n_bins, e.f_min, e.df, e.gmst = len(ev.detectors), ev.n_bins, ev.f_min, ev.df, ev.gmst
    keep = []
    for i, d in enumerate(ev.detectors):
        re = np.ascontiguousarray(d.data.real, dtype=np.float64)
        im = np.ascontiguousarray(d.data.imag, dtype=np.float64)
        ps = np.ascontiguousarray(d.psd, dtype=np.float64)
        keep += [re, im, ps]
        det = e.det[i]
        for j in range(3):
            det.vertex[j], det.x_arm[j], det.y_arm[j] = d.vertex[j], d.x_arm[j], d.y_arm[j]
        det.d_re = re.ctypes.data_as(C.POINTER(C.c_double))
        det.d_im = im.ctypes.data_as(C.POINTER(C.c_double))
        det.psd = ps.ctypes.data_as(C.POINTER(C.c_double))
    return e, keep


# ---------------------------------------------------------------- entry points
def ns_init(configs, events, device: int = 0):
    """configs: list of ns_config; events: list of synth.Event or ns_event.  Returns the handle."""
    lib = load()
    n = len(configs)
    cfg_arr = (ns_config * n)(*configs)
    ev_arr = (ns_event * n)()
    keep = []
    for i, ev in enumerate(events):
        if isinstance(ev, ns_event):
            ev_arr[i] = ev
        else:
            s, k = make_event(ev)
            ev_arr[i] = s
            keep.append(k)
    h = C.c_void_p()
    code = lib.ns_init(cfg_arr, ev_arr, n, device, C.byref(h))
    if code != NS_OK:
        raise GwnsError(code, lib.ns_last_error(None).decode())
    return h


def ns_waveform(h, event: int, theta, h_re, h_im):
    (pt, kind, st), (pr, _, _), (pi, _, _) = _same_kind(theta, h_re, h_im)
    return _check(_lib.ns_waveform(h, event, pt, theta.shape[0], pr, pi, kind, st), h)


def ns_likelihood_batch(h, event: int, theta, lnl):
    (pt, kind, st), (pl, _, _) = _same_kind(theta, lnl)
    return _check(_lib.ns_likelihood_batch(h, event, pt, theta.shape[0], pl, kind, st), h)


def ns_walk_batch(h, event: int, live_u, u0, lnl0, lnl_star: float, n_steps: int, iteration: int,
                  walker_offset: int, u_out, lnl_out, n_accept, n_like):
    ps = _same_kind(live_u, u0, lnl0, u_out, lnl_out, n_accept, n_like)
    kind, st = ps[0][1], ps[0][2]
    code = _lib.ns_walk_batch(h, event, ps[0][0], live_u.shape[0], ps[1][0], ps[2][0], float(lnl_star),
                              u0.shape[0], n_steps, iteration, walker_offset, ps[3][0], ps[4][0], ps[5][0],
                              ps[6][0], kind, st)
    return _check(code, h, allow_warning=True)


def ns_walk_batch_noalloc(h, event: int, live_u, u0, lnl0, lnl_star: float, n_steps: int, iteration: int,
                          walker_offset: int, u_out, lnl_out, n_accept, n_like):
    """The walk of ns_walk_batch without any device allocation; CUDA tensors only, enqueued
    on the current torch stream."""
    ps = _same_kind(live_u, u0, lnl0, u_out, lnl_out, n_accept, n_like)
    if ps[0][1] != NS_PTR_DEVICE:
        raise ValueError("ns_walk_batch_noalloc takes device (CUDA) tensors only")
    code = _lib.ns_walk_batch_noalloc(h, event, ps[0][0], live_u.shape[0], ps[1][0], ps[2][0], float(lnl_star),
                                      u0.shape[0], n_steps, iteration, walker_offset, ps[3][0], ps[4][0],
                                      ps[5][0], ps[6][0], ps[0][2])
    return _check(code, h)


def ns_step(h, max_batches: int, n_events: int = 1):
    prog = (ns_progress * n_events)()
    code = _check(_lib.ns_step(h, max_batches, prog), h, allow_warning=True)
    return code, [p.as_dict() for p in prog]


def ns_evidence(h, event: int = 0):
    lz, err, info = C.c_double(), C.c_double(), C.c_double()
    nl = C.c_int64()
    _check(_lib.ns_evidence(h, event, C.byref(lz), C.byref(err), C.byref(info), C.byref(nl)), h)
    return lz.value, err.value, info.value, nl.value


def ns_posterior(h, event: int = 0, cap: int | None = None):
    n = C.c_int64()
    _check(_lib.ns_posterior(h, event, None, None, 0, C.byref(n)), h)
    m = n.value if cap is None else min(cap, n.value)
    th = np.zeros((m, N_PARAMS))
    lw = np.zeros(m)
    _check(_lib.ns_posterior(h, event, th.ctypes.data, lw.ctypes.data, m, C.byref(n)), h)
    return th, lw


def ns_state_save(h, path: str):
    return _check(_lib.ns_state_save(h, path.encode()), h)


def ns_state_load(h, path: str):
    return _check(_lib.ns_state_load(h, path.encode()), h)


def ns_flow_num_params(h, event: int = 0) -> int:
    n = C.c_int32()
    _check(_lib.ns_flow_num_params(h, event, C.byref(n)), h)
    return n.value


def ns_flow_set(h, event: int, params, mu, sigma):
    p = np.ascontiguousarray(params, dtype=np.float32)
    m = np.ascontiguousarray(mu, dtype=np.float64)
    s = np.ascontiguousarray(sigma, dtype=np.float64)
    return _check(_lib.ns_flow_set(h, event, p.ctypes.data, m.ctypes.data, s.ctypes.data), h)


def ns_flow_get(h, event: int, n_dim: int):
    """(params float32 [n_params], mu [D], sigma [D])."""
    p = np.zeros(ns_flow_num_params(h, event), dtype=np.float32)
    m = np.zeros(n_dim)
    s = np.zeros(n_dim)
    _check(_lib.ns_flow_get(h, event, p.ctypes.data, m.ctypes.data, s.ctypes.data), h)
    return p, m, s


def ns_flow_logq(h, event: int, u, logq):
    (pu, kind, st), (pl, _, _) = _same_kind(u, logq)
    return _check(_lib.ns_flow_logq(h, event, pu, u.shape[0], pl, kind, st), h)


def ns_flow_sample(h, event: int, iteration: int, walker_offset: int, u_out, logq_out):
    """u_out [n][n_steps][D], logq_out [n][n_steps]."""
    (pu, kind, st), (pl, _, _) = _same_kind(u_out, logq_out)
    return _check(_lib.ns_flow_sample(h, event, iteration, walker_offset, u_out.shape[0], u_out.shape[1], pu, pl,
                                      kind, st), h)


def ns_flow_grad(h, event: int, u):
    """(mean -ln q, gradient float32 [n_params]) of host points u [n][D]."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    g = np.zeros(ns_flow_num_params(h, event), dtype=np.float32)
    loss = C.c_double()
    _check(_lib.ns_flow_grad(h, event, u.ctypes.data, u.shape[0], g.ctypes.data, C.byref(loss)), h)
    return loss.value, g


def ns_flow_train(h, event: int, u, epochs: int):
    """Losses before each of the epochs Adam steps on host points u [n][D]."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    losses = np.zeros(max(epochs, 1))
    _check(_lib.ns_flow_train(h, event, u.ctypes.data, u.shape[0], epochs, losses.ctypes.data), h)
    return losses[:epochs]


def ns_relbin_set(h, event: int, edges, theta0=None):
    """Relative-binning likelihood for the event around the fiducial theta0 [11], coarse-bin
    edges [n] (grid-bin indices, 0 .. n_bins); edges None restores the full likelihood."""
    if edges is None:
        return _check(_lib.ns_relbin_set(h, event, None, 0, None), h)
    e = np.ascontiguousarray(edges, dtype=np.int32)
    t = np.ascontiguousarray(theta0, dtype=np.float64)
    assert t.shape == (11,)
    return _check(_lib.ns_relbin_set(h, event, e.ctypes.data, e.shape[0], t.ctypes.data), h)


def ns_relbin_edges(f_min: float, df: float, n_bins: int, eps: float = 0.25) -> np.ndarray:
    """int32 coarse-bin edges [n_coarse + 1] (0, ..., n_bins) of the library's edge rule."""
    n = C.c_int32()
    code = _lib.ns_relbin_edges(float(f_min), float(df), int(n_bins), float(eps), None, 0, C.byref(n))
    if n.value <= 0:
        raise GwnsError(code, "ns_relbin_edges: bad grid or eps")
    out = np.zeros(n.value, dtype=np.int32)
    _check(_lib.ns_relbin_edges(float(f_min), float(df), int(n_bins), float(eps), out.ctypes.data, out.shape[0],
                                C.byref(n)), None)
    return out


def ns_hrss_batch(h, event: int, live_u, u0, lnl0, lnl_star: float, n_steps: int, iteration: int = 0,
                  walker_offset: int = 0):
    """Hit-and-run slice-sampling moves of host walkers u0 [n][D] against the survivors
    live_u [m][D]: (u_out, lnl_out, n_move, n_like)."""
    live_u = np.ascontiguousarray(live_u, dtype=np.float64)
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    lnl0 = np.ascontiguousarray(lnl0, dtype=np.float64)
    n = u0.shape[0]
    uo = np.zeros_like(u0)
    lo = np.zeros(n)
    nm = np.zeros(n, dtype=np.int32)
    nl = np.zeros(n, dtype=np.int32)
    _check(_lib.ns_hrss_batch(h, event, live_u.ctypes.data, live_u.shape[0], u0.ctypes.data, lnl0.ctypes.data,
                              float(lnl_star), n, n_steps, iteration, walker_offset, uo.ctypes.data,
                              lo.ctypes.data, nm.ctypes.data, nl.ctypes.data), h)
    return uo, lo, nm, nl


def ns_set_watchdog(h, budget_seconds: float):
    return _check(_lib.ns_set_watchdog(h, float(budget_seconds)), h)


def ns_set_abort(h, flag: bool):
    return _check(_lib.ns_set_abort(h, 1 if flag else 0), h)


def ns_batch_begin(h):
    return _check(_lib.ns_batch_begin(h), h)


def ns_batch_walk(h, walker_begin: int, walker_end: int):
    return _check(_lib.ns_batch_walk(h, int(walker_begin), int(walker_end)), h)


def ns_batch_walk_io(h, event: int, walker_begin: int, u, lnl, n_accept, n_like, n_bins, n_spec, write: bool):
    """Copy the walk outputs of walkers [walker_begin, walker_begin + len(lnl)) of one event out of
    the handle (write False) or into it (write True); arrays host (numpy) or CUDA tensors."""
    ps = _same_kind(u, lnl, n_accept, n_like, n_bins, n_spec)
    n = lnl.shape[0]
    return _check(_lib.ns_batch_walk_io(h, event, int(walker_begin), int(walker_begin) + n, ps[0][0], ps[1][0],
                                        ps[2][0], ps[3][0], ps[4][0], ps[5][0], ps[0][1], 1 if write else 0), h)


def ns_batch_end(h, n_events: int = 1):
    prog = (ns_progress * n_events)()
    code = _check(_lib.ns_batch_end(h, prog), h, allow_warning=True)
    return code, [p.as_dict() for p in prog]


def ns_free(h):
    if h is not None and _lib is not None:
        _lib.ns_free(h)


def ns_last_error(h=None) -> str:
    msg = load().ns_last_error(h)
    return msg.decode() if msg else ""
