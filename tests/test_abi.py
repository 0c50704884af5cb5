"""The C-ABI library loads, exports every symbol include/gwns.h declares, its struct
layouts match the binding, and bad arguments are rejected before any device work.
No compute call is made (these run without a GPU)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2509_04336_gb300 import build, gwns, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gwns.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return gwns.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ns_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert set(names) == set(gwns.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", gwns.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ns_[a-z_]+)\b", out))
    assert set(names) <= exported


def test_struct_layouts_match_header(tmp_path):
    probe = tmp_path / "probe.c"
    fields = {
        "ns_prior": ["kind", "periodic", "lo", "hi", "alpha", "value"],
        "ns_config": [f for f, _ in gwns.ns_config._fields_],
        "ns_detector": [f for f, _ in gwns.ns_detector._fields_],
        "ns_event": [f for f, _ in gwns.ns_event._fields_],
        "ns_progress": [f for f, _ in gwns.ns_progress._fields_],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for s, fs in fields.items():
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f in fs:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    probe.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c99", "-o", str(exe), str(probe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for s, fs in fields.items():
        cls = getattr(gwns, s)
        assert int(got[s]) == C.sizeof(cls), s
        for f in fs:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, f"{s}.{f}"


def _event_and_config():
    w = synth.workload("four_param_2det_taylorf2")
    w = synth.shrink(w, f_max=40.0)
    zero = lambda ev, i, th: 0.0 * synth.frequencies(ev.f_min, ev.df, ev.n_bins)
    ev = synth.make_event(w, lambda e, i, th: zero(e, i, th) + 1e-23, lambda a, b, p, df: 1.0)
    return w, ev


@pytest.mark.parametrize("mutate,code", [
    (lambda c, e: setattr(c, "n_live", 2), gwns.NS_EINVAL),
    (lambda c, e: setattr(c, "num_delete", 0), gwns.NS_EINVAL),
    (lambda c, e: setattr(c, "num_delete", c.n_live - 1), gwns.NS_EINVAL),
    (lambda c, e: setattr(c, "n_live", 5000), gwns.NS_EINVAL),
    (lambda c, e: setattr(c, "precision", 7), gwns.NS_EINVAL),
    (lambda c, e: setattr(c, "term_value", 0.0), gwns.NS_EINVAL),
    (lambda c, e: setattr(c.prior[0], "hi", c.prior[0].lo), gwns.NS_EINVAL),
    (lambda c, e: setattr(c.prior[0], "kind", 9), gwns.NS_EINVAL),
    (lambda c, e: setattr(e, "n_det", 0), gwns.NS_EINVAL),
    (lambda c, e: setattr(e, "df", -1.0), gwns.NS_EINVAL),
    (lambda c, e: e.det[0].psd.__setitem__(3, -1.0), gwns.NS_ENONFINITE),
    (lambda c, e: e.det[1].d_re.__setitem__(0, float("nan")), gwns.NS_ENONFINITE),
    (lambda c, e: setattr(c, "proposal", 5), gwns.NS_EINVAL),
    (lambda c, e: (setattr(c, "proposal", gwns.NS_PROPOSAL_DE_FLOW), setattr(c, "p_flow", 1.5)), gwns.NS_EINVAL),
    (lambda c, e: (setattr(c, "proposal", gwns.NS_PROPOSAL_DE_FLOW), setattr(c, "flow_layers", 17)), gwns.NS_EINVAL),
    (lambda c, e: (setattr(c, "proposal", gwns.NS_PROPOSAL_DE_FLOW), setattr(c, "flow_lr", -1.0)), gwns.NS_EINVAL),
    (lambda c, e: setattr(c, "hrss_moves", 1), gwns.NS_EINVAL),            # HRSS moves without HRSS
    (lambda c, e: (setattr(c, "proposal", gwns.NS_PROPOSAL_HRSS), setattr(c, "hrss_moves", -1)), gwns.NS_EINVAL),
    (lambda c, e: setattr(c, "flow_accept_weight", 10.0), gwns.NS_EINVAL),   # a flow weight without flow
    (lambda c, e: (setattr(c, "proposal", gwns.NS_PROPOSAL_DE_FLOW), setattr(c, "flow_accept_weight", 0.5)),
     gwns.NS_EINVAL),
    (lambda c, e: (setattr(c, "proposal", gwns.NS_PROPOSAL_DE_FLOW), setattr(c, "flow_accept_weight", float("nan"))),
     gwns.NS_EINVAL),
])
def test_init_rejects_bad_input_without_device_work(lib, mutate, code):
    w, ev = _event_and_config()
    cfg = gwns.make_config(w, synth.priors_with_injection(w, ev))
    evs, keep = gwns.make_event(ev)
    mutate(cfg, evs)
    h = C.c_void_p()
    got = lib.ns_init(C.byref(cfg), C.byref(evs), 1, 0, C.byref(h))
    assert got == code
    assert h.value is None
    assert len(gwns.ns_last_error(None)) > 0


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.ns_likelihood_batch(None, 0, None, 0, None, 0, None) == gwns.NS_EINVAL
    assert lib.ns_step(None, 1, None) == gwns.NS_EINVAL
    n = C.c_int32()
    assert lib.ns_flow_num_params(None, 0, C.byref(n)) == gwns.NS_EINVAL
    assert lib.ns_flow_logq(None, 0, None, 0, None, 0, None) == gwns.NS_EINVAL
    assert lib.ns_relbin_set(None, 0, None, 0, None) == gwns.NS_EINVAL
    assert lib.ns_hrss_batch(None, 0, None, 0, None, None, 0.0, 0, 0, 0, 0, None, None, None, None) == gwns.NS_EINVAL
    lib.ns_free(None)
