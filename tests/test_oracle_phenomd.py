"""Pins of the oracle's IMRPhenomD-form waveform: TaylorF2 limits, C1 continuity of every
region boundary, the Kerr quasi-normal-mode and final-spin fits at known points."""
import math

import numpy as np
import pytest

from oracle import likelihood as L, phenomd as P, taylorf2 as T
from oracle.constants import MSUN_S
from paper_2509_04336_gb300 import synth

CASES = [(10.0, 0.7, -0.34, 0.01), (35.0, 0.9, 0.4, -0.3), (20.0, 0.3, 0.8, -0.8), (15.0, 1.0, 0.0, 0.0)]


def test_qnm_fit_reproduces_schwarzschild_mode():
    # Schwarzschild l = 2 fundamental mode: M omega = 0.37367 - 0.08896 i (Chandrasekhar &
    # Detweiler 1975), quality factor Q = omega_R / (2 omega_I) = 2.100.
    om, qf = P.qnm22(0.0)
    assert abs(om - 0.37367) / 0.37367 < 0.02
    assert abs(qf - 0.37367 / (2 * 0.08896)) / 2.100 < 0.02
    # faster-spinning remnants ring at higher frequency and longer
    om2, q2 = P.qnm22(0.9)
    assert om2 > om and q2 > qf


def test_final_spin_limits():
    # equal masses without spin: 0.686 (numerical relativity); test-mass limit: the large body's spin
    assert abs(P.final_spin(0.25, 1.0, 0.0, 0.0) - 0.686) < 0.005
    for chi in (-0.5, 0.0, 0.7):
        assert abs(P.final_spin(1e-9, 1e-9, chi, 0.3) - chi) < 1e-6


@pytest.mark.parametrize("case", CASES)
def test_inspiral_is_taylorf2_without_pseudo_pn(case):
    mc, q, c1, c2 = case
    table = dict(P.DEFAULT_TABLE, sigma=(0.0, 0.0, 0.0))
    mtot, eta, delta = T.masses(mc, q)
    frd, fd = P.ringdown(eta, q, c1, c2, table)
    ins, _, _, (x1, _), _ = P.phase_parts(eta, delta, c1, c2, frd, fd, table)
    f = np.linspace(20.0, 0.95 * x1 / (mtot * MSUN_S), 50)
    got = ins(mtot * MSUN_S * f)[0]
    want = T.pn_phase(f, mc, q, c1, c2)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("case", CASES)
def test_low_frequency_limit_is_taylorf2(case):
    # the pseudo-PN terms scale as x^(4/3) and higher: relative to the phase they vanish as x -> 0
    mc, q, c1, c2 = case
    mtot, eta, delta = T.masses(mc, q)
    frd, fd = P.ringdown(eta, q, c1, c2)
    ins, _, _, _, _ = P.phase_parts(eta, delta, c1, c2, frd, fd)
    prev = None
    for x in (1e-3, 1e-4, 1e-5):
        d = abs(ins(np.array([x]))[0][0] - T.pn_phase([x / (mtot * MSUN_S)], mc, q, c1, c2)[0])
        rel = d / abs(T.pn_phase([x / (mtot * MSUN_S)], mc, q, c1, c2)[0])
        if prev is not None:
            assert rel < 0.05 * prev
        prev = rel
    assert prev < 1e-9


@pytest.mark.parametrize("case", CASES)
def test_c1_continuity_and_derivatives(case):
    mc, q, c1, c2 = case
    mtot, eta, delta = T.masses(mc, q)
    frd, fd = P.ringdown(eta, q, c1, c2)
    pins, pint, pmr, (x1, x2), _ = P.phase_parts(eta, delta, c1, c2, frd, fd)
    ains, aint, amr, (xa, xp) = P.amplitude_parts(eta, delta, c1, c2, frd, fd)
    for xb, left, right in ((x1, pins, pint), (x2, pint, pmr), (xa, ains, aint), (xp, aint, amr)):
        l, r = left(np.array([xb])), right(np.array([xb]))
        assert abs(l[0][0] - r[0][0]) <= 1e-10 * max(1.0, abs(l[0][0]))
        assert abs(l[1][0] - r[1][0]) <= 1e-8 * max(1.0, abs(l[1][0]))
    # the analytic derivatives are the derivatives (central differences)
    h = 1e-7
    for fn, x in ((pins, 0.01), (pint, 0.03), (pmr, 0.07), (ains, 0.01), (aint, 0.03), (amr, 0.09)):
        num = (fn(np.array([x + h]))[0][0] - fn(np.array([x - h]))[0][0]) / (2 * h)
        assert abs(num - fn(np.array([x]))[1][0]) <= 1e-6 * max(1.0, abs(num))
    # the ringdown shape peaks at x_p
    a = amr(np.array([xp - 1e-4, xp, xp + 1e-4]))[0]
    assert a[1] >= a[0] and a[1] >= a[2]


def test_amplitude_shape_limits_and_cutoff():
    th = synth.TABLE4_INJECTION.copy()
    mtot, _, _ = T.masses(th[0], th[1])
    f = np.array([1e-3, 1.0, 20.0, 0.199 / (mtot * MSUN_S), 0.201 / (mtot * MSUN_S)])
    _, shape, on = P.phase_and_amplitude(f, th)
    assert abs(shape[0] - 1.0) < 1e-4 and on[3] and not on[4]
    hp, hc = P.polarizations(f, th)
    assert hp[4] == 0 and hc[4] == 0


def test_phenomd_likelihood_zero_noise_and_snr():
    w = synth.shrink(synth.workload("bbh11_3det_8s_phenomd"), f_max=600.0)
    from dataclasses import replace
    w = replace(w, noise=False)
    ev = synth.make_event(w, lambda e, i, th: L.project(e, i, th, w.waveform), L.inner)
    assert L.log_likelihood(ev, ev.theta_inj, w.waveform) == 0.0
    assert abs(L.network_snr(ev, ev.theta_inj, w.waveform) - 30.0) < 1e-10
