"""Pins of the oracle's detector response, TaylorF2 waveform and likelihood against
closed forms, textbook special cases and exact invariances."""
import math

import numpy as np
import pytest

from oracle import detector, likelihood as L, taylorf2
from oracle.constants import C_SI, MSUN_S
from paper_2509_04336_gb300 import synth

GMST = synth.GMST_RAD


# ---------------- detector response -------------------------------------------------
def test_overhead_source_full_response():
    # Arms along x and y at the north pole; a source at the zenith sees |F|^2 = 1 and
    # arrives R/c before the geocentre.
    x, y, r = np.array([1.0, 0, 0]), np.array([0, 1.0, 0]), np.array([0, 0, 6.371e6])
    for psi in (0.0, 0.3, 1.1):
        fp, fc = detector.antenna_pattern(x, y, 0.7, math.pi / 2, psi, 0.2)
        assert abs(fp * fp + fc * fc - 1.0) < 1e-14
    assert abs(detector.time_delay(r, 0.1, math.pi / 2, 0.0) + 6.371e6 / C_SI) < 1e-18


@pytest.mark.parametrize("theta,phi", [(0.3, 0.2), (1.0, 2.0), (2.5, -1.2), (math.pi / 2, 0.7)])
def test_polar_detector_textbook_response(theta, phi):
    # Detector at the north pole with arms along x, y: F+^2 + Fx^2 equals
    # (1 + cos^2 th)^2 cos^2 2ph / 4 + cos^2 th sin^2 2ph for every psi (Thorne 1987).
    x, y = np.array([1.0, 0, 0]), np.array([0, 1.0, 0])
    dec, ra = math.pi / 2 - theta, phi
    want = 0.25 * (1 + math.cos(theta) ** 2) ** 2 * math.cos(2 * phi) ** 2 + (math.cos(theta) * math.sin(2 * phi)) ** 2
    for psi in (0.0, 0.9, 2.0):
        fp, fc = detector.antenna_pattern(x, y, ra, dec, psi, 0.0)
        assert abs(fp * fp + fc * fc - want) < 1e-13


def test_polarisation_angle_rotates_response_by_two_psi():
    v, x, y = synth.detector_vectors("L")
    f0 = complex(*detector.antenna_pattern(x, y, 1.0, -0.4, 0.0, GMST))
    for psi in (0.2, 1.3, 2.9):
        f = complex(*detector.antenna_pattern(x, y, 1.0, -0.4, psi, GMST))
        assert abs(abs(f) - abs(f0)) < 1e-14
        assert abs(f - f0 * np.exp(-2j * psi)) < 1e-13 or abs(f - f0 * np.exp(2j * psi)) < 1e-13


def test_time_delay_bounded_by_baseline():
    rh, _, _ = synth.detector_vectors("H")
    rl, _, _ = synth.detector_vectors("L")
    base = np.linalg.norm(rh - rl) / C_SI
    rng = np.random.default_rng(0)
    for _ in range(200):
        ra, dec = rng.uniform(0, 2 * math.pi), math.asin(rng.uniform(-1, 1))
        d = detector.time_delay(rh, ra, dec, GMST) - detector.time_delay(rl, ra, dec, GMST)
        assert abs(d) <= base * (1 + 1e-12)
    # a source along the baseline direction reaches the maximum
    n = (rl - rh) / np.linalg.norm(rl - rh)
    dec = math.asin(n[2])
    ra = math.atan2(n[1], n[0]) + GMST
    d = detector.time_delay(rh, ra, dec, GMST) - detector.time_delay(rl, ra, dec, GMST)
    assert abs(d - base) < 1e-15


# ---------------- TaylorF2 ---------------------------------------------------------
def test_newtonian_phase_closed_form():
    # 3/(128 eta v^5) = 3/128 (pi Mc f)^(-5/3): the leading phase depends on Mc alone.
    f = np.linspace(20, 60, 9)
    for mc, q in ((28.0, 0.8), (10.0, 0.25), (45.0, 1.0)):
        got = taylorf2.pn_phase(f, mc, q, 0.3, -0.2, pn_order=0)
        want = 3.0 / 128.0 * (math.pi * mc * MSUN_S * f) ** (-5.0 / 3.0)
        assert np.allclose(got, want, rtol=1e-13)


def test_newtonian_chirp_time():
    # (1/2 pi) dPsi_0/df = -tau_0 with tau_0 = 5/256 (pi f)^(-8/3) Mc^(-5/3) (geometric units).
    mc, f, h = 30.0, 40.0, 1e-4
    d = (taylorf2.pn_phase([f + h], mc, 0.7, 0, 0, 0)[0] - taylorf2.pn_phase([f - h], mc, 0.7, 0, 0, 0)[0]) / (2 * h)
    tau0 = 5.0 / 256.0 * (math.pi * f) ** (-8.0 / 3.0) * (mc * MSUN_S) ** (-5.0 / 3.0)
    assert abs(d / (2 * math.pi) + tau0) < 1e-8 * tau0


def test_exchange_symmetry():
    # (m1, chi1) <-> (m2, chi2): q -> 1/q with the spins swapped leaves the phase unchanged.
    f = np.linspace(20, 70, 11)
    a = taylorf2.pn_phase(f, 30.0, 0.6, 0.7, -0.3)
    b = taylorf2.pn_phase(f, 30.0, 1 / 0.6, -0.3, 0.7)
    assert np.allclose(a, b, rtol=1e-13, atol=1e-10)


def test_equal_mass_spin_structure():
    # delta = 0: the phase depends on the spins through chi_s and chi_a^2 only.
    f = np.linspace(20, 70, 11)
    a = taylorf2.pn_phase(f, 30.0, 1.0, 0.5, 0.1)
    b = taylorf2.pn_phase(f, 30.0, 1.0, 0.1, 0.5)
    assert np.allclose(a, b, rtol=1e-13)
    c = taylorf2.pn_phase(f, 30.0, 1.0, 0.3, 0.3)
    assert not np.allclose(a, c, rtol=1e-6)


def test_zero_spin_and_spin_terms_present():
    f = np.linspace(20, 70, 5)
    base = taylorf2.pn_phase(f, 30.0, 0.5, 0.0, 0.0)
    spun = taylorf2.pn_phase(f, 30.0, 0.5, 0.5, 0.0)
    assert np.all(np.abs(spun - base) > 1e-3)
    # aligned spins lengthen the inspiral: a positive 1.5PN spin-orbit term at low v
    a, _ = taylorf2.phase_coefficients(0.2, 0.4, 0.0, 0.0)
    b, _ = taylorf2.phase_coefficients(0.2, 0.4, 0.5, 0.5)
    assert b[3] > a[3]


def test_amplitude_distance_and_cutoff():
    f = np.array([20.0, 40.0, 60.0, 70.0])
    th = np.array([28.0, 0.8, 0.3, -0.2, 500.0, 0.4, 2.66, 1.3, 0.0, 1.38, -1.21])
    hp1, hc1 = taylorf2.polarizations(f, th)
    th2 = th.copy(); th2[4] = 1000.0
    hp2, _ = taylorf2.polarizations(f, th2)
    assert np.allclose(hp1, 2 * hp2, rtol=1e-14)
    fcut = taylorf2.cutoff_frequency(28.0, 0.8)
    assert 60.0 < fcut < 70.0 and hp1[3] == 0 and hp1[2] != 0
    # face-on: circular polarisation, hx = -i h+
    th3 = th.copy(); th3[5] = 0.0
    hp3, hc3 = taylorf2.polarizations(f, th3)
    assert np.allclose(hc3, -1j * hp3, rtol=1e-14)


# ---------------- likelihood --------------------------------------------------------
@pytest.fixture(scope="module")
def zero_noise_event():
    w = synth.workload("four_param_2det_taylorf2")
    return w, synth.make_event(w, L.project, L.inner)


def test_zero_noise_truth_has_zero_lnl_and_target_snr(zero_noise_event):
    w, ev = zero_noise_event
    assert L.log_likelihood(ev, ev.theta_inj) == 0.0
    assert abs(L.network_snr(ev, ev.theta_inj) - 20.0) < 1e-12
    # <h|h> scales exactly as d_L^-2
    th = ev.theta_inj.copy(); th[4] *= 2.0
    assert abs(L.network_snr(ev, th) - 10.0) < 1e-12
    # use_ratio: ln Lambda = ln L + <d|d>/2, and at the truth it equals SNR^2/2
    assert abs(L.log_likelihood(ev, ev.theta_inj, use_ratio=True) - 200.0) < 1e-9


def test_likelihood_polarisation_phase_invariance(zero_noise_event):
    # psi -> psi + pi/2 flips F+ and Fx; phi_c -> phi_c + pi/2 shifts Psi by -pi.
    _, ev = zero_noise_event
    th = np.array([30.0, 0.6, 0.1, 0.2, 800.0, 1.0, 0.5, 2.0, 0.01, 2.0, 0.3])
    th2 = th.copy(); th2[6] += math.pi / 2; th2[7] += math.pi / 2
    th3 = th.copy(); th3[6] += math.pi
    a, b, c = (L.log_likelihood(ev, x) for x in (th, th2, th3))
    assert abs(a - b) < 1e-9 * abs(a) and abs(a - c) < 1e-9 * abs(a)


def test_likelihood_brute_force_small_case():
    # A 4-bin two-detector event evaluated term by term with Python complex scalars.
    w = synth.shrink(synth.workload("four_param_2det_taylorf2"), f_max=20.75)
    ev = synth.make_event(w, L.project, L.inner)
    assert ev.n_bins == 4
    th = ev.theta_inj.copy(); th[0] = 27.5; th[8] = 0.003
    f = [20.0, 20.25, 20.5, 20.75]
    total = 0.0
    for d in ev.detectors:
        fp, fc = detector.antenna_pattern(d.x_arm, d.y_arm, th[9], th[10], th[6], ev.gmst)
        dt = detector.time_delay(d.vertex, th[9], th[10], ev.gmst)
        for k in range(4):
            hp, hc = taylorf2.polarizations(np.array([f[k]]), th)
            h = (fp * complex(hp[0]) + fc * complex(hc[0])) * complex(math.cos(-2 * math.pi * f[k] * dt), math.sin(-2 * math.pi * f[k] * dt))
            r = complex(d.data[k]) - h
            total += 4 * 0.25 * (r.real ** 2 + r.imag ** 2) / d.psd[k]
    assert abs(L.log_likelihood(ev, th) - (-0.5 * total)) < 1e-12 * abs(total)


def test_noise_normalisation():
    # E<n|n> = 2 per bin: the whitened noise power over 4017 x 3 bins is chi^2 with 2N dof.
    w = synth.workload("bbh11_3det_4s_taylorf2")
    f = synth.frequencies(w.f_min, w.df, w.n_bins)
    psd = synth.analytic_psd(f)
    tot, n = 0.0, 0
    for det in range(3):
        nz = synth.gaussian_noise(psd, w.df, 5, 0, det)
        tot += L.inner(nz, nz, psd, w.df); n += w.n_bins
    assert abs(tot - 2 * n) < 5 * math.sqrt(4 * n)
