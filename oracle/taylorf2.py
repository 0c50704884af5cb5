"""3.5PN aligned-spin TaylorF2 frequency-domain waveform (the workload waveform of the
TaylorF2 configurations; the paper's own analyses use IMRPhenomD, Sec. 3.3).

Stationary-phase waveform, Fourier convention h(f) = int h(t) exp(-2 pi i f t) dt:
  h+(f) = A(f) (1 + cos^2 iota)/2 exp(-i Psi(f)),   hx(f) = -i A(f) cos iota exp(-i Psi(f)),
  A(f)  = sqrt(5/24) pi^(-2/3) (G Mc/c^3)^(5/6) f^(-7/6) / (d_L/c)    (restricted amplitude),
  Psi(f) = 2 pi f t_c - 2 phi_c - pi/4 + 3/(128 eta v^5) sum_k (a_k + a_k^l ln v) v^k,
  v = (pi M f)^(1/3),
both zero above f_cut = 1/(6^(3/2) pi M) (test-mass ISCO; the paper is silent on the cutoff).

Phase coefficients a_k: non-spinning terms as collected in Buonanno, Iyer, Ochsner, Pan &
Sathyaprakash 2009 (Eq. 3.18); aligned-spin terms (1.5PN and 2.5PN spin-orbit, 2PN spin-spin,
3PN and 3.5PN spin-orbit) in the chi_s, chi_a, delta form collected in Khan et al. 2016
(IMRPhenomD paper, Appendix B).  Pins: the Newtonian phase equals 3/128 (pi Mc f)^(-5/3),
its frequency derivative gives the Newtonian chirp time, the phase is invariant under the
exchange (m1, chi1) <-> (m2, chi2), and equal-mass phases depend on the spins only through
chi_s and chi_a^2.  Every coefficient a_k, a_k^l (k >= 2) is pinned independently by the
stationary-phase derivation from the PN binding energy and flux of circular orbits, whose
test-mass parts are the exact Kerr binding energy (tests/test_oracle_taylorf2_spa.py).
"""
import math

import numpy as np

from .constants import EULER_GAMMA, MPC_SI, MSUN_S, C_SI

PI = math.pi


def masses(mc: float, q: float):
    """Total mass M [Msun], symmetric mass ratio eta, delta = (m1 - m2)/M for q = m2/m1."""
    eta = q / (1.0 + q) ** 2
    mtot = mc * eta ** (-0.6)
    delta = (1.0 - q) / (1.0 + q)
    return mtot, eta, delta


def phase_coefficients(eta: float, delta: float, chi1: float, chi2: float):
    """(a[0..7], a_log[0..7]) multiplying v^k and v^k ln v inside the bracket."""
    chis = 0.5 * (chi1 + chi2)
    chia = 0.5 * (chi1 - chi2)
    e2, e3 = eta * eta, eta * eta * eta
    a = np.zeros(8)
    al = np.zeros(8)
    a[0] = 1.0
    a[2] = 3715.0 / 756.0 + 55.0 * eta / 9.0
    a[3] = -16.0 * PI + 113.0 / 3.0 * delta * chia + (113.0 / 3.0 - 76.0 * eta / 3.0) * chis
    a[4] = (15293365.0 / 508032.0 + 27145.0 * eta / 504.0 + 3085.0 * e2 / 72.0
            + (-405.0 / 8.0 + 200.0 * eta) * chia * chia
            - 405.0 / 4.0 * delta * chia * chis
            + (-405.0 / 8.0 + 5.0 * eta / 2.0) * chis * chis)
    gamma_so = ((732985.0 / 2268.0 - 24260.0 * eta / 81.0 - 340.0 * e2 / 9.0) * chis
                + (732985.0 / 2268.0 + 140.0 * eta / 9.0) * delta * chia)
    a[5] = 38645.0 * PI / 756.0 - 65.0 * PI * eta / 9.0 - gamma_so
    al[5] = 3.0 * a[5]
    a[6] = (11583231236531.0 / 4694215680.0 - 6848.0 * EULER_GAMMA / 21.0 - 640.0 * PI * PI / 3.0
            + (-15737765635.0 / 3048192.0 + 2255.0 * PI * PI / 12.0) * eta
            + 76055.0 * e2 / 1728.0 - 127825.0 * e3 / 1296.0
            - 6848.0 / 21.0 * math.log(4.0)
            + PI * 2270.0 / 3.0 * delta * chia + PI * (2270.0 / 3.0 - 520.0 * eta) * chis)
    al[6] = -6848.0 / 21.0
    a[7] = (PI * (77096675.0 / 254016.0 + 378515.0 * eta / 1512.0 - 74045.0 * e2 / 756.0)
            + (-25150083775.0 / 3048192.0 + 10566655595.0 * eta / 762048.0
               - 1042165.0 * e2 / 3024.0 + 5345.0 * e3 / 36.0) * chis
            + (-25150083775.0 / 3048192.0 + 26804935.0 * eta / 6048.0 - 1985.0 * e2 / 48.0) * delta * chia)
    return a, al


def pn_phase(f, mc: float, q: float, chi1: float, chi2: float, pn_order: int = 7) -> np.ndarray:
    """3/(128 eta v^5) sum_{k<=pn_order} (a_k + a_k^l ln v) v^k  [rad]."""
    mtot, eta, delta = masses(mc, q)
    a, al = phase_coefficients(eta, delta, chi1, chi2)
    v = (PI * mtot * MSUN_S * np.asarray(f, dtype=np.float64)) ** (1.0 / 3.0)
    lnv = np.log(v)
    s = np.zeros_like(v)
    for k in range(pn_order + 1):
        s = s + (a[k] + al[k] * lnv) * v ** k
    return 3.0 / (128.0 * eta * v ** 5) * s


def cutoff_frequency(mc: float, q: float) -> float:
    mtot, _, _ = masses(mc, q)
    return 1.0 / (6.0 ** 1.5 * PI * mtot * MSUN_S)


def amplitude(f, mc: float, dist_mpc: float) -> np.ndarray:
    mc_s = mc * MSUN_S
    d_s = dist_mpc * MPC_SI / C_SI
    return math.sqrt(5.0 / 24.0) * PI ** (-2.0 / 3.0) * mc_s ** (5.0 / 6.0) * np.asarray(f, dtype=np.float64) ** (-7.0 / 6.0) / d_s


def polarizations(f, theta, cutoff: bool = True):
    """(h+, hx) [1/Hz] at frequencies f for the physical parameters theta [11]; cutoff=False
    continues the formula above f_cut (a smooth reference for relative binning)."""
    mc, q, chi1, chi2, dist, iota, _psi, phic, tc = (float(x) for x in theta[:9])
    f = np.asarray(f, dtype=np.float64)
    psi_f = 2.0 * PI * f * tc - 2.0 * phic - PI / 4.0 + pn_phase(f, mc, q, chi1, chi2)
    amp = amplitude(f, mc, dist)
    if cutoff:
        amp = np.where(f <= cutoff_frequency(mc, q), amp, 0.0)
    ci = math.cos(iota)
    e = np.exp(-1j * psi_f)
    hp = amp * 0.5 * (1.0 + ci * ci) * e
    hc = -1j * amp * ci * e
    return hp, hc
