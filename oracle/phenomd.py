"""IMRPhenomD-form aligned-spin inspiral-merger-ringdown waveform (the paper's analyses use
IMRPhenomD, Sec. 3.3).  The published IMRPhenomD calibration tables are not used: this is the
model's functional form with a stated form-only coefficient table (parity unpinned for physical
fidelity; the CUDA path implements the same form and table).

Geometric frequency x = M f (M the total mass in seconds).  With the TaylorF2 phase psi_TF2(x)
(oracle.taylorf2) and eta the symmetric mass ratio, the phase without the 2 pi f t_c - 2 phi_c - pi/4
part is, by region,
  inspiral      x < 0.018:  psi_TF2(x) + (3/4 s2 x^(4/3) + 3/5 s3 x^(5/3) + 1/2 s4 x^2) / eta
  intermediate  x < x2:     (b0 + b1 x + b2 ln x - b3 / (3 x^3)) / eta
  merger-ringdown x >= x2:  (a0 + a1 x - a2 / x + 4/3 a3 x^(3/4) + a4 atan((x - a5 f_RD) / f_damp)) / eta
with x2 = f_RD / 2, and (b0, b1), (a0, a1) fixed by continuity of the phase and its derivative at
the two boundaries.  The amplitude is K f^(-7/6) times a shape a(x):
  inspiral      x < 0.014:  1 + A2 v^2 + A3 v^3,  v = (pi x)^(1/3)  (1PN and 1.5PN amplitude terms)
  merger-ringdown x >= x_p: g1 g3 fd / ((x - fRD)^2 + (g3 fd)^2) exp(-g2 (x - fRD) / (g3 fd))
  intermediate: the cubic Hermite interpolant of value and slope at x = 0.014 and x_p,
with x_p = fRD + fd g3 (sqrt(1 - g2^2) - 1) / g2 the peak of the ringdown shape.  The waveform is
zero above x = 0.2.  The ringdown frequency fRD and damping fd (in units of 1/M) come from the
Kerr l = m = 2 fundamental quasi-normal mode fit of Berti, Cardoso & Will 2006 evaluated at the
remnant spin of the Rezzolla et al. 2008 final-spin formula and a remnant mass 1 - E_rad.

Pins: with the pseudo-PN coefficients zeroed the inspiral phase is TaylorF2; the phase and
amplitude are C1-continuous at every boundary; the QNM fit reproduces the Schwarzschild
l = 2 mode (M omega = 0.37367, Q = 2.10) to 2 %; the final-spin formula gives 0.686 for equal
masses without spin and reduces to the large body's spin in the test-mass limit.
"""
import math

import numpy as np

from .constants import MSUN_S
from . import taylorf2

PI = math.pi

# Form-only coefficient table (stand-in values, not the published calibration).
DEFAULT_TABLE = {
    "x_ins": 0.018,        # phase: end of the inspiral region
    "x_amp_ins": 0.014,    # amplitude: end of the inspiral region
    "x_cut": 0.2,          # no signal above
    "sigma": (50.0, -100.0, 40.0),      # s2, s3, s4
    "beta": (1.0, 1.0e-5),              # b2, b3
    "alpha": (0.01, 0.5, 0.05, 1.0),    # a2, a3, a4, a5
    "gamma": (0.006, 0.9, 1.3),         # g1, g2 (< 1: the ringdown shape has a peak), g3
    "erad": (0.0572, 0.498),            # E_rad = e1 eta + e2 eta^2
}


def final_spin(eta, q, chi1, chi2):
    """Remnant spin, Rezzolla et al. 2008 (aligned spins), q = m2/m1 <= 1."""
    at = (chi1 + chi2 * q * q) / (1.0 + q * q)
    s4, s5, t0, t2, t3 = -0.1229, 0.4537, -2.8904, -3.5171, 2.5763
    return at + at * eta * (s4 * at + s5 * eta + t0) + eta * (2.0 * math.sqrt(3.0) + t2 * eta + t3 * eta * eta)


def qnm22(af):
    """(M_f omega_R, Q) of the Kerr l = m = 2, n = 0 mode, Berti, Cardoso & Will 2006 fit."""
    om = 1.5251 - 1.1568 * (1.0 - af) ** 0.1292
    qf = 0.7000 + 1.4187 * (1.0 - af) ** (-0.4990)
    return om, qf


def ringdown(eta, q, chi1, chi2, table=None):
    """(fRD, fdamp) in units of 1/M."""
    t = DEFAULT_TABLE if table is None else table
    af = final_spin(eta, q, chi1, chi2)
    mf = 1.0 - (t["erad"][0] * eta + t["erad"][1] * eta * eta)
    om, qf = qnm22(af)
    f_rd = om / (2.0 * PI * mf)
    return f_rd, f_rd / (2.0 * qf)


def _tf2_phase_x(x, eta, delta, chi1, chi2):
    """TaylorF2 PN phase as a function of x = M f, and its derivative d/dx."""
    a, al = taylorf2.phase_coefficients(eta, delta, chi1, chi2)
    x = np.asarray(x, dtype=np.float64)
    v = (PI * x) ** (1.0 / 3.0)
    lnv = np.log(v)
    s = np.zeros_like(v)
    ds = np.zeros_like(v)
    for k in range(8):
        s = s + (a[k] + al[k] * lnv) * v ** (k - 5)
        # d/dx v^(k-5) (a + al ln v) = v^(k-5) / (3 x) ((k-5)(a + al ln v) + al)
        ds = ds + v ** (k - 5) / (3.0 * x) * ((k - 5) * (a[k] + al[k] * lnv) + al[k])
    c = 3.0 / (128.0 * eta)
    return c * s, c * ds


def phase_parts(eta, delta, chi1, chi2, f_rd, f_damp, table=None):
    """The region functions psi_ins, psi_int, psi_mr of x (continuity constants solved)."""
    t = DEFAULT_TABLE if table is None else table
    s2, s3, s4 = t["sigma"]
    b2, b3 = t["beta"]
    a2, a3, a4, a5 = t["alpha"]
    x1 = t["x_ins"]
    x2 = 0.5 * f_rd

    def ins(x):
        p, dp = _tf2_phase_x(x, eta, delta, chi1, chi2)
        x = np.asarray(x, dtype=np.float64)
        p = p + (0.75 * s2 * x ** (4.0 / 3.0) + 0.6 * s3 * x ** (5.0 / 3.0) + 0.5 * s4 * x * x) / eta
        dp = dp + (s2 * x ** (1.0 / 3.0) + s3 * x ** (2.0 / 3.0) + s4 * x) / eta
        return p, dp

    p1, dp1 = ins(np.array([x1]))
    b1 = eta * dp1[0] - b2 / x1 - b3 / x1 ** 4
    b0 = eta * p1[0] - b1 * x1 - b2 * math.log(x1) + b3 / (3.0 * x1 ** 3)

    def inter(x):
        x = np.asarray(x, dtype=np.float64)
        p = (b0 + b1 * x + b2 * np.log(x) - b3 / (3.0 * x ** 3)) / eta
        dp = (b1 + b2 / x + b3 / x ** 4) / eta
        return p, dp

    p2, dp2 = inter(np.array([x2]))

    def lor(x):
        return a4 * np.arctan((x - a5 * f_rd) / f_damp), a4 * f_damp / ((x - a5 * f_rd) ** 2 + f_damp ** 2)

    l2, dl2 = lor(x2)
    al1 = eta * dp2[0] - a2 / x2 ** 2 - a3 * x2 ** (-0.25) - dl2
    al0 = eta * p2[0] - al1 * x2 + a2 / x2 - (4.0 / 3.0) * a3 * x2 ** 0.75 - l2

    def mr(x):
        x = np.asarray(x, dtype=np.float64)
        l, dl = lor(x)
        p = (al0 + al1 * x - a2 / x + (4.0 / 3.0) * a3 * x ** 0.75 + l) / eta
        dp = (al1 + a2 / x ** 2 + a3 * x ** (-0.25) + dl) / eta
        return p, dp

    return ins, inter, mr, (x1, x2), {"b0": b0, "b1": b1, "a0": al0, "a1": al1}


def amplitude_parts(eta, delta, chi1, chi2, f_rd, f_damp, table=None):
    """Region functions of the amplitude shape a(x) and their derivatives."""
    t = DEFAULT_TABLE if table is None else table
    g1, g2, g3 = t["gamma"]
    xa = t["x_amp_ins"]
    chis, chia = 0.5 * (chi1 + chi2), 0.5 * (chi1 - chi2)
    A2 = -323.0 / 224.0 + 451.0 * eta / 168.0
    A3 = 27.0 * delta * chia / 8.0 + (27.0 / 8.0 - 11.0 * eta / 6.0) * chis

    def ins(x):
        x = np.asarray(x, dtype=np.float64)
        v = (PI * x) ** (1.0 / 3.0)
        a = 1.0 + A2 * v * v + A3 * v ** 3
        # dv/dx = v / (3 x)
        da = (2.0 * A2 * v + 3.0 * A3 * v * v) * v / (3.0 * x)
        return a, da

    gd = g3 * f_damp

    def mr(x):
        x = np.asarray(x, dtype=np.float64)
        d = x - f_rd
        e = np.exp(-g2 * d / gd)
        den = d * d + gd * gd
        a = g1 * gd / den * e
        da = a * (-2.0 * d / den - g2 / gd)
        return a, da

    xp = abs(f_rd + gd * (math.sqrt(1.0 - g2 * g2) - 1.0) / g2)
    y0, d0 = ins(np.array([xa]))
    y1, d1 = mr(np.array([xp]))
    y0, d0, y1, d1 = y0[0], d0[0], y1[0], d1[0]
    hspan = xp - xa

    def inter(x):
        x = np.asarray(x, dtype=np.float64)
        s = (x - xa) / hspan
        h00 = 2 * s ** 3 - 3 * s ** 2 + 1
        h10 = s ** 3 - 2 * s ** 2 + s
        h01 = -2 * s ** 3 + 3 * s ** 2
        h11 = s ** 3 - s ** 2
        a = h00 * y0 + h10 * hspan * d0 + h01 * y1 + h11 * hspan * d1
        dh00 = (6 * s ** 2 - 6 * s) / hspan
        dh10 = (3 * s ** 2 - 4 * s + 1) / hspan
        dh01 = (-6 * s ** 2 + 6 * s) / hspan
        dh11 = (3 * s ** 2 - 2 * s) / hspan
        da = dh00 * y0 + dh10 * hspan * d0 + dh01 * y1 + dh11 * hspan * d1
        return a, da

    return ins, inter, mr, (xa, xp)


def phase_and_amplitude(f, theta, table=None):
    """(Psi(f) without the t_c, phi_c terms, amplitude shape a(f), cutoff mask) for theta."""
    t = DEFAULT_TABLE if table is None else table
    mc, q, chi1, chi2 = (float(v) for v in theta[:4])
    mtot, eta, delta = taylorf2.masses(mc, q)
    f_rd, f_damp = ringdown(eta, q, chi1, chi2, t)
    x = mtot * MSUN_S * np.asarray(f, dtype=np.float64)
    pins, pint, pmr, (x1, x2), _ = phase_parts(eta, delta, chi1, chi2, f_rd, f_damp, t)
    ains, aint, amr, (xa, xp) = amplitude_parts(eta, delta, chi1, chi2, f_rd, f_damp, t)
    psi = np.where(x < x1, pins(x)[0], np.where(x < x2, pint(x)[0], pmr(x)[0]))
    amp = np.where(x < xa, ains(x)[0], np.where(x < xp, aint(x)[0], amr(x)[0]))
    on = x <= t["x_cut"]
    return psi, amp, on


def polarizations(f, theta, table=None, cutoff: bool = True):
    """(h+, hx) [1/Hz]: K f^(-7/6) a(f) with the TaylorF2 normalisation and polarisation factors;
    cutoff=False continues the merger-ringdown form above Mf = x_cut."""
    mc, q, chi1, chi2, dist, iota, _psi, phic, tc = (float(v) for v in theta[:9])
    f = np.asarray(f, dtype=np.float64)
    psi_pn, shape, on = phase_and_amplitude(f, theta, table)
    psi_f = 2.0 * PI * f * tc - 2.0 * phic - PI / 4.0 + psi_pn
    amp = taylorf2.amplitude(f, mc, dist) * shape
    if cutoff:
        amp = np.where(on, amp, 0.0)
    ci = math.cos(iota)
    e = np.exp(-1j * psi_f)
    return amp * 0.5 * (1.0 + ci * ci) * e, -1j * amp * ci * e
