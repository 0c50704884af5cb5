"""Independent pin of the oracle's TaylorF2 phase coefficients (oracle/taylorf2.py).

The TaylorF2 phase is the stationary-phase approximation of an adiabatic inspiral: with the
binding energy E(v) and the gravitational-wave flux F(v) of circular orbits (v = (pi M f)^(1/3),
units G = c = M = 1), energy balance dE/dt = -F gives
    t(v) = t_c + int^v G dv',  phi(v) = phi_c + int^v v'^3 G dv',  G = -E'(v) / F(v),
and the stationary-phase Fourier phase is Psi(f) = 2 pi f t(v) - 2 phi(v) - pi/4 with
2 pi f = 2 v^3.  Expanding G in v, integrating term by term and collecting
Psi = 2 pi f t_c - 2 phi_c - pi/4 + 3 / (128 eta v^5) sum_k (a_k + a_k^l ln v) v^k
gives every coefficient from E and F alone.  (Terms in v^5 without ln v and in v^8 are a
constant and a linear function of f: they are absorbed into phi_c and t_c.)

E and F are written here from the PN energy and flux of circular orbits (Blanchet, Living Rev.
Relativ. 17, 2 (2014): non-spinning to 3PN in E and 3.5PN in F; spin-orbit terms to 3.5PN; the
leading spin-spin terms of Kidder 1995 for black holes), a source separate from the phase
coefficients that the oracle restates.  Their test-mass parts are pinned to the exact binding
energy of circular equatorial orbits in the Kerr metric (Schwarzschild for zero spin), re-expanded
in x = (M Omega)^(2/3), and the spin-spin flux in the test-mass limit to the Kerr flux
coefficient 33/16 q^2 of Tagoshi, Shibata, Tanaka & Sasaki 1996.

The oracle claims: the non-spinning phase to 3.5PN, spin-orbit terms at 1.5, 2.5, 3 and 3.5PN and
the spin-spin terms at 2PN (no spin-squared terms at 3PN and above).  The derived coefficients
are compared with phase_coefficients term by term at several (eta, chi1, chi2).
"""
import functools
import math

import numpy as np
import pytest

from oracle import taylorf2

sp = pytest.importorskip("sympy")

v, x, L = sp.symbols("v x L", positive=True)          # L stands for ln v
eta, X1, X2, c1, c2 = sp.symbols("eta X1 X2 chi1 chi2", real=True)
gE = sp.EulerGamma
PI = sp.pi


def spin_combinations():
    """S_l / M^2 and Sigma_l / M^2 of aligned spins, delta = X1 - X2 (X_i = m_i / M)."""
    s = X1 ** 2 * c1 + X2 ** 2 * c2
    sig = X2 * c2 - X1 * c1
    return s, sig, X1 - X2


def energy_coeffs():
    """E = -(eta x / 2) (1 + sum_k e_k x^(k/2)), k = 2..7."""
    s, sig, d = spin_combinations()
    R = sp.Rational
    return {
        2: -R(3, 4) - eta / 12,
        3: R(14, 3) * s + 2 * d * sig,
        4: -R(27, 8) + R(19, 8) * eta - eta ** 2 / 24 + (-2 * eta * c1 * c2 - X1 ** 2 * c1 ** 2 - X2 ** 2 * c2 ** 2),
        5: (11 - R(61, 9) * eta) * s + d * (3 - R(10, 3) * eta) * sig,
        6: -R(675, 64) + (R(34445, 576) - R(205, 96) * PI ** 2) * eta - R(155, 96) * eta ** 2 - R(35, 5184) * eta ** 3,
        7: (R(135, 4) - R(367, 4) * eta + R(29, 12) * eta ** 2) * s + d * (R(27, 4) - 39 * eta + R(5, 4) * eta ** 2) * sig,
    }


def flux_coeffs():
    """F = (32/5) eta^2 x^5 (1 + sum_k f_k x^(k/2)), k = 2..7; f_6 carries ln x through L
    (ln x = 2 ln v)."""
    s, sig, d = spin_combinations()
    R = sp.Rational
    return {
        2: -R(1247, 336) - R(35, 12) * eta,
        3: 4 * PI - 4 * s - R(5, 4) * d * sig,
        4: (-R(44711, 9072) + R(9271, 504) * eta + R(65, 18) * eta ** 2
            + R(31, 8) * eta * c1 * c2 + R(33, 16) * (X1 ** 2 * c1 ** 2 + X2 ** 2 * c2 ** 2)),
        5: (-R(8191, 672) - R(583, 24) * eta) * PI + (-R(9, 2) + R(272, 9) * eta) * s
           + (-R(13, 16) + R(43, 4) * eta) * d * sig,
        6: (R(6643739519, 69854400) + R(16, 3) * PI ** 2 - R(1712, 105) * gE - R(856, 105) * (sp.log(16) + 2 * L)
            + (-R(134543, 7776) + R(41, 48) * PI ** 2) * eta - R(94403, 3024) * eta ** 2 - R(775, 324) * eta ** 3
            - 16 * PI * s - R(31, 6) * PI * d * sig),
        7: ((-R(16285, 504) + R(214745, 1728) * eta + R(193385, 3024) * eta ** 2) * PI
            + (R(476645, 6804) + R(6172, 189) * eta - R(2810, 27) * eta ** 2) * s
            + (R(9535, 336) + R(1849, 126) * eta - R(1501, 36) * eta ** 2) * d * sig),
    }


def _int_v_power_log(m, A, B):
    """int v^m (A + B ln v) dv (m != -1), with ln v written L."""
    return A * v ** (m + 1) / (m + 1) + B * (v ** (m + 1) * L / (m + 1) - v ** (m + 1) / (m + 1) ** 2)


def _mul(a, b, n=8):
    """Product of two truncated series in v (coefficient lists), to order v^(n-1)."""
    out = [0] * n
    for i, ai in enumerate(a):
        if ai == 0:
            continue
        for j in range(n - i):
            if b[j] != 0:
                out[i + j] += ai * b[j]
    return [sp.expand(c) for c in out]


@functools.lru_cache(maxsize=None)
def derived_coefficients():
    """{k: (a_k, a_k^l)} of the stationary-phase phase, as sympy expressions (L = ln v)."""
    e, f = energy_coeffs(), flux_coeffs()
    n = 8
    # -E'(v) / (eta v) with E = -(eta v^2 / 2)(1 + sum e_k v^k):
    # d/dv [v^(k+2) e_k] / 2 = (k + 2) e_k v^(k+1) / 2, plus the ln v derivative of e_k (none:
    # the energy has no logarithm to this order)
    num = [sp.Integer(1)] + [0] * (n - 1)
    for k, ek in e.items():
        assert not ek.has(L)
        num[k] += sp.Rational(k + 2, 2) * ek
    # 1 / (1 + u), u = sum f_k v^k: sum_j (-u)^j to order v^7
    u = [0] * n
    for k, fk in f.items():
        u[k] = fk
    inv = [sp.Integer(1)] + [0] * (n - 1)
    term = [sp.Integer(1)] + [0] * (n - 1)
    for _ in range(1, n):
        term = _mul(term, [-c for c in u], n)
        inv = [sp.expand(a + b) for a, b in zip(inv, term)]
    P = _mul(num, inv, n)          # G = (5 / (32 eta)) v^-9 sum_k P_k v^k
    out = {}
    for k in range(n):
        pk = sp.expand(P[k])
        A, B = pk.coeff(L, 0), pk.coeff(L, 1)
        assert sp.expand(pk - A - B * L) == 0
        # t: int v^(k-9) P_k,  phi: int v^(k-6) P_k; k = 5 in phi is the ln v case (no L there)
        T = _int_v_power_log(k - 9, A, B)
        if k == 5:
            assert B == 0
            Phi = A * L
        else:
            Phi = _int_v_power_log(k - 6, A, B)
        # Psi_k = (5 / (32 eta)) (2 v^3 T - 2 Phi), in units of 3 / (128 eta v^5): the bracket
        # term (a_k + a_k^l L) v^k
        br = sp.expand((2 * v ** 3 * T - 2 * Phi) * sp.Rational(5, 32) * sp.Rational(128, 3) * v ** 5)
        assert sp.expand(br.subs(v, 1) * v ** k - br) == 0
        br = br.subs(v, 1)
        out[k] = (sp.expand(br.coeff(L, 0)), sp.expand(br.coeff(L, 1)))
    return out


def _spin_parts(expr, order):
    """Part of a polynomial in (chi1, chi2) of the given total degree."""
    p = sp.Poly(sp.expand(expr), c1, c2)
    return sum(coef * c1 ** i * c2 ** j for (i, j), coef in p.terms() if i + j == order)


CASES = [(0.8, 0.3, -0.2), (0.25, 0.9, 0.7), (1.0, -0.5, 0.4), (0.5, 0.0, 0.0), (0.137, -0.99, 0.99), (0.6, 0.7, -0.3)]


def _num(expr, q, chi1, chi2):
    x1, x2 = 1.0 / (1.0 + q), q / (1.0 + q)
    val = expr.subs({X1: sp.Float(x1, 30), X2: sp.Float(x2, 30), eta: sp.Float(x1 * x2, 30),
                     c1: sp.Float(chi1, 30), c2: sp.Float(chi2, 30)})
    return float(sp.N(val, 30))


def _oracle(q, chi1, chi2):
    eta_, delta_ = q / (1.0 + q) ** 2, (1.0 - q) / (1.0 + q)
    return taylorf2.phase_coefficients(eta_, delta_, chi1, chi2)


def _claimed(k, a, which):
    """The part of a derived coefficient that the oracle claims: every non-spinning term,
    terms linear in the spins at every order, spin-squared terms only at 2PN."""
    if which == "log":
        return a
    keep = _spin_parts(a, 0) + _spin_parts(a, 1)
    if k == 4:
        keep += _spin_parts(a, 2)
    return keep


@pytest.mark.parametrize("q,chi1,chi2", CASES)
def test_phase_coefficients_follow_from_energy_and_flux(q, chi1, chi2):
    der = derived_coefficients()
    a, al = _oracle(q, chi1, chi2)
    assert a[0] == 1.0 and a[1] == 0.0 and al[0] == 0.0
    for k in range(2, 8):
        dk, dkl = der[k]
        want = _num(_claimed(k, dk, "lin"), q, chi1, chi2)
        want_l = _num(dkl, q, chi1, chi2)
        if k == 5:
            # the v^5 constant is absorbed into phi_c; the oracle's convention a_5 = a_5^l / 3
            assert abs(al[5] - want_l) <= 1e-12 * max(1.0, abs(want_l)), (k, al[5], want_l)
            assert abs(a[5] - al[5] / 3.0) <= 1e-13 * max(1.0, abs(a[5]))
            continue
        assert abs(a[k] - want) <= 1e-12 * max(1.0, abs(want)), (k, a[k], want)
        assert abs(al[k] - want_l) <= 1e-12 * max(1.0, abs(want_l)), (k, al[k], want_l)


def test_only_the_claimed_terms_are_left_out():
    # what the derivation has beyond the oracle: spin-squared terms at 3PN and 3.5PN (products
    # of lower-order spin terms here), nothing else
    der = derived_coefficients()
    for k in range(8):
        for part in der[k]:
            rest = sp.expand(part - _claimed(k, part, "log" if part is der[k][1] else "lin"))
            if k < 6:
                assert rest == 0, (k, rest)
            else:
                assert _spin_parts(rest, 0) == 0 and _spin_parts(rest, 1) == 0


def test_energy_test_mass_limit_is_the_kerr_binding_energy():
    # Circular equatorial orbits of a test mass around a Kerr black hole of spin chi (prograde
    # for chi > 0), r = M / u^2: E/mu = (1 - 2 u^2 + chi u^3) / sqrt(1 - 3 u^2 + 2 chi u^3) - 1,
    # M Omega = u^3 / (1 + chi u^3).  In x = (M Omega)^(2/3) the PN energy with eta -> 0 (body 1
    # the black hole, X1 = 1, X2 = 0) must agree to x^(9/2) (3.5PN), for every power of chi.
    chi, u = sp.symbols("chi u", real=True)
    ekerr = (1 - 2 * u ** 2 + chi * u ** 3) / sp.sqrt(1 - 3 * u ** 2 + 2 * chi * u ** 3) - 1
    # u as a series in y = sqrt(x): y^3 = u^3 / (1 + chi u^3) -> u = y (1 - chi y^3)^(-1/3)
    y = sp.symbols("y", positive=True)
    u_of_y = y * (1 - chi * y ** 3) ** sp.Rational(-1, 3)
    lhs = sp.expand(sp.series(ekerr.subs(u, u_of_y), y, 0, 10).removeO())
    e = energy_coeffs()
    pn = -(y ** 2 / 2) * (1 + sum(ek * y ** k for k, ek in e.items()))
    pn = sp.expand(pn.subs({eta: 0, X1: 1, X2: 0, c1: chi, c2: 0}))
    # the spin-squared terms beyond 2PN are not in the PN expression: compare what it holds
    diff = sp.expand(lhs - pn)
    p = sp.Poly(diff, y, chi)
    for (ky, kc), coef in p.terms():
        if ky <= 9 and (kc <= 1 or (kc == 2 and ky <= 6)):
            assert coef == 0, (ky, kc, coef)


def test_spin_spin_flux_test_mass_limit():
    # the Kerr test-mass flux carries (33/16) q^2 x^2 (Tagoshi et al. 1996)
    f4 = flux_coeffs()[4].subs({eta: 0, X1: 1, X2: 0, c2: 0})
    assert sp.expand(f4 - (sp.Rational(-44711, 9072) + sp.Rational(33, 16) * c1 ** 2)) == 0


@pytest.mark.parametrize("k,planted", [(2, ("3715.0 / 756.0", "3716.0 / 756.0")),
                                       (4, ("15293365.0 / 508032.0", "15293356.0 / 508032.0")),
                                       (6, ("6848.0 / 21.0 * math.log(4.0)", "6848.0 / 21.0 * math.log(2.0)")),
                                       (7, ("378515.0 * eta / 1512.0", "378515.0 * eta / 1521.0")),
                                       (3, ("113.0 / 3.0 * delta * chia", "113.0 / 3.0 * delta * chis")),
                                       (6, ("PI * (2270.0 / 3.0 - 520.0 * eta) * chis", "PI * (2270.0 / 3.0 + 520.0 * eta) * chis")),
                                       (7, ("26804935.0 * eta / 6048.0", "26804935.0 * eta / 6084.0"))])
def test_a_planted_typo_fails_the_pin(k, planted, monkeypatch):
    # a mistake in one constant of the oracle's coefficients is caught by the derivation
    import inspect
    src = inspect.getsource(taylorf2.phase_coefficients)
    assert planted[0] in src
    ns = dict(taylorf2.__dict__)
    exec(compile(src.replace(planted[0], planted[1], 1), "planted", "exec"), ns)
    monkeypatch.setattr(taylorf2, "phase_coefficients", ns["phase_coefficients"])
    with pytest.raises(AssertionError):
        for q, chi1, chi2 in CASES:
            test_phase_coefficients_follow_from_energy_and_flux(q, chi1, chi2)
