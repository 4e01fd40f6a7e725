"""Manufactured-solution pin of the oracle's coefficients against Eq. 1.

The paper does not print the matrices M, L, A of Eq. 8 (it defers them to
the literature); the oracle derives them from the Teukolsky master equation
(Eq. 1) with the coordinates of Eqs. 2-3 and the ansatz of Eq. 4.  This test
applies Eq. 1, exactly as printed, to Psi = e^{i m phi~} r^3 Phi for an
analytic Phi(t, r*(r), theta) with sympy in Boyer-Lindquist coordinates, and
compares with the reduced second-order operator built from the oracle's
double-precision coefficients:
    Phi_tt - b^2 Phi_{r*r*} + c_t Phi_t + c_* Phi_{r*} + c_0 Phi
        - q (Phi_thth + cot th Phi_th)   =   Eq.1[Psi] * (-Delta/(Sigma^2 r^3)) e^{-i m phi~}.
A dropped term, a wrong sign or a wrong power of r in any coefficient fails.
It also checks d b/d r* by a finite difference and the source prefactor.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O

sp = pytest.importorskip("sympy")

CASES = [
    (0.0, -2, 2, 4.3, 1.1),
    (0.7, -2, 2, 4.3, 1.1),
    (0.7, -2, 1, 2.9, 2.5),
    (0.9, 2, 3, 6.1, 0.4),
    (0.99, -2, 4, 1.6, 0.2),
    (0.5, 0, 0, 12.0, 1.7),
    (0.95, -1, -3, 25.0, 2.9),
]


def _teukolsky_lhs(a_v, s, m, r_v, th_v, with_source):
    t, r, th, ph = sp.symbols("t r theta phi", real=True)
    M = sp.Integer(1)
    a = sp.nsimplify(a_v)
    rp = M + sp.sqrt(M ** 2 - a ** 2)
    rm = M - sp.sqrt(M ** 2 - a ** 2)
    Delta = r ** 2 - 2 * M * r + a ** 2
    if a == 0:
        rstar = r + 2 * M * sp.log((r - rp) / (2 * M))
        phit = ph
    else:
        rstar = (r + 2 * M * rp / (rp - rm) * sp.log((r - rp) / (2 * M))
                 - 2 * M * rm / (rp - rm) * sp.log((r - rm) / (2 * M)))
        # Eq. 3 integrated: phi~ = phi + a/(r+ - r-) ln((r - r+)/(r - r-))
        phit = ph + a / (rp - rm) * sp.log((r - rp) / (r - rm))
    X = sp.Symbol("X", real=True)
    w = sp.Rational(3, 10) - sp.I * sp.Rational(1, 10)
    g = sp.exp(-(X - 3) ** 2 / 7) * sp.cos(X / 5)
    k = (1 + sp.cos(th)) ** 2 + sp.Rational(1, 3) * sp.sin(th) ** 2 * sp.cos(th)
    Phi = sp.exp(-sp.I * w * t) * g.subs(X, rstar) * k
    Psi = sp.exp(sp.I * m * phit) * r ** 3 * Phi                       # Eq. 4
    SigBL = r ** 2 + a ** 2 * sp.cos(th) ** 2
    # Eq. 1, left side, term by term as printed
    L = (-(((r ** 2 + a ** 2) ** 2) / Delta - a ** 2 * sp.sin(th) ** 2) * sp.diff(Psi, t, 2)
         - 4 * M * a * r / Delta * sp.diff(Psi, t, ph)
         - 2 * s * (r - M * (r ** 2 - a ** 2) / Delta + sp.I * a * sp.cos(th)) * sp.diff(Psi, t)
         + Delta ** (-s) * sp.diff(Delta ** (s + 1) * sp.diff(Psi, r), r)
         + 1 / sp.sin(th) * sp.diff(sp.sin(th) * sp.diff(Psi, th), th)
         + (1 / sp.sin(th) ** 2 - a ** 2 / Delta) * sp.diff(Psi, ph, 2)
         + 2 * s * (a * (r - M) / Delta + sp.I * sp.cos(th) / sp.sin(th) ** 2) * sp.diff(Psi, ph)
         - (s ** 2 * sp.cot(th) ** 2 - s) * Psi)
    Sig2 = (r ** 2 + a ** 2) ** 2 - a ** 2 * Delta * sp.sin(th) ** 2  # Eq. 7
    scale = (-Delta / (Sig2 * r ** 3)) * sp.exp(-sp.I * m * phit)
    subs = {t: sp.Rational(1, 2), r: sp.nsimplify(r_v), th: sp.nsimplify(th_v), ph: sp.Rational(1, 3)}
    lhs = complex(sp.N((L * scale).subs(subs), 30))
    # right side of Eq. 1 with T = e^{i m phi~} T_m, per unit T_m, after the same scaling
    rhs_pref = complex(sp.N((-4 * sp.pi * SigBL * r ** 0 * (-Delta / (Sig2 * r ** 3))).subs(subs), 30))
    T, RS = sp.symbols("T RS", real=True)
    Phi2 = sp.exp(-sp.I * w * T) * g.subs(X, RS) * k
    rs_v = sp.N(rstar.subs(r, sp.nsimplify(r_v)), 30)
    s2 = {T: sp.Rational(1, 2), RS: rs_v, th: sp.nsimplify(th_v)}
    D = lambda e: complex(sp.N(e.subs(s2), 30))
    derivs = dict(tt=D(sp.diff(Phi2, T, 2)), rr=D(sp.diff(Phi2, RS, 2)), t=D(sp.diff(Phi2, T)),
                  r=D(sp.diff(Phi2, RS)), f=D(Phi2), hh=D(sp.diff(Phi2, th, 2)), h=D(sp.diff(Phi2, th)))
    x = float(sp.N(sp.nsimplify(r_v) - rp, 30))
    return lhs, rhs_pref, derivs, x


@pytest.mark.parametrize("a,s,m,r,th", CASES)
def test_reduced_operator_matches_eq1(a, s, m, r, th):
    lhs, rhs_pref, d, x = _teukolsky_lhs(a, s, m, r, th, True)
    p = O.OracleProblem(s=s, m=m, M=1.0, a=a, Nr=8, Ntheta=8, rs_min=-10, rs_max=10, dt=0.1, rs_ext=0)
    c = O.point_coef(p, x, th)
    ct = c["ct_re"] + 1j * c["ct_im"]
    cs = c["cs_re"] + 1j * c["cs_im"]
    c0 = c["c0rad_re"] + 1j * c["c0rad_im"] + c["c0ang"]
    red = (d["tt"] - c["b"] ** 2 * d["rr"] + ct * d["t"] + cs * d["r"] + c0 * d["f"]
           - c["q"] * (d["hh"] + math.cos(th) / math.sin(th) * d["h"]))
    assert abs(red - lhs) <= 1e-12 * abs(lhs), (red, lhs)
    # source prefactor F / T_m
    assert abs(c["Fpref"] - rhs_pref.real) <= 1e-13 * abs(rhs_pref.real) and abs(rhs_pref.imag) < 1e-20


@pytest.mark.parametrize("a", [0.0, 0.7, 0.99])
def test_first_order_form_consistent(a):
    """With Pi = Phi_t + b Phi_{r*} (Eq. 5), Pi_t - b Pi_{r*} + c_t Pi - K Phi_{r*}
    + c_0 Phi - q L_th Phi must equal the reduced operator: K = b c_t - c_* - b b_{,r*}.
    b_{,r*} is checked against a finite difference of the oracle's b along r*."""
    p = O.OracleProblem(s=-2, m=2, M=1.0, a=a, Nr=8, Ntheta=8, rs_min=-10, rs_max=10, dt=0.1, rs_ext=0)
    for rs in (-30.0, 0.0, 2.5, 40.0):
        for th in (0.3, 1.2, 2.8):
            h = 1e-4
            bp = O.point_coef(p, O.x_of_rstar(1.0, a, rs + h), th)["b"]
            bm = O.point_coef(p, O.x_of_rstar(1.0, a, rs - h), th)["b"]
            c = O.point_coef(p, O.x_of_rstar(1.0, a, rs), th)
            fd = (bp - bm) / (2 * h)
            assert abs(c["b_rs"] - fd) <= 1e-7 * max(abs(fd), 1e-9) + 1e-12
            # K relation, term by term
            K = c["K_re"] + 1j * c["K_im"]
            expect = c["b"] * (c["ct_re"] + 1j * c["ct_im"]) - (c["cs_re"] + 1j * c["cs_im"]) - c["b"] * c["b_rs"]
            assert abs(K - expect) <= 1e-14 * max(1.0, abs(K))


def test_schwarzschild_coefficients_real():
    """a = 0: every coefficient is real, so Phi_R and Phi_I decouple."""
    p = O.OracleProblem(s=-2, m=2, M=1.0, a=0.0, Nr=8, Ntheta=8, rs_min=-10, rs_max=10, dt=0.1, rs_ext=0)
    for rs in (-50.0, 0.0, 10.0, 300.0):
        c = O.point_coef(p, O.x_of_rstar(1.0, 0.0, rs), 0.7)
        assert c["ct_im"] == 0.0 and c["cs_im"] == 0.0 and c["c0rad_im"] == 0.0 and c["K_im"] == 0.0
        assert c["b"] == pytest.approx(1.0, abs=1e-15)
