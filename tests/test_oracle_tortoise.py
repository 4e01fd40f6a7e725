"""Pins of the oracle's tortoise map (Eq. 2) and orbit frequency.

The oracle integrates Eq. 2 (dr*/dr = (r^2+a^2)/Delta) in closed form and
inverts it by a bracketed Newton iteration in ln(r - r_+).  These checks use
only facts independent of that code: the Schwarzschild closed form, a finite
difference of r*(r) against Eq. 2's right-hand side, and the round trip.
The orbit frequency of the source (Eq. 1's T slot, a circular equatorial
orbit) is pinned to the circular-geodesic condition of the Kerr metric,
differentiated by sympy.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O


@pytest.mark.parametrize("a", [0.0, 0.3, 0.7, 0.9, 0.99, 0.999])
def test_roundtrip_rstar(a):
    rp = 1.0 + math.sqrt(1.0 - a * a)
    for rs in [-500.0, -200.0, -100.0, -20.0, -1.0, 0.0, 3.0, 50.0, 600.0, 4000.0]:
        try:
            x = O.x_of_rstar(1.0, a, rs)
        except ValueError:
            # only possible for r* so deep that x underflows double precision
            assert a == 0.0 and rs <= -500.0
            continue
        back = O.rstar_of_x(1.0, a, x)
        # conditioning: d r* = (kappa-scale) d ln x, so |dx/x| ~ eps |r*| / (2 M r_+/(r_+ - r_-))
        assert abs(back - rs) <= 4e-14 * max(1.0, abs(rs)), (a, rs, back)
        assert x > 0.0


@pytest.mark.parametrize("a", [0.0, 0.5, 0.9, 0.99])
def test_derivative_matches_eq2(a):
    """d r*/dr = (r^2 + a^2)/Delta (Eq. 2), by a central difference in r."""
    rp = 1.0 + math.sqrt(1.0 - a * a)
    rm = 1.0 - math.sqrt(1.0 - a * a)
    for x in [1e-3, 0.05, 0.7, 3.0, 20.0, 300.0]:
        r = rp + x
        h = 1e-6 * x
        d = (O.rstar_of_x(1.0, a, x + h) - O.rstar_of_x(1.0, a, x - h)) / (2 * h)
        expect = (r * r + a * a) / ((r - rp) * (r - rm))
        assert abs(d - expect) <= 1e-7 * abs(expect)


def test_schwarzschild_closed_form():
    """a = 0: r* = r + 2M ln(r/2M - 1) (textbook tortoise coordinate)."""
    for r in [2.0001, 2.5, 3.0, 6.0, 10.0, 100.0, 1000.0]:
        assert abs(O.rstar_of_x(1.0, 0.0, r - 2.0) - (r + 2.0 * math.log(r / 2.0 - 1.0))) < 1e-12 * max(1, r)


def test_near_horizon_depth():
    """r* = -100M at a = 0 lies at r - 2M ~ 1e-22: x must come out positive
    and consistent with the Schwarzschild asymptotics x ~ 2M exp((r* - 2M)/2M)."""
    x = O.x_of_rstar(1.0, 0.0, -100.0)
    approx = 2.0 * math.exp((-100.0 - 2.0) / 2.0)
    assert 0.0 < x < 1e-20
    assert abs(x / approx - 1.0) < 1e-10


def _kerr_circular_omegas(M, a, r):
    """Both circular equatorial geodesic frequencies Omega = dphi/dt of the
    Kerr metric at Boyer-Lindquist radius r, derived here from the metric
    itself: on a circular orbit u = u^t (1, 0, 0, Omega) the radial geodesic
    equation reduces to
        d_r g_tt + 2 Omega d_r g_tphi + Omega^2 d_r g_phiphi = 0
    at theta = pi/2.  The metric components are those of the Kerr line
    element in Boyer-Lindquist coordinates (rho^2 = r^2 + a^2 cos^2 theta,
    Delta = r^2 - 2 M r + a^2); sympy differentiates them."""
    sp = __import__("sympy")
    rr, th, MM, aa = sp.symbols("r theta M a", positive=True)
    rho2 = rr**2 + aa**2 * sp.cos(th)**2
    g_tt = -(1 - 2 * MM * rr / rho2)
    g_tp = -2 * MM * aa * rr * sp.sin(th)**2 / rho2
    g_pp = (rr**2 + aa**2 + 2 * MM * aa**2 * rr * sp.sin(th)**2 / rho2) * sp.sin(th)**2
    sub = {rr: r, th: sp.pi / 2, MM: M, aa: a}
    c0, c1, c2 = (float(sp.diff(g, rr).subs(sub).evalf(30)) for g in (g_tt, g_tp, g_pp))
    W = sp.symbols("W")
    roots = sp.Poly(c2 * W**2 + 2 * c1 * W + c0, W).nroots(n=30)
    return sorted(float(x) for x in roots)


@pytest.mark.parametrize("a", [0.0, 0.5, 0.9, 0.99, 0.999])
@pytest.mark.parametrize("r0", [4.0, 6.0, 10.0, 15.0, 20.0])
def test_kepler_frequency_from_kerr_geodesics(a, r0):
    """The oracle's orbital frequency (it sets the source phase e^{-i m Omega t})
    is the prograde circular-orbit frequency of the Kerr metric: of the two
    roots of the circular-geodesic condition, the one that co-rotates with
    the hole (Omega > 0 for a >= 0, the larger root).  A dropped a-term, a
    wrong power of r0 or the retrograde branch fails this."""
    pytest.importorskip("sympy")
    lo, hi = _kerr_circular_omegas(1.0, a, r0)
    assert lo < 0.0 < hi
    got = O.kepler_omega(1.0, a, r0)
    assert abs(got - hi) <= 1e-13 * hi, (a, r0, got, hi)
    if a > 0.0:
        # the retrograde orbit is distinguishable at this tolerance
        assert abs(abs(lo) - hi) > 1e-6 * hi


def test_kepler_frequency_mass_scaling():
    """Omega scales as 1/M at fixed r0/M and a/M (the metric has no other
    length scale)."""
    for M in (0.5, 2.0, 7.0):
        assert abs(O.kepler_omega(M, 0.9 * M, 10.0 * M) * M - O.kepler_omega(1.0, 0.9, 10.0)) < 1e-15


def test_kepler_frequency_schwarzschild_newtonian_form():
    """a = 0: Kepler's third law Omega^2 r^3 = M holds exactly for circular
    Schwarzschild geodesics in Boyer-Lindquist time."""
    for r0 in (3.5, 6.0, 10.0, 100.0):
        w = O.kepler_omega(1.0, 0.0, r0)
        assert abs(w * w * r0**3 - 1.0) < 1e-14
