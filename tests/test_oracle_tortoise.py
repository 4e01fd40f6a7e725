"""Pins of the oracle's tortoise map (Eq. 2) and orbit frequency.

The oracle integrates Eq. 2 (dr*/dr = (r^2+a^2)/Delta) in closed form and
inverts it by a bracketed Newton iteration in ln(r - r_+).  These checks use
only facts independent of that code: the Schwarzschild closed form, a finite
difference of r*(r) against Eq. 2's right-hand side, and the round trip.
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


def test_kepler_frequency():
    """Prograde circular equatorial orbit, Omega = M^1/2 / (r0^3/2 + a M^1/2)."""
    assert abs(O.kepler_omega(1.0, 0.9, 10.0) - 1.0 / (10.0 ** 1.5 + 0.9)) < 1e-15
    assert abs(O.kepler_omega(1.0, 0.0, 6.0) - 6.0 ** -1.5) < 1e-15
    # value quoted for the 1024x32 workload (a=0.9, r0=10): 0.0307477/M
    assert abs(O.kepler_omega(1.0, 0.9, 10.0) - 0.0307477) < 1e-7
