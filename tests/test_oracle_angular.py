"""Pins of the oracle's angular operator (centred differences, Sec. 2.2).

A_th = -(d^2/dth^2 + cot th d/dth) + (m + s cos th)^2/sin^2 th - s on the
cell-centred theta grid with parity ghosts (even |m|: d Phi/d th = 0 at the
poles; odd |m|: Phi = 0).  At a = 0 its continuum eigenvalues are
(l - s)(l + s + 1), l >= max(|m|, |s|) (spin-weighted spherical harmonics,
Teukolsky 1973); the discrete ones must converge to them at second order.
A wrong ghost sign or a dropped cot term breaks the convergence.
"""
import numpy as np
import pytest

from oracle import oracle as O


def _matrix(s, m, N):
    p = O.OracleProblem(s=s, m=m, M=1.0, a=0.0, Nr=8, Ntheta=N, rs_min=-10, rs_max=10, dt=0.1, rs_ext=0)
    A = np.array([O.apply_atheta(p, np.eye(N)[k].astype(np.complex128)) for k in range(N)]).T
    return A.real, p


@pytest.mark.parametrize("s,m", [(-2, 2), (-2, 1), (-2, 3), (-2, 4), (-2, 0), (0, 0), (0, 1), (2, 2), (-1, 1)])
def test_eigenvalues_converge_second_order(s, m):
    lmin = max(abs(m), abs(s))
    exact = np.array([(l - s) * (l + s + 1) for l in range(lmin, lmin + 3)], dtype=float)
    errs = []
    for N in (32, 64, 128):
        A, _ = _matrix(s, m, N)
        ev = np.sort(np.linalg.eigvals(A).real)[:3]
        errs.append(np.abs(ev - exact).max())
    assert errs[-1] < 0.01 * exact.max()
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(order > 1.8), (errs, order)


@pytest.mark.parametrize("s,m", [(-2, 2), (-2, 1), (-2, 3), (0, 1)])
def test_eigenvalues_real_and_positive(s, m):
    A, _ = _matrix(s, m, 48)
    ev = np.linalg.eigvals(A)
    assert np.abs(ev.imag).max() < 1e-8 * np.abs(ev).max()
    assert ev.real.min() > 0


@pytest.mark.parametrize("s,m", [(-2, 2), (-2, 1), (-2, 3), (-2, 4)])
def test_lowest_harmonic_closed_form(s, m):
    """Y = sin(th/2)^{|m+s|} cos(th/2)^{|m-s|} is the lowest eigenfunction,
    eigenvalue (l-s)(l+s+1) with l = max(|m|,|s|); A_th Y - lambda Y = O(dth^2)."""
    lmin = max(abs(m), abs(s))
    lam = (lmin - s) * (lmin + s + 1)
    res = []
    for N in (64, 128, 256):
        _, p = _matrix(s, m, 4)
        p.Ntheta = N
        th = (np.arange(N) + 0.5) * np.pi / N
        Y = np.sin(th / 2) ** abs(m + s) * np.cos(th / 2) ** abs(m - s)
        r = O.apply_atheta(p, Y.astype(np.complex128)).real - lam * Y
        res.append(np.sqrt(np.mean(r[N // 8: -N // 8] ** 2)))
    order = np.log2(np.array(res[:-1]) / np.array(res[1:]))
    assert np.all(order > 1.8), (res, order)


def test_default_weights_project_lowest_harmonic():
    for (s, m) in [(-2, 2), (-2, 1), (-2, 3)]:
        p = O.OracleProblem(s=s, m=m, M=1.0, a=0.0, Nr=8, Ntheta=40, rs_min=-10, rs_max=10, dt=0.1, rs_ext=0)
        th = (np.arange(40) + 0.5) * np.pi / 40
        Y = np.sin(th / 2) ** abs(m + s) * np.cos(th / 2) ** abs(m - s)
        w = O.default_weights(p)
        assert abs(np.dot(w, Y) - 1.0) < 1e-14
        assert np.all(w >= 0)


def test_parity_ghosts():
    """Odd |m| means Phi = 0 at the poles: the antisymmetric ghost makes the
    first-cell stencil see -Phi_0 behind the pole; even |m| sees +Phi_0."""
    N = 16
    th = (np.arange(N) + 0.5) * np.pi / N
    e0 = np.zeros(N, complex); e0[0] = 1.0
    dth = np.pi / N
    for m, sign in [(2, 1.0), (1, -1.0)]:
        p = O.OracleProblem(s=0, m=m, M=1.0, a=0.0, Nr=8, Ntheta=N, rs_min=-10, rs_max=10, dt=0.1, rs_ext=0)
        out = O.apply_atheta(p, e0).real
        cot = np.cos(th[0]) / np.sin(th[0])
        lo_coef = -(1 - 0.5 * cot * dth) / dth ** 2
        expect = 2 / dth ** 2 + m * m / np.sin(th[0]) ** 2 + sign * lo_coef
        assert abs(out[0] - expect) < 1e-9 * abs(expect)
