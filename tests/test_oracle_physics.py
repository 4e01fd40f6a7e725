"""Physics pins of the oracle's split scheme.

C-T6  second-order self-convergence on three resolutions (r*, theta and t
      refined together), with and without a resolved source;
C-T7  the l=2 Schwarzschild quasinormal ringing (Leaver 1985) to 1 %;
C-7   the literal reading of Eqs. 12-14 (all of S explicit) is unstable at
      dt = dr*/2, while the split scheme stays bounded at the grids of the
      named workloads (its slow growth is the reflecting-wall mode of the
      radial boundary rows, bounded by 0.03/M here).
"""
import json
import os

import numpy as np
import pytest
from scipy.optimize import least_squares

from oracle import oracle as O
from paper_0909_4039_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _restrict(u):
    """coarse nodes = every other fine node; coarse theta cell = mean of its two fine cells"""
    v = u[:, ::2, :]
    return 0.5 * (v[:, :, 0::2] + v[:, :, 1::2])


def _run_level(Nr, Nth, T, amp, a=0.5, s=-2, m=2):
    lo, hi = -20.0, 40.0
    drs = (hi - lo) / (Nr - 1)
    p = O.OracleProblem(s=s, m=m, M=1.0, a=a, Nr=Nr, Ntheta=Nth, rs_min=lo, rs_max=hi, dt=0.5 * drs,
                        rs_ext=0.0, scheme=O.SCHEME_SPLIT, amp=amp, r0=8.0, sig_r=2.0, sig_th=0.5)
    th = (np.arange(Nth) + 0.5) * np.pi / Nth
    prof = np.cos(th / 2) ** 4 + 0.3 * np.sin(th) ** 2
    u0 = inputs.gaussian_pulse(Nr, Nth, lo, hi, 10.0, 3.0, prof) * (0.0 if amp else 1.0)
    nsteps = int(round(T / p.dt))
    u, _ = O.run(p, u0, nsteps)
    return u


@pytest.mark.parametrize("amp", [0.0, 1.0])
def test_second_order_self_convergence(amp):
    T = 8.0
    uc = _run_level(121, 8, T, amp)
    um = _run_level(241, 16, T, amp)
    uf = _run_level(481, 32, T, amp)
    e1 = np.linalg.norm(uc - _restrict(um))
    e2 = np.linalg.norm(_restrict(um) - _restrict(_restrict(uf)))
    order = np.log2(e1 / e2)
    assert 1.8 <= order <= 2.2, (e1, e2, order)


def _fit_damped(t, y):
    best = None
    for ph in np.linspace(0, 2 * np.pi, 8, endpoint=False):
        for w in (0.3, 0.37, 0.45):
            f = lambda x: x[0] * np.exp(-x[2] * t) * np.cos(x[1] * t + x[3]) - y
            r = least_squares(f, [np.abs(y).max(), w, 0.09, ph],
                              bounds=([-np.inf, 0.05, 0.0, -10], [np.inf, 2, 1, 20]))
            if best is None or r.cost < best.cost:
                best = r
    return best.x[1], best.x[2]


def test_schwarzschild_l2_ringdown():
    gold = json.load(open(os.path.join(GOLD, "qnm_schwarzschild_l2.json")))
    lo, hi, dr, Nth = -100.0, 300.0, 0.2, 16
    Nr = int(round((hi - lo) / dr)) + 1
    drs = (hi - lo) / (Nr - 1)
    p = O.OracleProblem(s=-2, m=2, M=1.0, a=0.0, Nr=Nr, Ntheta=Nth, rs_min=lo, rs_max=hi, dt=0.5 * drs,
                        rs_ext=100.0, scheme=O.SCHEME_SPLIT)
    th = (np.arange(Nth) + 0.5) * np.pi / Nth
    u0 = inputs.gaussian_pulse(Nr, Nth, lo, hi, 50.0, 5.0, np.cos(th / 2) ** 4)   # l=2 harmonic
    u, h = O.run(p, u0, int(260.0 / p.dt))
    t = np.arange(len(h)) * p.dt
    y = h.real
    assert np.abs(h.imag).max() == 0.0          # a = 0: real stays real
    tp = t[np.argmax(np.abs(y) * (t > 20))]
    sel = (t > tp + 30) & (t < tp + 90)
    wr, wi = _fit_damped(t[sel] - tp - 30, y[sel])
    tol = gold["tolerance_rel"]
    assert abs(wr - gold["omega_re"]) <= tol * abs(gold["omega_re"]), wr
    assert abs(wi + gold["omega_im"]) <= tol * abs(gold["omega_im"]), wi


def _growth_rate(Nr, Nth, a, m, lo, hi, T, scheme=O.SCHEME_SPLIT, seed=1):
    drs = (hi - lo) / (Nr - 1)
    p = O.OracleProblem(s=-2, m=m, M=1.0, a=a, Nr=Nr, Ntheta=Nth, rs_min=lo, rs_max=hi, dt=0.5 * drs,
                        rs_ext=500.0, scheme=scheme)
    u = inputs.random_state(Nr, Nth, seed=seed)
    n = int(T / p.dt)
    k1 = n // 2
    u, _ = O.run(p, u, k1)
    a1 = np.linalg.norm(u)
    u, _ = O.run(p, u, n - k1, n0=k1)
    return np.log(np.linalg.norm(u) / a1) / ((n - k1) * p.dt)


def test_literal_scheme_unstable_at_half_courant():
    """All of S explicit inside the LW stages acts as a midpoint rule on the
    stiff angular terms: it grows by orders of magnitude per step here."""
    w = inputs.PLAIN_1024x32
    drs = (w.rs_max - w.rs_min) / (w.Nr - 1)
    p = O.OracleProblem(s=w.s, m=w.m, M=1.0, a=w.a, Nr=w.Nr, Ntheta=w.Ntheta, rs_min=w.rs_min,
                        rs_max=w.rs_max, dt=0.5 * drs, rs_ext=w.rs_ext, scheme=O.SCHEME_LITERAL)
    u = inputs.random_state(w.Nr, w.Ntheta, seed=7)
    n0 = np.linalg.norm(u)
    u, _ = O.run(p, u, 12)
    assert np.linalg.norm(u) / n0 > 1e6


@pytest.mark.parametrize("Nr,Nth,a,m,T", [(1024, 32, 0.9, 2, 500.0), (1024, 32, 0.9, 4, 300.0),
                                           (2048, 32, 0.99, 4, 400.0)])
def test_split_scheme_bounded(Nr, Nth, a, m, T):
    rate = _growth_rate(Nr, Nth, a, m, -100.0, 600.0, T)
    assert rate < 0.03, rate


def test_plain_workload_bounded_with_source():
    """The 1024x32 workload (a = 0.9, orbit r0 = 10) from zero data for its
    2000 steps: the field stays bounded and the waveform is nonzero."""
    w = inputs.PLAIN_1024x32
    drs = (w.rs_max - w.rs_min) / (w.Nr - 1)
    p = O.OracleProblem(s=w.s, m=w.m, M=1.0, a=w.a, Nr=w.Nr, Ntheta=w.Ntheta, rs_min=w.rs_min,
                        rs_max=w.rs_max, dt=0.5 * drs, rs_ext=w.rs_ext, scheme=O.SCHEME_SPLIT,
                        amp=w.amp, r0=w.r0, sig_r=w.sig_r, sig_th=w.sig_th)
    u, h = O.run(p, None, w.steps)
    assert np.isfinite(u).all()
    assert np.abs(u).max() < 10.0
    assert np.abs(h[-200:]).max() > 0.0
