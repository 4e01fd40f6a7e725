"""Pins of the oracle's time step against an independent formulation.

C-T1: a second, naive implementation in numpy forms, at every point, the
real 4x4 matrices of the paper -- D (Eq. 11), M - D, A and the theta
stencil L (Eq. 9) -- acting on u = {Phi_R, Phi_I, Pi_R, Pi_I}, builds
S = T - (M - D) d_{r*} u - L u - A u (Eq. 12) and applies the two
Lax-Wendroff stages (Eqs. 13-14) literally.  The implicit half-step of the
split scheme is re-derived as a dense linear solve of the SDIRK stage
equations on the same real 4x4 blocks.  The oracle's complex-arithmetic
implementation must agree with both to rounding.

Also: linearity (zero stays zero, superposition, linear in the source
amplitude) and the a = 0 symmetries.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0909_4039_gb300 import inputs

GAM = 1.0 - 1.0 / np.sqrt(2.0)


def C(z):
    """real 2x2 block of multiplication by complex z"""
    return np.array([[z.real, -z.imag], [z.imag, z.real]])


def _prob(Nr=10, N=8, a=0.7, s=-2, m=2, scheme=O.SCHEME_LITERAL, amp=0.0, lo=-6.0, hi=12.0, cfl=0.5):
    drs = (hi - lo) / (Nr - 1)
    return O.OracleProblem(s=s, m=m, M=1.0, a=a, Nr=Nr, Ntheta=N, rs_min=lo, rs_max=hi, dt=cfl * drs,
                           rs_ext=0.0, scheme=scheme, amp=amp, r0=3.0, sig_r=1.5, sig_th=0.4)


def _blocks(p, rs, t):
    """Per theta cell: dict of 4x4 real D, MmD, A and scalars q, F at radius rs."""
    x = O.x_of_rstar(p.M, p.a, rs)
    N = p.Ntheta
    out = []
    src = p.source()
    rp = 1.0 + np.sqrt(1.0 - p.a ** 2)
    rs0 = O.rstar_of_x(p.M, p.a, src.r0 - rp)
    for j in range(N):
        th = (j + 0.5) * np.pi / N
        c = O.point_coef(p, x, th)
        D = np.diag([c["b"], c["b"], -c["b"], -c["b"]])
        MmD = np.zeros((4, 4))
        MmD[2:, :2] = -C(c["K_re"] + 1j * c["K_im"])
        A = np.zeros((4, 4))
        A[:2, 2:] = -np.eye(2)
        A[2:, 2:] = C(c["ct_re"] + 1j * c["ct_im"])
        A[2:, :2] = C(c["c0rad_re"] + 1j * c["c0rad_im"] + c["c0ang"])
        A_rad = A.copy()
        A_rad[2:, :2] = C(c["c0rad_re"] + 1j * c["c0rad_im"])
        G = np.exp(-(rs - rs0) ** 2 / (2 * src.sig_r ** 2) - (th - np.pi / 2) ** 2 / (2 * src.sig_th ** 2))
        F = c["Fpref"] * complex(src.amp_re, src.amp_im) * G * np.exp(-1j * p.m * src.Omega * t)
        out.append(dict(D=D, MmD=MmD, A=A, q=c["q"], F=F, c0ang=c["c0ang"]))
    return out


def _Ltheta(p, row):
    """L_th on a real theta row with parity ghosts (centred differences)."""
    N = p.Ntheta
    par = 1.0 if abs(p.m) % 2 == 0 else -1.0
    g = np.concatenate([[par * row[0]], row, [par * row[-1]]])
    th = (np.arange(N) + 0.5) * np.pi / N
    dth = np.pi / N
    return (g[2:] - 2 * g[1:-1] + g[:-2]) / dth ** 2 + np.cos(th) / np.sin(th) * (g[2:] - g[:-2]) / (2 * dth)


def _S(p, blk, ubar, du, t, full):
    """S = T - (M-D) du - L ubar - A ubar on a theta row; ubar, du: (N, 4)."""
    N = p.Ntheta
    S = np.zeros((N, 4))
    Lphi = np.stack([_Ltheta(p, ubar[:, 0]), _Ltheta(p, ubar[:, 1])], axis=1) if full else None
    for j in range(N):
        b = blk[j]
        Tv = np.array([0.0, 0.0, b["F"].real, b["F"].imag])
        S[j] = Tv - b["MmD"] @ du[j]
        if full:
            Lu = np.zeros(4)
            Lu[2:] = -b["q"] * Lphi[j]
            S[j] += -Lu - b["A"] @ ubar[j]
    return S


def _to4(u):
    return np.stack([u[0].real, u[0].imag, u[1].real, u[1].imag], axis=-1)  # (Nr, N, 4)


def _from4(v):
    return np.stack([v[..., 0] + 1j * v[..., 1], v[..., 2] + 1j * v[..., 3]])


def lw_numpy(p, u, n, full):
    Nr, N = p.Nr, p.Ntheta
    drs = (p.rs_max - p.rs_min) / (Nr - 1)
    dt = p.dt
    v = _to4(u)
    mid = np.zeros((Nr - 1, N, 4))
    for i in range(Nr - 1):                                    # Eq. 13
        rs = p.rs_min + (i + 0.5) * drs
        blk = _blocks(p, rs, n * dt)
        ubar = 0.5 * (v[i + 1] + v[i])
        du = (v[i + 1] - v[i]) / drs
        S = _S(p, blk, ubar, du, n * dt, full)
        for j in range(N):
            mid[i, j] = ubar[j] - 0.5 * dt * (blk[j]["D"] @ du[j] - S[j])
    new = np.zeros_like(v)
    for i in range(1, Nr - 1):                                 # Eq. 14
        rs = p.rs_min + i * drs
        blk = _blocks(p, rs, n * dt + 0.5 * dt)
        ut = 0.5 * (mid[i] + mid[i - 1])
        du = (mid[i] - mid[i - 1]) / drs
        S = _S(p, blk, ut, du, n * dt + 0.5 * dt, full)
        for j in range(N):
            new[i, j] = v[i, j] - dt * (blk[j]["D"] @ du[j] - S[j])
    return _from4(new)


def implicit_numpy(p, u, h):
    """SDIRK2 (gamma = 1 - 1/sqrt 2) step of length h on u_t = -(L + A) u,
    per r* row, by dense solves of the stage equations."""
    Nr, N = p.Nr, p.Ntheta
    drs = (p.rs_max - p.rs_min) / (Nr - 1)
    v = _to4(u)
    out = np.zeros_like(v)
    I = np.eye(4 * N)
    for i in range(1, Nr - 1):
        blk = _blocks(p, p.rs_min + i * drs, 0.0)
        J = np.zeros((4 * N, 4 * N))
        for j in range(N):
            J[4 * j:4 * j + 4, 4 * j:4 * j + 4] -= blk[j]["A"]
        # -L u: Pi rows get + q L_th Phi (real operator, per component)
        for k in range(N):
            e = np.zeros(N); e[k] = 1.0
            col = _Ltheta(p, e)
            for j in range(N):
                for comp in (0, 1):
                    J[4 * j + 2 + comp, 4 * k + comp] += blk[j]["q"] * col[j]
        x = v[i].reshape(-1)
        U1 = np.linalg.solve(I - GAM * h * J, x)
        U2 = np.linalg.solve(I - GAM * h * J, x + (1 - GAM) * h * J @ U1)
        out[i] = U2.reshape(N, 4)
    return _from4(out)


@pytest.mark.parametrize("a,m,N", [(0.7, 2, 8), (0.0, 1, 6), (0.95, 3, 5), (0.3, 0, 7)])
def test_literal_step_bruteforce(a, m, N):
    p = _prob(N=N, a=a, m=m, amp=0.8 - 0.3j)
    u = inputs.random_state(p.Nr, N, seed=11)
    ref = lw_numpy(p, u, 3, full=True)
    got = O.step(p, u, 3)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("a,m,N", [(0.7, 2, 8), (0.0, 1, 6), (0.95, 4, 5)])
def test_split_parts_bruteforce(a, m, N):
    p = _prob(N=N, a=a, m=m, amp=0.5 + 0.5j, scheme=O.SCHEME_SPLIT)
    u = inputs.random_state(p.Nr, N, seed=5)
    # implicit steps of length dt/2 and dt
    for h in (0.5 * p.dt, p.dt):
        ref_h = implicit_numpy(p, u, h)
        got_h = O.imp(p, u, h)
        assert np.abs(got_h - ref_h).max() <= 1e-12 * np.abs(ref_h).max()
    # derivative-only LW
    ref_lw = lw_numpy(p, u, 7, full=False)
    got_lw = O.lw(p, u, 7, full=False)
    assert np.abs(got_lw - ref_lw).max() <= 1e-12 * np.abs(ref_lw).max()
    # split steps: first s = LW C_{dt/2} u, then s' = LW C_dt s
    s1 = lw_numpy(p, implicit_numpy(p, u, 0.5 * p.dt), 7, full=False)
    got1 = O.step(p, u, 7, first=True)
    assert np.abs(got1 - s1).max() <= 1e-12 * np.abs(s1).max()
    s2 = lw_numpy(p, implicit_numpy(p, s1, p.dt), 8, full=False)
    got2 = O.step(p, s1, 8, first=False)
    assert np.abs(got2 - s2).max() <= 1e-12 * np.abs(s2).max()
    # a two-step run outputs u_2 = C_{dt/2} s_2 and samples u_1 = C_{dt/2} s_1
    w = O.default_weights(p)
    ie = O.extract_index(p)
    u2, h = O.run(p, u, 2, n0=7)
    ref_u2 = implicit_numpy(p, s2, 0.5 * p.dt)
    assert np.abs(u2 - ref_u2).max() <= 1e-12 * np.abs(ref_u2).max()
    ref_u1 = implicit_numpy(p, s1, 0.5 * p.dt)
    assert abs(h[1] - np.dot(w, ref_u1[0, ie])) <= 1e-12 * max(abs(h[1]), 1e-300) + 1e-300


def test_sdirk_half_step_is_second_order():
    """Local error of the implicit half-step vs the exact flow exp(h J) is O(h^3)."""
    from scipy.linalg import expm
    errs = []
    for cfl in (0.2, 0.1, 0.05):
        p = _prob(Nr=4, N=6, a=0.8, m=2, scheme=O.SCHEME_SPLIT, cfl=cfl)
        u = inputs.gaussian_pulse(4, 6, p.rs_min, p.rs_max, 3.0, 100.0,
                                  np.cos(((np.arange(6) + 0.5) * np.pi / 6) / 2) ** 4)
        u[1] = 0.3 * u[0]
        got = O.imp(p, u, 0.5 * p.dt)
        # exact flow for row 1 from the same dense J
        Nr, N = p.Nr, p.Ntheta
        drs = (p.rs_max - p.rs_min) / (Nr - 1)
        v = _to4(u)
        blk = _blocks(p, p.rs_min + drs, 0.0)
        J = np.zeros((4 * N, 4 * N))
        for j in range(N):
            J[4 * j:4 * j + 4, 4 * j:4 * j + 4] -= blk[j]["A"]
        for k in range(N):
            e = np.zeros(N); e[k] = 1.0
            col = _Ltheta(p, e)
            for j in range(N):
                for comp in (0, 1):
                    J[4 * j + 2 + comp, 4 * k + comp] += blk[j]["q"] * col[j]
        ex = (expm(0.5 * p.dt * J) @ v[1].reshape(-1)).reshape(N, 4)
        errs.append(np.abs(_to4(got)[1] - ex).max())
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(order > 2.7), (errs, order)


@pytest.mark.parametrize("scheme", [O.SCHEME_LITERAL, O.SCHEME_SPLIT])
def test_zero_stays_zero(scheme):
    p = _prob(Nr=40, N=8, scheme=scheme)
    u, h = O.run(p, np.zeros((2, 40, 8), complex), 20)
    assert np.all(u == 0) and np.all(h == 0)


@pytest.mark.parametrize("scheme", [O.SCHEME_LITERAL, O.SCHEME_SPLIT])
def test_superposition(scheme):
    p = _prob(Nr=40, N=8, scheme=scheme, amp=0.0)
    u = inputs.random_state(40, 8, seed=1)
    v = inputs.random_state(40, 8, seed=2)
    al, be = 0.7 - 0.2j, -1.3 + 0.4j
    lhs = O.step(p, al * u + be * v, 4)
    rhs = al * O.step(p, u, 4) + be * O.step(p, v, 4)
    assert np.abs(lhs - rhs).max() <= 1e-13 * np.abs(lhs).max()


def test_linear_in_source_amplitude():
    p1 = _prob(Nr=60, N=8, scheme=O.SCHEME_SPLIT, amp=1.0)
    p2 = _prob(Nr=60, N=8, scheme=O.SCHEME_SPLIT, amp=0.25 - 2.0j)
    p3 = _prob(Nr=60, N=8, scheme=O.SCHEME_SPLIT, amp=1.25 - 2.0j)
    u1, h1 = O.run(p1, None, 30)
    u2, h2 = O.run(p2, None, 30)
    u3, h3 = O.run(p3, None, 30)
    assert np.abs(u1).max() > 0
    assert np.abs(u3 - (u1 + u2)).max() <= 1e-13 * np.abs(u3).max()
    assert np.abs(h3 - (h1 + h2)).max() <= 1e-13 * max(np.abs(h3).max(), 1e-300)


def test_schwarzschild_real_data_stays_real():
    """a = 0 gives a real operator (C-T8): real data without a source stays real."""
    p = _prob(Nr=50, N=8, a=0.0, scheme=O.SCHEME_SPLIT)
    u = inputs.random_state(50, 8, seed=3).real.astype(np.complex128)
    out, _ = O.run(p, u, 25)
    assert np.abs(out.imag).max() == 0.0


def test_scalar_equatorial_reflection_symmetry():
    """s = 0, m = 0, a = 0.8: the operator commutes with th -> pi - th, so
    reflection-symmetric data stays symmetric."""
    p = _prob(Nr=50, N=8, a=0.8, s=0, m=0, scheme=O.SCHEME_SPLIT)
    u = inputs.random_state(50, 8, seed=4)
    u = 0.5 * (u + u[:, :, ::-1])
    out, _ = O.run(p, u, 25)
    assert np.abs(out - out[:, :, ::-1]).max() <= 1e-13 * np.abs(out).max()


def test_source_placement():
    """From zero data, the derivative-only LW step gives exactly
        Pi*_{i+1/2}  = (dt/2) F(r*_{i+1/2}, t^n)                     (Eq. 13)
        Pi^{n+1}_i   = dt [ b_i (Pi*_{i+1/2} - Pi*_{i-1/2})/dr* + F(r*_i, t^n + dt/2) ]   (Eq. 14)
    and Phi^{n+1} = 0: the source enters the Pi rows only, at the stated
    positions and time levels, with the prefactor of Eq. 1's right side."""
    p = _prob(Nr=41, N=9, a=0.6, amp=2.0 + 1.0j, lo=-10.0, hi=10.0, scheme=O.SCHEME_SPLIT)
    n = 5
    out = O.lw(p, np.zeros((2, 41, 9), complex), n, full=False)
    assert np.abs(out[0]).max() == 0.0
    drs = (p.rs_max - p.rs_min) / (p.Nr - 1)
    dt = p.dt
    mid = np.array([[b["F"] for b in _blocks(p, p.rs_min + (i + 0.5) * drs, n * dt)] for i in range(p.Nr - 1)])
    pstar = 0.5 * dt * mid
    ref = np.zeros((41, 9), complex)
    for i in range(1, 40):
        blk = _blocks(p, p.rs_min + i * drs, n * dt + 0.5 * dt)
        b = np.array([bb["D"][0, 0] for bb in blk])
        F = np.array([bb["F"] for bb in blk])
        ref[i] = dt * (b * (pstar[i] - pstar[i - 1]) / drs + F)
    assert np.abs(ref).max() > 1e-3
    assert np.abs(out[1] - ref).max() <= 1e-13 * np.abs(ref).max()
