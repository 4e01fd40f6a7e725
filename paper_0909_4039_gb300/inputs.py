"""Seeded synthetic inputs shared by the tests, the bench and the smoke entry.

This module holds workload descriptions and random-number generation only:
no coefficient, stencil or time-stepping arithmetic of the method lives here.
All workloads are synthetic (the paper uses no dataset): a circular-orbit
Gaussian source in the slot of the paper's particle source T (Sec. 2.1,
Eq. 1), zero or random initial data, and grids of the sizes below.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np


@dataclass(frozen=True)
class Workload:
    """One Teukolsky problem: grid, spin weight, mode, spin, source, steps."""
    name: str
    s: int
    m: int
    a: float
    Nr: int
    Ntheta: int
    rs_min: float
    rs_max: float
    steps: int
    r0: float = 10.0
    amp: complex = 1.0
    sig_r: float = 0.1
    sig_th: float = 0.1
    rs_ext: float = 500.0
    M: float = 1.0
    cfl: float = 0.5          # dt = cfl * dr*

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)

    @property
    def points(self) -> int:
        return self.Nr * self.Ntheta


# s=-2, m=2, a=0.9, 1024 x 32 over r* in [-100, 600], 2000 steps, orbit r0=10.
PLAIN_1024x32 = Workload("plain-fp64-1024x32", s=-2, m=2, a=0.9, Nr=1024, Ntheta=32,
                         rs_min=-100.0, rs_max=600.0, steps=2000, r0=10.0)

# s=-2, m=2, a=0.99, 16384 x 128 over r* in [-200, 1000], 20000 steps, orbit r0=6.
LARGE_16384x128 = Workload("single-16384x128", s=-2, m=2, a=0.99, Nr=16384, Ntheta=128,
                           rs_min=-200.0, rs_max=1000.0, steps=20000, r0=6.0)

# s=-2, m=2, a=0.7, 4096 x 64 over r* in [-100, 600], 8000 steps (adjoint case).
ADJOINT_4096x64 = Workload("adjoint-4096x64", s=-2, m=2, a=0.7, Nr=4096, Ntheta=64,
                           rs_min=-100.0, rs_max=600.0, steps=8000, r0=10.0)

# s=-2, m=2, a=0.999, 65536 x 256 over r* in [-500, 4000], 100000 steps.
LONG_65536x256 = Workload("long-65536x256", s=-2, m=2, a=0.999, Nr=65536, Ntheta=256,
                          rs_min=-500.0, rs_max=4000.0, steps=100000, r0=4.0)

WORKLOADS = {w.name: w for w in (PLAIN_1024x32, LARGE_16384x128, ADJOINT_4096x64, LONG_65536x256)}


def batched_instances(n: int = 64, seed: int = 0, steps: int = 10000) -> list[Workload]:
    """Uneven batch: a ~ U[0, 0.99], m ~ U{1..4}, r0 ~ U[6, 15],
    Nr ~ U{2048, 4096, 8192, 16384}, Ntheta ~ U{32, 64, 128}, r* in [-100, 600]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(n):
        a = float(rng.uniform(0.0, 0.99))
        m = int(rng.integers(1, 5))
        r0 = float(rng.uniform(6.0, 15.0))
        Nr = int(rng.choice([2048, 4096, 8192, 16384]))
        Nth = int(rng.choice([32, 64, 128]))
        out.append(Workload(f"batch{k}", s=-2, m=m, a=a, Nr=Nr, Ntheta=Nth, rs_min=-100.0,
                            rs_max=600.0, steps=steps, r0=r0))
    return out


def long_run_batch(n: int = 8) -> list[Workload]:
    """Eight long-run instances with r0 = linspace(4, 20, 8)."""
    return [LONG_65536x256.with_(name=f"long{k}", r0=float(r0))
            for k, r0 in enumerate(np.linspace(4.0, 20.0, n))]


def random_state(Nr: int, Ntheta: int, seed: int, zero_boundary: bool = True,
                 scale: float = 1.0) -> np.ndarray:
    """Complex128 state of shape (2, Nr, Ntheta), i.i.d. N(0,1) real and
    imaginary parts (numpy PCG64), with the radial boundary rows zeroed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = (rng.standard_normal((2, Nr, Ntheta)) + 1j * rng.standard_normal((2, Nr, Ntheta))) * scale
    if zero_boundary:
        u[:, 0, :] = 0.0
        u[:, -1, :] = 0.0
    return u


def gaussian_pulse(Nr: int, Ntheta: int, rs_min: float, rs_max: float, center: float,
                   width: float, theta_profile: np.ndarray | None = None) -> np.ndarray:
    """Smooth initial data: Phi = exp(-(r*-center)^2/(2 width^2)) * profile(theta)
    on the node/cell-centre grid, Pi = 0."""
    rs = rs_min + np.arange(Nr) * (rs_max - rs_min) / (Nr - 1)
    prof = np.ones(Ntheta) if theta_profile is None else np.asarray(theta_profile)
    u = np.zeros((2, Nr, Ntheta), dtype=np.complex128)
    u[0] = np.exp(-(rs[:, None] - center) ** 2 / (2.0 * width * width)) * prof[None, :]
    u[:, 0, :] = 0.0
    u[:, -1, :] = 0.0
    return u


def adjoint_target(nsamples: int, dt: float, seed: int = 1, omega_max: float = 0.5) -> np.ndarray:
    """Synthetic target waveform for the adjoint workload: complex Gaussian
    noise (numpy PCG64, `seed`) of `nsamples` samples spaced dt, low-passed
    to |omega| < omega_max (1/M) by zeroing the higher FFT bins."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.standard_normal(nsamples) + 1j * rng.standard_normal(nsamples)
    spec = np.fft.fft(z)
    omega = 2.0 * np.pi * np.fft.fftfreq(nsamples, d=dt)
    spec[np.abs(omega) >= omega_max] = 0.0
    return np.fft.ifft(spec)
