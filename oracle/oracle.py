"""ctypes binding of the FP64 CPU oracle (teuk_oracle.c).

TEST INFRASTRUCTURE.  The oracle is a plain, slow, independent restatement of
the Teukolsky time step of Khanna & McKennon (arXiv:0909.4039, Sec. 2,
Eqs. 1-14).  Only tests/, __graft_entry__.smoke() and bench.py's CPU legs
(cpu_baseline and the reference arm) may import this module.  The CUDA
library under paper_0909_4039_gb300/ never imports it and shares no code
with it.

Arrays: the state is a complex128 array of shape (2, Nr, Ntheta) (plane 0 is
Phi, plane 1 is Pi, Eqs. 4-5), C-contiguous.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
SRC = os.path.join(HERE, "teuk_oracle.c")

SCHEME_LITERAL = 0
SCHEME_SPLIT = 1

_lock = threading.Lock()
_lib = None


def _build_lib(path: str, extra: list[str], force: bool) -> str:
    os.makedirs(BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= max(os.path.getmtime(SRC),
                                              os.path.getmtime(os.path.join(HERE, "teuk_oracle.h")))):
        return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", *extra, "-fopenmp", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile teuk_oracle.c into oracle/_build/liboracle.so with gcc
    (ISO C, no floating-point contraction)."""
    return _build_lib(LIB_PATH, ["-ffp-contract=off"], force)


FMA_LIB_PATH = os.path.join(BUILD_DIR, "liboracle_fma.so")


def build_fma_variant(force: bool = False) -> str:
    """The same source compiled with fused multiply-adds wherever the
    compiler may contract a*b+c.  It computes the same method with a
    different rounding order; its disagreement with build() measures how
    strongly a run amplifies rounding (the floor any second FP64
    implementation, such as the GPU path, can be held to)."""
    extra = ["-ffp-contract=fast"]
    if platform.machine() in ("x86_64", "AMD64"):
        extra.append("-mfma")
    return _build_lib(FMA_LIB_PATH, extra, force)


def run_fma_variant(p: "OracleProblem", u0, nsteps: int, n0: int = 0):
    """run() with the FMA-contracted build of the oracle."""
    global _lib
    saved = lib()
    path = build_fma_variant()
    with _lock:
        _lib = None
    try:
        L = ctypes.CDLL(path)
        _bind(L)
        with _lock:
            _lib = L
        return run(p, u0, nsteps, n0)
    finally:
        with _lock:
            _lib = saved


class Grid(ctypes.Structure):
    _fields_ = [
        ("s", ctypes.c_int), ("m", ctypes.c_int),
        ("M", ctypes.c_double), ("a", ctypes.c_double),
        ("Nr", ctypes.c_long), ("Nth", ctypes.c_long),
        ("rs_min", ctypes.c_double), ("rs_max", ctypes.c_double),
        ("dt", ctypes.c_double), ("rs_ext", ctypes.c_double),
        ("scheme", ctypes.c_int), ("nthreads", ctypes.c_int),
    ]


class Source(ctypes.Structure):
    _fields_ = [
        ("amp_re", ctypes.c_double), ("amp_im", ctypes.c_double),
        ("r0", ctypes.c_double), ("sig_r", ctypes.c_double),
        ("sig_th", ctypes.c_double), ("Omega", ctypes.c_double),
    ]


class Coef(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "r", "x", "delta", "R", "sigma2", "b", "b_rs", "q",
        "ct_re", "ct_im", "cs_re", "cs_im", "c0rad_re", "c0rad_im", "c0ang",
        "K_re", "K_im", "Fpref")]


def _bind(L):
    dp = ctypes.POINTER(ctypes.c_double)
    gp = ctypes.POINTER(Grid)
    sp = ctypes.POINTER(Source)
    L.or_rstar_of_x.restype = ctypes.c_double
    L.or_rstar_of_x.argtypes = [ctypes.c_double] * 3
    L.or_x_of_rstar.restype = ctypes.c_int
    L.or_x_of_rstar.argtypes = [ctypes.c_double] * 3 + [dp]
    L.or_point_coef.restype = None
    L.or_point_coef.argtypes = [gp, ctypes.c_double, ctypes.c_double, ctypes.POINTER(Coef)]
    L.or_kepler_omega.restype = ctypes.c_double
    L.or_kepler_omega.argtypes = [ctypes.c_double] * 3
    L.or_apply_atheta.restype = None
    L.or_apply_atheta.argtypes = [gp, dp, dp]
    L.or_default_weights.restype = None
    L.or_default_weights.argtypes = [gp, dp]
    L.or_extract_index.restype = ctypes.c_long
    L.or_extract_index.argtypes = [gp]
    L.or_step.restype = ctypes.c_int
    L.or_step.argtypes = [gp, sp, ctypes.c_long, ctypes.c_int, dp, dp]
    L.or_run.restype = ctypes.c_int
    L.or_run.argtypes = [gp, sp, ctypes.c_long, ctypes.c_long, dp, dp, dp]
    L.or_imp.restype = ctypes.c_int
    L.or_imp.argtypes = [gp, ctypes.c_double, dp, dp]
    L.or_lw.restype = ctypes.c_int
    L.or_lw.argtypes = [gp, sp, ctypes.c_long, ctypes.c_int, dp, dp]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class OracleProblem:
    """One Teukolsky problem for the oracle: grid, scheme and source."""
    s: int
    m: int
    M: float
    a: float
    Nr: int
    Ntheta: int
    rs_min: float
    rs_max: float
    dt: float
    rs_ext: float
    scheme: int = SCHEME_SPLIT
    amp: complex = 0.0
    r0: float = 10.0
    sig_r: float = 0.1
    sig_th: float = 0.1
    Omega: float | None = None
    nthreads: int = 0

    def grid(self) -> Grid:
        return Grid(self.s, self.m, self.M, self.a, self.Nr, self.Ntheta, self.rs_min,
                    self.rs_max, self.dt, self.rs_ext, self.scheme, self.nthreads)

    def source(self) -> Source:
        Om = self.Omega
        if Om is None or not np.isfinite(Om):
            Om = kepler_omega(self.M, self.a, self.r0)
        amp = complex(self.amp)
        return Source(amp.real, amp.imag, self.r0, self.sig_r, self.sig_th, Om)


def rstar_of_x(M, a, x):
    return lib().or_rstar_of_x(M, a, x)


def x_of_rstar(M, a, rs):
    out = ctypes.c_double()
    rc = lib().or_x_of_rstar(M, a, rs, ctypes.byref(out))
    if rc != 0:
        raise ValueError(f"or_x_of_rstar failed rc={rc}")
    return out.value


def kepler_omega(M, a, r0):
    return lib().or_kepler_omega(M, a, r0)


def point_coef(p: OracleProblem, x: float, theta: float) -> dict:
    c = Coef()
    g = p.grid()
    lib().or_point_coef(ctypes.byref(g), x, theta, ctypes.byref(c))
    return {n: getattr(c, n) for n, _ in Coef._fields_}


def apply_atheta(p: OracleProblem, row: np.ndarray) -> np.ndarray:
    row = np.ascontiguousarray(row, dtype=np.complex128)
    out = np.empty_like(row)
    g = p.grid()
    lib().or_apply_atheta(ctypes.byref(g), _dp(row), _dp(out))
    return out


def default_weights(p: OracleProblem) -> np.ndarray:
    w = np.empty(p.Ntheta, dtype=np.float64)
    g = p.grid()
    lib().or_default_weights(ctypes.byref(g), _dp(w))
    return w


def extract_index(p: OracleProblem) -> int:
    g = p.grid()
    return int(lib().or_extract_index(ctypes.byref(g)))


def _state(u: np.ndarray, p: OracleProblem) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.complex128)
    if u.shape != (2, p.Nr, p.Ntheta):
        raise ValueError(f"state shape {u.shape} != {(2, p.Nr, p.Ntheta)}")
    return u


def step(p: OracleProblem, u: np.ndarray, n: int = 0, first: bool = True) -> np.ndarray:
    """Literal scheme: u^n -> u^{n+1}.  Split scheme: internal state
    s_n -> s_{n+1} (first=True: from a physical state, LW_n C_{dt/2} u)."""
    u = _state(u, p)
    out = np.empty_like(u)
    g, s = p.grid(), p.source()
    rc = lib().or_step(ctypes.byref(g), ctypes.byref(s), n, int(first), _dp(u), _dp(out))
    if rc != 0:
        raise RuntimeError(f"or_step rc={rc}")
    return out


def imp(p: OracleProblem, u: np.ndarray, h: float) -> np.ndarray:
    """Implicit SDIRK2 step of length h of the algebraic terms, every r* row."""
    u = _state(u, p)
    out = np.empty_like(u)
    g = p.grid()
    rc = lib().or_imp(ctypes.byref(g), float(h), _dp(u), _dp(out))
    if rc != 0:
        raise RuntimeError(f"or_imp rc={rc}")
    return out


def lw(p: OracleProblem, u: np.ndarray, n: int = 0, full: bool = True) -> np.ndarray:
    u = _state(u, p)
    out = np.empty_like(u)
    g, s = p.grid(), p.source()
    rc = lib().or_lw(ctypes.byref(g), ctypes.byref(s), n, int(full), _dp(u), _dp(out))
    if rc != 0:
        raise RuntimeError(f"or_lw rc={rc}")
    return out


def run(p: OracleProblem, u0: np.ndarray | None, nsteps: int, n0: int = 0,
        weights: np.ndarray | None = None):
    """Advance nsteps from step n0.  Returns (final state, h) where h[k] is the
    complex waveform sample of state n0+k, k = 0..nsteps."""
    if u0 is None:
        u = np.zeros((2, p.Nr, p.Ntheta), dtype=np.complex128)
    else:
        u = _state(u0, p).copy()
    h = np.empty(nsteps + 1, dtype=np.complex128)
    g, s = p.grid(), p.source()
    wp = None
    if weights is not None:
        weights = np.ascontiguousarray(weights, dtype=np.float64)
        wp = _dp(weights)
    rc = lib().or_run(ctypes.byref(g), ctypes.byref(s), n0, nsteps, _dp(u), wp, _dp(h))
    if rc != 0:
        raise RuntimeError(f"or_run rc={rc}")
    return u, h
