"""Helpers shared by the tests: one workload description drives both the
oracle (oracle/, FP64 CPU) and the CUDA library (through the C ABI)."""
from __future__ import annotations

import numpy as np

from paper_0909_4039_gb300 import inputs


def rel_l2(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def oracle_problem(w: inputs.Workload, scheme: str = "split", with_source: bool = True, nthreads: int = 0):
    from oracle import oracle as O
    drs = (w.rs_max - w.rs_min) / (w.Nr - 1)
    return O.OracleProblem(s=w.s, m=w.m, M=w.M, a=w.a, Nr=w.Nr, Ntheta=w.Ntheta, rs_min=w.rs_min,
                           rs_max=w.rs_max, dt=w.cfl * drs, rs_ext=w.rs_ext,
                           scheme=O.SCHEME_SPLIT if scheme == "split" else O.SCHEME_LITERAL,
                           amp=w.amp if with_source else 0.0, r0=w.r0, sig_r=w.sig_r, sig_th=w.sig_th,
                           nthreads=nthreads)


def gpu_stepper(w: inputs.Workload, precision: str = "fp64", scheme: str = "split", with_source: bool = True,
                wave_capacity: int | None = None, allow_unstable: bool = False):
    from paper_0909_4039_gb300 import teuk
    drs = (w.rs_max - w.rs_min) / (w.Nr - 1)
    st = teuk.Stepper(s=w.s, m=w.m, a=w.a, Nr=w.Nr, Ntheta=w.Ntheta, rstar_min=w.rs_min, rstar_max=w.rs_max,
                      dt=w.cfl * drs, rstar_extract=w.rs_ext, M=w.M, precision=precision, scheme=scheme,
                      allow_unstable=allow_unstable,
                      wave_capacity=wave_capacity or max(16, w.steps + 1))
    if with_source and w.amp != 0:
        st.set_source(w.amp, w.r0, w.sig_r, w.sig_th)
    return st
