"""Thin ctypes binding of libteuk (include/teuk.h).

Only argument marshalling happens here: every step of the time stepper runs
in the library's CUDA kernels.  PyTorch supplies device memory (caller-owned
buffers, as the ABI requires) and streams.  There is no CPU fallback: if
libteuk.so has not been built, or no GPU is present, the calls fail loudly.

The functions keep the C names (teuk_init_grid, teuk_set_source, teuk_step,
teuk_extract_waveform, ...); :class:`Stepper` bundles a context with its
three device buffers for convenience.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import _build

TEUK_OK = 0
TEUK_E_INVAL = 1
TEUK_E_CUDA = 2
TEUK_E_NONFINITE = 3
TEUK_E_UNSTABLE = 4
TEUK_E_TIMEOUT = 5
TEUK_E_STATE = 6
TEUK_E_RANGE = 7

TEUK_FP64 = 0
TEUK_FP32 = 1
TEUK_SCHEME_SPLIT = 0
TEUK_SCHEME_LITERAL = 1

EXPORTED = [
    "teuk_workspace_bytes", "teuk_init_grid", "teuk_set_source", "teuk_set_weights",
    "teuk_set_state", "teuk_get_state", "teuk_step", "teuk_extract_waveform",
    "teuk_current_step", "teuk_last_error", "teuk_status_string", "teuk_destroy",
    "teuk_tiling", "teuk_autotune", "teuk_set_tiling", "teuk_literal_step_static",
    "teuk_kernel_config", "teuk_set_persistent", "teuk_autotune_cold",
    "teuk_batch_workspace_bytes", "teuk_batch_create", "teuk_batch_step", "teuk_batch_tiling",
    "teuk_batch_set_tiling", "teuk_batch_steps_per_launch", "teuk_batch_set_steps_per_launch",
    "teuk_batch_autotune", "teuk_batch_last_error", "teuk_batch_destroy",
    "teuk_apply_step", "teuk_apply_sample", "teuk_adjoint_workspace_bytes", "teuk_adjoint_step", "teuk_dot",
    "teuk_set_tiling_steps", "teuk_state_level", "teuk_set_wait_limit", "teuk_fma_rate",
    "teuk_set_pipelined", "teuk_adjoint_step_spin", "teuk_apply_step_sample",
    "teuk_adjoint_prepare", "teuk_tape_bytes", "teuk_apply_step_tape", "teuk_adjoint_step_tape",
]


class TeukError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


_STATUS = {0: "TEUK_OK", 1: "TEUK_E_INVAL", 2: "TEUK_E_CUDA", 3: "TEUK_E_NONFINITE",
           4: "TEUK_E_UNSTABLE", 5: "TEUK_E_TIMEOUT", 6: "TEUK_E_STATE", 7: "TEUK_E_RANGE"}


class GridDesc(ctypes.Structure):
    """teuk_grid_desc"""
    _fields_ = [
        ("s", ctypes.c_int32), ("m", ctypes.c_int32),
        ("M", ctypes.c_double), ("a", ctypes.c_double),
        ("Nr", ctypes.c_int64), ("Ntheta", ctypes.c_int64),
        ("rstar_min", ctypes.c_double), ("rstar_max", ctypes.c_double),
        ("dt", ctypes.c_double), ("rstar_extract", ctypes.c_double),
        ("precision", ctypes.c_int32), ("scheme", ctypes.c_int32),
        ("allow_unstable", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def lib(load_only: bool = False):
    """Load libteuk.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_0909_4039_gb300._build.build() "
                           "(or __graft_entry__.build()); there is no CPU fallback")
    L = ctypes.CDLL(path)
    vp, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    sz = ctypes.POINTER(ctypes.c_size_t)
    gp = ctypes.POINTER(GridDesc)
    L.teuk_workspace_bytes.argtypes = [gp, sz, sz, sz]
    L.teuk_init_grid.argtypes = [gp, vp, vp, vp, i64, vp, ctypes.POINTER(vp)]
    L.teuk_set_source.argtypes = [vp, dbl, dbl, dbl, dbl, dbl, dbl]
    L.teuk_set_weights.argtypes = [vp, dp]
    L.teuk_set_state.argtypes = [vp, vp, i64, vp]
    L.teuk_get_state.argtypes = [vp, vp, ctypes.POINTER(i64), vp]
    L.teuk_step.argtypes = [vp, i64, vp]
    L.teuk_state_level.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int)]
    L.teuk_extract_waveform.argtypes = [vp, i64, i64, dp, dp, vp]
    L.teuk_current_step.argtypes = [vp]
    L.teuk_current_step.restype = i64
    L.teuk_last_error.argtypes = [vp]
    L.teuk_last_error.restype = ctypes.c_char_p
    L.teuk_status_string.argtypes = [ctypes.c_int]
    L.teuk_status_string.restype = ctypes.c_char_p
    L.teuk_destroy.argtypes = [vp]
    L.teuk_tiling.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                              ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int)]
    L.teuk_autotune.argtypes = [vp, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_int)]
    L.teuk_set_tiling.argtypes = [vp, ctypes.c_int]
    L.teuk_literal_step_static.argtypes = [vp, vp, vp, i64, vp]
    L.teuk_kernel_config.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.teuk_set_tiling_steps.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.teuk_set_tiling_steps.restype = ctypes.c_int
    L.teuk_set_persistent.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.teuk_autotune_cold.argtypes = [vp, ctypes.c_int, vp, ctypes.c_size_t, vp, ctypes.POINTER(ctypes.c_int)]
    L.teuk_set_wait_limit.argtypes = [vp, ctypes.c_int]
    L.teuk_set_pipelined.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.teuk_fma_rate.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, dp]
    for name in ("teuk_workspace_bytes", "teuk_init_grid", "teuk_set_source", "teuk_set_weights",
                 "teuk_set_state", "teuk_get_state", "teuk_step", "teuk_extract_waveform", "teuk_destroy",
                 "teuk_state_level",
                 "teuk_tiling", "teuk_autotune", "teuk_set_tiling", "teuk_literal_step_static",
                 "teuk_kernel_config", "teuk_set_persistent", "teuk_autotune_cold", "teuk_set_wait_limit",
                 "teuk_fma_rate", "teuk_set_pipelined"):
        getattr(L, name).restype = ctypes.c_int
    L.teuk_apply_step.argtypes = [vp, vp, vp, i64, ctypes.c_int, vp]
    L.teuk_apply_sample.argtypes = [vp, vp, ctypes.c_int, vp, vp]
    L.teuk_apply_step_sample.argtypes = [vp, vp, vp, i64, ctypes.c_int, vp, vp]
    L.teuk_adjoint_prepare.argtypes = [vp, vp, vp]
    L.teuk_tape_bytes.argtypes = [vp, sz]
    L.teuk_apply_step_tape.argtypes = [vp, vp, vp, i64, ctypes.c_int, vp, vp, vp]
    L.teuk_adjoint_step_tape.argtypes = [vp, vp, vp, vp, i64, ctypes.c_int, vp, vp, vp]
    L.teuk_adjoint_workspace_bytes.argtypes = [vp, sz]
    L.teuk_adjoint_step.argtypes = [vp, vp, vp, i64, ctypes.c_int, vp, vp, vp]
    L.teuk_adjoint_step_spin.argtypes = [vp, vp, vp, vp, i64, ctypes.c_int, vp, vp, vp]
    L.teuk_dot.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    for name in ("teuk_apply_step", "teuk_apply_sample", "teuk_adjoint_workspace_bytes", "teuk_adjoint_step",
                 "teuk_dot", "teuk_adjoint_step_spin", "teuk_apply_step_sample", "teuk_adjoint_prepare",
                 "teuk_tape_bytes", "teuk_apply_step_tape", "teuk_adjoint_step_tape"):
        getattr(L, name).restype = ctypes.c_int
    pvp = ctypes.POINTER(vp)
    ip = ctypes.POINTER(ctypes.c_int)
    L.teuk_batch_workspace_bytes.argtypes = [pvp, ctypes.c_int, sz]
    L.teuk_batch_create.argtypes = [pvp, ctypes.c_int, vp, ctypes.c_size_t, pvp]
    L.teuk_batch_step.argtypes = [vp, i64, vp]
    L.teuk_batch_tiling.argtypes = [vp, ip, ip, sz]
    L.teuk_batch_set_tiling.argtypes = [vp, ip]
    L.teuk_batch_steps_per_launch.argtypes = [vp, ip]
    L.teuk_batch_set_steps_per_launch.argtypes = [vp, ctypes.c_int]
    L.teuk_batch_autotune.argtypes = [vp, ctypes.c_int, vp]
    L.teuk_batch_last_error.argtypes = [vp]
    L.teuk_batch_last_error.restype = ctypes.c_char_p
    L.teuk_batch_destroy.argtypes = [vp]
    for name in ("teuk_batch_workspace_bytes", "teuk_batch_create", "teuk_batch_step", "teuk_batch_tiling",
                 "teuk_batch_set_tiling", "teuk_batch_steps_per_launch", "teuk_batch_set_steps_per_launch",
                 "teuk_batch_autotune", "teuk_batch_destroy"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int, ctx=None):
    if rc != TEUK_OK:
        msg = lib().teuk_last_error(ctx)
        raise TeukError(rc, msg.decode() if msg else "")


def make_desc(s, m, a, Nr, Ntheta, rstar_min, rstar_max, dt=0.0, rstar_extract=500.0, M=1.0,
              precision=TEUK_FP64, scheme=TEUK_SCHEME_SPLIT, allow_unstable=False) -> GridDesc:
    return GridDesc(int(s), int(m), float(M), float(a), int(Nr), int(Ntheta), float(rstar_min),
                    float(rstar_max), float(dt), float(rstar_extract), int(precision), int(scheme),
                    int(bool(allow_unstable)), 0)


def teuk_workspace_bytes(desc: GridDesc):
    a, b, c = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().teuk_workspace_bytes(ctypes.byref(desc), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def teuk_init_grid(desc: GridDesc, d_state: int, d_coef: int, d_wave: int, wave_capacity: int,
                   stream: int = 0):
    ctx = ctypes.c_void_p()
    _check(lib().teuk_init_grid(ctypes.byref(desc), d_state, d_coef, d_wave, wave_capacity, stream,
                                ctypes.byref(ctx)))
    return ctx


def teuk_set_source(ctx, amp: complex, r0: float, sigma_rstar: float, sigma_theta: float,
                    Omega: float = float("nan")):
    amp = complex(amp)
    _check(lib().teuk_set_source(ctx, amp.real, amp.imag, r0, sigma_rstar, sigma_theta, Omega), ctx)


def teuk_set_weights(ctx, w: np.ndarray | None):
    if w is None:
        _check(lib().teuk_set_weights(ctx, None), ctx)
    else:
        w = np.ascontiguousarray(w, dtype=np.float64)
        _check(lib().teuk_set_weights(ctx, w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), ctx)


def teuk_set_state(ctx, src_ptr: int, step: int, stream: int = 0):
    _check(lib().teuk_set_state(ctx, src_ptr, step, stream), ctx)


def teuk_get_state(ctx, dst_ptr: int, stream: int = 0) -> int:
    st = ctypes.c_int64()
    _check(lib().teuk_get_state(ctx, dst_ptr, ctypes.byref(st), stream), ctx)
    return st.value


def teuk_step(ctx, nsteps: int, stream: int = 0):
    _check(lib().teuk_step(ctx, int(nsteps), stream), ctx)


def teuk_state_level(ctx):
    """(byte offset of the current level in d_state, level bytes, shifted)."""
    off = ctypes.c_int64()
    nb = ctypes.c_size_t()
    sh = ctypes.c_int()
    _check(lib().teuk_state_level(ctx, ctypes.byref(off), ctypes.byref(nb), ctypes.byref(sh)), ctx)
    return off.value, nb.value, bool(sh.value)


def teuk_extract_waveform(ctx, first_step: int, count: int, want_rows: bool = False, Ntheta: int = 0,
                          stream: int = 0):
    h = np.empty(count, dtype=np.complex128)
    rows = np.empty((count, Ntheta), dtype=np.complex128) if want_rows else None
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib().teuk_extract_waveform(ctx, first_step, count, h.ctypes.data_as(dp),
                                       rows.ctypes.data_as(dp) if rows is not None else None, stream), ctx)
    return (h, rows) if want_rows else h


def teuk_current_step(ctx) -> int:
    return int(lib().teuk_current_step(ctx))


def teuk_tiling(ctx) -> dict:
    tr, th, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    sm = ctypes.c_size_t()
    _check(lib().teuk_tiling(ctx, ctypes.byref(tr), ctypes.byref(th), ctypes.byref(sm), ctypes.byref(g)), ctx)
    return {"tile_rows": tr.value, "threads": th.value, "smem_bytes": sm.value, "group": g.value}


def teuk_autotune(ctx, trial_steps: int = 20, stream: int = 0) -> int:
    tr = ctypes.c_int()
    _check(lib().teuk_autotune(ctx, int(trial_steps), stream, ctypes.byref(tr)), ctx)
    return tr.value


def teuk_autotune_cold(ctx, trial_steps: int, d_flush: int, flush_bytes: int, stream: int = 0) -> int:
    tr = ctypes.c_int()
    _check(lib().teuk_autotune_cold(ctx, int(trial_steps), d_flush, int(flush_bytes), stream, ctypes.byref(tr)), ctx)
    return tr.value


def teuk_set_tiling(ctx, tile_rows: int):
    _check(lib().teuk_set_tiling(ctx, int(tile_rows)), ctx)


def teuk_set_pipelined(ctx, tile_rows: int, threads: int = 256):
    _check(lib().teuk_set_pipelined(ctx, int(tile_rows), int(threads)), ctx)


def teuk_set_wait_limit(ctx, rounds: int):
    """Bound of the tiled kernels' waits on their state copies (test hook;
    rounds < 0 restores the default)."""
    _check(lib().teuk_set_wait_limit(ctx, int(rounds)), ctx)


def teuk_fma_rate(precision: str, iters: int, d_sink: int, stream: int) -> float:
    """Measured FMA throughput of the current device in flop/s (two per FMA)."""
    out = ctypes.c_double()
    prec = {"fp64": TEUK_FP64, "fp32": TEUK_FP32}[precision]
    _check(lib().teuk_fma_rate(prec, int(iters), d_sink, stream, ctypes.byref(out)))
    return out.value


def teuk_kernel_config(ctx) -> dict:
    pe, nc, gr, ks = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().teuk_kernel_config(ctx, ctypes.byref(pe), ctypes.byref(nc), ctypes.byref(gr), ctypes.byref(ks)), ctx)
    return {"persistent": pe.value == 1, "pipelined": pe.value == 2, "consumer_threads": nc.value,
            "grid": gr.value, "steps_per_launch": ks.value}


def teuk_set_tiling_steps(ctx, tile_rows: int, steps_per_launch: int):
    _check(lib().teuk_set_tiling_steps(ctx, int(tile_rows), int(steps_per_launch)), ctx)


def teuk_set_persistent(ctx, tile_rows: int, consumer_threads: int = 480):
    _check(lib().teuk_set_persistent(ctx, int(tile_rows), int(consumer_threads)), ctx)


def teuk_literal_step_static(ctx, d_in: int, d_out: int, n: int, stream: int = 0):
    """One literal-scheme step from d_in to d_out (device pointers in the
    context's state precision) with the library's static midpoint scratch;
    for callers that cannot allocate device memory.  See include/teuk.h."""
    _check(lib().teuk_literal_step_static(ctx, d_in, d_out, int(n), stream), ctx)


def teuk_destroy(ctx):
    _check(lib().teuk_destroy(ctx))


class Stepper:
    """A context plus its caller-owned device buffers (torch tensors)."""

    def __init__(self, s=-2, m=2, a=0.9, Nr=1024, Ntheta=32, rstar_min=-100.0, rstar_max=600.0,
                 dt=0.0, rstar_extract=500.0, M=1.0, precision="fp64", scheme="split",
                 allow_unstable=False, wave_capacity=4096, device=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libteuk needs a CUDA GPU; no CPU fallback exists")
        self.torch = torch
        self.device = torch.device(device or "cuda:0")
        prec = {"fp64": TEUK_FP64, "fp32": TEUK_FP32}[precision]
        sch = {"split": TEUK_SCHEME_SPLIT, "literal": TEUK_SCHEME_LITERAL}[scheme]
        self.desc = make_desc(s, m, a, Nr, Ntheta, rstar_min, rstar_max, dt, rstar_extract, M, prec, sch,
                              allow_unstable)
        self.Nr, self.Ntheta, self.precision = int(Nr), int(Ntheta), precision
        sb, cb, wb = teuk_workspace_bytes(self.desc)
        with torch.cuda.device(self.device):
            self.stream = stream or torch.cuda.Stream(device=self.device)
            self.d_state = torch.empty(sb, dtype=torch.uint8, device=self.device)
            self.d_coef = torch.empty(cb, dtype=torch.uint8, device=self.device)
            self.d_wave = torch.empty(wb * wave_capacity, dtype=torch.uint8, device=self.device)
        self.wave_capacity = wave_capacity
        self.ctx = teuk_init_grid(self.desc, self.d_state.data_ptr(), self.d_coef.data_ptr(),
                                  self.d_wave.data_ptr(), wave_capacity, self.stream.cuda_stream)
        drs = (rstar_max - rstar_min) / (Nr - 1)
        self.drs = drs
        self.dt = dt if dt > 0 else 0.5 * drs

    @property
    def sh(self) -> int:
        return self.stream.cuda_stream

    def autotune(self, trial_steps: int = 20, flush=None) -> int:
        """Measured choice of kernel and tile height.  With flush (a device
        tensor larger than the L2) every timed trial step starts cold."""
        if flush is None:
            return teuk_autotune(self.ctx, trial_steps, self.sh)
        return teuk_autotune_cold(self.ctx, trial_steps, flush.data_ptr(), flush.numel() * flush.element_size(),
                                  self.sh)

    def tiling(self) -> dict:
        out = teuk_tiling(self.ctx)
        out.update(teuk_kernel_config(self.ctx))
        return out

    def set_tiling(self, tile_rows: int, steps_per_launch: int = 1):
        if steps_per_launch == 1:
            teuk_set_tiling(self.ctx, tile_rows)
        else:
            teuk_set_tiling_steps(self.ctx, tile_rows, steps_per_launch)

    def set_persistent(self, tile_rows: int, consumer_threads: int = 480):
        teuk_set_persistent(self.ctx, tile_rows, consumer_threads)

    def set_pipelined(self, tile_rows: int, threads: int = 256):
        teuk_set_pipelined(self.ctx, tile_rows, threads)

    def set_source(self, amp=1.0, r0=10.0, sigma_rstar=0.1, sigma_theta=0.1, Omega=float("nan")):
        teuk_set_source(self.ctx, amp, r0, sigma_rstar, sigma_theta, Omega)

    def set_weights(self, w=None):
        teuk_set_weights(self.ctx, w)

    def set_state(self, u: np.ndarray, step: int = 0):
        u = np.ascontiguousarray(u, dtype=np.complex128)
        if u.shape != (2, self.Nr, self.Ntheta):
            raise ValueError(f"state shape {u.shape} != {(2, self.Nr, self.Ntheta)}")
        teuk_set_state(self.ctx, u.ctypes.data, step, self.sh)

    def set_state_device(self, u, step: int = 0):
        """u: torch complex128 CUDA tensor of shape (2, Nr, Ntheta)."""
        assert u.is_cuda and u.dtype == self.torch.complex128 and u.is_contiguous()
        teuk_set_state(self.ctx, u.data_ptr(), step, self.sh)

    def get_state(self) -> np.ndarray:
        out = np.empty((2, self.Nr, self.Ntheta), dtype=np.complex128)
        teuk_get_state(self.ctx, out.ctypes.data, self.sh)
        return out

    def step(self, n: int):
        teuk_step(self.ctx, n, self.sh)

    def level_view(self):
        """The current state level as a [2, Nr, Ntheta] complex tensor view of
        d_state (complex64 for the FP32 state), and whether it is the shifted
        split-scheme state.  Rows written through it are read by the next
        step; order the writes on self.stream."""
        import torch
        off, nb, shifted = teuk_state_level(self.ctx)
        dt = torch.complex64 if self.precision == "fp32" else torch.complex128
        v = self.d_state[off:off + nb].view(dt).view(2, self.Nr, self.Ntheta)
        return v, shifted

    def waveform(self, first: int, count: int, rows: bool = False):
        return teuk_extract_waveform(self.ctx, first, count, rows, self.Ntheta, self.sh)

    @property
    def current_step(self) -> int:
        return teuk_current_step(self.ctx)

    def synchronize(self):
        self.stream.synchronize()

    def close(self):
        if getattr(self, "ctx", None) is not None:
            teuk_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _bcheck(rc: int, batch=None):
    if rc != TEUK_OK:
        msg = lib().teuk_batch_last_error(batch)
        raise TeukError(rc, msg.decode() if msg else "")


class Batch:
    """Instances (Steppers of the split scheme) advanced together: one launch
    per step over every tile of every instance (teuk_batch_* in the C ABI).
    The steppers must outlive the batch and be stepped only through it."""

    def __init__(self, steppers, stream=None):
        import torch
        self.torch = torch
        self.steppers = list(steppers)
        if not self.steppers:
            raise ValueError("a batch needs at least one instance")
        n = len(self.steppers)
        self.device = self.steppers[0].device
        self.stream = stream or self.steppers[0].stream
        arr = (ctypes.c_void_p * n)(*[st.ctx for st in self.steppers])
        nbytes = ctypes.c_size_t()
        _bcheck(lib().teuk_batch_workspace_bytes(arr, n, ctypes.byref(nbytes)))
        self.d_ws = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8, device=self.device)
        base = self.d_ws.data_ptr()
        aligned = (base + 255) & ~255
        out = ctypes.c_void_p()
        _bcheck(lib().teuk_batch_create(arr, n, aligned, int(nbytes.value), ctypes.byref(out)))
        self.batch = out

    @property
    def sh(self) -> int:
        return self.stream.cuda_stream

    def _after_instances(self):
        # work queued on the instances' own streams comes first
        for st in self.steppers:
            if st.stream != self.stream:
                self.stream.wait_stream(st.stream)

    def _before_instances(self):
        # later work on an instance's stream sees the batched steps
        for st in self.steppers:
            if st.stream != self.stream:
                st.stream.wait_stream(self.stream)

    def step(self, nsteps: int):
        self._after_instances()
        _bcheck(lib().teuk_batch_step(self.batch, int(nsteps), self.sh), self.batch)
        self._before_instances()

    def autotune(self, trial_steps: int = 10) -> list:
        self._after_instances()
        _bcheck(lib().teuk_batch_autotune(self.batch, int(trial_steps), self.sh), self.batch)
        self._before_instances()
        return self.tiling()["tile_rows"]

    def tiling(self) -> dict:
        n = len(self.steppers)
        tr = (ctypes.c_int * n)()
        tot = ctypes.c_int()
        sm = ctypes.c_size_t()
        _bcheck(lib().teuk_batch_tiling(self.batch, tr, ctypes.byref(tot), ctypes.byref(sm)), self.batch)
        ks = ctypes.c_int()
        _bcheck(lib().teuk_batch_steps_per_launch(self.batch, ctypes.byref(ks)), self.batch)
        return {"tile_rows": list(tr), "total_tiles": tot.value, "smem_bytes": sm.value,
                "steps_per_launch": ks.value}

    def set_tiling(self, tile_rows=None, steps_per_launch=None):
        """Tile height per instance and/or time steps per launch (1 or 2)."""
        if steps_per_launch is not None:
            _bcheck(lib().teuk_batch_set_steps_per_launch(self.batch, int(steps_per_launch)), self.batch)
        if tile_rows is None:
            return
        n = len(self.steppers)
        if len(tile_rows) != n:
            raise ValueError("one tile height per instance")
        arr = (ctypes.c_int * n)(*[int(t) for t in tile_rows])
        _bcheck(lib().teuk_batch_set_tiling(self.batch, arr), self.batch)

    def synchronize(self):
        self.stream.synchronize()

    def close(self):
        if getattr(self, "batch", None) is not None:
            lib().teuk_batch_destroy(self.batch)
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
