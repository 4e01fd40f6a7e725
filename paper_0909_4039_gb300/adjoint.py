"""Gradients of waveform losses through the split stepper.

The forward map of the split scheme (see teuk_apply_step in include/teuk.h)
  s_1 = M_0(u_0),  s_{n+1} = M_n(s_n),  h_0 = E u_0,  h_n = E C_{dt/2} s_n
is differentiated in reverse mode: with g_n = dL/dRe h_n + i dL/dIm h_n,
  lam_N = C_{dt/2}^H E^H g_N,
  lam_n = M_n^H lam_{n+1} + C_{dt/2}^H E^H g_n,     lam_{u0} = M_0^H lam_1 + E^H g_0,
  dL/dp = sum_n Re <lam_{n+1}, dM_n/dp s_n> + sum_n Re conj(g_n) dh_n/dp|_s.
The transposed steps are the library's hand-written adjoint kernels
(teuk_adjoint_step).  The source amplitude A and the orbit radius r0 enter
only the source term, whose derivatives the adjoint kernel contracts on the
source patch.  The spin a enters every coefficient (through r(r*; a), the
pivots, the source prefactor, r0* and the Kepler frequency); its term
<lam_{n+1}, dM_n/da s_n> is the central difference (M_n(a+e) - M_n(a-e)) s_n / 2e
of two forward steps from the same state, contracted with lam_{n+1}
(truncation error O(e^2)).

The backward sweep needs s_n at every step: states are kept every
k ~ sqrt(N) steps during the forward run and each segment is recomputed from
its checkpoint before it is swept (sqrt(N) checkpointing with recompute).

Everything runs in the library's kernels on device buffers; PyTorch holds
the buffers and carries the gradients.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import inputs, teuk


@dataclass
class Params:
    """Differentiable parameters: source amplitude A (complex), orbit radius
    r0 (M) and spin a (M)."""
    amp: complex
    r0: float
    a: float


class Operator:
    """The step, sample and adjoint operators of one parameter set, on
    caller buffers.  `w` fixes the grid, mode and source widths; `prm` the
    differentiable parameters."""

    def __init__(self, w: inputs.Workload, prm: Params, precision: str = "fp64", device=None, stream=None):
        import torch
        self.torch = torch
        drs = (w.rs_max - w.rs_min) / (w.Nr - 1)
        self.st = teuk.Stepper(s=w.s, m=w.m, a=prm.a, Nr=w.Nr, Ntheta=w.Ntheta, rstar_min=w.rs_min,
                               rstar_max=w.rs_max, dt=w.cfl * drs, rstar_extract=w.rs_ext, M=w.M,
                               precision=precision, wave_capacity=4, device=device, stream=stream)
        self.st.set_source(prm.amp, prm.r0, w.sig_r, w.sig_th)
        self.w, self.prm, self.precision = w, prm, precision
        self.ctype = torch.complex64 if precision == "fp32" else torch.complex128
        self.shape = (2, w.Nr, w.Ntheta)
        nb = ctypes_size(lambda sz: teuk.lib().teuk_adjoint_workspace_bytes(self.st.ctx, sz))
        self.ws = torch.zeros(nb // 8, dtype=torch.float64, device=self.st.device)
        self.sh = self.st.sh

    def empty(self):
        return self.torch.empty(self.shape, dtype=self.ctype, device=self.st.device)

    def zeros(self):
        return self.torch.zeros(self.shape, dtype=self.ctype, device=self.st.device)

    def step(self, s_in, s_out, n: int, first: bool):
        teuk._check(teuk.lib().teuk_apply_step(self.st.ctx, s_in.data_ptr(), s_out.data_ptr(), int(n), int(first),
                                               self.sh), self.st.ctx)

    def sample(self, s, physical: bool, out_ptr: int):
        teuk._check(teuk.lib().teuk_apply_sample(self.st.ctx, s.data_ptr(), int(physical), out_ptr, self.sh),
                    self.st.ctx)

    def adjoint(self, lam_in, lam_out, n: int, first: bool, gseed_ptr):
        teuk._check(teuk.lib().teuk_adjoint_step(self.st.ctx, lam_in.data_ptr(), lam_out.data_ptr(), int(n),
                                                 int(first), gseed_ptr, self.ws.data_ptr(), self.sh), self.st.ctx)

    def dot(self, x, y, out_ptr: int):
        teuk._check(teuk.lib().teuk_dot(self.st.ctx, x.data_ptr(), y.data_ptr(), self.ws.data_ptr(), out_ptr,
                                        self.sh), self.st.ctx)

    def close(self):
        self.st.close()


def ctypes_size(call) -> int:
    import ctypes
    v = ctypes.c_size_t()
    rc = call(ctypes.byref(v))
    if rc != 0:
        raise teuk.TeukError(rc, "workspace query")
    return int(v.value)


def _ptr(t, k: int) -> int:
    """Device address of element k (in storage order) of a contiguous
    complex128 tensor."""
    return t.data_ptr() + 16 * k


def run_forward(op: Operator, nsteps: int, u0=None, every: int | None = None):
    """Waveform h_0..h_N (complex128, device) and the checkpoints: {0: u_0}
    and {n: s_n} for every n divisible by `every`.  Call on the operator's
    stream."""
    torch = op.torch
    h = torch.zeros(nsteps + 1, dtype=torch.complex128, device=op.st.device)
    u = op.zeros() if u0 is None else torch.as_tensor(u0).to(device=op.st.device, dtype=op.ctype).reshape(op.shape)
    ck = {0: u.clone()}
    op.sample(u, True, _ptr(h, 0))
    if nsteps == 0:
        return h, ck
    s, t = op.empty(), op.empty()
    op.step(u, s, 0, True)
    for n in range(1, nsteps + 1):
        if every and n % every == 0 and n < nsteps:
            ck[n] = s.clone()
        op.sample(s, False, _ptr(h, n))
        if n < nsteps:
            op.step(s, t, n, False)
            s, t = t, s
    return h, ck


def gradients(w: inputs.Workload, prm: Params, nsteps: int, grad_h, u0=None, precision: str = "fp64",
              every: int | None = None, wrt_a: bool = True, eps_a: float | None = None, device=None):
    """Reverse-mode derivatives of a loss whose gradient with respect to the
    waveform h_0..h_N is grad_h (complex, dL/dRe h + i dL/dIm h).  Returns
    dL/dRe A, dL/dIm A, dL/dr0, dL/da (None unless wrt_a) and the adjoint of
    the initial state (dL/dRe u_0 + i dL/dIm u_0), plus the waveform."""
    import torch
    op = Operator(w, prm, precision, device=device)
    every = every or max(1, int(round(math.sqrt(max(nsteps, 1)))))
    try:
        with torch.cuda.stream(op.st.stream):
            return _sweep(op, w, prm, nsteps, grad_h, u0, precision, every, wrt_a, eps_a, device)
    finally:
        op.close()


def _sweep(op, w, prm, nsteps, grad_h, u0, precision, every, wrt_a, eps_a, device):
    import torch
    h, ck = run_forward(op, nsteps, u0, every)
    g = grad_h.to(device=op.st.device, dtype=torch.complex128).contiguous()
    if g.numel() != nsteps + 1:
        raise ValueError("grad_h needs one entry per sample h_0..h_N")
    if wrt_a:
        eps = eps_a if eps_a is not None else (1e-4 if precision == "fp64" else 1e-3)
        opp = Operator(w, Params(prm.amp, prm.r0, prm.a + eps), precision, device=device, stream=op.st.stream)
        opm = Operator(w, Params(prm.amp, prm.r0, prm.a - eps), precision, device=device, stream=op.st.stream)
        dots = torch.zeros((nsteps + 1, 2), dtype=torch.complex128, device=op.st.device)
        samp = torch.zeros((nsteps + 1, 2), dtype=torch.complex128, device=op.st.device)
        tp, tm = op.empty(), op.empty()
    op.ws.zero_()
    lam, lam2 = op.zeros(), op.empty()
    # lam_N from the last sample alone (lam_{N+1} = 0)
    op.adjoint(lam, lam2, nsteps, nsteps == 0, _ptr(g, nsteps))
    lam, lam2 = lam2, lam
    bounds = sorted(k for k in ck) + [nsteps]
    for a, b in reversed(list(zip(bounds[:-1], bounds[1:]))):
        # states s_a .. s_b of this segment (s_0 is the physical u_0)
        states = [ck[a]]
        for n in range(a, b):
            nxt = op.empty()
            op.step(states[-1], nxt, n, n == 0)
            states.append(nxt)
        if wrt_a:
            # a-derivative of the samples h_n, n in (a, b]
            for n in range(max(a + 1, 1), b + 1):
                opp.sample(states[n - a], False, _ptr(samp, 2 * n))
                opm.sample(states[n - a], False, _ptr(samp, 2 * n + 1))
        for n in range(b - 1, a - 1, -1):
            sn = states[n - a]
            if wrt_a:
                # <lam_{n+1}, M_n(a +- e) s_n>
                opp.step(sn, tp, n, n == 0)
                opm.step(sn, tm, n, n == 0)
                op.dot(lam, tp, _ptr(dots, 2 * n))
                op.dot(lam, tm, _ptr(dots, 2 * n + 1))
            op.adjoint(lam, lam2, n, n == 0, _ptr(g, n))
            lam, lam2 = lam2, lam
        del states
    acc = op.ws[:4].cpu().numpy()
    out = {"dA_re": float(acc[0]), "dA_im": float(-acc[1]), "dr0": float(acc[2]), "du0": lam.clone(), "h": h}
    if wrt_a:
        d = dots.cpu().numpy()
        sp = samp.cpu().numpy()
        gn = g.cpu().numpy()
        step_term = np.sum((d[:nsteps, 0] - d[:nsteps, 1]).real)
        samp_term = np.sum((np.conj(gn[1:]) * (sp[1:, 0] - sp[1:, 1])).real)
        out["da"] = float((step_term + samp_term) / (2.0 * eps))
        opp.close()
        opm.close()
    else:
        out["da"] = None
    op.st.synchronize()
    return out


def waveform(w: inputs.Workload, prm: Params, nsteps: int, u0=None, precision: str = "fp64", device=None):
    """h_0..h_N for one parameter set (complex128, device)."""
    import torch
    op = Operator(w, prm, precision, device=device)
    try:
        with torch.cuda.stream(op.st.stream):
            h, _ = run_forward(op, nsteps, u0)
        op.st.synchronize()
        return h
    finally:
        op.close()


def _make_function():
    import torch

    class WaveformFunction(torch.autograd.Function):
        """h = waveform(A, r0, a) at the extraction node; params is a float64
        tensor (Re A, Im A, r0, a).  The backward pass runs the adjoint sweep
        with sqrt(N) checkpointing."""

        @staticmethod
        def forward(ctx, params, w, nsteps, precision):
            p = params.detach().cpu().numpy().astype(np.float64)
            prm = Params(complex(p[0], p[1]), float(p[2]), float(p[3]))
            ctx.w, ctx.nsteps, ctx.precision, ctx.prm = w, int(nsteps), precision, prm
            ctx.device = params.device
            h = waveform(w, prm, int(nsteps), precision=precision)
            return h.to(params.device)

        @staticmethod
        def backward(ctx, grad_h):
            r = gradients(ctx.w, ctx.prm, ctx.nsteps, grad_h, precision=ctx.precision)
            gp = torch.tensor([r["dA_re"], r["dA_im"], r["dr0"], r["da"]], dtype=torch.float64,
                              device=ctx.device)
            return gp, None, None, None

    return WaveformFunction


_WF = None


def waveform_fn(params, w: inputs.Workload, nsteps: int, precision: str = "fp64"):
    """Differentiable waveform: params = tensor (Re A, Im A, r0, a)."""
    global _WF
    if _WF is None:
        _WF = _make_function()
    return _WF.apply(params, w, nsteps, precision)
