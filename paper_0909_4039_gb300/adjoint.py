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
source patch.  The spin a enters every coefficient (through r(r*; a),
Delta and Sigma^2, the source prefactor, r0* and the Kepler frequency); its
terms <lam_{n+1}, dM_n/da s_n> and <g_n, d(E C_{dt/2})/da s_n> are contracted
inside the adjoint step from exact derivatives of the coefficient tables and
the forward stage values of s_n (teuk_adjoint_step_spin).  For checking,
spin="fd" takes them instead as central differences of two forward steps
at a +- e.

The spin term needs the forward stage values of every step.  By default
states are kept every k ~ sqrt(N) steps during the forward run, each segment
is recomputed from its checkpoint before it is swept, and the adjoint kernel
recomputes the implicit stage values from s_n (sqrt(N) checkpointing with
recompute).  With every = 1 every state is kept and no segment is
recomputed.  With tape=True every forward step records its stage values
(teuk_apply_step_tape, two states per step) and the sweep recomputes
nothing at all (teuk_adjoint_step_tape); the 4096 x 64 FP64 workload's 8000
steps take 134 GB, which one GPU's HBM holds.  Without the spin term the
adjoint step reads no state (the step is linear in s), so a sweep for the
source parameters alone recomputes nothing either.

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


# kernel launches issued through Operator (for launch accounting)
LAUNCHES = [0]


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
        # the spin adjoint's coefficient planes, once per operator (the zeros
        # above are queued on torch's stream)
        self.st.stream.wait_stream(torch.cuda.current_stream(self.st.device))
        rc = teuk.lib().teuk_adjoint_prepare(self.st.ctx, self.ws.data_ptr(), self.st.sh)
        if rc != 0:
            teuk._check(rc, self.st.ctx)
        L = teuk.lib()
        self._step, self._sample = L.teuk_apply_step, L.teuk_apply_sample
        self._step_sample = L.teuk_apply_step_sample
        self._adj, self._dot = L.teuk_adjoint_step, L.teuk_dot
        self._adjs = L.teuk_adjoint_step_spin
        self._step_tape, self._adjt = L.teuk_apply_step_tape, L.teuk_adjoint_step_tape
        self.tape_bytes = ctypes_size(lambda sz: teuk.lib().teuk_tape_bytes(self.st.ctx, sz))
        self._ctx, self._ws = self.st.ctx, self.ws.data_ptr()

    def empty(self):
        return self.torch.empty(self.shape, dtype=self.ctype, device=self.st.device)

    def zeros(self):
        return self.torch.zeros(self.shape, dtype=self.ctype, device=self.st.device)

    def _ok(self, rc):
        if rc != 0:
            teuk._check(rc, self._ctx)

    def step(self, s_in, s_out, n: int, first: bool):
        LAUNCHES[0] += 1
        self._ok(self._step(self._ctx, s_in.data_ptr(), s_out.data_ptr(), int(n), int(first), self.sh))

    def step_sample(self, s_in, s_out, n: int, first: bool, out_ptr: int):
        """step() plus the sample E C_{dt/2} s_out to out_ptr, in one launch."""
        LAUNCHES[0] += 1
        self._ok(self._step_sample(self._ctx, s_in.data_ptr(), s_out.data_ptr(), int(n), int(first), out_ptr,
                                   self.sh))

    def step_tape(self, s_in, s_out, n: int, first: bool, out_ptr: int, tape_ptr: int):
        """step_sample() that also writes the step's tape record at tape_ptr."""
        LAUNCHES[0] += 1
        self._ok(self._step_tape(self._ctx, s_in.data_ptr(), s_out.data_ptr(), int(n), int(first), out_ptr,
                                 tape_ptr, self.sh))

    def sample(self, s, physical: bool, out_ptr: int):
        LAUNCHES[0] += 1
        self._ok(self._sample(self._ctx, s.data_ptr(), int(physical), out_ptr, self.sh))

    def adjoint(self, lam_in, lam_out, n: int, first: bool, gseed_ptr):
        LAUNCHES[0] += 2     # the adjoint step and the reduction of its partial sums
        self._ok(self._adj(self._ctx, lam_in.data_ptr(), lam_out.data_ptr(), int(n), int(first), gseed_ptr,
                           self._ws, self.sh))

    def adjoint_spin(self, lam_in, lam_out, s, n: int, first: bool, gseed_ptr):
        """adjoint() plus the step's spin-derivative term (acc[4]); s = s_n."""
        LAUNCHES[0] += 2
        self._ok(self._adjs(self._ctx, lam_in.data_ptr(), lam_out.data_ptr(), s.data_ptr(), int(n), int(first),
                            gseed_ptr, self._ws, self.sh))

    def adjoint_tape(self, lam_in, lam_out, tape_ptr: int, n: int, first: bool, gseed_ptr):
        """adjoint_spin() with the stage values of step n read from its tape record."""
        LAUNCHES[0] += 2
        self._ok(self._adjt(self._ctx, lam_in.data_ptr(), lam_out.data_ptr(), tape_ptr, int(n), int(first),
                            gseed_ptr, self._ws, self.sh))

    def dot(self, x, y, out_ptr: int, z=None):
        """out = <x, y - z> (z None: <x, y>)."""
        LAUNCHES[0] += 2     # per-CTA partial sums and their fixed-order reduction
        self._ok(self._dot(self._ctx, x.data_ptr(), y.data_ptr(), None if z is None else z.data_ptr(), self._ws,
                           out_ptr, self.sh))

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


def run_forward(op: Operator, nsteps: int, u0=None, every: int | None = None, tape=None):
    """Waveform h_0..h_N (complex128, device), the checkpoints {0: u_0} and
    {n: s_n} for every n divisible by `every`, and the last state s_N (u_0
    when N = 0).  With `tape` (a device buffer of N records of
    op.tape_bytes) every step also writes its tape record n.  Call on the
    operator's stream."""
    torch = op.torch
    h = torch.zeros(nsteps + 1, dtype=torch.complex128, device=op.st.device)
    u = op.zeros() if u0 is None else torch.as_tensor(u0).to(device=op.st.device, dtype=op.ctype).reshape(op.shape)
    ck = {0: u.clone()}
    op.sample(u, True, _ptr(h, 0))
    if nsteps == 0:
        return h, ck, u
    s, t = op.empty(), op.empty()

    def adv(x, y, n):
        # one launch writes s_{n+1}, its sample h_{n+1} (and record n)
        if tape is None:
            op.step_sample(x, y, n, n == 0, _ptr(h, n + 1))
        else:
            op.step_tape(x, y, n, n == 0, _ptr(h, n + 1), tape.data_ptr() + n * op.tape_bytes)

    adv(u, s, 0)
    for n in range(1, nsteps):
        if every and n % every == 0:
            ck[n] = s.clone()
        adv(s, t, n)
        s, t = t, s
    return h, ck, s


class Forward:
    """A forward run kept for a backward sweep: the operator, the waveform
    and the checkpoints (sqrt(N) states), or the tape of every step."""

    def __init__(self, op, nsteps, h, ck, every, last=None, tape=None):
        self.op, self.nsteps, self.h, self.ck, self.every, self.last = op, nsteps, h, ck, every, last
        self.tape = tape

    def close(self):
        if self.op is not None:
            self.op.close()
            self.op = None
        self.ck = None
        self.last = None
        self.tape = None


def forward(w: inputs.Workload, prm: Params, nsteps: int, u0=None, precision: str = "fp64",
            every: int | None = None, device=None, tape: bool = False) -> Forward:
    """Forward run that keeps a state every `every` steps (default ~sqrt(N)),
    or with tape=True the tape record of every step (N x teuk_tape_bytes of
    device memory: two states per step; the backward sweep then recomputes
    nothing)."""
    import torch
    op = Operator(w, prm, precision, device=device)
    every = every or max(1, int(round(math.sqrt(max(nsteps, 1)))))
    tp = None
    if tape and nsteps > 0:
        tp = torch.empty(nsteps * op.tape_bytes // 8, dtype=torch.float64, device=op.st.device)
        every = 0
    caller = torch.cuda.current_stream(op.st.device)
    # u0 may come from work queued on the caller's stream
    op.st.stream.wait_stream(caller)
    with torch.cuda.stream(op.st.stream):
        if tp is not None:
            tp.record_stream(op.st.stream)
        h, ck, last = run_forward(op, nsteps, u0, every, tape=tp)
    # and the caller's later work reads h
    caller.wait_stream(op.st.stream)
    return Forward(op, nsteps, h, ck, every, last, tape=tp)


def backward(fw: Forward, grad_h, wrt_a: bool = True, eps_a: float | None = None, spin: str = "analytic") -> dict:
    """Reverse-mode derivatives of a loss whose gradient with respect to the
    waveform h_0..h_N of the forward run is grad_h (complex, dL/dRe h +
    i dL/dIm h): dL/dRe A, dL/dIm A, dL/dr0, dL/da (None unless wrt_a) and
    the adjoint of the initial state (dL/dRe u_0 + i dL/dIm u_0).
    spin = "analytic" contracts the spin term inside the adjoint steps;
    "fd" takes it as central differences of forward steps at a +- eps_a."""
    import torch
    op = fw.op
    # grad_h (autograd produces it on the caller's stream) is read by kernels
    # on the context's stream: order them after the work that wrote it
    caller = torch.cuda.current_stream(op.st.device)
    op.st.stream.wait_stream(caller)
    if torch.is_tensor(grad_h) and grad_h.is_cuda:
        grad_h.record_stream(op.st.stream)
    with torch.cuda.stream(op.st.stream):
        out = _sweep(fw, grad_h, wrt_a, eps_a, spin)
    caller.wait_stream(op.st.stream)
    return out


def gradients(w: inputs.Workload, prm: Params, nsteps: int, grad_h, u0=None, precision: str = "fp64",
              every: int | None = None, wrt_a: bool = True, eps_a: float | None = None, device=None,
              spin: str = "analytic", tape: bool = False):
    """forward() followed by backward(); returns backward's dictionary plus
    the waveform under "h"."""
    fw = forward(w, prm, nsteps, u0, precision, every, device, tape=tape)
    try:
        out = backward(fw, grad_h, wrt_a, eps_a, spin)
        out["h"] = fw.h
        return out
    finally:
        fw.close()


def _sweep(fw: Forward, grad_h, wrt_a, eps_a, spin="analytic"):
    import torch
    op, nsteps, ck = fw.op, fw.nsteps, fw.ck
    w, prm, precision = op.w, op.prm, op.precision
    g = torch.as_tensor(grad_h).to(device=op.st.device, dtype=torch.complex128).contiguous()
    if g.numel() != nsteps + 1:
        raise ValueError("grad_h needs one entry per sample h_0..h_N")
    if spin not in ("analytic", "fd"):
        raise ValueError("spin must be 'analytic' or 'fd'")
    analytic = wrt_a and spin == "analytic"
    if analytic and fw.last is None:
        raise ValueError("the forward run kept no last state")
    if fw.tape is not None and wrt_a and not analytic:
        raise ValueError("a taped forward run keeps no checkpoints: use spin='analytic'")
    if wrt_a and not analytic:
        eps = eps_a if eps_a is not None else (1e-4 if precision == "fp64" else 1e-3)
        dev = op.st.device
        opp = Operator(w, Params(prm.amp, prm.r0, prm.a + eps), precision, device=dev, stream=op.st.stream)
        opm = Operator(w, Params(prm.amp, prm.r0, prm.a - eps), precision, device=dev, stream=op.st.stream)
        dots = torch.zeros(nsteps + 1, dtype=torch.complex128, device=dev)
        samp = torch.zeros((nsteps + 1, 2), dtype=torch.complex128, device=dev)
        tp, tm = op.empty(), op.empty()
    op.ws[:8].zero_()   # the accumulators (the tail holds the coefficient planes)
    lam, lam2 = op.zeros(), op.empty()
    # lam_N from the last sample alone (lam_{N+1} = 0)
    if analytic:
        op.adjoint_spin(lam, lam2, fw.last, nsteps, nsteps == 0, _ptr(g, nsteps))
    else:
        op.adjoint(lam, lam2, nsteps, nsteps == 0, _ptr(g, nsteps))
    lam, lam2 = lam2, lam
    if fw.tape is not None and (analytic or not wrt_a):
        # the tape holds every step's stage values: nothing to recompute
        for n in range(nsteps - 1, -1, -1):
            if analytic:
                op.adjoint_tape(lam, lam2, fw.tape.data_ptr() + n * op.tape_bytes, n, n == 0, _ptr(g, n))
            else:
                op.adjoint(lam, lam2, n, n == 0, _ptr(g, n))
            lam, lam2 = lam2, lam
        ck = {}
    elif not wrt_a:
        # the adjoint of the linear step reads no state: no recompute either
        for n in range(nsteps - 1, -1, -1):
            op.adjoint(lam, lam2, n, n == 0, _ptr(g, n))
            lam, lam2 = lam2, lam
        ck = {}
    bounds = sorted(k for k in ck) + [nsteps] if ck else []
    for a, b in reversed(list(zip(bounds[:-1], bounds[1:]))):
        # states s_a .. s_b of this segment (s_0 is the physical u_0); the
        # adjoint steps n = b-1 .. a read s_n, so with the contracted spin
        # terms s_b is not needed (a checkpoint every step recomputes nothing)
        states = [ck[a]]
        last = b - 1 if analytic else b
        for n in range(a, last):
            nxt = op.empty()
            op.step(states[-1], nxt, n, n == 0)
            states.append(nxt)
        if wrt_a and not analytic:
            # a-derivative of the samples h_n, n in (a, b]
            for n in range(max(a + 1, 1), b + 1):
                opp.sample(states[n - a], False, _ptr(samp, 2 * n))
                opm.sample(states[n - a], False, _ptr(samp, 2 * n + 1))
        for n in range(b - 1, a - 1, -1):
            sn = states[n - a]
            if analytic:
                op.adjoint_spin(lam, lam2, sn, n, n == 0, _ptr(g, n))
            else:
                if wrt_a:
                    # <lam_{n+1}, (M_n(a + e) - M_n(a - e)) s_n>
                    opp.step(sn, tp, n, n == 0)
                    opm.step(sn, tm, n, n == 0)
                    op.dot(lam, tp, _ptr(dots, n), z=tm)
                op.adjoint(lam, lam2, n, n == 0, _ptr(g, n))
            lam, lam2 = lam2, lam
        del states
    acc = op.ws[:8].cpu().numpy()
    out = {"dA_re": float(acc[0]), "dA_im": float(-acc[1]), "dr0": float(acc[2]), "du0": lam.clone()}
    if analytic:
        out["da"] = float(acc[4])
    elif wrt_a:
        d = dots.cpu().numpy()
        sp = samp.cpu().numpy()
        gn = g.cpu().numpy()
        step_term = np.sum(d[:nsteps].real)
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
        op.st.stream.wait_stream(torch.cuda.current_stream(op.st.device))
        with torch.cuda.stream(op.st.stream):
            h, _, _ = run_forward(op, nsteps, u0)
        op.st.synchronize()
        return h
    finally:
        op.close()


def _make_function():
    import torch

    class WaveformFunction(torch.autograd.Function):
        """h = waveform(A, r0, a) at the extraction node; params is a float64
        tensor (Re A, Im A, r0, a).  The forward pass keeps sqrt(N)
        checkpoints; the backward pass sweeps the adjoint over them."""

        @staticmethod
        def forward(ctx, params, w, nsteps, precision):
            p = params.detach().cpu().numpy().astype(np.float64)
            prm = Params(complex(p[0], p[1]), float(p[2]), float(p[3]))
            ctx.device = params.device
            ctx.fw = forward(w, prm, int(nsteps), precision=precision)
            ctx.fw.op.st.synchronize()
            return ctx.fw.h.to(params.device)

        @staticmethod
        def backward(ctx, grad_h):
            try:
                r = backward(ctx.fw, grad_h)
            finally:
                ctx.fw.close()
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
