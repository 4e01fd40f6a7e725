"""Adjoint (transposed) stepper and waveform-loss gradients.

Pins, none of which uses the adjoint to check itself:
  * dot-product identities <y, M x> = <M^H y, x> for one step (regular and
    first), for the sample operator E C_{dt/2}, and for the whole map from
    the initial state to the waveform, to 1e-13 relative in FP64;
  * gradients of L = sum_n dt |h_n - target_n|^2 with respect to the source
    amplitude (Re A, Im A), the orbit radius r0 and the spin a against
    central finite differences of L computed by independent forward runs,
    on the GPU and with the FP64 oracle;
  * the torch.autograd.Function gives the same gradient as the sweep;
  * the adjoint workload (4096 x 64, a = 0.7, 8000 steps, low-passed noise
    target) at full size against central differences.
"""
import time

import numpy as np
import pytest

from paper_0909_4039_gb300 import inputs
from tests._common import oracle_problem, rel_l2

pytestmark = pytest.mark.gpu


def _w(Nr=90, Nth=16, a=0.7, m=2, steps=0, amp=0.0, r0=7.0, sig_r=0.6, sig_th=0.3):
    return inputs.Workload("adj", s=-2, m=m, a=a, Nr=Nr, Ntheta=Nth, rs_min=-40.0, rs_max=120.0, steps=steps,
                           r0=r0, amp=amp, sig_r=sig_r, sig_th=sig_th, rs_ext=80.0)


def _rand(shape, seed, device, dtype, zero_boundary=False):
    import torch
    u = inputs.random_state(shape[1], shape[2], seed=seed, zero_boundary=zero_boundary)
    return torch.as_tensor(u).to(device=device, dtype=dtype)


def _cdot(op, x, y):
    import torch
    out = torch.zeros(1, dtype=torch.complex128, device=x.device)
    op.dot(x, y, out.data_ptr())
    op.st.synchronize()
    return complex(out.item())


@pytest.mark.parametrize("Nr,Nth,m,first", [(90, 16, 2, False), (90, 16, 2, True), (70, 33, 3, False),
                                             (64, 128, 1, False), (50, 64, 4, True)])
def test_one_step_dot_product(Nr, Nth, m, first):
    """<y, M_n x> = <M_n^H y, x> with the source off (M_n linear)."""
    import torch
    from paper_0909_4039_gb300 import adjoint as A
    op = A.Operator(_w(Nr, Nth, m=m), A.Params(0.0, 7.0, 0.7), "fp64")
    with torch.cuda.stream(op.st.stream):
        x = _rand(op.shape, 1, op.st.device, op.ctype)
        y = _rand(op.shape, 2, op.st.device, op.ctype)
        Mx, MHy = op.empty(), op.empty()
        op.step(x, Mx, 5, first)
        op.adjoint(y, MHy, 5, first, None)
        lhs, rhs = _cdot(op, y, Mx), _cdot(op, MHy, x)
    scale = float(torch.linalg.vector_norm(y).item() * torch.linalg.vector_norm(Mx).item())
    assert abs(lhs - rhs) <= 1e-13 * scale, (lhs, rhs, scale)
    op.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("Nr,Nth,first", [(90, 16, False), (90, 16, True), (70, 33, False), (300, 64, False)])
def test_step_with_sample_equals_step_then_sample(Nr, Nth, first, precision):
    """teuk_apply_step_sample gives, bit for bit, the state of
    teuk_apply_step and the sample teuk_apply_sample takes of it."""
    import torch
    from paper_0909_4039_gb300 import adjoint as A
    op = A.Operator(_w(Nr, Nth, amp=0.4 + 0.2j), A.Params(0.4 + 0.2j, 7.0, 0.7), precision)
    with torch.cuda.stream(op.st.stream):
        x = _rand(op.shape, 4, op.st.device, op.ctype, zero_boundary=True)
        a, b = op.empty(), op.empty()
        h = torch.zeros(2, dtype=torch.complex128, device=op.st.device)
        op.step(x, a, 7, first)
        op.sample(a, False, h.data_ptr())
        op.step_sample(x, b, 7, first, h.data_ptr() + 16)
        op.st.synchronize()
    assert torch.equal(a, b)
    assert h[0].item() == h[1].item() and h[0].item() != 0
    op.close()


def test_sample_dot_product():
    """<g, E C_{dt/2} x> = <C_{dt/2}^H E^H g, x>: the adjoint step with a
    zero incoming adjoint returns the sample's adjoint."""
    import torch
    from paper_0909_4039_gb300 import adjoint as A
    op = A.Operator(_w(80, 32, m=2), A.Params(0.0, 7.0, 0.5), "fp64")
    with torch.cuda.stream(op.st.stream):
        x = _rand(op.shape, 3, op.st.device, op.ctype)
        h = torch.zeros(1, dtype=torch.complex128, device=op.st.device)
        g = torch.tensor([0.3 - 1.7j], dtype=torch.complex128, device=op.st.device)
        op.sample(x, False, h.data_ptr())
        lam = op.empty()
        op.adjoint(op.zeros(), lam, 9, False, g.data_ptr())
        lhs = complex(np.conj(g.item()) * h.item())
        rhs = _cdot(op, lam, x)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs), (lhs, rhs)
    op.close()


def test_whole_map_dot_product_initial_state():
    """G maps u_0 to (h_0..h_N) with the source off: <g, G u_0> equals
    <G^H g, u_0> where G^H g is the backward sweep's adjoint of u_0."""
    import torch
    from paper_0909_4039_gb300 import adjoint as A
    w = _w(100, 16, m=2)
    N = 60
    u0 = inputs.random_state(w.Nr, w.Ntheta, seed=11)
    prm = A.Params(0.0, 7.0, 0.7)
    h = A.waveform(w, prm, N, u0=u0).cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(5))
    g = rng.standard_normal(N + 1) + 1j * rng.standard_normal(N + 1)
    r = A.gradients(w, prm, N, torch.as_tensor(g), u0=u0, wrt_a=False, every=7)
    lhs = np.vdot(g, h)
    rhs = np.vdot(r["du0"].cpu().numpy().ravel(), u0.ravel())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs), (lhs, rhs)


def _loss(h, target, dt):
    return float(dt * np.sum(np.abs(h - target) ** 2))


def _fd_gradients(loss_of, prm, rel=1e-6):
    """Central differences of the loss in (Re A, Im A, r0, a).  L is
    quadratic in A, so its differences are exact there for any step."""
    from paper_0909_4039_gb300 import adjoint as A
    out = []
    for k, (name, h) in enumerate([("Ar", 1e-3), ("Ai", 1e-3), ("r0", rel * prm.r0), ("a", rel * max(prm.a, 0.1))]):
        def shifted(d):
            amp, r0, a = prm.amp, prm.r0, prm.a
            if k == 0:
                amp = amp + d
            elif k == 1:
                amp = amp + 1j * d
            elif k == 2:
                r0 = r0 + d
            else:
                a = a + d
            return loss_of(A.Params(amp, r0, a))
        out.append((shifted(h) - shifted(-h)) / (2 * h))
    return np.array(out)


def test_source_and_spin_gradients_against_gpu_differences():
    import torch
    from paper_0909_4039_gb300 import adjoint as A
    w = _w(220, 16, a=0.6, m=2, sig_r=0.8)
    N = 300
    dt = 0.5 * (w.rs_max - w.rs_min) / (w.Nr - 1)
    prm = A.Params(0.7 - 0.2j, 7.0, 0.6)
    target = 1e-3 * inputs.adjoint_target(N + 1, dt, seed=3)
    h = A.waveform(w, prm, N).cpu().numpy()
    r = A.gradients(w, prm, N, torch.as_tensor(2.0 * dt * (h - target)))
    got = np.array([r["dA_re"], r["dA_im"], r["dr0"], r["da"]])
    fd = _fd_gradients(lambda q: _loss(A.waveform(w, q, N).cpu().numpy(), target, dt), prm)
    assert np.all(np.abs(got - fd) <= 1e-6 * np.abs(fd) + 1e-12 * np.abs(fd).max()), (got, fd)


def test_gradients_against_oracle_differences():
    """The FP64 oracle's loss, differenced in each parameter, against the
    GPU adjoint gradient (small grid)."""
    import torch
    from oracle import oracle as O
    from paper_0909_4039_gb300 import adjoint as A
    w = _w(140, 8, a=0.5, m=2, sig_r=0.8)
    N = 160
    dt = 0.5 * (w.rs_max - w.rs_min) / (w.Nr - 1)
    prm = A.Params(0.9 + 0.4j, 6.5, 0.5)
    target = 1e-3 * inputs.adjoint_target(N + 1, dt, seed=4)
    h = A.waveform(w, prm, N).cpu().numpy()
    r = A.gradients(w, prm, N, torch.as_tensor(2.0 * dt * (h - target)))
    got = np.array([r["dA_re"], r["dA_im"], r["dr0"], r["da"]])

    def oracle_loss(q):
        wq = w.with_(a=q.a, r0=q.r0, amp=q.amp)
        _, ho = O.run(oracle_problem(wq), None, N)
        return _loss(ho, target, dt)

    fd = _fd_gradients(oracle_loss, prm)
    assert np.all(np.abs(got - fd) <= 1e-6 * np.abs(fd) + 1e-12 * np.abs(fd).max()), (got, fd)
    # the waveforms themselves agree at the FP64 parity tolerance
    _, ho = O.run(oracle_problem(w.with_(a=prm.a, r0=prm.r0, amp=prm.amp)), None, N)
    assert rel_l2(h, ho) <= 1e-12


def test_autograd_function_matches_sweep():
    import torch
    from paper_0909_4039_gb300 import adjoint as A
    w = _w(120, 16, a=0.4, m=2, sig_r=0.8)
    N = 90
    dt = 0.5 * (w.rs_max - w.rs_min) / (w.Nr - 1)
    target = torch.as_tensor(1e-3 * inputs.adjoint_target(N + 1, dt, seed=6), device="cuda")
    params = torch.tensor([0.5, -0.3, 8.0, 0.4], dtype=torch.float64, device="cuda", requires_grad=True)
    h = A.waveform_fn(params, w, N)
    loss = dt * torch.sum(torch.abs(h - target) ** 2)
    loss.backward()
    hn = h.detach().cpu().numpy()
    r = A.gradients(w, A.Params(0.5 - 0.3j, 8.0, 0.4), N, torch.as_tensor(2.0 * dt * (hn - target.cpu().numpy())))
    ref = np.array([r["dA_re"], r["dA_im"], r["dr0"], r["da"]])
    assert np.allclose(params.grad.cpu().numpy(), ref, rtol=1e-12, atol=0.0)


def test_adjoint_workload_4096x64_full_size():
    """The adjoint workload: 4096 x 64, a = 0.7, orbit r0 = 10, 8000 steps,
    target = low-passed complex noise (seed 1, |omega| < 0.5/M).  Gradient
    with respect to (Re A, Im A, r0, a) against central differences of GPU
    forward runs; prints the adjoint cost in forward-run units."""
    import torch
    from paper_0909_4039_gb300 import adjoint as A
    w = inputs.ADJOINT_4096x64
    N = w.steps
    dt = 0.5 * (w.rs_max - w.rs_min) / (w.Nr - 1)
    prm = A.Params(complex(w.amp), w.r0, w.a)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = A.waveform(w, prm, N).cpu().numpy()
    t_fwd = time.perf_counter() - t0
    scale = np.abs(h).max()
    target = scale * inputs.adjoint_target(N + 1, dt, seed=1)
    t0 = time.perf_counter()
    r = A.gradients(w, prm, N, torch.as_tensor(2.0 * dt * (h - target)))
    t_adj = time.perf_counter() - t0
    got = np.array([r["dA_re"], r["dA_im"], r["dr0"], r["da"]])
    fd = _fd_gradients(lambda q: _loss(A.waveform(w, q, N).cpu().numpy(), target, dt), prm)
    print(f"\nadjoint 4096x64x8000: grad {got}, central differences {fd}, "
          f"forward {t_fwd:.2f} s, gradient sweep {t_adj:.2f} s ({t_adj / t_fwd:.2f} forward runs)")
    assert np.all(np.abs(got - fd) <= 1e-5 * np.abs(fd) + 1e-10 * np.abs(fd).max()), (got, fd)


@pytest.mark.parametrize("first,m,Nth", [(False, 2, 16), (True, 2, 16), (False, 3, 33), (False, 1, 64)])
def test_one_step_spin_term_against_step_differences(first, m, Nth):
    """The spin term of one adjoint step, Re <lam, dM_n/da s> (+ the sample's
    Re <g, d(E C_{dt/2})/da s>), contracted inside teuk_adjoint_step_spin from
    the coefficient derivatives, against central differences of the step
    and sample operators at a +- e (independent forward evaluations), with
    the source on; FP64.  Also: the step's lam_n and source accumulators
    equal those of teuk_adjoint_step."""
    import torch
    from paper_0909_4039_gb300 import adjoint as A
    w = _w(110, Nth, a=0.6, m=m, sig_r=0.8)
    prm = A.Params(0.8 - 0.5j, 6.0, 0.6)
    n = 0 if first else 17
    eps = 1e-5
    op = A.Operator(w, prm, "fp64")
    opp = A.Operator(w, A.Params(prm.amp, prm.r0, prm.a + eps), "fp64", stream=op.st.stream)
    opm = A.Operator(w, A.Params(prm.amp, prm.r0, prm.a - eps), "fp64", stream=op.st.stream)
    with torch.cuda.stream(op.st.stream):
        s = _rand(op.shape, 21, op.st.device, op.ctype, zero_boundary=True)
        lam = _rand(op.shape, 22, op.st.device, op.ctype)
        g = torch.tensor([1.1 - 0.6j], dtype=torch.complex128, device=op.st.device)
        tp, tm = op.empty(), op.empty()
        opp.step(s, tp, n, first)
        opm.step(s, tm, n, first)
        fd = (_cdot(op, lam, tp) - _cdot(op, lam, tm)).real / (2 * eps)
        if not first:
            hp = torch.zeros(1, dtype=torch.complex128, device=op.st.device)
            hm = torch.zeros(1, dtype=torch.complex128, device=op.st.device)
            opp.sample(s, False, hp.data_ptr())
            opm.sample(s, False, hm.data_ptr())
            op.st.synchronize()
            fd += (np.conj(g.item()) * (hp.item() - hm.item())).real / (2 * eps)
        op.ws[:8].zero_()
        out_s = op.empty()
        op.adjoint_spin(lam, out_s, s, n, first, g.data_ptr())
        acc_s = op.ws[:8].clone()
        op.ws[:8].zero_()
        out_r = op.empty()
        op.adjoint(lam, out_r, n, first, g.data_ptr())
        acc_r = op.ws[:8].clone()
        op.st.synchronize()
    got = float(acc_s[4].item())
    assert abs(got - fd) <= 1e-7 * abs(fd) + 1e-12, (got, fd)
    assert rel_l2(out_s.cpu().numpy(), out_r.cpu().numpy()) <= 1e-13
    assert np.allclose(acc_s[:4].cpu().numpy(), acc_r[:4].cpu().numpy(), rtol=1e-12, atol=1e-300)
    for o in (op, opp, opm):
        o.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("first,m,Nth", [(False, 2, 16), (True, 2, 16), (False, 3, 33), (False, 1, 64)])
def test_tape_step_and_adjoint_equal_recompute(first, m, Nth, precision):
    """teuk_apply_step_tape gives the state and sample of
    teuk_apply_step_sample bit for bit, records the input's extraction row,
    and teuk_adjoint_step_tape reading that record gives, bit for bit, the
    lam_n and accumulators teuk_adjoint_step_spin gets by recomputing the
    stage values from s_n."""
    import torch
    from paper_0909_4039_gb300 import adjoint as A
    w = _w(150, Nth, a=0.6, m=m, sig_r=0.8)
    prm = A.Params(0.8 - 0.5j, 6.0, 0.6)
    n = 0 if first else 17
    op = A.Operator(w, prm, precision)
    with torch.cuda.stream(op.st.stream):
        s = _rand(op.shape, 31, op.st.device, op.ctype, zero_boundary=True)
        lam = _rand(op.shape, 32, op.st.device, op.ctype)
        g = torch.tensor([0.7 + 1.3j], dtype=torch.complex128, device=op.st.device)
        a, b = op.empty(), op.empty()
        h = torch.zeros(2, dtype=torch.complex128, device=op.st.device)
        tape = torch.full((op.tape_bytes // 8,), float("nan"), dtype=torch.float64, device=op.st.device)
        op.step_sample(s, a, n, first, h.data_ptr())
        op.step_tape(s, b, n, first, h.data_ptr() + 16, tape.data_ptr())
        op.ws[:8].zero_()
        out_s = op.empty()
        op.adjoint_spin(lam, out_s, s, n, first, g.data_ptr())
        acc_s = op.ws[:8].clone()
        op.ws[:8].zero_()
        out_t = op.empty()
        op.adjoint_tape(lam, out_t, tape.data_ptr(), n, first, g.data_ptr())
        acc_t = op.ws[:8].clone()
        op.st.synchronize()
    assert torch.equal(a, b) and h[0].item() == h[1].item()
    # the record: U1 and U2 of every row (finite, written), then the input's extraction row
    rec = tape.view(op.ctype)
    pl = 2 * w.Nr * w.Ntheta
    assert torch.isfinite(torch.view_as_real(rec[:2 * pl])).all()
    ie = int(round((w.rs_ext - w.rs_min) / ((w.rs_max - w.rs_min) / (w.Nr - 1))))   # the node nearest r*_ext
    xrow = rec[2 * pl:2 * pl + 2 * w.Ntheta].reshape(2, w.Ntheta)
    assert torch.equal(xrow, s[:, ie, :])
    assert torch.equal(out_s, out_t)
    assert torch.equal(acc_s, acc_t)
    op.close()


def test_taped_gradient_equals_checkpointed_gradient():
    """The whole gradient with the forward tape (store-all, no recompute)
    equals the sqrt(N)-checkpointed gradient, and the source-only sweep
    (no state needed) equals the source parts of the full one."""
    import torch
    from paper_0909_4039_gb300 import adjoint as A
    w = _w(200, 16, a=0.6, m=2, sig_r=0.8)
    N = 120
    dt = 0.5 * (w.rs_max - w.rs_min) / (w.Nr - 1)
    prm = A.Params(0.7 - 0.2j, 7.0, 0.6)
    target = 1e-3 * inputs.adjoint_target(N + 1, dt, seed=3)
    h = A.waveform(w, prm, N).cpu().numpy()
    gh = torch.as_tensor(2.0 * dt * (h - target))
    r_ck = A.gradients(w, prm, N, gh, every=11)
    r_tp = A.gradients(w, prm, N, gh, tape=True)
    r_src = A.gradients(w, prm, N, gh, wrt_a=False, every=11)
    for k in ("dA_re", "dA_im", "dr0", "da"):
        assert r_ck[k] == r_tp[k], (k, r_ck[k], r_tp[k])
    for k in ("dA_re", "dA_im", "dr0"):
        assert abs(r_src[k] - r_ck[k]) <= 1e-11 * abs(r_ck[k]), (k, r_src[k], r_ck[k])
    assert torch.equal(r_ck["du0"], r_tp["du0"])
    assert torch.equal(r_ck["h"], r_tp["h"])


def test_analytic_spin_gradient_matches_step_differences_sweep():
    """The whole sweep: dL/da from the contracted spin terms against the
    sweep that takes them as central differences of forward steps (FP64)."""
    import torch
    from paper_0909_4039_gb300 import adjoint as A
    w = _w(160, 16, a=0.55, m=2, sig_r=0.8)
    N = 120
    dt = 0.5 * (w.rs_max - w.rs_min) / (w.Nr - 1)
    prm = A.Params(0.6 + 0.2j, 7.5, 0.55)
    target = 1e-3 * inputs.adjoint_target(N + 1, dt, seed=9)
    h = A.waveform(w, prm, N).cpu().numpy()
    gh = torch.as_tensor(2.0 * dt * (h - target))
    ra = A.gradients(w, prm, N, gh, every=11)
    rf = A.gradients(w, prm, N, gh, every=11, spin="fd", eps_a=1e-5)
    assert abs(ra["da"] - rf["da"]) <= 1e-7 * abs(rf["da"]), (ra["da"], rf["da"])
    for k in ("dA_re", "dA_im", "dr0"):
        assert abs(ra[k] - rf[k]) <= 1e-11 * abs(rf[k]) + 1e-300, (k, ra[k], rf[k])


def test_adjoint_workload_grid_against_oracle_window():
    """The adjoint workload's grid (4096 x 64, a = 0.7, orbit r0 = 10, the
    sqrt(N) checkpointed sweep) over a window of 1000 steps: the gradient
    with respect to (Re A, Im A, r0, a) against central differences of the
    FP64 oracle's loss (independent code), each parameter shifted by 1e-6
    relative (1e-3 for A, where the loss is quadratic).  The waveform is
    taken at r* = 60M, which the signal reaches within the window (at 500M,
    1000 steps from zero data give a zero waveform and zero gradients)."""
    import torch
    from oracle import oracle as O
    from paper_0909_4039_gb300 import adjoint as A
    w = inputs.ADJOINT_4096x64.with_(rs_ext=60.0)
    N = 1000
    dt = 0.5 * (w.rs_max - w.rs_min) / (w.Nr - 1)
    prm = A.Params(complex(w.amp), w.r0, w.a)
    h = A.waveform(w, prm, N).cpu().numpy()
    target = (np.abs(h).max() + 1e-30) * inputs.adjoint_target(N + 1, dt, seed=1)
    r = A.gradients(w, prm, N, torch.as_tensor(2.0 * dt * (h - target)))
    got = np.array([r["dA_re"], r["dA_im"], r["dr0"], r["da"]])

    def oracle_loss(q):
        wq = w.with_(a=q.a, r0=q.r0, amp=q.amp)
        _, ho = O.run(oracle_problem(wq), None, N)
        return _loss(ho, target, dt)

    fd = _fd_gradients(oracle_loss, prm)
    print(f"\nadjoint 4096x64, 1000 steps: GPU {got}, oracle differences {fd}")
    assert np.all(np.abs(fd) > 0.0)
    assert np.all(np.abs(got - fd) <= 1e-6 * np.abs(fd) + 1e-12 * np.abs(fd).max()), (got, fd)


def test_fp32_gradient_of_the_adjoint_workload():
    """The FP32-state path's gradient on the full adjoint workload (4096 x 64,
    8000 steps, spin term contracted in the adjoint steps) against the FP64
    gradient, which the tests above pin to the oracle.  Measured: 5e-5 (Re A),
    2e-4 (Im A), 2e-5 (r0), 3e-5 (a); the spin term taken as central
    differences of FP32 forward steps instead was off by 2e-2."""
    import torch
    from paper_0909_4039_gb300 import adjoint as A
    w = inputs.ADJOINT_4096x64
    N = w.steps
    dt = 0.5 * (w.rs_max - w.rs_min) / (w.Nr - 1)
    prm = A.Params(complex(w.amp), w.r0, w.a)
    h = A.waveform(w, prm, N).cpu().numpy()
    target = np.abs(h).max() * inputs.adjoint_target(N + 1, dt, seed=1)
    r64 = A.gradients(w, prm, N, torch.as_tensor(2.0 * dt * (h - target)))
    h32 = A.waveform(w, prm, N, precision="fp32").cpu().numpy()
    r32 = A.gradients(w, prm, N, torch.as_tensor(2.0 * dt * (h32 - target)), precision="fp32")
    g64 = np.array([r64["dA_re"], r64["dA_im"], r64["dr0"], r64["da"]])
    g32 = np.array([r32["dA_re"], r32["dA_im"], r32["dr0"], r32["da"]])
    err = np.abs(g32 - g64) / np.abs(g64)
    print(f"\nFP32 gradient relative errors (Re A, Im A, r0, a): {err}")
    assert np.all(err < 2e-3), err
    assert err[3] < 1e-3, err


def test_adjoint_entry_points_reject_bad_calls():
    """Error paths of the spin adjoint and the taped step: another workspace
    than the prepared one, a missing sample address, an unaligned tape."""
    import ctypes
    import torch
    from paper_0909_4039_gb300 import adjoint as A
    from paper_0909_4039_gb300 import teuk
    L = teuk.lib()
    op = A.Operator(_w(60, 16), A.Params(0.3, 7.0, 0.5), "fp64")
    with torch.cuda.stream(op.st.stream):
        s, t, lam, lam2 = op.zeros(), op.zeros(), op.zeros(), op.zeros()
        other = torch.zeros_like(op.ws)
        rc = L.teuk_adjoint_step_spin(op.st.ctx, lam.data_ptr(), lam2.data_ptr(), s.data_ptr(), 3, 0, None,
                                      other.data_ptr(), op.sh)
        assert rc == 6   # TEUK_E_STATE: the workspace was not prepared
        rc = L.teuk_apply_step_sample(op.st.ctx, s.data_ptr(), t.data_ptr(), 3, 0, None, op.sh)
        assert rc == 1   # TEUK_E_INVAL: no sample address
        tape = torch.zeros(op.tape_bytes // 8 + 64, dtype=torch.float64, device=op.st.device)
        h = torch.zeros(1, dtype=torch.complex128, device=op.st.device)
        rc = L.teuk_apply_step_tape(op.st.ctx, s.data_ptr(), t.data_ptr(), 3, 0, h.data_ptr(),
                                    tape.data_ptr() + 8, op.sh)
        assert rc == 1   # TEUK_E_INVAL: unaligned tape
        size = ctypes.c_size_t()
        assert L.teuk_tape_bytes(op.st.ctx, ctypes.byref(size)) == 0 and size.value % 256 == 0
        assert size.value >= 16 * (4 * 60 * 16 + 2 * 16)
        # the prepared workspace works
        op.adjoint_spin(lam, lam2, s, 3, False, None)
        op.st.synchronize()
    op.close()
