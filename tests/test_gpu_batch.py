"""Batched instances (teuk_batch_*): uneven grids, spins, modes and sources
advanced together in one launch per step.

Each instance of a batch must compute exactly what it computes alone
(teuk_step): the batched kernel runs the same per-tile arithmetic with the
instance's own parameters, so states and waveforms are compared bit for bit
with single-instance runs, and small instances are compared with the FP64
oracle within the state precision's tolerance.  The full uneven batch of 64
instances (Nr in {2048..16384}, Ntheta in {32, 64, 128}) is checked on a
window of steps against single-instance runs of sampled instances.
"""
import numpy as np
import pytest

from paper_0909_4039_gb300 import inputs
from tests._common import gpu_stepper, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-4


def _mixed(precision="fp32"):
    spec = [
        # Nr, Ntheta, a, m, r0 (dr* <= 1 over r* in [-60, 240])
        (700, 128, 0.9, 2, 8.0),
        (341, 64, 0.3, 1, 7.0),
        (333, 32, 0.99, 4, 9.0),
        (1000, 16, 0.0, 3, 6.5),
        (457, 128, 0.7, 2, 12.0),
        (396, 64, 0.95, 4, 7.5),
    ]
    ws = []
    for k, (Nr, Nth, a, m, r0) in enumerate(spec):
        ws.append(inputs.Workload(f"mix{k}", s=-2, m=m, a=a, Nr=Nr, Ntheta=Nth, rs_min=-60.0, rs_max=240.0,
                                  steps=0, r0=r0, amp=0.8 - 0.2j * k, sig_r=0.9, sig_th=0.25, rs_ext=150.0))
    return ws


def _batch(steppers):
    from paper_0909_4039_gb300 import teuk
    return teuk.Batch(steppers)


@pytest.mark.parametrize("ks,nsteps", [(1, 130), (2, 130), (2, 41)])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_equals_instances_stepped_alone(precision, ks, nsteps):
    """Batched steps (first step, graph replays of 64 steps, a remainder;
    one or two steps per launch, an odd remainder as a one-step launch)
    give every instance the state and waveform it gets alone."""
    ws = _mixed()
    u0 = [inputs.random_state(w.Nr, w.Ntheta, seed=100 + k) for k, w in enumerate(ws)]
    alone = []
    for w, u in zip(ws, u0):
        st = gpu_stepper(w, precision, wave_capacity=nsteps + 1)
        st.set_state(u, 0)
        st.step(nsteps)
        alone.append((st.get_state(), st.waveform(0, nsteps + 1)))
        st.close()
    sts = [gpu_stepper(w, precision, wave_capacity=nsteps + 1) for w in ws]
    for st, u in zip(sts, u0):
        st.set_state(u, 0)
    b = _batch(sts)
    b.set_tiling(steps_per_launch=ks)
    assert b.tiling()["steps_per_launch"] == ks
    b.step(nsteps)
    b.synchronize()
    for k, st in enumerate(sts):
        assert st.current_step == nsteps
        u, h = st.get_state(), st.waveform(0, nsteps + 1)
        assert np.array_equal(u, alone[k][0]), (k, rel_l2(u, alone[k][0]))
        assert np.array_equal(h, alone[k][1]), k
    b.close()
    for st in sts:
        st.close()


@pytest.mark.parametrize("precision,tol", [("fp32", FP32_TOL), ("fp64", FP64_TOL)])
def test_batch_against_oracle(precision, tol):
    """Small instances of a batch against the FP64 oracle."""
    from oracle import oracle as O
    ws = [w for w in _mixed() if w.Nr <= 400]
    nsteps = 25
    u0 = [inputs.random_state(w.Nr, w.Ntheta, seed=7 + k) for k, w in enumerate(ws)]
    sts = [gpu_stepper(w, precision, wave_capacity=nsteps + 1) for w in ws]
    for st, u in zip(sts, u0):
        st.set_state(u, 0)
    b = _batch(sts)
    b.step(nsteps)
    b.synchronize()
    for w, st, u in zip(ws, sts, u0):
        uo, ho = O.run(oracle_problem(w), u, nsteps)
        assert rel_l2(st.get_state(), uo) <= tol, (w.name, rel_l2(st.get_state(), uo))
        assert rel_l2(st.waveform(0, nsteps + 1), ho) <= tol, w.name
    b.close()
    for st in sts:
        st.close()


def test_batch_mixed_first_steps_tiling_and_autotune():
    """Instances already stepped alone (shifted state) and fresh ones
    (physical state) start a batch together; tile heights set by hand and by
    the autotuner do not change the result."""
    ws = _mixed()
    u0 = [inputs.random_state(w.Nr, w.Ntheta, seed=300 + k) for k, w in enumerate(ws)]
    pre = [3 if k % 2 else 0 for k in range(len(ws))]
    results = []
    for mode in ("default", "manual", "manual-one-step", "autotune"):
        sts = [gpu_stepper(w, "fp32", wave_capacity=64) for w in ws]
        b = _batch(sts)
        assert b.tiling()["steps_per_launch"] == 2
        if mode.startswith("manual"):
            b.set_tiling([7 if w.Ntheta >= 64 else 30 for w in ws], 1 if mode.endswith("one-step") else None)
            assert b.tiling()["tile_rows"] == [7 if w.Ntheta >= 64 else 30 for w in ws]
        elif mode == "autotune":
            tr = b.autotune(3)
            assert all(t >= 1 for t in tr) and b.tiling()["steps_per_launch"] in (1, 2)
            for st in sts:
                assert st.current_step == 0 and np.abs(st.get_state()).max() == 0.0
        for st, u, k in zip(sts, u0, pre):
            st.set_state(u, 0)
            if k:
                st.step(k)          # before it is stepped through the batch
        b.step(20)
        b.synchronize()
        results.append([(st.current_step, st.get_state(), st.waveform(st.current_step - 20, 21)) for st in sts])
        b.close()
        for st in sts:
            st.close()
    for other in results[1:]:
        for (n0, u0_, h0), (n1, u1, h1) in zip(results[0], other):
            assert n0 == n1 and np.array_equal(u0_, u1) and np.array_equal(h0, h1)


def test_batch_rejects_incompatible_instances():
    from paper_0909_4039_gb300 import teuk
    w = inputs.Workload("rej", s=-2, m=2, a=0.5, Nr=100, Ntheta=32, rs_min=-50.0, rs_max=150.0, steps=0)
    a = gpu_stepper(w, "fp32", wave_capacity=8)
    b64 = gpu_stepper(w, "fp64", wave_capacity=8)
    wide = gpu_stepper(w.with_(Ntheta=200), "fp32", wave_capacity=8)
    lit = gpu_stepper(w, "fp32", scheme="literal", wave_capacity=8, allow_unstable=True)
    for group in ([a, b64], [a, wide], [a, lit], [a, a]):
        with pytest.raises(teuk.TeukError):
            teuk.Batch(group)
    b = teuk.Batch([a])
    before = b.tiling()
    for bad in ([0], [255]):
        with pytest.raises(teuk.TeukError):
            b.set_tiling(bad)
        assert b.tiling() == before
    b.set_tiling([31])
    assert b.tiling()["tile_rows"] == [31]
    for bad in (0, 3):
        with pytest.raises(teuk.TeukError):
            b.set_tiling(steps_per_launch=bad)
        assert b.tiling()["steps_per_launch"] == 2
    b.close()
    # Ntheta > 256: one step per launch only
    wider = gpu_stepper(w.with_(Ntheta=300), "fp32", wave_capacity=8)
    bw = teuk.Batch([wider])
    assert bw.tiling()["steps_per_launch"] == 1
    with pytest.raises(teuk.TeukError):
        bw.set_tiling(steps_per_launch=2)
    assert bw.tiling()["steps_per_launch"] == 1
    bw.close()
    for st in (a, b64, wide, lit, wider):
        st.close()


def test_uneven_batch_of_64_window():
    """The 64-instance uneven batch (seeded: a, m, r0, Nr, Ntheta drawn as
    stated in inputs.batched_instances) at full size: a window of batched
    steps from random states equals single-instance runs of sampled
    instances bit for bit, and the smallest sampled instance matches the
    oracle within the FP32 tolerance."""
    from oracle import oracle as O
    ws = inputs.batched_instances(64, seed=0, steps=12)
    nsteps = 12
    sts = [gpu_stepper(w, "fp32", wave_capacity=nsteps + 1) for w in ws]
    u0 = {}
    sample = sorted(range(64), key=lambda k: ws[k].points)[:2] + [int(np.argmax([w.points for w in ws])), 17, 42]
    for k, st in enumerate(sts):
        if k in sample:
            u0[k] = inputs.random_state(ws[k].Nr, ws[k].Ntheta, seed=1000 + k)
            st.set_state(u0[k], 0)
    b = _batch(sts)
    b.step(nsteps)
    b.synchronize()
    got = {k: (sts[k].get_state(), sts[k].waveform(0, nsteps + 1)) for k in sample}
    b.close()
    for st in sts:
        st.close()
    for k in sample:
        st = gpu_stepper(ws[k], "fp32", wave_capacity=nsteps + 1)
        st.set_state(u0[k], 0)
        st.step(nsteps)
        assert np.array_equal(st.get_state(), got[k][0]), k
        assert np.array_equal(st.waveform(0, nsteps + 1), got[k][1]), k
        st.close()
    k = sample[0]
    uo, ho = O.run(oracle_problem(ws[k]), u0[k], nsteps)
    assert rel_l2(got[k][0], uo) <= FP32_TOL
    assert rel_l2(got[k][1], ho) <= FP32_TOL


def test_batch_wide_theta_class():
    """Instances with 128 < Ntheta <= 256 (eight theta points per lane, the
    long-run workload's class) batch together and equal their solo runs."""
    ws = [inputs.Workload(f"wide{k}", s=-2, m=m, a=a, Nr=Nr, Ntheta=Nth, rs_min=-60.0, rs_max=240.0, steps=0,
                          r0=r0, amp=1.0 + 0.1j * k, sig_r=0.9, sig_th=0.2, rs_ext=150.0)
          for k, (Nr, Nth, a, m, r0) in enumerate([(400, 256, 0.999, 2, 5.0), (350, 200, 0.5, 3, 9.0),
                                                     (300, 136, 0.9, 1, 7.0)])]
    nsteps = 17
    u0 = [inputs.random_state(w.Nr, w.Ntheta, seed=50 + k) for k, w in enumerate(ws)]
    alone = []
    for w, u in zip(ws, u0):
        st = gpu_stepper(w, "fp32", wave_capacity=nsteps + 1)
        st.set_state(u, 0)
        st.step(nsteps)
        alone.append((st.get_state(), st.waveform(0, nsteps + 1)))
        st.close()
    sts = [gpu_stepper(w, "fp32", wave_capacity=nsteps + 1) for w in ws]
    for st, u in zip(sts, u0):
        st.set_state(u, 0)
    b = _batch(sts)
    b.step(nsteps)
    b.synchronize()
    for k, st in enumerate(sts):
        assert np.array_equal(st.get_state(), alone[k][0]), k
        assert np.array_equal(st.waveform(0, nsteps + 1), alone[k][1]), k
    b.close()
    for st in sts:
        st.close()


def test_long_run_batch_full_size_window():
    """The long-run workload at full size (65536 x 256, a = 0.999) in the
    batched launch configuration its eight-instance run uses (Ntheta = 256
    class, two steps per launch): two instances (r0 = 4 and 20) step
    together for seven steps.  The first starts from random data over every
    tile and is compared with the FP64 oracle within the FP32 tolerance; the
    second (zero data, its own source) equals its solo run bit for bit."""
    from oracle import oracle as O
    ws = inputs.long_run_batch(2)
    nsteps = 7
    u0 = inputs.random_state(ws[0].Nr, ws[0].Ntheta, seed=77)
    sts = [gpu_stepper(w, "fp32", wave_capacity=nsteps + 1) for w in ws]
    sts[0].set_state(u0, 0)
    b = _batch(sts)
    til = b.tiling()
    assert til["steps_per_launch"] == 2, til
    b.step(nsteps)
    b.synchronize()
    got = [(st.get_state(), st.waveform(0, nsteps + 1)) for st in sts]
    b.close()
    for st in sts:
        st.close()
    solo = gpu_stepper(ws[1], "fp32", wave_capacity=nsteps + 1)
    solo.step(nsteps)
    assert np.array_equal(solo.get_state(), got[1][0])
    assert np.array_equal(solo.waveform(0, nsteps + 1), got[1][1])
    solo.close()
    uo, ho = O.run(oracle_problem(ws[0]), u0, nsteps)
    assert rel_l2(got[0][0], uo) <= FP32_TOL, rel_l2(got[0][0], uo)
    assert rel_l2(got[0][1], ho) <= FP32_TOL, rel_l2(got[0][1], ho)
