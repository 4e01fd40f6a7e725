"""Failure detection without a GPU fault: a bounded device wait that runs out.

The tiled step kernels wait on mbarriers for the bulk copies of their state
tiles, and every wait is bounded.  teuk_set_wait_limit shortens the bound of
a tile's waits on its state copy; with 0 rounds the wait gives up at once,
while the copies are legitimately in flight.  The tile then records the
timeout in the context's control block, waits (with the default bound) for
its own copies to land, and returns without writing its rows.  No kernel
traps, faults or hangs: nothing waits on anything that is not already on its
way.

Checked here, through the C ABI: the timeout reaches the host as
TEUK_E_TIMEOUT from teuk_extract_waveform; the context stays usable; after
teuk_set_state (which clears the flags) a run with the default bound equals
an undisturbed run bit for bit, state and waveform.
"""
import numpy as np
import pytest

from paper_0909_4039_gb300 import inputs
from tests._common import gpu_stepper

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_wait_that_runs_out_reports_timeout_and_context_recovers(precision):
    from paper_0909_4039_gb300 import teuk
    w = inputs.Workload("timeout", s=-2, m=2, a=0.9, Nr=300, Ntheta=32, rs_min=-60.0, rs_max=140.0, steps=12,
                        r0=8.0, amp=1.0, sig_r=0.8, sig_th=0.3, rs_ext=100.0)
    u0 = inputs.random_state(w.Nr, w.Ntheta, seed=41)

    ref = gpu_stepper(w, precision)
    ref.set_state(u0, 0)
    ref.step(w.steps)
    s_ref = ref.get_state()
    h_ref = ref.waveform(1, w.steps)
    ref.close()

    st = gpu_stepper(w, precision)
    assert not st.tiling()["persistent"]
    teuk.teuk_set_wait_limit(st.ctx, 0)
    st.set_state(u0, 0)
    st.step(3)
    with pytest.raises(teuk.TeukError) as e:
        st.waveform(1, 3)
    assert e.value.code == teuk.TEUK_E_TIMEOUT
    assert "did not complete" in str(e.value)

    # the flag stays until a new run starts
    with pytest.raises(teuk.TeukError) as e2:
        st.waveform(1, 1)
    assert e2.value.code == teuk.TEUK_E_TIMEOUT

    teuk.teuk_set_wait_limit(st.ctx, -1)
    st.set_state(u0, 0)
    st.step(w.steps)
    s = st.get_state()
    h = st.waveform(1, w.steps)
    st.close()
    assert np.array_equal(s, s_ref)
    assert np.array_equal(h, h_ref)
