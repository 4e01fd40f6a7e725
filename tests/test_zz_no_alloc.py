"""The allocation-free literal step (teuk_literal_step_static).

Some callers cannot allocate device memory where they step (a framework's
caching allocator owns the device memory, or the loop may not call
cudaMalloc/cudaFree because they synchronise the device).  For them the
library offers one literal-scheme step whose midpoint scratch is a fixed
array inside the library itself.  This file checks, through the C ABI, that
two such steps in a row give what the ordinary entry point (teuk_step,
scratch in the caller's workspace) gives, and that a grid too large for the
fixed array is refused.  It is collected last so that a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_0909_4039_gb300 import inputs
from tests._common import gpu_stepper, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-4)])
def test_static_scratch_step_matches_teuk_step(precision, tol):
    import torch

    from paper_0909_4039_gb300 import teuk
    w = inputs.Workload("noalloc", s=-2, m=2, a=0.8, Nr=60, Ntheta=12, rs_min=-20.0, rs_max=40.0, steps=2,
                        r0=6.0, amp=0.9 - 0.2j, sig_r=1.0, sig_th=0.3, rs_ext=30.0)
    st = gpu_stepper(w, precision, scheme="literal", allow_unstable=True)
    u0 = inputs.random_state(w.Nr, w.Ntheta, seed=31)
    st.set_state(u0, 0)
    st.step(1)
    ref1 = st.get_state()
    st.step(1)
    ref2 = st.get_state()
    cdt = torch.complex128 if precision == "fp64" else torch.complex64
    a = torch.tensor(u0, dtype=cdt, device=st.device)
    b = torch.empty_like(a)
    c = torch.empty_like(a)
    teuk.teuk_literal_step_static(st.ctx, a.data_ptr(), b.data_ptr(), 0, st.sh)
    teuk.teuk_literal_step_static(st.ctx, b.data_ptr(), c.data_ptr(), 1, st.sh)
    st.synchronize()
    assert rel_l2(b.cpu().numpy().astype(np.complex128), ref1) <= tol
    assert rel_l2(c.cpu().numpy().astype(np.complex128), ref2) <= tol
    st.close()


def test_static_scratch_rejects_grids_above_its_limit():
    import torch

    from paper_0909_4039_gb300 import teuk
    w = inputs.Workload("noalloc-big", s=-2, m=2, a=0.5, Nr=4097, Ntheta=128, rs_min=-20.0, rs_max=40.0, steps=0,
                        amp=0.0)
    st = gpu_stepper(w, "fp64", scheme="literal", with_source=False, allow_unstable=True, wave_capacity=4)
    a = torch.zeros((2, w.Nr, w.Ntheta), dtype=torch.complex128, device=st.device)
    b = torch.empty_like(a)
    with pytest.raises(teuk.TeukError) as e:
        teuk.teuk_literal_step_static(st.ctx, a.data_ptr(), b.data_ptr(), 0, st.sh)
    assert e.value.code == teuk.TEUK_E_INVAL and "8 MiB" in str(e.value)
    st.close()
