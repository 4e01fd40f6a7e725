"""One grid stepped as r* slabs with halo rows (slabs.SlabStepper, the
virtual-slab form of the single-instance decomposition on one GPU) against
the same grid stepped whole.

The grid's r* nodes are exact binary fractions (r* in [-64, 64], dr* = 1/2),
so every slab context builds bit for bit the coefficients, pivots, source
patch and extraction node of the whole grid at the same r*, and the owned
rows of the slabs must equal the whole grid's rows bit for bit: state and
waveform, with two or three halo rows (one or two steps between exchanges),
with a source crossing a slab edge, over an odd number of steps (a short
last chunk).
"""
import numpy as np
import pytest

from paper_0909_4039_gb300 import inputs

pytestmark = pytest.mark.gpu


def _kw(precision, Nr=257, Ntheta=32):
    return dict(s=-2, m=2, a=0.9, Nr=Nr, Ntheta=Ntheta, rstar_min=-64.0, rstar_max=64.0, dt=0.25,
                rstar_extract=40.0, precision=precision, wave_capacity=128)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("nslabs,halo", [(3, 2), (3, 3), (2, 3), (5, 3)])
def test_slabs_equal_whole_grid_bitwise(precision, nslabs, halo):
    from paper_0909_4039_gb300 import slabs, teuk
    steps = 41
    kw = _kw(precision)
    u0 = inputs.random_state(kw["Nr"], kw["Ntheta"], seed=9)
    # source near r* = 16 (r0 = 12 at a = 0.9), a patch of about +-18 rows that
    # crosses the edge between the second and third of three slabs (row 171)
    src = (0.8 - 0.3j, 12.0, 2.0, 0.3)
    whole = teuk.Stepper(**kw)
    whole.set_source(*src)
    whole.set_state(u0, 0)
    whole.step(steps)
    ref_u, ref_h = whole.get_state(), whole.waveform(0, steps + 1)
    whole.close()

    sl = slabs.SlabStepper(nslabs, halo, **kw)
    sl.set_source(*src)
    sl.set_state(u0, 0)
    sl.step(steps)
    assert sl.current_step == steps
    got_u, got_h = sl.get_state(), sl.waveform(0, steps + 1)
    sl.close()
    assert np.array_equal(got_u, ref_u), float(np.abs(got_u - ref_u).max())
    assert np.array_equal(got_h, ref_h)


def test_slab_contexts_see_the_whole_grid_rstar():
    """Each slab's r* range is the whole grid's rows g0 .. g0+rows-1."""
    from paper_0909_4039_gb300 import slabs
    kw = _kw("fp64")
    sl = slabs.SlabStepper(3, 3, **kw)
    for g, st in zip(sl.geoms, sl.slabs):
        assert st.Nr == g.rows
        assert st.desc.rstar_min == -64.0 + 0.5 * g.g0
        assert st.desc.rstar_max == -64.0 + 0.5 * (g.g0 + g.rows - 1)
    i_ext = int(round((40.0 + 64.0) / 0.5))
    assert sl.geoms[sl.owner].a <= i_ext < sl.geoms[sl.owner].b
    sl.close()


def test_state_level_offset_and_shifted_flag():
    """teuk_state_level: the level flips with every step launch, the state is
    physical after set_state and shifted after a split step, and rows
    written through the view are what the next step reads."""
    from paper_0909_4039_gb300 import teuk
    kw = _kw("fp64", Nr=65)
    st = teuk.Stepper(**kw)
    u0 = inputs.random_state(65, 32, seed=3)
    import torch
    st.set_state(u0, 0)
    st.synchronize()
    off0, nb, shifted = teuk.teuk_state_level(st.ctx)
    assert not shifted and nb == 2 * 65 * 32 * 16 and off0 in (0, nb)
    v, _ = st.level_view()
    assert np.array_equal(v.cpu().numpy(), u0)          # the physical state, in place
    st.step(1)
    off1, _, shifted = teuk.teuk_state_level(st.ctx)
    assert shifted and off1 != off0
    # a zeroed level stays zero under the (linear, source-free) step; the
    # writes are ordered after the step's stream and before the next step
    st.synchronize()
    v, _ = st.level_view()
    v.zero_()
    torch.cuda.synchronize()
    st.step(3)
    assert np.abs(st.get_state()).max() == 0.0
    st.close()
