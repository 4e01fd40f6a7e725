"""CPU-side checks of the C ABI: the library loads, exports every function
include/teuk.h declares, and its host-side validation returns the documented
status codes without touching a GPU (no compute call is made here)."""
import ctypes
import os
import re

import pytest

from paper_0909_4039_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    from paper_0909_4039_gb300 import teuk
    return teuk


def _declared():
    src = open(os.path.join(ROOT, "include", "teuk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(teuk_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("teuk_init_grid", "teuk_set_source", "teuk_step", "teuk_extract_waveform"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    L = lib.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert sorted(lib.EXPORTED) == _declared()


def test_status_strings(lib):
    L = lib.lib()
    for code, name in [(0, b"TEUK_OK"), (1, b"TEUK_E_INVAL"), (4, b"TEUK_E_UNSTABLE"), (7, b"TEUK_E_RANGE")]:
        assert L.teuk_status_string(code) == name


def _desc(lib, **kw):
    base = dict(s=-2, m=2, a=0.9, Nr=1024, Ntheta=32, rstar_min=-100.0, rstar_max=600.0)
    base.update(kw)
    return lib.make_desc(**base)


def test_workspace_sizes(lib):
    sb, cb, wb = lib.teuk_workspace_bytes(_desc(lib, precision=lib.TEUK_FP64))
    assert sb == 2 * 2 * 1024 * 32 * 16
    assert wb == 16 * 33
    sb32, cb32, _ = lib.teuk_workspace_bytes(_desc(lib, precision=lib.TEUK_FP32))
    assert sb32 == sb // 2
    assert cb > 0 and cb32 > 0


@pytest.mark.parametrize("bad", [dict(Nr=2), dict(Ntheta=0), dict(Ntheta=4096), dict(a=1.0), dict(a=-1.2),
                                 dict(rstar_max=-200.0), dict(s=3), dict(M=0.0), dict(precision=7),
                                 dict(scheme=9), dict(dt=float("nan"))])
def test_invalid_descriptors(lib, bad):
    with pytest.raises(lib.TeukError) as e:
        lib.teuk_workspace_bytes(_desc(lib, **bad))
    assert e.value.code == lib.TEUK_E_INVAL


def test_init_rejects_bad_buffers_before_any_device_call(lib):
    d = _desc(lib)
    with pytest.raises(lib.TeukError) as e:
        lib.teuk_init_grid(d, 0, 0, 0, 16)
    assert e.value.code == lib.TEUK_E_INVAL
    with pytest.raises(lib.TeukError) as e:
        lib.teuk_init_grid(d, 0x1000, 0x2001, 0x3000, 16)      # misaligned; never dereferenced
    assert e.value.code == lib.TEUK_E_INVAL


def test_courant_guard(lib):
    # dt = 1.2 dr*: radial Courant number above 1
    d = _desc(lib, dt=1.2 * 700.0 / 1023)
    with pytest.raises(lib.TeukError) as e:
        lib.teuk_init_grid(d, 0x1000, 0x2000, 0x3000, 16)
    assert e.value.code == lib.TEUK_E_UNSTABLE


def test_literal_scheme_guard(lib):
    """The literal reading of Eqs. 12-14 is refused at dt = dr*/2 (it grows
    every step); the check is host arithmetic, no device call."""
    d = _desc(lib, scheme=lib.TEUK_SCHEME_LITERAL)
    with pytest.raises(lib.TeukError) as e:
        lib.teuk_init_grid(d, 0x1000, 0x2000, 0x3000, 16)
    assert e.value.code == lib.TEUK_E_UNSTABLE
    assert "literal" in str(e.value)


def test_null_context_calls(lib):
    L = lib.lib()
    assert L.teuk_step(None, 1, None) == lib.TEUK_E_STATE
    assert L.teuk_set_source(None, 1.0, 0.0, 10.0, 0.1, 0.1, float("nan")) == lib.TEUK_E_STATE
    assert L.teuk_destroy(None) == lib.TEUK_OK
    assert L.teuk_current_step(None) == -1
