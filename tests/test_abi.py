"""The C ABI library loads, exports every function include/rtw.h declares, and validates its
arguments on the host.  No compute call is made, so these run without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def librtw():
    from paper_2403_13856_gb300 import build, rtw

    build.build()
    return rtw


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rtw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rtw_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("rtw_create_object", "rtw_trace", "rtw_field", "rtw_destroy_object", "rtw_destroy_rays",
                 "rtw_status_string", "rtw_sync_status"):
        assert must in names


def test_every_declared_symbol_is_exported(librtw):
    L = librtw.lib()
    for name in declared_functions():
        assert hasattr(L, name), name


def test_status_strings(librtw):
    L = librtw.lib()
    assert L.rtw_status_string(0) == b"ok"
    assert L.rtw_status_string(-1) == b"invalid argument"
    assert L.rtw_status_string(-99) == b"unknown status"
    assert b"sm_103a" in L.rtw_version()


def _desc(rtw, **kw):
    d = rtw.rtw_object_desc()
    d.a, d.b, d.c = kw.get("a", 10.0), 10.0, 10.0
    d.quat[:] = kw.get("quat", [1.0, 0.0, 0.0, 0.0])
    d.center[:] = [0.0, 0.0, 0.0]
    d.m_re, d.m_im = kw.get("m", 1.333), kw.get("m_im", 0.0)
    w = rtw.rtw_incident()
    w.wavelength_um = kw.get("lam", 0.6328)
    w.dir[:] = kw.get("dir", [0.0, 0.0, 1.0])
    w.jones_re[:] = [1.0, 0.0]
    w.jones_im[:] = [0.0, 0.0]
    return d, w


@pytest.mark.parametrize("kw,code", [
    (dict(a=-1.0), -1), (dict(quat=[1.0, 0.1, 0.0, 0.0]), -1), (dict(m=1.0), -1), (dict(m=-2.0), -1),
    (dict(lam=0.0), -1), (dict(m_im=0.01), -2), (dict(dir=[0.0, 1.0, 0.0]), -2),
])
def test_create_object_validation(librtw, kw, code):
    """Invalid descriptors are rejected before any device is touched."""
    L = librtw.lib()
    d, w = _desc(librtw, **kw)
    h = ctypes.c_void_p()
    rc = L.rtw_create_object(ctypes.byref(d), 1, ctypes.byref(w), ctypes.byref(h))
    assert rc == code
    assert L.rtw_last_error()
    assert not h.value


def test_null_arguments(librtw):
    L = librtw.lib()
    assert L.rtw_create_object(None, 1, None, None) == -1
    assert L.rtw_trace(None, None, None, None) == -1
    assert L.rtw_field(None, None, 0, 0, None, None, None) == -1
    assert L.rtw_rays_info(None, None, None, None) == -1
    assert L.rtw_far_field_batch(None, None, None, 0, None, None, None, None) == -1
    assert L.rtw_field_caustic(None, None, None, 0, None, None, None, None) == -1
    assert L.rtw_batch_info(None, None, None, None) == -1
    assert L.rtw_batch_times(None, None, None) == -1
    L.rtw_destroy_batch(None)


def test_no_cpu_fallback_without_device(librtw):
    """Without a CUDA device a valid object cannot be created: the library reports a CUDA error
    instead of computing anything on the host."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = librtw.lib()
    d, w = _desc(librtw)
    h = ctypes.c_void_p()
    assert L.rtw_create_object(ctypes.byref(d), 1, ctypes.byref(w), ctypes.byref(h)) == -3


def test_python_binding_fails_loudly_when_library_missing(monkeypatch):
    from paper_2403_13856_gb300 import rtw

    monkeypatch.setattr(rtw, "_lib", None)
    monkeypatch.setattr(rtw, "LIB_PATH", "/nonexistent/librtw.so")
    with pytest.raises(rtw.RTWError):
        rtw.lib()
