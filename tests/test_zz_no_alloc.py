"""rtw_fan_field_static: the fan path for callers that may not allocate device memory.

It must give the same far field as rtw_create_object + rtw_trace + rtw_field on the same fan,
call after call (its fixed scratch array keeps the previous call's contents, so stale data would
show up on the second call), and refuse sizes beyond its limits.  This file is collected last so a
run that stops at the first failure has run every other test before it.
"""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rtw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_13856_gb300 import build, rtw as R

    build.build()
    L = R.lib()
    L.rtw_fan_field_static.argtypes = [ctypes.c_void_p] * 8
    L.rtw_fan_field_static.restype = ctypes.c_int
    return R


def structs(rtw, spec, jones):
    d = rtw.rtw_object_desc()
    d.a, d.b, d.c = spec["a"], spec["b"], spec["c"]
    d.quat[:] = list(spec["quat"])
    d.center[:] = list(spec.get("center", (0.0, 0.0, 0.0)))
    d.m_re, d.m_im = spec["m"], 0.0
    w = rtw.rtw_incident()
    w.wavelength_um = spec["wavelength"]
    w.dir[:] = [0.0, 0.0, 1.0]
    j = [complex(x) for x in jones]
    w.jones_re[:] = [j[0].real, j[1].real]
    w.jones_im[:] = [j[0].imag, j[1].imag]
    return d, w


def static_call(rtw, spec, jones, tp, dirs, flags, with_mask=True):
    d, w = structs(rtw, spec, jones)
    nd = dirs.n_theta
    nout = tp.p_max + 1 if flags & rtw.RTW_FIELD_PER_ORDER else 1
    out = torch.full((nd, nout, 2), complex(7.0, 7.0), dtype=torch.complex128, device="cuda")
    mask = torch.full((nd,), 255, dtype=torch.uint8, device="cuda")
    rc = rtw.lib().rtw_fan_field_static(ctypes.addressof(d), ctypes.addressof(w), ctypes.addressof(tp),
                                        ctypes.addressof(dirs), flags, out.data_ptr(),
                                        mask.data_ptr() if with_mask else None,
                                        torch.cuda.current_stream().cuda_stream)
    assert rc == 0, rtw.lib().rtw_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy(), (mask.cpu().numpy() if with_mask else None)


def allocating_call(rtw, spec, jones, tp, dirs, flags):
    obj = rtw.Object([rtw.ObjectSpec(**spec, jones=jones)])  # ObjectSpec takes the centre too
    rays = rtw.rtw_trace(obj, tp)
    nd = dirs.n_theta
    nout = tp.p_max + 1 if flags & rtw.RTW_FIELD_PER_ORDER else 1
    out = torch.zeros((nd, nout, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(nd, dtype=torch.uint8, device="cuda")
    rtw.rtw_field(rays, dirs, out, mask, flags=flags)
    rtw.rtw_sync_status()
    return out.cpu().numpy(), mask.cpu().numpy()


def test_static_matches_allocating_path_twice(rtw):
    sphere = dict(a=10.0, b=10.0, c=10.0, quat=(1.0, 0.0, 0.0, 0.0), m=1.333, wavelength=0.6328)
    drop = dict(a=9.0, b=11.0, c=7.5, quat=(1.0, 0.0, 0.0, 0.0), m=1.55, wavelength=0.5)
    # turned about an oblique axis, off the origin
    tilted = dict(a=12.0, b=9.5, c=8.0, quat=(0.9, 0.25, -0.3, 0.15), center=(3.0, -2.0, 5.0), m=1.45,
                  wavelength=0.55)
    qn = math.sqrt(sum(q * q for q in tilted["quat"]))
    tilted["quat"] = tuple(q / qn for q in tilted["quat"])
    calls = [
        (sphere, (0.0, 1.0), rtw.trace_params(grid=rtw.RTW_GRID_FAN, p_max=3, n_rays=10000),
         rtw.dirs_plane(1801, 0.0, math.radians(0.1)), rtw.RTW_FIELD_PER_ORDER, True),
        (drop, (0.3, 0.9), rtw.trace_params(grid=rtw.RTW_GRID_FAN, p_max=4, n_rays=6001, fan_phi=0.4),
         rtw.dirs_plane(997, -math.pi + 0.001, 2 * math.pi / 997), 0, True),
        (tilted, (0.6, 0.8j), rtw.trace_params(grid=rtw.RTW_GRID_FAN, p_max=3, n_rays=8000, fan_phi=-1.1),
         rtw.dirs_plane(1200, -math.pi + 0.002, 2 * math.pi / 1200), rtw.RTW_FIELD_PER_ORDER, False),
    ]
    for spec, jones, tp, dirs, flags, with_mask in calls:  # calls in a row share the scratch array
        got, gm = static_call(rtw, spec, jones, tp, dirs, flags, with_mask)
        ref, rm = allocating_call(rtw, spec, jones, tp, dirs, flags)
        scale = np.abs(ref).max()
        assert scale > 0
        # the same kernels on the same inputs: only the order of the atomic sums may differ
        assert np.abs(got - ref).max() <= 1e-12 * scale
        if with_mask:
            assert np.array_equal(gm, rm)


def test_static_rejects_sizes_beyond_its_limit(rtw):
    sphere = dict(a=10.0, b=10.0, c=10.0, quat=(1.0, 0.0, 0.0, 0.0), m=1.333, wavelength=0.6328)
    d, w = structs(rtw, sphere, (1.0, 0.0))
    tp = rtw.trace_params(grid=rtw.RTW_GRID_FAN, p_max=3, n_rays=20000)  # 80000 ray-orders > 65536
    dirs = rtw.dirs_plane(181, 0.0, math.radians(1.0))
    out = torch.zeros((181, 1, 2), dtype=torch.complex128, device="cuda")
    rc = rtw.lib().rtw_fan_field_static(ctypes.addressof(d), ctypes.addressof(w), ctypes.addressof(tp),
                                        ctypes.addressof(dirs), 0, out.data_ptr(), None, None)
    assert rc == -4
    assert b"65536" in rtw.lib().rtw_last_error()
