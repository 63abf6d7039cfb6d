"""Physical optics at the 3-D caustics of a square-grid field on the GPU (rtw_field_caustic) against the
oracle's or_field_grid_caustic on the same rays and directions.

Weights agree to 1e-9 and masks exactly.  Fields: the ray sum (weight 0) within the FP64 path's 1e-6 of
the largest component; where a weight is above 0 the aperture integral adds single-precision terms --
each term w U dA rounded to FP32 (relative 6e-8), its phase within a 16 x 16 ray block taken in FP32
and reduced to [-pi, pi] before one FP32 sincos (a few 1e-7 rad), and at most 256 of them summed in
FP32 before the FP64 accumulation -- so its error is bounded by a small multiple of 1e-6 of the sum of
the terms' magnitudes, which the oracle reports per direction and order (l1):
    |F_gpu - F_oracle| <= 1e-6 max |F| + 2e-5 l1.
Cases: the sphere's rainbow (the case the oracle pins by the fan's PO and Table 1) and a tilted
ellipsoid with four orders; the summed-order output; argument checks.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

M_WATER = 1.333
LAM = 0.6328


@pytest.fixture(scope="module")
def rtw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_13856_gb300 import build, rtw as R

    build.build()
    R.lib()
    return R


def caustic_gpu(rtw, spec, jones, h, p_max, nt, nph, tile, per_order=True, flags_trace=None):
    g = rtw.Object([rtw.ObjectSpec(**spec, jones=jones)])
    tp = rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, spacing=h,
                          flags=rtw.RTW_TRACE_APERTURE if flags_trace is None else flags_trace)
    rays = rtw.rtw_trace(g, tp)
    nd, npo = nt * nph, p_max + 1
    out = torch.zeros((nd, npo if per_order else 1, 2), dtype=torch.complex128, device="cuda")
    mask = torch.zeros(nd, dtype=torch.uint8, device="cuda")
    w = torch.zeros((nd, npo), dtype=torch.float64, device="cuda")
    rtw.rtw_field_caustic(rays, rtw.dirs_grid(nt, nph), rtw.caustic_params(tile=tile), out, mask, w,
                          flags=rtw.RTW_FIELD_PER_ORDER if per_order else 0)
    rtw.rtw_sync_status()
    return out.cpu().numpy(), mask.cpu().numpy(), w.cpu().numpy(), rays


def compare(oracle_mod, o, got, gmask, gw, nt, nph, p_max, tile, h):
    ref, rmask, rw, corders, l1, hits = o.field_grid_caustic(p_max, nt, nph, tile=tile, h=h)
    F = oracle_mod.complex_field(ref.reshape(-1, 4)).reshape(nt * nph, p_max + 1, 2)
    assert np.abs(gw - rw).max() <= 1e-9
    assert np.array_equal(gmask, rmask)
    scale = np.abs(F).max()
    err = np.abs(got - F).max(-1)
    bound = 1e-6 * scale + 2e-5 * l1
    worst = np.max((err - 1e-6 * scale) / np.maximum(l1, 1e-300), initial=0.0)
    print(f"corrected (direction, order) pairs {int((rw > 0).sum())}; max |dF| / max |F| = {err.max() / scale:.2e}; "
          f"max excess / l1 = {worst:.2e}")
    assert np.all(err <= bound)
    assert (rw > 0).any() and ((corders >> 1) != 0).any()
    return ref, rmask, rw


def test_caustic_sphere_rainbow_matches_oracle(rtw, oracle_mod):
    a, h, nt, nph, tile = 50.0, 0.2, 360, 31, (8, 2)
    spec = dict(a=a, b=a, c=a, quat=(1.0, 0.0, 0.0, 0.0), m=M_WATER, wavelength=LAM)
    got, gmask, gw, _ = caustic_gpu(rtw, spec, (0.0, 1.0), h, 2, nt, nph, tile)
    o = oracle_mod.Object(a, a, a, m=M_WATER, wavelength=LAM, jones=(0.0, 1.0))
    compare(oracle_mod, o, got, gmask, gw, nt, nph, 2, tile, h)


def test_caustic_tilted_ellipsoid_matches_oracle(rtw, oracle_mod):
    h, nt, nph, tile = 0.12, 90, 60, (8, 4)
    quat = (0.9, 0.25, -0.3, 0.15)
    qn = math.sqrt(sum(q * q for q in quat))
    quat = tuple(q / qn for q in quat)
    spec = dict(a=14.0, b=11.0, c=9.0, quat=quat, m=M_WATER, wavelength=LAM)
    got, gmask, gw, _ = caustic_gpu(rtw, spec, (0.6, 0.8j), h, 3, nt, nph, tile)
    o = oracle_mod.Object(14.0, 11.0, 9.0, quat=quat, m=M_WATER, wavelength=LAM, jones=(0.6, 0.8j))
    compare(oracle_mod, o, got, gmask, gw, nt, nph, 3, tile, h)


def test_caustic_summed_orders(rtw):
    a, h, nt, nph, tile = 20.0, 0.15, 120, 41, (8, 4)
    spec = dict(a=a, b=0.9 * a, c=0.8 * a, quat=(1.0, 0.0, 0.0, 0.0), m=M_WATER, wavelength=LAM)
    per, pm, pw, _ = caustic_gpu(rtw, spec, (1.0, 0.0), h, 3, nt, nph, tile)
    tot, tm, tw, _ = caustic_gpu(rtw, spec, (1.0, 0.0), h, 3, nt, nph, tile, per_order=False)
    assert np.array_equal(pm, tm) and np.array_equal(pw, tw)
    assert np.abs(tot[:, 0] - per.sum(1)).max() <= 1e-12 * np.abs(per).max()


def test_caustic_arguments(rtw):
    spec = dict(a=10.0, b=10.0, c=10.0, quat=(1.0, 0.0, 0.0, 0.0), m=M_WATER, wavelength=LAM)
    g = rtw.Object([rtw.ObjectSpec(**spec, jones=(1.0, 0.0))])
    plain = rtw.rtw_trace(g, rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=2, spacing=0.5))
    ap = rtw.rtw_trace(g, rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=2, spacing=0.5,
                                           flags=rtw.RTW_TRACE_APERTURE))
    nt, nph = 30, 20
    out = torch.zeros((nt * nph, 3, 2), dtype=torch.complex128, device="cuda")
    d = rtw.dirs_grid(nt, nph)
    with pytest.raises(rtw.RTWError):  # no aperture records
        rtw.rtw_field_caustic(plain, d, rtw.caustic_params(), out, flags=rtw.RTW_FIELD_PER_ORDER)
    for cp in (rtw.caustic_params(tile=(20, 20)), rtw.caustic_params(tile=(-1, 4)),
               rtw.caustic_params(po=(0.2, 0.1)), rtw.caustic_params(cone=(1.0, 1.6)),
               rtw.caustic_params(p_min=4)):
        with pytest.raises(rtw.RTWError):
            rtw.rtw_field_caustic(ap, d, cp, out, flags=rtw.RTW_FIELD_PER_ORDER)
    with pytest.raises(rtw.RTWError):  # windows are not taken
        rtw.rtw_field_caustic(ap, rtw.dirs_grid(nt, nph, (0, 10, 0, 10)), rtw.caustic_params(), out,
                              flags=rtw.RTW_FIELD_PER_ORDER)
    with pytest.raises(rtw.RTWError):  # 16 x 16 tiles of this coarse grid: a cone reaches pi/2
        rtw.rtw_field_caustic(ap, d, rtw.caustic_params(), out, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_field_caustic(ap, d, rtw.caustic_params(tile=(4, 2)), out, flags=rtw.RTW_FIELD_PER_ORDER)
    rtw.rtw_sync_status()
