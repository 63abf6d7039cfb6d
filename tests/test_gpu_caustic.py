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


def test_caustic_full_size_blend(rtw):
    """The ellipsoid workload at full size (4e6 rays, orders 0..5, 512 x 1024 directions, default
    widths and tiles, as the benchmark times it), checked by properties that hold at any size: the
    field of every order is (1 - s) F_rays + s F_PO with F_rays the plain field (rtw_field) and F_PO
    the field of a call whose widths give every direction s = 1 (the same tiles and cones), within
    the single-precision terms' 1e-6 of the largest component; s lies in [0, 1]; the caustic bit is
    left only where order 0 (not corrected) put it."""
    import math

    from paper_2403_13856_gb300 import workloads as W

    spec, cfg = W.ELLIPSOID, W.ELLIPSOID_GRID
    p_max, nt, nph = cfg["p_max"], cfg["n_theta"], cfg["n_phi"]
    nd = nt * nph
    g = rtw.Object([rtw.ObjectSpec(**spec, jones=(1.0, 0.0))])
    rays = rtw.rtw_trace(g, rtw.trace_params(grid=rtw.RTW_GRID_SQUARE, p_max=p_max, n_rays=cfg["n_rays"],
                                             flags=rtw.RTW_TRACE_APERTURE))
    d = rtw.dirs_grid(nt, nph)
    per = rtw.RTW_FIELD_PER_ORDER
    plain = torch.zeros((nd, p_max + 1, 2), dtype=torch.complex128, device="cuda")
    pm = torch.zeros(nd, dtype=torch.uint8, device="cuda")
    rtw.rtw_field(rays, d, plain, pm, flags=per)
    blend = torch.zeros_like(plain)
    bm = torch.zeros_like(pm)
    w = torch.zeros((nd, p_max + 1), dtype=torch.float64, device="cuda")
    rtw.rtw_field_caustic(rays, d, rtw.caustic_params(), blend, bm, w, flags=per)
    L = max(spec["a"], spec["b"], spec["c"])
    aw = (spec["wavelength"] / L) ** (2.0 / 3.0)
    fw = 1.0 / math.sqrt(2.0 * math.pi / spec["wavelength"] * L)
    full = rtw.caustic_params(po=(3.5, 3.6), cone=(3 * aw + 3 * fw, 3 * aw + 6 * fw))
    po = torch.zeros_like(plain)
    w1 = torch.zeros_like(w)
    rtw.rtw_field_caustic(rays, d, full, po, None, w1, flags=per)
    rtw.rtw_sync_status()
    corrected = (w > 0).any(0)  # the orders with caustic directions
    assert bool(corrected[1:].any()) and not bool(corrected[0])
    for p in range(1, p_max + 1):
        if corrected[p]:
            assert bool((w1[:, p] == 1.0).all())
    assert bool((w >= 0).all()) and bool((w <= 1).all())
    s = w[..., None]
    want = (1.0 - s) * plain + s * po
    want[:, ~corrected] = plain[:, ~corrected]
    scale = plain.abs().max().item()
    err = (blend - want).abs().max().item()
    print(f"full size: corrected (direction, order) pairs {int((w > 0).sum().item())}, "
          f"max |blend - (1 - s) F_rays - s F_PO| / max |F| = {err / scale:.2e}")
    assert err <= 1e-6 * scale
    # masks: the PO bit where a weight is positive; the caustic bit only where the plain field had
    # it and no corrected order removed it (order 0 keeps its own)
    assert bool(((bm & 4) != 0).eq((w > 0).any(1)).all())
    assert bool((((bm & 1) != 0) <= ((pm & 1) != 0)).all())
    assert ((bm & 1) != 0).float().mean().item() < ((pm & 1) != 0).float().mean().item()
