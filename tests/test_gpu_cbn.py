"""The paper's final occupancy network, CBN + SoftZ (Appendix, Eq. 7 and
Eq. 8), through the C ABI against the FP64 oracle: the field at ragged batch
sizes, the coarse-to-fine localization and the render, at the plain FP32
parity bar (occupancy <= 1e-4; sets, volumes and counts identical unless an
oracle value lies within 1e-4 of 0.5), and the forms a CBN context refuses."""
import numpy as np
import pytest

from oracle import field, localize, render
from paper_2007_13988_gb300 import pifu, synth

from gpu_common import COLOUR_TOL, DEPTH_TOL, OCC_TOL, Ctx, ambiguous_rays, compare_volume

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    c = Ctx(synth.tiny_cbn(0))
    yield c
    c.close()


@pytest.fixture(scope="module")
def full():
    c = Ctx(synth.full_cbn(0))
    yield c
    c.close()


def occ_oracle(w, P, calib=None):
    return field.occupancy(w.occ_net, w.occ_map, w.calib if calib is None else calib, P)


@pytest.mark.parametrize("m", [1, 31, 33, 4099])
def test_cbn_query_tiny_ragged(tiny, m):
    P = synth.query_points(m, seed=20 + m)
    got = tiny.query(P)
    assert np.max(np.abs(got - occ_oracle(tiny.w, P))) <= OCC_TOL


def test_cbn_query_full_near_surface_and_yaw(full):
    w = full.w
    P = synth.distill_points(w.fig, 6000, 21)
    got = full.query(P)
    want = occ_oracle(w, P)
    err = np.abs(got - want)
    print("CBN full query: max %.2e, points within 0.1 of 0.5: %d"
          % (err.max(), int(np.sum(np.abs(want - 0.5) < 0.1))))
    assert err.max() <= OCC_TOL
    cal = synth.calib_yaw(30.0)
    P = synth.query_points(3000, seed=22)
    assert np.max(np.abs(full.query(P, calib=cal) - occ_oracle(w, P, cal))) <= OCC_TOL


def test_cbn_query_depth_outside_unit_range(tiny):
    # a 30-degree yaw sends corners of the volume past |P_z| = 1, where SoftZ
    # clamps (reading of Eq. 7's domain)
    cal = synth.calib_yaw(30.0, scale=1.3)
    P = synth.query_points(2000, seed=23)
    z = field.project(cal, P)[2]
    assert np.any(np.abs(z) > 1.0)
    assert np.max(np.abs(tiny.query(P, calib=cal) - occ_oracle(tiny.w, P, cal))) <= OCC_TOL


@pytest.fixture(scope="module")
def tiny_levels(tiny):
    w = tiny.w
    return localize.hierarchical(lambda P: occ_oracle(w, P), w.n0, w.num_levels)


def test_cbn_localize_tiny(tiny, tiny_levels):
    vol = tiny.localize()
    b, e, v = tiny.volume_host(vol)
    res = compare_volume(b, e, v, tiny_levels, vol)
    print("CBN tiny localization:", res)


def test_cbn_localize_full_128(full):
    w = full.w
    lv = localize.hierarchical(lambda P: occ_oracle(w, P), 32, 3)
    vol = full.localize(n0=32, levels=3)
    b, e, v = full.volume_host(vol)
    res = compare_volume(b, e, v, lv, vol)
    print("CBN full 32^3 -> 128^3:", res)


def test_cbn_render_tiny(tiny, tiny_levels):
    w = tiny.w
    tiny.localize()
    fine = tiny_levels[-1]
    R = 64
    o_rgb, o_depth, o_hit = render.render(fine.values, R, w.col_net, w.occ_map, w.col_map, w.calib)
    depth, rgb, mask = tiny.render(R)
    ok = ~ambiguous_rays(fine.values, R)
    assert np.array_equal(mask[ok], o_hit[ok])
    hit = ok & o_hit
    assert hit.sum() > 0
    assert np.max(np.abs(depth[hit] - o_depth[hit])) <= DEPTH_TOL
    assert np.max(np.abs(rgb[ok] - o_rgb[ok])) <= COLOUR_TOL


def test_cbn_refused_forms(tiny):
    import torch
    w = tiny.w
    for prec in (pifu.PIFU_PREC_FP8, pifu.PIFU_PREC_FP8_MIXED):
        with pytest.raises(pifu.PifuError) as ei:
            tiny.localize(precision=prec)
        assert ei.value.status == pifu.PIFU_ERR_UNSUPPORTED
    with pytest.raises(pifu.PifuError) as ei:
        pifu.pifu_calibrate_fp8(tiny.ctx, tiny.occ, w.calib, w.n0)
    assert ei.value.status == pifu.PIFU_ERR_UNSUPPORTED
    d = torch.empty((64, 64), dtype=torch.float32, device="cuda")
    rgb = torch.empty((64, 64, 3), dtype=torch.float32, device="cuda")
    m = torch.empty((64, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(pifu.PifuError) as ei:
        pifu.pifu_frame(tiny.ctx, tiny.occ, tiny.col, w.calib, w.n0, w.num_levels, 64, 64, d, rgb,
                        m, precision=pifu.PIFU_PREC_MIXED)
    assert ei.value.status == pifu.PIFU_ERR_UNSUPPORTED
