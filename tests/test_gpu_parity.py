"""CUDA path (through the C ABI) against the FP64 oracle, element by element,
on seeded synthetic inputs: the field (Eq. 1, Eq. 2), the coarse-to-fine
localization (Sec. 3.2) and the mesh-free render (Eq. 3)."""
import numpy as np
import pytest

from oracle import field, localize, render
from paper_2007_13988_gb300 import synth

from gpu_common import (COLOUR_TOL, DEPTH_TOL, OCC_TOL, Ctx, ambiguous_rays, check_localization,
                        check_render, localized)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    c = Ctx(synth.tiny(0))
    yield c
    c.close()


@pytest.fixture(scope="module")
def full():
    c = Ctx(synth.full(0))
    yield c
    c.close()


def occ_oracle(w, P, calib=None):
    return field.occupancy(w.occ_net, w.occ_map, w.calib if calib is None else calib, P)


# ---------------------------------------------------------------- field ------

@pytest.mark.parametrize("m", [1, 7, 129, 4099, 65536 + 37])
def test_query_tiny_ragged_sizes(tiny, m):
    P = synth.query_points(m, seed=100 + m) * np.float32(1.2)   # some points outside the volume
    got = tiny.query(P)
    want = occ_oracle(tiny.w, P)
    assert np.max(np.abs(got - want)) <= OCC_TOL


def test_query_full_random_points(full):
    P = synth.query_points(3000, seed=7)
    got = full.query(P)
    want = occ_oracle(full.w, P)
    err = np.max(np.abs(got - want))
    assert err <= OCC_TOL, err


# FP32 batches of up to 2048 points run in one fused launch whose cluster
# size follows the batch (16-CTA clusters for one tile up to 2-CTA clusters
# for about 76 tiles and more): one batch per regime, ragged tails included.
@pytest.mark.parametrize("m", [16, 130, 300, 700, 1216, 2048])
def test_query_full_fused_cluster_sizes(full, m):
    P = synth.query_points(m, seed=300 + m)
    got = full.query(P)
    want = occ_oracle(full.w, P)
    err = np.max(np.abs(got - want))
    assert err <= OCC_TOL, err


def test_query_full_near_surface_points(full):
    # points on the finest grid next to the figure, where o changes fastest
    w = full.w
    c = localize.node_coords(256)
    rng = np.random.default_rng(3)
    k = rng.integers(0, 257, 20000)
    j = rng.integers(0, 257, 20000)
    i = rng.integers(0, 257, 20000)
    P = np.stack([c[i], c[j], c[k]], 1)
    o = occ_oracle(w, P)
    sel = np.abs(o - 0.5) < 0.45
    if sel.sum() < 50:
        sel[:50] = True
    P = P[sel][:2000].astype(np.float32)
    got = full.query(P)
    want = occ_oracle(w, P)
    assert np.max(np.abs(got - want)) <= OCC_TOL


def test_query_yaw_calibration(full):
    cal = synth.calib_yaw(30.0)
    P = synth.query_points(2000, seed=8)
    got = full.query(P, calib=cal)
    want = occ_oracle(full.w, P, calib=cal)
    assert np.max(np.abs(got - want)) <= OCC_TOL


def test_query_empty_is_noop(tiny):
    assert tiny.query(np.zeros((0, 3), np.float32)).shape == (0,)


@pytest.mark.parametrize("which", ["tiny", "full"])
def test_query_colour(which, tiny, full):
    c = tiny if which == "tiny" else full
    w = c.w
    P = synth.query_points(1500, seed=9)
    got = c.query_colour(P)
    want = field.colour(w.col_net, w.occ_map, w.col_map, w.calib, P)
    assert np.max(np.abs(got - want)) <= COLOUR_TOL
    # the FP32 path is far inside the bar; keep the margin visible
    assert np.max(np.abs(got - want)) <= 1e-5


# --------------------------------------------------------- localization ------

@pytest.fixture(scope="module")
def tiny_oracle(tiny):
    w = tiny.w
    return localize.hierarchical(lambda P: occ_oracle(w, P), w.n0, w.num_levels)


def test_localize_tiny_matches_oracle(tiny, tiny_oracle):
    res, _, vol = check_localization(tiny, tiny_oracle, lambda P: occ_oracle(tiny.w, P))
    assert vol.n == 64 and vol.num_levels == 3
    print("tiny localization:", res)


@pytest.mark.parametrize("n0,levels", [(2, 1), (8, 1), (2, 4), (8, 3), (32, 2)])
def test_localize_tiny_schedules(tiny, n0, levels):
    w = tiny.w
    f = lambda P: occ_oracle(w, P)
    lv = localize.hierarchical(f, n0, levels)
    check_localization(tiny, lv, f, n0=n0, levels=levels)


def test_localize_tiny_yaw(tiny):
    w = tiny.w
    cal = synth.calib_yaw(30.0)
    f = lambda P: occ_oracle(w, P, cal)
    lv = localize.hierarchical(f, w.n0, w.num_levels)
    check_localization(tiny, lv, f, calib=cal)


@pytest.fixture(scope="module")
def full_oracle_128(full):
    w = full.w
    return localize.hierarchical(lambda P: occ_oracle(w, P), 32, 3)


def test_localize_full_shapes_128(full, full_oracle_128):
    check_localization(full, full_oracle_128, lambda P: occ_oracle(full.w, P), n0=32, levels=3)


@pytest.fixture(scope="module")
def full_oracle_256(full):
    w = full.w
    return localize.hierarchical(lambda P: occ_oracle(w, P), 32, 4)


def test_localize_full_size_256(full, full_oracle_256):
    # the full-size workload: 32^3 -> 256^3 with the 257-1024-512-256-128-1 MLP
    res, _, vol = check_localization(full, full_oracle_256, lambda P: occ_oracle(full.w, P))
    assert vol.n == 256
    print("full-size localization:", res)


def test_localize_not_converged_is_reported(tiny, tiny_oracle):
    # the tiny figure needs several conflict rounds at 32^3 and 64^3
    assert max(l.conflict_rounds for l in tiny_oracle) > 1
    from paper_2007_13988_gb300 import pifu
    with pytest.raises(pifu.PifuError) as ei:
        tiny.localize(max_rounds=1)
    assert ei.value.status == pifu.PIFU_ERR_NOT_CONVERGED
    tiny.localize()   # the context stays usable


def test_localize_rejects_bad_arguments(tiny):
    from paper_2007_13988_gb300 import pifu
    for kw in (dict(n0=3), dict(n0=0), dict(levels=0), dict(levels=9), dict(n0=256, levels=3)):
        with pytest.raises(pifu.PifuError) as ei:
            tiny.localize(**kw)
        assert ei.value.status == pifu.PIFU_ERR_ARG


# --------------------------------------------------------------- render ------

def test_render_tiny(tiny, tiny_oracle):
    res = check_render(tiny, localized(tiny, tiny_oracle), 64, bg=(0.25, 0.5, 0.75))
    print("tiny render:", res)


@pytest.mark.parametrize("R", [32, 96, 128])
def test_render_tiny_other_sizes(tiny, tiny_oracle, R):
    check_render(tiny, localized(tiny, tiny_oracle), R)


def test_render_full_size_512(full, full_oracle_256):
    res = check_render(full, localized(full, full_oracle_256), 512)
    print("full render:", res)


def test_render_before_localize_is_a_state_error():
    from paper_2007_13988_gb300 import pifu
    c = Ctx(synth.tiny(1))
    try:
        with pytest.raises(pifu.PifuError) as ei:
            c.render(16)
        assert ei.value.status == pifu.PIFU_ERR_STATE
    finally:
        c.close()
