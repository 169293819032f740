"""The whole-GPU FP32 network (the MIXED forms' FP32-accurate passes of at
most 64 points in the default re-check form) against the FP64 oracle,
through the C ABI.  A MIXED query of at most 256 points is one FP32-accurate
pass over all its points (batches that small go straight to that
arithmetic), so its values are the pass's own: sizes of at most 64 cover one
point, the 4-point register tile and its ragged edges, and one to eight
point groups; the larger ones check the hand-over to the cluster network.
The forms' agreement, determinism, the tiny network (three layers, one grid
barrier) and the bounded grid-barrier wait are covered too."""
import numpy as np
import pytest

from oracle import field, localize
from paper_2007_13988_gb300 import synth

from gpu_common import OCC_TOL, Ctx, check_localization

pytestmark = pytest.mark.gpu

MIXED = 2
# Two FP32 forms of the same network differ only in the order of their sums:
# a few FP32 roundings of each layer's pre-activations.
FORMS_TOL = 2e-6


@pytest.fixture(scope="module")
def full():
    c = Ctx(synth.full(0))
    yield c
    c.close()


@pytest.fixture(scope="module")
def tiny():
    c = Ctx(synth.tiny(0))
    yield c
    c.close()


def occ_oracle(w, P):
    return field.occupancy(w.occ_net, w.occ_map, w.calib, P)


def near_points(w, n, seed):
    """Points of the volume with occupancies spread over (0, 1): random
    points and jittered copies of the oracle's near-0.5 points among them."""
    rng = np.random.default_rng(seed)
    P = synth.query_points(20000, seed=seed)
    o = occ_oracle(w, P)
    band = P[np.abs(o - 0.5) < 0.45]
    pick = band[rng.integers(0, len(band), n // 2)] + rng.normal(0.0, 2e-3, (n // 2, 3))
    return np.concatenate([pick, P[: n - n // 2]]).astype(np.float32)


@pytest.fixture(scope="module")
def pts_full(full):
    return near_points(full.w, 192, 11)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 15, 16, 17, 24, 31, 33, 48, 63, 64, 65, 100, 129,
                               192])
def test_grid_pass_matches_oracle(full, pts_full, m):
    P = pts_full[:m]
    got = full.query(P, precision=MIXED, margin=0.5)
    want = occ_oracle(full.w, P)
    err = np.max(np.abs(got - want))
    print("m = %d: max |error| %.2e" % (m, err))
    assert err <= OCC_TOL, err


@pytest.mark.parametrize("m", [1, 7, 40, 64, 150])
def test_grid_pass_tiny_network(tiny, m):
    P = near_points(tiny.w, m, 12)
    got = tiny.query(P, precision=MIXED, margin=0.5)
    want = occ_oracle(tiny.w, P)
    err = np.max(np.abs(got - want))
    assert err <= OCC_TOL, err


def test_grid_pass_is_deterministic_and_agrees_with_cluster_form(full, pts_full):
    pifu = full.pifu
    for m in (9, 40, 64):
        P = pts_full[:m]
        a = full.query(P, precision=MIXED, margin=0.5)
        b = full.query(P, precision=MIXED, margin=0.5)
        assert np.array_equal(a, b), m   # every sum in a fixed order
        pifu.pifu_set_recheck(full.ctx, pifu.PIFU_RECHECK_SIMT)
        try:
            s = full.query(P, precision=MIXED, margin=0.5)
        finally:
            pifu.pifu_set_recheck(full.ctx, pifu.PIFU_RECHECK_TENSOR)
        print("m = %d: whole-GPU vs cluster FP32: max |difference| %.2e"
              % (m, np.max(np.abs(a - s))))
        assert np.max(np.abs(a - s)) <= FORMS_TOL, (m, np.max(np.abs(a - s)))


def test_tiny_mixed_localization_all_values_fp32_accurate(tiny):
    # With the margin at 0.5 every occupancy of a MIXED localization comes
    # from an FP32-accurate pass: the conflict rounds' small batches on the
    # whole-GPU network, the larger re-check passes on the cluster network.
    # So the comparison with the oracle is the exact one of the FP32 form.
    w = tiny.w
    f = lambda P: occ_oracle(w, P)
    lv = localize.hierarchical(f, w.n0, w.num_levels)
    res, _, vol = check_localization(tiny, lv, f, precision=MIXED, margin=0.5)
    print("tiny MIXED, margin 0.5:", res, list(vol.rechecked_per_level)[: w.num_levels])


def test_grid_barrier_wait_reports_timeout_and_recovers(tiny):
    # The tiny network has no split-TF32 form, so with the test hook on, the
    # timeout of a MIXED localization comes from the whole-GPU kernel's grid
    # barrier (no copy in flight there: the hook defers the weight copies).
    # The cluster kernel has no such wait: in the SIMT form the same call
    # succeeds.  Afterwards the context localizes correctly again.
    pifu = tiny.pifu
    w = tiny.w
    pifu.pifu_test_starve_wait(tiny.ctx, 1)
    try:
        with pytest.raises(pifu.PifuError) as ei:
            tiny.localize(precision=MIXED)
        assert ei.value.status == pifu.PIFU_ERR_TIMEOUT
        pifu.pifu_set_recheck(tiny.ctx, pifu.PIFU_RECHECK_SIMT)
        try:
            tiny.localize(precision=MIXED)
        finally:
            pifu.pifu_set_recheck(tiny.ctx, pifu.PIFU_RECHECK_TENSOR)
    finally:
        pifu.pifu_test_starve_wait(tiny.ctx, 0)
    f = lambda P: occ_oracle(w, P)
    lv = localize.hierarchical(f, w.n0, w.num_levels)
    check_localization(tiny, lv, f, precision=MIXED, margin=0.5)
