"""The MIXED forms' FP32 passes on the tensor cores against the FP64 oracle,
through the C ABI.  The pass splits every FP32 operand into two TF32 values
(hi = tf32(v), lo = tf32(v - hi)) and forms each product as
hi*hi + hi*lo + lo*hi with FP32 accumulation (pifu_set_recheck,
PIFU_RECHECK_TENSOR, the default).  With the margin at 0.5 every occupancy of
a MIXED query goes through that pass, so the query's values are the pass's
own: they must meet the oracle within the occupancy tolerance, at batch
sizes that cover ragged 128-point tiles, the split-K forms (fewer tiles than
SMs) and the unsplit ones, and more than one 16,384-point pass.  Passes of
at most 192 points run the SIMT network in the default form and the
split-TF32 network with PIFU_RECHECK_TENSOR_ALL (tested here at small
sizes); the SIMT form (PIFU_RECHECK_SIMT) stays covered for the large passes
too."""
import numpy as np
import pytest

from oracle import field, localize
from paper_2007_13988_gb300 import synth

from gpu_common import OCC_TOL, Ctx, check_mixed_values

pytestmark = pytest.mark.gpu

MIXED = 2
# Split TF32 keeps about 2^-22 of every product; FP32 keeps 2^-24.  The two
# forms' values may differ by a few FP32 roundings of the layer sums, far
# below the occupancy tolerance.
FORMS_TOL = 2e-5


@pytest.fixture(scope="module")
def full():
    c = Ctx(synth.full(0))
    yield c
    c.close()


def occ_oracle(w, P):
    return field.occupancy(w.occ_net, w.occ_map, w.calib, P)


@pytest.fixture(scope="module")
def oracle256(full):
    w = full.w
    return localize.hierarchical(lambda P: occ_oracle(w, P), w.n0, w.num_levels)


@pytest.fixture(scope="module")
def near_surface(oracle256):
    """Points where 0.05 < o < 0.95: the oracle's finest-level nodes (32^3 ->
    256^3) in that band, in a seeded order, then jittered copies of them.
    Their BF16 occupancies are not saturated, so a MIXED query with the margin
    at 0.5 re-checks every one of them."""
    lv = oracle256[-1]
    n1 = 257
    q = np.flatnonzero(lv.evaluated.ravel() & (np.abs(lv.values.ravel() - 0.5) < 0.45))
    rng = np.random.default_rng(5)
    q = q[rng.permutation(len(q))]
    cc = localize.node_coords(256)
    P = np.stack([cc[q % n1], cc[(q // n1) % n1], cc[q // (n1 * n1)]], 1)
    extra = P[rng.integers(0, len(P), 20000)] + rng.normal(0.0, 2e-3, (20000, 3))
    return np.concatenate([P, extra]).astype(np.float32)


# Passes of more than 192 points run the split-TF32 network (fewer: the
# SIMT network).  513 and 545: four full 128-point tiles and a ragged one of
# 1 or 33 points; 700-2305: split K (fewer (point, neuron) tiles than SMs in
# some layers); 5000: layers 1-2 unsplit; 16384 + 129: two passes.
@pytest.mark.parametrize("m", [513, 545, 700, 1000, 2305, 5000, 16384 + 129])
def test_tensor_recheck_matches_oracle(full, near_surface, m):
    P = near_surface[:m]
    want = occ_oracle(full.w, P)
    assert np.count_nonzero(np.abs(want - 0.5) < 0.45) > 192   # a split-TF32 pass
    got = full.query(P, precision=MIXED, margin=0.5)
    err = np.max(np.abs(got - want))
    print("m = %d: max |error| %.2e" % (m, err))
    assert err <= OCC_TOL, err


# Every pass on the split-TF32 network, the small ones included: one 32-point
# group, either side of a group, a ragged second tile, and every layer split.
@pytest.mark.parametrize("m", [1, 31, 33, 100, 129, 192])
def test_tensor_all_small_batches_match_oracle(full, near_surface, m):
    pifu = full.pifu
    P = near_surface[:m]
    pifu.pifu_set_recheck(full.ctx, pifu.PIFU_RECHECK_TENSOR_ALL)
    try:
        got = full.query(P, precision=MIXED, margin=0.5)
    finally:
        pifu.pifu_set_recheck(full.ctx, pifu.PIFU_RECHECK_TENSOR)
    want = occ_oracle(full.w, P)
    err = np.max(np.abs(got - want))
    print("all-tensor m = %d: max |error| %.2e" % (m, err))
    assert err <= OCC_TOL, err


def test_tensor_and_simt_forms_agree(full, near_surface):
    P = near_surface[-3000:]
    pifu = full.pifu
    a = full.query(P, precision=MIXED, margin=0.5)
    b = full.query(P, precision=MIXED, margin=0.5)
    assert np.array_equal(a, b)   # the split-K sums are taken in a fixed order
    pifu.pifu_set_recheck(full.ctx, pifu.PIFU_RECHECK_SIMT)
    try:
        s = full.query(P, precision=MIXED, margin=0.5)
    finally:
        pifu.pifu_set_recheck(full.ctx, pifu.PIFU_RECHECK_TENSOR)
    want = occ_oracle(full.w, P)
    assert np.max(np.abs(s - want)) <= OCC_TOL
    print("tensor vs SIMT re-check: max |difference| %.2e, tensor vs oracle %.2e, SIMT vs "
          "oracle %.2e" % (np.max(np.abs(a - s)), np.max(np.abs(a - want)),
                           np.max(np.abs(s - want))))
    assert np.max(np.abs(a - s)) <= FORMS_TOL, np.max(np.abs(a - s))


@pytest.mark.parametrize("form", ["tensor", "simt"])
def test_mixed_localization_band_values(full, oracle256, form):
    # a MIXED localization (32^3 -> 256^3; the finest level re-checks more
    # than 192 points at once) with either re-check form: every stored
    # occupancy within 0.02 of 0.5 meets the oracle within OCC_TOL
    pifu = full.pifu
    if form == "simt":
        pifu.pifu_set_recheck(full.ctx, pifu.PIFU_RECHECK_SIMT)
    try:
        vol = full.localize(precision=MIXED)
        res = check_mixed_values(full, vol, oracle256, lambda P: occ_oracle(full.w, P))
    finally:
        pifu.pifu_set_recheck(full.ctx, pifu.PIFU_RECHECK_TENSOR)
    print("%s re-check: %s, rechecked %s" % (form, res, list(vol.rechecked_per_level)[:4]))
    assert res["in_band"] > 0
    assert max(vol.rechecked_per_level[i] for i in range(vol.num_levels)) > 192


def test_set_recheck_rejects_unknown_form(full):
    with pytest.raises(Exception):
        full.pifu.pifu_set_recheck(full.ctx, 7)


def test_starved_wait_reports_timeout_and_context_recovers(full, oracle256):
    # The split-K units of a tile wait for each other's partial tiles (a
    # cross-CTA flag wait, no bulk copy or MMA in flight).  The test hook makes
    # that wait need an arrival that never comes: it gives up after its poll
    # limit, the kernel returns, and the call reports PIFU_ERR_TIMEOUT; then
    # the same context localizes correctly again, host-driven and as a graph.
    import torch
    pifu = full.pifu
    w = full.w
    R = 256
    depth = torch.empty((R, R), dtype=torch.float32, device="cuda")
    rgb = torch.empty((R, R, 3), dtype=torch.float32, device="cuda")
    mask = torch.empty((R, R), dtype=torch.uint8, device="cuda")

    def frame():
        v = pifu.pifu_frame(full.ctx, full.occ, full.col, w.calib, w.n0, w.num_levels, R, R,
                            depth, rgb, mask, precision=MIXED)
        torch.cuda.synchronize()
        return v

    pifu.pifu_test_starve_wait(full.ctx, 1)
    try:
        with pytest.raises(pifu.PifuError) as e1:
            full.localize(precision=MIXED)
        assert e1.value.status == pifu.PIFU_ERR_TIMEOUT
        with pytest.raises(pifu.PifuError) as e2:
            frame()
        assert e2.value.status == pifu.PIFU_ERR_TIMEOUT
    finally:
        pifu.pifu_test_starve_wait(full.ctx, 0)
    field_fn = lambda P: occ_oracle(w, P)
    res = check_mixed_values(full, full.localize(precision=MIXED), oracle256, field_fn)
    assert res["in_band"] > 0
    res = check_mixed_values(full, frame(), oracle256, field_fn)
    assert res["in_band"] > 0
