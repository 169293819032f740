"""The two octree baselines of Fig. 3 (binarized subdivision, threshold
subdivision) through pifu_localize, against the FP64 oracle's
octree_binarized / octree_threshold, and the Fig. 3 trade-off at full size.

Rules (plain FP32 form, tests/parity_rules.py): evaluated values within
OCC_TOL; for the threshold form also the interpolated values at the other
nodes (convex combinations of values within OCC_TOL).  Evaluated sets,
binarized results and per-level counts are identical at every level to the
oracle's, where the oracle follows the library's decision wherever its own is
within rounding: a value within NEAR_HALF of 0.5, or (threshold form) a
corner deviation within DEV_TOL of the threshold (where the binarized value
of an interpolated node within NEAR_HALF of 0.5 may also go either way)."""
import numpy as np
import pytest

from oracle import field, localize, metrics
from paper_2007_13988_gb300 import pifu, synth

from gpu_common import Ctx, check_localization

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


def oracle_field(w):
    return lambda P: field.occupancy(w.occ_net, w.occ_map, w.calib, P)


def gpu_volume(c, vol):
    occ, ev, val = pifu.volume_tensors(vol)
    n, rw = vol.n, vol.row_words
    b = pifu.unpack_bits(occ.cpu().numpy(), n, rw)
    e = pifu.unpack_bits(ev.cpu().numpy(), n, rw)
    v = val.cpu().numpy().astype(np.float64).reshape((n + 1,) * 3)
    return b, e, v


def check(c, base, kind, threshold=None, **kw):
    res, _, vol = check_localization(c, base, oracle_field(c.w), kind=kind, threshold=threshold,
                                     **kw)
    assert all(r == 0 for r in vol.conflict_rounds[:len(base)])
    return res


@pytest.mark.parametrize("n0,levels", [(16, 3), (8, 4), (2, 3)])
def test_binarized_octree_matches_oracle(tiny, n0, levels):
    lv = localize.octree_binarized(oracle_field(tiny.w), n0, levels)
    res = check(tiny, lv, "binarized", n0=n0, levels=levels)
    print("binarized octree %d -> %d: %s" % (n0, n0 << (levels - 1), res))


@pytest.mark.parametrize("threshold", [0.0, 0.05, 0.2, 0.4, 1.0])
def test_threshold_octree_matches_oracle(tiny, threshold):
    w = tiny.w
    lv = localize.octree_threshold(oracle_field(w), w.n0, w.num_levels, threshold)
    res = check(tiny, lv, "threshold", threshold)
    print("threshold octree thr %.2f: %s" % (threshold, res))
    if threshold == 1.0:           # no deviation of values in [0, 1] exceeds 1
        assert res["evals"][0][1:] == [0] * (w.num_levels - 1)


def test_octrees_full_shapes_128(full):
    w = full.w
    f = oracle_field(w)
    lv = localize.octree_binarized(f, 32, 3)
    check(full, lv, "binarized", n0=32, levels=3)
    lv = localize.octree_threshold(f, 32, 3, 0.08)
    check(full, lv, "threshold", 0.08, n0=32, levels=3)


def main_body(b, cell):
    """The 26-connected components of an inside set with at least `cell`
    voxels (the volume of one coarsest cell): what a coarse-to-fine search can
    see at all.  The synthetic field also has islands of 1 to 3 voxels away
    from the figure that lie between the coarsest nodes."""
    from scipy import ndimage
    lab, _ = ndimage.label(b, structure=np.ones((3, 3, 3)))
    sz = np.bincount(lab.ravel())
    sz[0] = 0
    return sz[lab] >= cell


def fig3(full, n0, levels, thresholds):
    N = n0 << (levels - 1)
    cell = (N // n0) ** 3
    bb, _, _ = gpu_volume(full, full.localize(n0=N, levels=1))
    body_bb = main_body(bb, cell)

    def run(**kw):
        vol = full.localize(n0=n0, levels=levels, **kw)
        b, _, _ = gpu_volume(full, vol)
        return ((N + 1) ** 3 / int(vol.n_eval), metrics.iou(b, bb),
                metrics.iou(main_body(b, cell), body_bb))

    ours = run()
    binz = run(subdivision=pifu.PIFU_SUBDIV_BINARIZED)
    thr = [run(subdivision=pifu.PIFU_SUBDIV_THRESHOLD, threshold=t) for t in thresholds]
    print("Fig. 3, %d^3 -> %d^3 (acceleration, IoU, main-body IoU): method %s binarized %s "
          "thresholds %s" % (n0, N, ours, binz, thr))
    return ours, binz, thr


def test_fig3_tradeoff_full_size(full):
    """32^3 -> 256^3 in FP32 against the brute-force 256^3 grid: the method
    reproduces the figure exactly (islands smaller than a coarsest cell aside)
    and is more accurate than the binarized octree; raising the threshold
    trades accuracy for fewer evaluations, and no threshold that evaluates
    fewer nodes than the method is as accurate."""
    ours, binz, thr = fig3(full, 32, 4, (0.05, 0.08, 0.12, 0.2, 0.3, 0.4))
    assert ours[2] >= 0.9999
    assert binz[1] < ours[1]
    acc = [a for a, _, _ in thr]
    assert all(x < y for x, y in zip(acc, acc[1:]))
    assert all(i < ours[1] for a, i, _ in thr if a >= ours[0])


def test_fig3_coarse_start(full):
    """8^3 -> 64^3: with few coarse nodes across the figure, both octree
    baselines lose most of it while the conflict rounds of the method
    recover all of it."""
    ours, binz, thr = fig3(full, 8, 4, (0.05, 0.2))
    assert ours[2] >= 0.9999
    assert binz[1] < 0.8 and all(i < 0.8 for _, i, _ in thr)


def test_octree_arguments(tiny):
    with pytest.raises(pifu.PifuError) as ei:
        tiny.localize(subdivision=3)
    assert ei.value.status == pifu.PIFU_ERR_ARG
    with pytest.raises(pifu.PifuError) as ei:
        tiny.localize(subdivision=pifu.PIFU_SUBDIV_THRESHOLD, threshold=-0.1)
    assert ei.value.status == pifu.PIFU_ERR_ARG
