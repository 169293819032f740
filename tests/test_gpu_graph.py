"""Graph form (pifu_frame): localization + render as one CUDA graph with
device-resident batch sizes and conditional WHILE nodes for the conflict
loops.  Checked against the FP64 oracle, for determinism across relaunches,
and for its error paths (device-side non-convergence, capacity)."""
import numpy as np
import pytest

from oracle import field, localize, metrics, render
from paper_2007_13988_gb300 import pifu, synth

from gpu_common import Ctx, ambiguous_rays, check_mixed_values, depth_step

pytestmark = pytest.mark.gpu


def run_frame(c, R, precision=pifu.PIFU_PREC_MIXED, **kw):
    import torch
    depth = torch.empty((R, R), dtype=torch.float32, device="cuda")
    rgb = torch.empty((R, R, 3), dtype=torch.float32, device="cuda")
    mask = torch.empty((R, R), dtype=torch.uint8, device="cuda")
    w = c.w
    vol = pifu.pifu_frame(c.ctx, c.occ, c.col, w.calib, kw.pop("n0", w.n0),
                          kw.pop("levels", w.num_levels), R, R, depth, rgb, mask,
                          precision=precision, **kw)
    torch.cuda.synchronize()
    return vol, depth.cpu().numpy().astype(np.float64), rgb.cpu().numpy().astype(np.float64), \
        mask.cpu().numpy().astype(bool)


@pytest.fixture(scope="module")
def full():
    c = Ctx(synth.full(0))
    yield c
    c.close()


@pytest.fixture(scope="module")
def full_oracle(full):
    w = full.w
    return localize.hierarchical(lambda P: field.occupancy(w.occ_net, w.occ_map, w.calib, P),
                                 w.n0, w.num_levels)


def check_against_oracle(c, vol, depth, rgb, mask, levels, R, iou_min, rgb_tol, steps=1):
    w = c.w
    b, e, v = c.volume_host(vol)
    fine = levels[-1]
    iou = metrics.iou(b, fine.binary)
    assert iou >= iou_min, iou
    o_rgb, o_depth, o_hit = render.render(fine.values, R, w.col_net, w.occ_map, w.col_map, w.calib)
    ok = ~ambiguous_rays(fine.values, R)
    agree = np.count_nonzero(mask[ok] == o_hit[ok]) / np.count_nonzero(ok)
    assert agree >= 0.999, agree
    both = ok & o_hit & mask
    derr = float(np.max(np.abs(depth[both] - o_depth[both])))
    assert derr <= steps * depth_step(vol.n), derr
    d = rgb[both] - o_rgb[both]
    psnr = 10 * np.log10(1.0 / np.mean(d * d))
    assert np.max(np.abs(d)) <= rgb_tol
    return iou, agree, psnr, derr


def test_graph_frame_mixed_matches_oracle(full, full_oracle):
    vol, depth, rgb, mask = run_frame(full, 512)
    iou, agree, psnr, derr = check_against_oracle(full, vol, depth, rgb, mask, full_oracle, 512,
                                                  0.999, 0.05)
    w = full.w
    mv = check_mixed_values(full, vol, full_oracle,
                            lambda P: field.occupancy(w.occ_net, w.occ_map, w.calib, P))
    print("graph mixed: IoU %.6f, mask agreement %.6f, depth max %.2e, colour PSNR %.1f dB, "
          "evals %d, rounds %s, %s" % (iou, agree, derr, psnr, vol.n_eval,
                                       list(vol.conflict_rounds)[:4], mv))
    assert psnr >= 40.0
    # the device-side counters are those of the method: evaluations within
    # the near-0.5 set differences of the oracle's
    assert abs(vol.n_eval - sum(l.n_eval for l in full_oracle)) <= 200


def test_graph_frame_relaunch_is_deterministic(full):
    v1, d1, r1, m1 = run_frame(full, 512)
    v2, d2, r2, m2 = run_frame(full, 512)   # cached graph
    assert np.array_equal(m1, m2)
    assert np.array_equal(np.nan_to_num(d1, nan=-9), np.nan_to_num(d2, nan=-9))
    assert np.array_equal(r1, r2)
    assert v1.n_eval == v2.n_eval


def test_async_frames_equal_the_synchronous_frame(full):
    # pifu_frame_async launches the same graph without waiting: three frames
    # back to back, then pifu_frame_wait, give pifu_frame's outputs bit for bit
    import torch
    v1, d1, r1, m1 = run_frame(full, 512)
    R = 512
    depth = torch.empty((R, R), dtype=torch.float32, device="cuda")
    rgb = torch.empty((R, R, 3), dtype=torch.float32, device="cuda")
    mask = torch.empty((R, R), dtype=torch.uint8, device="cuda")
    w = full.w
    args = (full.ctx, full.occ, full.col, w.calib, w.n0, w.num_levels, R, R, depth, rgb, mask)
    vs = pifu.pifu_frame(*args, precision=pifu.PIFU_PREC_MIXED)   # captures this output set
    for _ in range(3):
        pifu.pifu_frame_async(*args, precision=pifu.PIFU_PREC_MIXED)
    va = pifu.pifu_frame_wait(full.ctx, torch.cuda.current_stream())
    d2 = depth.cpu().numpy().astype(np.float64)
    assert np.array_equal(mask.cpu().numpy().astype(bool), m1)
    assert np.array_equal(np.nan_to_num(d2, nan=-9), np.nan_to_num(d1, nan=-9))
    assert np.array_equal(rgb.cpu().numpy().astype(np.float64), r1)
    assert va.n_eval == v1.n_eval == vs.n_eval
    assert list(va.conflict_rounds)[:4] == list(v1.conflict_rounds)[:4]
    b1, e1, _ = full.volume_host(v1)
    ba, ea, _ = full.volume_host(va)
    assert np.array_equal(b1, ba) and np.array_equal(e1, ea)


def test_graph_frame_bf16(full, full_oracle):
    # no FP32 re-check: a BF16 decision near 0.5 may move a ray's first
    # inside sample by a node, and its crossing by up to two intervals
    vol, depth, rgb, mask = run_frame(full, 512, precision=pifu.PIFU_PREC_BF16)
    check_against_oracle(full, vol, depth, rgb, mask, full_oracle, 512, 0.99, 0.05, steps=2)


def test_graph_frame_follows_new_inputs(full):
    # same buffers, new contents: the cached graph reads whatever is there
    import torch
    w2 = synth.full(5)
    saved = full.occ.clone()
    try:
        full.occ.copy_(torch.from_numpy(w2.occ_map).cuda())
        vol, depth, rgb, mask = run_frame(full, 512)
        lv = localize.hierarchical(lambda P: field.occupancy(w2.occ_net, w2.occ_map, w2.calib, P),
                                   w2.n0, w2.num_levels)
        b, e, v = full.volume_host(vol)
        # figure 5's occupancy through figure 0's network weights would not
        # match: the maps differ but the networks are the same construction
        # with the same seed, so compare against the oracle with those weights
        lv0 = localize.hierarchical(
            lambda P: field.occupancy(full.w.occ_net, w2.occ_map, w2.calib, P), w2.n0,
            w2.num_levels)
        assert metrics.iou(b, lv0[-1].binary) >= 0.999
    finally:
        full.occ.copy_(saved)


def test_graph_frame_tiny_and_not_converged():
    c = Ctx(synth.tiny(0))
    try:
        w = c.w
        lv = localize.hierarchical(lambda P: field.occupancy(w.occ_net, w.occ_map, w.calib, P),
                                   w.n0, w.num_levels)
        vol, depth, rgb, mask = run_frame(c, 64)
        b, e, v = c.volume_host(vol)
        assert metrics.iou(b, lv[-1].binary) >= 0.99
        assert [int(vol.conflict_rounds[i]) for i in range(3)] == [l.conflict_rounds for l in lv]
        with pytest.raises(pifu.PifuError) as ei:
            run_frame(c, 64, max_rounds=1)
        assert ei.value.status == pifu.PIFU_ERR_NOT_CONVERGED
        vol, depth, rgb, mask = run_frame(c, 64)   # usable afterwards
    finally:
        c.close()


def test_graph_frame_capacity_is_checked(full):
    with pytest.raises(pifu.PifuError) as ei:
        run_frame(full, 1025)   # 1025^2 pixels > 1,048,576
    assert ei.value.status == pifu.PIFU_ERR_CAPACITY
