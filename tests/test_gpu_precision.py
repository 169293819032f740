"""The precision form at 512^3 effective resolution (32^3 -> 512^3, five
levels): tensor-core layers with FP32 re-evaluation of the occupancies within
0.02 of 0.5, against the FP64 oracle's hierarchical result at the same
resolution (IoU, Chamfer distance in fine voxels, colour of the render),
host-driven and as one CUDA graph."""
import numpy as np
import pytest

from oracle import field, localize, metrics, render
from paper_2007_13988_gb300 import pifu, synth

from gpu_common import Ctx, ambiguous_rays

pytestmark = pytest.mark.gpu

LEVELS = 5          # 32 -> 64 -> 128 -> 256 -> 512
R = 512


@pytest.fixture(scope="module")
def full():
    c = Ctx(synth.full(0))
    yield c
    c.close()


@pytest.fixture(scope="module")
def oracle512(full):
    w = full.w
    lv = localize.hierarchical(lambda P: field.occupancy(w.occ_net, w.occ_map, w.calib, P),
                               w.n0, LEVELS)
    o_rgb, o_depth, o_hit = render.render(lv[-1].values, R, w.col_net, w.occ_map, w.col_map,
                                          w.calib)
    return lv, o_rgb, o_hit


def filled(b, e, v):
    return np.where(e, v, b.astype(np.float64))


def check_volume(c, vol, lv, label):
    b, e, v = c.volume_host(vol)
    fine = lv[-1]
    iou = metrics.iou(b, fine.binary)
    ch = metrics.chamfer_voxels(filled(b, e, v), fine.values)
    n_or = sum(l.n_eval for l in lv)
    print("%s: IoU %.6f, Chamfer %.4f fine voxels, evaluations %d (oracle %d), rechecked %d"
          % (label, iou, ch, vol.n_eval, n_or,
             sum(int(vol.rechecked_per_level[i]) for i in range(LEVELS))))
    assert vol.n == 512
    assert iou >= 0.995
    assert ch <= 0.25
    # the method's own work, within the near-0.5 differences of the oracle's
    assert abs(vol.n_eval - n_or) <= 0.01 * n_or
    return b, e


def test_mixed_512_host_driven(full, oracle512):
    lv, _, _ = oracle512
    vol = full.localize(levels=LEVELS, precision=pifu.PIFU_PREC_MIXED)
    check_volume(full, vol, lv, "mixed 512^3 host-driven")


def test_mixed_512_graph_frame(full, oracle512):
    import torch
    lv, o_rgb, o_hit = oracle512
    w = full.w
    depth = torch.empty((R, R), dtype=torch.float32, device="cuda")
    rgb = torch.empty((R, R, 3), dtype=torch.float32, device="cuda")
    mask = torch.empty((R, R), dtype=torch.uint8, device="cuda")
    vol = pifu.pifu_frame(full.ctx, full.occ, full.col, w.calib, w.n0, LEVELS, R, R, depth, rgb,
                          mask, precision=pifu.PIFU_PREC_MIXED)
    torch.cuda.synchronize()
    check_volume(full, vol, lv, "mixed 512^3 graph")
    m = mask.cpu().numpy().astype(bool)
    ok = ~ambiguous_rays(lv[-1].values, R)
    agree = np.count_nonzero(m[ok] == o_hit[ok]) / np.count_nonzero(ok)
    both = ok & m & o_hit
    d = rgb.cpu().numpy().astype(np.float64)[both] - o_rgb[both]
    psnr = 10 * np.log10(1.0 / np.mean(d * d))
    print("mixed 512^3 graph render: mask agreement %.6f, colour PSNR %.1f dB" % (agree, psnr))
    assert agree >= 0.999
    assert psnr >= 40.0


# ---- FP8 form: the 1024-wide layer's output and the 512-wide layer in E4M3 --

@pytest.fixture(scope="module")
def fp8(full):
    w = full.w
    with pytest.raises(pifu.PifuError) as ei:
        full.query(np.zeros((4, 3)), precision=pifu.PIFU_PREC_FP8)
    assert ei.value.status == pifu.PIFU_ERR_STATE   # not calibrated yet
    pifu.pifu_calibrate_fp8(full.ctx, full.occ, w.calib, w.n0)
    return full


def test_fp8_query_error_is_bounded(fp8):
    """E4M3 (3 mantissa bits) for the 1024-wide layer's output and the
    512-wide layer's weights on it, the input rows in BF16: the error of the
    occupancy against FP64 is bounded in distribution, and the FP32
    re-evaluation of FP8_MIXED restores the plain tolerance near 0.5."""
    w = fp8.w
    P = synth.distill_points(w.fig, 20000, 99)
    o = field.occupancy(w.occ_net, w.occ_map, w.calib, P)
    o8 = fp8.query(P, precision=pifu.PIFU_PREC_FP8)
    e = np.abs(o8 - o)
    print("fp8 query: max %.4f p99 %.4f median %.5f" % (e.max(), np.quantile(e, 0.99),
                                                        np.median(e)))
    assert np.median(e) <= 0.01
    assert np.quantile(e, 0.99) <= 0.06
    assert e.max() <= 0.25
    om = fp8.query(P, precision=pifu.PIFU_PREC_FP8_MIXED, margin=0.02)
    near = np.abs(om - 0.5) < 0.02
    assert np.max(np.abs(om[near] - o[near])) <= 1e-4


def test_fp8_mixed_256_matches_oracle(fp8):
    w = fp8.w
    lv = localize.hierarchical(lambda P: field.occupancy(w.occ_net, w.occ_map, w.calib, P),
                               w.n0, w.num_levels)
    vol = fp8.localize(precision=pifu.PIFU_PREC_FP8_MIXED)
    b, e, v = fp8.volume_host(vol)
    iou = metrics.iou(b, lv[-1].binary)
    ch = metrics.chamfer_voxels(filled(b, e, v), lv[-1].values)
    print("fp8 mixed 256^3: IoU %.6f, Chamfer %.4f fine voxels, evaluations %d (oracle %d)"
          % (iou, ch, vol.n_eval, sum(l.n_eval for l in lv)))
    assert iou >= 0.995


def test_fp8_mixed_512_graph_frame(fp8, oracle512):
    import torch
    lv, o_rgb, o_hit = oracle512
    w = fp8.w
    depth = torch.empty((R, R), dtype=torch.float32, device="cuda")
    rgb = torch.empty((R, R, 3), dtype=torch.float32, device="cuda")
    mask = torch.empty((R, R), dtype=torch.uint8, device="cuda")
    vol = pifu.pifu_frame(fp8.ctx, fp8.occ, fp8.col, w.calib, w.n0, LEVELS, R, R, depth, rgb,
                          mask, precision=pifu.PIFU_PREC_FP8_MIXED)
    torch.cuda.synchronize()
    b, e, v = fp8.volume_host(vol)
    iou = metrics.iou(b, lv[-1].binary)
    ch = metrics.chamfer_voxels(filled(b, e, v), lv[-1].values)
    m = mask.cpu().numpy().astype(bool)
    both = m & o_hit
    d = rgb.cpu().numpy().astype(np.float64)[both] - o_rgb[both]
    psnr = 10 * np.log10(1.0 / np.mean(d * d))
    print("fp8 mixed 512^3 graph: IoU %.6f, Chamfer %.4f fine voxels, colour PSNR %.1f dB, "
          "mask disagreement %d px" % (iou, ch, psnr, int(np.count_nonzero(m != o_hit))))
    assert iou >= 0.995
    assert psnr >= 40.0
