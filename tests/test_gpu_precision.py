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
