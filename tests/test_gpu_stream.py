"""The batched video-stream form (config 4: animated subjects of different
scales, BF16 feature maps, frames evaluated together) against the FP64
oracle, frame by frame: each frame of a batch is compared with the oracle's
coarse-to-fine localization (Sec. 3.2) and render (Eq. 3) on the same
BF16-rounded maps.

Bars: occupancy IoU >= 0.995 and colour PSNR >= 40 dB for every precision
(the benchmark spec's); in MIXED also every stored occupancy within the 0.02
re-check band within OCC_TOL of the oracle's (it was evaluated again in
FP32) and every decision the same as the oracle's at nodes whose exact
occupancy is more than 0.06 from 0.5; the depth of rays that both hit
within one depth interval."""
import numpy as np
import pytest

from oracle import field, localize, metrics, render
from paper_2007_13988_gb300 import distill, pifu, synth

from gpu_common import Ctx, ambiguous_rays, check_mixed_values, depth_step

pytestmark = pytest.mark.gpu

R = 512


def torch():
    import torch as _t
    return _t


@pytest.fixture(scope="module")
def ctx():
    c = Ctx(synth.full(0))
    yield c
    c.close()


@pytest.fixture(scope="module")
def frames():
    """The stream's smallest- and largest-scale subjects (of 8, seed 100), one
    frame each, with their maps as BF16 on the device and as the BF16-rounded
    float64 values the oracle reads."""
    t = torch()
    subj = synth.stream(n_figures=8, frames=64, seed=100)
    order = np.argsort([s.scale for s in subj])
    out = []
    for i, tt in ((int(order[0]), 5), (int(order[-1]), 40)):
        g_o, g_t = subj[i].maps(tt)
        o16 = t.from_numpy(g_o).cuda().to(t.bfloat16).contiguous()
        c16 = t.from_numpy(g_t).cuda().to(t.bfloat16).contiguous()
        out.append({"subject": i, "scale": subj[i].scale, "t": tt, "occ": o16, "col": c16,
                    "occ_r": o16.float().cpu().numpy().astype(np.float64),
                    "col_r": c16.float().cpu().numpy().astype(np.float64)})
    return out


@pytest.fixture(scope="module")
def oracle_frames(ctx, frames):
    w = ctx.w
    res = []
    for fr in frames:
        f = lambda P, m=fr["occ_r"]: field.occupancy(w.occ_net, m, w.calib, P)
        lv = localize.hierarchical(f, w.n0, w.num_levels)
        rgb, depth, hit = render.render(lv[-1].values, R, w.col_net, fr["occ_r"], fr["col_r"],
                                        w.calib)
        res.append((f, lv, rgb, depth, hit))
    return res


def run_batch(c, frames, precision, **kw):
    t = torch()
    B = len(frames)
    d = t.empty((B, R, R), dtype=t.float32, device="cuda")
    rgb = t.empty((B, R, R, 3), dtype=t.float32, device="cuda")
    m = t.empty((B, R, R), dtype=t.uint8, device="cuda")
    w = c.w
    vols = pifu.pifu_frames(c.ctx, [fr["occ"] for fr in frames], [fr["col"] for fr in frames],
                            [w.calib] * B, w.n0, w.num_levels, R, R, d, rgb, m,
                            precision=precision, **kw)
    t.cuda.synchronize()
    return vols, d.cpu().numpy().astype(np.float64), rgb.cpu().numpy().astype(np.float64), \
        m.cpu().numpy().astype(bool)


def check_frame(c, vol, depth, rgb, mask, ofr, mixed):
    f, lv, o_rgb, o_depth, o_hit = ofr
    b, e, v = c.volume_host(vol)
    fine = lv[-1]
    iou = metrics.iou(b, fine.binary)
    ok = ~ambiguous_rays(fine.values, R)
    both = ok & mask & o_hit
    d = rgb[both] - o_rgb[both]
    psnr = 10 * np.log10(1.0 / np.mean(d * d))
    derr = float(np.max(np.abs(depth[both] - o_depth[both])))
    res = {"iou": iou, "psnr": psnr, "depth_err": derr,
           "mask_agree": float(np.mean(mask[ok] == o_hit[ok])),
           "evals": int(vol.n_eval), "evals_oracle": int(sum(l.n_eval for l in lv))}
    assert iou >= 0.995, res
    assert psnr >= 40.0, res
    if mixed:
        res.update(check_mixed_values(c, vol, lv, f))
        assert derr <= depth_step(vol.n), res
    return res


def test_stream_batch_mixed_matches_oracle(ctx, frames, oracle_frames):
    vols, depth, rgb, mask = run_batch(ctx, frames, pifu.PIFU_PREC_MIXED)
    for k, (fr, ofr) in enumerate(zip(frames, oracle_frames)):
        res = check_frame(ctx, vols[k], depth[k], rgb[k], mask[k], ofr, mixed=True)
        print("stream MIXED subject %d (scale %.2f) frame %d: %s"
              % (fr["subject"], fr["scale"], fr["t"], res))


@pytest.fixture(scope="module")
def fp8_surrogate(ctx, frames):
    """FP8 scales from the first frame, and a surrogate distilled as the
    surrogate tests do it."""
    w = ctx.w
    pifu.pifu_calibrate_fp8(ctx.ctx, frames[0]["occ"], w.calib, w.n0)
    x, y = distill.build_samples(ctx.ctx, n_figures=12, per_figure=200000, seed0=1000)
    distill.train(ctx.ctx, x, y, steps=4000, batch=4096, lr=3e-3)
    margin, _ = distill.calibrate_margin(ctx.ctx, seeds=[2000, 2001], per_figure=100000)
    assert margin < 0.5     # the surrogate decides some points itself
    return margin


def test_stream_batch_fp8_mixed_surrogate_matches_oracle(ctx, frames, oracle_frames,
                                                         fp8_surrogate):
    vols, depth, rgb, mask = run_batch(ctx, frames, pifu.PIFU_PREC_FP8_MIXED,
                                       use_surrogate=True, surrogate_margin=fp8_surrogate)
    for k, (fr, ofr) in enumerate(zip(frames, oracle_frames)):
        res = check_frame(ctx, vols[k], depth[k], rgb[k], mask[k], ofr, mixed=False)
        print("stream FP8_MIXED + surrogate (margin %.3f) subject %d (scale %.2f) frame %d: %s"
              % (fp8_surrogate, fr["subject"], fr["scale"], fr["t"], res))
