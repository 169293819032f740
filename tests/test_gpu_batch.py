"""Batched form: B frames in lockstep (pifu_frames), BF16 feature maps and
the tile autotuner.  Each frame of a batch must make the same decisions as
the same frame run alone (every MLP row is computed independently of its
batch neighbours, and a frame whose frontier is empty is unchanged by the
batch's extra rounds);
BF16 maps are checked against the FP64 oracle on the BF16-rounded values."""
import numpy as np
import pytest

from oracle import field, localize, metrics
from paper_2007_13988_gb300 import pifu, synth

from gpu_common import OCC_TOL, Ctx, to_dev

pytestmark = pytest.mark.gpu

R = 256


def torch():
    import torch as _t
    return _t


@pytest.fixture(scope="module")
def ctx():
    # A lockstep round's FP32-accurate pass holds several frames' points, so
    # its size can put the batch on split TF32 (passes of more than 192
    # points) where the frame alone runs the SIMT network; the two may take
    # the other side of 0.5 at a node within about 1e-5 of it.  The equality
    # checks below compare the method's steps, so both sides use one
    # arithmetic: the SIMT network for every pass.
    c = Ctx(synth.full(0))
    c.pifu.pifu_set_recheck(c.ctx, c.pifu.PIFU_RECHECK_SIMT)
    yield c
    c.close()


def stream_frames(n, t0=0):
    subj = synth.stream(n_figures=n, frames=64, seed=300)
    out = []
    for i, s in enumerate(subj):
        g_o, g_t = s.maps(t0 + 5 * i)
        out.append((to_dev(g_o), to_dev(g_t)))
    return subj, out


def outputs(B):
    t = torch()
    return (t.empty((B, R, R), dtype=t.float32, device="cuda"),
            t.empty((B, R, R, 3), dtype=t.float32, device="cuda"),
            t.empty((B, R, R), dtype=t.uint8, device="cuda"))


def host_volume(c, vol):
    b, e, v = c.volume_host(vol)
    return b, e, np.nan_to_num(v, nan=-1.0)


def test_batch_equals_single_frames(ctx):
    w = ctx.w
    B = 3
    subj, maps = stream_frames(B)
    calibs = [w.calib] * B
    d, rgb, m = outputs(B)
    vols = pifu.pifu_frames(ctx.ctx, [o for o, _ in maps], [t for _, t in maps], calibs, w.n0,
                            w.num_levels, R, R, d, rgb, m, precision=pifu.PIFU_PREC_MIXED)
    torch().cuda.synchronize()
    batch = [(host_volume(ctx, v), d[f].cpu().numpy(), rgb[f].cpu().numpy(), m[f].cpu().numpy(),
              [int(v.evals_per_level[i]) for i in range(w.num_levels)])
             for f, v in enumerate(vols)]
    rounds_batch = [int(vols[0].conflict_rounds[i]) for i in range(w.num_levels)]
    for f in range(B):
        d1, rgb1, m1 = (x[:1].contiguous() for x in outputs(1))
        v1 = pifu.pifu_frame(ctx.ctx, maps[f][0], maps[f][1], w.calib, w.n0, w.num_levels, R, R,
                             d1[0], rgb1[0], m1[0], precision=pifu.PIFU_PREC_MIXED)
        torch().cuda.synchronize()
        (bb, be, bv), bd, brgb, bm, bev = batch[f]
        sb, se, sv = host_volume(ctx, v1)
        # the decisions are the same; a round that has at most 256 points in
        # one form runs in FP32 there and in BF16 + FP32 re-check in the
        # other, so values agree to BF16 rounding away from 0.5
        assert np.array_equal(bb, sb) and np.array_equal(be, se), f
        assert np.max(np.abs(bv[be] - sv[se])) <= 0.03, f
        assert bev == [int(v1.evals_per_level[i]) for i in range(w.num_levels)]
        sm = m1[0].cpu().numpy()
        assert np.mean(bm == sm) >= 0.9999
        both = (bm == 1) & (sm == 1)
        assert np.max(np.abs(bd[both] - d1[0].cpu().numpy()[both])) <= 2.0 / 256
        assert np.max(np.abs(brgb[both] - rgb1[0].cpu().numpy()[both])) <= 0.05
        # the batch runs as many rounds as its slowest frame
        assert all(rb >= int(v1.conflict_rounds[i]) for i, rb in enumerate(rounds_batch))
    print("batch of %d: evaluations %s, rounds %s, scales %s"
          % (B, [b[4] for b in batch], rounds_batch, [round(s.scale, 2) for s in subj]))


def test_batch_graph_is_reused_with_new_maps(ctx):
    """Map pointers and calibrations are device data: a second batch of other
    frames relaunches the captured graph and gives those frames' results
    (the same decisions as the frame alone; values to BF16 rounding)."""
    w = ctx.w
    _, maps_a = stream_frames(2, t0=0)
    _, maps_b = stream_frames(2, t0=31)
    d, rgb, m = outputs(2)
    args = (w.n0, w.num_levels, R, R, d, rgb, m)
    pifu.pifu_frames(ctx.ctx, [o for o, _ in maps_a], [t for _, t in maps_a], [w.calib] * 2, *args)
    vb = pifu.pifu_frames(ctx.ctx, [o for o, _ in maps_b], [t for _, t in maps_b], [w.calib] * 2,
                          *args)
    torch().cuda.synchronize()
    got = host_volume(ctx, vb[1])
    d1, rgb1, m1 = outputs(1)
    v1 = pifu.pifu_frame(ctx.ctx, maps_b[1][0], maps_b[1][1], w.calib, w.n0, w.num_levels, R, R,
                         d1[0], rgb1[0], m1[0])
    torch().cuda.synchronize()
    want = host_volume(ctx, v1)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    assert np.max(np.abs(got[2][got[1]] - want[2][want[1]])) <= 0.03


def test_batch_arguments(ctx):
    w = ctx.w
    _, maps = stream_frames(2)
    t = torch()
    with pytest.raises(pifu.PifuError) as ei:
        small = to_dev(np.zeros((64, 64, 256), np.float32))
        pifu.pifu_frames(ctx.ctx, [maps[0][0], small], None, [w.calib] * 2, w.n0, 2, 64, 64)
    assert ei.value.status == pifu.PIFU_ERR_ARG
    with pytest.raises(pifu.PifuError) as ei:
        pifu.pifu_frames(ctx.ctx, [maps[0][0]], None, [w.calib], w.n0, 2, 64, 64,
                         precision=pifu.PIFU_PREC_FP32)
    assert ei.value.status == pifu.PIFU_ERR_UNSUPPORTED
    del t


def test_bf16_maps_match_oracle_on_rounded_values(ctx):
    """BF16 storage of the feature map: the plain FP32 arithmetic on it equals
    the oracle evaluated on the same BF16-rounded values (<= 1e-4), and the
    MIXED localization matches the oracle's on that map."""
    t = torch()
    w = ctx.w
    occ16 = t.from_numpy(w.occ_map).cuda().to(t.bfloat16).contiguous()
    occ_r = occ16.float().cpu().numpy().astype(np.float64)
    P = synth.distill_points(w.fig, 4096, 12)
    want = field.occupancy(w.occ_net, occ_r, w.calib, P)
    out = t.empty(len(P), dtype=t.float32, device="cuda")
    pifu.pifu_query_ex(ctx.ctx, occ16, w.calib, to_dev(P.astype(np.float32)), out, precision=0)
    t.cuda.synchronize()
    assert np.max(np.abs(out.cpu().numpy() - want)) <= OCC_TOL
    lv = localize.hierarchical(lambda Q: field.occupancy(w.occ_net, occ_r, w.calib, Q), w.n0, 3)
    vol = pifu.pifu_localize(ctx.ctx, occ16, w.calib, w.n0, 3, precision=pifu.PIFU_PREC_MIXED)
    b, e, v = ctx.volume_host(vol)
    iou = metrics.iou(b, lv[-1].binary)
    print("bf16 map, 32^3 -> 128^3 mixed: IoU %.6f" % iou)
    assert iou >= 0.999


def test_autotune_keeps_results(ctx):
    w = ctx.w
    d, rgb, m = outputs(1)
    before = pifu.pifu_frame(ctx.ctx, ctx.occ, ctx.col, w.calib, w.n0, w.num_levels, R, R, d[0],
                             rgb[0], m[0])
    torch().cuda.synchronize()
    vb = host_volume(ctx, before)
    rgb_b = rgb.cpu().numpy()
    chosen = pifu.pifu_autotune(ctx.ctx, 65536)
    print("autotune (BN, ms):", chosen)
    assert chosen and all(bn in (64, 128, 256, pifu.PIFU_TILE_PAIR) for bn, _ in chosen)
    after = pifu.pifu_frame(ctx.ctx, ctx.occ, ctx.col, w.calib, w.n0, w.num_levels, R, R, d[0],
                            rgb[0], m[0])
    torch().cuda.synchronize()
    va = host_volume(ctx, after)
    for a, b in zip(va, vb):
        assert np.array_equal(a, b)
    np.testing.assert_array_equal(rgb.cpu().numpy(), rgb_b)
