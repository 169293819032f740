"""The paper's final occupancy network, CBN + SoftZ (Appendix, Eq. 7 and
Eq. 8), through the C ABI against the FP64 oracle: the field at ragged batch
sizes, the coarse-to-fine localization and the render, at the plain FP32
parity bar (occupancy <= 1e-4; sets, volumes, counts and rounds identical at
every level, with the oracle following the library's side of 0.5 where its
own value lies within 1e-4 of it), and the forms a CBN context refuses."""
import numpy as np
import pytest

from oracle import field, localize, render
from paper_2007_13988_gb300 import pifu, synth

from gpu_common import COLOUR_TOL, DEPTH_TOL, OCC_TOL, Ctx, ambiguous_rays, check_localization

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
    res, _, _ = check_localization(tiny, tiny_levels, lambda P: occ_oracle(tiny.w, P))
    print("CBN tiny localization:", res)


def test_cbn_localize_full_128(full):
    w = full.w
    f = lambda P: occ_oracle(w, P)
    lv = localize.hierarchical(f, 32, 3)
    res, _, _ = check_localization(full, lv, f, n0=32, levels=3)
    print("CBN full 32^3 -> 128^3:", res)


def test_cbn_render_tiny(tiny, tiny_levels):
    w = tiny.w
    _, lv, _ = check_localization(tiny, tiny_levels, lambda P: occ_oracle(w, P))
    fine = lv[-1]
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
                        m, precision=pifu.PIFU_PREC_FP8_MIXED)
    assert ei.value.status == pifu.PIFU_ERR_UNSUPPORTED


# ---- tensor-core (tcgen05, BF16 operands, FP32 accumulation) form ---------------

BF16, MIXED = pifu.PIFU_PREC_BF16, pifu.PIFU_PREC_MIXED


def bf16_round(a):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def emulate_tc(net, c, z):
    """The kernel's arithmetic in float64: statistics folded into the linear
    layers as the library folds them (products in double, stored in FP32,
    MMA operands in BF16), BF16 features and block outputs a, FP32 epilogue
    values, the last layer on the unrounded a."""
    f64 = np.float64
    eps = f64(np.float32(net.eps))
    s = [1.0 / np.sqrt(np.asarray(v, f64) + eps) for v in net.var]
    WzT = (s[0][:, None] * np.asarray(net.Wz, f64)).astype(np.float32).astype(f64)
    bz = (s[0] * (np.asarray(net.bz, f64) - np.asarray(net.mu[0], f64))).astype(np.float32)
    p = np.clip(0.5 * (z + 1.0), 0.0, 1.0)
    x = (net.n_z - 1) * p
    i = np.minimum(np.floor(x).astype(int), net.n_z - 2)
    t = x - i
    n = (1 - t)[:, None] * WzT[:, i].T + t[:, None] * WzT[:, i + 1].T + bz.astype(f64)
    cb = bf16_round(c)
    for blk in range(net.n_blocks):
        g = cb @ bf16_round(net.Gg[blk]).T + np.asarray(net.gg[blk], f64)
        b = cb @ bf16_round(net.Gb[blk]).T + np.asarray(net.gb[blk], f64)
        a = np.maximum(g * n + b, 0.0)
        if blk + 1 == net.n_blocks:
            logit = a @ np.asarray(net.W[blk], f64)[0] + f64(net.b[blk][0])
            return 1.0 / (1.0 + np.exp(-logit))
        W = bf16_round((s[blk + 1][:, None] * np.asarray(net.W[blk], f64)).astype(np.float32))
        bl = (s[blk + 1] * (np.asarray(net.b[blk], f64) - np.asarray(net.mu[blk + 1], f64)))
        n = bf16_round(a) @ W.T + bl.astype(np.float32).astype(f64)


@pytest.mark.parametrize("K,m", [(64, 1), (64, 300), (128, 3001)])
def test_cbn_tc_matches_bf16_emulation(K, m):
    """Hand-sized CBN networks (C = 128: two K-blocks of features; three
    blocks) on BF16-valued maps at texel centres and depths on a 1/64 grid, so
    the kernel's inputs are exact; ragged tile counts."""
    C, n_z, nb = 128, 64, 3
    rng = np.random.default_rng(11 + K)
    u = lambda *sh: rng.uniform(-1, 1, sh)
    net = synth.CbnNet(
        C=C, n_z=n_z, width=K,
        Wz=u(K, n_z).astype(np.float32), bz=(0.1 * u(K)).astype(np.float32),
        Gg=[bf16_round(0.1 * u(K, C)).astype(np.float32) for _ in range(nb)],
        gg=[(1 + 0.1 * u(K)).astype(np.float32) for _ in range(nb)],
        Gb=[bf16_round(0.1 * u(K, C)).astype(np.float32) for _ in range(nb)],
        gb=[(0.1 * u(K)).astype(np.float32) for _ in range(nb)],
        mu=[(0.2 * u(K)).astype(np.float32) for _ in range(nb)],
        var=[rng.uniform(0.5, 1.5, K).astype(np.float32) for _ in range(nb)],
        W=[(u(K, K) * np.sqrt(6.0 / K)).astype(np.float32) for _ in range(nb - 1)]
          + [(u(1, K) * np.sqrt(3.0 / K)).astype(np.float32)],
        b=[(0.1 * u(K)).astype(np.float32) for _ in range(nb - 1)] + [np.zeros(1, np.float32)])
    w = synth.tiny(0)
    H = W = 32
    fmap = bf16_round(rng.standard_normal((H, W, C))).astype(np.float32)
    w.occ_map = np.ascontiguousarray(fmap)
    w.occ_net = net
    w.col_net = synth.colour_net(C + 1, (64, 3), (), 5)
    c = Ctx(w)
    try:
        i = rng.integers(0, W, m)
        j = rng.integers(0, H, m)
        z = rng.integers(-64, 65, m) / 64.0
        P = np.stack([(2 * i + 1) / W - 1, (2 * j + 1) / H - 1, z], 1).astype(np.float32)
        want = emulate_tc(net, fmap[j, i].astype(np.float64), z)
        got = c.query(P, precision=BF16)
        err = np.abs(got - want)
        print("CBN tc K=%d m=%d: max %.2e mean %.2e" % (K, m, err.max(), err.mean()))
        # differences only from FP32-vs-FP64 accumulation order flipping a
        # BF16 rounding of a block output
        assert err.max() <= 2e-3
        assert err.mean() <= 1e-4
    finally:
        c.close()


def test_cbn_bf16_query_against_oracle(full):
    w = full.w
    P = synth.query_points(4000, seed=24)
    want = occ_oracle(w, P)
    got = full.query(P, precision=BF16)
    err = np.abs(got - want)
    print("CBN bf16 occupancy error vs oracle: max %.3g mean %.3g" % (err.max(), err.mean()))
    assert err.mean() <= 5e-3
    assert np.count_nonzero((got >= 0.5) != (want >= 0.5)) <= 0.01 * len(P)


def test_cbn_mixed_query_decisions_match_oracle(full):
    w = full.w
    c = localize.node_coords(256)
    rng = np.random.default_rng(25)
    k, j, i = (rng.integers(0, 257, 60000) for _ in range(3))
    P = np.stack([c[i], c[j], c[k]], 1)
    o = occ_oracle(w, P)
    P = P[np.abs(o - 0.5) < 0.3][:3000].astype(np.float32)
    want = occ_oracle(w, P)
    got = full.query(P, precision=MIXED)
    near = np.abs(want - 0.5) < 0.015
    assert np.max(np.abs(got[near] - want[near])) <= OCC_TOL
    assert np.array_equal(got >= 0.5, want >= 0.5)


@pytest.fixture(scope="module")
def full_levels(full):
    w = full.w
    return localize.hierarchical(lambda P: occ_oracle(w, P), w.n0, w.num_levels)


def test_cbn_mixed_localization_256(full, full_levels):
    from oracle import metrics
    vol = full.localize(precision=MIXED, margin=0.02)
    b, e, v = full.volume_host(vol)
    iou = metrics.iou(b, full_levels[-1].binary)
    print("CBN mixed 32^3 -> 256^3: IoU %.6f, evals %d (oracle %d), rechecked %s"
          % (iou, vol.n_eval, sum(l.n_eval for l in full_levels), list(vol.rechecked_per_level)[:4]))
    assert iou >= 0.999
    vb = full.localize(precision=BF16)
    bb, _, _ = full.volume_host(vb)
    assert metrics.iou(bb, full_levels[-1].binary) >= 0.97


# ---- graph forms -------------------------------------------------------------------

def frame_outputs(B, R):
    import torch
    return (torch.empty((B, R, R), dtype=torch.float32, device="cuda"),
            torch.empty((B, R, R, 3), dtype=torch.float32, device="cuda"),
            torch.empty((B, R, R), dtype=torch.uint8, device="cuda"))


@pytest.mark.parametrize("prec", [BF16, MIXED])
def test_cbn_graph_frame_equals_host_driven(full, prec):
    """The per-frame CUDA graph runs the same kernels on the same points as
    pifu_localize + pifu_render (every point's arithmetic is independent of
    its batch neighbours), so volume and render are identical."""
    import torch
    w = full.w
    R = 256
    d, rgb, m = (x[0] for x in frame_outputs(1, R))
    vol = pifu.pifu_frame(full.ctx, full.occ, full.col, w.calib, w.n0, w.num_levels, R, R, d, rgb,
                          m, precision=prec)
    torch.cuda.synchronize()
    gb, ge, gv = full.volume_host(vol)
    g = (d.cpu().numpy(), rgb.cpu().numpy(), m.cpu().numpy())
    n_graph = int(vol.n_eval)
    hv = full.localize(precision=prec)
    hb, he, hvv = full.volume_host(hv)
    h = full.render(R, precision=BF16)
    print("CBN graph vs host (%s): evaluations %d / %d" % (prec, n_graph, int(hv.n_eval)))
    assert np.array_equal(gb, hb) and np.array_equal(ge, he)
    np.testing.assert_array_equal(np.nan_to_num(gv, nan=-1), np.nan_to_num(hvv, nan=-1))
    assert n_graph == int(hv.n_eval)
    np.testing.assert_array_equal(g[2].astype(bool), h[2])
    np.testing.assert_array_equal(np.nan_to_num(g[0], nan=-9), np.nan_to_num(h[0].astype(np.float32), nan=-9))
    np.testing.assert_array_equal(g[1], h[1].astype(np.float32))


def test_cbn_batch_equals_single_frames(full):
    """Two frames of the animated stream in lockstep make the decisions each
    makes alone (values to BF16 rounding: a round of at most 256 points runs
    in FP32 alone and in BF16 + re-check in the batch)."""
    import torch
    w = full.w
    R = 256
    subj = synth.stream(n_figures=2, frames=64, seed=300)
    maps = [[torch.from_numpy(x).cuda() for x in s.maps(7 * i)] for i, s in enumerate(subj)]
    d, rgb, m = frame_outputs(2, R)
    vols = pifu.pifu_frames(full.ctx, [o for o, _ in maps], [t for _, t in maps], [w.calib] * 2,
                            w.n0, w.num_levels, R, R, d, rgb, m, precision=MIXED)
    torch.cuda.synchronize()
    for f in range(2):
        bb, be, bv = full.volume_host(vols[f])
        d1, rgb1, m1 = (x[0] for x in frame_outputs(1, R))
        v1 = pifu.pifu_frame(full.ctx, maps[f][0], maps[f][1], w.calib, w.n0, w.num_levels, R, R,
                             d1, rgb1, m1, precision=MIXED)
        torch.cuda.synchronize()
        sb, se, sv = full.volume_host(v1)
        assert np.array_equal(bb, sb) and np.array_equal(be, se), f
        assert np.max(np.abs(np.nan_to_num(bv, nan=0) - np.nan_to_num(sv, nan=0))) <= 0.03
        assert np.mean(m[f].cpu().numpy() == m1.cpu().numpy()) >= 0.9999
