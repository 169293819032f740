"""The paper's view-culled final level (Sec. 3.2), through the C ABI, against
the FP64 oracle's culled level computed on the oracle's own localization:
plain FP32 at the parity tolerances, the MIXED graph form at the benchmark's
shape (32^3 -> 256^3 localized, the culled 512 level at 512^2), and the graph
form against the host-driven form."""
import numpy as np
import pytest

from oracle import field, localize, render
from paper_2007_13988_gb300 import pifu, synth

from gpu_common import COLOUR_TOL, DEPTH_TOL, NEAR_HALF, Ctx, depth_step

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    c = Ctx(synth.full(0))
    yield c
    c.close()


def oracle_culled(w, levels, R):
    f = lambda P: field.occupancy(w.occ_net, w.occ_map, w.calib, P)
    lv = localize.hierarchical(f, w.n0, levels)
    rgb, depth, hit, res = render.render_culled(f, lv[-1].binary, R, w.col_net, w.occ_map,
                                                w.col_map, w.calib)
    return lv, rgb, depth, hit, res


def near_half_rays(res):
    """Rays whose evaluated values up to the first inside node come within
    NEAR_HALF of 0.5 (an FP32-vs-FP64 flip can change their first node)."""
    v = res["values"]
    k = np.arange(v.shape[2])[None, None, :]
    upto = np.where(res["hit"], res["i_max"], v.shape[2] - 1)[..., None]
    return ((np.abs(v - 0.5) < NEAR_HALF) & res["evaluated"] & (k <= upto)).any(axis=2)


def test_culled_fp32_matches_oracle(full):
    w = full.w
    levels, R = 3, 256                 # 32 -> 128 localized, the culled level at 256
    lv, o_rgb, o_depth, o_hit, res = oracle_culled(w, levels, R)
    vol = full.localize(levels=levels, precision=pifu.PIFU_PREC_FP32)
    depth, rgb, mask = full.render(R, precision=pifu.PIFU_PREC_FP32, final_level=1)
    n_gpu = int(full.pifu.pifu_sync_stats(full.ctx).evals_per_level[levels])
    ok = ~near_half_rays(res)
    print("culled fp32: candidates GPU %d oracle %d, hits %d, near-0.5 rays %d"
          % (n_gpu, res["n_eval"], int(o_hit.sum()), int((~ok).sum())))
    assert abs(n_gpu - res["n_eval"]) <= 0.001 * res["n_eval"] + 10
    assert np.array_equal(mask[ok], o_hit[ok])
    both = ok & mask & o_hit
    assert np.max(np.abs(depth[both] - o_depth[both])) <= DEPTH_TOL
    assert np.max(np.abs(rgb[both] - o_rgb[both])) <= COLOUR_TOL
    # far fewer evaluations than the finest level localized densely
    assert res["n_eval"] < 0.02 * R * R * (R + 1)


def test_culled_graph_mixed_at_benchmark_shape(full):
    import torch
    w = full.w
    R = 512
    lv, o_rgb, o_depth, o_hit, res = oracle_culled(w, w.num_levels, R)
    depth = torch.empty((R, R), dtype=torch.float32, device="cuda")
    rgb = torch.empty((R, R, 3), dtype=torch.float32, device="cuda")
    mask = torch.empty((R, R), dtype=torch.uint8, device="cuda")
    vol = pifu.pifu_frame(full.ctx, full.occ, full.col, w.calib, w.n0, w.num_levels, R, R, depth,
                          rgb, mask, precision=pifu.PIFU_PREC_MIXED, final_level=1)
    torch.cuda.synchronize()
    m = mask.cpu().numpy().astype(bool)
    d = depth.cpu().numpy().astype(np.float64)
    c = rgb.cpu().numpy().astype(np.float64)
    ok = ~near_half_rays(res)
    agree = np.mean(m[ok] == o_hit[ok])
    both = ok & m & o_hit
    err = c[both] - o_rgb[both]
    psnr = 10 * np.log10(1.0 / np.mean(err * err))
    n_cull = int(vol.evals_per_level[w.num_levels])
    print("culled mixed graph 512: candidates %d (oracle %d), mask agreement %.6f, depth max %.2e, "
          "colour PSNR %.1f dB" % (n_cull, res["n_eval"], agree, np.abs(d[both] - o_depth[both]).max(),
                                   psnr))
    assert agree >= 0.999
    assert np.abs(d[both] - o_depth[both]).max() <= depth_step(2 * vol.n)
    assert psnr >= 40.0
    assert abs(n_cull - res["n_eval"]) <= 0.01 * res["n_eval"]


def test_culled_graph_equals_host_driven(full):
    import torch
    w = full.w
    R = 256
    levels = 3
    depth = torch.empty((R, R), dtype=torch.float32, device="cuda")
    rgb = torch.empty((R, R, 3), dtype=torch.float32, device="cuda")
    mask = torch.empty((R, R), dtype=torch.uint8, device="cuda")
    pifu.pifu_frame(full.ctx, full.occ, full.col, w.calib, w.n0, levels, R, R, depth, rgb, mask,
                    precision=pifu.PIFU_PREC_BF16, final_level=1)
    torch.cuda.synchronize()
    g = (depth.cpu().numpy(), rgb.cpu().numpy(), mask.cpu().numpy())
    full.localize(levels=levels, precision=pifu.PIFU_PREC_BF16)
    h = full.render(R, precision=pifu.PIFU_PREC_BF16, final_level=1)
    np.testing.assert_array_equal(g[2].astype(bool), h[2])
    np.testing.assert_array_equal(np.nan_to_num(g[0], nan=-9), np.nan_to_num(h[0].astype(np.float32), nan=-9))
    np.testing.assert_array_equal(g[1], h[1].astype(np.float32))


def test_culled_arguments(full):
    w = full.w
    full.localize(levels=2, precision=pifu.PIFU_PREC_FP32)
    with pytest.raises(pifu.PifuError) as ei:
        full.render(96, final_level=1)        # not a power of two
    assert ei.value.status == pifu.PIFU_ERR_ARG
    with pytest.raises(pifu.PifuError) as ei:
        full.render(64, width=64, height=32, final_level=1)
    assert ei.value.status == pifu.PIFU_ERR_ARG
