"""Pins of the oracle's mesh-free render (Sec. 3.2, Eq. 3) against closed
forms: the analytic ray-capsule intersection, a plane, and the tie rule."""
import numpy as np
import pytest

from oracle import field, localize, metrics, render
from paper_2007_13988_gb300 import synth


def plane_volume(N, z0, slope):
    z = localize.node_coords(N)
    v = np.clip(0.5 + slope * (z0 - z), 0.0, 1.0)     # inside behind z = z0
    return np.broadcast_to(v[:, None, None], (N + 1, N + 1, N + 1)).copy()


def test_plane_depth_is_exact():
    N, R = 32, 16
    vol = plane_volume(N, z0=0.2109375, slope=3.0)
    depth, hit, k = render.first_crossing(vol, R)
    assert hit.all()
    np.testing.assert_allclose(depth, 0.2109375, atol=1e-14)


def test_first_crossing_smallest_index_and_miss():
    N, R = 8, 4
    vol = np.zeros((N + 1,) * 3)
    vol[6] = 1.0          # depth node 6 -> k = 2 from the observer
    vol[2] = 1.0          # a farther inside region, k = 6
    vol[:, :, :2] = 0.0   # columns x in {0, 1} empty
    depth, hit, k = render.first_crossing(vol, R)
    # pixels whose bilinear footprint touches only columns >= 2 hit at k = 2
    c = render.pixel_centres(R)
    fx = (c + 1) * N / 2
    full = np.floor(fx) >= 2
    assert (k[:, full] == 2).all()
    # crossing between k=1 (value 0) and k=2 (value 1): half-way
    zk = 1 - 2 * np.arange(N + 1) / N
    np.testing.assert_allclose(depth[:, full], (zk[1] + zk[2]) / 2)
    # pixels entirely over the empty columns miss; background is applied
    empty = np.ceil(fx) <= 1
    assert not hit[:, empty].any()
    net = type("N", (), {"d_in": 1, "W": [np.zeros((3, 1))], "b": [np.zeros(3)], "skip": (), "slope": 0.01})()
    rgb, d2, h2 = render.render(vol, R, net, np.zeros((2, 2, 0), np.float32), None,
                                synth.calib_identity(), background=(0.1, 0.2, 0.3))
    np.testing.assert_array_equal(rgb[:, empty], np.broadcast_to([0.1, 0.2, 0.3], rgb[:, empty].shape))
    np.testing.assert_allclose(rgb[h2], 0.5)


@pytest.mark.parametrize("n0,levels,R", [(16, 3, 64), (8, 4, 64), (16, 3, 128)])
def test_depth_matches_ray_capsule_intersection(n0, levels, R):
    # With f_O replaced by sigmoid(-sdf / tau) of the capsule figure, the
    # rendered depth is the figure's front surface along each pixel ray
    # (closed form: per capsule, sphere and cylinder quadratics), within one
    # fine voxel.
    fig = synth.capsule_figure(0)
    n_fine = n0 << (levels - 1)
    tau = 0.5 * 2.0 / n_fine
    f = lambda P: field.capsule_occupancy(fig.a, fig.b, fig.r, P, tau)
    lv = localize.hierarchical(f, n0, levels)
    depth, hit, _ = render.first_crossing(lv[-1].values, R)
    c = render.pixel_centres(R)
    uu, vv = np.meshgrid(c, c, indexing="xy")
    front, _, ahit = synth.z_ray_figure(fig, uu, vv)
    both = hit & ahit
    assert both.sum() > 0.9 * ahit.sum()
    err = np.abs(depth[both] - front[both])
    assert err.max() <= 2.0 / n_fine
    # hit masks disagree only on rays grazing the silhouette: a ray that the
    # render hits passes within one voxel of the figure and vice versa
    h = 2.0 / n_fine
    mism = hit ^ ahit
    if mism.any():
        jj, ii = np.nonzero(mism)
        near = [min(np.hypot(uu[j, i] - a, vv[j, i] - b) for a, b in
                    zip(uu[ahit], vv[ahit])) if not ahit[j, i] else 0.0 for j, i in zip(jj, ii)]
        assert max(near) <= 1.5 * h


def test_metrics_closed_forms():
    a = np.zeros((4, 4, 4), bool); a[:2] = True
    b = np.zeros((4, 4, 4), bool); b[:3] = True
    assert metrics.iou(a, b) == 2 / 3
    x = np.zeros((8, 8, 3)); y = x + 0.1
    assert abs(metrics.psnr(x, y) - 20.0) < 1e-9
    # two planes shifted by a quarter voxel: Chamfer = 0.25 voxel
    N = 16
    v1 = plane_volume(N, z0=0.0, slope=N / 4)
    v2 = plane_volume(N, z0=0.25 * 2 / N, slope=N / 4)
    assert abs(metrics.chamfer_voxels(v1, v2) - 0.25) < 1e-9


def test_render_colours_the_surface_point():
    # Colour net reading phi_O[0] and P_z of a map whose channel 0 holds the
    # texel's u: the render must query f_T at (x_pixel, y_pixel, z*).
    N, R = 16, 8
    vol = plane_volume(N, z0=-0.3046875, slope=2.0)
    H = W = 16
    u = (2 * np.arange(W) + 1) / W - 1
    occ = np.broadcast_to(u[None, :, None], (H, W, 1)).astype(np.float32).copy()
    Wt = np.zeros((3, 2)); Wt[0, 0] = 1.0; Wt[1, 1] = 1.0
    net = type("N", (), {"d_in": 2, "W": [Wt], "b": [np.zeros(3)], "skip": (), "slope": 0.01})()
    rgb, depth, hit = render.render(vol, R, net, occ, None, synth.calib_identity())
    c = render.pixel_centres(R)
    assert hit.all()
    # pixel centres lie between the outermost texel centres: u is exact
    np.testing.assert_allclose(rgb[:, :, 0], np.broadcast_to((np.tanh(c)[None, :] + 1) / 2, (R, R)), atol=1e-12)
    np.testing.assert_allclose(rgb[:, :, 1], (np.tanh(-0.3046875) + 1) / 2, atol=1e-12)
    np.testing.assert_allclose(rgb[:, :, 2], 0.5)


# ---- view-culled final level -------------------------------------------------

def capsule_setup(n0, levels):
    fig = synth.capsule_figure(0)
    n_f = n0 << levels                # the final level doubles the last localized one
    tau = 0.5 * 2.0 / n_f
    f = lambda P: field.capsule_occupancy(fig.a, fig.b, fig.r, P, tau)
    lv = localize.hierarchical(f, n0, levels)
    return fig, f, lv, n_f


def test_culled_plane_crossing_closed_form():
    """A half-space, occupancy 0.5 + s (z0 - z) clipped to [0, 1].  Along a
    ray the upsampled binarized level is 0, then 1/2 at the one fine node
    between the coarse outside and inside nodes, then 1: that node is the only
    one evaluated, and the crossing interpolates its value with its
    neighbour's tentative 0 or 1."""
    z0, slope = 0.2109375, 3.0
    f = lambda P: np.clip(0.5 + slope * (z0 - P[:, 2]), 0.0, 1.0)
    N_c, R = 16, 16
    N_f = 2 * N_c
    h = 2.0 / N_f
    coarse = plane_volume(N_c, z0, slope) >= 0.5
    res = render.culled_final_level(f, coarse, R)
    assert res["hit"].all()
    assert (res["evaluated"].sum(axis=2) == 1).all()
    zc = localize.node_coords(N_c)
    z_in = zc[coarse[:, 0, 0]].max()          # nearest coarse inside node
    z_m = z_in + h                              # the fine node between it and the outside one
    o_m = 0.5 + slope * (z0 - z_m)
    if o_m >= 0.5:
        want = (z_m + h) - (0.5 / o_m) * h      # between tentative 0 and o_m
    else:
        want = z_m - (0.5 - o_m) / (1.0 - o_m) * h   # between o_m and tentative 1
    np.testing.assert_allclose(res["depth"], want, atol=1e-13)


def test_culled_invariants():
    fig, f, lv, n_f = capsule_setup(8, 3)
    R = n_f
    res = render.culled_final_level(f, lv[-1].binary, R)
    T, ev, sh = res["T"], res["evaluated"], res["shadow"]
    # nothing behind the first fully inside tentative node is evaluated
    assert not (ev & sh).any()
    # only ambiguous (fractional) tentative nodes are evaluated
    assert ((T[ev] > 0) & (T[ev] < 1)).all()
    # shadow nodes start right after the nearest node with T = 1
    o_max = T.max(axis=2)
    jj, ii = np.nonzero(o_max >= 1)
    for j, i in zip(jj[:200], ii[:200]):
        first_one = int(np.argmax(T[j, i] >= 1))
        assert not sh[j, i, :first_one + 1].any() and sh[j, i, first_one + 1:].all()
    # a hit's first inside node is preceded only by outside nodes
    v = res["values"]
    hj, hi = np.nonzero(res["hit"])
    for j, i in zip(hj[:500], hi[:500]):
        k = res["i_max"][j, i]
        assert v[j, i, k] >= 0.5 and (v[j, i, :k] < 0.5).all()
    # far fewer evaluations than the dense final level
    assert res["n_eval"] < 0.05 * T.size


@pytest.mark.parametrize("n0,levels", [(8, 3), (16, 2)])
def test_culled_depth_matches_ray_capsule_intersection(n0, levels):
    fig, f, lv, n_f = capsule_setup(n0, levels)
    R = n_f
    res = render.culled_final_level(f, lv[-1].binary, R)
    depth, hit = res["depth"], res["hit"]
    c = render.pixel_centres(R)
    uu, vv = np.meshgrid(c, c, indexing="xy")
    front, _, ahit = synth.z_ray_figure(fig, uu, vv)
    both = hit & ahit
    assert both.sum() > 0.9 * ahit.sum()
    assert np.abs(depth[both] - front[both]).max() <= 2.0 / n_f


def test_culled_matches_dense_columns():
    """Brute force: the network at every node of every pixel column, then the
    first inside node.  Where the coarse level is right the culled level finds
    the same first inside node (its one evaluated node per ray decides which
    side of it the surface lies), and its depth is within one fine voxel of
    the dense linear crossing."""
    fig, f, lv, n_f = capsule_setup(8, 3)
    R = n_f
    res = render.culled_final_level(f, lv[-1].binary, R)
    c = render.pixel_centres(R)
    zk = 1 - 2 * np.arange(n_f + 1) / n_f
    jj, ii, kk = np.meshgrid(np.arange(R), np.arange(R), np.arange(n_f + 1), indexing="ij")
    P = np.stack([c[ii.ravel()], c[jj.ravel()], zk[kk.ravel()]], axis=1)
    dense = f(P).reshape(R, R, n_f + 1)
    inside = dense >= 0.5
    dhit = inside.any(axis=2)
    assert np.mean(dhit == res["hit"]) >= 0.995
    both = dhit & res["hit"]
    kd = np.argmax(inside, axis=2)
    assert np.mean(kd[both] == res["i_max"][both]) >= 0.99
    zd = np.full(dense.shape[:2], np.nan)
    for j, i in zip(*np.nonzero(both)):
        k = kd[j, i]
        if k == 0:
            zd[j, i] = 1.0
        else:
            tt = (0.5 - dense[j, i, k - 1]) / (dense[j, i, k] - dense[j, i, k - 1])
            zd[j, i] = zk[k - 1] + tt * (zk[k] - zk[k - 1])
    assert np.nanmax(np.abs(zd[both] - res["depth"][both])) <= 2.0 / n_f
