"""Degenerate scenes through the C ABI, against the FP64 oracle: no subject
(every node outside) and a volume that is inside everywhere.  The
constructed f_O computes min(f - z, z - b, mask - 1/2) scaled, so a map with
mask 0 (front = back = -1) puts every node far outside, and mask 1 with
front = 2, back = -2 puts every node inside.  Level 0 is then the only level
with evaluations (no interpolated value is strictly between 0 and 1), the
conflict loops never run, and the render is all background or all hits at
the observer's plane (depth +1)."""
import copy

import numpy as np
import pytest

from oracle import field, localize, render
from paper_2007_13988_gb300 import pifu, synth

from gpu_common import COLOUR_TOL, OCC_TOL, Ctx

pytestmark = pytest.mark.gpu


def scene(kind):
    w = copy.copy(synth.full(0))
    occ = w.occ_map.copy()
    if kind == "empty":
        occ[:, :, 0] = -1.0
        occ[:, :, 1] = -1.0
        occ[:, :, 2] = 0.0
    else:
        occ[:, :, 0] = 2.0
        occ[:, :, 1] = -2.0
        occ[:, :, 2] = 1.0
    w.occ_map = np.ascontiguousarray(occ)
    return w


@pytest.fixture(scope="module", params=["empty", "full"])
def case(request):
    c = Ctx(scene(request.param))
    yield request.param, c
    c.close()


def test_degenerate_localization_matches_oracle(case):
    kind, c = case
    w = c.w
    f = lambda P: field.occupancy(w.occ_net, w.occ_map, w.calib, P)
    lv = localize.hierarchical(f, w.n0, w.num_levels)
    n0_nodes = (w.n0 + 1) ** 3
    assert [l.n_eval for l in lv] == [n0_nodes] + [0] * (w.num_levels - 1)
    for prec in (pifu.PIFU_PREC_FP32, pifu.PIFU_PREC_MIXED):
        vol = c.localize(precision=prec)
        b, e, v = c.volume_host(vol)
        assert [int(vol.evals_per_level[i]) for i in range(w.num_levels)] == \
            [n0_nodes] + [0] * (w.num_levels - 1)
        assert list(vol.conflict_rounds)[:w.num_levels] == [0] * w.num_levels
        assert not e.any()                     # nothing evaluated at the finest level
        assert np.array_equal(b, lv[-1].binary)
        assert b.all() if kind == "full" else not b.any()


def test_degenerate_render(case):
    kind, c = case
    w = c.w
    R = 256
    f = lambda P: field.occupancy(w.occ_net, w.occ_map, w.calib, P)
    lv = localize.hierarchical(f, w.n0, 2)
    c.localize(levels=2)
    depth, rgb, mask = c.render(R, background=(0.25, 0.5, 0.75))
    if kind == "empty":
        assert not mask.any()
        assert np.isnan(depth).all()
        np.testing.assert_array_equal(rgb.reshape(-1, 3), np.tile([0.25, 0.5, 0.75], (R * R, 1)))
    else:
        assert mask.all()
        assert np.all(depth == 1.0)            # the first sample, at the observer's plane
        o_rgb, o_depth, o_hit = render.render(lv[-1].values, R, w.col_net, w.occ_map, w.col_map,
                                              w.calib)
        assert o_hit.all() and np.all(o_depth == 1.0)
        assert np.max(np.abs(rgb - o_rgb)) <= COLOUR_TOL


def test_degenerate_graph_frame(case):
    import torch
    kind, c = case
    w = c.w
    R = 256
    d = torch.empty((R, R), dtype=torch.float32, device="cuda")
    rgb = torch.empty((R, R, 3), dtype=torch.float32, device="cuda")
    m = torch.empty((R, R), dtype=torch.uint8, device="cuda")
    vol = pifu.pifu_frame(c.ctx, c.occ, c.col, w.calib, w.n0, w.num_levels, R, R, d, rgb, m,
                          precision=pifu.PIFU_PREC_MIXED)
    torch.cuda.synchronize()
    assert int(vol.n_eval) == (w.n0 + 1) ** 3
    mh = m.cpu().numpy().astype(bool)
    assert mh.all() if kind == "full" else not mh.any()


def test_degenerate_query_values(case):
    kind, c = case
    w = c.w
    P = synth.query_points(4096, seed=31)
    got = c.query(P)
    want = field.occupancy(w.occ_net, w.occ_map, w.calib, P)
    assert np.max(np.abs(got - want)) <= OCC_TOL
    assert (want > 0.99).all() if kind == "full" else (want < 0.01).all()
