"""Pins of the oracle's coarse-to-fine localization (Sec. 3.2) against brute
force, closed forms and a differently written fixed-point computation."""
import itertools
from collections import deque

import numpy as np
import pytest

from oracle import field, localize
from paper_2007_13988_gb300 import synth


def test_upsample_tentative_hand_example():
    # 2x2x2 coarse nodes -> 3x3x3 fine nodes.  Only coarse node (z=0,y=0,x=0)
    # is inside.  Fine (0,0,0) sits on it: 1.  Fine (0,0,1) is between it and
    # an outside node: 1/2.  Fine (1,1,1), the centre: 1/8.  Fine (2,2,2): 0.
    c = np.zeros((2, 2, 2), dtype=bool)
    c[0, 0, 0] = True
    T = localize.upsample_tentative(c)
    assert T.shape == (3, 3, 3)
    assert T[0, 0, 0] == 1.0 and T[0, 0, 1] == 0.5 and T[0, 1, 1] == 0.25
    assert T[1, 1, 1] == 0.125 and T[2, 2, 2] == 0.0 and T[0, 0, 2] == 0.0


def test_upsample_tentative_is_trilinear_brute_force():
    rng = np.random.default_rng(0)
    c = rng.random((4, 5, 3)) < 0.5
    T = localize.upsample_tentative(c)
    for k, j, i in itertools.product(range(7), range(9), range(5)):
        # trilinear weights at coarse position (i/2, j/2, k/2)
        acc = 0.0
        for kk, jj, ii in itertools.product(range(4), range(5), range(3)):
            w = (max(0, 1 - abs(k / 2 - kk)) * max(0, 1 - abs(j / 2 - jj))
                 * max(0, 1 - abs(i / 2 - ii)))
            acc += w * c[kk, jj, ii]
        assert T[k, j, i] == acc


def test_dilate26_brute_force():
    rng = np.random.default_rng(1)
    m = rng.random((6, 7, 5)) < 0.05
    out = localize.dilate26(m)
    want = np.zeros_like(m)
    for k, j, i in zip(*np.nonzero(m)):
        for dk, dj, di in itertools.product((-1, 0, 1), repeat=3):
            a, b, c = k + dk, j + dj, i + di
            if 0 <= a < 6 and 0 <= b < 7 and 0 <= c < 5:
                want[a, b, c] = True
    np.testing.assert_array_equal(out, want)


def capsule_field(fig, n_fine):
    tau = 0.5 * 2.0 / n_fine
    return lambda P: field.capsule_occupancy(fig.a, fig.b, fig.r, P, tau)


def surface_cells(values):
    """Cells whose 8 corner nodes are not all on one side of 0.5."""
    b = values >= 0.5
    anyin = np.zeros(tuple(s - 1 for s in b.shape), dtype=bool)
    allin = np.ones_like(anyin)
    for dz, dy, dx in itertools.product((0, 1), repeat=3):
        s = b[dz:dz + anyin.shape[0], dy:dy + anyin.shape[1], dx:dx + anyin.shape[2]]
        anyin |= s
        allin &= s
    return anyin & ~allin


@pytest.mark.parametrize("n0,levels", [(8, 3), (16, 2), (16, 3), (8, 4), (4, 5)])
def test_hierarchical_equals_brute_force_on_capsule_figure(n0, levels):
    # Sec. 3.2 / Sec. 4: the localization retains the brute-force result.
    # Analytic stand-in for f_O: sigmoid(-sdf / tau), a connected figure,
    # at finest grids of 32^3 and 64^3.  (At 16^3 the capsules, radius
    # 0.03-0.08, are thinner than one cell of 0.125 and the figure falls
    # apart into pieces the coarse levels cannot see.)
    fig = synth.capsule_figure(0)
    n_fine = n0 << (levels - 1)
    f = capsule_field(fig, n_fine)
    lv = localize.hierarchical(f, n0, levels)
    d = localize.dense(f, n_fine)
    fine = lv[-1]
    np.testing.assert_array_equal(fine.binary, d.binary)
    # every corner of every brute-force surface cell was evaluated, with the
    # brute-force value
    cells = surface_cells(d.values)
    corners = np.zeros_like(fine.evaluated)
    for dz, dy, dx in itertools.product((0, 1), repeat=3):
        corners[dz:dz + cells.shape[0], dy:dy + cells.shape[1], dx:dx + cells.shape[2]] |= cells
    assert fine.evaluated[corners].all()
    np.testing.assert_array_equal(fine.values[corners], d.values[corners])
    # and it evaluated fewer points than brute force (the acceleration factor)
    assert sum(l.n_eval for l in lv) < d.n_eval


def least_fixed_point(N, T, o):
    """Evaluated set by a worklist search, written independently of the
    oracle: start from candidates and their 1-ring; whenever a node is
    evaluated and conflicts, push its 1-ring."""
    n1 = N + 1
    cand = (T > 0) & (T < 1)
    E = np.zeros_like(cand)
    work = deque()
    for k, j, i in zip(*np.nonzero(cand)):
        for d in itertools.product((-1, 0, 1), repeat=3):
            a, b, c = k + d[0], j + d[1], i + d[2]
            if 0 <= a < n1 and 0 <= b < n1 and 0 <= c < n1 and not E[a, b, c]:
                E[a, b, c] = True
                work.append((a, b, c))
    while work:
        k, j, i = work.popleft()
        if (o[k, j, i] >= 0.5) != (T[k, j, i] >= 0.5):
            for d in itertools.product((-1, 0, 1), repeat=3):
                a, b, c = k + d[0], j + d[1], i + d[2]
                if 0 <= a < n1 and 0 <= b < n1 and 0 <= c < n1 and not E[a, b, c]:
                    E[a, b, c] = True
                    work.append((a, b, c))
    return E


def test_evaluated_set_is_least_fixed_point_with_network_field():
    w = synth.tiny(0)
    f = lambda P: field.occupancy(w.occ_net, w.occ_map, w.calib, P)
    lv = localize.hierarchical(f, 8, 3)   # 8 -> 16 -> 32
    dense32 = localize.dense(f, 32)
    for l in lv[1:]:
        o = localize.dense(f, l.N).values if l.N != 32 else dense32.values
        E = least_fixed_point(l.N, l.tentative, o)
        np.testing.assert_array_equal(l.evaluated, E)
        # same points, other batch composition: BLAS may round differently
        np.testing.assert_allclose(l.values[E], o[E], rtol=0, atol=1e-13)
        # unevaluated nodes keep a tentative value of exactly 0 or 1
        assert np.isin(l.values[~E], (0.0, 1.0)).all()


def test_evaluated_nodes_are_justified():
    # Every evaluated node is a candidate, a 1-ring neighbour of a candidate,
    # or a 1-ring neighbour of a conflict (Sec. 3.2).
    w = synth.tiny(0)
    f = lambda P: field.occupancy(w.occ_net, w.occ_map, w.calib, P)
    lv = localize.hierarchical(f, 16, 3)
    for l in lv[1:]:
        cand = (l.tentative > 0) & (l.tentative < 1)
        conflict = l.evaluated & ((l.values >= 0.5) != (l.tentative >= 0.5))
        ok = localize.dilate26(cand) | localize.dilate26(conflict)
        assert not (l.evaluated & ~ok).any()
        # at termination every conflict's whole 1-ring is evaluated
        assert not (localize.dilate26(conflict) & ~l.evaluated).any()


def test_isolated_thin_capsule_is_missed():
    # Reading of the "retains the accuracy" claim: a component that contains
    # no coarse node and touches no detected band is never seen.  A lone
    # sphere of radius 0.04 between the nodes of a 4^3 grid (spacing 0.5).
    a = np.array([[0.3, 0.3, 0.3]])
    r = np.array([0.04])
    f = lambda P: field.capsule_occupancy(a, a, r, P, tau=2.0 / 64 / 2)
    lv = localize.hierarchical(f, 4, 4)
    d = localize.dense(f, 32)
    assert d.binary.sum() > 0
    assert lv[-1].binary.sum() == 0


# ---- octree baselines (Fig. 3) ---------------------------------------------------

def affine_field(P):
    return 0.31 + 0.27 * P[:, 0] - 0.19 * P[:, 1] + 0.11 * P[:, 2]


def test_threshold_octree_affine_field_closed_forms():
    # tri-linear interpolation reproduces an affine field exactly
    n0, L = 4, 3
    big = localize.octree_threshold(affine_field, n0, L, threshold=10.0)
    assert [l.n_eval for l in big] == [(n0 + 1) ** 3, 0, 0]
    P = localize.grid_points(n0 << (L - 1))
    np.testing.assert_allclose(big[-1].values.ravel(), affine_field(P), atol=1e-14)
    # threshold 0: every node between coarse nodes deviates (the gradient
    # is non-zero on every axis), nodes on coarse nodes do not
    zero = localize.octree_threshold(affine_field, n0, L, threshold=0.0)
    for l in zero[1:]:
        assert l.n_eval == (l.N + 1) ** 3 - (l.N // 2 + 1) ** 3


def test_binarized_octree_single_inside_node():
    # one inside coarse node: exactly the fine nodes of the 8 cells around it
    # other than itself (its own fine node interpolates to 1, its
    # neighbours to fractions, everything else to 0) are evaluated
    n0 = 4
    centre = np.array([0.0, 0.0, 0.0])
    f = lambda P: (np.abs(P - centre).max(axis=1) < 0.1).astype(np.float64)
    lv = localize.octree_binarized(f, n0, 2)
    ev = lv[1].evaluated
    k, j, i = np.nonzero(ev)
    assert len(k) == 26                      # the 3x3x3 block around fine node (4, 4, 4), less it
    assert set(map(tuple, np.stack([k, j, i], 1) - 4)) == {
        (a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)} - {(0, 0, 0)}


def test_fig3_ordering_on_capsules():
    """On the capsule figure (32^3 -> 64^3 from 16^3): the method keeps the
    brute-force result, the binarized octree loses surface, and the
    threshold subdivision trades evaluations for accuracy monotonically."""
    from oracle import metrics
    n0, L = 16, 3
    fig = synth.capsule_figure(0)
    tau = 0.5 * 2.0 / (n0 << (L - 1))
    f = lambda P: field.capsule_occupancy(fig.a, fig.b, fig.r, P, tau)
    brute = localize.dense(f, n0 << (L - 1))
    ours = localize.hierarchical(f, n0, L)
    binz = localize.octree_binarized(f, n0, L)
    iou = lambda lv: metrics.iou(lv[-1].binary, brute.binary)
    assert iou(ours) == 1.0
    assert iou(binz) < iou(ours)
    accel, ious = [], []
    for thr in (0.05, 0.08, 0.12, 0.2, 0.3, 0.4):
        lv = localize.octree_threshold(f, n0, L, thr)
        accel.append(localize.acceleration_factor(lv))
        ious.append(iou(lv))
    assert all(a < b for a, b in zip(accel, accel[1:]))      # higher threshold, fewer evaluations
    assert ious[0] >= ious[-1]
    # at the threshold that evaluates about as many nodes as the method,
    # the method is more accurate
    a_ours = localize.acceleration_factor(ours)
    k = int(np.argmin([abs(a - a_ours) for a in accel]))
    assert ious[k] < 1.0
