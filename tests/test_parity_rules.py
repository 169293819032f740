"""The comparison rules of the GPU parity tests (tests/parity_rules.py),
checked on the CPU with evaluators made from the oracle itself: the oracle
equals itself; an evaluator that takes the other side of 0.5 at nodes within
NEAR_HALF of it (as FP32 rounding may) is accepted, with the consequences of
that decision followed through the later levels; one planted mistake
anywhere else (a decision far from 0.5, a node evaluated or skipped, a value
off by twice the tolerance, a round count) is refused."""
import numpy as np
import pytest

from oracle import field, localize
from paper_2007_13988_gb300 import synth

import parity_rules as pr


def as_eval(levels):
    out = []
    for lv in levels:
        v = np.where(lv.evaluated, lv.values, np.nan)
        out.append(pr.EvalLevel(lv.N, lv.binary.copy(), lv.evaluated.copy(), v, lv.n_eval,
                                lv.conflict_rounds))
    return out


@pytest.fixture(scope="module")
def tiny():
    w = synth.tiny(0)
    f = lambda P: field.occupancy(w.occ_net, w.occ_map, w.calib, P)
    return f, localize.hierarchical(f, w.n0, w.num_levels), w


def test_oracle_equals_itself(tiny):
    f, lv, w = tiny
    theirs = as_eval(lv)
    got, trues, stats = pr.flip_aware(f, w.n0, theirs, base=lv)
    res = pr.compare(theirs, got, trues)
    assert stats["flipped"] == 0
    assert [r["eval_symdiff"] for r in res["levels"]] == [0] * len(lv)


@pytest.mark.parametrize("plant", ["bin", "eval_add", "eval_drop", "value", "rounds", "count"])
def test_one_planted_mistake_is_refused(tiny, plant):
    f, lv, w = tiny
    theirs = as_eval(lv)
    g = theirs[-1]
    # a node far from 0.5 that the oracle evaluated, and one it did not
    far = np.flatnonzero((g.evaluated & (np.abs(np.nan_to_num(g.values) - 0.5) > 0.2)).ravel())
    off = np.flatnonzero((~g.evaluated).ravel())
    assert len(far) and len(off)
    if plant == "bin":
        g.binary.ravel()[far[0]] ^= True
    elif plant == "eval_add":
        g.evaluated.ravel()[off[0]] = True
    elif plant == "eval_drop":
        g.evaluated.ravel()[far[0]] = False
    elif plant == "value":
        g.values.ravel()[far[0]] += 2 * pr.OCC_TOL
    elif plant == "rounds":
        g.rounds += 1
    else:
        g.n_eval += 1
    got, trues, _ = pr.flip_aware(f, w.n0, theirs, base=lv)
    with pytest.raises(pr.ParityError):
        pr.compare(theirs, got, trues)


def plane_field(x0, s=20.0):
    """Occupancy of the half-space x < x0 with a soft edge of slope s."""
    return lambda P: 1.0 / (1.0 + np.exp(-s * (x0 - np.asarray(P)[:, 0])))


def test_a_flip_near_half_is_followed_through_the_levels():
    # the plane x = 0 of nodes sits 5e-5 above 0.5 at every level; the other
    # evaluator puts it 5e-5 below, which moves the surface by one coarse
    # cell: its next levels select, evaluate and binarize other nodes
    logit = np.log((0.5 + 5e-5) / (0.5 - 5e-5))
    x0 = logit / 20.0
    exact = plane_field(x0)

    def flipped(P):
        o = exact(P)
        at0 = np.abs(np.asarray(P)[:, 0]) < 1e-12
        o[at0] = 1.0 - o[at0]
        return o

    n0, L = 4, 4
    mine = localize.hierarchical(exact, n0, L)
    theirs_lv = localize.hierarchical(flipped, n0, L)
    assert pr.near_decisions(mine) > 0
    # the flip changes the finest level beyond the flipped nodes themselves
    assert np.count_nonzero(mine[-1].evaluated ^ theirs_lv[-1].evaluated) > 0
    theirs = as_eval(theirs_lv)
    got, trues, stats = pr.flip_aware(exact, n0, theirs, base=mine)
    pr.compare(theirs, got, trues)
    assert stats["flipped"] > 0
    # the values compared are the oracle's own, not the substituted ones
    assert np.nanmax(np.abs(trues[-1] - np.where(got[-1].evaluated, got[-1].values, np.nan))) > 0


def test_a_flip_far_from_half_is_refused():
    exact = plane_field(0.013)          # no node within NEAR_HALF of 0.5

    def wrong(P):
        o = exact(P)
        pick = np.abs(np.asarray(P)[:, 0] - 0.5) < 1e-12   # o ~ 1e-4, far from 0.5
        o[pick] = 1.0 - o[pick]
        return o

    n0, L = 4, 3
    mine = localize.hierarchical(exact, n0, L)
    assert pr.near_decisions(mine) == 0
    theirs = as_eval(localize.hierarchical(wrong, n0, L))
    got, trues, _ = pr.flip_aware(exact, n0, theirs, base=mine)
    with pytest.raises(pr.ParityError):
        pr.compare(theirs, got, trues)


def test_binarized_octree_flip_is_followed():
    logit = np.log((0.5 + 5e-5) / (0.5 - 5e-5))
    exact = plane_field(logit / 20.0)

    def flipped(P):
        o = exact(P)
        at0 = np.abs(np.asarray(P)[:, 0]) < 1e-12
        o[at0] = 1.0 - o[at0]
        return o

    mine = localize.octree_binarized(exact, 4, 3)
    theirs = as_eval(localize.octree_binarized(flipped, 4, 3))
    got, trues, stats = pr.flip_aware(exact, 4, theirs, base=mine, kind="binarized")
    pr.compare(theirs, got, trues, rounds=False)
    assert stats["flipped"] > 0


def test_threshold_octree_decision_in_the_band_is_followed(tiny):
    f, _, w = tiny
    thr = 0.2
    mine = localize.octree_threshold(f, w.n0, w.num_levels, thr)
    theirs_lv = localize.octree_threshold(f, w.n0, w.num_levels, thr)
    theirs = []
    for lv in theirs_lv:
        theirs.append(pr.EvalLevel(lv.N, lv.binary.copy(), lv.evaluated.copy(), lv.values.copy(),
                                   lv.n_eval, 0))
    # the other evaluator takes the other decision at one node of the last
    # level whose deviation is within the band: accepted.  Its value there is
    # then the evaluated one instead of the interpolated mean.
    _, dev = localize.corner_mean_deviation(theirs_lv[-2].values)
    band = np.flatnonzero((np.abs(dev - thr) < pr.DEV_TOL).ravel())
    g = theirs[-1]
    assert len(band) > 0
    if len(band):
        k = band[0]
        g.evaluated.ravel()[k] ^= True
        N = g.N
        P, idx = localize.points_of(N, np.arange(g.values.size).reshape(g.values.shape) == k)
        if g.evaluated.ravel()[k]:
            g.values.ravel()[k] = f(P)[0]
            g.n_eval += 1
        else:
            g.values.ravel()[k] = localize.upsample_tentative(theirs_lv[-2].values).ravel()[k]
            g.n_eval -= 1
        g.binary.ravel()[k] = g.values.ravel()[k] >= 0.5
    got, trues, stats = pr.flip_aware(f, w.n0, theirs, base=mine, kind="threshold",
                                      threshold=thr)
    pr.compare(theirs, got, trues, rounds=False, threshold=thr)
    # a decision outside the band is refused
    out = np.flatnonzero((np.abs(dev - thr) > 0.05).ravel())
    g.evaluated.ravel()[out[0]] ^= True
    with pytest.raises(pr.ParityError):
        pr.compare(theirs, got, trues, rounds=False, threshold=thr)
