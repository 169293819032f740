"""Comparison rules for a localization (Sec. 3.2) computed in FP32 against the
FP64 oracle, with no GPU in them (tests/test_parity_rules.py checks them on
the CPU; the GPU parity tests apply them to the library's results).

Why a plain set comparison is not enough.  FP32 arithmetic may put a node
whose exact occupancy lies within NEAR_HALF of 0.5 on the other side of the
threshold.  Every later step of the method then follows that decision: the
next level's tentative values, its candidates, its conflict rounds.  So the
oracle's levels are recomputed with the other evaluator's value substituted
at exactly those nodes, level by level (the "flip-aware" oracle), and the
evaluator must then equal it: identical evaluated sets, binarized volumes,
per-level evaluation counts and conflict rounds at every level, and values
within OCC_TOL of the oracle's own (unsubstituted) values at every evaluated
node.  A node that is not within NEAR_HALF of 0.5 is never substituted, so
one wrong decision there, or one node evaluated or skipped wrongly, fails.

The same holds for the octree baselines of Fig. 3: the binarized octree
decides at 0.5 like the method; the threshold octree decides on a corner
deviation, where the substitution is the other evaluator's decision at the
nodes whose deviation lies within DEV_TOL of the threshold.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from oracle import localize

OCC_TOL = 1e-4
NEAR_HALF = 1e-4
DEV_TOL = 4 * OCC_TOL     # a deviation is a difference of two values within OCC_TOL


@dataclasses.dataclass
class EvalLevel:
    """One level as an evaluator computed it."""
    N: int
    binary: np.ndarray      # [N+1]^3 bool
    evaluated: np.ndarray   # [N+1]^3 bool
    values: np.ndarray      # [N+1]^3 float64, NaN where not evaluated (threshold form: everywhere)
    n_eval: int
    rounds: int


def node_index(P, N):
    """Linear indices of node positions P [M, 3] of a level with N cells."""
    i = np.rint((np.asarray(P, np.float64) + 1.0) * (N / 2.0)).astype(np.int64)
    n1 = N + 1
    return (i[:, 2] * n1 + i[:, 1]) * n1 + i[:, 0]


class _LevelField:
    """The oracle's field at the nodes of one level, with the evaluator's
    value at the nodes where the oracle's lies within NEAR_HALF of 0.5 (and
    the evaluator evaluated the node).  Records the unsubstituted values."""

    def __init__(self, field, N, theirs, cache, stats):
        self.field, self.N, self.theirs, self.cache, self.stats = field, N, theirs, cache, stats
        self.true = np.full((N + 1,) * 3, np.nan)

    def __call__(self, P):
        idx = node_index(P, self.N)
        o = np.empty(len(idx))
        miss = np.ones(len(idx), bool)
        if self.cache is not None:
            have = self.cache.evaluated.ravel()[idx]
            o[have] = self.cache.values.ravel()[idx[have]]
            miss = ~have
        if miss.any():
            o[miss] = self.field(np.asarray(P)[miss])
        self.true.ravel()[idx] = o
        if self.theirs is None:
            return o
        g = self.theirs.values.ravel()[idx]
        sub = (np.abs(o - 0.5) < NEAR_HALF) & ~np.isnan(g)
        self.stats["substituted"] += int(sub.sum())
        self.stats["flipped"] += int(np.count_nonzero((g[sub] >= 0.5) != (o[sub] >= 0.5)))
        out = o.copy()
        out[sub] = g[sub]
        return out


def flip_aware(field, n0, theirs, base=None, kind="method", threshold=None):
    """The oracle's levels following the evaluator's side of 0.5 (or of the
    threshold) wherever the oracle's own decision is within rounding of it.

    theirs: one EvalLevel per level (None entries: no substitution there).
    base: the plain oracle levels of the same schedule, whose values are
    reused where they were evaluated (the field is evaluated only at new
    nodes).  kind: "method", "binarized" or "threshold".
    Returns (levels, true values per level, stats)."""
    stats = {"substituted": 0, "flipped": 0, "dev_substituted": 0, "dev_flipped": 0}
    L = len(theirs)
    trues = []

    def fld(l, N):
        cache = base[l] if base is not None and l < len(base) and base[l].N == N else None
        th = theirs[l] if kind != "threshold" else None
        f = _LevelField(field, N, th, cache, stats)
        trues.append(f.true)
        return f

    levels = [localize.dense(fld(0, n0), n0)]
    for l in range(1, L):
        coarse = levels[-1]
        N = 2 * coarse.N
        f = fld(l, N)
        if kind == "method":
            levels.append(localize.refine(f, coarse))
        elif kind == "binarized":
            levels.append(localize.refine_binarized(f, coarse))
        else:
            # the threshold rule with the evaluator's decision in the band
            mean, dev = localize.corner_mean_deviation(coarse.values)
            ev = dev > threshold
            band = np.abs(dev - threshold) < DEV_TOL
            if theirs[l] is not None and band.any():
                stats["dev_substituted"] += int(band.sum())
                stats["dev_flipped"] += int(np.count_nonzero(ev[band] != theirs[l].evaluated[band]))
                ev = np.where(band, theirs[l].evaluated, ev)
            values = mean.copy()
            n = localize.evaluate_mask(f, N, ev, values)
            levels.append(localize.Level(N=N, values=values, evaluated=ev, tentative=mean,
                                         selected=ev, n_eval=n, conflict_rounds=0))
    return levels, trues, stats


def near_decisions(levels, threshold=None):
    """Oracle decisions an FP32 evaluator may take the other way: values within
    NEAR_HALF of 0.5 and (threshold form) deviations within DEV_TOL of the
    threshold."""
    n = 0
    for l, lv in enumerate(levels):
        n += int(np.count_nonzero(np.abs(lv.values[lv.evaluated] - 0.5) < NEAR_HALF))
        if threshold is not None and l > 0:
            _, dev = localize.corner_mean_deviation(levels[l - 1].values)
            n += int(np.count_nonzero(np.abs(dev - threshold) < DEV_TOL))
    return n


class ParityError(AssertionError):
    pass


def compare(theirs, levels, trues, rounds=True, threshold=None):
    """Exact comparison of the evaluator's levels (None entries are skipped)
    with flip-aware oracle levels.  Raises ParityError with the figures."""
    res = {"levels": []}
    for l, (g, o, tv) in enumerate(zip(theirs, levels, trues)):
        if g is None:
            continue
        both = g.evaluated & o.evaluated
        err = float(np.max(np.abs(g.values[both] - tv[both]))) if both.any() else 0.0
        r = {
            "N": o.N,
            "eval_symdiff": int(np.count_nonzero(g.evaluated ^ o.evaluated)),
            "n_eval": (int(g.n_eval), int(o.n_eval)),
            "rounds": (int(g.rounds), int(o.conflict_rounds)),
            "max_abs_err": err,
        }
        if threshold is None:
            r["bin_diff"] = int(np.count_nonzero(g.binary ^ o.binary))
        else:
            # interpolated values everywhere: the decision at 0.5 of a value
            # within NEAR_HALF of it may go either way; elsewhere it is unique,
            # and everywhere it must be the evaluator's own value's
            vo = o.values
            sure = np.abs(vo - 0.5) >= NEAR_HALF
            r["bin_diff"] = int(np.count_nonzero((g.binary ^ o.binary) & sure))
            r["bin_self"] = int(np.count_nonzero(g.binary != (g.values >= 0.5)))
            r["max_abs_err_all"] = float(np.max(np.abs(g.values - vo)))
        res["levels"].append(r)
        bad = (r["eval_symdiff"] != 0 or r["bin_diff"] != 0 or r["n_eval"][0] != r["n_eval"][1]
               or (rounds and r["rounds"][0] != r["rounds"][1]) or err > OCC_TOL
               or r.get("bin_self", 0) != 0 or r.get("max_abs_err_all", 0.0) > OCC_TOL + 1e-6)
        if bad:
            raise ParityError(res)
    return res
