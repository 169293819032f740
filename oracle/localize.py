"""Sec. 3.2, "Octree-based Robust Surface Localization", in float64.

Grid.  A level of resolution N has N cells and N+1 nodes per axis at
x_i = -1 + 2 i / N.  Arrays are indexed [z][y][x], i.e. node (i, j, k) has
linear index (k (N+1) + j) (N+1) + i.  Level l+1 doubles N, so even fine
indices coincide with coarse nodes.

Algorithm (one finer level, the steps in the paper's order):
 1. binarize the coarser level's values at 0.5 (inside iff o >= 0.5);
 2. tri-linearly interpolate the binarized values onto the fine nodes, giving
    the tentative value T in {0, 1/8, ..., 1};
 3. boundary candidates: T neither 0 nor 1;
 4. dilate the candidates by their 1-ring (26-neighbourhood; neighbours
    outside the grid are dropped);
 5. evaluate the selected nodes with the network;
 6. conflicts: evaluated nodes whose binarized prediction differs from the
    binarized tentative value; evaluate the not yet evaluated 1-ring
    neighbours of the conflicts, and repeat until no new node is added;
 7. the level's value is the prediction where evaluated, else T (which is 0
    or 1 there).
The coarsest level is evaluated densely.  Brute force (the PIFu baseline the
paper accelerates) evaluates every node of the finest level.

Pins: tests/test_oracle_localize.py (hierarchical equals brute force on every
surface cell for the analytic capsule field at 16^3-64^3; a full enumeration
of a 16^3 grid; the fixed-point characterisation of the evaluated set; a
hand-made 1-D-like case; the documented miss of an isolated thin capsule).
"""
from __future__ import annotations

import dataclasses

import numpy as np

F64 = np.float64


def node_coords(N):
    """Coordinates of the N+1 nodes of one axis: -1 + 2 i / N."""
    return -1.0 + 2.0 * np.arange(N + 1, dtype=F64) / N


def grid_points(N):
    """All (N+1)^3 node positions as [M, 3] (x, y, z), linear order [z][y][x]."""
    c = node_coords(N)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def points_of(N, mask):
    """Positions of the nodes where ``mask`` ([N+1]^3 bool) is set, with their
    linear indices, in increasing linear order."""
    idx = np.flatnonzero(mask.ravel())
    n1 = N + 1
    i = idx % n1
    j = (idx // n1) % n1
    k = idx // (n1 * n1)
    c = node_coords(N)
    return np.stack([c[i], c[j], c[k]], axis=1), idx


def upsample_tentative(coarse_bin):
    """Tri-linear interpolation of a binarized coarse level onto the next level.

    A fine node at index i along an axis sits on coarse node i/2 if i is even
    and half-way between coarse nodes (i-1)/2 and (i+1)/2 if i is odd; the
    tri-linear weight of every involved corner is therefore a product of 1 or
    1/2 per axis, and the value is the mean of the 1, 2, 4 or 8 corners.
    """
    a = np.asarray(coarse_bin, dtype=F64)
    for axis in range(3):
        n = a.shape[axis]
        shape = list(a.shape)
        shape[axis] = 2 * n - 1
        out = np.empty(shape, dtype=F64)
        even = [slice(None)] * 3
        odd = [slice(None)] * 3
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        even[axis] = slice(0, None, 2)
        odd[axis] = slice(1, None, 2)
        lo[axis] = slice(0, n - 1)
        hi[axis] = slice(1, n)
        out[tuple(even)] = a
        out[tuple(odd)] = 0.5 * (a[tuple(lo)] + a[tuple(hi)])
        a = out
    return a


def dilate26(mask):
    """Union of every set node's 26-neighbourhood (Chebyshev radius 1) and
    itself, restricted to the grid: out[n] = OR of mask over the 27 nodes
    n + (dx, dy, dz), d in {-1, 0, 1}^3, that lie in the grid."""
    m = np.asarray(mask, dtype=bool)
    out = np.zeros_like(m)
    if not m.any():
        return out
    # Work inside the bounding box of the set nodes grown by one (same result).
    nz = np.nonzero(m)
    lo = [max(int(v.min()) - 1, 0) for v in nz]
    hi = [min(int(v.max()) + 2, s) for v, s in zip(nz, m.shape)]
    sub = m[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
    pad = np.pad(sub, 1, constant_values=False)
    acc = np.zeros_like(sub)
    S = sub.shape
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                acc |= pad[1 + dz:1 + dz + S[0], 1 + dy:1 + dy + S[1], 1 + dx:1 + dx + S[2]]
    out[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] = acc
    return out


@dataclasses.dataclass
class Level:
    N: int                      # cells per axis
    values: np.ndarray          # [N+1]^3 float64: prediction where evaluated, else tentative
    evaluated: np.ndarray       # [N+1]^3 bool
    tentative: np.ndarray | None  # [N+1]^3 float64 (None for the dense coarsest level)
    selected: np.ndarray | None   # candidates + 1-ring (before the conflict loop)
    n_eval: int
    conflict_rounds: int        # number of conflict-neighbour evaluation rounds

    @property
    def binary(self):
        return self.values >= 0.5


def evaluate_mask(field, N, mask, values):
    """Evaluate ``field`` at the nodes of ``mask`` and write them into ``values``."""
    P, idx = points_of(N, mask)
    if len(idx):
        values.ravel()[idx] = field(P)
    return len(idx)


def dense(field, N):
    """Brute force: evaluate every node of the N^3 grid."""
    vals = np.empty((N + 1,) * 3, dtype=F64)
    vals.ravel()[:] = field(grid_points(N))
    ev = np.ones((N + 1,) * 3, dtype=bool)
    return Level(N=N, values=vals, evaluated=ev, tentative=None, selected=None,
                 n_eval=vals.size, conflict_rounds=0)


def refine(field, coarse: Level, max_rounds=100000):
    """One finer level of the coarse-to-fine localization (steps 1-7 above)."""
    N = 2 * coarse.N
    coarse_bin = coarse.values >= 0.5                       # 1. binarize
    T = upsample_tentative(coarse_bin)                      # 2. interpolate
    cand = (T > 0.0) & (T < 1.0)                            # 3. candidates
    sel = dilate26(cand)                                    # 4. 1-ring dilation
    o = np.full(T.shape, np.nan)
    n_eval = evaluate_mask(field, N, sel, o)                # 5. evaluate
    E = sel.copy()
    rounds = 0
    while True:                                             # 6. conflicts
        conflict = E & ((o >= 0.5) != (T >= 0.5))
        frontier = dilate26(conflict) & ~E
        if not frontier.any():
            break
        if rounds >= max_rounds:
            raise RuntimeError("conflict loop did not converge")
        n_eval += evaluate_mask(field, N, frontier, o)
        E |= frontier
        rounds += 1
    values = np.where(E, o, T)                              # 7. level values
    return Level(N=N, values=values, evaluated=E, tentative=T, selected=sel,
                 n_eval=n_eval, conflict_rounds=rounds)


def hierarchical(field, n0, num_levels):
    """Coarse-to-fine localization: dense at resolution n0, then num_levels-1
    refinements, each doubling the resolution.  Returns the list of levels."""
    levels = [dense(field, n0)]
    for _ in range(num_levels - 1):
        levels.append(refine(field, levels[-1]))
    return levels


# ---- the octree baselines of Fig. 3 (Sec. 3.2) ---------------------------------
#
# Two subdivision rules the paper compares against, each dense at the coarsest
# level and one pass per finer level (no dilation, no conflict rounds):
#  * binarized octree (the subdivision of the occupancy-network paper cited
#    there): binarize the coarser level, interpolate tri-linearly, evaluate
#    the nodes whose interpolated value is neither 0 nor 1 (the cells whose
#    corners straddle the boundary); every other node keeps its 0 / 1 value;
#  * threshold subdivision: for every fine node, the coarse values it
#    interpolates from (its 1, 2, 4 or 8 coarse corners, continuous values);
#    evaluate it when their maximum absolute deviation from their mean exceeds
#    the threshold, else give it that mean (tri-linear interpolation).
# The acceleration factor of Fig. 3 divides the brute-force node count by the
# evaluated count.


def corner_mean_deviation(coarse_vals):
    """(mean, deviation) for every node of the next level: the mean of the
    coarse values it interpolates from and their maximum absolute deviation
    from that mean."""
    c = np.asarray(coarse_vals, dtype=F64)
    Nc = c.shape[0] - 1
    idx = np.arange(2 * Nc + 1)
    lo, hi = idx // 2, (idx + 1) // 2
    mean = upsample_tentative(c)
    dev = np.zeros_like(mean)
    for kz in (lo, hi):
        for jy in (lo, hi):
            for ix in (lo, hi):
                dev = np.maximum(dev, np.abs(c[np.ix_(kz, jy, ix)] - mean))
    return mean, dev


def refine_binarized(field, coarse: Level):
    """One finer level of the binarized-octree baseline."""
    N = 2 * coarse.N
    T = upsample_tentative(coarse.values >= 0.5)
    ev = (T > 0.0) & (T < 1.0)
    values = T.copy()
    n = evaluate_mask(field, N, ev, values)
    return Level(N=N, values=values, evaluated=ev, tentative=T, selected=ev,
                 n_eval=n, conflict_rounds=0)


def octree_binarized(field, n0, num_levels):
    """Binarized-octree baseline; returns the levels."""
    levels = [dense(field, n0)]
    for _ in range(num_levels - 1):
        levels.append(refine_binarized(field, levels[-1]))
    return levels


def refine_threshold(field, coarse: Level, threshold):
    """One finer level of the threshold-subdivision baseline."""
    N = 2 * coarse.N
    mean, dev = corner_mean_deviation(coarse.values)
    ev = dev > threshold
    values = mean.copy()
    n = evaluate_mask(field, N, ev, values)
    return Level(N=N, values=values, evaluated=ev, tentative=mean, selected=ev,
                 n_eval=n, conflict_rounds=0)


def octree_threshold(field, n0, num_levels, threshold):
    """Threshold-subdivision baseline; returns the levels."""
    levels = [dense(field, n0)]
    for _ in range(num_levels - 1):
        levels.append(refine_threshold(field, levels[-1], threshold))
    return levels


def acceleration_factor(levels):
    """Brute-force evaluations at the finest level / evaluations made."""
    return (levels[-1].N + 1) ** 3 / sum(l.n_eval for l in levels)
