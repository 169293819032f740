"""Shared set-up for the GPU parity tests: device copies of a workload, a
library context, and the comparison rules of the plain FP32 path.

Tolerances (plain FP32 form against the FP64 oracle):
* occupancy: max-abs error <= 1e-4;
* localization: evaluated sets, binarized volumes, evaluation counts and
  conflict rounds identical at every level to the oracle's, where the oracle
  follows the library's side of 0.5 at the nodes whose exact occupancy lies
  within 1e-4 of it (tests/parity_rules.py; such nodes are counted);
* depth: within 1e-3 of the volume extent (2), i.e. 2e-3 in NDC, on rays
  whose samples up to the crossing stay 1e-4 away from 0.5;
* colour: max-abs error <= 1e-3.
"""
from __future__ import annotations

import numpy as np

import parity_rules as pr
from oracle import field, render
from parity_rules import NEAR_HALF, OCC_TOL
DEPTH_TOL = 1e-3 * 2.0
COLOUR_TOL = 1e-3


def depth_step(N):
    """One depth interval of a ray sampled at the depth nodes of an N-cell
    level, 2 / N in NDC.  Two renders that agree on a ray's first inside
    sample put its crossing in the same interval, so their depths differ by
    less than this whatever the error of the samples.  This bounds the
    tensor-core forms, whose occupancies away from the FP32 re-check band
    keep their BF16 rounding (up to a few 1e-2), which the linear crossing
    solve passes on to the depth in proportion to the interval."""
    return 2.0 / N


def check_mixed_values(c, vol, base, field, margin=0.02, sure=0.06):
    """MIXED forms at the finest level: every stored occupancy within `margin`
    of 0.5 was evaluated again in FP32, so it is within OCC_TOL of the
    oracle's; and every decision at a node whose exact occupancy is more than
    `sure` from 0.5 (about twice the largest BF16 error seen) is the
    oracle's.  Returns the figures."""
    b, e, v = c.volume_host(vol)
    fine = base[-1]
    idx = np.flatnonzero(e.ravel())
    o = np.empty(len(idx))
    have = fine.evaluated.ravel()[idx]
    o[have] = fine.values.ravel()[idx[have]]
    if (~have).any():
        from oracle import localize
        n1 = vol.n + 1
        q = idx[~have]
        cc = localize.node_coords(vol.n)
        P = np.stack([cc[q % n1], cc[(q // n1) % n1], cc[q // (n1 * n1)]], 1)
        o[~have] = field(P)
    g = v.ravel()[idx]
    band = np.abs(g - 0.5) < margin
    far = np.abs(o - 0.5) > sure
    res = {"in_band": int(band.sum()),
           "band_err": float(np.max(np.abs(g[band] - o[band]))) if band.any() else 0.0,
           "far_flips": int(np.count_nonzero((g[far] >= 0.5) != (o[far] >= 0.5)))}
    assert res["band_err"] <= OCC_TOL, res
    assert res["far_flips"] == 0, res
    return res


def torch():
    import torch as _t
    return _t


def to_dev(a):
    t = torch()
    return t.from_numpy(np.ascontiguousarray(a)).cuda()


class Ctx:
    """A libpifu context plus device copies of one workload's inputs."""

    def __init__(self, w):
        from paper_2007_13988_gb300 import pifu
        self.pifu = pifu
        self.w = w
        self.ctx = pifu.pifu_create(pifu.blob_from_nets(w.occ_net, w.col_net))
        self.occ = to_dev(w.occ_map)
        self.col = None if w.col_map is None else to_dev(w.col_map)
        self.calib = w.calib

    def close(self):
        if self.ctx is not None:
            self.pifu.pifu_destroy(self.ctx)
            self.ctx = None

    def query(self, P, calib=None, precision=0, margin=0.02):
        t = torch()
        pts = to_dev(np.asarray(P, np.float32))
        out = t.empty(len(P), dtype=t.float32, device="cuda")
        self.pifu.pifu_query_ex(self.ctx, self.occ, self.calib if calib is None else calib, pts,
                                out, precision, margin)
        t.cuda.synchronize()
        return out.cpu().numpy().astype(np.float64)

    def query_colour(self, P, calib=None):
        t = torch()
        pts = to_dev(np.asarray(P, np.float32))
        out = t.empty((len(P), 3), dtype=t.float32, device="cuda")
        self.pifu.pifu_query_colour(self.ctx, self.occ, self.col,
                                    self.calib if calib is None else calib, pts, out)
        t.cuda.synchronize()
        return out.cpu().numpy().astype(np.float64)

    def localize(self, n0=None, levels=None, calib=None, **kw):
        w = self.w
        vol = self.pifu.pifu_localize(self.ctx, self.occ, self.calib if calib is None else calib,
                                      w.n0 if n0 is None else n0,
                                      w.num_levels if levels is None else levels, **kw)
        return vol

    def volume_host(self, vol):
        """(binary [n+1]^3, evaluated [n+1]^3, values [n+1]^3 with NaN where
        not evaluated) copied to the host."""
        occ, ev, val = self.pifu.volume_tensors(vol)
        n, rw = vol.n, vol.row_words
        b = self.pifu.unpack_bits(occ.cpu().numpy(), n, rw)
        e = self.pifu.unpack_bits(ev.cpu().numpy(), n, rw)
        v = val.cpu().numpy().astype(np.float64).reshape((n + 1,) * 3)
        v = np.where(e, v, np.nan)
        return b, e, v

    def render(self, R, calib=None, background=(0.0, 0.0, 0.0), width=None, height=None,
               precision=0, final_level=0):
        t = torch()
        W = R if width is None else width
        H = R if height is None else height
        depth = t.empty((H, W), dtype=t.float32, device="cuda")
        rgb = t.empty((H, W, 3), dtype=t.float32, device="cuda")
        mask = t.empty((H, W), dtype=t.uint8, device="cuda")
        self.pifu.pifu_render(self.ctx, W, H, self.occ, self.col,
                              self.calib if calib is None else calib, depth, rgb, mask,
                              background=background, precision=precision,
                              final_level=final_level)
        t.cuda.synchronize()
        return (depth.cpu().numpy().astype(np.float64), rgb.cpu().numpy().astype(np.float64),
                mask.cpu().numpy().astype(bool))


def near_half_count(levels):
    """Oracle-evaluated values within NEAR_HALF of 0.5 over all levels."""
    return pr.near_decisions(levels)


def eval_level(c, vol, l, full_values=False):
    """The finest level of a localization as the comparison rules take it
    (l: its index in the schedule, for the per-level counters)."""
    occ, ev, val = c.pifu.volume_tensors(vol)
    n, rw = vol.n, vol.row_words
    b = c.pifu.unpack_bits(occ.cpu().numpy(), n, rw)
    e = c.pifu.unpack_bits(ev.cpu().numpy(), n, rw)
    v = val.cpu().numpy().astype(np.float64).reshape((n + 1,) * 3)
    if not full_values:
        v = np.where(e, v, np.nan)
    return pr.EvalLevel(n, b, e, v, int(vol.evals_per_level[l]), int(vol.conflict_rounds[l]))


def check_localization(c, base, field, n0=None, levels=None, calib=None, kind="method",
                       threshold=None, **kw):
    """Localize through the library and compare with the oracle exactly
    (tests/parity_rules.py): every level's evaluated set, binarized volume,
    evaluation count and conflict rounds equal the flip-aware oracle's, and
    every evaluated value is within OCC_TOL of the oracle's.

    base: the plain oracle levels of this schedule; field: the oracle's field
    (evaluated only at nodes base did not evaluate).  When some oracle
    decision is within rounding of its threshold, the library's levels are
    taken one by one from localizations with 1, 2, ... levels (the first
    levels of a schedule do not depend on the later ones), so that the
    oracle follows the library's side of each such decision.
    Returns (the figures, the flip-aware oracle levels, the last volume)."""
    w = c.w
    n0 = w.n0 if n0 is None else n0
    L = w.num_levels if levels is None else levels
    if kind == "binarized":
        kw["subdivision"] = c.pifu.PIFU_SUBDIV_BINARIZED
    elif kind == "threshold":
        kw["subdivision"] = c.pifu.PIFU_SUBDIV_THRESHOLD
        kw["threshold"] = threshold
    full_values = kind == "threshold"
    near = pr.near_decisions(base, threshold)
    theirs = []
    if near > 0:
        for l in range(L - 1):
            v = c.localize(n0=n0, levels=l + 1, calib=calib, **kw)
            theirs.append(eval_level(c, v, l, full_values))
    # the full schedule last: it stays the context's volume for a render
    vol = c.localize(n0=n0, levels=L, calib=calib, **kw)
    final = eval_level(c, vol, L - 1, full_values)
    # the counters of every level
    counts = [int(vol.evals_per_level[l]) for l in range(L)]
    rounds = [int(vol.conflict_rounds[l]) for l in range(L)]
    if near == 0:
        theirs = [None] * (L - 1) + [final]
        got = base
        trues = [np.where(lv.evaluated, lv.values, np.nan) for lv in base]
        stats = {"substituted": 0, "flipped": 0}
    else:
        theirs.append(final)
        got, trues, stats = pr.flip_aware(field, n0, theirs, base=base, kind=kind,
                                          threshold=threshold)
    res = pr.compare(theirs, got, trues, rounds=kind == "method", threshold=threshold)
    res.update(near=near, **stats)
    res["evals"] = (counts, [int(lv.n_eval) for lv in got])
    res["rounds"] = (rounds, [int(lv.conflict_rounds) for lv in got])
    assert res["evals"][0] == res["evals"][1], res
    assert res["rounds"][0] == res["rounds"][1], res
    return res, got, vol


def ambiguous_rays(values, R):
    """Pixels whose oracle ray samples, up to and including the first
    crossing (all samples on a miss), come within NEAR_HALF of 0.5."""
    from oracle import render as orender
    V = orender.ray_columns(values, R)
    inside = V >= 0.5
    hit = inside.any(axis=2)
    k = np.where(hit, np.argmax(inside, axis=2), V.shape[2] - 1)
    ks = np.arange(V.shape[2])[None, None, :]
    upto = ks <= k[..., None]
    return ((np.abs(V - 0.5) < NEAR_HALF) & upto).any(axis=2)


def check_render(c, levels, R, calib=None, bg=(0.0, 0.0, 0.0)):
    w = c.w
    fine = levels[-1]
    o_rgb, o_depth, o_hit = render.render(fine.values, R, w.col_net, w.occ_map, w.col_map,
                                          w.calib if calib is None else calib, background=bg)
    depth, rgb, mask = c.render(R, calib=calib, background=bg)
    amb = ambiguous_rays(fine.values, R)
    ok = ~amb
    assert np.array_equal(mask[ok], o_hit[ok])
    hit = ok & o_hit
    assert hit.sum() > 0
    assert np.max(np.abs(depth[hit] - o_depth[hit])) <= DEPTH_TOL
    assert np.all(np.isnan(depth[ok & ~o_hit]))
    assert np.max(np.abs(rgb[ok] - o_rgb[ok])) <= COLOUR_TOL
    return {"hits": int(o_hit.sum()), "ambiguous": int(amb.sum()),
            "depth_err": float(np.max(np.abs(depth[hit] - o_depth[hit]))),
            "rgb_err": float(np.max(np.abs(rgb[ok] - o_rgb[ok])))}


def localized(c, base):
    """Localize (checked against the oracle) and return the oracle's levels
    that follow the library's side of 0.5 at near-0.5 nodes."""
    w = c.w
    _, lv, _ = check_localization(c, base,
                                  lambda P: field.occupancy(w.occ_net, w.occ_map, w.calib, P))
    return lv
