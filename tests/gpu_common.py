"""Shared set-up for the GPU parity tests: device copies of a workload, a
library context, and the comparison rules of the plain FP32 path.

Tolerances (plain FP32 form against the FP64 oracle):
* occupancy: max-abs error <= 1e-4;
* binarized decisions and evaluated sets: identical, except where an
  oracle value lies within 1e-4 of 0.5 (such points are counted and the
  comparison then only bounds the difference);
* depth: within 1e-3 of the volume extent (2), i.e. 2e-3 in NDC, on rays
  whose samples up to the crossing stay 1e-4 away from 0.5;
* colour: max-abs error <= 1e-3.
"""
from __future__ import annotations

import numpy as np

OCC_TOL = 1e-4
NEAR_HALF = 1e-4
DEPTH_TOL = 1e-3 * 2.0
COLOUR_TOL = 1e-3


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
    n = 0
    for l in levels:
        v = l.values[l.evaluated]
        n += int(np.count_nonzero(np.abs(v - 0.5) < NEAR_HALF))
    return n


def compare_volume(gpu_b, gpu_e, gpu_v, levels, stats):
    """Check a GPU-localized finest level against the oracle's levels.

    Returns a dict of the figures.  Exact set equality is required when no
    oracle value lies within NEAR_HALF of 0.5; otherwise the differences are
    reported and bounded."""
    fine = levels[-1]
    near = near_half_count(levels)
    both = gpu_e & fine.evaluated
    err = float(np.max(np.abs(gpu_v[both] - fine.values[both]))) if both.any() else 0.0
    res = {
        "near_half": near,
        "eval_symdiff": int(np.count_nonzero(gpu_e ^ fine.evaluated)),
        "bin_diff": int(np.count_nonzero(gpu_b ^ fine.binary)),
        "max_abs_err": err,
        "evals_gpu": [int(stats.evals_per_level[i]) for i in range(len(levels))],
        "evals_oracle": [int(l.n_eval) for l in levels],
        "rounds_gpu": [int(stats.conflict_rounds[i]) for i in range(len(levels))],
        "rounds_oracle": [int(l.conflict_rounds) for l in levels],
    }
    assert err <= OCC_TOL, res
    if near == 0:
        assert res["eval_symdiff"] == 0, res
        assert res["bin_diff"] == 0, res
        assert res["evals_gpu"] == res["evals_oracle"], res
        assert res["rounds_gpu"] == res["rounds_oracle"], res
    else:
        # a flip at a near-0.5 point may shift the refinement locally
        assert res["bin_diff"] <= 64 * near, res
        assert res["eval_symdiff"] <= 4096 * near, res
    return res


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
