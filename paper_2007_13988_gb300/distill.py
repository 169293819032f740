"""Distillation of the occupancy surrogate f_S from f_O, on the GPU.

Training tuples (features, depth, occupancy) come from f_O itself: for each
of several seeded capsule figures (random pose and scale), points are drawn
near the surface and uniformly (synth.distill_points), the library gathers
their input rows and evaluates f_O in FP32 (pifu_surrogate_samples), and the
library's own kernels train f_S with BCE + Adam (pifu_surrogate_train).  The
fall-back margin is calibrated on held-out figures: a high quantile of
|f_S - 1/2| among points where f_S and f_O disagree on the side of 0.5, so
that nearly all of f_S's wrong decisions fall back to f_O.  The decisions
that remain wrong only steer the coarse levels: the finest level always runs
f_O, and its conflict loop re-evaluates wherever a wrong coarse decision left
the surface out.  PyTorch only holds the device buffers.
"""
from __future__ import annotations

import numpy as np

from . import pifu, synth


def figure_inputs(seed, C=256, H=128, W=128, scale_range=(0.7, 1.2)):
    rng = np.random.default_rng(seed)
    fig = synth.capsule_figure(seed, scale=float(rng.uniform(*scale_range)), jitter=0.04)
    return fig, synth.feature_map(fig, H, W, C, seed)


def build_samples(ctx, n_figures, per_figure, seed0=1000, C=256, H=128, W=128):
    """(x [N][ldx], y [N]) device tensors of distillation tuples, rows shuffled."""
    import torch
    ldx = (C + 1 + 7) // 8 * 8
    N = n_figures * per_figure
    x = torch.empty((N, ldx), dtype=torch.float32, device="cuda")
    y = torch.empty(N, dtype=torch.float32, device="cuda")
    calib = synth.calib_identity()
    for f in range(n_figures):
        fig, fmap = figure_inputs(seed0 + f, C, H, W)
        occ = torch.from_numpy(fmap).cuda()
        pts = torch.from_numpy(synth.distill_points(fig, per_figure, seed0 + 7919 * (f + 1))).cuda()
        sl = slice(f * per_figure, (f + 1) * per_figure)
        pifu.pifu_surrogate_samples(ctx, occ, calib, pts, x[sl], y[sl])
    torch.cuda.synchronize()
    perm = torch.randperm(N, device="cuda", generator=torch.Generator(device="cuda").manual_seed(seed0))
    return x[perm].contiguous(), y[perm].contiguous()


def train(ctx, x, y, steps=4000, batch=4096, lr=3e-3, h1=128, h2=64, seed=0):
    """Initialise and train f_S; returns the (first, last) batch losses."""
    pifu.pifu_surrogate_init(ctx, h1, h2, seed)
    return pifu.pifu_surrogate_train(ctx, x, y, batch=batch, steps=steps, lr=lr)


def calibrate_margin(ctx, seeds, per_figure=200000, precision=pifu.PIFU_PREC_BF16, quantile=0.99,
                     C=256, H=128, W=128):
    """(margin, held-out sign disagreement) from held-out figures: the
    `quantile` of |f_S - 1/2| over the points where f_S and f_O disagree."""
    import torch
    calib = synth.calib_identity()
    gaps = []
    disagree = 0
    total = 0
    for sd in seeds:
        fig, fmap = figure_inputs(sd, C, H, W)
        occ = torch.from_numpy(fmap).cuda()
        pts = torch.from_numpy(synth.distill_points(fig, per_figure, sd + 31)).cuda()
        o_s = torch.empty(per_figure, dtype=torch.float32, device="cuda")
        o_f = torch.empty(per_figure, dtype=torch.float32, device="cuda")
        pifu.pifu_surrogate_query(ctx, occ, calib, pts, o_s, precision)
        pifu.pifu_query(ctx, occ, calib, pts, o_f)
        torch.cuda.synchronize()
        wrong = (o_s >= 0.5) != (o_f >= 0.5)
        disagree += int(wrong.sum().item())
        total += per_figure
        if wrong.any():
            gaps.append((o_s[wrong] - 0.5).abs().cpu().numpy())
    if not gaps:
        return 0.0, 0.0
    g = np.concatenate(gaps)
    return float(min(0.5, np.quantile(g, quantile))), disagree / max(1, total)
