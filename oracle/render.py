"""Sec. 3.2, "Mesh-free Rendering", in float64.

The volume is aligned with the target view: x and y are the pixel axes and z
runs along the camera ray, higher z nearer to the observer (Sec. 3.2).

Reading used for a render of R x R pixels over a level of N cells:
* pixel (i, j) has its centre at x = (2i+1)/R - 1, y = (2j+1)/R - 1;
* along the ray the samples are the node depths z_k = 1 - 2k/N, k = 0..N,
  counted from the observer (k = 0 nearest, so the first crossing wins ties
  at the smallest index, matching the argmax convention of Sec. 3.2);
* the sample value v_k is the bilinear interpolation in (x, y) of the four
  node columns around the pixel centre at depth node k;
* the surface is the first k with v_k >= 0.5; its depth is the linear 0.5
  crossing between samples k-1 and k (z = 1 if k = 0), i.e. the two nodes are
  "interpolated by the predicted occupancy value";
* Eq. 3: R(q) = T(P(q), I) where the ray hits, else the background B (and a
  transparent mask).

Pins: tests/test_oracle_render.py (depth against the closed-form ray-capsule
intersection for the analytic capsule field, within one fine voxel; a
half-space volume with a known plane; the smallest-index tie rule).
Colour values are pinned only through the field's own pins (the colour
weights are seeded and have no closed form).
"""
from __future__ import annotations

import numpy as np

from . import field as _field

F64 = np.float64


def pixel_centres(R):
    return (2.0 * np.arange(R, dtype=F64) + 1.0) / R - 1.0


def ray_columns(values, R):
    """Bilinear (x, y) interpolation of node columns at every pixel centre.

    values: [N+1]^3 indexed [z][y][x].  Returns V [R, R, N+1] with
    V[j, i, k] = value at pixel (i, j), depth node k counted from the observer
    (depth node index N - k in the array).
    """
    N = values.shape[0] - 1
    c = pixel_centres(R)
    f = (c + 1.0) * N / 2.0                 # continuous node coordinate
    i0 = np.minimum(np.floor(f).astype(np.int64), N - 1)
    w = f - i0
    vz = values[::-1]                        # vz[k] = depth node N - k
    # along y (rows j) then x (columns i)
    rows = (1 - w)[None, :, None] * vz[:, i0, :] + w[None, :, None] * vz[:, i0 + 1, :]
    cols = (1 - w)[None, None, :] * rows[:, :, i0] + w[None, None, :] * rows[:, :, i0 + 1]
    return np.transpose(cols, (1, 2, 0))    # [j, i, k]


def first_crossing(values, R):
    """Depth map, hit mask and first-crossing index of an R x R render.

    Returns (depth [R, R] float64 with NaN on misses, hit [R, R] bool,
    k [R, R] int64 with -1 on misses)."""
    N = values.shape[0] - 1
    V = ray_columns(values, R)
    inside = V >= 0.5
    hit = inside.any(axis=2)
    k = np.where(hit, np.argmax(inside, axis=2), -1)     # argmax: smallest index
    zk = 1.0 - 2.0 * np.arange(N + 1, dtype=F64) / N
    depth = np.full((R, R), np.nan)
    jj, ii = np.nonzero(hit)
    kk = k[jj, ii]
    first = kk == 0
    depth[jj[first], ii[first]] = 1.0
    jn, in_, kn = jj[~first], ii[~first], kk[~first]
    v0 = V[jn, in_, kn - 1]
    v1 = V[jn, in_, kn]
    t = (0.5 - v0) / (v1 - v0)
    depth[jn, in_] = zk[kn - 1] + t * (zk[kn] - zk[kn - 1])
    return depth, hit, k


def render(values, R, col_net, occ_map, col_map, calib, background=(0.0, 0.0, 0.0)):
    """Eq. 3: RGB [R, R, 3], depth, hit mask.  Hit pixels get T(P(q), I) at the
    surface point P(q) = (x, y, z*); misses get the background."""
    depth, hit, _ = first_crossing(values, R)
    rgb = np.empty((R, R, 3), dtype=F64)
    rgb[:] = np.asarray(background, dtype=F64)
    c = pixel_centres(R)
    jj, ii = np.nonzero(hit)
    if len(jj):
        P = np.stack([c[ii], c[jj], depth[jj, ii]], axis=1)
        rgb[jj, ii] = _field.colour(col_net, occ_map, col_map, calib, P)
    return rgb, depth, hit
