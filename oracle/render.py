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


# ---- the paper's view-culled final level (Sec. 3.2, "Mesh-free Rendering") ----
#
# Reading used: the render's pixel columns are the final level's columns (the
# grid's x, y are the pixel axes): pixel (i, j) at its centre, depth nodes
# z_k = 1 - 2k/N_f (k = 0 nearest) of the final level, N_f = 2 N_c where N_c
# is the last localized level.  Steps, in the paper's order:
#  1. upsample the binarized level N_c by tri-linear interpolation to every
#     (pixel, depth node): the tentative value T;
#  2. argmax along the ray: O_max = max_k T, i_max = the smallest k reaching it;
#  3. if O_max = 1, the nodes behind i_max (k > i_max) are shadow nodes;
#  4. the remaining nodes with an interpolated value strictly between 0 and 1
#     (the ambiguous band around 0.5) are evaluated with the network; every
#     other node keeps T (0 or 1, or its fraction behind the shadow line);
#  5. binarize (>= 0.5) and argmax again; a pixel hits when some node is
#     inside, and its surface lies between the nodes i_max - 1 and i_max,
#     interpolated linearly by their values (z = 1 when i_max = 0);
#  6. Eq. 3 colours the surface point.


def tentative_columns(coarse_binary, R, N_f):
    """T [R, R, N_f + 1]: tri-linear interpolation of the binarized level
    (bool [N_c+1]^3, [z][y][x]) at pixel centres and final-level depth nodes
    (k counted from the observer)."""
    N_c = coarse_binary.shape[0] - 1
    B = np.asarray(coarse_binary, dtype=F64)
    Vc = ray_columns(B, R)                   # [j, i, kc], kc = coarse depth from the observer
    zk = 1.0 - 2.0 * np.arange(N_f + 1, dtype=F64) / N_f
    fz = (1.0 - zk) * N_c / 2.0              # coarse depth coordinate from the observer
    k0 = np.minimum(np.floor(fz).astype(np.int64), N_c - 1)
    wz = fz - k0
    return (1.0 - wz)[None, None, :] * Vc[:, :, k0] + wz[None, None, :] * Vc[:, :, k0 + 1]


def culled_final_level(field, coarse_binary, R, N_f=None):
    """The view-culled final level.  field(P [m, 3]) -> occupancy [m].

    Returns a dict: depth [R, R] (NaN on misses), hit [R, R] bool, values
    [R, R, N_f+1] (network output where evaluated, else T), evaluated
    [R, R, N_f+1] bool, shadow [R, R, N_f+1] bool, T, i_max [R, R] (-1 on
    misses), n_eval."""
    N_c = coarse_binary.shape[0] - 1
    if N_f is None:
        N_f = 2 * N_c
    T = tentative_columns(coarse_binary, R, N_f)
    # 2. argmax along the ray (smallest index among the maxima)
    o_max = T.max(axis=2)
    i_max = np.argmax(T >= o_max[..., None], axis=2)
    # 3. shadow nodes
    k = np.arange(N_f + 1)[None, None, :]
    shadow = (o_max[..., None] >= 1.0) & (k > i_max[..., None])
    # 4. evaluate the non-shadow ambiguous nodes
    ev = (~shadow) & (T > 0.0) & (T < 1.0)
    values = T.copy()
    jj, ii, kk = np.nonzero(ev)
    c = pixel_centres(R)
    zk = 1.0 - 2.0 * np.arange(N_f + 1, dtype=F64) / N_f
    if len(jj):
        P = np.stack([c[ii], c[jj], zk[kk]], axis=1)
        values[jj, ii, kk] = field(P)
    # 5. binarize, argmax again, crossing
    inside = values >= 0.5
    hit = inside.any(axis=2)
    first = np.where(hit, np.argmax(inside, axis=2), -1)
    depth = np.full((R, R), np.nan)
    hj, hi = np.nonzero(hit)
    hk = first[hj, hi]
    at0 = hk == 0
    depth[hj[at0], hi[at0]] = 1.0
    nj, ni, nk = hj[~at0], hi[~at0], hk[~at0]
    v0 = values[nj, ni, nk - 1]
    v1 = values[nj, ni, nk]
    t = (0.5 - v0) / (v1 - v0)
    depth[nj, ni] = zk[nk - 1] + t * (zk[nk] - zk[nk - 1])
    return {"depth": depth, "hit": hit, "values": values, "evaluated": ev, "shadow": shadow,
            "T": T, "i_max": first, "n_eval": int(ev.sum())}


def render_culled(field, coarse_binary, R, col_net, occ_map, col_map, calib,
                  background=(0.0, 0.0, 0.0), N_f=None):
    """Eq. 3 over the view-culled final level: (rgb, depth, hit, result dict)."""
    res = culled_final_level(field, coarse_binary, R, N_f)
    depth, hit = res["depth"], res["hit"]
    rgb = np.empty((R, R, 3), dtype=F64)
    rgb[:] = np.asarray(background, dtype=F64)
    c = pixel_centres(R)
    jj, ii = np.nonzero(hit)
    if len(jj):
        P = np.stack([c[ii], c[jj], depth[jj, ii]], axis=1)
        rgb[jj, ii] = _field.colour(col_net, occ_map, col_map, calib, P)
    return rgb, depth, hit, res
