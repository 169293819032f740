"""Accuracy metrics used to compare reconstructions (Sec. 4 reports Chamfer and
point-to-surface distances; the paper gives no formula, so the plain
definitions are used).

* IoU over the binarized nodes of one grid: |A and B| / |A or B|.
* Chamfer distance in voxels: symmetric mean nearest-neighbour distance
  between the surface point sets of two volumes, where a volume's surface
  points are the linear 0.5 crossings on its grid edges, in units of the
  grid spacing.
* PSNR of two images in [0, 1]: 10 log10(1 / MSE).
"""
from __future__ import annotations

import numpy as np

F64 = np.float64


def iou(a, b):
    a = np.asarray(a, dtype=bool)
    b = np.asarray(b, dtype=bool)
    union = np.count_nonzero(a | b)
    return 1.0 if union == 0 else np.count_nonzero(a & b) / union


def edge_crossings(values):
    """Points where the linear interpolation of ``values`` ([z][y][x]) crosses
    0.5 on grid edges, in index units, as [n, 3] (x, y, z)."""
    v = np.asarray(values, dtype=F64)
    pts = []
    for axis in range(3):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[axis] = slice(0, -1)
        hi[axis] = slice(1, None)
        a = v[tuple(lo)]
        b = v[tuple(hi)]
        cross = (a >= 0.5) != (b >= 0.5)
        k, j, i = np.nonzero(cross)
        t = (0.5 - a[k, j, i]) / (b[k, j, i] - a[k, j, i])
        p = np.stack([i, j, k], axis=1).astype(F64)
        p[:, 2 - axis] += t
        pts.append(p)
    return np.concatenate(pts, axis=0)


def _nn_dist(src, dst):
    """Distance from every point of src to its nearest point of dst."""
    from scipy.spatial import cKDTree
    return cKDTree(dst).query(src, k=1)[0]


def chamfer_voxels(values_a, values_b):
    """Symmetric mean nearest-neighbour distance between the 0.5 edge
    crossings of two volumes on the same grid, in voxels."""
    pa = edge_crossings(values_a)
    pb = edge_crossings(values_b)
    if len(pa) == 0 or len(pb) == 0:
        return 0.0 if len(pa) == len(pb) else float("inf")
    return 0.5 * (_nn_dist(pa, pb).mean() + _nn_dist(pb, pa).mean())


def psnr(a, b, peak=1.0):
    mse = float(np.mean((np.asarray(a, F64) - np.asarray(b, F64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(peak * peak / mse)
