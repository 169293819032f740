"""Eq. 1 and Eq. 2 of Sec. 3.1 in float64.

O(P) = f_O(Phi(P_xy, g_O(I)), P_z)                                  (Eq. 1)
T(P) = f_T(Phi(P_xy, g_T(I)), Phi(P_xy, g_O(I)), P_z)               (Eq. 2)

Readings where the paper is silent (each also listed in the design notes):
* P is in the volume's NDC; a 3x4 affine calibration maps it to the input
  view, (u, v, P_z) = C [P, 1] (orthographic / weak perspective, Sec. 3.1 and
  Sec. 4 data rendering).
* Phi is bilinear sampling (Sec. 3.1 cites the spatial transformer) with
  texel centres at u = (2i+1)/W - 1 ("align corners" false), row index
  increasing with v, indices clamped to the border.
* The MLP input is [phi, P_z] for f_O and [phi_T, phi_O, P_z] for f_T, in the
  argument order of Eq. 1 / Eq. 2.  A skip layer's input is [h, x].
* Hidden activation leaky-ReLU (slope stored with the weights; the paper
  states LeakyReLU for f_T without a slope), sigmoid on f_O's output, tanh on
  f_T's output mapped to [0, 1] as (t + 1) / 2.

* The paper's final f_O (Appendix) lifts the feature with conditional batch
  normalization and takes the depth as a soft one-hot vector (Eq. 7, Eq. 8):
  ``soft_z`` and ``cbn_mlp``.

Pins: tests/test_oracle_field.py (texel-centre sampling returns stored values,
a map linear in (u, v) is reproduced exactly, border clamping, MLP against an
explicit per-neuron loop, the Table A1 flop count; the colour mapping, input
order and a constructed colour network's closed form end to end; SoftZ
closed forms, batch-normalization statistics, a hand-built CBN network, the
constructed CBN network's closed form).
"""
from __future__ import annotations

import numpy as np

F64 = np.float64


def project(calib, P):
    """(u, v, z_in) = C [P, 1] for P [M, 3]; C is the 3x4 calibration."""
    C = np.asarray(calib, dtype=F64).reshape(3, 4)
    P = np.asarray(P, dtype=F64)
    q = P @ C[:, :3].T + C[:, 3]
    return q[:, 0], q[:, 1], q[:, 2]


def sample_bilinear(fmap, u, v):
    """Phi: bilinear sample of a channel-last [H][W][C] map at NDC (u, v).

    Texel (i, j) has its centre at u = (2i+1)/W - 1, v = (2j+1)/H - 1, so the
    continuous texel coordinate is s = ((u + 1) W - 1) / 2.  The four taps
    are (i0, j0), (i0+1, j0), (i0, j0+1), (i0+1, j0+1) with i0 = floor(s),
    weights (1-a)(1-b), a(1-b), (1-a)b, ab; tap indices are clamped to the
    map (border replicate) while the weights are kept.
    """
    F = np.asarray(fmap)
    H, W, _ = F.shape
    u = np.asarray(u, dtype=F64)
    v = np.asarray(v, dtype=F64)
    s = ((u + 1.0) * W - 1.0) / 2.0
    t = ((v + 1.0) * H - 1.0) / 2.0
    i0 = np.floor(s)
    j0 = np.floor(t)
    a = (s - i0)[:, None]
    b = (t - j0)[:, None]
    i0 = i0.astype(np.int64)
    j0 = j0.astype(np.int64)
    i1 = np.clip(i0 + 1, 0, W - 1)
    j1 = np.clip(j0 + 1, 0, H - 1)
    i0 = np.clip(i0, 0, W - 1)
    j0 = np.clip(j0, 0, H - 1)
    f00 = F[j0, i0].astype(F64)
    f10 = F[j0, i1].astype(F64)
    f01 = F[j1, i0].astype(F64)
    f11 = F[j1, i1].astype(F64)
    return (1 - a) * (1 - b) * f00 + a * (1 - b) * f10 + (1 - a) * b * f01 + a * b * f11


def leaky_relu(x, slope):
    return np.where(x >= 0, x, slope * x)


def mlp(net, x):
    """Forward pass of a concatenation MLP in float64 (returns the last
    layer's pre-activation).  Layer l computes W_l z + b_l with z = [h, x] if
    l is a skip layer, else h; leaky-ReLU after every layer but the last."""
    x = np.asarray(x, dtype=F64)
    h = x
    L = len(net.W)
    for l in range(L):
        z = np.concatenate([h, x], axis=1) if (l in net.skip and l > 0) else h
        h = z @ np.asarray(net.W[l], dtype=F64).T + np.asarray(net.b[l], dtype=F64)
        if l < L - 1:
            h = leaky_relu(h, net.slope)
    return h


def sigmoid(t):
    return 1.0 / (1.0 + np.exp(-t))


def soft_z(pz, n):
    """Soft one-hot depth Z (Appendix, "Depth Representation", Eq. 7): with
    P'_z = (P_z + 1) / 2 and x = (n - 1) P'_z, Z_i = 1 + floor(x) - x at
    i = floor(x), x - floor(x) at i = floor(x) + 1, 0 elsewhere.
    Readings: P'_z is clamped to [0, 1] (Eq. 7 is stated for -1 <= P_z <= 1);
    at P'_z = 1 the second index is n, whose weight is 0, and is dropped."""
    p = np.clip(0.5 * (np.asarray(pz, dtype=F64) + 1.0), 0.0, 1.0)
    x = (n - 1) * p
    i = np.floor(x).astype(np.int64)
    Z = np.zeros((len(p), n), dtype=F64)
    rows = np.arange(len(p))
    Z[rows, i] = 1.0 + i - x
    k = i + 1 < n
    Z[rows[k], i[k] + 1] = x[k] - i[k]
    return Z


def cbn_mlp(net, c, Z):
    """The CBN lifting of the Appendix ("Pixel-aligned 3D Lifting", Eq. 8) in
    float64; returns the logit.  h_0 = Wz Z + bz; block i normalizes its
    input with the running statistics, f = gamma_i(c) (h - mu_i) /
    sqrt(var_i + eps) + beta_i(c) with gamma_i(c) = Gg_i c + gg_i and
    beta_i(c) = Gb_i c + gb_i, applies ReLU, then its linear layer."""
    c = np.asarray(c, dtype=F64)
    h = np.asarray(Z, dtype=F64) @ np.asarray(net.Wz, F64).T + np.asarray(net.bz, F64)
    for i in range(net.n_blocks):
        norm = (h - np.asarray(net.mu[i], F64)) / np.sqrt(np.asarray(net.var[i], F64) + net.eps)
        gamma = c @ np.asarray(net.Gg[i], F64).T + np.asarray(net.gg[i], F64)
        beta = c @ np.asarray(net.Gb[i], F64).T + np.asarray(net.gb[i], F64)
        a = np.maximum(gamma * norm + beta, 0.0)
        h = a @ np.asarray(net.W[i], F64).T + np.asarray(net.b[i], F64)
    return h


def occupancy_logit(net, occ_map, calib, P, chunk=8192):
    """Pre-sigmoid value of f_O at points P [M, 3] (Eq. 1): the concatenation
    MLP on [phi, P_z], or (a network of kind "cbn") the CBN lifting
    conditioned on phi with the SoftZ depth."""
    P = np.asarray(P, dtype=F64).reshape(-1, 3)
    out = np.empty(len(P), dtype=F64)
    for s in range(0, len(P), chunk):
        u, v, z = project(calib, P[s:s + chunk])
        phi = sample_bilinear(occ_map, u, v)
        if getattr(net, "kind", "mlp") == "cbn":
            out[s:s + chunk] = cbn_mlp(net, phi, soft_z(z, net.n_z))[:, 0]
        else:
            x = np.concatenate([phi, z[:, None]], axis=1)
            out[s:s + chunk] = mlp(net, x)[:, 0]
    return out


def occupancy(net, occ_map, calib, P, chunk=8192):
    """O(P) in [0, 1] (Eq. 1): sigmoid of f_O at the sampled feature and depth."""
    return sigmoid(occupancy_logit(net, occ_map, calib, P, chunk))


def colour(net, occ_map, col_map, calib, P, chunk=8192):
    """T(P, I) as RGB in [0, 1] (Eq. 2): f_T on [phi_T, phi_O, P_z], tanh output
    mapped by (t + 1) / 2.  With no colour map f_T reads [phi_O, P_z]."""
    P = np.asarray(P, dtype=F64).reshape(-1, 3)
    out = np.empty((len(P), 3), dtype=F64)
    for s in range(0, len(P), chunk):
        u, v, z = project(calib, P[s:s + chunk])
        parts = []
        if col_map is not None:
            parts.append(sample_bilinear(col_map, u, v))
        parts.append(sample_bilinear(occ_map, u, v))
        parts.append(z[:, None])
        t = mlp(net, np.concatenate(parts, axis=1))
        out[s:s + chunk] = (np.tanh(t) + 1.0) / 2.0
    return out


def capsule_sdf(a, b, r, P):
    """Signed distance to a union of capsules (segment a_k b_k, radius r_k)."""
    P = np.asarray(P, dtype=F64).reshape(-1, 3)
    d = np.full(len(P), np.inf)
    for ak, bk, rk in zip(np.asarray(a, F64), np.asarray(b, F64), np.asarray(r, F64)):
        ab = bk - ak
        L2 = float(ab @ ab)
        t = np.clip(((P - ak) @ ab) / L2, 0.0, 1.0) if L2 > 0 else np.zeros(len(P))
        q = ak + t[:, None] * ab
        d = np.minimum(d, np.linalg.norm(P - q, axis=1) - rk)
    return d


def capsule_occupancy(a, b, r, P, tau):
    """Analytic stand-in for f_O: sigmoid(-sdf / tau).  Used only to pin the
    localization and the render against closed forms."""
    return sigmoid(-capsule_sdf(a, b, r, P) / tau)
