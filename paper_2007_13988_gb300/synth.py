"""Seeded synthetic inputs for the pixel-aligned occupancy field.

This module produces the *inputs* of the method and nothing else: a stick
figure of capsules, the channel-last feature maps an image encoder would have
produced for it, a calibration matrix, query points and MLP weights.  It holds
none of the method's arithmetic (no bilinear sampling, no MLP evaluation, no
localization, no rendering), so that the CPU oracle and the CUDA path can both
consume it without sharing any computation.

Stand-in for the paper's data.  The paper reconstructs people from real
images through a trained HRNet encoder (256 channels at 128x128, Appendix,
"Image Encoder") and trained MLPs (Sec. 3.1).  Neither images nor weights are
available, so:

* the subject is a 15-capsule stick figure inside [-1, 1]^3;
* feature channels 0-2 are the figure's orthographic front depth, back depth
  and silhouette mask sampled at texel centres, the other channels N(0, 1);
* the occupancy MLP's weights are *constructed* (not trained) so that its
  0.5 level set follows the figure: a group of "carrier" units computes
  min(front - z, back-to-z distance) and propagates it through every hidden
  layer, while the remaining units are Kaiming-uniform random and add a small
  texel-scale perturbation to the output logit.  The architecture (widths,
  skip concatenation, leaky-ReLU, sigmoid) is exactly the evaluated one.
* the colour MLP's weights are Kaiming-uniform from the seed.

All arrays are float32 and C-contiguous; every random draw comes from
``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import dataclasses
import math

import os

import numpy as np

LEAKY_SLOPE = 0.01

# --------------------------------------------------------------------------
# Capsule figure
# --------------------------------------------------------------------------

# Joint template of a standing figure facing +z (the viewer), in NDC.
_JOINTS = {
    "head_top": (0.0, 0.80, 0.00),
    "head_base": (0.0, 0.64, 0.00),
    "neck": (0.0, 0.52, 0.00),
    "chest": (0.0, 0.42, 0.00),
    "pelvis": (0.0, 0.02, 0.00),
    "hip_l": (-0.11, -0.04, 0.00),
    "hip_r": (0.11, -0.04, 0.00),
    "shoulder_l": (-0.20, 0.42, 0.00),
    "shoulder_r": (0.20, 0.42, 0.00),
    "elbow_l": (-0.36, 0.18, 0.06),
    "elbow_r": (0.36, 0.18, 0.06),
    "wrist_l": (-0.46, -0.04, 0.14),
    "wrist_r": (0.46, -0.04, 0.14),
    "knee_l": (-0.13, -0.46, 0.04),
    "knee_r": (0.13, -0.46, 0.04),
    "ankle_l": (-0.13, -0.86, -0.02),
    "ankle_r": (0.13, -0.86, -0.02),
}

# (name, joint a, joint b, nominal radius); radii lie in [0.03, 0.08].
_SEGMENTS = (
    ("head", "head_base", "head_top", 0.075),
    ("neck", "neck", "head_base", 0.040),
    ("torso", "pelvis", "chest", 0.080),
    ("hip_l", "pelvis", "hip_l", 0.060),
    ("hip_r", "pelvis", "hip_r", 0.060),
    ("shoulder_l", "chest", "shoulder_l", 0.050),
    ("shoulder_r", "chest", "shoulder_r", 0.050),
    ("upper_arm_l", "shoulder_l", "elbow_l", 0.045),
    ("upper_arm_r", "shoulder_r", "elbow_r", 0.045),
    ("forearm_l", "elbow_l", "wrist_l", 0.035),
    ("forearm_r", "elbow_r", "wrist_r", 0.035),
    ("thigh_l", "hip_l", "knee_l", 0.060),
    ("thigh_r", "hip_r", "knee_r", 0.060),
    ("shin_l", "knee_l", "ankle_l", 0.045),
    ("shin_r", "knee_r", "ankle_r", 0.045),
)

R_MIN, R_MAX = 0.03, 0.08


@dataclasses.dataclass
class Figure:
    """A union of capsules: segment endpoints a[i], b[i] and radius r[i]."""

    a: np.ndarray  # [K, 3] float64
    b: np.ndarray  # [K, 3] float64
    r: np.ndarray  # [K] float64
    names: tuple


def capsule_figure(seed: int = 0, scale: float = 1.0, jitter: float = 0.02,
                   radius_jitter: float = 0.15, perturb: np.ndarray | None = None) -> Figure:
    """Seeded 15-capsule stick figure inside [-1, 1]^3.

    Joints get N(0, jitter) offsets, radii a relative jitter (clamped to
    [0.03, 0.08]), and the whole figure is scaled about the origin by
    ``scale`` (radii scale too, then clamp).  ``perturb`` adds per-joint
    offsets on top (used for animated frames).
    """
    rng = np.random.default_rng(seed)
    names = list(_JOINTS)
    pos = np.array([_JOINTS[n] for n in names], dtype=np.float64)
    pos = pos + rng.normal(0.0, jitter, size=pos.shape)
    if perturb is not None:
        pos = pos + perturb
    pos = pos * scale
    idx = {n: i for i, n in enumerate(names)}
    a = np.stack([pos[idx[s[1]]] for s in _SEGMENTS])
    b = np.stack([pos[idx[s[2]]] for s in _SEGMENTS])
    r0 = np.array([s[3] for s in _SEGMENTS])
    r = r0 * (1.0 + rng.uniform(-radius_jitter, radius_jitter, size=r0.shape)) * scale
    r = np.clip(r, R_MIN, R_MAX)
    return Figure(a=a, b=b, r=r, names=tuple(s[0] for s in _SEGMENTS))


def _z_ray_capsule_interval(u, v, a, b, r):
    """Interval [t0, t1] of z where the ray (u, v, z) lies inside one capsule.

    u, v: arrays of the same shape.  Returns (t0, t1, hit).  The capsule is the
    union of two spheres and a finite cylinder, each convex, so the interval
    of the union is the min/max over the pieces that the ray meets.
    """
    t0 = np.full(u.shape, np.inf)
    t1 = np.full(u.shape, -np.inf)
    # Spheres at both ends.
    for c in (a, b):
        d2 = r * r - (u - c[0]) ** 2 - (v - c[1]) ** 2
        ok = d2 >= 0
        s = np.sqrt(np.where(ok, d2, 0.0))
        t0 = np.where(ok, np.minimum(t0, c[2] - s), t0)
        t1 = np.where(ok, np.maximum(t1, c[2] + s), t1)
    # Finite cylinder: |(p - a) - ((p - a).d) d|^2 = r^2 with 0 <= (p - a).d <= |ab|.
    ab = b - a
    L = float(np.linalg.norm(ab))
    if L > 0:
        d = ab / L
        # p(t) - a = w + t e_z with w = (u - a_x, v - a_y, -a_z)
        wx, wy, wz = u - a[0], v - a[1], -a[2] + np.zeros_like(u)
        wd = wx * d[0] + wy * d[1] + wz * d[2]
        # perpendicular part: q(t) = w - (w.d) d + t (e_z - d_z d)
        qx, qy, qz = wx - wd * d[0], wy - wd * d[1], wz - wd * d[2]
        ex, ey, ez = -d[2] * d[0], -d[2] * d[1], 1.0 - d[2] * d[2]
        A = ex * ex + ey * ey + ez * ez
        B = 2.0 * (qx * ex + qy * ey + qz * ez)
        Cq = qx * qx + qy * qy + qz * qz - r * r
        if A > 1e-12:
            disc = B * B - 4 * A * Cq
            ok = disc >= 0
            sq = np.sqrt(np.where(ok, disc, 0.0))
            c0 = (-B - sq) / (2 * A)
            c1 = (-B + sq) / (2 * A)
            # axial coordinate s(t) = wd + t d_z must lie in [0, L]
            if abs(d[2]) > 1e-12:
                s0 = (0.0 - wd) / d[2]
                s1 = (L - wd) / d[2]
                lo, hi = np.minimum(s0, s1), np.maximum(s0, s1)
                c0, c1 = np.maximum(c0, lo), np.minimum(c1, hi)
            else:
                inside_slab = (wd >= 0) & (wd <= L)
                ok = ok & inside_slab
            ok = ok & (c0 <= c1)
            t0 = np.where(ok, np.minimum(t0, c0), t0)
            t1 = np.where(ok, np.maximum(t1, c1), t1)
        else:
            # Axis parallel to z: the cylinder is hit iff the ray is within r of the axis.
            ok = (qx * qx + qy * qy) <= r * r
            lo = min(a[2], b[2])
            hi = max(a[2], b[2])
            t0 = np.where(ok, np.minimum(t0, lo), t0)
            t1 = np.where(ok, np.maximum(t1, hi), t1)
    hit = t1 >= t0
    return t0, t1, hit


def z_ray_figure(fig: Figure, u, v):
    """Front (max z), back (min z) and hit mask of rays along z through (u, v)."""
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    front = np.full(u.shape, -np.inf)
    back = np.full(u.shape, np.inf)
    anyhit = np.zeros(u.shape, dtype=bool)
    for k in range(len(fig.r)):
        t0, t1, hit = _z_ray_capsule_interval(u, v, fig.a[k], fig.b[k], fig.r[k])
        front = np.where(hit, np.maximum(front, t1), front)
        back = np.where(hit, np.minimum(back, t0), back)
        anyhit |= hit
    front = np.where(anyhit, front, -1.0)
    back = np.where(anyhit, back, -1.0)
    return front, back, anyhit


def texel_centres(H: int, W: int):
    """NDC (u, v) of texel centres, shape [H, W]: u = (2i+1)/W - 1, v = (2j+1)/H - 1."""
    u = (2.0 * np.arange(W) + 1.0) / W - 1.0
    v = (2.0 * np.arange(H) + 1.0) / H - 1.0
    return np.meshgrid(u, v, indexing="xy")


def feature_map(fig: Figure, H: int, W: int, C: int, seed: int) -> np.ndarray:
    """Channel-last [H][W][C] float32 map standing in for the encoder's g_O(I).

    Channels 0-2: orthographic front depth, back depth and mask at texel
    centres (misses: front = back = -1, mask = 0).  Channels 3..C-1: N(0, 1)
    drawn from ``seed + 1``.
    """
    assert C >= 3
    uu, vv = texel_centres(H, W)
    front, back, hit = z_ray_figure(fig, uu, vv)
    rng = np.random.default_rng(seed + 1)
    f = rng.standard_normal((H, W, C), dtype=np.float32)
    f[:, :, 0] = front
    f[:, :, 1] = back
    f[:, :, 2] = hit.astype(np.float32)
    return np.ascontiguousarray(f, dtype=np.float32)


def colour_map(fig: Figure, H: int, W: int, C: int, seed: int) -> np.ndarray:
    """Second channel-last map standing in for g_T(I): N(0, 1) from ``seed + 2``,
    channels 0-2 a smooth colour of the front-most capsule (0 on misses)."""
    uu, vv = texel_centres(H, W)
    rng = np.random.default_rng(seed + 2)
    m = rng.standard_normal((H, W, C), dtype=np.float32)
    best = np.full(uu.shape, -np.inf)
    col = np.zeros(uu.shape + (3,))
    palette = np.random.default_rng(seed + 3).uniform(0.1, 0.9, size=(len(fig.r), 3))
    for k in range(len(fig.r)):
        t0, t1, hit = _z_ray_capsule_interval(uu, vv, fig.a[k], fig.b[k], fig.r[k])
        nearer = hit & (t1 > best)
        best = np.where(nearer, t1, best)
        shade = 0.75 + 0.25 * np.cos(3.0 * uu + 2.0 * vv)
        col = np.where(nearer[..., None], palette[k] * shade[..., None], col)
    m[:, :, :3] = col
    return np.ascontiguousarray(m, dtype=np.float32)


# --------------------------------------------------------------------------
# Video stream: seeded figures animated by per-frame joint perturbations
# --------------------------------------------------------------------------

class StreamFigure:
    """One animated subject of a stream: its seed, scale and per-joint phases."""

    def __init__(self, seed: int, scale: float, frames: int, amp: float = 0.03):
        self.seed = seed
        self.scale = scale
        self.frames = frames
        self.amp = amp
        self.phase = np.random.default_rng(seed + 7).uniform(0.0, 2.0 * np.pi,
                                                              size=(len(_JOINTS), 3))
        self._noise_o = None
        self._noise_t = None

    def figure(self, t: int) -> Figure:
        """The figure at frame t: joints moved by amp sin(2 pi t / frames + phase)."""
        perturb = self.amp * np.sin(2.0 * np.pi * t / self.frames + self.phase)
        return capsule_figure(self.seed, scale=self.scale, jitter=0.04, perturb=perturb)

    def texture(self, H: int = 128, W: int = 128, C: int = 256):
        """(g_O, g_T) of frame 0; their N(0, 1) channels 3.. are the subject's
        fixed texture for every frame."""
        if self._noise_o is None or self._noise_o.shape != (H, W, C):
            self._noise_o = feature_map(self.figure(0), H, W, C, self.seed)
            self._noise_t = colour_map(self.figure(0), H, W, C, self.seed)
        return self._noise_o, self._noise_t

    def geometry(self, t: int, H: int = 128, W: int = 128):
        """Channels 0-2 of g_O (front depth, back depth, mask) and of g_T
        (colour) at frame t, as [H][W][3] float32 arrays."""
        fig = self.figure(t)
        uu, vv = texel_centres(H, W)
        front, back, hit = z_ray_figure(fig, uu, vv)
        geo = np.stack([front, back, hit.astype(np.float32)], axis=-1).astype(np.float32)
        return geo, colour_map(fig, H, W, 3, self.seed)

    def maps(self, t: int, H: int = 128, W: int = 128, C: int = 256):
        """(g_O, g_T) float32 maps of frame t: the fixed texture with the
        frame's geometry and colour channels."""
        g_o, g_t = (m.copy() for m in self.texture(H, W, C))
        geo, col = self.geometry(t, H, W)
        g_o[:, :, :3] = geo
        g_t[:, :, :3] = col
        return g_o, g_t


def stream(n_figures: int = 8, frames: int = 64, seed: int = 100,
           scale_range=(0.5, 1.3)) -> list:
    """The subjects of a video stream: independent seeded figures with scales
    uniform in scale_range (so their surface-cell fractions differ)."""
    rng = np.random.default_rng(seed)
    scales = rng.uniform(scale_range[0], scale_range[1], size=n_figures)
    return [StreamFigure(seed + 1000 * (i + 1), float(scales[i]), frames) for i in range(n_figures)]


# --------------------------------------------------------------------------
# Calibration and query points
# --------------------------------------------------------------------------

def calib_identity() -> np.ndarray:
    """3x4 affine map volume NDC -> input view (u, v, z): the identity."""
    c = np.zeros((3, 4), dtype=np.float32)
    c[0, 0] = c[1, 1] = c[2, 2] = 1.0
    return c


def calib_yaw(deg: float, scale: float = 1.0) -> np.ndarray:
    """Orthographic input view rotated by ``deg`` about the y axis."""
    t = math.radians(deg)
    c = np.zeros((3, 4), dtype=np.float64)
    c[0, 0], c[0, 2] = math.cos(t), math.sin(t)
    c[1, 1] = 1.0
    c[2, 0], c[2, 2] = -math.sin(t), math.cos(t)
    c[:, :3] *= scale
    return c.astype(np.float32)


def distill_points(fig: Figure, n: int, seed: int, near_frac: float = 0.5,
                   sigma: float = 0.02) -> np.ndarray:
    """Training points for distillation: a fraction near the figure's surface
    (a point on a random capsule's surface plus N(0, sigma) jitter, the
    importance sampling PIFu trains with) and the rest uniform in [-1, 1]^3."""
    rng = np.random.default_rng(seed)
    n_near = int(n * near_frac)
    k = rng.integers(0, len(fig.r), n_near)
    t = rng.uniform(0, 1, n_near)[:, None]
    axis = fig.a[k] + t * (fig.b[k] - fig.a[k])
    u = rng.standard_normal((n_near, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    near = axis + fig.r[k][:, None] * u + rng.normal(0, sigma, (n_near, 3))
    uni = rng.uniform(-1, 1, (n - n_near, 3))
    P = np.concatenate([near, uni], 0)
    return np.clip(P[rng.permutation(n)], -1, 1).astype(np.float32)


def query_points(n: int, seed: int) -> np.ndarray:
    """n points uniform in [-1, 1]^3, float32 [n, 3]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(n, 3)).astype(np.float32)


# --------------------------------------------------------------------------
# MLP weights
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Net:
    """An MLP of the concatenation family (Sec. 3.1; Appendix, Pixel-aligned 3D
    Lifting, the "MLP" variant): layer l maps [h_{l-1}, x] (if l is in
    ``skip``) or h_{l-1} to width[l]; leaky-ReLU between layers; the last
    layer's activation is ``out_act`` ("sigmoid" or "tanh01")."""

    d_in: int
    widths: tuple           # output width of every layer, last = n_out
    skip: tuple             # 0-based indices of layers whose input is [h, x]
    W: list                 # W[l]: float32 [width[l], fan_in(l)], row-major
    b: list                 # b[l]: float32 [width[l]]
    out_act: str
    slope: float = LEAKY_SLOPE

    def fan_in(self, l: int) -> int:
        prev = self.d_in if l == 0 else self.widths[l - 1]
        return prev + (self.d_in if l in self.skip else 0)

    @property
    def n_params(self) -> int:
        return sum(w.size + bb.size for w, bb in zip(self.W, self.b))

    def flops_per_point(self) -> int:
        return sum(2 * w.shape[0] * w.shape[1] for w in self.W)


def _kaiming_uniform(rng, n_out, n_in, gain=math.sqrt(2.0 / (1.0 + LEAKY_SLOPE ** 2))):
    bound = gain * math.sqrt(3.0 / n_in)
    return rng.uniform(-bound, bound, size=(n_out, n_in))


def occupancy_net(C: int, widths, skip, seed: int, logit_scale: float,
                  noise_logit: float = 0.25, carriers: int = 16,
                  mask_gain: float = 1.0) -> Net:
    """Constructed occupancy MLP f_O whose 0.5 level set follows the figure.

    Input x = [phi_0 .. phi_{C-1}, z] with phi_0 = front depth f, phi_1 = back
    depth b, phi_2 = mask.  The field's signed distance is

        M = min(f - z, z - b, mask_gain (mask - 1/2)),

    positive inside the figure and clearly negative off the silhouette.  With
    leaky-ReLU g (slope s), g(t) - g(-t) = (1+s) t and g(t) + g(-t) = (1-s)|t|,
    so a +/- pair of units carries a signed value or its magnitude linearly:

    * layer 0 carries A = f - b, B = f + b - 2z and Cm = mask_gain (mask - 1/2),
      giving m = min(f - z, z - b) = A/2 - |B|/2 and Cm as linear read-outs;
    * layer 1 carries S = m + Cm and D = m - Cm, so M = S/2 - |D|/2;
    * later hidden layers pass M on in +/- pairs;
    * the output logit is ``logit_scale * M`` plus a random projection of the
      non-carrier units scaled to about ``noise_logit``.

    Every unit pair is replicated ``carriers`` times with random gains in
    [0.5, 1.5]; all other weights are Kaiming-uniform random.
    """
    rng = np.random.default_rng(seed)
    s = LEAKY_SLOPE
    d_in = C + 1
    widths = tuple(widths)
    L = len(widths)
    assert widths[-1] == 1 and L >= 3
    R = carriers
    net_W, net_b = [], []
    for l in range(L):
        fan = (d_in if l == 0 else widths[l - 1]) + (d_in if l in skip else 0)
        n_out = widths[l]
        if l == L - 1:
            W = np.zeros((n_out, fan))
            b = np.zeros(n_out)
        else:
            W = _kaiming_uniform(rng, n_out, fan)
            b = rng.uniform(-0.1, 0.1, size=n_out)
        net_W.append(W)
        net_b.append(b)

    def pairs(W, b, first, inputs_w, prev_width):
        """Write R +/- unit pairs carrying the linear form ``inputs_w`` (over
        the previous layer's units, length prev_width) at rows first.. and
        return the read-out vectors for the signed value and the magnitude."""
        g = rng.uniform(0.5, 1.5, size=R)
        rows = slice(first, first + 2 * R)
        W[rows, :] = 0.0
        b[rows] = 0.0
        signed = np.zeros(W.shape[0])
        mag = np.zeros(W.shape[0])
        for r in range(R):
            W[first + r, :prev_width] = g[r] * inputs_w
            W[first + R + r, :prev_width] = -g[r] * inputs_w
            signed[first + r] = 1.0 / ((1 + s) * g[r] * R)
            signed[first + R + r] = -1.0 / ((1 + s) * g[r] * R)
            mag[first + r] = 1.0 / ((1 - s) * g[r] * R)
            mag[first + R + r] = 1.0 / ((1 - s) * g[r] * R)
        return signed, mag

    # Layer 0 over x: A, B, Cm.
    iz = C
    wA = np.zeros(d_in); wA[0], wA[1] = 1.0, -1.0
    wB = np.zeros(d_in); wB[0], wB[1], wB[iz] = 1.0, 1.0, -2.0
    wC = np.zeros(d_in); wC[2] = mask_gain
    assert 6 * R <= widths[0]
    A_s, _ = pairs(net_W[0], net_b[0], 0, wA, d_in)
    _, B_m = pairs(net_W[0], net_b[0], 2 * R, wB, d_in)
    C_s, _ = pairs(net_W[0], net_b[0], 4 * R, wC, d_in)
    net_b[0][4 * R:6 * R] = 0.0
    # Cm = mask_gain * (mask - 1/2): fold the -1/2 into the bias of the C pair.
    for r in range(R):
        g = net_W[0][4 * R + r, 2] / mask_gain
        net_b[0][4 * R + r] = -0.5 * mask_gain * g
        net_b[0][5 * R + r] = 0.5 * mask_gain * g
    m_lin = 0.5 * A_s - 0.5 * B_m          # read-out of m from layer-0 units
    c_lin = C_s                            # read-out of Cm
    # Layer 1: S = m + Cm, D = m - Cm.
    assert 4 * R <= widths[1]
    S_s, _ = pairs(net_W[1], net_b[1], 0, m_lin + c_lin, widths[0])
    _, D_m = pairs(net_W[1], net_b[1], 2 * R, m_lin - c_lin, widths[0])
    M_lin = 0.5 * S_s - 0.5 * D_m          # read-out of M from layer-1 units
    n_carrier = 4 * R
    # Layers 2 .. L-2 pass M on.
    for l in range(2, L - 1):
        assert 2 * R <= widths[l]
        M_lin, _ = pairs(net_W[l], net_b[l], 0, M_lin, widths[l - 1])
        n_carrier = 2 * R
    # Output: logit = scale * M + noise projection of the non-carrier units.
    prev = widths[L - 2]
    WL = net_W[L - 1]
    WL[0, :prev] = logit_scale * M_lin
    n_rand = prev - n_carrier
    proj = rng.uniform(-1.0, 1.0, size=n_rand) * math.sqrt(3.0 / n_rand)
    WL[0, n_carrier:prev] += noise_logit * proj
    net_b[L - 1][:] = 0.0
    return Net(d_in=d_in, widths=widths, skip=tuple(skip),
               W=[np.ascontiguousarray(w, dtype=np.float32) for w in net_W],
               b=[np.ascontiguousarray(bb, dtype=np.float32) for bb in net_b],
               out_act="sigmoid")


def colour_net(d_in: int, widths, skip, seed: int) -> Net:
    """Colour MLP f_T (Sec. 3.1, Eq. 2; Appendix: 1024-512-256-128-3, skips,
    leaky-ReLU, tanh on the last layer).  Kaiming-uniform weights from seed."""
    rng = np.random.default_rng(seed)
    Ws, bs = [], []
    widths = tuple(widths)
    for l, n_out in enumerate(widths):
        fan = (d_in if l == 0 else widths[l - 1]) + (d_in if l in skip else 0)
        if l == len(widths) - 1:
            W = rng.uniform(-1, 1, size=(n_out, fan)) * math.sqrt(3.0 / fan)
            b = rng.uniform(-0.2, 0.2, size=n_out)
        else:
            W = _kaiming_uniform(rng, n_out, fan)
            b = rng.uniform(-0.1, 0.1, size=n_out)
        Ws.append(np.ascontiguousarray(W, dtype=np.float32))
        bs.append(np.ascontiguousarray(b, dtype=np.float32))
    return Net(d_in=d_in, widths=widths, skip=tuple(skip), W=Ws, b=bs, out_act="tanh01")


@dataclasses.dataclass
class CbnNet:
    """f_O of the paper's final model (Appendix, "Depth Representation" and
    "Pixel-aligned 3D Lifting"): the depth P_z enters as its soft one-hot
    vector Z of ``n_z`` channels (Eq. 7) through a linear layer of ``width``
    outputs, followed by ``n_blocks`` blocks of conditional batch
    normalization (Eq. 8) with gamma(c) = Gg c + gg and beta(c) = Gb c + gb
    linear in the pixel-aligned feature c, ReLU, and a linear layer; the last
    block's linear layer has one output, the logit.  mu / var are the
    normalization's running statistics (inference)."""

    C: int
    n_z: int
    width: int
    Wz: np.ndarray          # [width][n_z]
    bz: np.ndarray          # [width]
    Gg: list                # per block [width][C]
    gg: list                # per block [width]
    Gb: list                # per block [width][C]
    gb: list                # per block [width]
    mu: list                # per block [width]
    var: list               # per block [width]
    W: list                 # per block [width][width], the last [1][width]
    b: list                 # per block [width], the last [1]
    eps: float = 1e-5
    out_act: str = "sigmoid"
    kind: str = "cbn"

    @property
    def n_blocks(self) -> int:
        return len(self.W)

    @property
    def n_params(self) -> int:
        arrs = [self.Wz, self.bz] + self.Gg + self.gg + self.Gb + self.gb + self.W + self.b
        return sum(a.size for a in arrs)

    def flops_per_point(self) -> int:
        mats = [self.Wz] + self.Gg + self.Gb + self.W
        return sum(2 * m.shape[0] * m.shape[1] for m in mats)


def occupancy_cbn_net(C: int, seed: int, logit_scale: float, width: int = 128,
                      n_blocks: int = 5, n_z: int = 64, noise_logit: float = 0.25,
                      carriers: int = 8, mask_gain: float = 1.0) -> CbnNet:
    """Constructed CBN + SoftZ occupancy network whose 0.5 level set follows
    the figure: its logit is ``logit_scale * M`` plus a texel-scale random
    perturbation, M = min(f - z, z - b, mask_gain (mask - 1/2)) as in
    ``occupancy_net``.

    Conditional batch normalization acts channel by channel, so a carrier unit
    of block i reads channel u of h_{i-1} (normalized with the running
    statistics) scaled by a constant gamma, plus beta(c), linear in the
    feature; ReLU pairs carry values as in ``occupancy_net`` (slope 0:
    r(t) - r(-t) = t, r(t) + r(-t) = |t|):

    * the SoftZ layer gives z exactly on the channels whose Wz row is
      zeta (2 j / (n_z - 1) - 1) (the two weights of Z sum to 1 and their
      centroid is (n_z - 1) P'_z);
    * block 1 carries A = f - b and Cm = mask_gain (mask - 1/2) through beta
      alone and B = f + b - 2z through gamma z + beta;
    * the linear layer after it forms S = m + Cm and D = m - Cm,
      m = A/2 - |B|/2, block 2 carries them, and M = S/2 - |D|/2;
    * blocks 3 .. n_blocks pass M on; the last linear layer reads it out.

    Every unit pair is replicated ``carriers`` times with gains in [0.5, 1.5];
    the other units are random (gamma near 1, small beta(c), Kaiming linear
    layers, running statistics mu in [-0.2, 0.2], var in [0.5, 1.5])."""
    rng = np.random.default_rng(seed)
    R = carriers
    K = width
    assert 6 * R <= K and n_blocks >= 3
    relu_gain = math.sqrt(2.0)
    Wz = _kaiming_uniform(rng, K, n_z, relu_gain)
    bz = rng.uniform(-0.1, 0.1, size=K)
    Gg, gg, Gb, gb, mu, var, W, b = [], [], [], [], [], [], [], []
    for i in range(n_blocks):
        Gg.append(0.1 * rng.uniform(-1, 1, size=(K, C)) * math.sqrt(3.0 / C))
        gg.append(np.ones(K))
        Gb.append(0.1 * rng.uniform(-1, 1, size=(K, C)) * math.sqrt(3.0 / C))
        gb.append(rng.uniform(-0.1, 0.1, size=K))
        mu.append(rng.uniform(-0.2, 0.2, size=K))
        var.append(rng.uniform(0.5, 1.5, size=K))
        if i < n_blocks - 1:
            W.append(_kaiming_uniform(rng, K, K, relu_gain))
            b.append(rng.uniform(-0.1, 0.1, size=K))
        else:
            W.append(np.zeros((1, K)))
            b.append(np.zeros(1))
    # float32 running statistics: the construction's constants use the
    # stored values
    mu = [m.astype(np.float32).astype(np.float64) for m in mu]
    var = [v.astype(np.float32).astype(np.float64) for v in var]
    scale = [1.0 / np.sqrt(v + 1e-5) for v in var]

    def constant_gamma(i, u, gamma, beta):
        Gg[i][u, :] = 0.0
        gg[i][u] = gamma
        Gb[i][u, :] = 0.0
        gb[i][u] = beta

    def readouts(first, gains):
        """Signed and magnitude read-outs (length K) of the R pairs at units
        first .. first + 2R (first R the + units)."""
        signed = np.zeros(K)
        mag = np.zeros(K)
        for r in range(R):
            signed[first + r] = 1.0 / (gains[r] * R)
            signed[first + R + r] = -1.0 / (gains[r] * R)
            mag[first + r] = 1.0 / (gains[r] * R)
            mag[first + R + r] = 1.0 / (gains[r] * R)
        return signed, mag

    # block 0 (the first CBN block)
    gA, gB, gC = (rng.uniform(0.5, 1.5, size=R) for _ in range(3))
    for r in range(R):
        for sgn, off in ((1.0, 0), (-1.0, R)):
            u = off + r                       # A = f - b through beta
            constant_gamma(0, u, 0.0, 0.0)
            Gb[0][u, 0], Gb[0][u, 1] = sgn * gA[r], -sgn * gA[r]
            u = 2 * R + off + r               # B = f + b - 2z
            zeta = rng.uniform(0.5, 1.5)
            Wz[u, :] = zeta * (2.0 * np.arange(n_z) / (n_z - 1) - 1.0)
            bz[u] = 0.0
            gam = -2.0 * sgn * gB[r] / (scale[0][u] * zeta)
            constant_gamma(0, u, gam, -2.0 * sgn * gB[r] * mu[0][u] / zeta)
            Gb[0][u, 0], Gb[0][u, 1] = sgn * gB[r], sgn * gB[r]
            u = 4 * R + off + r               # Cm = mask_gain (mask - 1/2)
            constant_gamma(0, u, 0.0, -0.5 * sgn * gC[r] * mask_gain)
            Gb[0][u, 2] = sgn * gC[r] * mask_gain
    A_s, _ = readouts(0, gA)
    _, B_m = readouts(2 * R, gB)
    C_s, _ = readouts(4 * R, gC)
    m_lin = 0.5 * A_s - 0.5 * B_m
    forms = [m_lin + C_s, m_lin - C_s]        # S, D over block 0's units

    def carry(i, form_rows):
        """Linear layer i - 1 writes each form of form_rows onto 2R channels
        (gains lambda); block i carries it in R +/- pairs; returns the
        read-out gains."""
        gains = []
        for q, form in enumerate(form_rows):
            g = rng.uniform(0.5, 1.5, size=R)
            gains.append(g)
            for r in range(R):
                for sgn, off in ((1.0, 0), (-1.0, R)):
                    u = 2 * R * q + off + r
                    lam = rng.uniform(0.5, 1.5)
                    W[i - 1][u, :] = lam * form
                    b[i - 1][u] = 0.0
                    constant_gamma(i, u, sgn * g[r] / (scale[i][u] * lam),
                                   sgn * g[r] * mu[i][u] / lam)
        return gains

    gS, gD = carry(1, forms)
    S_s, _ = readouts(0, gS)
    _, D_m = readouts(2 * R, gD)
    M_lin = 0.5 * S_s - 0.5 * D_m
    for i in range(2, n_blocks):
        (gM,) = carry(i, [M_lin])
        M_lin, _ = readouts(0, gM)
    n_rand = K - 2 * R
    proj = rng.uniform(-1.0, 1.0, size=n_rand) * math.sqrt(3.0 / n_rand)
    W[-1][0, :] = logit_scale * M_lin
    W[-1][0, 2 * R:] += noise_logit * proj
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return CbnNet(C=C, n_z=n_z, width=K, Wz=f32(Wz), bz=f32(bz), Gg=[f32(a) for a in Gg],
                  gg=[f32(a) for a in gg], Gb=[f32(a) for a in Gb], gb=[f32(a) for a in gb],
                  mu=[f32(a) for a in mu], var=[f32(a) for a in var], W=[f32(a) for a in W],
                  b=[f32(a) for a in b])


# --------------------------------------------------------------------------
# Workload presets
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    fig: Figure
    occ_map: np.ndarray        # [H][W][C_O] float32
    col_map: np.ndarray | None  # [H][W][C_T] float32 or None (colour MLP reads only g_O)
    calib: np.ndarray          # [3][4] float32
    occ_net: Net
    col_net: Net
    n0: int                    # coarsest level resolution (cells per axis)
    num_levels: int
    render: int                # R x R render


def tiny(seed: int = 0, calib=None) -> Workload:
    """Plain method, tiny: C = 32 at 64x64, MLP 33-128-64-1, levels 16->32->64,
    64x64 render, colour MLP 33-128-64-3 reading g_O only."""
    fig = capsule_figure(seed)
    C = 32
    occ = feature_map(fig, 64, 64, C, seed)
    onet = occupancy_net(C, (128, 64, 1), (), seed + 10, logit_scale=0.65 * 64, carriers=8)
    cnet = colour_net(C + 1, (128, 64, 3), (), seed + 11)
    return Workload("tiny 16^3->64^3, 64^2 render, C=32 FP32", fig, occ, None,
                    calib_identity() if calib is None else calib, onet, cnet,
                    n0=16, num_levels=3, render=64)


def full(seed: int = 0, calib=None, num_levels: int = 4, n0: int = 32, render: int = 512) -> Workload:
    """Plain method at full size: 256x128x128 FP32 maps, f_O 257-1024-512-256-128-1
    with the input re-concatenated at layers 2-4, f_T 513-1024-512-256-128-3,
    levels 32^3 -> 256^3, 512x512 render."""
    fig = capsule_figure(seed)
    C = 256
    occ = feature_map(fig, 128, 128, C, seed)
    col = colour_map(fig, 128, 128, C, seed)
    n_fine = n0 << (num_levels - 1)
    onet = occupancy_net(C, (1024, 512, 256, 128, 1), (1, 2, 3), seed + 10,
                         logit_scale=0.65 * n_fine, carriers=16)
    cnet = colour_net(2 * C + 1, (1024, 512, 256, 128, 3), (1, 2, 3), seed + 11)
    return Workload(f"full {n0}^3->{n_fine}^3, {render}^2 render, C=256 FP32", fig, occ, col,
                    calib_identity() if calib is None else calib, onet, cnet,
                    n0=n0, num_levels=num_levels, render=render)


def fitted_occupancy_net(which: str, base: Net) -> Net:
    """f_O of the ``which`` ("tiny" or "full") workload fitted to its seed-0
    figure: the architecture of ``base``, the stored weights of
    tests/golden/fitted_occ_<which>.npz (written once by
    tests/golden/fit_occupancy.py: 2000 Adam steps of BCE on 65,536 points
    against the capsules' occupancy)."""
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests",
                        "golden", "fitted_occ_%s.npz" % which)
    z = np.load(path)
    L = len(base.widths)
    W = [np.ascontiguousarray(z["W%d" % l], dtype=np.float32) for l in range(L)]
    b = [np.ascontiguousarray(z["b%d" % l], dtype=np.float32) for l in range(L)]
    for l in range(L):
        assert W[l].shape == (base.widths[l], base.fan_in(l)), (which, l, W[l].shape)
    return Net(base.d_in, base.widths, base.skip, W, b, base.out_act, base.slope)


def tiny_fitted(calib=None) -> Workload:
    """The tiny workload (seed 0) with its fitted f_O."""
    w = tiny(0, calib)
    w.occ_net = fitted_occupancy_net("tiny", w.occ_net)
    w.name = "tiny 16^3->64^3, 64^2 render, C=32 FP32, fitted f_O"
    return w


def full_fitted(calib=None, num_levels: int = 4, n0: int = 32, render: int = 512) -> Workload:
    """The full-size workload (seed 0) with its fitted f_O."""
    w = full(0, calib, num_levels=num_levels, n0=n0, render=render)
    w.occ_net = fitted_occupancy_net("full", w.occ_net)
    w.name = w.name + ", fitted f_O"
    return w


def tiny_cbn(seed: int = 0, calib=None) -> Workload:
    """The tiny workload with the CBN + SoftZ f_O (C = 32, width 64, four
    blocks, n_z = 64), levels 16 -> 32 -> 64, 64x64 render."""
    w = tiny(seed, calib)
    w.occ_net = occupancy_cbn_net(32, seed + 12, logit_scale=0.65 * 64, width=64, n_blocks=4,
                                  carriers=4)
    w.name = "tiny CBN+SoftZ 16^3->64^3, 64^2 render, C=32 FP32"
    return w


def full_cbn(seed: int = 0, calib=None, num_levels: int = 4, n0: int = 32,
             render: int = 512) -> Workload:
    """The full-size frame with the paper's final f_O: SoftZ (64) -> 128, five
    CBN blocks of 128 channels conditioned on the 256-channel feature, one
    output; the colour MLP and the maps are those of ``full``."""
    w = full(seed, calib, num_levels, n0, render)
    n_fine = n0 << (num_levels - 1)
    w.occ_net = occupancy_cbn_net(256, seed + 12, logit_scale=0.65 * n_fine)
    w.name = f"full CBN+SoftZ {n0}^3->{n_fine}^3, {render}^2 render, C=256 FP32"
    return w
