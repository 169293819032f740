"""Pins of the oracle's field (Eq. 1 / Eq. 2, Sec. 3.1) to facts that do not
come from the oracle itself: closed forms of bilinear sampling, hand-built
networks with known outputs, the network that the generator constructs to
compute a closed-form signed distance, and the paper's Table A1 cost."""
import math
import os

import numpy as np
import pytest

from oracle import field
from paper_2007_13988_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def texel_uv(i, j, W, H):
    return (2.0 * i + 1.0) / W - 1.0, (2.0 * j + 1.0) / H - 1.0


def test_texel_centres_return_stored_values():
    # power-of-two sizes, as the encoder's maps: texel centres are exact in
    # binary floating point, so the sample is the stored value bit for bit
    rng = np.random.default_rng(1)
    F = rng.standard_normal((8, 16, 5)).astype(np.float32)
    jj, ii = np.meshgrid(np.arange(8), np.arange(16), indexing="ij")
    u, v = texel_uv(ii.ravel(), jj.ravel(), 16, 8)
    out = field.sample_bilinear(F, u, v)
    np.testing.assert_array_equal(out, F.reshape(-1, 5).astype(np.float64))


def test_linear_map_reproduced_in_interior():
    # A map linear in the texel coordinates is reproduced exactly by bilinear
    # interpolation anywhere between the outermost texel centres.
    H, W = 6, 8
    jj, ii = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    alpha, beta, gamma = 0.75, -1.25, 0.5
    F = (alpha * ii + beta * jj + gamma)[..., None].astype(np.float64)
    rng = np.random.default_rng(2)
    s = rng.uniform(0, W - 1, 200)
    t = rng.uniform(0, H - 1, 200)
    u = (2 * s + 1) / W - 1
    v = (2 * t + 1) / H - 1
    out = field.sample_bilinear(F, u, v)[:, 0]
    np.testing.assert_allclose(out, alpha * s + beta * t + gamma, rtol=0, atol=1e-12)


def test_border_clamp_and_row_direction():
    H, W = 4, 5
    F = np.arange(H * W, dtype=np.float64).reshape(H, W, 1)
    # Far outside on each side: the nearest edge texel (border replicate).
    out = field.sample_bilinear(F, np.array([-5.0, 5.0, -5.0, 5.0]),
                                np.array([-5.0, -5.0, 5.0, 5.0]))[:, 0]
    np.testing.assert_array_equal(out, [F[0, 0, 0], F[0, W - 1, 0], F[H - 1, 0, 0], F[H - 1, W - 1, 0]])
    # Row index grows with v: v = +1 - 1/H is the centre of the last row.
    u, v = texel_uv(2, H - 1, W, H)
    assert field.sample_bilinear(F, np.array([u]), np.array([v]))[0, 0] == F[H - 1, 2, 0]
    # Half-way between two texel centres along u: their mean.
    u0, v0 = texel_uv(1, 2, W, H)
    u1, _ = texel_uv(2, 2, W, H)
    mid = field.sample_bilinear(F, np.array([(u0 + u1) / 2]), np.array([v0]))[0, 0]
    assert mid == (F[2, 1, 0] + F[2, 2, 0]) / 2


def test_projection_closed_forms():
    P = np.array([[0.25, -0.5, 0.75], [1.0, 0.0, 0.0]])
    u, v, z = field.project(synth.calib_identity(), P)
    np.testing.assert_array_equal(np.stack([u, v, z], 1), P)
    c = synth.calib_yaw(90.0).astype(np.float64)
    u, v, z = field.project(c, np.array([[1.0, 0.3, 0.0]]))
    # 90 degrees about y: x axis -> -z in the input view, y unchanged.
    np.testing.assert_allclose([u[0], v[0], z[0]], [0.0, 0.3, -1.0], atol=1e-7)


class _Net:
    def __init__(self, d_in, W, b, skip=(), slope=0.01):
        self.d_in, self.W, self.b, self.skip, self.slope = d_in, W, b, tuple(skip), slope


def test_mlp_hand_built_skip_and_slope():
    # x = (x0, x1, x2).  Layer 0: h = [x0, -x1] through leaky-ReLU.
    # Layer 1 (skip): input [h0, h1, x0, x1, x2]; picks 2 h0 + 3 x2 - h1.
    # Layer 2: out = h' (one unit) -> known closed form.
    W0 = np.array([[1.0, 0, 0], [0, -1.0, 0]])
    b0 = np.zeros(2)
    W1 = np.array([[2.0, -1.0, 0, 0, 3.0]])
    b1 = np.array([0.5])
    W2 = np.array([[1.0]])
    b2 = np.array([-0.25])
    net = _Net(3, [W0, W1, W2], [b0, b1, b2], skip=(1,), slope=0.1)
    X = np.array([[1.0, 2.0, 0.1], [-1.0, -2.0, -4.0], [0.5, 0.0, -0.1]])

    def lr(t):
        return t if t >= 0 else 0.1 * t

    want = []
    for x0, x1, x2 in X:
        h0, h1 = lr(x0), lr(-x1)
        g = lr(2 * h0 - h1 + 3 * x2 + 0.5)
        want.append(g - 0.25)
    np.testing.assert_allclose(field.mlp(net, X)[:, 0], want, rtol=0, atol=1e-15)


def test_colour_output_mapping():
    # Zero weights: the output is the bias; T = (tanh(b) + 1) / 2 per channel.
    b_last = np.array([0.3, -2.0, 0.0])
    net = _Net(3, [np.zeros((4, 3)), np.zeros((3, 4))], [np.zeros(4), b_last])
    F = np.zeros((2, 2, 2), dtype=np.float32)
    rgb = field.colour(net, F, None, synth.calib_identity(), np.array([[0.1, 0.2, 0.3]]))
    np.testing.assert_allclose(rgb[0], (np.tanh(b_last) + 1) / 2, atol=1e-15)


@pytest.mark.parametrize("C,widths,skip,R", [(32, (128, 64, 1), (), 8),
                                             (48, (256, 128, 64, 32, 1), (1, 2, 3), 4)])
def test_constructed_network_computes_closed_form(C, widths, skip, R):
    # With the noise projection off, the generator's network computes
    # logit = scale * min(f - z, z - b, mask - 1/2) by construction (the
    # identities g(t) - g(-t) = 1.01 t and g(t) + g(-t) = 0.99 |t| of the
    # leaky-ReLU).  The oracle's forward pass must reproduce that closed form.
    net = synth.occupancy_net(C, widths, skip, seed=5, logit_scale=7.0, noise_logit=0.0, carriers=R)
    rng = np.random.default_rng(3)
    n = 500
    x = rng.standard_normal((n, C + 1))
    x[:, 0] = rng.uniform(-1, 1, n)        # front
    x[:, 1] = x[:, 0] - rng.uniform(0, 0.6, n)  # back <= front
    x[:, 2] = rng.uniform(0, 1, n)         # mask
    x[:, C] = rng.uniform(-1, 1, n)        # z
    f, b, m, z = x[:, 0], x[:, 1], x[:, 2], x[:, C]
    want = 7.0 * np.minimum(np.minimum(f - z, z - b), m - 0.5)
    got = field.mlp(net, x)[:, 0]
    # float32 weights (gains and 1/gain read-outs rounded): ~1e-6 relative.
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-5)


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                out[k.strip()] = float(v)
    return out


def test_table_a1_mlp_cost_pins_full_size_shapes():
    # Table A1: the concatenation MLP costs +9.7 GFLOPS per 4096 calls.
    g = _golden("table_a1_mlp_cost.txt")
    w = synth.full(0)
    flops = sum(2 * W.shape[0] * W.shape[1] for W in w.occ_net.W)
    assert flops == 2363392
    assert round(flops * g["calls"] / 1e9, 1) == g["gflops_concat_mlp"]
    # ... and the skip pattern matters: without the skips it would be 7.6.
    no_skip = 2 * (257 * 1024 + 1024 * 512 + 512 * 256 + 256 * 128 + 128)
    assert round(no_skip * 4096 / 1e9, 1) != g["gflops_concat_mlp"]


def test_capsule_sdf_closed_forms():
    a = np.array([[0.0, 0.0, 0.0]])
    b = np.array([[0.0, 1.0, 0.0]])
    r = np.array([0.1])
    P = np.array([[0.1, 0.5, 0.0],    # on the cylinder wall
                  [0.0, 1.1, 0.0],    # on the top cap
                  [0.0, -0.3, 0.4],   # 0.5 from a, outside
                  [0.0, 0.5, 0.0]])   # on the axis
    np.testing.assert_allclose(field.capsule_sdf(a, b, r, P), [0.0, 0.0, 0.4, -0.1], atol=1e-15)
    o = field.capsule_occupancy(a, b, r, P, tau=0.05)
    np.testing.assert_allclose(o, [0.5, 0.5, 1 / (1 + math.exp(8.0)), 1 / (1 + math.exp(-2.0))], atol=1e-15)


def test_projection_translation_column():
    c = synth.calib_identity().astype(np.float64)
    c[:, 3] = [0.125, -0.25, 0.5]
    u, v, z = field.project(c, np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]]))
    np.testing.assert_array_equal(np.stack([u, v, z], 1), [[0.125, -0.25, 0.5], [0.625, 0.25, 1.0]])


def test_occupancy_end_to_end_closed_form_at_texel_centres():
    # f_O built to compute scale * min(f - z, z - b, mask - 1/2) (noise off),
    # evaluated through projection + sampling at texel centres, where the
    # sampled features are the stored ones: O = sigmoid(closed form).  Pins
    # the input order [phi, P_z] and the sigmoid.
    w = synth.tiny(0)
    net = synth.occupancy_net(32, (128, 64, 1), (), seed=4, logit_scale=9.0, noise_logit=0.0, carriers=8)
    rng = np.random.default_rng(5)
    i = rng.integers(0, 64, 300)
    j = rng.integers(0, 64, 300)
    z = rng.uniform(-1, 1, 300)
    u, v = texel_uv(i, j, 64, 64)
    P = np.stack([u, v, z], 1)
    F = w.occ_map.astype(np.float64)
    want = 9.0 * np.minimum(np.minimum(F[j, i, 0] - z, z - F[j, i, 1]), F[j, i, 2] - 0.5)
    got = field.occupancy(net, w.occ_map, w.calib, P)
    np.testing.assert_allclose(got, 1 / (1 + np.exp(-want)), rtol=0, atol=1e-5)


def test_colour_input_order():
    # f_T input is [phi_T, phi_O, P_z] (Eq. 2 argument order).  A one-layer
    # net whose three outputs read phi_T[0], phi_O[0] and P_z.
    H, W = 4, 4
    T = np.full((H, W, 2), 0.25, np.float32)
    O = np.full((H, W, 3), -0.5, np.float32)
    Wt = np.zeros((3, 6))
    Wt[0, 0] = 1.0      # phi_T[0]
    Wt[1, 2] = 1.0      # phi_O[0]
    Wt[2, 5] = 1.0      # P_z
    net = _Net(6, [Wt], [np.zeros(3)])
    rgb = field.colour(net, O, T, synth.calib_identity(), np.array([[0.0, 0.0, 0.75]]))
    np.testing.assert_allclose(rgb[0], (np.tanh([0.25, -0.5, 0.75]) + 1) / 2, atol=1e-15)


def _passthrough_colour_net(d, n_hidden, width, A, c, slope, alpha):
    """A colour MLP whose hidden layers carry the input x unchanged in the
    pair form [x, -x] through leaky-ReLU (lrelu(x) - lrelu(-x) = (1 + s) x),
    each skip layer rebuilding it from h_{l-1} (weight alpha) and from its x
    segment (weight 1 - alpha), and whose last layer (also a skip layer)
    outputs A x + c.  So f_T(x) = A x + c exactly, whatever the depth."""
    assert width >= 2 * d
    inv = 1.0 / (1.0 + slope)
    Ws, bs = [], []
    for l in range(n_hidden + 1):
        last = l == n_hidden
        n_out = A.shape[0] if last else width
        fan_h = d if l == 0 else width
        Wh = np.zeros((n_out, fan_h))
        Wx = np.zeros((n_out, d))
        T = A if last else np.vstack([np.eye(d), -np.eye(d)])   # the map applied to x
        if l == 0:
            Wh[:T.shape[0], :d] = T   # layer 0 reads x only
        else:
            # x = (h[:d] - h[d:2d]) / (1 + s)
            rebuild = np.hstack([np.eye(d), -np.eye(d)]) * inv
            Wh[:T.shape[0], :2 * d] = alpha * (T @ rebuild)
            Wx[:T.shape[0], :] = (1.0 - alpha) * T
        Ws.append(Wh if l == 0 else np.hstack([Wh, Wx]))
        bs.append(c.copy() if last else np.zeros(n_out))
    return _Net(d, Ws, bs, skip=tuple(range(1, n_hidden + 1)), slope=slope)


@pytest.mark.parametrize("n_hidden,alpha", [(1, 0.5), (4, 0.25)])
def test_colour_end_to_end_closed_form_at_texel_centres(n_hidden, alpha):
    # T(P) = (tanh(A [phi_T, phi_O, P_z] + c) + 1) / 2 for a network built to
    # compute A x + c (above), sampled at texel centres where phi is the
    # stored texel: pins the input order, the skip concatenation [h, x] in
    # every layer including the last, the leaky-ReLU slope and the tanh
    # mapping, end to end through projection and sampling.
    rng = np.random.default_rng(11)
    H = W = 8
    CT, CO = 3, 4
    T = rng.standard_normal((H, W, CT)).astype(np.float32)
    O = rng.standard_normal((H, W, CO)).astype(np.float32)
    d = CT + CO + 1
    A = rng.uniform(-0.5, 0.5, (3, d))
    c = rng.uniform(-0.2, 0.2, 3)
    net = _passthrough_colour_net(d, n_hidden, 2 * d + 3, A, c, slope=0.2, alpha=alpha)
    i = rng.integers(0, W, 200)
    j = rng.integers(0, H, 200)
    z = rng.uniform(-1, 1, 200)
    u, v = texel_uv(i, j, W, H)
    P = np.stack([u, v, z], 1)
    x = np.concatenate([T[j, i].astype(np.float64), O[j, i].astype(np.float64), z[:, None]], 1)
    want = (np.tanh(x @ A.T + c) + 1.0) / 2.0
    got = field.colour(net, O, T, synth.calib_identity(), P)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
    # a plausible mistake fails: phi_O before phi_T
    swapped = np.concatenate([x[:, CT:CT + CO], x[:, :CT], x[:, -1:]], 1)
    assert np.max(np.abs((np.tanh(swapped @ A.T + c) + 1) / 2 - got)) > 1e-3


# ---- CBN + SoftZ (Appendix, Eq. 7 and Eq. 8) ------------------------------------

def test_soft_z_closed_forms():
    n = 64
    # Eq. 7's two weights are the linear "hat" basis of the n nodes x = 0..n-1
    # at x = (n - 1) (P_z + 1) / 2: Z_i = max(0, 1 - |x - i|)
    pz = np.concatenate([np.linspace(-1, 1, 1001), [-1.0, 1.0, 0.0]])
    Z = field.soft_z(pz, n)
    x = (n - 1) * (pz + 1) / 2
    hat = np.maximum(0.0, 1.0 - np.abs(x[:, None] - np.arange(n)[None, :]))
    np.testing.assert_allclose(Z, hat, rtol=0, atol=1e-12)
    np.testing.assert_allclose(Z.sum(axis=1), 1.0, atol=1e-12)
    assert np.count_nonzero(Z, axis=1).max() <= 2
    # the centroid recovers the depth: sum_i (2 i / (n - 1) - 1) Z_i = P_z
    np.testing.assert_allclose(Z @ (2 * np.arange(n) / (n - 1) - 1), pz, atol=1e-12)
    # end points and the midpoint, worked by hand
    assert Z[-3, 0] == 1.0 and Z[-2, n - 1] == 1.0
    assert Z[-1, 31] == 0.5 and Z[-1, 32] == 0.5
    # outside [-1, 1] the depth is clamped (reading)
    np.testing.assert_array_equal(field.soft_z([1.5, -3.0], n), field.soft_z([1.0, -1.0], n))
    # a small case by hand: n = 5, P_z = -0.5 -> x = 1 exactly; P_z = 0.25 -> x = 2.5
    Z5 = field.soft_z([-0.5, 0.25], 5)
    np.testing.assert_array_equal(Z5, [[0, 1, 0, 0, 0], [0, 0, 0.5, 0.5, 0]])


class _Cbn:
    def __init__(self, **kw):
        self.__dict__.update(kw)
        self.kind = "cbn"
        self.n_blocks = len(self.W)


def test_cbn_hand_built():
    """Two channels, one-dimensional feature c, n_z = 3, two blocks, worked
    by hand.  var = 1e-5 makes eps matter (scale 1/sqrt(2e-5))."""
    net = _Cbn(C=1, n_z=3, width=2, eps=1e-5,
               Wz=np.array([[1.0, 2.0, 3.0], [0.0, 0.0, 1.0]]), bz=np.array([0.5, -1.0]),
               Gg=[np.array([[1.0], [0.0]]), np.array([[0.0], [2.0]])],
               gg=[np.array([0.0, 1.0]), np.array([1.0, 0.5])],
               Gb=[np.array([[0.0], [1.0]]), np.array([[-1.0], [0.0]])],
               gb=[np.array([0.25, 0.0]), np.array([0.0, 0.1])],
               mu=[np.array([1.0, -1.0]), np.array([0.0, 2.0])],
               var=[np.array([3.0 - 1e-5, 1e-5]), np.array([1.0 - 1e-5, 4.0 - 1e-5])],
               W=[np.array([[1.0, -1.0], [2.0, 0.0]]), np.array([[1.0, 1.0]])],
               b=[np.array([0.0, 1.0]), np.array([-0.5])])
    c = np.array([[2.0]])
    Z = np.array([[0.0, 0.5, 0.5]])
    # h0 = [1*0 + 2*.5 + 3*.5 + .5, .5 - 1] = [3, -0.5]
    # block 0: norm = [(3 - 1)/sqrt(3), (-0.5 + 1)/sqrt(2e-5)]
    #          gamma = [2, 1], beta = [0.25, 2]
    n0 = (3.0 - 1.0) / math.sqrt(3.0)
    n1 = 0.5 / math.sqrt(2e-5)
    a = [max(2 * n0 + 0.25, 0.0), max(1 * n1 + 2.0, 0.0)]
    h1 = [a[0] - a[1], 2 * a[0] + 1.0]
    # block 1: norm = [h1_0 / 1, (h1_1 - 2) / 2]; gamma = [1, 4.5]; beta = [-2, 0.1]
    a2 = [max(1.0 * h1[0] - 2.0, 0.0), max(4.5 * (h1[1] - 2.0) / 2.0 + 0.1, 0.0)]
    want = a2[0] + a2[1] - 0.5
    assert abs(field.cbn_mlp(net, c, Z)[0, 0] - want) <= 1e-12 * max(1.0, abs(want))
    # a second input where the first channel's ReLU cuts: c = -1
    # block 0: gamma = [-1, 1], beta = [0.25, -1]
    c = np.array([[-1.0]])
    a = [max(-1 * n0 + 0.25, 0.0), max(1 * n1 - 1.0, 0.0)]
    h1 = [a[0] - a[1], 2 * a[0] + 1.0]
    # block 1: gamma = [1, 2 (-1) + 0.5] = [1, -1.5]; beta = [1, 0.1]
    a2 = [max(1.0 * h1[0] + 1.0, 0.0), max(-1.5 * (h1[1] - 2.0) / 2.0 + 0.1, 0.0)]
    want = a2[0] + a2[1] - 0.5
    assert abs(field.cbn_mlp(net, c, Z)[0, 0] - want) <= 1e-12 * max(1.0, abs(want))


def test_cbn_batch_statistics():
    """With the running statistics equal to a batch's own mean and variance,
    gamma(c) = 1 and beta(c) = 0, the normalized batch has mean 0 and
    variance var / (var + eps) per channel (read through a ReLU-free pair:
    r(t) - r(-t) = t)."""
    rng = np.random.default_rng(4)
    n_z, K, C, M = 8, 3, 4, 4000
    Wz = rng.standard_normal((K, n_z))
    bz = rng.standard_normal(K)
    Z = field.soft_z(rng.uniform(-1, 1, M), n_z)
    h0 = Z @ Wz.T + bz
    mu, var = h0.mean(axis=0), h0.var(axis=0)
    # block 0 duplicates each channel with gamma +1 / -1; its linear layer
    # takes the difference of each pair (= the normalized value)
    Wz2 = np.concatenate([Wz, Wz])
    net = _Cbn(C=C, n_z=n_z, width=2 * K, eps=1e-5, Wz=Wz2, bz=np.concatenate([bz, bz]),
               Gg=[np.zeros((2 * K, C)), np.zeros((1, 2 * K))],
               gg=[np.concatenate([np.ones(K), -np.ones(K)]), np.ones(1)],
               Gb=[np.zeros((2 * K, C)), np.zeros((1, 2 * K))], gb=[np.zeros(2 * K), np.zeros(1)],
               mu=[np.concatenate([mu, mu]), np.zeros(1)],
               var=[np.concatenate([var, var]), np.ones(1)],
               W=[np.concatenate([np.eye(K), -np.eye(K)], axis=1)], b=[np.zeros(K)])
    net.n_blocks = 1
    out = field.cbn_mlp(net, rng.standard_normal((M, C)), Z)
    np.testing.assert_allclose(out.mean(axis=0), 0.0, atol=1e-12)
    np.testing.assert_allclose(out.var(axis=0), var / (var + 1e-5), rtol=1e-12)


@pytest.mark.parametrize("C,width,n_blocks,R", [(16, 64, 3, 4), (256, 128, 5, 8)])
def test_constructed_cbn_network_computes_closed_form(C, width, n_blocks, R):
    # logit = scale * min(f - z, z - b, mask - 1/2) by construction (ReLU pair
    # identities, constant gamma compensating the running statistics, the
    # SoftZ centroid).  The oracle's forward pass must reproduce it.
    net = synth.occupancy_cbn_net(C, seed=6, logit_scale=7.0, width=width, n_blocks=n_blocks,
                                  noise_logit=0.0, carriers=R)
    rng = np.random.default_rng(9)
    n = 500
    c = rng.standard_normal((n, C))
    c[:, 0] = rng.uniform(-1, 1, n)
    c[:, 1] = c[:, 0] - rng.uniform(0, 0.6, n)
    c[:, 2] = rng.uniform(0, 1, n)
    z = rng.uniform(-1, 1, n)
    f, b, m = c[:, 0], c[:, 1], c[:, 2]
    want = 7.0 * np.minimum(np.minimum(f - z, z - b), m - 0.5)
    got = field.cbn_mlp(net, c, field.soft_z(z, net.n_z))[:, 0]
    np.testing.assert_allclose(got, want, rtol=0, atol=5e-5)


def test_cbn_full_size_cost():
    """Shapes of the paper's final f_O under the reading of the design notes:
    SoftZ 64 -> 128, five CBN blocks of 128 channels conditioned on the
    256-channel feature, 128-wide linear layers, one output.  Table A1 quotes
    3.0 GFLOPS per 4096 calls; this reading costs 3.29 (the input layer and
    the 128-wide linear layers cannot be dropped without contradicting the
    text), within 10%."""
    net = synth.occupancy_cbn_net(256, seed=0, logit_scale=1.0)
    f = net.flops_per_point()
    assert f == 2 * (64 * 128 + 5 * 2 * 256 * 128 + 4 * 128 * 128 + 128)
    assert abs(f * 4096 / 1e9 - 3.0) / 3.0 < 0.10


def test_cbn_occupancy_end_to_end_closed_form_at_texel_centres():
    # the CBN + SoftZ f_O built to compute scale * min(f - z, z - b, mask - 1/2)
    # (noise off), through projection, sampling and SoftZ at texel centres:
    # pins the conditioning on phi and the depth path through Eq. 7
    w = synth.tiny(0)
    net = synth.occupancy_cbn_net(32, seed=4, logit_scale=9.0, width=64, n_blocks=4,
                                  noise_logit=0.0, carriers=4)
    rng = np.random.default_rng(5)
    i = rng.integers(0, 64, 300)
    j = rng.integers(0, 64, 300)
    z = rng.uniform(-1, 1, 300)
    u, v = texel_uv(i, j, 64, 64)
    P = np.stack([u, v, z], 1)
    F = w.occ_map.astype(np.float64)
    want = 9.0 * np.minimum(np.minimum(F[j, i, 0] - z, z - F[j, i, 1]), F[j, i, 2] - 0.5)
    got = field.occupancy(net, w.occ_map, w.calib, P)
    np.testing.assert_allclose(got, 1 / (1 + np.exp(-want)), rtol=0, atol=1e-5)
