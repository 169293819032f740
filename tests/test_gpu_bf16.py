"""Tensor-core (tcgen05, BF16 operands, FP32 accumulation) form of the MLP.

1. Kernel numerics, isolated: a hand-sized network whose inputs are exactly
   representable in BF16 (texel-centre samples of a BF16-valued map, depths
   on a 1/64 grid, BF16-valued weights), against a numpy emulation of the
   same arithmetic (float64 sums, BF16 rounding of every stored activation).
   Covers all tile widths (256, 128, 64 outputs), skip segments, ragged M.
2. The BF16 form against the FP64 oracle: its occupancy error, and the
   localized volume's IoU, are reported and bounded.
"""
import numpy as np
import pytest

from oracle import field, localize, metrics
from paper_2007_13988_gb300 import synth

from gpu_common import Ctx, to_dev

pytestmark = pytest.mark.gpu

BF16 = 1


def bf16_round(a):
    """Round float64/float32 values to the nearest BF16 (ties to even)."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def make_net(C, widths, skip, seed):
    rng = np.random.default_rng(seed)
    d_in = C + 1
    Ws, bs = [], []
    for l, n in enumerate(widths):
        fan = (d_in if l == 0 else widths[l - 1]) + (d_in if l in skip else 0)
        W = rng.uniform(-1, 1, (n, fan)) * np.sqrt(3.0 / fan)
        Ws.append(bf16_round(W).astype(np.float32))
        bs.append(rng.uniform(-0.1, 0.1, n).astype(np.float32))
    return synth.Net(d_in=d_in, widths=tuple(widths), skip=tuple(skip), W=Ws, b=bs,
                     out_act="sigmoid")


def emulate(net, X):
    """BF16-operand / FP32-accumulate MLP with every stored activation rounded
    to BF16 (as the kernels store them); the last layer reads BF16 and
    accumulates in float."""
    x = bf16_round(X)
    h = x
    L = len(net.W)
    for l in range(L):
        z = np.concatenate([h, x], 1) if (l in net.skip and l > 0) else h
        t = z @ net.W[l].astype(np.float64).T + net.b[l].astype(np.float64)
        if l < L - 1:
            t = np.where(t >= 0, t, net.slope * t)
            h = bf16_round(t)
        else:
            h = t
    return 1.0 / (1.0 + np.exp(-h[:, 0]))


@pytest.mark.parametrize("m", [1, 200, 3001])
def test_tc_layers_match_bf16_emulation(m):
    C = 60   # d_in = 61: the x segment spans one K-block with a ragged edge
    occ_net = make_net(C, (256, 128, 64, 64, 1), (1, 2), seed=3)
    w = synth.tiny(0)
    rng = np.random.default_rng(4)
    H = W = 32
    fmap = bf16_round(rng.standard_normal((H, W, C))).astype(np.float32)
    w.occ_map = np.ascontiguousarray(fmap)
    w.occ_net = occ_net
    w.col_net = synth.colour_net(C + 1, (64, 3), (), 5)
    c = Ctx(w)
    try:
        i = rng.integers(0, W, m)
        j = rng.integers(0, H, m)
        z = rng.integers(-64, 65, m) / 64.0
        P = np.stack([(2 * i + 1) / W - 1, (2 * j + 1) / H - 1, z], 1).astype(np.float32)
        X = np.concatenate([fmap[j, i].astype(np.float64), z[:, None]], 1)
        want = emulate(occ_net, X)
        got = c.query(P, precision=BF16)
        # differences only from FP32-vs-FP64 accumulation order flipping a
        # BF16 rounding of a stored activation
        assert np.max(np.abs(got - want)) <= 2e-3, np.max(np.abs(got - want))
        assert np.mean(np.abs(got - want)) <= 1e-4
    finally:
        c.close()


def pair_workload(m, seed=11):
    """A hand-sized f_O whose first three hidden layers are multiples of 256
    wide (so the CTA-pair form applies to them) on BF16-exact inputs."""
    C = 60
    occ_net = make_net(C, (512, 256, 256, 128, 1), (1, 2, 3), seed=seed)
    w = synth.tiny(0)
    rng = np.random.default_rng(seed + 1)
    H = W = 32
    fmap = bf16_round(rng.standard_normal((H, W, C))).astype(np.float32)
    w.occ_map = np.ascontiguousarray(fmap)
    w.occ_net = occ_net
    w.col_net = synth.colour_net(C + 1, (64, 3), (), 5)
    i = rng.integers(0, W, m)
    j = rng.integers(0, H, m)
    z = rng.integers(-64, 65, m) / 64.0
    P = np.stack([(2 * i + 1) / W - 1, (2 * j + 1) / H - 1, z], 1).astype(np.float32)
    X = np.concatenate([fmap[j, i].astype(np.float64), z[:, None]], 1)
    return w, P, X


# tuned layers of pair_workload's nets, in the autotuner's order: f_O's four
# hidden layers (the last one carries the fused last layer), then f_T's one
SINGLE = [256, 256, 256, 128, 64]


# m: one row; the odd CTA's half holds one row; whole 256-row pair tiles plus
# a tail only the even CTA covers; a tail both cover; several waves
@pytest.mark.parametrize("m", [1, 129, 256 * 40 + 100, 256 * 40 + 200, 70001])
def test_pair_form_matches_single_cta_form(m):
    """The CTA-pair form (two CTAs on a 256 x 256 tile, cta_group::2 MMAs)
    adds the same products in the same K order as the single-CTA form, so
    the outputs are equal bit for bit; both stay within the emulation bound."""
    from paper_2007_13988_gb300 import pifu
    w, P, X = pair_workload(m)
    want = emulate(w.occ_net, X)
    c = Ctx(w)
    try:
        pair = [pifu.PIFU_TILE_PAIR] * 3 + SINGLE[3:]
        got = {}
        for name, codes in (("single", SINGLE), ("pair", pair), ("mixed", [512, 256, 512, 128, 64])):
            pifu.pifu_set_tiles(c.ctx, codes)
            got[name] = c.query(P, precision=BF16)
            assert np.max(np.abs(got[name] - want)) <= 2e-3, name
        np.testing.assert_array_equal(got["pair"], got["single"])
        np.testing.assert_array_equal(got["mixed"], got["single"])
    finally:
        c.close()


def test_set_tiles_refusals():
    from paper_2007_13988_gb300 import pifu
    w, P, _ = pair_workload(300)
    c = Ctx(w)
    try:
        before = c.query(P, precision=BF16)
        bad = [SINGLE[:-1],                       # one layer short
               SINGLE + [64],                     # one too many
               [96] + SINGLE[1:],                 # not a tile code
               [256, 256, 256, 512, 64],          # the pair form on the 128-wide layer
               [256, 256, 256, 64, 64],           # the fused layer must keep its code
               [256, 256, 256, 128, 512]]         # the pair form on a 64-wide layer
        for codes in bad:
            with pytest.raises(pifu.PifuError) as e:
                pifu.pifu_set_tiles(c.ctx, codes)
            assert e.value.status == pifu.PIFU_ERR_ARG
        np.testing.assert_array_equal(c.query(P, precision=BF16), before)
    finally:
        c.close()


@pytest.fixture(scope="module")
def full():
    c = Ctx(synth.full(0))
    yield c
    c.close()


def test_bf16_query_against_oracle(full):
    w = full.w
    P = synth.query_points(4000, seed=21)
    want = field.occupancy(w.occ_net, w.occ_map, w.calib, P)
    got = full.query(P, precision=BF16)
    fp32 = full.query(P)
    err = np.abs(got - want)
    print("bf16 occupancy error vs oracle: max %.3g mean %.3g; fp32 max %.3g"
          % (err.max(), err.mean(), np.abs(fp32 - want).max()))
    assert err.mean() <= 5e-3
    flips = np.count_nonzero((got >= 0.5) != (want >= 0.5))
    assert flips <= 0.01 * len(P)


def test_bf16_localization_iou(full):
    w = full.w
    vol = full.localize(precision=BF16)
    b, e, v = full.volume_host(vol)
    counts = {}
    for line in open("tests/golden/full_frame_counts.txt"):
        line = line.split("#")[0].strip()
        if "=" in line:
            k, x = line.split("=")
            counts[k.strip()] = int(x)
    # oracle's finest binarized volume, from a dense evaluation restricted to
    # nodes that either side evaluated, plus both sides' 0/1 elsewhere
    lv = localize.hierarchical(lambda P: field.occupancy(w.occ_net, w.occ_map, w.calib, P),
                               w.n0, w.num_levels)
    iou = metrics.iou(b, lv[-1].binary)
    print("bf16 localization: IoU %.5f, evals %d (oracle %d)" % (iou, vol.n_eval,
                                                                counts["evals_total"]))
    assert iou >= 0.97


MIXED = 2


def test_mixed_query_decisions_match_oracle(full):
    # points on the finest grid near the figure, where o is close to 0.5
    w = full.w
    c = localize.node_coords(256)
    rng = np.random.default_rng(9)
    k, j, i = (rng.integers(0, 257, 60000) for _ in range(3))
    P = np.stack([c[i], c[j], c[k]], 1)
    o = field.occupancy(w.occ_net, w.occ_map, w.calib, P)
    P = P[np.abs(o - 0.5) < 0.3][:3000].astype(np.float32)
    want = field.occupancy(w.occ_net, w.occ_map, w.calib, P)
    got = full.query(P, precision=MIXED)
    near = np.abs(want - 0.5) < 0.015
    # re-evaluated points carry FP32 accuracy; every decision matches
    assert np.max(np.abs(got[near] - want[near])) <= 1e-4
    assert np.array_equal(got >= 0.5, want >= 0.5)


def test_mixed_localization_matches_oracle(full):
    w = full.w
    vol = full.localize(precision=MIXED, margin=0.02)
    b, e, v = full.volume_host(vol)
    lv = localize.hierarchical(lambda P: field.occupancy(w.occ_net, w.occ_map, w.calib, P),
                               w.n0, w.num_levels)
    iou = metrics.iou(b, lv[-1].binary)
    sym = int(np.count_nonzero(e ^ lv[-1].evaluated))
    print("mixed localization: IoU %.6f, eval symdiff %d, rechecked %s"
          % (iou, sym, list(vol.rechecked_per_level)[:4]))
    assert iou >= 0.999
