"""The learned surrogate f_S: its training kernels against the FP64 oracle's
BCE gradients and Adam step, its distillation tuples against the oracle's
field, and what it gains in the localization (fewer f_O evaluations at the
coarse levels) at unchanged accuracy against the oracle."""
import numpy as np
import pytest

from oracle import field, localize, metrics, train
from paper_2007_13988_gb300 import distill, pifu, synth

from gpu_common import OCC_TOL, Ctx, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    c = Ctx(synth.full(0))
    yield c
    c.close()


def unpack(params, d_in, h1, h2):
    """Unpadded parameter vector -> (Ws, bs) for the oracle."""
    o = 0
    Ws, bs = [], []
    for n_out, fan in ((h1, d_in), (h2, h1), (1, h2)):
        Ws.append(params[o:o + n_out * fan].reshape(n_out, fan).astype(np.float64))
        o += n_out * fan
        bs.append(params[o:o + n_out].astype(np.float64))
        o += n_out
    return Ws, bs


def samples(c, n, seed):
    import torch
    w = c.w
    P = synth.distill_points(w.fig, n, seed)
    ldx = (w.occ_net.d_in + 7) // 8 * 8
    x = torch.empty((n, ldx), dtype=torch.float32, device="cuda")
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    pifu.pifu_surrogate_samples(c.ctx, c.occ, w.calib, to_dev(P), x, y)
    torch.cuda.synchronize()
    return P, x, y


def test_distillation_tuples_match_oracle(full):
    w = full.w
    P, x, y = samples(full, 512, 3)
    xs = x.cpu().numpy().astype(np.float64)
    u, v, z = field.project(w.calib, P)
    phi = field.sample_bilinear(w.occ_map, u, v)
    np.testing.assert_allclose(xs[:, :256], phi, rtol=0, atol=1e-5)
    np.testing.assert_allclose(xs[:, 256], z, rtol=0, atol=1e-6)
    assert np.all(xs[:, 257:] == 0)
    want = field.occupancy(w.occ_net, w.occ_map, w.calib, P)
    assert np.max(np.abs(y.cpu().numpy() - want)) <= OCC_TOL


def test_gradients_match_oracle_backward(full):
    h1, h2 = 128, 64
    pifu.pifu_surrogate_init(full.ctx, h1, h2, seed=7)
    d_in = full.w.occ_net.d_in
    n = pifu.surrogate_param_count(h1, h2, d_in)
    params = pifu.pifu_surrogate_params(full.ctx, n)
    P, x, y = samples(full, 1024, 5)
    loss, grad = pifu.pifu_surrogate_grad(full.ctx, x, y, n)
    Ws, bs = unpack(params, d_in, h1, h2)
    X = x.cpu().numpy().astype(np.float64)[:, :d_in]
    o_loss, dWs, dbs = train.loss_and_grads(Ws, bs, X, y.cpu().numpy(), 0.01)
    want = np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in zip(dWs, dbs)])
    assert abs(loss - o_loss) <= 1e-5 * max(1.0, abs(o_loss))
    rel = np.linalg.norm(grad - want) / np.linalg.norm(want)
    assert rel <= 1e-4, rel
    assert np.max(np.abs(grad - want)) <= 1e-4 * np.max(np.abs(want)) + 1e-7


def test_adam_step_matches_oracle(full):
    h1, h2 = 128, 64
    pifu.pifu_surrogate_init(full.ctx, h1, h2, seed=11)
    d_in = full.w.occ_net.d_in
    n = pifu.surrogate_param_count(h1, h2, d_in)
    before = pifu.pifu_surrogate_params(full.ctx, n).astype(np.float64)
    P, x, y = samples(full, 2048, 9)
    _, grad = pifu.pifu_surrogate_grad(full.ctx, x, y, n)
    pifu.pifu_surrogate_train(full.ctx, x, y, batch=2048, steps=1, lr=1e-3)
    after = pifu.pifu_surrogate_params(full.ctx, n).astype(np.float64)
    want, _, _ = train.adam_step(before, grad.astype(np.float64), np.zeros(n), np.zeros(n), 1, 1e-3)
    # first Adam step moves every parameter with a non-negligible gradient by
    # lr in the gradient's direction
    big = np.abs(grad) > 1e-6
    np.testing.assert_allclose(after[big], want[big], rtol=0, atol=2e-6)


@pytest.fixture(scope="module")
def trained(full):
    x, y = distill.build_samples(full.ctx, n_figures=12, per_figure=200000, seed0=1000)
    first, last = distill.train(full.ctx, x, y, steps=4000, batch=4096, lr=3e-3)
    margin, disagree = distill.calibrate_margin(full.ctx, seeds=[2000, 2001], per_figure=100000)
    return first, last, margin, disagree


def test_training_learns_the_decision(full, trained):
    first, last, margin, disagree = trained
    print("surrogate: loss %.4f -> %.4f, held-out sign disagreement %.4f, margin %.3f"
          % (first, last, disagree, margin))
    assert last < 0.5 * first
    assert disagree <= 0.15


def test_surrogate_localization_gain(full, trained):
    first, last, margin, disagree = trained
    w = full.w
    lv = localize.hierarchical(lambda P: field.occupancy(w.occ_net, w.occ_map, w.calib, P),
                               w.n0, w.num_levels)
    base = full.localize(precision=pifu.PIFU_PREC_MIXED)
    coarse_fo = sum(int(base.evals_per_level[i]) for i in range(w.num_levels - 1))
    vol = full.localize(precision=pifu.PIFU_PREC_MIXED, use_surrogate=True,
                        surrogate_margin=margin)
    b, e, v = full.volume_host(vol)
    iou = metrics.iou(b, lv[-1].binary)
    fallback = sum(int(vol.fallback_per_level[i]) for i in range(w.num_levels - 1))
    coarse = sum(int(vol.evals_per_level[i]) for i in range(w.num_levels - 1))
    print("surrogate localization: IoU %.6f, coarse f_O evaluations %d -> %d (fallback %.3f)"
          % (iou, coarse_fo, fallback, fallback / max(1, coarse)))
    assert iou >= 0.995
    # the gain: far fewer full-network evaluations at the coarse levels
    assert fallback < 0.5 * coarse_fo


def test_surrogate_graph_frame_matches_host_path(full, trained):
    """The graph form runs the same f_S / f_O decisions as the host-driven
    form (device-sized fall-back queue instead of a host read)."""
    import torch
    first, last, margin, disagree = trained
    w = full.w
    host = full.localize(precision=pifu.PIFU_PREC_MIXED, use_surrogate=True,
                         surrogate_margin=margin)
    hb, he, hv = full.volume_host(host)
    h_fallback = [int(host.fallback_per_level[i]) for i in range(w.num_levels)]
    h_evals = [int(host.evals_per_level[i]) for i in range(w.num_levels)]
    R = 512
    depth = torch.empty((R, R), dtype=torch.float32, device="cuda")
    rgb = torch.empty((R, R, 3), dtype=torch.float32, device="cuda")
    mask = torch.empty((R, R), dtype=torch.uint8, device="cuda")
    vol = pifu.pifu_frame(full.ctx, full.occ, full.col, w.calib, w.n0, w.num_levels, R, R,
                          depth, rgb, mask, precision=pifu.PIFU_PREC_MIXED,
                          use_surrogate=True, surrogate_margin=margin)
    torch.cuda.synchronize()
    gb, ge, gv = full.volume_host(vol)
    assert [int(vol.fallback_per_level[i]) for i in range(w.num_levels)] == h_fallback
    assert [int(vol.evals_per_level[i]) for i in range(w.num_levels)] == h_evals
    assert h_fallback[-1] == 0          # the finest level never uses f_S
    assert np.array_equal(gb, hb) and np.array_equal(ge, he)
    # committed values: BF16 away from 0.5 in both forms, except that the host
    # form evaluates a fall-back batch of at most 256 points in FP32 outright
    np.testing.assert_allclose(gv[ge], hv[he], rtol=0, atol=0.03)



# ---- point OHEM (Sec. 3.3, Eq. 6) for the surrogate's tuples -------------------

def test_ohem_sampling_matches_oracle(full):
    """The sampler draws the oracle's indices: integer weights (exact prefix
    sums in float64), the same splitmix64 counters and the same search."""
    import torch
    pifu.pifu_surrogate_init(full.ctx, 128, 64, seed=1)
    m, B = 50000, 4096
    rng = np.random.default_rng(4)
    w = rng.integers(0, 9, size=m).astype(np.float32)
    pifu.pifu_surrogate_ohem_init(full.ctx, m)
    pifu.pifu_surrogate_ohem_weights(full.ctx, m, w)
    idx = torch.empty(B, dtype=torch.int32, device="cuda")
    for seed, step in ((0, 0), (12345, 7), (2 ** 40 + 3, 4000)):
        pifu.pifu_surrogate_ohem_sample(full.ctx, seed, step, idx)
        want = train.ohem_sample(w, seed, step, B)
        np.testing.assert_array_equal(idx.cpu().numpy(), want)
    assert not np.any(w[idx.cpu().numpy()] == 0)   # zero-weight tuples are never drawn


def test_ohem_step_reweights_by_eq6(full):
    """One OHEM step: the drawn tuples' weights become Eq. 6 of their BCE
    under the parameters before the step (the oracle's forward pass)."""
    h1, h2 = 128, 64
    pifu.pifu_surrogate_init(full.ctx, h1, h2, seed=3)
    d_in = full.w.occ_net.d_in
    n = pifu.surrogate_param_count(h1, h2, d_in)
    params = pifu.pifu_surrogate_params(full.ctx, n)
    m, B = 8192, 1024
    P, x, y = samples(full, m, 21)
    pifu.pifu_surrogate_ohem_init(full.ctx, m)
    pifu.pifu_surrogate_train_ohem(full.ctx, x, y, batch=B, steps=1, lr=1e-3, seed=9)
    wgpu = pifu.pifu_surrogate_ohem_weights(full.ctx, m).astype(np.float64)
    drawn = np.unique(train.ohem_sample(np.ones(m), 9, 0, B))
    Ws, bs = unpack(params, d_in, h1, h2)
    X = x.cpu().numpy().astype(np.float64)[drawn, :d_in]
    Z, _ = train.forward(Ws, bs, X, 0.01)
    t = Z[-1][:, 0]
    yy = y.cpu().numpy().astype(np.float64)[drawn]
    L = np.logaddexp(0.0, t) - yy * t
    np.testing.assert_allclose(wgpu[drawn], train.ohem_inverse_probability(L, 0.7, 0.0),
                               rtol=1e-4)
    undrawn = np.setdiff1d(np.arange(m), drawn)
    assert np.all(wgpu[undrawn] == 1.0)


def test_ohem_training_learns(full, trained):
    """Training with point OHEM lowers the loss; its held-out sign
    disagreement is reported beside uniform sampling at the same steps."""
    x, y = distill.build_samples(full.ctx, n_figures=6, per_figure=200000, seed0=1000)
    pifu.pifu_surrogate_init(full.ctx, 128, 64, seed=0)
    pifu.pifu_surrogate_ohem_init(full.ctx, x.shape[0])
    first, last = pifu.pifu_surrogate_train_ohem(full.ctx, x, y, batch=4096, steps=3000, lr=3e-3,
                                                 seed=5)
    margin, disagree = distill.calibrate_margin(full.ctx, seeds=[2000, 2001], per_figure=100000)
    print("surrogate with point OHEM: loss %.4f -> %.4f, held-out sign disagreement %.4f, "
          "margin %.3f (uniform sampling, more steps and tuples: %.4f)"
          % (first, last, disagree, margin, trained[3]))
    assert disagree <= 0.15
