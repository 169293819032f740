"""Pins of the oracle's training arithmetic (BCE loss of Sec. 3.1, Adam of
the appendix) against central finite differences and hand-computed values."""
import math

import numpy as np

from oracle import train


def small_net(seed=0, dims=(7, 5, 4, 1)):
    rng = np.random.default_rng(seed)
    Ws = [rng.standard_normal((dims[i + 1], dims[i])) * 0.7 for i in range(len(dims) - 1)]
    bs = [rng.standard_normal(dims[i + 1]) * 0.1 for i in range(len(dims) - 1)]
    return Ws, bs


def test_bce_closed_forms():
    assert abs(train.bce_with_logits([0.0], [0.3]) - math.log(2.0)) < 1e-15
    # y = 1: -log sigmoid(t)
    assert abs(train.bce_with_logits([2.0], [1.0]) - math.log1p(math.exp(-2.0))) < 1e-15
    # y = 0: -log(1 - sigmoid(t))
    assert abs(train.bce_with_logits([-1.5], [0.0]) - math.log1p(math.exp(-1.5))) < 1e-15


def test_gradients_match_central_differences():
    Ws, bs = small_net(1)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((9, 7))
    y = rng.uniform(0, 1, 9)
    slope = 0.01
    loss, dWs, dbs = train.loss_and_grads(Ws, bs, X, y, slope)
    h = 1e-6
    for l in range(len(Ws)):
        for idx in [(0, 0), (Ws[l].shape[0] - 1, Ws[l].shape[1] - 1), (0, Ws[l].shape[1] // 2)]:
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[l][idx] += h
            Wm[l][idx] -= h
            num = (train.loss_and_grads(Wp, bs, X, y, slope)[0]
                   - train.loss_and_grads(Wm, bs, X, y, slope)[0]) / (2 * h)
            assert abs(num - dWs[l][idx]) < 1e-8, (l, idx)
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[l][0] += h
        bm[l][0] -= h
        num = (train.loss_and_grads(Ws, bp, X, y, slope)[0]
               - train.loss_and_grads(Ws, bm, X, y, slope)[0]) / (2 * h)
        assert abs(num - dbs[l][0]) < 1e-8


def test_adam_first_steps_by_hand():
    # Step 1: m = 0.1 g, v = 0.001 g^2, bias-corrected m_hat = g, v_hat = g^2,
    # so the update is lr * g / (|g| + eps) = lr * sign(g) (up to eps).
    w, m, v = train.adam_step(np.array([1.0, -2.0]), np.array([0.5, -4.0]), np.zeros(2),
                              np.zeros(2), 1, lr=0.1)
    np.testing.assert_allclose(w, [1.0 - 0.1, -2.0 + 0.1], atol=1e-7)
    np.testing.assert_allclose(m, [0.05, -0.4])
    np.testing.assert_allclose(v, [0.00025, 0.016])
    # Step 2 with the same gradient: m_hat = g, v_hat = g^2 again.
    w2, _, _ = train.adam_step(w, np.array([0.5, -4.0]), m, v, 2, lr=0.1)
    np.testing.assert_allclose(w2, [1.0 - 0.2, -2.0 + 0.2], atol=1e-7)


def test_ohem_eq6_closed_forms():
    # beta = 0: the inverse probability is exp(L / alpha); L = 0 gives 1 / (1 + beta)
    L = np.array([0.0, 0.35, 0.7, 1.4])
    np.testing.assert_allclose(train.ohem_inverse_probability(L, 0.7, 0.0), np.exp(L / 0.7),
                               rtol=1e-15)
    assert abs(train.ohem_inverse_probability([0.0], 0.7, 10.0)[0] - 1.0 / 11.0) < 1e-16
    # harder points (larger loss) are drawn more often
    assert np.all(np.diff(train.ohem_inverse_probability(L, 0.7, 0.0)) > 0)


def test_splitmix64_published_outputs():
    # the generator's first outputs from state 0 (published reference values)
    s, z = train.splitmix64_next(0)
    assert z == 0xE220A8397B1DCDAF
    s, z = train.splitmix64_next(s)
    assert z == 0x6E789E6AA1B965F4


def test_ohem_sampling_frequencies():
    w = np.array([1.0, 2.0, 7.0, 0.0, 10.0])
    idx = train.ohem_sample(w, seed=3, step=5, B=20000)
    freq = np.bincount(idx, minlength=len(w)) / len(idx)
    np.testing.assert_allclose(freq, w / w.sum(), atol=0.015)
    assert freq[3] == 0.0


def skip_net(seed=3, d_in=6, widths=(5, 4, 3, 1), skip=(1, 2)):
    rng = np.random.default_rng(seed)
    Ws, bs = [], []
    prev = d_in
    for l, w in enumerate(widths):
        fan = prev + (d_in if (l in skip and l > 0) else 0)
        Ws.append(rng.standard_normal((w, fan)) * 0.6)
        bs.append(rng.standard_normal(w) * 0.1)
        prev = w
    return Ws, bs


def test_concat_gradients_match_central_differences():
    # every weight and bias of a net whose layers 1 and 2 read [h, x]
    Ws, bs = skip_net()
    skip = (1, 2)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((11, 6))
    y = (rng.uniform(0, 1, 11) > 0.5).astype(float)
    slope = 0.01
    _, dWs, dbs = train.loss_and_grads_concat(Ws, bs, X, y, slope, skip)
    h = 1e-6

    def loss(Ws_, bs_):
        return train.loss_and_grads_concat(Ws_, bs_, X, y, slope, skip)[0]

    for l in range(len(Ws)):
        for idx in np.ndindex(*Ws[l].shape):
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[l][idx] += h
            Wm[l][idx] -= h
            num = (loss(Wp, bs) - loss(Wm, bs)) / (2 * h)
            assert abs(num - dWs[l][idx]) < 1e-8, (l, idx)
        for k in range(len(bs[l])):
            bp = [b.copy() for b in bs]
            bm = [b.copy() for b in bs]
            bp[l][k] += h
            bm[l][k] -= h
            num = (loss(Ws, bp) - loss(Ws, bm)) / (2 * h)
            assert abs(num - dbs[l][k]) < 1e-8, (l, k)


def test_concat_forward_is_the_field_mlp():
    # the trainer's logit is the inference network's (oracle.field.mlp, the
    # same concatenation family written for Eq. 1)
    from types import SimpleNamespace

    from oracle import field
    Ws, bs = skip_net(seed=5)
    X = np.random.default_rng(6).standard_normal((8, 6))
    net = SimpleNamespace(W=Ws, b=bs, skip=(1, 2), slope=0.01)
    Z, _ = train.forward_concat(Ws, bs, X, 0.01, (1, 2))
    assert np.allclose(Z[-1], field.mlp(net, X), rtol=0, atol=1e-13)


def test_concat_without_skips_is_the_plain_trainer():
    Ws, bs = small_net(7)
    X = np.random.default_rng(8).standard_normal((5, 7))
    y = np.random.default_rng(9).uniform(0, 1, 5)
    a = train.loss_and_grads(Ws, bs, X, y, 0.01)
    b = train.loss_and_grads_concat(Ws, bs, X, y, 0.01, ())
    assert abs(a[0] - b[0]) < 1e-15
    for l in range(len(Ws)):
        assert np.allclose(a[1][l], b[1][l], rtol=0, atol=1e-15)
        assert np.allclose(a[2][l], b[2][l], rtol=0, atol=1e-15)
