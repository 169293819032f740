"""Training arithmetic of the distilled occupancy surrogate, in float64.

The paper trains f_O with a binary cross-entropy loss (Sec. 3.1) and uses
Adam for the texture network (Appendix, Training procedure).  The surrogate
is an MLP of the same family (no skips): h_l = g(W_l h_{l-1} + b_l) with
leaky-ReLU g, logit t = W_L h_{L-1} + b_L, target y in [0, 1] (the full
network's occupancy), and the mean BCE over a batch of B points

    L = (1/B) sum_b [ softplus(t_b) - y_b t_b ]
      = (1/B) sum_b -[ y_b log s(t_b) + (1 - y_b) log(1 - s(t_b)) ],

whose gradient with respect to t_b is (s(t_b) - y_b) / B.  Backward
propagation is the chain rule layer by layer: dW_l = dZ_l^T H_{l-1},
db_l = column sums of dZ_l, dH_{l-1} = dZ_l W_l, dZ_{l-1} = dH_{l-1} * g'(Z).

Adam (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

The concatenation MLP with skip layers (the full f_O's family, fitted once to
the figures by tests/golden/fit_occupancy.py) has its own forward and
backward below.

Pins: tests/test_oracle_train.py (central finite differences of the loss,
with and without skips; a hand-computed Adam step; BCE closed forms).
"""
from __future__ import annotations

import numpy as np

F64 = np.float64


def leaky(z, slope):
    return np.where(z >= 0, z, slope * z)


def leaky_grad(z, slope):
    return np.where(z >= 0, 1.0, slope)


def bce_with_logits(t, y):
    """Mean BCE of logits t against targets y (numerically stable form)."""
    t = np.asarray(t, F64)
    y = np.asarray(y, F64)
    return float(np.mean(np.logaddexp(0.0, t) - y * t))


def forward(Ws, bs, X, slope):
    """Pre-activations Z_l and activations H_l (H_0 = X); the last Z is the logit."""
    H = [np.asarray(X, F64)]
    Z = []
    L = len(Ws)
    for l in range(L):
        z = H[-1] @ np.asarray(Ws[l], F64).T + np.asarray(bs[l], F64)
        Z.append(z)
        if l < L - 1:
            H.append(leaky(z, slope))
    return Z, H


def loss_and_grads(Ws, bs, X, y, slope):
    """Mean BCE loss and its gradients (dW_l, db_l) for one batch."""
    Z, H = forward(Ws, bs, X, slope)
    t = Z[-1][:, 0]
    B = len(t)
    loss = bce_with_logits(t, y)
    s = 1.0 / (1.0 + np.exp(-t))
    dz = ((s - np.asarray(y, F64)) / B)[:, None]
    L = len(Ws)
    dWs = [None] * L
    dbs = [None] * L
    for l in range(L - 1, -1, -1):
        dWs[l] = dz.T @ H[l]
        dbs[l] = dz.sum(axis=0)
        if l > 0:
            dh = dz @ np.asarray(Ws[l], F64)
            dz = dh * leaky_grad(Z[l - 1], slope)
    return loss, dWs, dbs


# ---- the concatenation MLP with skips (Sec. 3.1, f_O of the "MLP" variant) ----
#
# Layer l reads z_l = [h_{l-1}, x] when l is a skip layer (l > 0), else
# h_{l-1} (h_{-1} = x); Z_l = z_l W_l^T + b_l, h_l = g(Z_l) but for the last
# layer, whose Z is the logit.  Backward: dZ_l gives dW_l = dZ_l^T z_l and
# db_l = column sums of dZ_l; dz_l = dZ_l W_l, whose first columns are
# dh_{l-1} (the trailing d_in columns of a skip layer are the gradient with
# respect to x, which no parameter needs), and dZ_{l-1} = dh_{l-1} * g'(Z_{l-1}).


def forward_concat(Ws, bs, X, slope, skip):
    """Pre-activations Z_l and layer inputs z_l of the concatenation MLP."""
    X = np.asarray(X, F64)
    h = X
    Z, zin = [], []
    L = len(Ws)
    for l in range(L):
        z = np.concatenate([h, X], axis=1) if (l in skip and l > 0) else h
        zin.append(z)
        pre = z @ np.asarray(Ws[l], F64).T + np.asarray(bs[l], F64)
        Z.append(pre)
        if l < L - 1:
            h = leaky(pre, slope)
    return Z, zin


def loss_and_grads_concat(Ws, bs, X, y, slope, skip):
    """Mean BCE loss and its gradients (dW_l, db_l) of the concatenation MLP."""
    Z, zin = forward_concat(Ws, bs, X, slope, skip)
    t = Z[-1][:, 0]
    B = len(t)
    loss = bce_with_logits(t, y)
    s = 1.0 / (1.0 + np.exp(-t))
    dz = ((s - np.asarray(y, F64)) / B)[:, None]
    L = len(Ws)
    dWs = [None] * L
    dbs = [None] * L
    for l in range(L - 1, -1, -1):
        dWs[l] = dz.T @ zin[l]
        dbs[l] = dz.sum(axis=0)
        if l > 0:
            width_prev = np.asarray(Ws[l - 1]).shape[0]
            dh = (dz @ np.asarray(Ws[l], F64))[:, :width_prev]
            dz = dh * leaky_grad(Z[l - 1], slope)
    return loss, dWs, dbs


def adam_step(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns new (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


# ---- point OHEM (Sec. 3.3, Eq. 6) ----------------------------------------------
#
# Each training point m carries the inverse of its sampling probability,
#     P^-1_pt(m) = 1 / (exp(-L_BCE(m) / alpha_p) + beta_p),
# recomputed from its binary cross-entropy whenever it is in a mini-batch and
# used, after normalisation, as the probability of drawing it again.  The
# draws use uniforms from splitmix64 (Steele, Lea and Flood; the constants of
# the published generator), one 64-bit output per (seed, step, draw) counter,
# and inverse-CDF search on the float64 prefix sums of the weights.

MASK64 = (1 << 64) - 1


def ohem_inverse_probability(loss, alpha=0.7, beta=0.0):
    """Eq. 6 for points."""
    loss = np.asarray(loss, F64)
    return 1.0 / (np.exp(-loss / alpha) + beta)


def splitmix64_next(state):
    """One step of splitmix64: (new state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


def draw_uniform(seed, step, i):
    """Uniform in [0, 1) for draw i of step `step`: the first splitmix64 output
    from the state seed ^ (step << 32) ^ i, top 53 bits."""
    state = (seed ^ ((step & 0xFFFFFFFF) << 32) ^ i) & MASK64
    _, z = splitmix64_next(state)
    return (z >> 11) * (1.0 / 9007199254740992.0)


def ohem_sample(weights, seed, step, B):
    """B indices drawn with probability proportional to weights."""
    w = np.asarray(weights, F64)
    cdf = np.cumsum(w)
    total = cdf[-1]
    u = np.array([draw_uniform(seed, step, i) for i in range(B)]) * total
    idx = np.searchsorted(cdf, u, side="right")
    return np.minimum(idx, len(w) - 1)
