"""Fits the occupancy networks f_O of the tiny and the full-size workloads to
their capsule figures once and stores the weights (tests/golden/fitted_occ_*.npz).

The workloads' description: the weights are fitted by the generator with 2000
Adam steps of BCE on 65,536 points against the capsules' occupancy.  Read as:
a fixed training set of 65,536 points per figure, half uniform in the volume
[-1, 1]^3 and half near the capsule surfaces (a point on a capsule's surface
moved by N(0, 0.02) per coordinate), target 1 inside the union of capsules
and 0 outside; mini-batches of 4096 points in seeded random order; Adam with
learning rate 1e-3 (Kingma & Ba's defaults otherwise); the network's input
x = [Phi(P_xy, g(I)), P_z] through the workload's calibration and feature map
(Eq. 1), its architecture and skips the workload's.  Every step of the
arithmetic is the oracle's (oracle.field for the input rows and the figure's
signed distance, oracle.train for the loss, the gradients and Adam, all in
float64); the stored weights are rounded to float32, the type the library
reads.  Only this script writes the files; nothing reads the CUDA path.

    python tests/golden/fit_occupancy.py [tiny|full|both]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import field, train  # noqa: E402
from paper_2007_13988_gb300 import synth  # noqa: E402

POINTS = 65536
STEPS = 2000
BATCH = 4096
LR = 1e-3
NEAR_SIGMA = 0.02


def training_set(w, seed):
    """(x rows [POINTS, d_in], targets [POINTS]) for workload w."""
    rng = np.random.default_rng(seed)
    fig = w.fig
    n_u = POINTS // 2
    P_u = rng.uniform(-1.0, 1.0, (n_u, 3))
    n_s = POINTS - n_u
    a = np.asarray(fig.a, np.float64)
    b = np.asarray(fig.b, np.float64)
    r = np.asarray(fig.r, np.float64)
    # capsule k drawn by its surface area (side 2 pi r L plus the two caps 4 pi r^2)
    L = np.linalg.norm(b - a, axis=1)
    area = 2 * np.pi * r * L + 4 * np.pi * r * r
    k = rng.choice(len(r), size=n_s, p=area / area.sum())
    t = rng.uniform(0.0, 1.0, n_s)
    d = rng.standard_normal((n_s, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    q = a[k] + t[:, None] * (b[k] - a[k])
    # the point of the capsule's surface in direction d from its axis point q
    P_s = q + r[k][:, None] * d + rng.normal(0.0, NEAR_SIGMA, (n_s, 3))
    P = np.concatenate([P_u, np.clip(P_s, -1.0, 1.0)])
    y = (field.capsule_sdf(a, b, r, P) < 0.0).astype(np.float64)
    u, v, z = field.project(w.calib, P)
    phi = field.sample_bilinear(w.occ_map, u, v)
    X = np.concatenate([phi, z[:, None]], axis=1)
    return X, y


def init_weights(net, seed):
    """He-normal hidden layers, a small last layer, zero biases."""
    rng = np.random.default_rng(seed)
    Ws, bs = [], []
    L = len(net.widths)
    for l in range(L):
        fan = net.fan_in(l)
        std = np.sqrt(2.0 / fan) if l < L - 1 else 0.1 / np.sqrt(fan)
        Ws.append(rng.standard_normal((net.widths[l], fan)) * std)
        bs.append(np.zeros(net.widths[l]))
    return Ws, bs


def fit(w, seed):
    net = w.occ_net
    X, y = training_set(w, seed)
    Ws, bs = init_weights(net, seed + 1)
    mW = [np.zeros_like(a) for a in Ws]
    vW = [np.zeros_like(a) for a in Ws]
    mb = [np.zeros_like(a) for a in bs]
    vb = [np.zeros_like(a) for a in bs]
    rng = np.random.default_rng(seed + 2)
    order = rng.permutation(POINTS)
    pos = 0
    hist = []
    t0 = time.time()
    for step in range(1, STEPS + 1):
        if pos + BATCH > POINTS:
            order = rng.permutation(POINTS)
            pos = 0
        idx = order[pos:pos + BATCH]
        pos += BATCH
        loss, dWs, dbs = train.loss_and_grads_concat(Ws, bs, X[idx], y[idx], net.slope, net.skip)
        for l in range(len(Ws)):
            Ws[l], mW[l], vW[l] = train.adam_step(Ws[l], dWs[l], mW[l], vW[l], step, LR)
            bs[l], mb[l], vb[l] = train.adam_step(bs[l], dbs[l], mb[l], vb[l], step, LR)
        if step % 200 == 0 or step == 1:
            hist.append((step, loss))
            print("  step %4d loss %.5f (%.0f s)" % (step, loss, time.time() - t0), flush=True)
    # training-set accuracy of the decision at 0.5
    Z, _ = train.forward_concat(Ws, bs, X, net.slope, net.skip)
    acc = float(np.mean((Z[-1][:, 0] > 0) == (y > 0.5)))
    return Ws, bs, hist, acc


def main():
    which = sys.argv[1] if len(sys.argv) > 1 else "both"
    jobs = []
    if which in ("tiny", "both"):
        jobs.append(("tiny", synth.tiny(0), 7001))
    if which in ("full", "both"):
        jobs.append(("full", synth.full(0), 7002))
    for name, w, seed in jobs:
        print("fitting f_O of the %s workload (%s)" % (name, w.name), flush=True)
        Ws, bs, hist, acc = fit(w, seed)
        out = os.path.join(HERE, "fitted_occ_%s.npz" % name)
        arrays = {}
        for l in range(len(Ws)):
            arrays["W%d" % l] = Ws[l].astype(np.float32)
            arrays["b%d" % l] = bs[l].astype(np.float32)
        np.savez_compressed(out, **arrays, loss=np.array(hist, np.float64),
                            train_accuracy=np.float64(acc))
        print("  training-set accuracy %.4f; wrote %s" % (acc, out), flush=True)


if __name__ == "__main__":
    main()
