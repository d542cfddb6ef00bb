"""FP64 CPU oracle of the single-pulse candidate classifier -- TEST INFRASTRUCTURE.

The paper plans automatic transient detection (Sec. 5) without naming a
method; this is the small network the batched dedispersion feeds: a patch of
32 DM trials x 256 series samples (channels = trials) goes through

    3 x [Conv1d(32 -> 32, kernel 7, zero padding 3) + ReLU],
    max-pool 2 after the first and the second block,
    global average over time -> Linear(32 -> 4) -> softmax cross-entropy.

Parameters (21,732): conv weights w_l[co][ci][k] and biases b_l[co] for
l = 1..3, then the linear layer fc_w[4][32], fc_b[4], in that flat order.
Forward and backward are plain loops over the definitions in FP64; the
tests pin the backward pass against finite differences of the forward pass.
"""
from __future__ import annotations

import numpy as np

C = 32          # channels (DM trials)
K = 7           # kernel width
PAD = 3
T = 256         # samples per patch
NCLS = 4        # dispersed pulse, broadband RFI, narrowband RFI, noise
CONV = C * C * K


def n_params() -> int:
    return 3 * (CONV + C) + NCLS * C + NCLS


def unpack(theta: np.ndarray):
    """Flat parameter vector -> (list of (w, b) per conv layer, fc_w, fc_b)."""
    theta = np.asarray(theta, dtype=np.float64)
    layers, o = [], 0
    for _ in range(3):
        w = theta[o:o + CONV].reshape(C, C, K)
        o += CONV
        b = theta[o:o + C]
        o += C
        layers.append((w, b))
    fw = theta[o:o + NCLS * C].reshape(NCLS, C)
    o += NCLS * C
    fb = theta[o:o + NCLS]
    return layers, fw, fb


def conv1d(x, w, b):
    """y[n, co, t] = b[co] + sum_{ci, k} w[co, ci, k] x[n, ci, t + k - PAD] (zero outside)."""
    n, ci, t = x.shape
    xp = np.zeros((n, ci, t + 2 * PAD))
    xp[:, :, PAD:PAD + t] = x
    y = np.zeros((n, w.shape[0], t))
    for k in range(K):
        y += np.einsum("oc,nct->not", w[:, :, k], xp[:, :, k:k + t])
    return y + b[None, :, None]


def forward(theta, x):
    """Logits and the intermediate values the backward pass needs."""
    layers, fw, fb = unpack(theta)
    cache = []
    h = np.asarray(x, dtype=np.float64)
    for l, (w, b) in enumerate(layers):
        z = conv1d(h, w, b)
        a = np.maximum(z, 0.0)
        if l < 2:
            n, c, t = a.shape
            r = a.reshape(n, c, t // 2, 2)
            idx = np.argmax(r, axis=3)            # first of two on ties
            p = np.take_along_axis(r, idx[..., None], 3)[..., 0]
        else:
            idx, p = None, a
        cache.append((h, z, idx))
        h = p
    g = h.mean(axis=2)                            # global average pool
    logits = g @ fw.T + fb
    return logits, (cache, h, g)


def softmax_xent(logits, labels):
    """Mean cross-entropy over the batch and d loss / d logits."""
    z = logits - logits.max(axis=1, keepdims=True)
    p = np.exp(z)
    p /= p.sum(axis=1, keepdims=True)
    n = len(labels)
    loss = -np.mean(np.log(p[np.arange(n), labels]))
    d = p.copy()
    d[np.arange(n), labels] -= 1.0
    return loss, d / n, p


def backward(theta, x, labels):
    """(loss, gradient of the mean cross-entropy w.r.t. theta, probabilities)."""
    layers, fw, fb = unpack(theta)
    logits, (cache, hlast, g) = forward(theta, x)
    loss, dlog, prob = softmax_xent(logits, labels)
    grads = []
    d_fw = dlog.T @ g
    d_fb = dlog.sum(axis=0)
    dg = dlog @ fw
    dh = np.repeat(dg[:, :, None], hlast.shape[2], axis=2) / hlast.shape[2]
    for l in range(2, -1, -1):
        h_in, z, idx = cache[l]
        w, b = layers[l]
        if l < 2:                                  # undo the max-pool
            n, c, t2 = dh.shape
            da = np.zeros((n, c, t2, 2))
            np.put_along_axis(da, idx[..., None], dh[..., None], 3)
            da = da.reshape(n, c, 2 * t2)
        else:
            da = dh
        dz = da * (z > 0)
        n, ci, t = h_in.shape
        xp = np.zeros((n, ci, t + 2 * PAD))
        xp[:, :, PAD:PAD + t] = h_in
        dw = np.zeros_like(w)
        for k in range(K):
            dw[:, :, k] = np.einsum("not,nct->oc", dz, xp[:, :, k:k + t])
        db = dz.sum(axis=(0, 2))
        dxp = np.zeros_like(xp)
        for k in range(K):
            dxp[:, :, k:k + t] += np.einsum("oc,not->nct", w[:, :, k], dz)
        dh = dxp[:, :, PAD:PAD + t]
        grads.append((dw, db))
    grads.reverse()
    flat = []
    for dw, db in grads:
        flat += [dw.ravel(), db]
    flat += [d_fw.ravel(), d_fb]
    return loss, np.concatenate(flat), prob


def adam_step(theta, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; returns new (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(rng_uniform: np.ndarray) -> np.ndarray:
    """He-uniform conv weights and uniform linear weights from uniforms in (0, 1)."""
    u = np.asarray(rng_uniform, dtype=np.float64)
    theta = np.zeros(n_params())
    o = 0
    bound = np.sqrt(6.0 / (C * K))
    for _ in range(3):
        theta[o:o + CONV] = (2 * u[o:o + CONV] - 1) * bound
        o += CONV + C                               # biases start at zero
    bf = np.sqrt(6.0 / C)
    theta[o:o + NCLS * C] = (2 * u[o:o + NCLS * C] - 1) * bf * 0.5
    return theta


def patch(series: np.ndarray, d0: int, t0: int, rows: int = C, cols: int = T) -> np.ndarray:
    """Rows d0.. and samples t0.. of a series block (indices outside repeat the
    nearest edge), less the mean, over the standard deviation (population; a
    constant patch keeps scale 1), in FP64."""
    series = np.asarray(series, dtype=np.float64)
    ndm, n = series.shape
    d = np.clip(np.arange(d0, d0 + rows), 0, ndm - 1)
    t = np.clip(np.arange(t0, t0 + cols), 0, n - 1)
    p = series[np.ix_(d, t)]
    mu = p.mean()
    sd = np.sqrt(np.mean((p - mu) ** 2))
    return (p - mu) / (sd if sd > 0 else 1.0)
