"""FP64 reference of the proposal network (TEST INFRASTRUCTURE ONLY).

The network flags decimated blocks worth a full-resolution search.  It is not
from the paper (the paper has no learned part); it is defined here, and this
file is its definition, written plainly in numpy:

  input   x[256]: one block of the x16-decimated, normalised series
  conv l  a_l[c][p] = bf16(relu(b_l[c] + sum_{ci,k} bf16(W_l[c][ci][k]) a_{l-1}[ci][p + k - 4]))
          (l = 1, 2, 3; 16 channels; kernel 9, zero padding of 4; a_0 = bf16(x), one channel;
          the layer-3 activations are kept unrounded: they only feed the pool)
  pool    g[c] = max_p a_3[c][p]
  head    z = b_4 + sum_c W_4[c] g[c],  p = sigmoid(z)
  loss    BCE(p, y) = softplus(z) - y z

The input blocks come from ``decimate``: 16-sample sums of a row, centred and
scaled to unit variance.

bf16(v) rounds to the nearest bfloat16 (ties to even); bf16=False drops the
rounding (the exact function, used to check the gradients by finite
differences).  Gradients pass the roundings unchanged (straight-through); the
max pool sends its gradient to the first maximum of each channel.

Parameter vector (float, 4817 entries): W1[16][9], b1[16], W2[16][16][9], b2[16],
W3[16][16][9], b3[16], W4[16], b4.
"""
from __future__ import annotations

import numpy as np

C, K, P, PAD = 16, 9, 256, 4
SHAPES = [("W1", (C, 1, K)), ("b1", (C,)), ("W2", (C, C, K)), ("b2", (C,)), ("W3", (C, C, K)),
          ("b3", (C,)), ("W4", (C,)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def decimate(x, mu, sigma, factor=16):
    """The network's input series: x16 decimation of each row, normalised.

    d[r][j] = (sum_{i < factor} x[r][factor j + i] - factor mu_r) / (sqrt(factor) sigma_r)
    for j < nt // factor (a trailing partial block is dropped): the sum of a
    block of white noise N(mu_r, sigma_r^2) has mean factor mu_r and deviation
    sqrt(factor) sigma_r, so d is N(0, 1) noise.  Plain loops in FP64."""
    x = np.asarray(x, np.float64)
    ndm, nt = x.shape
    mu = np.broadcast_to(np.asarray(mu, np.float64), (ndm,))
    sigma = np.broadcast_to(np.asarray(sigma, np.float64), (ndm,))
    nb = nt // factor
    out = np.empty((ndm, nb))
    for r in range(ndm):
        for j in range(nb):
            acc = 0.0
            for i in range(factor):
                acc += x[r, factor * j + i]
            out[r, j] = (acc - factor * mu[r]) / (np.sqrt(factor) * sigma[r])
    return out


def unpack(theta):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + n], np.float64).reshape(shp)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SHAPES])


def bf16(v):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(v, np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _conv(a, W, b):
    """b[c] + sum_{ci,k} W[c][ci][k] a[ci][p + k - 4] for every p (zero padding)."""
    ci_n = a.shape[0]
    ap = np.zeros((ci_n, P + 2 * PAD))
    ap[:, PAD:PAD + P] = a
    out = np.empty((W.shape[0], P))
    for c in range(W.shape[0]):
        acc = np.full(P, b[c])
        for ci in range(ci_n):
            for k in range(K):
                acc += W[c, ci, k] * ap[ci, k:k + P]
        out[c] = acc
    return out


def forward(theta, x, rounding=True):
    """Returns (z, cache) for one block x[256]."""
    q = unpack(theta)
    rd = bf16 if rounding else (lambda v: np.asarray(v, np.float64))
    W1, W2, W3 = rd(q["W1"]), rd(q["W2"]), rd(q["W3"])
    a0 = rd(np.asarray(x, np.float64).reshape(1, P))
    h1 = _conv(a0, W1, q["b1"])
    a1 = rd(np.maximum(h1, 0.0))
    h2 = _conv(a1, W2, q["b2"])
    a2 = rd(np.maximum(h2, 0.0))
    h3 = _conv(a2, W3, q["b3"])
    a3 = np.maximum(h3, 0.0)
    arg = np.argmax(a3, axis=1)  # first maximum
    g = a3[np.arange(C), arg]
    z = float(q["b4"][0] + np.dot(q["W4"], g))
    return z, dict(a0=a0, a1=a1, a2=a2, h1=h1, h2=h2, h3=h3, g=g, arg=arg, W1=W1, W2=W2, W3=W3, q=q)


def loss_of(z, y):
    return float(np.logaddexp(0.0, z) - y * z)


def backward(theta, x, y, rounding=True):
    """(loss, gradient vector) of one block with label y."""
    z, cc = forward(theta, x, rounding)
    q = cc["q"]
    dz = 1.0 / (1.0 + np.exp(-z)) - y
    g = {name: np.zeros(shp) for name, shp in SHAPES}
    g["W4"] = dz * cc["g"]
    g["b4"][0] = dz
    dh3 = np.zeros((C, P))
    for c in range(C):
        p = cc["arg"][c]
        if cc["h3"][c, p] > 0.0:
            dh3[c, p] = dz * q["W4"][c]

    def conv_back(dh, a_in, W):
        ci_n = a_in.shape[0]
        ap = np.zeros((ci_n, P + 2 * PAD))
        ap[:, PAD:PAD + P] = a_in
        dW = np.zeros(W.shape)
        da = np.zeros((ci_n, P + 2 * PAD))
        for c in range(W.shape[0]):
            for ci in range(ci_n):
                for k in range(K):
                    dW[c, ci, k] = np.dot(dh[c], ap[ci, k:k + P])
                    da[ci, k:k + P] += W[c, ci, k] * dh[c]
        return dW, dh.sum(axis=1), da[:, PAD:PAD + P]

    g["W3"], g["b3"], da2 = conv_back(dh3, cc["a2"], cc["W3"])
    dh2 = da2 * (cc["h2"] > 0.0)
    g["W2"], g["b2"], da1 = conv_back(dh2, cc["a1"], cc["W2"])
    dh1 = da1 * (cc["h1"] > 0.0)
    g["W1"], g["b1"], _ = conv_back(dh1, cc["a0"], cc["W1"])
    return loss_of(z, y), pack(g)


def batch_gradient(theta, X, Y, rounding=True):
    """Mean loss and mean gradient over blocks X[n][256], labels Y[n]."""
    tot, grad = 0.0, np.zeros(N_PARAMS)
    for x, y in zip(X, Y):
        l, gr = backward(theta, x, float(y), rounding)
        tot += l
        grad += gr
    return tot / len(X), grad / len(X)


def adam(theta, m, v, grad, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (step counts from 1); returns new (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed):
    """He-style initial parameters (float32 values)."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shp in SHAPES:
        if name.startswith("W"):
            fan_in = shp[1] * shp[2] if len(shp) == 3 else shp[0]
            d[name] = rng.normal(0.0, np.sqrt(2.0 / fan_in), shp)
        else:
            d[name] = np.zeros(shp)
    return pack(d).astype(np.float32)
