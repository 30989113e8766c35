"""FP64 reference of the learned warm start: a small proposal network.

TEST INFRASTRUCTURE ONLY: the test-suite and the package smoke check are
the only callers; nothing here imports the CUDA package.

The network has no counterpart in the paper: it is the amortised warm start
of the method (q for a new instance's users predicted from their data, plain
QEM continuing from there).  For one user with N items:

  features   f = [ sum_n x_n y_n (D), sum_n x_n (D), sum_n y_n (1) ]      (2D + 1 = 37)
  layers     h1 = relu(W1 f + b1)   (128)
             h2 = relu(W2 h1 + b2)  (128)
             o  = W3 h2 + b3        (2D = 36)
  proposal   q_net = N(mu = o[:D], diag sigma^2),  sigma = exp(o[D:])

Loss of a batch: the mean over users of the Gaussian KL divergence from the
QEM proposal N(m, diag s^2) to q_net, summed over dimensions,

  KL = sum_d [ log(sigma_d / s_d) + (s_d^2 + (m_d - mu_d)^2) / (2 sigma_d^2) - 1/2 ],

  dKL/dmu_d        = (mu_d - m_d) / sigma_d^2
  dKL/dlog sigma_d = 1 - (s_d^2 + (m_d - mu_d)^2) / sigma_d^2 .

Mixed precision: with bf16=True the operands of every matrix product (the
features or activations, and the weights) are rounded to BF16 (round to
nearest, ties to even) and the products summed exactly (FP64 here, FP32 on
the GPU); the backward pass uses the same rounded operands (the rounding is
passed straight through).

Adam (Kingma & Ba, ICLR 2015): m = b1 m + (1 - b1) g; v = b2 v + (1 - b2) g^2;
theta -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Flat parameter layout: W1 [128][37], b1 [128], W2 [128][128], b2 [128],
W3 [36][128], b3 [36] (row-major, rows = outputs).
"""
from __future__ import annotations

import numpy as np

SIZES = (37, 128, 128, 36)


def n_params(sizes=SIZES) -> int:
    return sum(o * i + o for i, o in zip(sizes[:-1], sizes[1:]))


def unpack(theta: np.ndarray, sizes=SIZES) -> list:
    out, off = [], 0
    for i, o in zip(sizes[:-1], sizes[1:]):
        W = theta[off:off + o * i].reshape(o, i)
        off += o * i
        b = theta[off:off + o]
        off += o
        out.append((W, b))
    return out


def features(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """x [n, N, D], y [n, N] -> [n, 2D + 1]."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    return np.concatenate([np.einsum("und,un->ud", x, y), x.sum(1), y.sum(1, keepdims=True)], axis=1)


def round_bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    u = np.ascontiguousarray(np.asarray(a, np.float32)).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta: np.ndarray, f: np.ndarray, bf16: bool = False):
    """Network output o [n, 36] and the values the backward pass needs."""
    rnd = round_bf16 if bf16 else (lambda a: np.asarray(a, np.float64))
    layers = unpack(np.asarray(theta, np.float64))
    a = np.asarray(f, np.float64)
    cache = []
    for j, (W, b) in enumerate(layers):
        ar, Wr = rnd(a), rnd(W)
        z = ar @ Wr.T + b
        cache.append((ar, Wr, z))
        a = np.maximum(z, 0.0) if j + 1 < len(layers) else z
    return a, cache


def kl(o: np.ndarray, m: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Per-user KL(N(m, s^2) || N(o[:D], exp(o[D:])^2)) summed over dimensions."""
    D = m.shape[1]
    mu, ls = o[:, :D], o[:, D:]
    sig2 = np.exp(2.0 * ls)
    return np.sum(ls - np.log(s) + (s * s + (m - mu) ** 2) / (2.0 * sig2) - 0.5, axis=1)


def loss_grad(theta: np.ndarray, f: np.ndarray, m: np.ndarray, s: np.ndarray, bf16: bool = False):
    """Mean KL over the batch and its gradient (flat, the parameter layout)."""
    o, cache = forward(theta, f, bf16)
    n, D = m.shape
    mu, ls = o[:, :D], o[:, D:]
    sig2 = np.exp(2.0 * ls)
    loss = float(np.mean(kl(o, m, s)))
    g_o = np.concatenate([(mu - m) / sig2, 1.0 - (s * s + (m - mu) ** 2) / sig2], axis=1) / n
    grads = []
    g = g_o
    for j in range(len(cache) - 1, -1, -1):
        ar, Wr, z = cache[j]
        if j + 1 < len(cache):
            g = g * (z > 0.0)
        grads.append((g.T @ ar, g.sum(0)))
        g = g @ Wr
    flat = []
    for gW, gb in reversed(grads):
        flat += [gW.reshape(-1), gb]
    return loss, np.concatenate(flat)


def adam(theta, grad, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step (t >= 1); returns the new (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
