"""FP64 reference of the E-step of a two-level model whose leaf plate is a chain.

TEST INFRASTRUCTURE ONLY: the test-suite and the benchmark's CPU-baseline
and reference legs are the only callers.  Nothing here imports the CUDA package.

The chain plate follows the autoregressive timeseries of App. F's Covid
model: every region c of an instance has T daily latents z_{c,0..T-1}; the
first day's prior depends on the instance's root latent, every later day's on
the previous day,

  z_{c,0} | g   ~ the leaf level's prior given the root sample (N(g, a I), or
                  N(g[:D], diag exp g[D:])),
  z_{c,d} | z_{c,d-1} ~ N(z_{c,d-1}, b I)        (random walk, b = prior_b),

each day has its own observations and its own factorised Gaussian proposal,
and under massively parallel sampling each (region, day) is its own latent
with its own sample index.  Eq. mp_iw then factorises along each chain
(Sec. 6's recursion with the previous day as the parent), leaves to root:

  h_{c,d}[k]     = sum_n log p(x | z_{c,d}^k) - log q_{c,d}(z_{c,d}^k)       (Eq. rmp)
  S_{c,d}[j, k]  = log N(z_{c,d}^k; z_{c,d-1}^j, b I) + h_{c,d}[k] + B_{c,d+1}[k]   (d >= 1)
  B_{c,d}[j]     = log (1/K) sum_k exp S_{c,d}[j, k]          (B_{c,T} = 0)
  S_{c,0}[p, k]  = log p(z_{c,0}^k | g^p) + h_{c,0}[k] + B_{c,1}[k]
  L_c[p]         = log (1/K) sum_k exp S_{c,0}[p, k]                          (Eq. Prmp)
  A[p]           = log p(g^p) - log q(g^p) + sum_c L_c[p],   log P_MP = LSE A - log K,
and root to leaves (Eq. mmp with indicator moments):
  W = softmax A,
  w_{c,0}[k] = sum_p W[p] exp(S_{c,0}[p, k] - L_c[p] - log K),
  w_{c,d}[k] = sum_j w_{c,d-1}[j] exp(S_{c,d}[j, k] - B_{c,d}[j] - log K),
  moments    = sum_k w[k] (z^k, (z^k)^2) per (region, day).

Layout: the leaf level's elements are (region, day) pairs, element c T + d;
q per level [n, 2, dim] (loc, scale); eps per level [n, K, dim].
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

LIK_NONE, LIK_GAUSS, LIK_BERNOULLI_LOGIT, LIK_POISSON_LOG = 0, 1, 2, 3
PRIOR_STD_NORMAL, PRIOR_NORMAL_FIXED_VAR, PRIOR_NORMAL_MEAN_LOGVAR = 0, 1, 2


def _lognorm(x, mean, var):
    return -0.5 * (np.log(2.0 * math.pi * var) + (x - mean) ** 2 / var)


def _loglik(lik, lik_var, x, y, z):
    """x [N, D], y [N], z [K, D] -> [K]."""
    if lik == LIK_NONE:
        return np.zeros(z.shape[0])
    s = z @ x.T
    if lik == LIK_GAUSS:
        return _lognorm(y[None, :], s, lik_var).sum(1)
    if lik == LIK_BERNOULLI_LOGIT:
        return (y[None, :] * s - np.logaddexp(0.0, s)).sum(1)
    if lik == LIK_POISSON_LOG:
        return (y[None, :] * s - np.exp(s) - special.gammaln(y[None, :] + 1.0)).sum(1)
    raise ValueError("likelihood not supported on a chain level")


def _lse(a, axis):
    m = np.max(a, axis=axis, keepdims=True)
    m = np.where(np.isfinite(m), m, 0.0)
    return np.squeeze(m + np.log(np.sum(np.exp(a - m), axis=axis, keepdims=True)), axis=axis)


def _first_prior(u, z, g):
    """log p(z_{c,0}^k | g^p) for all (p, k): z [K, D], g [K, 2D or D] -> [K_p, K]."""
    D = u.dim
    if u.prior == PRIOR_NORMAL_FIXED_VAR:
        return _lognorm(z[None, :, :], g[:, None, :], u.prior_a).sum(-1)
    if u.prior == PRIOR_NORMAL_MEAN_LOGVAR:
        return _lognorm(z[None, :, :], g[:, None, :D], np.exp(g[:, None, D:])).sum(-1)
    raise ValueError("first-day prior must be N(parent, a I) or N(mean, diag exp logvar)")


def estep(model, q, K: int, eps, root_extra=None) -> dict:
    """One E-step in FP64 of a model [root level, chain level] (every instance).

    root_extra: [n_inst, K] or None; added to each root's sum over its chains
    (the sums of chains the model does not hold: a sharded plate).

    Returns log_pmp [n_inst], w per level ([n0, K], [n1, K]), mom per level
    ([n, 2, dim]), z per level, and the chain's tables: L [n_chains, K]
    (first day, per root sample) and B [n1, K] (B_{c,d} for d >= 1, 0 at d = 0).
    """
    r, u = model.levels
    T = int(getattr(u, "chain", 1) or 1)
    assert r.prior == PRIOR_STD_NORMAL and r.lik == LIK_NONE and u.n % T == 0
    D0, D = r.dim, u.dim
    q0 = np.asarray(q[0], np.float64).reshape(r.n, 2, D0)
    q1 = np.asarray(q[1], np.float64).reshape(u.n, 2, D)
    z0 = q0[:, None, 0, :] + q0[:, None, 1, :] * np.asarray(eps[0], np.float64).reshape(r.n, K, D0)
    z1 = q1[:, None, 0, :] + q1[:, None, 1, :] * np.asarray(eps[1], np.float64).reshape(u.n, K, D)
    n_ch = u.n // T
    chain_par = np.asarray(u.parent, np.int64)[::T]
    lK = math.log(K)
    h = np.zeros((u.n, K))
    for e in range(u.n):
        x = np.asarray(u.x[e], np.float64).reshape(-1, D) if u.lik else None
        y = np.asarray(u.y[e], np.float64) if u.lik else None
        h[e] = _loglik(u.lik, u.lik_var, x, y, z1[e]) - _lognorm(z1[e], q1[e, 0], q1[e, 1] ** 2).sum(1)

    def S_step(e):
        """S_{c,d}[j, k] of element e = c T + d, d >= 1 (without the B term)."""
        return _lognorm(z1[e][None, :, :], z1[e - 1][:, None, :], u.prior_b).sum(-1) + h[e][None, :]

    B = np.zeros((u.n, K))
    L = np.zeros((n_ch, K))
    S0 = {}
    for c in range(n_ch):
        e0 = c * T
        nxt = np.zeros(K)                       # B_{c,d+1}
        for d in range(T - 1, 0, -1):
            e = e0 + d
            B[e] = _lse(S_step(e) + nxt[None, :], axis=1) - lK
            nxt = B[e]
        g = z0[chain_par[c]]
        S0[c] = _first_prior(u, z1[e0], g) + h[e0][None, :] + nxt[None, :]
        L[c] = _lse(S0[c], axis=1) - lK
    log_pmp = np.zeros(r.n)
    w0 = np.zeros((r.n, K))
    w1 = np.zeros((u.n, K))
    for i in range(r.n):
        f0 = (_lognorm(z0[i], 0.0, r.prior_a) - _lognorm(z0[i], q0[i, 0], q0[i, 1] ** 2)).sum(1)
        A = f0 + L[chain_par == i].sum(0) + (0.0 if root_extra is None else np.asarray(root_extra, np.float64)[i])
        lse = float(_lse(A, axis=0))
        log_pmp[i] = lse - lK
        w0[i] = np.exp(A - lse)
    for c in range(n_ch):
        e0 = c * T
        i = chain_par[c]
        P = np.exp(S0[c] - L[c][:, None] - lK)   # P(k | p): rows sum to one
        w1[e0] = w0[i] @ P
        for d in range(1, T):
            e = e0 + d
            nxt = B[e + 1] if d + 1 < T else np.zeros(K)
            P = np.exp(S_step(e) + nxt[None, :] - B[e][:, None] - lK)
            w1[e] = w1[e - 1] @ P
    mom0 = np.stack([np.einsum("ik,ikd->id", w0, z0), np.einsum("ik,ikd->id", w0, z0 ** 2)], 1)
    mom1 = np.stack([np.einsum("ek,ekd->ed", w1, z1), np.einsum("ek,ekd->ed", w1, z1 ** 2)], 1)
    return {"log_pmp": log_pmp, "w": [w0, w1], "mom": [mom0, mom1], "z": [z0, z1], "L": L, "B": B}
