"""FP64 reference of the E-step with a parent-conditioned (non-factorised)
massively parallel proposal and the permutation copy scheme.

TEST INFRASTRUCTURE ONLY: the test-suite and the benchmark's CPU-baseline
and reference legs are the only callers.  Nothing here imports the CUDA
package.

App. A.2 defines Q_MP(z) = prod_i Q_MP(z_i | z_j, j in qa(i)) from a
single-sample proposal Q(z_i' | z_j') and a scheme that picks which of the K
parent copies each child copy is drawn from; the paper's experiments use a
uniformly random permutation.  Here the child's single-sample proposal is a
Gaussian centred on its parent's sample (a residual proposal):

  Q(z_i | z_p) = N(z_i; z_p[:D] + loc_i, diag scale_i^2),
  z_i^k = z_p^{s_i(k)}[:D] + loc_i + scale_i eps_i^k,     s_i a permutation of 0..K-1.

With s_i given, the density of copy k under Q_MP given all parent copies is
Q(z_i^k | z_p^{s_i(k)}): it depends on k alone, so Eq. rmp's denominator is a
per-sample term and Eq. mp_iw keeps the factorisation of the factorised case:

  h_i[k]      = sum_n log p(x_in | z_i^k) - log N(z_i^k; z_p^{s_i(k)}[:D] + loc_i, scale_i^2)
  L_i[p]      = log (1/K) sum_k exp(log p(z_i^k | z_p^p) + h_i[k])           (Eq. Prmp)
  A[p]        = log p(z_root^p) - log q(z_root^p) + sum_i L_i[p],   log P_MP = LSE A - log K
  W = softmax A;  P_i(k | p) = exp(log p(z_i^k | z_p^p) + h_i[k] - L_i[p] - log K)
  w_i[k]      = sum_p W[p] P_i(k | p)                                        (Eq. mmp)

The M-step of the residual proposal matches the moments of the residual
d_i = z_i - z_p[:D] under the estimator's joint weights of (parent sample,
child sample), W[p] P_i(k | p):

  E d   = E z_i - E z_p[:D],
  E d^2 = E z_i^2 - 2 E[z_i z_p[:D]] + E z_p[:D]^2,
  E[z_i z_p[:D]] = sum_k z_i^k (sum_p W[p] P_i(k | p) z_p^p[:D])     (pairwise moment).

Two-level models (root with the N(0, a I) prior and a factorised Gaussian
proposal; children with the N(parent, a I) or N(mean, diag exp logvar)
prior); q per level [n, 2, dim] (loc, scale; the children's loc is the
residual offset), eps per level [n, K, dim], perm [n_1, K] (s_i).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

LIK_NONE, LIK_GAUSS, LIK_BERNOULLI_LOGIT, LIK_POISSON_LOG = 0, 1, 2, 3
PRIOR_NORMAL_FIXED_VAR, PRIOR_NORMAL_MEAN_LOGVAR = 1, 2


def _lognorm(x, mean, var):
    return -0.5 * (np.log(2.0 * math.pi * var) + (x - mean) ** 2 / var)


def _loglik(lik, lik_var, x, y, z):
    if lik == LIK_NONE:
        return np.zeros(z.shape[0])
    s = z @ x.T
    if lik == LIK_GAUSS:
        return _lognorm(y[None, :], s, lik_var).sum(1)
    if lik == LIK_BERNOULLI_LOGIT:
        return (y[None, :] * s - np.logaddexp(0.0, s)).sum(1)
    if lik == LIK_POISSON_LOG:
        return (y[None, :] * s - np.exp(s) - special.gammaln(y[None, :] + 1.0)).sum(1)
    raise ValueError("likelihood not supported here")


def _lse(a, axis):
    m = np.max(a, axis=axis, keepdims=True)
    m = np.where(np.isfinite(m), m, 0.0)
    return np.squeeze(m + np.log(np.sum(np.exp(a - m), axis=axis, keepdims=True)), axis=axis)


def child_prior(u, z, zp):
    """log p(z^k | zp^p) for all (p, k): z [K, D], zp [K, Dp] -> [K_p, K]."""
    D = u.dim
    if u.prior == PRIOR_NORMAL_FIXED_VAR:
        return _lognorm(z[None, :, :], zp[:, None, :D], u.prior_a).sum(-1)
    if u.prior == PRIOR_NORMAL_MEAN_LOGVAR:
        return _lognorm(z[None, :, :], zp[:, None, :D], np.exp(zp[:, None, D:])).sum(-1)
    raise ValueError("child prior must be N(parent, a I) or N(mean, diag exp logvar)")


def draw_perm(seed: int, it: int, n: int, K: int) -> np.ndarray:
    """The counter-based parent-copy permutations [n, K]: per element e the K
    keys are word (k mod 4) of Philox4x32-10 (the oracle's own generator) with
    counter (k div 4, e mod 2^32, (e div 2^32) | 2^30, it) and key seed; copies
    ordered by (key, k), perm[e][rank] = k."""
    from oracle import oracle as O
    key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]
    out = np.zeros((n, K), np.int64)
    for e in range(n):
        keys = np.zeros(K, np.uint64)
        for k0 in range(0, K, 4):
            w = O.philox4x32_10([k0 >> 2, e & 0xFFFFFFFF, ((e >> 32) & 0xFFFFFFFF) | 0x40000000, it & 0xFFFFFFFF], key)
            for j in range(min(4, K - k0)):
                keys[k0 + j] = w[j]
        out[e] = np.lexsort((np.arange(K), keys))
    return out


def samples(model, q, K: int, eps, perm):
    """The reparameterised draws: root z = loc + scale eps; child z^k = z_p^{s(k)}[:D] + loc + scale eps^k."""
    r, u = model.levels
    D = u.dim
    q0 = np.asarray(q[0], np.float64).reshape(r.n, 2, r.dim)
    q1 = np.asarray(q[1], np.float64).reshape(u.n, 2, D)
    z0 = q0[:, None, 0, :] + q0[:, None, 1, :] * np.asarray(eps[0], np.float64).reshape(r.n, K, r.dim)
    perm = np.asarray(perm, np.int64).reshape(u.n, K)
    par = np.asarray(u.parent, np.int64)
    base = z0[par[:, None], perm, :D]                                 # [n1, K, D] z_p^{s(k)}[:D]
    z1 = base + q1[:, None, 0, :] + q1[:, None, 1, :] * np.asarray(eps[1], np.float64).reshape(u.n, K, D)
    return z0, z1, base


def estep(model, q, K: int, eps, perm) -> dict:
    """One E-step in FP64.  Returns log_pmp [n_inst], w per level, mom per level
    ([n, 2, dim]: the root's (E z, E z^2); the children's residual moments
    (E d, E d^2)), zmom1 (the children's (E z, E z^2)), cross [n1, D]
    (E[z_i z_p[:D]]), z per level, logL [n1, K]."""
    r, u = model.levels
    D = u.dim
    q0 = np.asarray(q[0], np.float64).reshape(r.n, 2, r.dim)
    q1 = np.asarray(q[1], np.float64).reshape(u.n, 2, D)
    z0, z1, base = samples(model, q, K, eps, perm)
    par = np.asarray(u.parent, np.int64)
    lK = math.log(K)
    S = np.zeros((u.n, K, K))
    for e in range(u.n):
        x = np.asarray(u.x[e], np.float64).reshape(-1, D) if u.lik else None
        y = np.asarray(u.y[e], np.float64) if u.lik else None
        h = _loglik(u.lik, u.lik_var, x, y, z1[e]) - _lognorm(z1[e], base[e] + q1[e, 0], q1[e, 1] ** 2).sum(1)
        S[e] = child_prior(u, z1[e], z0[par[e]]) + h[None, :]
    logL = _lse(S, axis=2) - lK
    log_pmp = np.zeros(r.n)
    w0 = np.zeros((r.n, K))
    for i in range(r.n):
        f0 = (_lognorm(z0[i], 0.0, r.prior_a) - _lognorm(z0[i], q0[i, 0], q0[i, 1] ** 2)).sum(1)
        A = f0 + logL[par == i].sum(0)
        lse = float(_lse(A, axis=0))
        log_pmp[i] = lse - lK
        w0[i] = np.exp(A - lse)
    w1 = np.zeros((u.n, K))
    cross = np.zeros((u.n, D))
    for e in range(u.n):
        J = w0[par[e]][:, None] * np.exp(S[e] - logL[e][:, None] - lK)   # joint weights [p, k]
        w1[e] = J.sum(0)
        cross[e] = np.einsum("pk,kd,pd->d", J, z1[e], z0[par[e]][:, :D])
    mom0 = np.stack([np.einsum("ik,ikd->id", w0, z0), np.einsum("ik,ikd->id", w0, z0 ** 2)], 1)
    zmom1 = np.stack([np.einsum("ek,ekd->ed", w1, z1), np.einsum("ek,ekd->ed", w1, z1 ** 2)], 1)
    pm1, pm2 = mom0[par, 0, :D], mom0[par, 1, :D]
    mom1 = np.stack([zmom1[:, 0] - pm1, zmom1[:, 1] - 2.0 * cross + pm2], 1)
    return {"log_pmp": log_pmp, "w": [w0, w1], "mom": [mom0, mom1], "zmom1": zmom1, "cross": cross,
            "z": [z0, z1], "logL": logL}
