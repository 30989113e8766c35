"""FP64 reference of the E-step with the root's two halves as separate latents.

TEST INFRASTRUCTURE ONLY: the test-suite, the package smoke check and the
benchmark's CPU-baseline leg are the only callers.  Nothing here imports the
CUDA package.

The grouped path gives the root of a two-level model (hierarchical logistic
regression, App. F's MovieLens model) one index k for the pair (mu, psi).  In
that model mu and psi are separate latents (the global mean and the global
log-variance), so under massively parallel sampling each has its own index
and a user's prior factor p(z_m | mu, psi) depends on two parent indices: the
K^(number of parents) tables of the Limitations section (grouping latents,
as the grouped path does, is the alternative that section names).  With
every latent its own index, Eq. mp_iw factorises over the users given
(k_mu, k_psi):

  f_mu[a]      = log N(mu^a; 0, v I) - log q(mu^a)                 (likewise f_psi[b])
  h_m[k]       = sum_n log p(x_mn | z_m^k) - log q_m(z_m^k)          (Eq. rmp)
  S_m[a, b, k] = log N(z_m^k; mu^a, diag exp(psi^b)) + h_m[k]
  L_m[a, b]    = log (1/K) sum_k exp S_m[a, b, k]                    (Eq. Prmp, user summed out)
  A[a, b]      = f_mu[a] + f_psi[b] + sum_m L_m[a, b]
  log P_MP     = log (1/K^2) sum_{a, b} exp A[a, b]
  W[a, b]      = exp(A[a, b]) / sum exp A                            (joint root weights)
  w_mu[a]      = sum_b W[a, b],   w_psi[b] = sum_a W[a, b]            (Eq. mmp, indicator moments)
  w_m[k]       = sum_{a, b} W[a, b] exp(S_m[a, b, k] - L_m[a, b] - log K)
  moments      = sum_k w[k] (z^k, (z^k)^2) per latent, mu with w_mu, psi with w_psi.

Samples are the reparameterised draws z = loc + scale * eps (Gaussian q), the
same eps for both halves of the root as for the grouped root: mu^a is
dimensions [0, D) of root sample a and psi^b dimensions [D, 2D) of root
sample b.  Densities are written out here with numpy (log N, log-sigmoid via
logaddexp, Poisson via gammaln).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

LIK_NONE, LIK_GAUSS, LIK_BERNOULLI_LOGIT, LIK_POISSON_LOG = 0, 1, 2, 3


def _lognorm(x, mean, var):
    return -0.5 * (np.log(2.0 * math.pi * var) + (x - mean) ** 2 / var)


def _loglik(lik: int, lik_var: float, x, y, z):
    """x [N, D], y [N], z [K, D] -> [K] summed log-likelihood of the element's observations."""
    if lik == LIK_NONE:
        return np.zeros(z.shape[0])
    s = z @ x.T                                   # [K, N]
    if lik == LIK_GAUSS:
        return _lognorm(y[None, :], s, lik_var).sum(1)
    if lik == LIK_BERNOULLI_LOGIT:
        return (y[None, :] * s - np.logaddexp(0.0, s)).sum(1)
    if lik == LIK_POISSON_LOG:
        return (y[None, :] * s - np.exp(s) - special.gammaln(y[None, :] + 1.0)).sum(1)
    raise ValueError("likelihood not supported by the split root")


def _lse(a, axis=None):
    m = np.max(a, axis=axis, keepdims=True)
    m = np.where(np.isfinite(m), m, 0.0)
    out = m + np.log(np.sum(np.exp(a - m), axis=axis, keepdims=True))
    return np.squeeze(out, axis=axis) if axis is not None else float(out.reshape(()))


def estep(model, q, K: int, eps) -> dict:
    """One split-root E-step in FP64 over every instance of a two-level model.

    model: levels[0] = roots (dim 2D, N(0, prior_a I) prior, Gaussian q, no
    likelihood), levels[1] = users (dim D, prior N(mu, diag exp(psi)));
    q: per level [n, 2, dim] (loc, scale); eps: per level [n, K, dim].
    Returns log_pmp [n_inst]; w_mu, w_psi [n_inst, K]; w (users) [n1, K];
    logL [n1, K, K] (L_m[a, b]); mom per level [n, 2, dim]; z per level.
    """
    r, u = model.levels
    D = u.dim
    assert r.dim == 2 * D and u.prior == 2 and r.prior == 0 and r.lik == LIK_NONE
    q0 = np.asarray(q[0], np.float64).reshape(r.n, 2, 2 * D)
    q1 = np.asarray(q[1], np.float64).reshape(u.n, 2, D)
    z0 = q0[:, None, 0, :] + q0[:, None, 1, :] * np.asarray(eps[0], np.float64).reshape(r.n, K, 2 * D)
    z1 = q1[:, None, 0, :] + q1[:, None, 1, :] * np.asarray(eps[1], np.float64).reshape(u.n, K, D)
    par = np.asarray(u.parent, np.int64)
    log_pmp = np.zeros(r.n)
    w_mu, w_psi = np.zeros((r.n, K)), np.zeros((r.n, K))
    w1 = np.zeros((u.n, K))
    logL = np.zeros((u.n, K, K))
    mom0, mom1 = np.zeros((r.n, 2, 2 * D)), np.zeros((u.n, 2, D))
    for i in range(r.n):
        mu, psi = z0[i, :, :D], z0[i, :, D:]
        # root factors of each half: prior N(0, v) minus the proposal's log density
        f_mu = (_lognorm(mu, 0.0, r.prior_a) - _lognorm(mu, q0[i, 0, :D], q0[i, 1, :D] ** 2)).sum(1)
        f_psi = (_lognorm(psi, 0.0, r.prior_a) - _lognorm(psi, q0[i, 0, D:], q0[i, 1, D:] ** 2)).sum(1)
        users = np.nonzero(par == i)[0]
        prec = np.exp(-psi)                                               # [K_b, D]
        lognorm_b = -0.5 * (D * math.log(2.0 * math.pi) + psi.sum(1))     # [K_b]

        def S_of(m):
            # S[a, b, k] = sum_d log N(z_m^k_d; mu^a_d, exp(psi^b_d)) + h_m[k]
            #            = lognorm_b[b] - 1/2 sum_d prec[b, d] (z_m^k_d - mu^a_d)^2 + h_m[k]
            h = _loglik(u.lik, u.lik_var, np.asarray(u.x[m], np.float64).reshape(-1, D) if u.lik else None,
                        np.asarray(u.y[m], np.float64) if u.lik else None, z1[m]) \
                - _lognorm(z1[m], q1[m, 0], q1[m, 1] ** 2).sum(1)
            sq = (z1[m][None, :, :] - mu[:, None, :]) ** 2                # [K_a, K, D]
            quad = (sq.reshape(K * K, D) @ prec.T).reshape(K, K, K)       # [a, k, b]
            return lognorm_b[None, :, None] - 0.5 * quad.transpose(0, 2, 1) + h[None, None, :]

        A = f_mu[:, None] + f_psi[None, :]
        for m in users:
            logL[m] = _lse(S_of(m), axis=2) - math.log(K)
            A = A + logL[m]
        lse = _lse(A)
        log_pmp[i] = lse - 2.0 * math.log(K)
        W = np.exp(A - lse)
        w_mu[i], w_psi[i] = W.sum(1), W.sum(0)
        for m in users:
            P = np.exp(S_of(m) - logL[m][:, :, None] - math.log(K))      # P(k | a, b): rows sum to one
            w1[m] = np.einsum("ab,abk->k", W, P)
            mom1[m, 0] = w1[m] @ z1[m]
            mom1[m, 1] = w1[m] @ (z1[m] ** 2)
        mom0[i, 0, :D], mom0[i, 1, :D] = w_mu[i] @ mu, w_mu[i] @ mu ** 2
        mom0[i, 0, D:], mom0[i, 1, D:] = w_psi[i] @ psi, w_psi[i] @ psi ** 2
    return {"log_pmp": log_pmp, "w_mu": w_mu, "w_psi": w_psi, "w": w1, "logL": logL,
            "mom": [mom0, mom1], "z": [z0, z1]}
