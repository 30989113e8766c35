"""Pins of the chain-plate oracle (oracle/chain.py): a two-level model whose
leaf plate is a daily random walk per region (the Covid model's
autoregressive timeseries, App. F), every (region, day) its own latent.

* brute force: literal enumeration of every index vector over the root and
  all days (oracle/brute.py, scipy densities) for Poisson-log and Gaussian
  observations, one- and two-dimensional latents, several instances, and a
  first day under a (mean, log-variance) root;
* special case: chains of length 1 are an ordinary two-level model, whose
  estimator the C oracle computes (shared noise);
* closed form: on a linear-Gaussian chain (Gaussian days) the average of
  P_MP / p(y) over independent draws is 1, p(y) from Gaussian conditioning,
  and the moments approach the exact posterior marginals as K grows;
* weights of every latent sum to one.
"""
import copy

import numpy as np
import pytest

from oracle import brute
from oracle import chain as C
from oracle import oracle as O
from paper_2503_08264_gb300 import synth as S


def _mean_logvar_first_day(model):
    """The same chain with a (mean, log-variance) root and day 0 ~ N(mean, diag exp logvar)."""
    m = copy.deepcopy(model)
    m.levels[0].dim = 2 * m.levels[1].dim
    m.levels[1].prior = S.PRIOR_NORMAL_MEAN_LOGVAR
    return m


def _cases():
    yield "poisson_R1_T3_K3", S.chain_poisson(n_inst=1, R=1, T=3, D=1, seed=1), 3
    yield "mean_logvar_day0_R2_T2_K3", _mean_logvar_first_day(S.chain_poisson(n_inst=1, R=2, T=2, D=1, seed=9)), 3
    yield "poisson_R2_T2_K3", S.chain_poisson(n_inst=1, R=2, T=2, D=1, seed=2), 3
    yield "gauss_D2_R1_T3_K3", S.chain_poisson(n_inst=1, R=1, T=3, D=2, seed=3, lik=S.LIK_GAUSS, n_obs=2), 3
    yield "poisson_R1_T4_K2", S.chain_poisson(n_inst=1, R=1, T=4, D=1, seed=4, n_obs=3), 2
    yield "two_instances_R1_T2_K3", S.chain_poisson(n_inst=2, R=1, T=2, D=1, seed=5), 3


@pytest.mark.parametrize("name,model,K", list(_cases()), ids=lambda v: v if isinstance(v, str) else "")
def test_chain_matches_enumeration(name, model, K):
    q = S.random_q(model, seed=11, loc_scale=0.4, sd_lo=0.4, sd_hi=1.0)
    eps = S.noise(model, K, seed=12)
    o = C.estep(model, q, K, eps)
    for inst in range(model.n_inst):
        b = brute.estep_instance_chain(model, q, o["z"], K, inst)
        np.testing.assert_allclose(o["log_pmp"][inst], b["log_pmp"], rtol=1e-12)
        for (l, e), we in b["w"].items():
            np.testing.assert_allclose(o["w"][l][e], we, rtol=1e-10, atol=1e-14)
            np.testing.assert_allclose(o["mom"][l][e], b["mom"][(l, e)], rtol=1e-10, atol=1e-13)


def test_chain_of_length_one_is_the_tree_estimator():
    model = S.chain_poisson(n_inst=2, R=5, T=1, D=2, seed=21, n_obs=3)
    K = 16
    q = S.random_q(model, seed=22, loc_scale=0.4, sd_lo=0.4, sd_hi=1.0)
    eps = S.noise(model, K, seed=23)
    a = C.estep(model, q, K, eps)
    g = O.estep(model, q, K, eps=eps)
    np.testing.assert_allclose(a["log_pmp"], g["log_pmp"], rtol=1e-12)
    for l in range(2):
        np.testing.assert_allclose(a["w"][l], g["w"][l], rtol=1e-10, atol=1e-14)
        np.testing.assert_allclose(a["mom"][l], g["mom"][l], rtol=1e-10, atol=1e-13)


def test_chain_weights_sum_to_one():
    model = S.chain_poisson(n_inst=2, R=3, T=6, D=1, seed=31)
    K = 24
    o = C.estep(model, S.random_q(model, seed=32), K, S.noise(model, K, seed=33))
    for l in range(2):
        np.testing.assert_allclose(o["w"][l].sum(1), 1.0, rtol=1e-12)
    assert np.all(np.isfinite(o["B"])) and np.all(np.isfinite(o["L"]))


def _chain_gauss_exact(model):
    """log p(y) and the posterior of (g, z) for the linear-Gaussian chain:
    g ~ N(0, a0), z_{c,0} = g + N(0, a), z_{c,d} = z_{c,d-1} + N(0, b),
    y_{c,d} = x z_{c,d} + N(0, v) (D = 1, one observation per day)."""
    from scipy import stats
    r, u = model.levels
    T = u.chain
    n = u.n
    A = np.zeros((n + 1, n + 1))          # latent = A @ innovations (g first)
    var = np.zeros(n + 1)
    var[0] = r.prior_a
    A[0, 0] = 1.0
    for e in range(n):
        prev = 0 if e % T == 0 else e        # index of the parent in the latent vector
        A[e + 1] = A[prev]
        A[e + 1, e + 1] = 1.0
        var[e + 1] = u.prior_a if e % T == 0 else u.prior_b
    C = A @ np.diag(var) @ A.T
    P = np.zeros((n, n + 1))
    P[np.arange(n), np.arange(n) + 1] = u.x[:, 0, 0].astype(np.float64)
    Sy = P @ C @ P.T + u.lik_var * np.eye(n)
    y = u.y[:, 0].astype(np.float64)
    lpy = stats.multivariate_normal(np.zeros(n), Sy).logpdf(y)
    G = C @ P.T @ np.linalg.inv(Sy)
    return lpy, G @ y, C - G @ P @ C


def test_chain_gaussian_unbiased_evidence_and_exact_marginals():
    """E[P_MP] = p(y) (Sec. 3.2) with p(y) from Gaussian conditioning, and the
    MPIW moments approach the exact posterior marginals as K grows (App. C)."""
    import math
    model = S.chain_poisson(n_inst=1, R=2, T=5, D=1, seed=41, lik=S.LIK_GAUSS, lik_var=0.3)
    lpy, mean, cov = _chain_gauss_exact(model)
    sd = np.sqrt(np.diag(cov))
    q = [np.array([[[mean[0]], [1.3 * sd[0]]]]), np.stack([mean[1:], 1.3 * sd[1:]], 1)[:, :, None]]
    K, R = 8, 300
    ratios = np.array([math.exp(C.estep(model, q, K, S.noise(model, K, seed=500 + s))["log_pmp"][0] - lpy)
                       for s in range(R)])
    se = ratios.std(ddof=1) / math.sqrt(R)
    assert abs(ratios.mean() - 1.0) < 4 * se + 1e-3, (ratios.mean(), se)
    errs = []
    q0 = S.initial_q(model)
    for K in (16, 512):
        o = C.estep(model, q0, K, S.noise(model, K, seed=7))
        m1 = np.concatenate([o["mom"][0][:, 0, 0], o["mom"][1][:, 0, 0]])
        errs.append(np.max(np.abs(m1 - mean) / sd))
    assert errs[1] < 0.5 and errs[1] < errs[0], errs
