"""Pins of the split-root oracle (oracle/split_root.py): the E-step of a
two-level model whose root halves, the global mean mu and the global
log-variance psi, are separate latents with their own sample indices.

* brute force: literal enumeration of every index vector
  (k_mu, k_psi, k_1, ..., k_M) with scipy densities (oracle/brute.py), for
  Bernoulli-logit, Gaussian and Poisson-log users and for several instances;
* special case: with K = 1 there is one index vector, so the split and the
  grouped estimators coincide (the C oracle computes the grouped one);
* invariant: the split estimator sums over all (k_mu, k_psi) pairs, so
  permuting the psi samples alone leaves log P_MP, the mu weights and every
  user's weights unchanged and permutes the psi weights (the grouped
  estimator, which pairs k_mu = k_psi, changes);
* unbiasedness: with Gaussian users, E[P_MP] = p(x), p(x) by one-dimensional
  Gauss-Hermite quadrature over psi of a closed-form Gaussian density;
* weights of every latent sum to one.
"""
import copy

import numpy as np
import pytest

from oracle import brute
from oracle import oracle as O
from oracle import split_root as R
from paper_2503_08264_gb300 import synth as S


def _with_lik(model, lik: int, seed: int):
    """The same two-level model with the users' observations redrawn for another likelihood."""
    m = copy.deepcopy(model)
    u = m.levels[1]
    rng = np.random.default_rng(seed)
    u.x = (0.5 * rng.standard_normal(u.x.shape)).astype(np.float32)
    if lik == S.LIK_GAUSS:
        u.y = rng.standard_normal(u.y.shape).astype(np.float32)
        u.lik_var = 0.7
    else:
        u.y = rng.poisson(1.5, size=u.y.shape).astype(np.float32)
    u.lik = lik
    return m


def _cases():
    yield "logistic_M2_K3", S.hier_logistic(M=2, N=3, D=2, seed=1), 3
    yield "logistic_M3_K3", S.hier_logistic(M=3, N=4, D=3, seed=2), 3
    yield "logistic_M2_K4", S.hier_logistic(M=2, N=2, D=2, seed=3), 4
    yield "gauss_M2_K3", _with_lik(S.hier_logistic(M=2, N=3, D=2, seed=4), S.LIK_GAUSS, 5), 3
    yield "poisson_M2_K3", _with_lik(S.hier_logistic(M=2, N=3, D=2, seed=6), S.LIK_POISSON_LOG, 7), 3
    yield "batch3_M2_K3", S.hier_logistic_batch(3, M=2, N=3, D=2, seed=8), 3


@pytest.mark.parametrize("name,model,K", list(_cases()), ids=lambda v: v if isinstance(v, str) else "")
def test_split_root_matches_enumeration(name, model, K):
    q = S.random_q(model, seed=21, loc_scale=0.4, sd_lo=0.4, sd_hi=1.0)
    eps = S.noise(model, K, seed=22)
    o = R.estep(model, q, K, eps)
    for inst in range(model.n_inst):
        b = brute.estep_instance_split_root(model, q, o["z"], K, inst)
        assert b["n"] == 2 + int(np.sum(model.levels[1].parent == inst))
        np.testing.assert_allclose(o["log_pmp"][inst], b["log_pmp"], rtol=1e-12)
        np.testing.assert_allclose(o["w_mu"][inst], b["w_mu"], rtol=1e-10, atol=1e-14)
        np.testing.assert_allclose(o["w_psi"][inst], b["w_psi"], rtol=1e-10, atol=1e-14)
        for e, we in b["w"].items():
            np.testing.assert_allclose(o["w"][e], we, rtol=1e-10, atol=1e-14)
            np.testing.assert_allclose(o["mom"][1][e], b["mom"][e], rtol=1e-10, atol=1e-13)


def test_split_root_one_sample_is_the_grouped_estimator():
    model = S.hier_logistic_batch(2, M=4, N=3, D=3, seed=31)
    q = S.random_q(model, seed=32, loc_scale=0.4, sd_lo=0.4, sd_hi=1.0)
    eps = S.noise(model, 1, seed=33)
    o = R.estep(model, q, 1, eps)
    g = O.estep(model, q, 1, eps=eps)
    np.testing.assert_allclose(o["log_pmp"], g["log_pmp"], rtol=1e-12)
    for l in range(2):
        np.testing.assert_allclose(o["mom"][l], g["mom"][l], rtol=1e-12, atol=1e-14)


def test_split_root_invariant_to_permuting_one_half():
    model = S.hier_logistic(M=6, N=4, D=3, seed=41)
    K, D = 8, 3
    q = S.random_q(model, seed=42, loc_scale=0.4, sd_lo=0.4, sd_hi=1.0)
    eps = S.noise(model, K, seed=43)
    perm = np.random.default_rng(44).permutation(K)
    eps_p = [e.copy() for e in eps]
    eps_p[0][:, :, D:] = eps[0][:, perm, D:]
    a, b = R.estep(model, q, K, eps), R.estep(model, q, K, eps_p)
    np.testing.assert_allclose(b["log_pmp"], a["log_pmp"], rtol=1e-13)
    np.testing.assert_allclose(b["w_mu"], a["w_mu"], rtol=1e-11, atol=1e-15)
    np.testing.assert_allclose(b["w_psi"][:, :], a["w_psi"][:, perm], rtol=1e-11, atol=1e-15)
    np.testing.assert_allclose(b["w"], a["w"], rtol=1e-11, atol=1e-15)
    np.testing.assert_allclose(b["mom"][0], a["mom"][0], rtol=1e-11, atol=1e-14)
    # the grouped estimator pairs the halves sample by sample, so it changes
    ga, gb = O.estep(model, q, K, eps=eps), O.estep(model, q, K, eps=eps_p)
    assert abs(ga["log_pmp"][0] - gb["log_pmp"][0]) > 1e-6


def test_split_root_weights_sum_to_one():
    model = S.hier_logistic_batch(3, M=5, N=4, D=4, seed=51)
    K = 16
    q = S.random_q(model, seed=52)
    o = R.estep(model, q, K, S.noise(model, K, seed=53))
    np.testing.assert_allclose(o["w_mu"].sum(1), 1.0, rtol=1e-12)
    np.testing.assert_allclose(o["w_psi"].sum(1), 1.0, rtol=1e-12)
    np.testing.assert_allclose(o["w"].sum(1), 1.0, rtol=1e-12)
    assert np.all(np.isfinite(o["logL"]))


def test_split_root_estimator_is_unbiased():
    """E[P_MP] = p(x) (Sec. 3.2) for the split estimator.  Users with Gaussian
    observations, D = 1, x = 1: given psi the data are Gaussian with covariance
    1 (mu) + e^psi (user) + v I (noise), so p(x) = E_psi N(x; 0, Sigma(psi)),
    one Gauss-Hermite quadrature over psi ~ N(0, 1)."""
    import math
    from scipy import stats
    model = S.hier_logistic(M=2, N=3, D=1, seed=61)
    u = model.levels[1]
    v = 0.5
    rng = np.random.default_rng(62)
    u.lik, u.lik_var = S.LIK_GAUSS, v
    u.x = np.ones_like(u.x)
    u.y = (0.7 + rng.standard_normal(u.y.shape)).astype(np.float32)
    y = u.y.astype(np.float64).reshape(-1)
    M, N = u.y.shape
    blk = np.kron(np.eye(M), np.ones((N, N)))

    def lpx_given(psi):
        return stats.multivariate_normal(np.zeros(M * N), np.ones((M * N, M * N)) + math.exp(psi) * blk
                                         + v * np.eye(M * N)).logpdf(y)

    xs, ws = np.polynomial.hermite_e.hermegauss(60)            # nodes for the weight exp(-x^2 / 2)
    lpx = np.log(np.sum(ws / math.sqrt(2 * math.pi) * np.exp([lpx_given(t) for t in xs])))
    q = S.random_q(model, seed=63, loc_scale=0.0, sd_lo=0.8, sd_hi=0.8)
    q[0][0, 0, 0] = 0.7                                           # mu near the data mean
    K, reps = 8, 400
    ratios = np.array([math.exp(R.estep(model, q, K, S.noise(model, K, seed=900 + s))["log_pmp"][0] - lpx)
                       for s in range(reps)])
    se = ratios.std(ddof=1) / math.sqrt(reps)
    assert abs(ratios.mean() - 1.0) < 4 * se + 1e-3, (ratios.mean(), se)
    assert np.log(ratios).mean() < 0
