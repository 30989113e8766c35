"""Pins of the parent-conditioned proposal oracle (oracle/conditional.py):
children drawn from N(z_p^{s(k)} + loc, scale^2), parent copy s(k) chosen by a
uniformly random permutation (App. A.2's copy scheme), residual moments for
the M-step.

* brute force: literal enumeration of every index vector with scipy
  densities, the proposal term of each child copy taken at the parent copy it
  was drawn from; log P_MP, weights, moments and the pairwise moment
  E[z_i z_p] (1e-12);
* unbiasedness: on the conjugate Gaussian hierarchy the average of
  P_MP / p(x) over independent draws (noise and permutations) is 1 within
  its Monte Carlo error, p(x) in closed form; the same estimator with the
  proposal term taken at the combination's parent copy instead has a mean
  log ratio significantly above 0, which no unbiased estimator can have
  (Jensen), so the pin tells the two readings of Eq. rmp apart;
* residual moments: E d = E z_i - E z_p and E d^2 = E z_i^2 - 2 E[z_i z_p] +
  E z_p^2 equal the moments of d = z_i - z_p under the enumerated joint weights,
  and approach the exact posterior of d on the conjugate hierarchy as K grows;
* the counter-based permutations are permutations, uniform, and change with
  the iteration.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import brute
from oracle import conditional as QC
from paper_2503_08264_gb300 import synth as S


def _perms(model, K, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.permutation(K) for _ in range(model.levels[1].n)])


def _cases():
    yield "conj_gauss_M2_K3", S.conjugate_gaussian(M=2, N=3, seed=1), 3
    yield "conj_gauss_M3_K3", S.conjugate_gaussian(M=3, N=2, seed=2), 3
    yield "logistic_M2_K4", S.hier_logistic(M=2, N=3, D=2, seed=3), 4
    yield "logistic_batch2_M2_K3", S.hier_logistic_batch(2, M=2, N=3, D=2, seed=4), 3


@pytest.mark.parametrize("name,model,K", list(_cases()), ids=lambda v: v if isinstance(v, str) else "")
def test_conditional_matches_enumeration(name, model, K):
    q = S.random_q(model, seed=11, loc_scale=0.3, sd_lo=0.4, sd_hi=1.0)
    eps = S.noise(model, K, seed=12)
    perm = _perms(model, K, 13)
    o = QC.estep(model, q, K, eps, perm)
    D = model.levels[1].dim
    for inst in range(model.n_inst):
        b = brute.estep_instance_conditional(model, q, o["z"], perm, K, inst)
        np.testing.assert_allclose(o["log_pmp"][inst], b["log_pmp"], rtol=1e-12)
        for (l, e), we in b["w"].items():
            np.testing.assert_allclose(o["w"][l][e], we, rtol=1e-10, atol=1e-14)
            ref = b["mom"][(l, e)]
            got = o["mom"][0][e] if l == 0 else o["zmom1"][e]
            np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-13)
            if l == 1:
                np.testing.assert_allclose(o["cross"][e], b["cross"][e], rtol=1e-10, atol=1e-13)
                # residual moments from the enumerated pieces
                p = model.levels[1].parent[e]
                pm = b["mom"][(0, p)][:, :D]
                d1 = ref[0] - pm[0]
                d2 = ref[1] - 2 * b["cross"][e] + pm[1]
                np.testing.assert_allclose(o["mom"][1][e], np.stack([d1, d2]), rtol=1e-10, atol=1e-12)


def _conj_exact(model):
    """log p(x) and the posterior of (mu, z) for mu~N(0,1), z_m~N(mu,1), x_mn~N(z_m,v)."""
    lv = model.levels[1]
    M, N, v = lv.n, lv.n_obs, lv.lik_var
    x = lv.y.astype(np.float64).reshape(-1)
    P = np.zeros((M * N, M + 1))
    for m in range(M):
        P[m * N:(m + 1) * N, 1 + m] = 1.0
    C = np.ones((M + 1, M + 1))
    C[1:, 1:] += np.eye(M)
    Sx = P @ C @ P.T + v * np.eye(M * N)
    lpx = stats.multivariate_normal(np.zeros(M * N), Sx).logpdf(x)
    G = C @ P.T @ np.linalg.inv(Sx)
    return lpx, G @ x, C - G @ P @ C


def test_conditional_proposal_is_unbiased_and_the_other_reading_is_not():
    model = S.conjugate_gaussian(M=4, N=8, seed=5)
    lpx, mean, cov = _conj_exact(model)
    M = model.levels[1].n
    # residual d_m = z_m - mu under the posterior
    d_mean = mean[1:] - mean[0]
    d_sd = np.sqrt(np.diag(cov)[1:] + cov[0, 0] - 2 * cov[0, 1:])
    q = [np.array([[[mean[0]], [1.2 * math.sqrt(cov[0, 0])]]]),
         np.stack([d_mean, 1.2 * d_sd], 1)[:, :, None]]
    K, R = 8, 400
    good, other = [], []
    for s in range(R):
        eps = S.noise(model, K, seed=1000 + s)
        perm = _perms(model, K, 5000 + s)
        good.append(math.exp(QC.estep(model, q, K, eps, perm)["log_pmp"][0] - lpx))
        # the other reading: the proposal term at the combination's parent copy,
        # enumerated over (k_mu, k_1..k_M) by the factorisation over users
        z0, z1, _ = QC.samples(model, q, K, eps, perm)
        u = model.levels[1]
        f0 = (stats.norm.logpdf(z0[0, :, 0], 0, 1) - stats.norm.logpdf(z0[0, :, 0], q[0][0, 0, 0], q[0][0, 1, 0]))
        A = f0.copy()
        for e in range(M):
            lik = stats.norm.logpdf(u.y[e][None, :], z1[e][:, 0][:, None], math.sqrt(u.lik_var)).sum(1)
            pr = stats.norm.logpdf(z1[e][None, :, 0], z0[0][:, None, 0], 1.0)
            qq = stats.norm.logpdf(z1[e][None, :, 0], z0[0][:, None, 0] + q[1][e, 0, 0], q[1][e, 1, 0])
            Se = pr + lik[None, :] - qq
            A = A + np.log(np.exp(Se).mean(1))
        other.append(np.exp(A).mean() / math.exp(lpx))
    good, other = np.array(good), np.array(other)
    se = good.std(ddof=1) / math.sqrt(R)
    assert abs(good.mean() - 1.0) < 4 * se + 1e-3, (good.mean(), se)
    assert np.log(good).mean() < 0                      # Jensen: E log P_MP <= log p(x)
    # the other reading has no finite variance (the proposal term of a copy at a
    # parent copy it was not drawn from can vanish), so test it through Jensen:
    # an unbiased positive estimator has E log(ratio) <= 0
    lo = np.log(other)
    assert lo.mean() > 4 * lo.std(ddof=1) / math.sqrt(R), (lo.mean(), lo.std())


def test_conditional_weights_sum_to_one():
    model = S.hier_logistic_batch(2, M=6, N=4, D=3, seed=21)
    K = 16
    o = QC.estep(model, S.random_q(model, seed=22), K, S.noise(model, K, seed=23), _perms(model, K, 24))
    for l in range(2):
        np.testing.assert_allclose(o["w"][l].sum(1), 1.0, rtol=1e-12)


def test_counter_based_permutations_are_uniform_permutations():
    n, K = 2000, 8
    perm = QC.draw_perm(seed=77, it=3, n=n, K=K)
    assert np.all(np.sort(perm, axis=1) == np.arange(K))            # every row is a permutation
    # the parent copy of child copy 0 is uniform over the K copies (chi-square, 7 dof, 0.1% level)
    counts = np.bincount(perm[:, 0], minlength=K)
    chi2 = ((counts - n / K) ** 2 / (n / K)).sum()
    assert chi2 < 24.3, counts
    # different iterations and elements give different permutations
    other = QC.draw_perm(seed=77, it=4, n=n, K=K)
    assert np.mean(np.all(other == perm, axis=1)) < 0.01


def test_conditional_residual_moments_approach_exact_posterior():
    """On the conjugate hierarchy the residual d_m = z_m - mu has an exact
    Gaussian posterior (mean and variance from Gaussian conditioning); the
    residual moments the M-step consumes approach them as K grows (App. C)."""
    model = S.conjugate_gaussian(M=6, N=8, seed=31)
    model.levels[1].qcond = 1
    _, mean, cov = _conj_exact(model)
    d_mean = mean[1:] - mean[0]
    d_var = np.diag(cov)[1:] + cov[0, 0] - 2 * cov[0, 1:]
    q = [np.array([[[0.0], [1.0]]]), np.stack([np.zeros(6), np.ones(6)], 1)[:, :, None]]
    errs = []
    for K in (32, 1024):
        o = QC.estep(model, q, K, S.noise(model, K, seed=32), _perms(model, K, 33))
        m1, m2 = o["mom"][1][:, 0, 0], o["mom"][1][:, 1, 0]
        v = m2 - m1 ** 2
        errs.append(max(np.max(np.abs(m1 - d_mean) / np.sqrt(d_var)), np.max(np.abs(v / d_var - 1.0))))
    assert errs[1] < 0.3 and errs[1] < errs[0], errs
