"""Pins of the FP64 oracle against things other than itself.

* brute force: literal enumeration of all K^n index vectors (oracle/brute.py,
  scipy densities) on tiny 2- and 3-level trees and on single-latent models;
* closed forms: conjugate Gaussian / Gamma-Poisson / Beta-Bernoulli marginal
  likelihoods and posteriors (textbook conjugacy, scipy for the Gaussians);
* invariants: weights sum to one, exact reparameterisation invariance
  (App. E), unbiasedness of P_MP (Sec. 3.2), EMA closed form (App. D);
* special cases: a single latent is global importance weighting (App. A.1);
* library routines: digamma / trigamma against scipy; M-step round trips;
* published known-answer vectors for the counter-based generator.
"""
import math
import os

import numpy as np
import pytest
from scipy import special, stats

from oracle import brute
from oracle import oracle as O
from paper_2503_08264_gb300 import synth as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _tiny_models():
    yield "conj_gauss", S.conjugate_gaussian(M=3, N=4, seed=1), 4
    yield "hier_logistic", S.hier_logistic(M=3, N=3, D=2, seed=2), 4
    yield "three_level", S.batched_three_level(n_inst=1, D=2, seed=3, groups=(2, 2), units=(1, 2)), 3
    yield "gamma_poisson", S.gamma_poisson(n_inst=3, N=5, seed=4), 6
    yield "beta_bernoulli", S.beta_bernoulli(n_inst=3, N=5, seed=5), 6


@pytest.mark.parametrize("name,model,K", list(_tiny_models()), ids=lambda v: v if isinstance(v, str) else "")
def test_recursion_matches_enumeration(name, model, K):
    q = S.random_q(model, seed=11) if model.levels[0].qfam == S.Q_GAUSS else S.initial_q(model)
    eps = S.noise(model, K, seed=12)
    o = O.estep(model, q, K, eps=eps)
    for inst in range(model.n_inst):
        b = brute.estep_instance(model, q, o["z"], K, inst)
        assert abs(o["log_pmp"][inst] - b["log_pmp"]) <= 1e-11 * max(1.0, abs(b["log_pmp"]))
        for (l, e), wb in b["w"].items():
            np.testing.assert_allclose(o["w"][l][e], wb, rtol=1e-9, atol=1e-13)
            np.testing.assert_allclose(o["mom"][l][e], b["mom"][(l, e)], rtol=1e-9, atol=1e-12)


def test_three_level_two_instances_enumeration():
    model = S.batched_three_level(n_inst=2, D=1, seed=7, groups=(1, 2), units=(1, 2))
    K = 3
    q = S.random_q(model, seed=1)
    eps = S.noise(model, K, seed=2)
    o = O.estep(model, q, K, eps=eps)
    for inst in range(2):
        b = brute.estep_instance(model, q, o["z"], K, inst)
        assert abs(o["log_pmp"][inst] - b["log_pmp"]) <= 1e-11 * abs(b["log_pmp"])
        for (l, e), wb in b["w"].items():
            np.testing.assert_allclose(o["w"][l][e], wb, rtol=1e-9, atol=1e-13)


def test_samples_are_location_scale_of_noise():
    model = S.hier_logistic(M=4, N=2, D=3, seed=0)
    K = 5
    q = S.random_q(model, seed=3)
    eps = S.noise(model, K, seed=4)
    o = O.estep(model, q, K, eps=eps)
    for l in range(2):
        qq = q[l].astype(np.float64)
        ref = qq[:, None, 0, :] + qq[:, None, 1, :] * eps[l].astype(np.float64)
        np.testing.assert_array_equal(o["z"][l], ref)


def test_weights_sum_to_one_and_constant_moment():
    model = S.batched_three_level(n_inst=3, D=4, seed=8, groups=(2, 4), units=(2, 5))
    K = 16
    o = O.estep(model, S.random_q(model, seed=5), K, eps=S.noise(model, K, seed=6))
    for l in range(3):
        np.testing.assert_allclose(o["w"][l].sum(axis=1), 1.0, atol=1e-12)
        assert (o["w"][l] >= 0).all()


# --------------------------------------------------------------------------- closed forms
def _gauss_root_only(N=10, v=0.5, seed=0, n_inst=2):
    rng = np.random.default_rng(seed)
    mu = rng.standard_normal(n_inst)
    y = (mu[:, None] + math.sqrt(v) * rng.standard_normal((n_inst, N))).astype(np.float32)
    lv = S.Level(n=n_inst, dim=1, prior=S.PRIOR_STD_NORMAL, prior_a=1.0, lik=S.LIK_GAUSS,
                 lik_var=v, n_obs=N, x=np.ones((n_inst, N, 1), np.float32), y=y)
    return S.Model([lv])


def test_exact_posterior_proposal_gives_exact_evidence_gaussian():
    """q = exact posterior => r_k == p(x) for every draw (so log P_MP = log p(x))."""
    v, N = 0.5, 10
    model = _gauss_root_only(N=N, v=v)
    y = model.levels[0].y.astype(np.float64)
    prec = 1.0 + N / v
    mean = (y.sum(1) / v) / prec
    q = [np.stack([mean, np.full_like(mean, 1 / math.sqrt(prec))], 1)[:, :, None].astype(np.float64)]
    K = 64
    o = O.estep(model, q, K, eps=S.noise(model, K, seed=1))
    for i in range(model.n_inst):
        cov = np.ones((N, N)) + v * np.eye(N)
        lpx = stats.multivariate_normal(np.zeros(N), cov).logpdf(y[i])
        assert abs(o["log_pmp"][i] - lpx) < 1e-10 * abs(lpx)
        np.testing.assert_allclose(o["w"][0][i], 1.0 / K, rtol=1e-10)


def test_exact_posterior_proposal_gamma_poisson_and_beta_bernoulli():
    K = 32
    gp = S.gamma_poisson(n_inst=3, N=7, a0=2.0, b0=1.5, seed=3)
    y = gp.levels[0].y.astype(np.float64)
    a = 2.0 + y.sum(1)
    b = 1.5 + y.shape[1]
    q = [np.stack([a, np.full_like(a, b)], 1)[:, :, None]]
    o = O.estep(gp, q, K, eps=S.noise(gp, K, seed=4))
    lpy = (special.gammaln(a) - special.gammaln(2.0) + 2.0 * np.log(1.5) - a * np.log(b)
           - special.gammaln(y + 1).sum(1))
    np.testing.assert_allclose(o["log_pmp"], lpy, rtol=1e-11)
    np.testing.assert_allclose(o["w"][0], 1.0 / K, rtol=1e-9)

    bb = S.beta_bernoulli(n_inst=3, N=9, a0=2.0, b0=3.0, seed=5)
    y = bb.levels[0].y.astype(np.float64)
    a = 2.0 + y.sum(1)
    b = 3.0 + y.shape[1] - y.sum(1)
    q = [np.stack([a, b], 1)[:, :, None]]
    o = O.estep(bb, q, K, eps=S.noise(bb, K, seed=6))
    lpy = special.betaln(a, b) - special.betaln(2.0, 3.0)
    np.testing.assert_allclose(o["log_pmp"], lpy, rtol=1e-11)


def _conj_gauss_exact(model):
    """Linear-Gaussian conditioning for mu~N(0,1), z_m~N(mu,1), x_mn~N(z_m,v)."""
    lv = model.levels[1]
    M, N, v = lv.n, lv.n_obs, lv.lik_var
    x = lv.y.astype(np.float64).reshape(-1)
    P = np.zeros((M * N, M + 1))
    for m in range(M):
        P[m * N:(m + 1) * N, 1 + m] = 1.0
    C = np.ones((M + 1, M + 1))
    C[1:, 1:] += np.eye(M)                           # Cov(z_m, z_m') = 1 + delta
    Sx = P @ C @ P.T + v * np.eye(M * N)
    lpx = stats.multivariate_normal(np.zeros(M * N), Sx).logpdf(x)
    G = C @ P.T @ np.linalg.inv(Sx)
    mean = G @ x
    cov = C - G @ P @ C
    return lpx, mean, cov


def test_conjugate_gaussian_unbiased_evidence():
    """E[P_MP] = p(x) (Sec. 3.2): average of P_MP / p(x) over seeds is 1."""
    model = S.conjugate_gaussian(M=8, N=16, seed=0)
    lpx, mean, cov = _conj_gauss_exact(model)
    sd = np.sqrt(np.diag(cov))
    q = [np.array([[[mean[0]], [1.3 * sd[0]]]]),
         np.stack([mean[1:], 1.3 * sd[1:]], 1)[:, :, None]]
    K, R = 16, 300
    ratios = np.array([math.exp(O.estep(model, q, K, seed=s)["log_pmp"][0] - lpx) for s in range(R)])
    se = ratios.std(ddof=1) / math.sqrt(R)
    assert abs(ratios.mean() - 1.0) < 4 * se + 1e-3
    # Jensen: E log P_MP <= log p(x)
    assert np.log(ratios).mean() < 0


def test_conjugate_gaussian_moments_converge_with_K():
    """MPIW moments -> exact posterior moments as K grows (App. C)."""
    model = S.conjugate_gaussian(M=8, N=16, seed=1)
    _, mean, cov = _conj_gauss_exact(model)
    sd = np.sqrt(np.diag(cov))
    q = [np.array([[[0.0], [1.0]]]), np.stack([np.zeros(8), np.ones(8)], 1)[:, :, None]]
    errs = []
    for K in (64, 1024):
        o = O.estep(model, q, K, seed=3)
        m1 = np.concatenate([o["mom"][0][:, 0, 0], o["mom"][1][:, 0, 0]])
        errs.append(np.max(np.abs(m1 - mean) / sd))
    assert errs[1] < 0.5
    assert errs[1] < errs[0]


def test_reparameterisation_invariance():
    """App. E: scaling every latent by 1/alpha with matched model and q leaves
    the weights unchanged and maps the moments by (alpha m1, alpha^2 m2)."""
    alpha = 1.0 / 100.0
    model = S.conjugate_gaussian(M=5, N=6, seed=2)
    rep = S.conjugate_gaussian(M=5, N=6, seed=2)
    rep.levels[0].prior_a = 1.0 / alpha ** 2
    rep.levels[1].prior_a = 1.0 / alpha ** 2
    rep.levels[1].x = np.full(model.levels[1].x.shape, alpha, np.float64)
    K = 32
    q = [x.astype(np.float64) for x in S.random_q(model, seed=3)]
    qr = [x / alpha for x in q]
    eps = S.noise(model, K, seed=4)
    o = O.estep(model, q, K, eps=eps)
    r = O.estep(rep, qr, K, eps=eps)
    for l in range(2):
        np.testing.assert_allclose(r["w"][l], o["w"][l], rtol=1e-9, atol=1e-14)
        np.testing.assert_allclose(alpha * r["mom"][l][:, 0], o["mom"][l][:, 0], rtol=1e-9, atol=1e-13)
        np.testing.assert_allclose(alpha ** 2 * r["mom"][l][:, 1], o["mom"][l][:, 1], rtol=1e-9)
    # log P_MP is invariant too: the Jacobian alpha^n appears in P and in Q
    np.testing.assert_allclose(r["log_pmp"], o["log_pmp"], rtol=1e-10)


def test_single_latent_is_global_importance_weighting():
    """App. A.1: with n = 1, w = softmax(log r) and log P = logsumexp(log r) - log K."""
    model = _gauss_root_only(N=6, v=0.7, n_inst=1)
    K = 50
    q = [np.array([[[0.3], [0.8]]])]
    eps = S.noise(model, K, seed=9)
    o = O.estep(model, q, K, eps=eps)
    z = 0.3 + 0.8 * eps[0][0, :, 0].astype(np.float64)
    y = model.levels[0].y[0].astype(np.float64)
    logr = (stats.norm.logpdf(z, 0, 1) + stats.norm.logpdf(y[None, :], z[:, None], math.sqrt(0.7)).sum(1)
            - stats.norm.logpdf(z, 0.3, 0.8))
    np.testing.assert_allclose(o["w"][0][0], special.softmax(logr), rtol=1e-10)
    assert abs(o["log_pmp"][0] - (special.logsumexp(logr) - math.log(K))) < 1e-10


# --------------------------------------------------------------------------- M-step / EMA
def test_special_functions_against_scipy():
    xs = np.concatenate([np.linspace(0.01, 3, 40), np.linspace(3, 200, 40)])
    for x in xs:
        assert abs(O.digamma(x) - special.digamma(x)) < 1e-12 * max(1, abs(special.digamma(x)))
        assert abs(O.trigamma(x) - special.polygamma(1, x)) < 1e-12 * special.polygamma(1, x)
    assert abs(O.digamma(1.0) + np.euler_gamma) < 1e-15


def test_mstep_round_trips():
    mu = np.array([[-1.5, 0.0, 2.0]])
    sd = np.array([[0.1, 1.0, 3.0]])
    m = np.stack([mu, mu ** 2 + sd ** 2], 1)
    q = O.mstep(O.Q_GAUSS, m)
    np.testing.assert_allclose(q[:, 0], mu, rtol=1e-14)
    np.testing.assert_allclose(q[:, 1], sd, rtol=1e-12)
    a = np.array([[0.3, 1.0, 7.5, 120.0]])
    b = np.array([[2.0, 0.5, 1.0, 30.0]])
    m = np.stack([a / b, special.digamma(a) - np.log(b)], 1)
    q = O.mstep(O.Q_GAMMA, m)
    np.testing.assert_allclose(q[:, 0], a, rtol=1e-10)
    np.testing.assert_allclose(q[:, 1], b, rtol=1e-10)
    a = np.array([[0.5, 2.0, 40.0, 3.0]])
    b = np.array([[0.7, 5.0, 3.0, 300.0]])
    m = np.stack([special.digamma(a) - special.digamma(a + b), special.digamma(b) - special.digamma(a + b)], 1)
    q = O.mstep(O.Q_BETA, m)
    np.testing.assert_allclose(q[:, 0], a, rtol=1e-10)
    np.testing.assert_allclose(q[:, 1], b, rtol=1e-10)


@pytest.mark.timeout(60)
def test_mstep_outside_the_family_domain_gives_nan():
    """Statistics no Gamma or Beta has (Jensen: E log z < log E z, and
    e^{E log z} + e^{E log(1-z)} < 1) give NaN parameters, promptly; the
    special functions are NaN outside x > 0 (their recurrences would not end
    at x = -inf)."""
    for x in (0.0, -1.0, -np.inf, -1e300, np.nan):
        assert np.isnan(O.digamma(x)) and np.isnan(O.trigamma(x))
    la = np.log(0.6)
    m = np.array([[[la, la + 1e-3, la, np.nan, -0.9]], [[np.log(0.4) + 1e-12, np.log(0.4) - 1e-3, -np.inf, la, -0.7]]])
    m = np.moveaxis(m, 0, 1)                       # [n=1][2][D=5]
    q = O.mstep(O.Q_BETA, m)
    assert np.all(np.isnan(q[0, :, :4]))           # A + B >= 1, -inf, NaN
    assert np.all(np.isfinite(q[0, :, 4])) and np.all(q[0, :, 4] > 0)
    a, b = q[0, 0, 4], q[0, 1, 4]
    np.testing.assert_allclose([special.digamma(a) - special.digamma(a + b),
                                special.digamma(b) - special.digamma(a + b)], [-0.9, -0.7], rtol=1e-10)
    g = np.array([[[2.0, 2.0, -1.0], [np.log(2.0), np.log(2.0) + 0.1, 0.0]]])  # s = 0, s < 0, E z < 0
    qg = O.mstep(O.Q_GAMMA, g)
    assert np.all(np.isnan(qg))


def test_gauss_mstep_variance_floor():
    m = np.array([[[2.0], [4.0]]])   # var 0: the single-dominant-sample pathology (Sec. 4)
    q = O.mstep(O.Q_GAUSS, m, var_floor=1e-6)
    assert q[0, 1, 0] == pytest.approx(math.sqrt(1e-6 * 4.0))


def test_ema_closed_form():
    """With m_0 = 0 and a constant estimate c, m_t = (1 - (1-lambda)^t) c
    (App. D's geometric series, in Alg. 1's convention lambda = new weight)."""
    c = np.array([1.5, -2.0, 0.25])
    lam = 0.3
    m = np.zeros(3)
    for t in range(1, 25):
        m = O.ema(m, c, lam)
        np.testing.assert_allclose(m, (1 - (1 - lam) ** t) * c, rtol=1e-13)


# --------------------------------------------------------------------------- samplers and RNG
def test_philox_known_answers():
    with open(os.path.join(GOLD, "philox4x32_10_kat.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(t) for t in out] == v[6:10]


def test_counter_noise_is_standard_normal():
    e = O.draw_noise(seed=123, it=7, level=1, n=64, K=256, nps=6).reshape(-1)
    assert abs(e.mean()) < 0.02 and abs(e.var() - 1) < 0.03
    assert stats.kstest(e, "norm").pvalue > 1e-3
    e2 = O.draw_noise(seed=123, it=8, level=1, n=64, K=256, nps=6).reshape(-1)
    assert abs(np.corrcoef(e, e2)[0, 1]) < 0.02


def test_gamma_and_beta_samplers_ks():
    K = 4000
    gp = S.gamma_poisson(n_inst=2, N=3, seed=0)
    q = [np.array([[[0.6], [2.0]], [[4.5], [0.5]]])]
    o = O.estep(gp, q, K, eps=S.noise(gp, K, seed=1))
    for i, (a, b) in enumerate([(0.6, 2.0), (4.5, 0.5)]):
        assert stats.kstest(o["z"][0][i, :, 0], stats.gamma(a, scale=1 / b).cdf).pvalue > 1e-3
    bb = S.beta_bernoulli(n_inst=2, N=3, seed=0)
    q = [np.array([[[0.5], [0.8]], [[3.0], [7.0]]])]
    o = O.estep(bb, q, K, eps=S.noise(bb, K, seed=2))
    for i, (a, b) in enumerate([(0.5, 0.8), (3.0, 7.0)]):
        assert stats.kstest(o["z"][0][i, :, 0], stats.beta(a, b).cdf).pvalue > 1e-3


def test_instances_are_independent_and_subset_noise_matches():
    """Instances share nothing: the oracle on a sub-model of a few instances,
    with the counter-based noise those elements have in the full model, gives
    the full model's numbers for them (the basis of sampled parity at full
    size)."""
    K = 8
    full = S.batched_three_level(n_inst=7, D=3, seed=41, groups=(1, 3), units=(0, 4), n_obs=2)
    q = S.random_q(full, seed=42, loc_scale=0.3, sd_lo=0.4, sd_hi=0.9)
    ref = O.estep(full, q, K, seed=17, it=3)
    sub, keep = S.subset(full, [5, 2])
    assert [lv.n for lv in sub.levels] == [len(k) for k in keep]
    eps = [O.draw_noise_at(17, 3, l, keep[l], K, lv.noise_per_sample(), lv.qfam) for l, lv in enumerate(sub.levels)]
    got = O.estep(sub, [q[l][keep[l]] for l in range(3)], K, eps=eps)
    np.testing.assert_allclose(got["log_pmp"], ref["log_pmp"][keep[0]], rtol=1e-13)
    for l in range(3):
        np.testing.assert_allclose(got["mom"][l], ref["mom"][l][keep[l]], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(got["w"][l], ref["w"][l][keep[l]], rtol=1e-12, atol=1e-15)


def test_predictive_special_cases():
    """A weight vector on one sample gives that sample's log-likelihood; equal
    samples give it whatever the weights; Jensen's inequality against the
    weighted mean of the log-likelihoods."""
    rng = np.random.default_rng(61)
    n, K, D, N = 3, 7, 4, 5
    z = rng.standard_normal((n, K, D)) * 0.5
    x = rng.standard_normal((n, N, D))
    y = (rng.random((n, N)) < 0.4).astype(np.float64)
    one = np.zeros((n, K))
    one[:, 2] = 1.0
    s = np.einsum("ekd,end->ekn", z, x)
    ll = (y[:, None, :] * s - np.logaddexp(0.0, s)).sum(-1)      # Bernoulli-logit by hand
    np.testing.assert_allclose(O.predictive(z, one, 2, x, y), ll[:, 2], rtol=1e-12)
    same = np.repeat(z[:, :1], K, axis=1)
    w = rng.dirichlet(np.ones(K), size=n)
    np.testing.assert_allclose(O.predictive(same, w, 2, x, y), ll[:, 0] * 0 + (y * (x @ z[:, 0][..., None])[..., 0]
                               - np.logaddexp(0.0, (x @ z[:, 0][..., None])[..., 0])).sum(-1), rtol=1e-12)
    assert np.all(O.predictive(z, w, 2, x, y) >= (w * ll).sum(1) - 1e-12)
    yc = rng.poisson(2.0, (n, N)).astype(np.float64)
    lp = (yc[:, None, :] * s - np.exp(s) - np.vectorize(math.lgamma)(yc + 1.0)[:, None, :]).sum(-1)
    np.testing.assert_allclose(O.predictive(z, one, 3, x, yc), lp[:, 2], rtol=1e-12)
