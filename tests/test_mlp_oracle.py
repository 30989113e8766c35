"""Pins of the FP64 warm-start network reference (oracle/mlp.py), independent
of the CUDA path: central finite differences of the loss, the Gaussian KL
against numerical integration of its definition, BF16 rounding against the
library conversion, the first Adam step's closed form, a hand-wired network,
and the user features by explicit loops."""
import numpy as np
import pytest
from scipy import integrate, stats

from oracle import mlp as M


def _random_case(n=7, seed=0, scale=0.2):
    rng = np.random.default_rng(seed)
    theta = rng.standard_normal(M.n_params()) * scale
    f = rng.standard_normal((n, 37))
    m = rng.standard_normal((n, 18))
    s = rng.uniform(0.3, 1.5, (n, 18))
    return theta, f, m, s


def test_parameter_count():
    assert M.n_params() == 128 * 37 + 128 + 128 * 128 + 128 + 36 * 128 + 36 == 26020


def test_gradient_matches_central_differences():
    theta, f, m, s = _random_case()
    _, g = M.loss_grad(theta, f, m, s)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(M.n_params(), 60, replace=False),
                          [0, 128 * 37, 128 * 37 + 128, M.n_params() - 37, M.n_params() - 1]])
    h = 1e-4

    def at(i, d):
        t = theta.copy()
        t[i] += d
        return M.loss_grad(t, f, m, s)[0]

    for i in idx:  # fourth-order central difference
        fd = (-at(i, 2 * h) + 8 * at(i, h) - 8 * at(i, -h) + at(i, -2 * h)) / (12 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])


def test_kl_matches_numerical_integration():
    cases = [(0.0, 1.0, 1.0, np.log(2.0)), (0.3, 0.5, -0.2, np.log(0.7)), (-1.0, 2.0, 0.5, 0.0)]
    for m, s, mu, ls in cases:
        p, qd = stats.norm(m, s), stats.norm(mu, np.exp(ls))
        ref = integrate.quad(lambda z: p.pdf(z) * (p.logpdf(z) - qd.logpdf(z)), m - 12 * s, m + 12 * s,
                             epsabs=1e-13, epsrel=1e-12)[0]
        o = np.zeros((1, 36))
        o[0, 0], o[0, 18] = mu, ls
        mm, ss = np.zeros((1, 18)), np.ones((1, 18))
        mm[0, 0], ss[0, 0] = m, s
        # the other 17 dimensions are N(0,1) against N(0,1): zero
        assert abs(M.kl(o, mm, ss)[0] - ref) < 1e-9
    o = np.concatenate([np.full((1, 18), 0.4), np.log(np.full((1, 18), 0.9))], axis=1)
    assert abs(M.kl(o, np.full((1, 18), 0.4), np.full((1, 18), 0.9))[0]) < 1e-14


def test_bf16_rounding_matches_library_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    a = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-6, 6, 4000),
                        [1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -1.0 - 2.0 ** -8, 0.0, 65504.0]])
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.round_bf16(a), ref)
    assert M.round_bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0          # tie to even
    assert M.round_bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6


def test_first_adam_step_closed_form():
    rng = np.random.default_rng(4)
    theta = rng.standard_normal(50)
    g = rng.standard_normal(50)
    new, m, v = M.adam(theta, g, np.zeros(50), np.zeros(50), t=1, lr=1e-2, eps=1e-8)
    np.testing.assert_allclose(new, theta - 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_hand_wired_network():
    """Unit 0 of each layer copies feature 3 through both ReLUs; unit 18 of the
    output reads feature 36 negated plus 0.25; all else zero."""
    theta = np.zeros(M.n_params())
    (W1, b1), (W2, b2), (W3, b3) = M.unpack(theta)
    W1[0, 3] = 1.0
    W1[1, 36] = 1.0
    W2[0, 0] = 2.0
    W2[1, 1] = 1.0
    W3[0, 0] = 1.5
    W3[18, 1] = -1.0
    b3[18] = 0.25
    f = np.zeros((3, 37))
    f[:, 3] = [1.0, -2.0, 0.5]
    f[:, 36] = [4.0, 0.0, 1.0]
    o, _ = M.forward(theta, f)
    np.testing.assert_allclose(o[:, 0], 1.5 * 2.0 * np.maximum(f[:, 3], 0))
    np.testing.assert_allclose(o[:, 18], -f[:, 36] + 0.25)
    assert np.count_nonzero(o[:, 1:18]) == 0 and np.count_nonzero(o[:, 19:]) == 0


def test_features_by_loops():
    rng = np.random.default_rng(5)
    x = (rng.random((4, 5, 18)) < 0.3).astype(np.float32)
    y = (rng.random((4, 5)) < 0.5).astype(np.float32)
    f = M.features(x, y)
    for u in range(4):
        for d in range(18):
            assert f[u, d] == sum(x[u, n, d] * y[u, n] for n in range(5))
            assert f[u, 18 + d] == sum(x[u, n, d] for n in range(5))
        assert f[u, 36] == sum(y[u, n] for n in range(5))
