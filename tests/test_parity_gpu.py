"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, on the
same seeded inputs (shared supplied noise, or each side's own implementation
of the same counter-based stream).

Tolerances (relative, the definitions of the error targets):
  log P_MP   |d| <= tol * |log P_MP|
  moments    |d m1| <= tol * max(|m1|, sd_q),  |d m2| <= tol * max(|m2|, sd_q^2)
  weights    |d w| <= tol_w per sample (weights lie in [0, 1])
FP32 path: tol = 1e-5 for log P_MP, moments and weights (the FP32 target).
The path keeps every sample-independent constant in FP64 and centres each
element's FP32 factor on its maximum, so the FP32 work happens near zero for
the samples that carry weight; what remains is ~1e-7 rounding per log-factor.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2503_08264_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_08264_gb300 import build
    build.build()
    O.build()


def _plan(model, K, precision="fp32", **kw):
    from paper_2503_08264_gb300 import qem
    return qem.Plan(model, K, precision=precision, **kw)


def moment_errors(model, q, got, ref):
    out = []
    for l, lv in enumerate(model.levels):
        g, r = got[l].astype(np.float64), ref[l]
        if lv.qfam == S.Q_GAUSS:
            sd = np.asarray(q[l], np.float64)[:, 1, :]
            s1 = np.maximum(np.abs(r[:, 0]), sd)
            s2 = np.maximum(np.abs(r[:, 1]), sd ** 2)
        else:
            s1 = np.maximum(np.abs(r[:, 0]), 1.0)
            s2 = np.maximum(np.abs(r[:, 1]), 1.0)
        out.append(max(np.max(np.abs(g[:, 0] - r[:, 0]) / s1, initial=0.0),
                       np.max(np.abs(g[:, 1] - r[:, 1]) / s2, initial=0.0)))
    return out


def run_pair(model, K, q, eps=None, seed=0, it=0, precision="fp32", tuning=None):
    plan = _plan(model, K, precision)
    if tuning:
        plan.set_tuning(**tuning)
    qd = plan.flat(q)
    ed = plan.flat(eps) if eps is not None else None
    mom, _ = plan.estep(qd, ed, seed=seed, it=it)
    lp = plan.log_pmp()
    w = plan.split_w(plan.weights())
    z = plan.split_z(plan.samples())
    got = {"log_pmp": lp, "mom": plan.split_q(mom), "w": w, "z": z}
    plan.close()
    ref = O.estep(model, q, K, eps=eps, seed=seed, it=it)
    return got, ref


def assert_parity(model, q, got, ref, tol_lp, tol_m, tol_w):
    lp_err = np.max(np.abs(got["log_pmp"] - ref["log_pmp"]) / np.abs(ref["log_pmp"]))
    m_err = moment_errors(model, q, got["mom"], ref["mom"])
    w_err = [np.max(np.abs(got["w"][l] - ref["w"][l]), initial=0.0) for l in range(len(model.levels))]
    msg = f"log_pmp rel {lp_err:.2e}, moments {['%.2e' % e for e in m_err]}, weights {['%.2e' % e for e in w_err]}"
    print(msg)
    assert lp_err <= tol_lp, msg
    assert max(m_err) <= tol_m, msg
    assert max(w_err) <= tol_w, msg
    for l in range(len(model.levels)):
        if model.levels[l].n:
            np.testing.assert_allclose(got["w"][l].sum(1), 1.0, atol=1e-5)


def test_conjugate_gaussian_fp32():
    model = S.conjugate_gaussian(M=8, N=16, seed=0)
    K = 16
    q = S.initial_q(model)
    eps = S.noise(model, K, seed=1)
    got, ref = run_pair(model, K, q, eps)
    assert_parity(model, q, got, ref, 1e-5, 1e-5, 1e-5)


def test_hier_logistic_fp32_movielens_shape():
    model = S.hier_logistic(M=300, N=5, seed=0)
    K = 128
    q = S.random_q(model, seed=2)
    eps = S.noise(model, K, seed=3)
    got, ref = run_pair(model, K, q, eps)
    assert_parity(model, q, got, ref, 1e-5, 1e-5, 1e-5)


def test_hier_logistic_ragged_k_multiple_tiles():
    model = S.hier_logistic(M=37, N=4, seed=5)
    K = 200          # two row tiles of 128 and a ragged chunk tail
    q = S.random_q(model, seed=6)
    eps = S.noise(model, K, seed=7)
    got, ref = run_pair(model, K, q, eps)
    np.testing.assert_allclose(got["z"][1], ref["z"][1], rtol=1e-6, atol=1e-6)
    assert_parity(model, q, got, ref, 1e-5, 1e-5, 1e-5)


def test_three_level_ragged_plates_fp32():
    model = S.batched_three_level(n_inst=5, D=8, seed=3, groups=(0, 6), units=(0, 15))
    K = 96
    q = S.random_q(model, seed=4)
    eps = S.noise(model, K, seed=5)
    got, ref = run_pair(model, K, q, eps)
    assert_parity(model, q, got, ref, 1e-5, 1e-5, 1e-5)


def test_single_sample_k1():
    model = S.hier_logistic(M=9, N=3, D=4, seed=1)
    q = S.random_q(model, seed=2)
    eps = S.noise(model, 1, seed=3)
    got, ref = run_pair(model, 1, q, eps)
    assert_parity(model, q, got, ref, 1e-5, 1e-5, 1e-6)


def test_gamma_and_beta_root_models():
    for model, K in ((S.gamma_poisson(n_inst=6, N=9, seed=1), 64), (S.beta_bernoulli(n_inst=6, N=9, seed=2), 64)):
        q = S.initial_q(model)
        eps = S.noise(model, K, seed=3)
        got, ref = run_pair(model, K, q, eps)
        np.testing.assert_allclose(got["z"][0], ref["z"][0], rtol=1e-5)
        assert_parity(model, q, got, ref, 1e-5, 1e-5, 1e-5)


def test_counter_based_noise_matches_oracle_stream():
    model = S.hier_logistic(M=50, N=5, seed=9)
    K = 64
    q = S.random_q(model, seed=1)
    got, ref = run_pair(model, K, q, eps=None, seed=1234, it=17)
    np.testing.assert_allclose(got["z"][1], ref["z"][1], rtol=1e-5, atol=1e-5)
    assert_parity(model, q, got, ref, 1e-5, 1e-5, 1e-5)


def test_estep_is_deterministic():
    model = S.batched_three_level(n_inst=3, D=8, seed=1, groups=(2, 4), units=(3, 9))
    K = 64
    plan = _plan(model, K)
    qd = plan.flat(S.random_q(model, seed=1))
    a, la = plan.estep(qd, None, seed=5, it=1)
    a, la = a.clone(), la.clone()
    b, lb = plan.estep(qd, None, seed=5, it=1)
    assert torch.equal(a, b) and torch.equal(la, lb)
    plan.close()


def test_mstep_matches_oracle():
    rng = np.random.default_rng(0)
    # Gaussian: random moments including the variance-floor case
    model = S.hier_logistic(M=20, N=2, D=3, seed=0)
    plan = _plan(model, 8)
    qs = S.random_q(model, seed=3)
    mh = []
    for lv in model.levels:
        a = rng.standard_normal((lv.n, lv.dim))
        v = rng.uniform(0.0, 2.0, (lv.n, lv.dim))
        v[0, 0] = 0.0                      # floor case
        mh.append(np.stack([a, a * a + v], 1))
    mp = []
    for lv in model.levels:
        a = rng.standard_normal((lv.n, lv.dim))
        mp.append(np.stack([a, a * a + 1.0], 1))
    lam = 0.3
    mom_d = plan.flat(mh, torch.float64)
    m_d = plan.flat(mp, torch.float64)
    q_d = plan.flat(qs)
    plan.mstep(mom_d, m_d, q_d, lam)
    torch.cuda.synchronize()
    m_got = plan.split_q(m_d)
    q_got = plan.split_q(q_d)
    for l in range(2):
        m_ref = O.ema(mp[l], mh[l], lam)
        np.testing.assert_allclose(m_got[l], m_ref, rtol=1e-14, atol=1e-14)
        q_ref = O.mstep(O.Q_GAUSS, m_ref, var_floor=1e-10)
        np.testing.assert_allclose(q_got[l], q_ref, rtol=2e-7, atol=1e-30)
    plan.close()
    # Gamma and Beta M-steps (EMA + moment matching through digamma Newton)
    for model, fam in ((S.gamma_poisson(n_inst=5, N=2), O.Q_GAMMA), (S.beta_bernoulli(n_inst=5, N=2), O.Q_BETA)):
        plan = _plan(model, 8)
        a = rng.uniform(0.3, 30, (5, 1))
        b = rng.uniform(0.3, 30, (5, 1))
        from scipy import special
        if fam == O.Q_GAMMA:
            m = np.stack([a / b, special.digamma(a) - np.log(b)], 1)
        else:
            m = np.stack([special.digamma(a) - special.digamma(a + b), special.digamma(b) - special.digamma(a + b)], 1)
        m_d = plan.flat([m], torch.float64)
        q_d = plan.flat([np.ones((5, 2, 1))])
        plan.mstep(None, m_d, q_d, 1.0)
        torch.cuda.synchronize()
        q_ref = O.mstep(fam, m)
        np.testing.assert_allclose(plan.split_q(q_d)[0], q_ref, rtol=2e-7)
        np.testing.assert_allclose(plan.split_q(q_d)[0][:, 0], a, rtol=1e-6)
        plan.close()


def test_mstep_outside_the_family_domain_raises_numeric():
    """Beta statistics with e^{E log z} + e^{E log(1-z)} just above 1 (reachable
    through rounding when the weights collapse) have no solution: the M-step
    keeps that element's previous parameters, fits the others, and the next
    qem_log_pmp reports QEM_ERR_NUMERIC."""
    from scipy import special
    from paper_2503_08264_gb300 import _lib as L
    model = S.beta_bernoulli(n_inst=4, N=3, seed=1)
    plan = _plan(model, 8)
    q0 = [np.full((4, 2, 1), 2.0)]
    q_d = plan.flat(q0)
    plan.estep(q_d, None, seed=1, it=1)
    assert np.all(np.isfinite(plan.log_pmp()))
    a = np.array([[1.5], [3.0], [0.7], [9.0]])
    b = np.array([[2.5], [0.8], [4.0], [2.0]])
    m = np.stack([special.digamma(a) - special.digamma(a + b), special.digamma(b) - special.digamma(a + b)], 1)
    m[2, 0, 0] = np.log(0.5) + 1e-9
    m[2, 1, 0] = np.log(0.5) + 1e-9          # A + B = 1 + 2e-9
    m_d = plan.flat([m], torch.float64)
    plan.mstep(None, m_d, q_d, 1.0)
    torch.cuda.synchronize()
    got = plan.split_q(q_d)[0]
    np.testing.assert_array_equal(got[2], q0[0][2])
    keep = [0, 1, 3]
    np.testing.assert_allclose(got[keep, 0], a[keep], rtol=1e-6)
    np.testing.assert_allclose(got[keep, 1], b[keep], rtol=1e-6)
    with pytest.raises(L.QemError) as ei:
        plan.log_pmp()
    assert ei.value.code == L.QEM_ERR_NUMERIC
    plan.close()


def test_ema_schedule_theorem_1():
    """sched_p replaces lambda by t^-p (Thm. 1's schedule)."""
    model = S.gamma_poisson(n_inst=2, N=2)
    plan = _plan(model, 4)
    m = [np.array([[[1.0], [0.0]], [[2.0], [0.1]]])]
    mh = [np.array([[[3.0], [0.5]], [[1.0], [-0.4]]])]
    for t in (1, 2, 7):
        m_d = plan.flat(m, torch.float64)
        q_d = plan.flat([np.ones((2, 2, 1))])
        plan.mstep(plan.flat(mh, torch.float64), m_d, q_d, 0.0, sched_p=0.6, t=t)
        torch.cuda.synchronize()
        lam = t ** -0.6
        np.testing.assert_allclose(plan.split_q(m_d)[0], (1 - lam) * m[0] + lam * mh[0], rtol=1e-14)
    plan.close()


def test_qem_run_matches_oracle_loop():
    """Alg. 1 for T iterations on the device (graph-replayed) against the oracle
    loop with each side's own draw of the same counter-based noise."""
    model = S.conjugate_gaussian(M=8, N=16, seed=0)
    K, T, lam, seed = 16, 20, 0.5, 99
    plan = _plan(model, K)
    q0 = S.initial_q(model)
    m0 = [np.stack([q[:, 0], q[:, 0] ** 2 + q[:, 1] ** 2], 1).astype(np.float64) for q in q0]
    m_d = plan.flat(m0, torch.float64)
    q_d = plan.flat(q0)
    trace = torch.empty(T * plan.n_inst, dtype=torch.float64, device="cuda")
    plan.run(T, lam, m_d, q_d, seed=seed, trace=trace)
    torch.cuda.synchronize()
    m_ref = [x.copy() for x in m0]
    q_ref = [O.mstep(O.Q_GAUSS, x) for x in m_ref]
    lps = []
    for t in range(1, T + 1):
        r = O.estep(model, q_ref, K, seed=seed, it=t)
        lps.append(r["log_pmp"][0])
        m_ref = [O.ema(m_ref[l], r["mom"][l], lam) for l in range(2)]
        q_ref = [O.mstep(O.Q_GAUSS, x) for x in m_ref]
    got_m = plan.split_q(m_d)
    for l in range(2):
        np.testing.assert_allclose(got_m[l], m_ref[l], rtol=5e-4, atol=5e-4)
    np.testing.assert_allclose(trace.cpu().numpy(), np.array(lps), rtol=1e-4)
    plan.close()


def test_non_finite_proposal_reports_numeric_error():
    from paper_2503_08264_gb300 import _lib as L
    model = S.hier_logistic(M=4, N=2, D=2, seed=0)
    plan = _plan(model, 16)
    q = S.random_q(model, seed=0)
    q[0][0, 0, 0] = np.nan
    plan.estep(plan.flat(q), None)
    with pytest.raises(L.QemError) as ei:
        plan.log_pmp()
    assert ei.value.code == L.QEM_ERR_NUMERIC
    plan.close()
