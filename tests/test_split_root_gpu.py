"""GPU parity of the split-root E-step (qem_estep_split_root): the global mean
and log-variance of the hierarchical model as separate latents with their
own sample indices (K^2 parent index pairs per user), against the FP64
split-root oracle on the same noise.

Tolerances as the FP32 parity tests (test_parity_gpu.py): 1e-5 relative for
log P_MP and the moments, 1e-5 absolute for the weights.  Cases span several
row tiles of the K^2-row forward and a ragged tail (K^2 not a multiple of
the 128-row block), several instances of uneven size, Poisson-log users, the
in-kernel counter-based noise, the MovieLens shape at K = 128, and a short
EM loop through the M-step.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from oracle import split_root as R
from paper_2503_08264_gb300 import synth as S

from test_parity_gpu import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_08264_gb300 import build
    build.build()
    O.build()


def _poisson_users(model, seed):
    u = model.levels[1]
    rng = np.random.default_rng(seed)
    u.x = (0.4 * rng.standard_normal(u.x.shape)).astype(np.float32)
    u.y = rng.poisson(1.5, size=u.y.shape).astype(np.float32)
    u.lik = S.LIK_POISSON_LOG
    return model


def _run(model, K, q, eps, seed=0, it=0, precision="fp32"):
    from paper_2503_08264_gb300 import qem
    plan = qem.Plan(model, K, precision=precision)
    qd = plan.flat(q)
    ed = plan.flat(eps) if eps is not None else None
    mom, lp_dev, rw = plan.estep_split_root(qd, ed, seed=seed, it=it)
    torch.cuda.synchronize()
    lp = plan.log_pmp()
    w = plan.split_w(plan.weights())
    got = {"log_pmp": lp, "mom": plan.split_q(mom), "w": w, "rw": rw.cpu().numpy(),
           "lp_dev": lp_dev.cpu().numpy()}
    plan.close()
    return got


def _check(model, q, got, ref, tol=1e-5):
    np.testing.assert_array_equal(got["lp_dev"], got["log_pmp"])
    assert_parity(model, q, got, {"log_pmp": ref["log_pmp"], "mom": ref["mom"], "w": [ref["w_mu"], ref["w"]]},
                  tol, tol, tol)
    np.testing.assert_allclose(got["rw"][:, 0], ref["w_mu"], atol=tol, rtol=0)
    np.testing.assert_allclose(got["rw"][:, 1], ref["w_psi"], atol=tol, rtol=0)
    np.testing.assert_allclose(got["rw"].sum(2), 1.0, atol=1e-5)


@pytest.mark.parametrize("K", [16, 50, 96])
def test_split_root_matches_oracle(K):
    model = S.hier_logistic(M=40, N=5, seed=81)
    q = S.random_q(model, seed=82)
    eps = S.noise(model, K, seed=83)
    _check(model, q, _run(model, K, q, eps), R.estep(model, q, K, eps))


def test_split_root_uneven_instances_poisson_users():
    model = S.hier_logistic_batch(3, M=12, N=4, D=6, seed=84)
    keep = np.nonzero(model.levels[1].parent != 1)[0][:-5]    # instance sizes 12, 0, 7
    u = model.levels[1]
    for f in ("parent", "x", "y"):
        setattr(u, f, getattr(u, f)[keep])
    u.n = len(keep)
    model = _poisson_users(model, 85)
    K = 40
    q = S.random_q(model, seed=86, loc_scale=0.3, sd_lo=0.3, sd_hi=0.8)
    eps = S.noise(model, K, seed=87)
    _check(model, q, _run(model, K, q, eps), R.estep(model, q, K, eps))


def test_split_root_counter_based_noise():
    model = S.hier_logistic(M=25, N=5, seed=88)
    K, seed, it = 64, 1234, 3
    q = S.random_q(model, seed=89)
    eps = [O.draw_noise(seed, it, l, lv.n, K, lv.noise_per_sample()) for l, lv in enumerate(model.levels)]
    _check(model, q, _run(model, K, q, None, seed=seed, it=it), R.estep(model, q, K, eps))


def test_split_root_movielens_shape_k128():
    model = S.hier_logistic(M=300, N=5, seed=90)
    K = 128
    q = S.random_q(model, seed=91)
    eps = S.noise(model, K, seed=92)
    _check(model, q, _run(model, K, q, eps), R.estep(model, q, K, eps))


def test_split_root_plan_precision_does_not_matter():
    model = S.hier_logistic(M=10, N=5, seed=93)
    K = 128
    q = S.random_q(model, seed=94)
    eps = S.noise(model, K, seed=95)
    a = _run(model, K, q, eps, precision="fp32")
    b = _run(model, K, q, eps, precision="bf16x3")
    np.testing.assert_array_equal(a["log_pmp"], b["log_pmp"])
    for l in range(2):
        np.testing.assert_array_equal(a["mom"][l], b["mom"][l])


def test_split_root_em_loop_matches_oracle():
    """Three iterations of Alg. 1 with the split-root E-step, EMA + M-step on the GPU."""
    from paper_2503_08264_gb300 import qem
    model = S.hier_logistic(M=20, N=5, D=6, seed=96)
    K, T, lam = 24, 3, 0.5
    plan = qem.Plan(model, K, precision="fp32")
    q0 = S.initial_q(model)
    qd = plan.flat(q0)
    m = plan.mean_params(qd)
    qd_next = torch.empty_like(qd)
    plan.mstep(None, m, qd_next, lam, t=1)
    qd = qd_next
    m_ref = [np.stack([q[:, 0], q[:, 0] ** 2 + q[:, 1] ** 2], 1) for q in (np.asarray(x, np.float64) for x in q0)]
    q_ref = [O.mstep(S.Q_GAUSS, mm) for mm in m_ref]
    for t in range(1, T + 1):
        eps = S.noise(model, K, seed=100 + t)
        mom, _, _ = plan.estep_split_root(qd, plan.flat(eps))
        plan.mstep(mom, m, qd, lam, t=t)
        ref = R.estep(model, q_ref, K, eps)
        m_ref = [O.ema(m_ref[l], ref["mom"][l], lam) for l in range(2)]
        q_ref = [O.mstep(S.Q_GAUSS, m_ref[l]) for l in range(2)]
    torch.cuda.synchronize()
    got = plan.split_q(qd)
    for l in range(2):
        np.testing.assert_allclose(got[l], q_ref[l], rtol=1e-4, atol=1e-4)
    plan.close()


def test_split_root_rejects_unsupported_models():
    from paper_2503_08264_gb300 import _lib as L
    from paper_2503_08264_gb300 import qem
    model = S.batched_three_level(n_inst=2, D=4, seed=97, groups=(2, 3), units=(2, 3))
    plan = qem.Plan(model, 8, precision="fp32")
    q = plan.flat(S.random_q(model, seed=98))
    with pytest.raises(L.QemError) as e:
        plan.estep_split_root(q)
    assert e.value.code == L.QEM_ERR_UNSUPPORTED
    plan.close()
