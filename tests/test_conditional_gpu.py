"""GPU parity of the parent-conditioned proposal (qcond: App. A.2's
non-factorised Q_MP with the permutation copy scheme) against the FP64
oracle (oracle/conditional.py) on the same noise and permutations.

Tolerances as the FP32 parity tests: 1e-5 relative for log P_MP and the
moments (the children's moments are the residual's (E d, E d^2)), 1e-5
absolute for the weights.  Cases: the MovieLens-shaped model (mean/log-
variance prior, D = 18) and the conjugate Gaussian hierarchy with a ragged
K, supplied permutations; the counter-based permutations against the
oracle's own generator; the single-launch EM loop against the host loop.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import conditional as QC
from oracle import oracle as O
from paper_2503_08264_gb300 import synth as S

from test_parity_gpu import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_08264_gb300 import build
    build.build()
    O.build()


def _perms(n, K, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.permutation(K) for _ in range(n)]).astype(np.int32)


def _run(model, K, q, eps, perm, seed=0, it=0):
    from paper_2503_08264_gb300 import qem
    plan = qem.Plan(model, K, precision="fp32")
    plan.set_perm(perm)
    qd = plan.flat(q)
    ed = plan.flat(eps) if eps is not None else None
    mom, _ = plan.estep(qd, ed, seed=seed, it=it)
    torch.cuda.synchronize()
    got = {"log_pmp": plan.log_pmp(), "mom": plan.split_q(mom), "w": plan.split_w(plan.weights())}
    plan.close()
    return got


def _cond(model):
    model.levels[1].qcond = 1
    return model


@pytest.mark.parametrize("name,model,K", [
    ("logistic_M40_K64", _cond(S.hier_logistic(M=40, N=5, seed=121)), 64),
    ("conj_gauss_M8_K100", _cond(S.conjugate_gaussian(M=8, N=16, seed=122)), 100),
    ("logistic_batch3_M10_K32", _cond(S.hier_logistic_batch(3, M=10, N=4, D=6, seed=123)), 32),
], ids=lambda v: v if isinstance(v, str) else "")
def test_conditional_supplied_permutations_match_oracle(name, model, K):
    q = S.random_q(model, seed=124, loc_scale=0.2, sd_lo=0.3, sd_hi=0.8)
    eps = S.noise(model, K, seed=125)
    perm = _perms(model.levels[1].n, K, 126)
    assert_parity(model, q, _run(model, K, q, eps, perm), QC.estep(model, q, K, eps, perm), 1e-5, 1e-5, 1e-5)


def test_conditional_counter_based_permutations_match_oracle_generator():
    model = _cond(S.hier_logistic(M=30, N=5, D=8, seed=127))
    K, seed, it = 48, 4321, 5
    q = S.random_q(model, seed=128, loc_scale=0.2, sd_lo=0.3, sd_hi=0.8)
    eps = S.noise(model, K, seed=129)
    perm = QC.draw_perm(seed, it, model.levels[1].n, K)
    assert_parity(model, q, _run(model, K, q, eps, None, seed=seed, it=it), QC.estep(model, q, K, eps, perm),
                  1e-5, 1e-5, 1e-5)


def test_conditional_single_launch_loop_matches_host_loop():
    from paper_2503_08264_gb300 import qem
    model = _cond(S.hier_logistic_batch(2, M=12, N=5, D=6, seed=130))
    K, T_it, lam, seed = 64, 4, 0.5, 11
    plan = qem.Plan(model, K, precision="fp32")
    q0 = plan.flat(S.initial_q(model))
    m0 = plan.mean_params(q0)
    m_h, q_h = m0.clone(), torch.empty_like(q0)
    plan.mstep(None, m_h, q_h, lam, t=1)
    mom = torch.empty(plan.q_len, dtype=torch.float64, device="cuda")
    for t in range(1, T_it + 1):
        plan.estep(q_h, None, seed=seed, it=t, moments=mom)
        plan.mstep(mom, m_h, q_h, lam, t=t)
    m_r, q_r = m0.clone(), torch.empty_like(q0)
    plan.run(T_it, lam, m_r, q_r, seed=seed)
    torch.cuda.synchronize()
    assert torch.equal(m_r, m_h) and torch.equal(q_r, q_h)
    assert np.all(np.isfinite(plan.log_pmp()))
    plan.close()


def test_conditional_rejects_unsupported_plans():
    from paper_2503_08264_gb300 import _lib as L
    from paper_2503_08264_gb300 import qem
    model = _cond(S.hier_logistic(M=4, N=3, D=4, seed=131))
    with pytest.raises(L.QemError) as e:
        qem.Plan(model, 128, precision="bf16x3")
    assert e.value.code == L.QEM_ERR_UNSUPPORTED
    plain = qem.Plan(S.hier_logistic(M=4, N=3, D=4, seed=131), 16, precision="fp32")
    with pytest.raises(L.QemError) as e:
        plain.set_perm(np.zeros((4, 16), np.int32))
    assert e.value.code == L.QEM_ERR_INVALID_ARG
    plain.close()
