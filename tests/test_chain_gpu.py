"""GPU parity of chain plates (the daily random walk per region of the Covid
model's timeseries, every (region, day) its own latent) against the FP64
chain oracle on the same noise.

Tolerances as the FP32 parity tests: 1e-5 relative for log P_MP and the
moments, 1e-5 absolute for the weights.  Cases: Poisson-log days with
one-dimensional latents, Gaussian days with three-dimensional latents and a
ragged K, several instances, the in-kernel counter-based noise, the Covid
shape (92 regions x 109 days, K = 128), and the single-launch EM loop
(qem_run) against the host loop.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import chain as C
from oracle import oracle as O
from paper_2503_08264_gb300 import synth as S

from test_parity_gpu import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_08264_gb300 import build
    build.build()
    O.build()


def _run(model, K, q, eps, seed=0, it=0):
    from paper_2503_08264_gb300 import qem
    plan = qem.Plan(model, K, precision="fp32")
    qd = plan.flat(q)
    ed = plan.flat(eps) if eps is not None else None
    mom, _ = plan.estep(qd, ed, seed=seed, it=it)
    torch.cuda.synchronize()
    got = {"log_pmp": plan.log_pmp(), "mom": plan.split_q(mom), "w": plan.split_w(plan.weights())}
    plan.close()
    return got


@pytest.mark.parametrize("R,T,K", [(4, 7, 64), (3, 12, 32), (1, 2, 128)])
def test_chain_poisson_matches_oracle(R, T, K):
    model = S.chain_poisson(n_inst=1, R=R, T=T, D=1, seed=101 + T)
    q = S.random_q(model, seed=102, loc_scale=0.3, sd_lo=0.2, sd_hi=0.6)
    eps = S.noise(model, K, seed=103)
    assert_parity(model, q, _run(model, K, q, eps), C.estep(model, q, K, eps), 1e-5, 1e-5, 1e-5)


def test_chain_gaussian_three_dims_ragged_k_two_instances():
    model = S.chain_poisson(n_inst=2, R=3, T=5, D=3, seed=104, lik=S.LIK_GAUSS, n_obs=2)
    K = 100
    q = S.random_q(model, seed=105, loc_scale=0.3, sd_lo=0.3, sd_hi=0.8)
    eps = S.noise(model, K, seed=106)
    assert_parity(model, q, _run(model, K, q, eps), C.estep(model, q, K, eps), 1e-5, 1e-5, 1e-5)


def test_chain_counter_based_noise():
    model = S.chain_poisson(n_inst=1, R=5, T=9, D=1, seed=107)
    K, seed, it = 64, 99, 2
    q = S.random_q(model, seed=108, loc_scale=0.3, sd_lo=0.2, sd_hi=0.6)
    eps = [O.draw_noise(seed, it, l, lv.n, K, lv.noise_per_sample()) for l, lv in enumerate(model.levels)]
    assert_parity(model, q, _run(model, K, q, None, seed=seed, it=it), C.estep(model, q, K, eps),
                  1e-5, 1e-5, 1e-5)


def test_chain_covid_shape_k128():
    """Daily counts here reach ~2.5e3, so the Poisson-log factor multiplies
    any rounding of s - s0 by y: the sampler forms s - s0 from the element's
    FP64 centre loc.x - s0 plus the scaled noise (never through the rounded
    sample z) and the factor as (y - e^s0)(s - s0) - e^s0 (e^(s-s0) - 1 - (s-s0)),
    which keeps every output at the FP32 target of 1e-5."""
    model = S.chain_poisson(n_inst=1, R=92, T=109, D=1, seed=109)
    K = 128
    q = S.random_q(model, seed=110, loc_scale=0.3, sd_lo=0.2, sd_hi=0.6)
    eps = S.noise(model, K, seed=111)
    assert_parity(model, q, _run(model, K, q, eps), C.estep(model, q, K, eps), 1e-5, 1e-5, 1e-5)


def test_chain_single_launch_loop_matches_host_loop():
    from paper_2503_08264_gb300 import qem
    model = S.chain_poisson(n_inst=2, R=6, T=10, D=1, seed=112)
    K, T_it, lam, seed = 64, 5, 0.5, 3
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


def test_chain_rejects_unsupported_plans():
    from paper_2503_08264_gb300 import _lib as L
    from paper_2503_08264_gb300 import qem
    model = S.chain_poisson(n_inst=1, R=2, T=4, D=1, seed=113)
    with pytest.raises(L.QemError) as e:
        qem.Plan(model, 128, precision="bf16x3")
    assert e.value.code == L.QEM_ERR_UNSUPPORTED
    model.levels[1].parent = model.levels[1].parent.copy()
    model.levels[1].chain = 3            # 8 days are not whole chains of 3
    with pytest.raises(L.QemError) as e:
        qem.Plan(model, 16, precision="fp32")
    assert e.value.code == L.QEM_ERR_INVALID_ARG
