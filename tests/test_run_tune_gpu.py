"""GPU tests of batching: the single-launch device loop (qem_run) and the
launch-shape autotuner (qem_tune).

* qem_run runs T iterations of Alg. 1 as one graph launch (a conditional
  while node); on a batch of uneven three-level instances with the
  split-BF16 contraction it reproduces, bit for bit, the host loop of
  qem_estep / qem_mstep with the same noise stream, and a second call
  (the cached graph) does too.
* qem_tune picks launch shapes from its candidate sets; an autotuned plan
  still matches the FP64 oracle at the path's tolerance; a second plan of the
  same shapes takes the cached choice.
* Checkpoint and resume: a run of T1 iterations, then a run of T2 from
  t0 = T1 + 1 on its saved mean parameters, equals one run of T1 + T2 bit
  for bit (mean parameters, proposal and the log P_MP trace), with the noise
  stream and Thm. 1's schedule both keyed by the iteration t.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2503_08264_gb300 import synth as S

from test_parity_gpu import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_08264_gb300 import build
    build.build()
    O.build()


def test_qem_run_single_launch_matches_host_loop():
    from paper_2503_08264_gb300 import qem
    model = S.batched_three_level(n_inst=12, D=8, seed=61, groups=(0, 6), units=(0, 30))
    K, T, lam, seed = 256, 6, 0.5, 7
    plan = qem.Plan(model, K, precision="bf16x3")
    q0 = plan.flat(S.initial_q(model))
    m0 = plan.mean_params(q0)
    # host loop: Q_1 = set(m_0), then E-step and EMA + M-step per iteration
    m_h, q_h = m0.clone(), torch.empty_like(q0)
    plan.mstep(None, m_h, q_h, lam, t=1)
    mom = torch.empty(plan.q_len, dtype=torch.float64, device="cuda")
    lps = []
    for t in range(1, T + 1):
        _, lp = plan.estep(q_h, None, seed=seed, it=t, moments=mom)
        lps.append(lp.clone())
        plan.mstep(mom, m_h, q_h, lam, t=t)
    torch.cuda.synchronize()
    for rep in range(2):
        m_r, q_r = m0.clone(), torch.empty_like(q0)
        trace = torch.full((T * plan.n_inst,), np.nan, dtype=torch.float64, device="cuda")
        plan.run(T, lam, m_r, q_r, seed=seed, trace=trace)
        torch.cuda.synchronize()
        assert torch.equal(m_r, m_h), f"call {rep}: mean parameters differ"
        assert torch.equal(q_r, q_h), f"call {rep}: proposal parameters differ"
        assert torch.equal(trace.view(T, -1), torch.stack(lps)), f"call {rep}: log P_MP trace differs"
    # a shorter run reuses the graph and stops after its own T
    m_r, q_r = m0.clone(), torch.empty_like(q0)
    plan.run(2, lam, m_r, q_r, seed=seed)
    m_2, q_2 = m0.clone(), torch.empty_like(q0)
    plan.mstep(None, m_2, q_2, lam, t=1)
    for t in range(1, 3):
        plan.estep(q_2, None, seed=seed, it=t, moments=mom)
        plan.mstep(mom, m_2, q_2, lam, t=t)
    torch.cuda.synchronize()
    assert torch.equal(m_r, m_2)
    plan.close()


@pytest.mark.parametrize("precision,K,tol", [("fp32", 128, 1e-5), ("bf16x3", 256, 1e-3)])
def test_autotuned_plan_matches_oracle_and_caches(precision, K, tol):
    """The tuner's choice (FP32 tiles, or the tensor-core schedules of a
    split-BF16 plan) gives results within the path's tolerance, and the
    cached choice is reapplied without timing."""
    from paper_2503_08264_gb300 import _lib as L
    from paper_2503_08264_gb300 import qem
    model = S.hier_logistic(M=300, N=5, seed=71)
    q = S.random_q(model, seed=72, loc_scale=0.3, sd_lo=0.3, sd_hi=0.8)
    eps = S.noise(model, K, seed=73)
    plan = qem.Plan(model, K, precision=precision, tile=L.QEM_TILE_AUTO)
    qd = plan.flat(q)
    mom, _ = plan.estep(qd, plan.flat(eps))   # tunes first (outside any capture)
    choice = plan.tuning()
    print("tuned", choice)
    assert choice["sample_threads"] in (64, 128, 256)
    assert choice["mom_threads"] in (128, 256, 512)
    assert choice["fwd_rows"] in (64, 128, 256) and choice["fwd_chunk"] in (16, 32, 64)
    assert choice["tc_sched"] in (0, 1, 2, 3)
    got = {"log_pmp": plan.log_pmp(), "mom": plan.split_q(mom), "w": plan.split_w(plan.weights())}
    ref = O.estep(model, q, K, eps=eps)
    assert_parity(model, q, got, ref, tol, tol, tol)
    # every candidate of every knob is a valid launch: force each one
    forced = plan.tune(qd, force=True)
    assert forced == plan.tuning()
    plan.close()
    # same shapes: the cached choice is applied without timing
    plan2 = qem.Plan(model, K, precision=precision)
    assert plan2.tune(plan2.flat(q)) == forced
    plan2.close()


@pytest.mark.parametrize("case", ["bf16x3_hier_logistic", "fp32_chain"])
def test_run_resumes_bit_identically(case):
    from paper_2503_08264_gb300 import qem
    if case == "bf16x3_hier_logistic":
        model, K, prec = S.hier_logistic(M=60, N=5, seed=81), 256, "bf16x3"
    else:
        model, K, prec = S.chain_poisson(n_inst=2, R=5, T=12, D=1, seed=82), 64, "fp32"
    T1, T2, lam, sched_p, seed = 4, 5, 0.5, 0.6, 17
    plan = qem.Plan(model, K, precision=prec)
    q0 = plan.flat(S.initial_q(model))
    m0 = plan.mean_params(q0)
    n = plan.n_inst
    # one run of T1 + T2
    m_a, q_a = m0.clone(), torch.empty_like(q0)
    tr_a = torch.empty((T1 + T2) * n, dtype=torch.float64, device="cuda")
    plan.run(T1 + T2, lam, m_a, q_a, sched_p=sched_p, seed=seed, trace=tr_a)
    # T1, a checkpoint of the mean parameters (host copy), then T2 from t0 = T1 + 1
    m_b, q_b = m0.clone(), torch.empty_like(q0)
    tr_b1 = torch.empty(T1 * n, dtype=torch.float64, device="cuda")
    plan.run(T1, lam, m_b, q_b, sched_p=sched_p, seed=seed, trace=tr_b1)
    saved = m_b.cpu()
    m_c, q_c = saved.cuda(), torch.empty_like(q0)
    tr_b2 = torch.empty(T2 * n, dtype=torch.float64, device="cuda")
    plan.run(T2, lam, m_c, q_c, sched_p=sched_p, seed=seed, trace=tr_b2, t0=T1 + 1)
    torch.cuda.synchronize()
    assert torch.equal(m_c, m_a)
    assert torch.equal(q_c, q_a)
    assert torch.equal(torch.cat([tr_b1, tr_b2]), tr_a)
    # a resume from another t gives another run (the schedule and the noise move with t)
    m_d, q_d = saved.cuda(), torch.empty_like(q0)
    plan.run(T2, lam, m_d, q_d, sched_p=sched_p, seed=seed, t0=T1 + 2)
    torch.cuda.synchronize()
    assert not torch.equal(m_d, m_a)
    plan.close()
