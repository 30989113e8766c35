"""GPU tests of the tensor-core (tcgen05) contraction path.

* the operand layout / descriptor path, through the diagnostic GEMM entry
  point, against a plain fp32 matmul of the same BF16 operands;
* the E-step with split-BF16 operands (BF16X3) against the FP64 oracle at the
  mixed-precision tolerance (1e-3 relative: log P_MP, moments relative to
  max(|m|, sd_q) or sd_q^2, weights absolute);
* plain BF16 and TF32 report their errors (kept for the precision study: the
  parent's operand rows are shared by all of its children, so their rounding
  adds up over the plate sum instead of averaging out);
* the element-resident and streaming schedules agree to FP32 summation
  order (the same MMAs; each row's exponentials are added in another order).
"""
import ctypes as C

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


def canonical(x: torch.Tensor) -> torch.Tensor:
    """[R, F] -> the K-major core-matrix layout (8 x 8 blocks, row groups major)."""
    R, F = x.shape
    return x.view(R // 8, 8, F // 8, 8).permute(0, 2, 1, 3).contiguous().view(-1)


@pytest.mark.parametrize("fk,n", [(16, 16), (48, 64), (112, 256), (128, 128), (32, 240)])
def test_diag_gemm_matches_matmul(fk, n):
    from paper_2503_08264_gb300 import _lib as L
    g = torch.Generator().manual_seed(fk * 1000 + n)
    A = torch.randn(128, fk, generator=g).to(torch.bfloat16)
    B = torch.randn(n, fk, generator=g).to(torch.bfloat16)
    ref = A.float() @ B.float().T
    Ad, Bd = canonical(A).cuda(), canonical(B).cuda()
    out = torch.zeros(128, n, dtype=torch.float32, device="cuda")
    rc = L.load().qem_diag_tc_gemm(C.c_void_p(Ad.data_ptr()), C.c_void_p(Bd.data_ptr()), fk, n,
                                   C.c_void_p(out.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    np.testing.assert_allclose(out.cpu().numpy(), ref.numpy(), rtol=1e-5, atol=1e-4)


from test_parity_gpu import assert_parity, moment_errors, run_pair  # noqa: E402


@pytest.mark.parametrize("M,K", [(300, 128), (40, 256), (13, 1024)])
def test_bf16x3_hier_logistic_parity(M, K):
    model = S.hier_logistic(M=M, N=5, seed=11)
    q = S.random_q(model, seed=12, loc_scale=0.3, sd_lo=0.3, sd_hi=0.8)
    eps = S.noise(model, K, seed=13)
    got, ref = run_pair(model, K, q, eps, precision="bf16x3")
    assert_parity(model, q, got, ref, 1e-3, 1e-3, 1e-3)


def test_bf16x3_three_level_parity():
    model = S.batched_three_level(n_inst=6, D=8, seed=21, groups=(0, 5), units=(0, 12))
    K = 256
    q = S.random_q(model, seed=22, loc_scale=0.3, sd_lo=0.3, sd_hi=0.8)
    eps = S.noise(model, K, seed=23)
    got, ref = run_pair(model, K, q, eps, precision="bf16x3")
    assert_parity(model, q, got, ref, 1e-3, 1e-3, 1e-3)


def test_bf16x3_from_initial_proposal():
    """q0 = N(0, I) (App. F): very uneven weights, the overflow-rescale path."""
    model = S.hier_logistic(M=64, N=10, seed=31)
    K = 512
    q = S.initial_q(model)
    eps = S.noise(model, K, seed=32)
    got, ref = run_pair(model, K, q, eps, precision="bf16x3")
    assert_parity(model, q, got, ref, 1e-3, 1e-3, 1e-3)


def test_plain_bf16_reports_error():
    model = S.hier_logistic(M=100, N=5, seed=41)
    K = 256
    q = S.random_q(model, seed=42, loc_scale=0.3, sd_lo=0.3, sd_hi=0.8)
    eps = S.noise(model, K, seed=43)
    got, ref = run_pair(model, K, q, eps, precision="bf16")
    lp = np.max(np.abs(got["log_pmp"] - ref["log_pmp"]) / np.abs(ref["log_pmp"]))
    print("plain bf16: log_pmp rel", lp, "moments", moment_errors(model, q, got["mom"], ref["mom"]))
    assert lp < 1e-2


@pytest.mark.parametrize("precision,tol", [("bf16x3", 1e-3), ("fp32", 1e-5)])
def test_dense_parent_weights(precision, tol):
    """Few children per parent: the parents' weights stay spread, so the
    adjoint runs over hundreds of kept parent samples (the tensor-core adjoint
    for the split-BF16 path)."""
    model = S.batched_three_level(n_inst=4, D=8, seed=51, groups=(2, 3), units=(1, 2))
    K = 256
    q = S.initial_q(model)
    eps = S.noise(model, K, seed=52)
    got, ref = run_pair(model, K, q, eps, precision=precision)
    rel = 2.0 ** -40 if precision == "fp32" else 2.0 ** -24   # the adjoint's compaction threshold
    kept = [(r > rel * r.max(1, keepdims=True)).sum(1).min() for r in ref["w"][:2]]
    print("min kept parent samples per level", kept)
    assert min(kept) > 16
    assert_parity(model, q, got, ref, tol, tol, tol)


def _estep_with(model, K, q, eps, precision, **tuning):
    from paper_2503_08264_gb300 import qem
    plan = qem.Plan(model, K, precision=precision)
    if tuning:
        plan.set_tuning(**tuning)
    mom, _ = plan.estep(plan.flat(q), plan.flat(eps))
    out = {"log_pmp": plan.log_pmp(), "mom": mom.cpu().numpy(), "w": plan.weights().cpu().numpy(),
           "tuning": plan.tuning()}
    plan.close()
    return out


@pytest.mark.parametrize("precision", ["bf16x3", "tf32"])
@pytest.mark.parametrize("M,K", [(300, 128), (200, 256), (40, 384), (3, 640), (13, 1024)])
def test_schedules_agree(precision, M, K):
    """Both element-resident kernels (tc_sched 3) against the streaming ones:
    K = 128 (one 128-column chunk), 256, 384 and 640 (a ragged last chunk),
    1024 (four resident chunks, two adjoint passes); M > 152 wraps elements
    around the CTAs."""
    model = S.hier_logistic(M=M, N=5, seed=61)
    q = S.random_q(model, seed=62, loc_scale=0.3, sd_lo=0.3, sd_hi=0.8)
    eps = S.noise(model, K, seed=63)
    res = _estep_with(model, K, q, eps, precision, tc_sched=3)
    stream = _estep_with(model, K, q, eps, precision, tc_sched=0)
    assert res["tuning"]["tc_sched"] == 3 and stream["tuning"]["tc_sched"] == 0
    np.testing.assert_allclose(res["log_pmp"], stream["log_pmp"], rtol=1e-7)
    np.testing.assert_allclose(res["w"], stream["w"], rtol=1e-5, atol=1e-9)
    # moments relative to max(|m|, sd_q) (the parity tests' measure): near-zero
    # means are sums of +-1e-3 terms whose FP32 summation order shows at 1e-7
    plan_q = [np.asarray(x, np.float64) for x in q]
    off, split_r, split_s = 0, [], []
    for lv in model.levels:
        n = lv.n * 2 * lv.dim
        split_r.append(res["mom"][off:off + n].reshape(lv.n, 2, lv.dim))
        split_s.append(stream["mom"][off:off + n].reshape(lv.n, 2, lv.dim))
        off += n
    assert max(moment_errors(model, plan_q, split_r, split_s)) < 1e-5


@pytest.mark.parametrize("K", [384, 512, 640, 1024])
def test_resident_adjoint_dense_root_weights(K):
    """Flat root weights (the root's proposal equal to its prior, few users):
    the root keeps most of its K samples, so every element's resident adjoint
    (tc_sched 3) runs over full chunks of 256 and a ragged last one; against
    the oracle at the mixed-precision tolerance.  K = 384 (three row blocks
    in a pass) and 640 (passes of four and one) give odd row-block counts,
    where a row block's tiles alternate between the two epilogue groups from
    chunk to chunk."""
    model = S.hier_logistic(M=3, N=2, seed=65)
    q = S.random_q(model, seed=66, loc_scale=0.1, sd_lo=0.9, sd_hi=1.1)
    q[0][:, 0, :] = 0.0
    q[0][:, 1, :] = 1.0
    eps = S.noise(model, K, seed=67)
    got, ref = run_pair(model, K, q, eps, precision="bf16x3", tuning={"tc_sched": 3})
    kept = (ref["w"][0] > 2.0 ** -24 * ref["w"][0].max(1, keepdims=True)).sum(1).min()
    print("kept root samples", kept)
    assert kept > K // 2
    assert_parity(model, q, got, ref, 1e-3, 1e-3, 1e-3)


def test_tune_set_rejects_values_outside_the_candidates():
    from paper_2503_08264_gb300 import _lib as L
    from paper_2503_08264_gb300 import qem
    plan = qem.Plan(S.hier_logistic(M=4, N=2, seed=0), 128, precision="bf16x3")
    with pytest.raises(L.QemError) as ei:
        plan.set_tuning(tc_sched=4)
    assert ei.value.code == L.QEM_ERR_INVALID_ARG
    with pytest.raises(L.QemError):
        plan.set_tuning(sample_threads=96)
    plan.close()


@pytest.mark.parametrize("M,K", [(300, 128), (40, 256), (13, 1024)])
def test_tf32_reports_error(M, K):
    """kind::tf32 with one product per k-step: errors reported (like plain
    BF16, not held to the mixed-precision tolerance)."""
    model = S.hier_logistic(M=M, N=5, seed=11)
    q = S.random_q(model, seed=12, loc_scale=0.3, sd_lo=0.3, sd_hi=0.8)
    eps = S.noise(model, K, seed=13)
    got, ref = run_pair(model, K, q, eps, precision="tf32")
    lp = np.max(np.abs(got["log_pmp"] - ref["log_pmp"]) / np.abs(ref["log_pmp"]))
    w = [np.max(np.abs(got["w"][l] - ref["w"][l])) for l in range(2)]
    print(f"tf32 M={M} K={K}: log_pmp rel {lp:.2e}, moments",
          ["%.2e" % e for e in moment_errors(model, q, got["mom"], ref["mom"])], "weights", ["%.2e" % e for e in w])
    assert lp < 1e-2
    for l in range(2):
        np.testing.assert_allclose(got["w"][l].sum(1), 1.0, atol=1e-5)


def test_tf32_three_level_reports_error():
    model = S.batched_three_level(n_inst=6, D=8, seed=21, groups=(0, 5), units=(0, 12))
    K = 256
    q = S.random_q(model, seed=22, loc_scale=0.3, sd_lo=0.3, sd_hi=0.8)
    eps = S.noise(model, K, seed=23)
    got, ref = run_pair(model, K, q, eps, precision="tf32")
    lp = np.max(np.abs(got["log_pmp"] - ref["log_pmp"]) / np.abs(ref["log_pmp"]))
    print(f"tf32 three-level: log_pmp rel {lp:.2e}, moments",
          ["%.2e" % e for e in moment_errors(model, q, got["mom"], ref["mom"])])
    assert lp < 1e-2


def test_expired_wait_reports_timeout_and_the_next_plan_works():
    """A device wait that runs out: with the test hook on, the contraction's
    MMA-issuing thread first waits on a barrier that nothing completes before
    the teardown (a flag nothing sets); the wait ends after timeout_s = 10 ms,
    every role of the CTA stops at its next wait, the CTA waits for its own
    copies and MMAs under a separate bound before it frees TMEM and exits, and
    qem_log_pmp reports QEM_ERR_TIMEOUT; under each tensor-core schedule (the
    forward's and the adjoint's resident and streaming kernels).  The context
    stays usable: a fresh plan in the same process then matches the oracle.
    (A short timeout_s alone makes no wait run out: mbarrier.try_wait
    suspends until the phase completes, and the copies land within that.)"""
    from paper_2503_08264_gb300 import _lib as L
    from paper_2503_08264_gb300 import qem
    model = S.hier_logistic(M=40, N=5, seed=91)
    K = 256
    q = S.random_q(model, seed=92, loc_scale=0.3, sd_lo=0.3, sd_hi=0.8)
    eps = S.noise(model, K, seed=93)
    for sched in (1, 0, 3, 2):
        plan = qem.Plan(model, K, precision="bf16x3", timeout_s=0.01)
        plan.set_tuning(tc_sched=sched)
        plan.test_expire_wait(True)
        plan.estep(plan.flat(q), plan.flat(eps))
        with pytest.raises(L.QemError) as ei:
            plan.log_pmp()
        assert ei.value.code == L.QEM_ERR_TIMEOUT, (sched, ei.value.code)
        plan.close()
    got, ref = run_pair(model, K, q, eps, precision="bf16x3")
    assert_parity(model, q, got, ref, 1e-3, 1e-3, 1e-3)


def test_plans_of_different_shapes_coexist():
    """Kernels are opted into the maximum dynamic shared memory once: a plan
    with smaller operands made after a larger one must not lower the limit
    the larger plan's launches need (K = 1024 rows need ~220 KB per CTA)."""
    from paper_2503_08264_gb300 import qem
    big_model = S.hier_logistic(M=24, N=5, seed=95)
    small_model = S.hier_logistic(M=24, N=5, seed=96)
    big = qem.Plan(big_model, 1024, precision="bf16x3")
    small = qem.Plan(small_model, 256, precision="bf16x3")
    q_small = S.random_q(small_model, seed=97, loc_scale=0.3, sd_lo=0.3, sd_hi=0.8)
    small.estep(small.flat(q_small), small.flat(S.noise(small_model, 256, seed=98)))
    small.log_pmp()
    small.close()
    q = S.random_q(big_model, seed=99, loc_scale=0.3, sd_lo=0.3, sd_hi=0.8)
    eps = S.noise(big_model, 1024, seed=100)
    mom, _ = big.estep(big.flat(q), big.flat(eps))
    torch.cuda.synchronize()
    got = {"log_pmp": big.log_pmp(), "mom": big.split_q(mom), "w": big.split_w(big.weights())}
    big.close()
    assert_parity(big_model, q, got, O.estep(big_model, q, 1024, eps=eps), 1e-3, 1e-3, 1e-3)
