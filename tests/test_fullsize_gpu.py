"""Parity at the full workload sizes, in the launch configuration the benchmark
times (split-BF16 contraction, a plan on its own stream, noise drawn in the
kernels from the counter-based stream).

* Hierarchical logistic regression, 5000 users x 10 items, K = 1024: the
  whole E-step (5.2e9 log-factor pairs) against the FP64 oracle, which draws
  the same noise from its own Philox4x32-10; about 20 s of oracle time on 16
  host cores.
* Batched three-level model, 256 instances, K = 256: the full batch on the
  GPU; the first, the largest and the last instance against the oracle run on
  the sub-model of those instances with the noise their elements have in the
  full model (instances share nothing, so this is exact sampled parity).

Tolerance: the mixed-precision 1e-3 (log P_MP relative; moments relative to
max(|m|, sd_q) and max(|m2|, sd_q^2); weights absolute).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2503_08264_gb300 import synth as S

from test_parity_gpu import assert_parity

pytestmark = pytest.mark.gpu

TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_08264_gb300 import build
    build.build()
    O.build()


def _gpu_estep(model, K, q, seed, it):
    from paper_2503_08264_gb300 import qem
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plan = qem.Plan(model, K, precision="bf16x3", stream=stream)
        qd = plan.flat(q)
        mom, _ = plan.estep(qd, None, seed=seed, it=it)
        got = {"log_pmp": plan.log_pmp(), "mom": plan.split_q(mom), "w": plan.split_w(plan.weights())}
    stream.synchronize()
    plan.close()
    return got


def test_hier_logistic_5000_users_k1024_full_estep():
    model = S.hier_logistic(M=5000, N=10, seed=1000)
    K = 1024
    q = S.random_q(model, seed=1001, loc_scale=0.3, sd_lo=0.3, sd_hi=0.8)
    got = _gpu_estep(model, K, q, seed=77, it=5)
    ref = O.estep(model, q, K, seed=77, it=5)
    assert_parity(model, q, got, ref, TOL, TOL, TOL)


def test_batched_three_level_256_k256_sampled_instances():
    model = S.batched_three_level(n_inst=256, seed=1000)
    K = 256
    q = S.random_q(model, seed=1002, loc_scale=0.3, sd_lo=0.3, sd_hi=0.8)
    got = _gpu_estep(model, K, q, seed=78, it=6)
    units_per_inst = np.bincount(model.levels[1].parent[model.levels[2].parent], minlength=256)
    ids = sorted({0, int(np.argmax(units_per_inst)), 255})
    sub, keep = S.subset(model, ids)
    q_sub = [q[l][keep[l]] for l in range(len(model.levels))]
    eps = [O.draw_noise_at(78, 6, l, keep[l], K, lv.noise_per_sample(), lv.qfam) for l, lv in enumerate(sub.levels)]
    ref = O.estep(sub, q_sub, K, eps=eps)
    got_sub = {"log_pmp": got["log_pmp"][keep[0]],
               "mom": [got["mom"][l][keep[l]] for l in range(len(keep))],
               "w": [got["w"][l][keep[l]] for l in range(len(keep))]}
    print("instances", ids, "units", [int(units_per_inst[i]) for i in ids])
    assert_parity(sub, q_sub, got_sub, ref, TOL, TOL, TOL)
    # the instances not compared still produce finite, normalised results
    assert np.all(np.isfinite(got["log_pmp"]))
    for l in range(len(model.levels)):
        if model.levels[l].n:
            np.testing.assert_allclose(got["w"][l].sum(1), 1.0, atol=1e-5)
