"""The sharded E-step through the C ABI (qem_estep_shard_forward / _finish,
qem_set_elem_base) on one GPU: the shards of one instance run one after the
other in this process (no kernel waits on another), their root plate sums G_r
are added on the device in place of the all-reduce between processes, and the
reassembled log P_MP, weights and moments are checked against the FP64
oracle of the whole model at the parity tolerances; with the in-kernel noise
and each shard's element base, against one plan holding the whole model.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import chain as OC
from oracle import oracle as O
from paper_2503_08264_gb300 import shard as SH
from paper_2503_08264_gb300 import synth as S

from test_parity_gpu import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_08264_gb300 import build
    build.build()
    O.build()


def _model(name):
    if name == "hier_logistic":
        return S.hier_logistic(M=150, N=5, D=18, seed=61), 128
    if name == "three_level":
        return S.batched_three_level(n_inst=3, D=4, seed=62, groups=(3, 6), units=(2, 30)), 64
    return S.chain_poisson(n_inst=1, R=6, T=9, D=1, seed=63), 64


def _sharded(model, K, world, precision, q=None, eps=None, seed=0, it=0):
    """Run the E-step as `world` shards; return (per-shard log_pmp, assembled w, mom)."""
    from paper_2503_08264_gb300 import qem
    plans, ranges_of = [], []
    for lo, hi in SH.child_ranges(model, world):
        sub, ranges = SH.shard_model(model, lo, hi)
        p = qem.Plan(sub, K, precision=precision)
        p.set_elem_base([a for a, _ in ranges])
        plans.append(p)
        ranges_of.append(ranges)
    qd = [p.flat(SH.take(q, r)) for p, r in zip(plans, ranges_of)]
    ed = [None if eps is None else p.flat(SH.take(eps, r)) for p, r in zip(plans, ranges_of)]
    Gs = [p.shard_forward(qq, ee, seed, it) for p, qq, ee in zip(plans, qd, ed)]
    G = torch.stack(Gs).sum(0)
    outs = [p.shard_finish(G) for p in plans]
    torch.cuda.synchronize()
    lps = [p.log_pmp() for p in plans]
    w = SH.assemble([p.split_w(p.weights()) for p in plans], ranges_of)
    m = SH.assemble([p.split_q(o[0]) for p, o in zip(plans, outs)], ranges_of)
    for p in plans:
        p.close()
    return lps, w, m


def _whole_oracle(model, q, K, eps):
    if int(getattr(model.levels[1], "chain", 1) or 1) > 1:
        return OC.estep(model, q, K, eps)
    return O.estep(model, q, K, eps)


@pytest.mark.parametrize("name,precision,world,tol", [
    ("hier_logistic", "fp32", 3, (1e-5, 1e-5, 1e-5)),
    ("three_level", "fp32", 2, (1e-5, 1e-5, 1e-5)),
    ("chain", "fp32", 3, (1e-5, 1e-5, 1e-5)),
    ("hier_logistic", "bf16x3", 2, (1e-3, 1e-3, 1e-3)),
])
def test_sharded_estep_matches_whole_model_oracle(name, precision, world, tol):
    model, K = _model(name)
    q = S.random_q(model, seed=64, loc_scale=0.3, sd_lo=0.3, sd_hi=0.8)
    eps = S.noise(model, K, seed=65)
    lps, w, m = _sharded(model, K, world, precision, q, eps)
    for lp in lps[1:]:
        np.testing.assert_array_equal(lp, lps[0])   # the root step is identical on every shard
    ref = _whole_oracle(model, q, K, eps)
    assert_parity(model, q, {"log_pmp": lps[0], "w": w, "mom": m}, ref, *tol)


@pytest.mark.parametrize("name", ["hier_logistic", "three_level"])
def test_sharded_in_kernel_noise_draws_the_whole_models_samples(name):
    """With each shard's element base the counter-based noise is the whole
    model's: the sharded E-step matches one plan of the whole model (FP32
    summation order apart)."""
    from paper_2503_08264_gb300 import qem
    model, K = _model(name)
    q = S.random_q(model, seed=66, loc_scale=0.3, sd_lo=0.3, sd_hi=0.8)
    lps, w, m = _sharded(model, K, 2, "fp32", q, None, seed=5, it=3)
    whole = qem.Plan(model, K, precision="fp32")
    mom, _ = whole.estep(whole.flat(q), None, seed=5, it=3)
    torch.cuda.synchronize()
    ref = {"log_pmp": whole.log_pmp(), "w": whole.split_w(whole.weights()), "mom": whole.split_q(mom)}
    whole.close()
    np.testing.assert_allclose(lps[0], ref["log_pmp"], rtol=1e-7)
    for l in range(len(model.levels)):
        np.testing.assert_allclose(w[l], ref["w"][l], rtol=1e-4, atol=1e-7)
        np.testing.assert_allclose(m[l], ref["mom"][l], rtol=1e-5, atol=1e-6)
    from paper_2503_08264_gb300 import _lib as L
    plan = qem.Plan(SH.shard_model(model, *SH.child_ranges(model, 2)[1])[0], K, precision="fp32")
    with pytest.raises(L.QemError):
        plan.set_elem_base([0, -1] + [0] * (len(model.levels) - 2))
    plan.close()


def test_shard_entry_points_reject_a_one_level_plan():
    from paper_2503_08264_gb300 import _lib as L
    from paper_2503_08264_gb300 import qem
    model = S.Model([S.Level(n=2, dim=2, prior=S.PRIOR_STD_NORMAL)])
    plan = qem.Plan(model, 32)
    q = plan.flat(S.random_q(model, seed=1))
    G = torch.zeros((2, 32), dtype=torch.float64, device="cuda")
    with pytest.raises(L.QemError) as e:
        plan.shard_forward(q, None, 0, 0, G)
    assert e.value.code == L.QEM_ERR_UNSUPPORTED
    plan.close()
