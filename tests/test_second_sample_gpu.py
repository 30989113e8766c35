"""GPU tests of the second-sample estimates (the remark after Theorem 1):
log P_MP from a fresh draw (qem_log_pmp_fresh) and the moments normalised by
it (qem_moments_rescale), against the FP64 oracle composed the same way."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2503_08264_gb300 import synth as S

from test_parity_gpu import moment_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_08264_gb300 import build
    build.build()
    O.build()


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_fresh_draw_with_the_estep_stream_repeats_its_log_pmp(precision):
    from paper_2503_08264_gb300 import qem
    model = S.batched_three_level(n_inst=5, D=8, seed=81, groups=(1, 4), units=(1, 20))
    K = 128
    plan = qem.Plan(model, K, precision=precision)
    q = plan.flat(S.random_q(model, seed=82, loc_scale=0.3, sd_lo=0.3, sd_hi=0.8))
    _, lp = plan.estep(q, None, seed=9, it=4)
    lp_e = lp.clone()
    lp_f = plan.log_pmp_fresh(q, seed=9, it=4)
    torch.cuda.synchronize()
    assert torch.equal(lp_e, lp_f)
    plan.close()


def test_second_sample_moments_match_oracle():
    from paper_2503_08264_gb300 import qem
    model = S.batched_three_level(n_inst=4, D=8, seed=83, groups=(1, 4), units=(1, 15))
    K = 64
    q = S.random_q(model, seed=84, loc_scale=0.3, sd_lo=0.4, sd_hi=0.9)
    plan = qem.Plan(model, K, precision="fp32")
    qd = plan.flat(q)
    mom, lp_same = plan.estep(qd, None, seed=21, it=2)
    lp_same = lp_same.clone()
    lp_new = plan.log_pmp_fresh(qd, seed=21, it=1002)
    plan.moments_rescale(lp_same, lp_new, mom)
    got_mom = plan.split_q(mom)
    got_new = lp_new.cpu().numpy()
    plan.close()
    a = O.estep(model, q, K, seed=21, it=2)
    b = O.estep(model, q, K, seed=21, it=1002)
    np.testing.assert_allclose(got_new, b["log_pmp"], rtol=1e-5)
    ratio = np.exp(a["log_pmp"] - b["log_pmp"])
    inst = [np.arange(model.levels[0].n)]
    for l in range(1, len(model.levels)):
        inst.append(inst[-1][model.levels[l].parent])
    ref = [a["mom"][l] * ratio[inst[l]][:, None, None] for l in range(len(model.levels))]
    print("P_MP(z) / P_MP(z_new) per instance", ratio)
    # the ratio multiplies both moments: compare relative to the rescaled scale
    errs = moment_errors(model, [np.stack([qq[:, 0], qq[:, 1] * r[:, None]], 1) for qq, r in
                                 zip(q, [ratio[i] for i in inst])], got_mom, ref)
    print("moment errors", errs)
    assert max(errs) < 1e-4
