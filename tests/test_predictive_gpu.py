"""GPU tests of the predictive log-likelihood of held-out data (qem_predictive)
against the FP64 oracle's, both from their own E-step on the same noise."""
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


@pytest.mark.parametrize("case,precision,tol", [("logistic", "fp32", 1e-5), ("logistic", "bf16x3", 1e-3),
                                                ("poisson", "fp32", 1e-5)])
def test_predictive_matches_oracle(case, precision, tol):
    from paper_2503_08264_gb300 import qem
    rng = np.random.default_rng(91)
    if case == "logistic":
        model = S.hier_logistic(M=60, N=5, seed=92)
        level, K, N = 1, 128, 4
        x_new = (rng.random((60, N, 18)) < 0.3).astype(np.float32)
        y_new = (rng.random((60, N)) < 0.5).astype(np.float32)
    else:
        model = S.batched_three_level(n_inst=3, D=8, seed=93, groups=(1, 3), units=(2, 9))
        level, K, N = 2, 128, 3
        nu = model.levels[2].n
        x_new = (rng.standard_normal((nu, N, 8)) * np.sqrt(1 / 8)).astype(np.float32)
        y_new = rng.poisson(1.5, (nu, N)).astype(np.float32)
    q = S.random_q(model, seed=94, loc_scale=0.3, sd_lo=0.3, sd_hi=0.8)
    eps = S.noise(model, K, seed=95)
    plan = qem.Plan(model, K, precision=precision)
    plan.estep(plan.flat(q), plan.flat(eps))
    got = plan.predictive(level, x_new, y_new).cpu().numpy()
    plan.close()
    ref = O.estep(model, q, K, eps=eps)
    lv = model.levels[level]
    want = O.predictive(ref["z"][level], ref["w"][level], lv.lik, x_new, y_new, lv.lik_var)
    err = np.max(np.abs(got - want) / np.maximum(np.abs(want), 1.0))
    print(case, precision, "max relative error", err)
    assert err < tol
