"""GPU test of the allocation-free single-level E-step.

Callers that cannot allocate device memory at the moment they need an
E-step (a runtime whose memory pool forbids outside allocations, a
latency-bound loop) use qem_estep_single_noalloc, whose scratch is a
library-wide device array.  It must give the same moments and log P_MP as the
planned E-step on the same single-level model and inputs, on consecutive
calls (the shared scratch keeps the previous call's contents).
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2503_08264_gb300 import synth as S

pytestmark = pytest.mark.gpu


def _root_gauss(n=5, N=7, seed=0):
    rng = np.random.default_rng(seed)
    y = (rng.standard_normal((n, 1)) + 0.6 * rng.standard_normal((n, N))).astype(np.float32)
    lv = S.Level(n=n, dim=1, prior=S.PRIOR_STD_NORMAL, prior_a=1.0, lik=S.LIK_GAUSS, lik_var=0.36, n_obs=N,
                 x=np.ones((n, N, 1), np.float32), y=y)
    return S.Model([lv])


@pytest.mark.parametrize("name", ["gauss", "gamma_poisson", "beta_bernoulli"])
def test_noalloc_matches_planned_estep_on_consecutive_calls(name):
    from paper_2503_08264_gb300 import build, qem
    from paper_2503_08264_gb300 import _lib as L
    build.build()
    model = {"gauss": lambda: _root_gauss(),
             "gamma_poisson": lambda: S.gamma_poisson(n_inst=6, N=9, seed=1),
             "beta_bernoulli": lambda: S.beta_bernoulli(n_inst=6, N=9, seed=2)}[name]()
    K = 64
    plan = qem.Plan(model, K, precision="fp32")
    q = plan.flat(S.initial_q(model) if name != "gauss" else S.random_q(model, seed=3))
    lv = model.levels[0]
    x_d, y_d = [t for t in plan._keep if isinstance(t, torch.Tensor)][:2]
    desc = L.LevelDesc()
    desc.n, desc.dim, desc.prior = lv.n, lv.dim, lv.prior
    desc.prior_a, desc.prior_b = float(lv.prior_a), float(lv.prior_b)
    desc.lik, desc.lik_var, desc.n_obs, desc.qfam = lv.lik, float(lv.lik_var), lv.n_obs, lv.qfam
    desc.x, desc.y = x_d.data_ptr(), y_d.data_ptr()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for eps_seed in (4, None):  # supplied noise, then the in-kernel counter-based stream
        eps = plan.flat(S.noise(model, K, seed=eps_seed)) if eps_seed is not None else None
        mom_ref, lp_ref = plan.estep(q, eps, seed=11, it=2)
        torch.cuda.synchronize()
        for call in range(2):
            mom = torch.full((plan.q_len,), float("nan"), dtype=torch.float64, device="cuda")
            lp = torch.full((plan.n_inst,), float("nan"), dtype=torch.float64, device="cuda")
            rc = L.load().qem_estep_single_noalloc(
                C.byref(desc), K, C.c_void_p(q.data_ptr()), C.c_void_p(eps.data_ptr()) if eps is not None else None,
                11, 2, C.c_void_p(mom.data_ptr()), C.c_void_p(lp.data_ptr()), stream)
            assert rc == 0, L.load().qem_status_string(rc)
            torch.cuda.synchronize()
            np.testing.assert_allclose(lp.cpu().numpy(), lp_ref.cpu().numpy(), rtol=1e-5)
            np.testing.assert_allclose(mom.cpu().numpy(), mom_ref.cpu().numpy(), rtol=1e-5, atol=1e-7)
    plan.close()


def test_noalloc_rejects_oversize_and_tree_levels():
    from paper_2503_08264_gb300 import build
    from paper_2503_08264_gb300 import _lib as L
    build.build()
    desc = L.LevelDesc()
    desc.n, desc.dim, desc.prior, desc.prior_a, desc.qfam = 100000, 16, S.PRIOR_STD_NORMAL, 1.0, S.Q_GAUSS
    dummy = torch.zeros(4, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    assert L.load().qem_estep_single_noalloc(C.byref(desc), 4096, p, None, 0, 0, p, p, None) == L.QEM_ERR_UNSUPPORTED
    par = np.zeros(1, np.int64)
    desc.n, desc.parent = 1, par.ctypes.data
    assert L.load().qem_estep_single_noalloc(C.byref(desc), 8, p, None, 0, 0, p, p, None) == L.QEM_ERR_INVALID_ARG
