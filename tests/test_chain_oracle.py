"""Pins of the chain-plate oracle (oracle/chain.py): a two-level model whose
leaf plate is a daily random walk per region (the Covid model's
autoregressive timeseries, App. F), every (region, day) its own latent.

* brute force: literal enumeration of every index vector over the root and
  all days (oracle/brute.py, scipy densities) for Poisson-log and Gaussian
  observations, one- and two-dimensional latents, several instances;
* special case: chains of length 1 are an ordinary two-level model, whose
  estimator the C oracle computes (shared noise);
* weights of every latent sum to one.
"""
import copy

import numpy as np
import pytest

from oracle import brute
from oracle import chain as C
from oracle import oracle as O
from paper_2503_08264_gb300 import synth as S


def _cases():
    yield "poisson_R1_T3_K3", S.chain_poisson(n_inst=1, R=1, T=3, D=1, seed=1), 3
    yield "poisson_R2_T2_K3", S.chain_poisson(n_inst=1, R=2, T=2, D=1, seed=2), 3
    yield "gauss_D2_R1_T3_K3", S.chain_poisson(n_inst=1, R=1, T=3, D=2, seed=3, lik=S.LIK_GAUSS, n_obs=2), 3
    yield "poisson_R1_T4_K2", S.chain_poisson(n_inst=1, R=1, T=4, D=1, seed=4, n_obs=3), 2
    yield "two_instances_R1_T2_K3", S.chain_poisson(n_inst=2, R=1, T=2, D=1, seed=5), 3


@pytest.mark.parametrize("name,model,K", list(_cases()), ids=lambda v: v if isinstance(v, str) else "")
def test_chain_matches_enumeration(name, model, K):
    q = S.random_q(model, seed=11, loc_scale=0.4, sd_lo=0.4, sd_hi=1.0)
    eps = S.noise(model, K, seed=12)
    o = C.estep(model, q, K, eps)
    for inst in range(model.n_inst):
        b = brute.estep_instance_chain(model, q, o["z"], K, inst)
        np.testing.assert_allclose(o["log_pmp"][inst], b["log_pmp"], rtol=1e-12)
        for (l, e), we in b["w"].items():
            np.testing.assert_allclose(o["w"][l][e], we, rtol=1e-10, atol=1e-14)
            np.testing.assert_allclose(o["mom"][l][e], b["mom"][(l, e)], rtol=1e-10, atol=1e-13)


def test_chain_of_length_one_is_the_tree_estimator():
    model = S.chain_poisson(n_inst=2, R=5, T=1, D=2, seed=21, n_obs=3)
    K = 16
    q = S.random_q(model, seed=22, loc_scale=0.4, sd_lo=0.4, sd_hi=1.0)
    eps = S.noise(model, K, seed=23)
    a = C.estep(model, q, K, eps)
    g = O.estep(model, q, K, eps=eps)
    np.testing.assert_allclose(a["log_pmp"], g["log_pmp"], rtol=1e-12)
    for l in range(2):
        np.testing.assert_allclose(a["w"][l], g["w"][l], rtol=1e-10, atol=1e-14)
        np.testing.assert_allclose(a["mom"][l], g["mom"][l], rtol=1e-10, atol=1e-13)


def test_chain_weights_sum_to_one():
    model = S.chain_poisson(n_inst=2, R=3, T=6, D=1, seed=31)
    K = 24
    o = C.estep(model, S.random_q(model, seed=32), K, S.noise(model, K, seed=33))
    for l in range(2):
        np.testing.assert_allclose(o["w"][l].sum(1), 1.0, rtol=1e-12)
    assert np.all(np.isfinite(o["B"])) and np.all(np.isfinite(o["L"]))
