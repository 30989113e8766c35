"""Seeded synthetic workloads for the QEM E-step.

This module only *describes* models and *draws* data and noise.  It holds none
of the estimator's arithmetic (no log-densities, no importance weights, no
moments), so both the CUDA path and the CPU oracle can take their inputs from
it without sharing any of the method.

A model is a plate tree of levels (Sec. 3.2 and App. A.2 of the paper: one
latent per plate element, K samples per latent, a factorised proposal).  Level
0 holds one root latent per independent instance; every element of level l>0
has one parent element at level l-1, and elements are stored grouped by
parent (parent indices non-decreasing), which makes every plate a contiguous
CSR segment.

The workloads follow the model definitions of App. F (MovieLens, Eq. in
App. F.3) and the conjugate hierarchies used to pin the estimator:

* ``conjugate_gaussian``  mu~N(0,1), z_m~N(mu,1), x_mn~N(z_m,0.5^2)
* ``hier_logistic``       mu,psi~N(0,I_18), z_m~N(mu,diag e^psi), y~Bern(sigmoid(z.x))
* ``batched_three_level`` mu~N(0,I_8), z_g~N(mu,I), z_u~N(z_g,0.5^2 I), y~Pois(exp(w.z_u))
* ``gamma_poisson`` / ``beta_bernoulli``  single-latent conjugate pairs for the
  Gamma and Beta proposal families.
* ``chain_poisson``       g~N(0,I); per region a daily random walk z_{c,0}~N(g,a I),
  z_{c,d}~N(z_{c,d-1},b I); y~Pois(exp(z.x)) (the Covid model's chain plate, App. F)

A chain level (``chain`` = T > 1, the leaf level of a two-level model) holds
T consecutive elements per region, element c T + d for day d; all T share the
region's parent, the first day's prior is the level's prior given the parent
and every later day's is N(previous day, prior_b I).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# prior kinds of a level (how p(z_e | z_parent) is defined)
PRIOR_STD_NORMAL = 0      # N(0, prior_a * I)                      (roots)
PRIOR_NORMAL_FIXED_VAR = 1  # N(z_parent, prior_a * I), dim(parent) == dim
PRIOR_NORMAL_MEAN_LOGVAR = 2  # N(z_parent[:D], diag exp(z_parent[D:])), dim(parent) == 2D
PRIOR_GAMMA = 3           # Gamma(shape=prior_a, rate=prior_b)      (roots, D=1)
PRIOR_BETA = 4            # Beta(prior_a, prior_b)                   (roots, D=1)

# likelihood kinds of a level; s = z . x_n is the linear predictor
LIK_NONE = 0
LIK_GAUSS = 1             # y ~ N(s, lik_var)
LIK_BERNOULLI_LOGIT = 2   # y ~ Bernoulli(sigmoid(s))
LIK_POISSON_LOG = 3       # y ~ Poisson(exp(s))
LIK_POISSON_RATE = 4      # y ~ Poisson(z)        (D=1, z>0)
LIK_BERNOULLI_PROB = 5    # y ~ Bernoulli(z)      (D=1, 0<z<1)

# proposal families; the two q parameters per dimension are
Q_GAUSS = 0               # (loc, scale)
Q_GAMMA = 1               # (shape, rate)
Q_BETA = 2                # (a, b)

# Marsaglia-Tsang attempts carried by the supplied noise of a Gamma sample
GAMMA_TRIES = 8


@dataclass
class Level:
    n: int
    dim: int
    prior: int
    prior_a: float = 1.0
    prior_b: float = 1.0
    lik: int = LIK_NONE
    lik_var: float = 1.0
    n_obs: int = 0
    qfam: int = Q_GAUSS
    parent: np.ndarray | None = None   # int64 [n], non-decreasing
    x: np.ndarray | None = None        # float32 [n, n_obs, dim]
    y: np.ndarray | None = None        # float32 [n, n_obs]
    chain: int = 1                     # T > 1: elements form chains of T days (leaf level)
    qcond: int = 0                     # 1: proposal centred on a permuted parent copy (leaf level)

    def noise_per_sample(self) -> int:
        """Number of N(0,1)/U(0,1) numbers one sample of this level consumes."""
        if self.qfam == Q_GAUSS:
            return self.dim
        if self.qfam == Q_GAMMA:
            return self.dim * (2 * GAMMA_TRIES + 1)
        return self.dim * 2 * (2 * GAMMA_TRIES + 1)


@dataclass
class Model:
    levels: list
    name: str = ""
    truth: dict = field(default_factory=dict)

    @property
    def n_inst(self) -> int:
        return self.levels[0].n

    def pairs(self, K: int) -> int:
        """K_parent * K_child log-factor pairs of one E-step."""
        return int(sum(lv.n for lv in self.levels[1:])) * K * K


def _x_obs(rng, n, n_obs, dim, p=None, scale=None):
    if p is not None:
        return (rng.random((n, n_obs, dim)) < p).astype(np.float32)
    return (rng.standard_normal((n, n_obs, dim)) * scale).astype(np.float32)


def conjugate_gaussian(M: int = 8, N: int = 16, seed: int = 0, obs_var: float = 0.25) -> Model:
    """mu ~ N(0,1); z_m ~ N(mu,1); x_mn ~ N(z_m, obs_var)."""
    rng = np.random.default_rng(seed)
    mu = rng.standard_normal()
    z = mu + rng.standard_normal(M)
    y = (z[:, None] + np.sqrt(obs_var) * rng.standard_normal((M, N))).astype(np.float32)
    root = Level(n=1, dim=1, prior=PRIOR_STD_NORMAL, prior_a=1.0)
    users = Level(n=M, dim=1, prior=PRIOR_NORMAL_FIXED_VAR, prior_a=1.0,
                  lik=LIK_GAUSS, lik_var=obs_var, n_obs=N,
                  parent=np.zeros(M, np.int64),
                  x=np.ones((M, N, 1), np.float32), y=y)
    return Model([root, users], name=f"conjugate_gaussian_M{M}_N{N}",
                 truth={"mu": mu, "z": z})


def hier_logistic(M: int = 300, N: int = 5, D: int = 18, seed: int = 0, p_feat: float = 0.3) -> Model:
    """MovieLens-shaped hierarchical logistic regression (App. F.3).

    Root = the grouped (mu, psi) pair as one 2D-dimensional latent; users
    z_m ~ N(mu, diag exp(psi)); binary genre features per (user, item).
    """
    rng = np.random.default_rng(seed)
    mu = rng.standard_normal(D)
    psi = rng.standard_normal(D)
    z = mu + np.exp(0.5 * psi) * rng.standard_normal((M, D))
    x = _x_obs(rng, M, N, D, p=p_feat)
    s = np.einsum("mnd,md->mn", x.astype(np.float64), z)
    y = (rng.random((M, N)) < 1.0 / (1.0 + np.exp(-s))).astype(np.float32)
    root = Level(n=1, dim=2 * D, prior=PRIOR_STD_NORMAL, prior_a=1.0)
    users = Level(n=M, dim=D, prior=PRIOR_NORMAL_MEAN_LOGVAR, lik=LIK_BERNOULLI_LOGIT,
                  n_obs=N, parent=np.zeros(M, np.int64), x=x, y=y)
    return Model([root, users], name=f"hier_logistic_M{M}_N{N}",
                 truth={"mu": mu, "psi": psi, "z": z})


def hier_logistic_batch(n_inst: int, M: int = 300, N: int = 5, D: int = 18, seed: int = 0,
                        p_feat: float = 0.3) -> Model:
    """n_inst independent hierarchical logistic instances in one model (instance
    i is hier_logistic(M, N, D, seed + i); roots are the instances)."""
    parts = [hier_logistic(M=M, N=N, D=D, seed=seed + i, p_feat=p_feat) for i in range(n_inst)]
    root = Level(n=n_inst, dim=2 * D, prior=PRIOR_STD_NORMAL, prior_a=1.0)
    users = Level(n=n_inst * M, dim=D, prior=PRIOR_NORMAL_MEAN_LOGVAR, lik=LIK_BERNOULLI_LOGIT, n_obs=N,
                  parent=np.repeat(np.arange(n_inst, dtype=np.int64), M),
                  x=np.concatenate([p.levels[1].x for p in parts]), y=np.concatenate([p.levels[1].y for p in parts]))
    return Model([root, users], name=f"hier_logistic_batch{n_inst}_M{M}_N{N}")


def mlp_init(seed: int, sizes=(37, 128, 128, 36), out_scale: float = 0.1) -> np.ndarray:
    """Initial warm-start network parameters (flat layout W1, b1, W2, b2, W3,
    b3): He-normal weights (std sqrt(2 / fan_in)), the output layer scaled by
    out_scale, zero biases."""
    rng = np.random.default_rng(seed)
    out = []
    for j, (i, o) in enumerate(zip(sizes[:-1], sizes[1:])):
        W = rng.standard_normal((o, i)) * np.sqrt(2.0 / i)
        if j == len(sizes) - 2:
            W *= out_scale
        out += [W.reshape(-1), np.zeros(o)]
    return np.concatenate(out).astype(np.float32)


def batched_three_level(n_inst: int = 256, D: int = 8, seed: int = 0,
                        groups=(5, 40), units=(10, 200), n_obs: int = 4,
                        unit_var: float = 0.25) -> Model:
    """Independent 3-level instances with uneven plates.

    mu ~ N(0,I_D); G ~ U{groups}; z_g ~ N(mu, I); units per group ~ U{units};
    z_u ~ N(z_g, unit_var I); n_obs obs y ~ Poisson(exp(w.z_u)), w ~ N(0, I/D).
    """
    rng = np.random.default_rng(seed)
    G = rng.integers(groups[0], groups[1] + 1, size=n_inst)       # may be 0: an empty plate
    gpar = np.repeat(np.arange(n_inst, dtype=np.int64), G)
    U = rng.integers(units[0], units[1] + 1, size=int(G.sum()))
    upar = np.repeat(np.arange(int(G.sum()), dtype=np.int64), U)
    mu = rng.standard_normal((n_inst, D))
    zg = mu[gpar] + rng.standard_normal((len(gpar), D))
    zu = zg[upar] + np.sqrt(unit_var) * rng.standard_normal((len(upar), D))
    w = _x_obs(rng, len(upar), n_obs, D, scale=np.sqrt(1.0 / D))
    rate = np.exp(np.einsum("und,ud->un", w.astype(np.float64), zu))
    y = rng.poisson(np.minimum(rate, 1e6)).astype(np.float32)
    root = Level(n=n_inst, dim=D, prior=PRIOR_STD_NORMAL, prior_a=1.0)
    grp = Level(n=len(gpar), dim=D, prior=PRIOR_NORMAL_FIXED_VAR, prior_a=1.0, parent=gpar)
    unit = Level(n=len(upar), dim=D, prior=PRIOR_NORMAL_FIXED_VAR, prior_a=unit_var,
                 lik=LIK_POISSON_LOG, n_obs=n_obs, parent=upar, x=w, y=y)
    return Model([root, grp, unit], name=f"batched_three_level_{n_inst}",
                 truth={"mu": mu, "zg": zg, "zu": zu})


def gamma_poisson(n_inst: int = 4, N: int = 20, a0: float = 2.0, b0: float = 1.0, seed: int = 0) -> Model:
    """lambda ~ Gamma(a0, b0) (rate b0); y_n ~ Poisson(lambda); one latent per instance."""
    rng = np.random.default_rng(seed)
    lam = rng.gamma(a0, 1.0 / b0, size=n_inst)
    y = rng.poisson(lam[:, None], size=(n_inst, N)).astype(np.float32)
    root = Level(n=n_inst, dim=1, prior=PRIOR_GAMMA, prior_a=a0, prior_b=b0,
                 lik=LIK_POISSON_RATE, n_obs=N, qfam=Q_GAMMA,
                 x=np.ones((n_inst, N, 1), np.float32), y=y)
    return Model([root], name="gamma_poisson", truth={"lam": lam})


def beta_bernoulli(n_inst: int = 4, N: int = 20, a0: float = 2.0, b0: float = 3.0, seed: int = 0) -> Model:
    """theta ~ Beta(a0, b0); y_n ~ Bernoulli(theta); one latent per instance."""
    rng = np.random.default_rng(seed)
    th = rng.beta(a0, b0, size=n_inst)
    y = (rng.random((n_inst, N)) < th[:, None]).astype(np.float32)
    root = Level(n=n_inst, dim=1, prior=PRIOR_BETA, prior_a=a0, prior_b=b0,
                 lik=LIK_BERNOULLI_PROB, n_obs=N, qfam=Q_BETA,
                 x=np.ones((n_inst, N, 1), np.float32), y=y)
    return Model([root], name="beta_bernoulli", truth={"theta": th})


def chain_poisson(n_inst: int = 1, R: int = 92, T: int = 109, D: int = 1, seed: int = 0, first_var: float = 0.5,
                  step_var: float = 0.05, n_obs: int = 1, lik: int = LIK_POISSON_LOG, lik_var: float = 1.0) -> Model:
    """Daily random walks under a global latent (the Covid model's chain plate,
    App. F, with Poisson counts in place of its negative binomial):
    g ~ N(0, I_D) per instance; per region c, z_{c,0} ~ N(g, first_var I),
    z_{c,d} ~ N(z_{c,d-1}, step_var I); y_{c,d,n} ~ Poisson(exp(z_{c,d} . x)) with
    x = 1 for D = 1 and x ~ N(0, I/D) otherwise (or Gaussian y, lik = LIK_GAUSS)."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n_inst, D))
    z = np.empty((n_inst, R, T, D))
    z[:, :, 0] = g[:, None, :] + np.sqrt(first_var) * rng.standard_normal((n_inst, R, D))
    for d in range(1, T):
        z[:, :, d] = z[:, :, d - 1] + np.sqrt(step_var) * rng.standard_normal((n_inst, R, D))
    n = n_inst * R * T
    z = z.reshape(n, D)
    if D == 1:
        x = np.ones((n, n_obs, 1), np.float32)
    else:
        x = (rng.standard_normal((n, n_obs, D)) / np.sqrt(D)).astype(np.float32)
    s = np.einsum("end,ed->en", x.astype(np.float64), z)
    if lik == LIK_GAUSS:
        y = (s + np.sqrt(lik_var) * rng.standard_normal(s.shape)).astype(np.float32)
    else:
        y = rng.poisson(np.exp(np.minimum(s, 20.0))).astype(np.float32)
    root = Level(n=n_inst, dim=D, prior=PRIOR_STD_NORMAL, prior_a=1.0)
    days = Level(n=n, dim=D, prior=PRIOR_NORMAL_FIXED_VAR, prior_a=first_var, prior_b=step_var, lik=lik,
                 lik_var=lik_var, n_obs=n_obs, parent=np.repeat(np.arange(n_inst, dtype=np.int64), R * T),
                 x=x, y=y, chain=T)
    return Model([root, days], name=f"chain_poisson_R{R}_T{T}", truth={"g": g, "z": z})


def subset(model: Model, inst_ids) -> tuple:
    """The sub-model of the instances inst_ids (roots), with every descendant.

    Returns (sub_model, keep) where keep[l] holds, in order, the indices in the
    full model of the elements of level l that the sub-model keeps (so per-
    element arrays of the full model are sliced with keep[l]).
    """
    keep = [np.unique(np.asarray(inst_ids, np.int64))]
    levels = [Level(**{**model.levels[0].__dict__, "n": len(keep[0]),
                       "x": None if model.levels[0].x is None else model.levels[0].x[keep[0]],
                       "y": None if model.levels[0].y is None else model.levels[0].y[keep[0]]})]
    for lv in model.levels[1:]:
        prev = keep[-1]
        sel = np.nonzero(np.isin(lv.parent, prev))[0].astype(np.int64)
        pos = np.searchsorted(prev, lv.parent[sel]).astype(np.int64)
        keep.append(sel)
        levels.append(Level(**{**lv.__dict__, "n": len(sel), "parent": pos,
                               "x": None if lv.x is None else lv.x[sel],
                               "y": None if lv.y is None else lv.y[sel]}))
    return Model(levels, name=f"{model.name}_subset{len(keep[0])}"), keep


def initial_q(model: Model) -> list:
    """Initial proposal of App. F: N(0, I) for Gaussian latents; the prior otherwise.

    Returns one float32 array [n, 2, dim] per level (parameter pair per dim).
    """
    out = []
    for lv in model.levels:
        q = np.empty((lv.n, 2, lv.dim), np.float32)
        if lv.qfam == Q_GAUSS:
            q[:, 0, :] = 0.0
            q[:, 1, :] = 1.0
        else:
            q[:, 0, :] = lv.prior_a
            q[:, 1, :] = lv.prior_b
        out.append(q)
    return out


def random_q(model: Model, seed: int, loc_scale: float = 0.5, sd_lo: float = 0.3, sd_hi: float = 1.2) -> list:
    """A seeded, non-trivial Gaussian proposal (for parity cases away from q0)."""
    rng = np.random.default_rng(seed)
    out = []
    for lv in model.levels:
        q = np.empty((lv.n, 2, lv.dim), np.float32)
        q[:, 0, :] = loc_scale * rng.standard_normal((lv.n, lv.dim))
        q[:, 1, :] = rng.uniform(sd_lo, sd_hi, size=(lv.n, lv.dim))
        out.append(q)
    return out


def noise(model: Model, K: int, seed: int) -> list:
    """Supplied noise, one float32 array [n, K, noise_per_sample] per level.

    Gaussian levels take N(0,1) draws.  Gamma/Beta levels take, per dimension
    and per Gamma variate, GAMMA_TRIES (normal, uniform) pairs followed by one
    extra uniform (the Marsaglia-Tsang attempts and the shape<1 boost).
    """
    rng = np.random.default_rng(seed)
    out = []
    for lv in model.levels:
        if lv.qfam == Q_GAUSS:
            out.append(rng.standard_normal((lv.n, K, lv.dim), dtype=np.float32))
            continue
        nvar = 1 if lv.qfam == Q_GAMMA else 2
        blk = 2 * GAMMA_TRIES + 1
        e = np.empty((lv.n, K, lv.dim * nvar, blk), np.float32)
        e[..., 0:2 * GAMMA_TRIES:2] = rng.standard_normal(e[..., 0:2 * GAMMA_TRIES:2].shape)
        e[..., 1:2 * GAMMA_TRIES:2] = rng.uniform(1e-7, 1.0, e[..., 1:2 * GAMMA_TRIES:2].shape)
        e[..., -1] = rng.uniform(1e-7, 1.0, e[..., -1].shape)
        out.append(e.reshape(lv.n, K, lv.dim * nvar * blk))
    return out


def flat(arrays: list) -> np.ndarray:
    """Concatenate per-level arrays into the flat level-major buffer the ABI takes."""
    return np.concatenate([np.ascontiguousarray(a).reshape(-1) for a in arrays])


def split(buf: np.ndarray, model: Model, per_elt) -> list:
    """Inverse of ``flat``: per_elt(level) gives the element count of one element."""
    out, off = [], 0
    for lv in model.levels:
        sz = lv.n * per_elt(lv)
        out.append(buf[off:off + sz])
        off += sz
    return out
