"""Literal MPIW by enumeration of every index vector k in {1..K}^n.

TEST INFRASTRUCTURE ONLY.  This is Eq. (mp_iw) of the paper written out with
no factorisation at all: for one model instance with n latents (every plate
element of every level is its own latent with its own index k_i),

    log r_k  = sum_i [ log p(z_i^{k_i} | z_pa(i)^{k_pa(i)}) + log p(x_i | z_i^{k_i})
                       - log q_i(z_i^{k_i}) ]                          (Eq. rmp)
    P_MP     = K^-n sum_k r_k                                          (Eq. Prmp)
    w_i[k]   = sum_{k : k_i = k} r_k / sum_k r_k                       (Eq. mmp, m = 1[k_i = k])
    m_i      = sum_k w_i[k] T(z_i^k)

All densities come from scipy.stats / scipy.special (library routines that
share nothing with either the oracle in C or the CUDA path).  Only feasible
for n log2 K up to ~20.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
from scipy import special, stats

Q_GAUSS, Q_GAMMA, Q_BETA = 0, 1, 2


def _log_prior(lv, z, zp):
    if lv.prior == 0:
        return stats.norm.logpdf(z, 0.0, math.sqrt(lv.prior_a)).sum()
    if lv.prior == 1:
        return stats.norm.logpdf(z, zp, math.sqrt(lv.prior_a)).sum()
    if lv.prior == 2:
        D = lv.dim
        return stats.norm.logpdf(z, zp[:D], np.exp(0.5 * zp[D:])).sum()
    if lv.prior == 3:
        return stats.gamma.logpdf(z, lv.prior_a, scale=1.0 / lv.prior_b).sum()
    return stats.beta.logpdf(z, lv.prior_a, lv.prior_b).sum()


def _log_lik(lv, e, z):
    if lv.lik == 0:
        return 0.0
    x = np.asarray(lv.x[e], np.float64)
    y = np.asarray(lv.y[e], np.float64)
    s = x @ z
    if lv.lik == 1:
        return stats.norm.logpdf(y, s, math.sqrt(lv.lik_var)).sum()
    if lv.lik == 2:
        return (y * special.log_expit(s) + (1 - y) * special.log_expit(-s)).sum()
    if lv.lik == 3:
        return stats.poisson.logpmf(y, np.exp(s)).sum()
    if lv.lik == 4:
        return stats.poisson.logpmf(y, z[0]).sum()
    return stats.bernoulli.logpmf(y, z[0]).sum()


def _log_q(lv, qe, z):
    a, b = np.asarray(qe[0], np.float64), np.asarray(qe[1], np.float64)
    if lv.qfam == Q_GAUSS:
        return stats.norm.logpdf(z, a, b).sum()
    if lv.qfam == Q_GAMMA:
        return stats.gamma.logpdf(z, a, scale=1.0 / b).sum()
    return stats.beta.logpdf(z, a, b).sum()


def _T(lv, z):
    if lv.qfam == Q_GAUSS:
        return np.stack([z, z * z])
    if lv.qfam == Q_GAMMA:
        return np.stack([z, np.log(z)])
    return np.stack([np.log(z), np.log1p(-z)])


def instance_latents(model, inst: int):
    """(level, element) of every latent of one instance, parents before children."""
    lat = [(0, inst)]
    frontier = [inst]
    for l in range(1, len(model.levels)):
        par = model.levels[l].parent
        nxt = [int(e) for e in np.nonzero(np.isin(par, frontier))[0]]
        lat += [(l, e) for e in nxt]
        frontier = nxt
    return lat


def estep_instance(model, q, z, K: int, inst: int = 0) -> dict:
    """Enumerate all K^n index vectors of one instance.

    q: per level [n, 2, dim] proposal parameters; z: per level [n, K, dim]
    samples (the draws themselves, so the check does not depend on how they
    were produced).  Returns log_pmp, and w / mom keyed by (level, element).
    """
    lat = instance_latents(model, inst)
    idx = {le: i for i, le in enumerate(lat)}
    n = len(lat)
    unary = np.zeros((n, K))
    pair = {}
    for i, (l, e) in enumerate(lat):
        lv = model.levels[l]
        for k in range(K):
            zk = np.asarray(z[l][e, k], np.float64)
            u = _log_lik(lv, e, zk) - _log_q(lv, q[l][e], zk)
            if l == 0:
                u += _log_prior(lv, zk, None)
            unary[i, k] = u
        if l > 0:
            p = int(lv.parent[e])
            pi = idx[(l - 1, p)]
            f = np.zeros((K, K))
            for kp in range(K):
                zp = np.asarray(z[l - 1][p, kp], np.float64)
                for k in range(K):
                    f[kp, k] = _log_prior(lv, np.asarray(z[l][e, k], np.float64), zp)
            pair[i] = (pi, f)
    logr = []
    combos = list(itertools.product(range(K), repeat=n))
    for kv in combos:
        s = sum(unary[i, kv[i]] for i in range(n))
        s += sum(f[kv[pi], kv[i]] for i, (pi, f) in pair.items())
        logr.append(s)
    logr = np.array(logr)
    mx = logr.max()
    terms = np.exp(logr - mx)
    tot = math.fsum(terms)
    log_pmp = mx + math.log(tot) - n * math.log(K)
    combos = np.array(combos)
    w, mom = {}, {}
    for i, (l, e) in enumerate(lat):
        wi = np.array([math.fsum(terms[combos[:, i] == k]) for k in range(K)]) / tot
        w[(l, e)] = wi
        lv = model.levels[l]
        T = _T(lv, np.asarray(z[l][e], np.float64))      # [2, K, dim]
        mom[(l, e)] = np.einsum("k,skd->sd", wi, T)
    return {"log_pmp": log_pmp, "w": w, "mom": mom, "n": n}


def estep_instance_split_root(model, q, z, K: int, inst: int = 0) -> dict:
    """Enumeration for a two-level model whose root halves are separate latents.

    The root sample rows z[0][inst, k] = (mu^k, psi^k) are read as two latents,
    mu (dimensions [0, D)) and psi ([D, 2D)), each with its own index, so the
    index vector is (k_mu, k_psi, k_1, ..., k_M) and a user's prior factor
    N(z_m; mu^{k_mu}, diag exp(psi^{k_psi})) takes both parent indices.  The
    root prior N(0, v I) and the proposal are products over dimensions, so
    each half keeps its own part of them.  Returns log_pmp, w_mu, w_psi,
    w / mom of the users keyed by element, n.
    """
    r, u = model.levels
    D = u.dim
    q0 = np.asarray(q[0][inst], np.float64)
    users = [int(e) for e in np.nonzero(np.asarray(u.parent) == inst)[0]]
    n = 2 + len(users)
    mu = np.asarray(z[0][inst][:, :D], np.float64)
    psi = np.asarray(z[0][inst][:, D:], np.float64)
    sd0 = math.sqrt(r.prior_a)
    un_mu = np.array([stats.norm.logpdf(mu[k], 0.0, sd0).sum() - stats.norm.logpdf(mu[k], q0[0, :D], q0[1, :D]).sum()
                      for k in range(K)])
    un_psi = np.array([stats.norm.logpdf(psi[k], 0.0, sd0).sum()
                       - stats.norm.logpdf(psi[k], q0[0, D:], q0[1, D:]).sum() for k in range(K)])
    un_u, pair = [], []
    for e in users:
        ze = np.asarray(z[1][e], np.float64)
        un_u.append(np.array([_log_lik(u, e, ze[k]) - _log_q(u, q[1][e], ze[k]) for k in range(K)]))
        f = np.zeros((K, K, K))
        for a in range(K):
            for b in range(K):
                zp = np.concatenate([mu[a], psi[b]])
                for k in range(K):
                    f[a, b, k] = _log_prior(u, ze[k], zp)
        pair.append(f)
    combos = np.array(list(itertools.product(range(K), repeat=n)))
    logr = un_mu[combos[:, 0]] + un_psi[combos[:, 1]]
    for j in range(len(users)):
        logr = logr + un_u[j][combos[:, 2 + j]] + pair[j][combos[:, 0], combos[:, 1], combos[:, 2 + j]]
    mx = logr.max()
    terms = np.exp(logr - mx)
    tot = math.fsum(terms)
    out = {"log_pmp": mx + math.log(tot) - n * math.log(K), "n": n, "w": {}, "mom": {}}
    marg = [np.array([math.fsum(terms[combos[:, i] == k]) for k in range(K)]) / tot for i in range(n)]
    out["w_mu"], out["w_psi"] = marg[0], marg[1]
    for j, e in enumerate(users):
        ze = np.asarray(z[1][e], np.float64)
        out["w"][e] = marg[2 + j]
        out["mom"][e] = np.stack([marg[2 + j] @ ze, marg[2 + j] @ ze ** 2])
    return out


def estep_instance_chain(model, q, z, K: int, inst: int = 0) -> dict:
    """Enumeration for a two-level model whose leaf level is a chain plate.

    Latents: the instance's root and every (region, day) element of its
    chains (element c T + d), each with its own index.  The first day of a
    region takes the level's prior given the root sample; day d >= 1 takes
    N(z_{c,d-1}, prior_b I).  Returns log_pmp, w / mom keyed by (level,
    element), n.
    """
    r, u = model.levels
    T = int(u.chain)
    elems = [int(e) for e in np.nonzero(np.asarray(u.parent) == inst)[0]]
    lat = [(0, inst)] + [(1, e) for e in elems]
    idx = {le: i for i, le in enumerate(lat)}
    n = len(lat)
    unary = np.zeros((n, K))
    pair = {}
    for i, (l, e) in enumerate(lat):
        lv = model.levels[l]
        for k in range(K):
            zk = np.asarray(z[l][e, k], np.float64)
            unary[i, k] = _log_lik(lv, e, zk) - _log_q(lv, q[l][e], zk) + (_log_prior(lv, zk, None) if l == 0 else 0.0)
        if l == 1:
            first = e % T == 0
            pi = idx[(0, inst)] if first else idx[(1, e - 1)]
            f = np.zeros((K, K))
            for kp in range(K):
                zp = np.asarray(z[0][inst, kp] if first else z[1][e - 1, kp], np.float64)
                for k in range(K):
                    zk = np.asarray(z[1][e, k], np.float64)
                    f[kp, k] = (_log_prior(u, zk, zp) if first
                                else stats.norm.logpdf(zk, zp, math.sqrt(u.prior_b)).sum())
            pair[i] = (pi, f)
    combos = np.array(list(itertools.product(range(K), repeat=n)))
    logr = np.zeros(len(combos))
    for i in range(n):
        logr += unary[i][combos[:, i]]
    for i, (pi, f) in pair.items():
        logr += f[combos[:, pi], combos[:, i]]
    mx = logr.max()
    terms = np.exp(logr - mx)
    tot = math.fsum(terms)
    w, mom = {}, {}
    for i, (l, e) in enumerate(lat):
        wi = np.array([math.fsum(terms[combos[:, i] == k]) for k in range(K)]) / tot
        w[(l, e)] = wi
        ze = np.asarray(z[l][e], np.float64)
        mom[(l, e)] = np.stack([wi @ ze, wi @ ze ** 2])
    return {"log_pmp": mx + math.log(tot) - n * math.log(K), "w": w, "mom": mom, "n": n}


def estep_instance_conditional(model, q, z, perm, K: int, inst: int = 0) -> dict:
    """Enumeration for a two-level model whose children use the parent-
    conditioned proposal N(z_p^{s(k)}[:D] + loc, diag scale^2) with the
    permutation copy scheme: copy k of child i was drawn from parent copy
    perm[i][k], so Eq. rmp's proposal term of copy k is that density.
    Returns log_pmp, w / mom ((E z, E z^2)) keyed by (level, element), the
    pairwise moment cross[e] = E[z_e z_parent[:D]], n.
    """
    r, u = model.levels
    D = u.dim
    users = [int(e) for e in np.nonzero(np.asarray(u.parent) == inst)[0]]
    lat = [(0, inst)] + [(1, e) for e in users]
    n = len(lat)
    z0 = np.asarray(z[0][inst], np.float64)
    unary = np.zeros((n, K))
    for k in range(K):
        unary[0, k] = _log_prior(r, z0[k], None) - _log_q(r, q[0][inst], z0[k])
    pair = []
    for i, e in enumerate(users, start=1):
        ze = np.asarray(z[1][e], np.float64)
        loc, sc = np.asarray(q[1][e][0], np.float64), np.asarray(q[1][e][1], np.float64)
        for k in range(K):
            mean = z0[int(perm[e][k])][:D] + loc
            unary[i, k] = _log_lik(u, e, ze[k]) - stats.norm.logpdf(ze[k], mean, sc).sum()
        f = np.array([[_log_prior(u, ze[k], z0[kp]) for k in range(K)] for kp in range(K)])
        pair.append(f)
    combos = np.array(list(itertools.product(range(K), repeat=n)))
    logr = np.zeros(len(combos))
    for i in range(n):
        logr += unary[i][combos[:, i]]
    for i, f in enumerate(pair, start=1):
        logr += f[combos[:, 0], combos[:, i]]
    mx = logr.max()
    terms = np.exp(logr - mx)
    tot = math.fsum(terms)
    out = {"log_pmp": mx + math.log(tot) - n * math.log(K), "n": n, "w": {}, "mom": {}, "cross": {}}
    for i, (l, e) in enumerate(lat):
        wi = np.array([math.fsum(terms[combos[:, i] == k]) for k in range(K)]) / tot
        ze = np.asarray(z[l][e], np.float64)
        out["w"][(l, e)] = wi
        out["mom"][(l, e)] = np.stack([wi @ ze, wi @ ze ** 2])
        if l == 1:
            prod = ze[combos[:, i]] * z0[combos[:, 0]][:, :D]            # [combos, D]
            out["cross"][e] = np.array([math.fsum(terms * prod[:, d]) for d in range(D)]) / tot
    return out
