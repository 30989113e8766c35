"""ctypes front-end of the FP64 CPU oracle (``qem_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, the package smoke check and the
benchmark's CPU-baseline leg are the only callers.  Nothing here imports the
CUDA package; models are read duck-typed (``levels[l].n``, ``.dim``, ...), so
the oracle depends on no code of the path it checks.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qem_oracle.c")
_LIB = os.path.join(_HERE, "libqem_oracle.so")

Q_GAUSS, Q_GAMMA, Q_BETA = 0, 1, 2
GAMMA_TRIES = 8


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: it also builds on the Arm host)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Level(C.Structure):
    _fields_ = [("n", C.c_int64), ("dim", C.c_int), ("prior", C.c_int),
                ("prior_a", C.c_double), ("prior_b", C.c_double),
                ("lik", C.c_int), ("lik_var", C.c_double), ("n_obs", C.c_int), ("qfam", C.c_int),
                ("parent", C.c_void_p), ("x", C.c_void_p), ("y", C.c_void_p), ("q", C.c_void_p),
                ("eps", C.c_void_p), ("z", C.c_void_p), ("w", C.c_void_p), ("mom", C.c_void_p),
                ("logL", C.c_void_p), ("H_extra", C.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_estep.restype = C.c_int
        _lib.orc_estep.argtypes = [C.c_int, C.POINTER(_Level), C.c_int, C.c_uint64, C.c_uint64, C.c_void_p]
        _lib.orc_digamma.restype = C.c_double
        _lib.orc_digamma.argtypes = [C.c_double]
        _lib.orc_trigamma.restype = C.c_double
        _lib.orc_trigamma.argtypes = [C.c_double]
        _lib.orc_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.orc_draw_noise_at.argtypes = [C.c_uint64, C.c_uint64, C.c_int, C.c_void_p, C.c_int64, C.c_int,
                                           C.c_int, C.c_int, C.c_void_p]
        _lib.orc_draw_noise.argtypes = [C.c_uint64, C.c_uint64, C.c_int, C.c_int64, C.c_int, C.c_int,
                                        C.c_int, C.c_void_p]
        for nm in ("orc_mstep_gamma", "orc_mstep_beta"):
            getattr(_lib, nm).argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_void_p]
        _lib.orc_mstep_gauss.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_double, C.c_void_p]
        _lib.orc_ema.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_double]
        _lib.orc_max_threads.restype = C.c_int
    return _lib


def _p(a):
    return a.ctypes.data if a is not None else None


def noise_per_sample(lv) -> int:
    if lv.qfam == Q_GAUSS:
        return lv.dim
    return lv.dim * (1 if lv.qfam == Q_GAMMA else 2) * (2 * GAMMA_TRIES + 1)


def estep(model, q, K: int, eps=None, seed: int = 0, it: int = 0, root_extra=None) -> dict:
    """One MPIW E-step in FP64.

    q:   per level, array [n, 2, dim] of proposal parameters
    eps: per level, array [n, K, noise_per_sample] of supplied noise, or None
         to draw it from the counter-based stream (seed, it)
    root_extra: [n_inst, K] or None; added to the root's sum over its children
         (the plate sums of children the model does not hold: a sharded plate)
    Returns log_pmp [n_inst] and per level z, w (marginal weights), mom
    (E_w[T(z)], [n, 2, dim]) and logL (levels > 0: [n, K_parent]).
    """
    L = len(model.levels)
    keep = []
    arr = (_Level * L)()
    out = {"z": [], "w": [], "mom": [], "logL": []}
    for l, lv in enumerate(model.levels):
        c = arr[l]
        c.n, c.dim, c.prior = lv.n, lv.dim, lv.prior
        c.prior_a, c.prior_b = float(lv.prior_a), float(lv.prior_b)
        c.lik, c.lik_var, c.n_obs, c.qfam = lv.lik, float(lv.lik_var), lv.n_obs, lv.qfam
        par = None if lv.parent is None else np.ascontiguousarray(lv.parent, np.int64)
        x = None if lv.x is None else np.ascontiguousarray(lv.x, np.float64)
        y = None if lv.y is None else np.ascontiguousarray(lv.y, np.float64)
        qq = np.ascontiguousarray(q[l], np.float64).reshape(lv.n, 2, lv.dim)
        ee = None if eps is None else np.ascontiguousarray(eps[l], np.float64).reshape(lv.n, K, -1)
        z = np.zeros((lv.n, K, lv.dim))
        w = np.zeros((lv.n, K))
        mom = np.zeros((lv.n, 2, lv.dim))
        logL = np.zeros((lv.n, K))
        keep += [par, x, y, qq, ee]
        c.parent, c.x, c.y, c.q, c.eps = _p(par), _p(x), _p(y), _p(qq), _p(ee)
        c.z, c.w, c.mom, c.logL = _p(z), _p(w), _p(mom), _p(logL)
        out["z"].append(z); out["w"].append(w); out["mom"].append(mom); out["logL"].append(logL)
    if root_extra is not None:
        hx = np.ascontiguousarray(root_extra, np.float64).reshape(model.levels[0].n, K)
        keep.append(hx)
        arr[0].H_extra = _p(hx)
    lp = np.zeros(model.levels[0].n)
    rc = lib().orc_estep(L, arr, K, seed, it, _p(lp))
    if rc != 0:
        raise ValueError(f"oracle estep failed ({rc})")
    out["log_pmp"] = lp
    return out


def mstep(qfam: int, m: np.ndarray, var_floor: float = 1e-10) -> np.ndarray:
    """Mean parameters [n, 2, D] -> proposal parameters [n, 2, D] (FP64)."""
    m = np.ascontiguousarray(m, np.float64)
    n, _, D = m.shape
    out = np.zeros_like(m)
    if qfam == Q_GAUSS:
        lib().orc_mstep_gauss(_p(m), n, D, var_floor, _p(out))
    elif qfam == Q_GAMMA:
        lib().orc_mstep_gamma(_p(m), n, D, _p(out))
    else:
        lib().orc_mstep_beta(_p(m), n, D, _p(out))
    return out


def ema(m: np.ndarray, m_hat: np.ndarray, lam: float) -> np.ndarray:
    m = np.ascontiguousarray(m, np.float64).copy()
    mh = np.ascontiguousarray(m_hat, np.float64)
    lib().orc_ema(_p(m), _p(mh), m.size, lam)
    return m


def digamma(x: float) -> float:
    return lib().orc_digamma(x)


def trigamma(x: float) -> float:
    return lib().orc_trigamma(x)


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, np.uint32).copy()
    k = np.asarray(key, np.uint32).copy()
    o = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def draw_noise(seed: int, it: int, level: int, n: int, K: int, nps: int, qfam: int = Q_GAUSS) -> np.ndarray:
    out = np.zeros((n, K, nps))
    lib().orc_draw_noise(seed, it, level, n, K, nps, qfam, _p(out))
    return out


def draw_noise_at(seed: int, it: int, level: int, idx, K: int, nps: int, qfam: int = Q_GAUSS) -> np.ndarray:
    """draw_noise for the elements idx of a level (their indices in the full model)."""
    idx = np.ascontiguousarray(idx, np.int64)
    out = np.zeros((len(idx), K, nps))
    lib().orc_draw_noise_at(seed, it, level, _p(idx), len(idx), K, nps, qfam, _p(out))
    return out


def max_threads() -> int:
    return lib().orc_max_threads()


def predictive(z: np.ndarray, w: np.ndarray, lik: int, x_new, y_new, lik_var: float = 1.0) -> np.ndarray:
    """Predictive log-likelihood of held-out data from weighted samples (FP64):

        out[e] = log sum_k w[e, k] prod_n p(y_new[e, n] | z[e, k], x_new[e, n])

    z [n, K, D], w [n, K] (each row summing to one), x_new [n, N, D] (unused by
    the Poisson-rate and Bernoulli-probability likelihoods), y_new [n, N].
    Densities from scipy (library routines independent of the C oracle).
    """
    from scipy import special, stats
    z = np.asarray(z, np.float64)
    w = np.asarray(w, np.float64)
    y = np.asarray(y_new, np.float64)
    if lik in (4, 5):                       # Poisson-rate, Bernoulli-probability: z is the parameter
        zz = z[:, :, 0][:, :, None]
        if lik == 4:
            ll = stats.poisson.logpmf(y[:, None, :], zz).sum(-1)
        else:
            ll = (y[:, None, :] * np.log(zz) + (1 - y[:, None, :]) * np.log1p(-zz)).sum(-1)
    else:
        s = np.einsum("ekd,end->ekn", z, np.asarray(x_new, np.float64))
        yy = y[:, None, :]
        if lik == 1:                        # Gaussian
            ll = stats.norm.logpdf(yy, s, np.sqrt(lik_var)).sum(-1)
        elif lik == 2:                      # Bernoulli-logit
            ll = (yy * special.log_expit(s) + (1 - yy) * special.log_expit(-s)).sum(-1)
        elif lik == 3:                      # Poisson-log
            ll = stats.poisson.logpmf(yy, np.exp(s)).sum(-1)
        else:
            raise ValueError("no likelihood")
    return special.logsumexp(ll, b=w, axis=1)
