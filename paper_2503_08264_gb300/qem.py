"""Python binding of libqem: the C-ABI calls under the same names, taking torch
CUDA tensors, plus a small ``Plan`` owner object.

Argument marshalling only (pointers, sizes, the current stream); every step
of the E-step and M-step runs in the library's kernels.  PyTorch supplies
device memory and streams.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L
from . import synth as S

PREC = {"fp32": L.QEM_PREC_FP32, "bf16": L.QEM_PREC_BF16, "bf16x3": L.QEM_PREC_BF16X3, "tf32": L.QEM_PREC_TF32}


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream_handle(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------------- raw ABI, same names
def qem_plan(desc: L.ModelDesc, opts: L.PlanOpts) -> C.c_void_p:
    h = C.c_void_p()
    L.check(L.load().qem_plan(C.byref(desc), C.byref(opts), C.byref(h)), "qem_plan")
    return h


def qem_plan_destroy(h) -> None:
    L.check(L.load().qem_plan_destroy(h), "qem_plan_destroy")


def qem_estep(h, q_params, eps, seed: int, it: int, moments, log_pmp=None) -> None:
    L.check(L.load().qem_estep(h, _ptr(q_params), _ptr(eps), seed, it, _ptr(moments), _ptr(log_pmp)), "qem_estep")


def qem_estep_split_root(h, q_params, eps, seed: int, it: int, moments, log_pmp=None, root_weights=None) -> None:
    L.check(L.load().qem_estep_split_root(h, _ptr(q_params), _ptr(eps), seed, it, _ptr(moments), _ptr(log_pmp),
                                          _ptr(root_weights)), "qem_estep_split_root")


def qem_mstep(h, moments, mean_params, q_params, lam: float, sched_p: float = 0.0, t: int = 1) -> None:
    L.check(L.load().qem_mstep(h, _ptr(moments), _ptr(mean_params), _ptr(q_params), lam, sched_p, t), "qem_mstep")


def qem_mean_params(h, q_params, mean_params) -> None:
    L.check(L.load().qem_mean_params(h, _ptr(q_params), _ptr(mean_params)), "qem_mean_params")


def qem_log_pmp(h, n_inst: int) -> np.ndarray:
    out = np.zeros(n_inst, np.float64)
    L.check(L.load().qem_log_pmp(h, out.ctypes.data_as(C.c_void_p)), "qem_log_pmp")
    return out


def qem_weights(h, weights) -> None:
    L.check(L.load().qem_weights(h, _ptr(weights)), "qem_weights")


def qem_samples(h, z) -> None:
    L.check(L.load().qem_samples(h, _ptr(z)), "qem_samples")


def qem_tune(h, q_params, flags: int = 0) -> None:
    L.check(L.load().qem_tune(h, _ptr(q_params), flags), "qem_tune")


def qem_tune_get(h) -> dict:
    a = (C.c_int * 5)()
    L.check(L.load().qem_tune_get(h, a), "qem_tune_get")
    return {"sample_threads": a[0], "mom_threads": a[1], "fwd_rows": a[2], "fwd_chunk": a[3], "tc_sched": a[4]}


def qem_run(h, T: int, t0: int, lam: float, sched_p: float, seed: int, mean_params, q_params, moments,
            trace=None) -> None:
    L.check(L.load().qem_run(h, T, t0, lam, sched_p, seed, _ptr(mean_params), _ptr(q_params), _ptr(moments),
                             _ptr(trace)), "qem_run")


def qem_profile_enable(h, on: bool) -> None:
    L.check(L.load().qem_profile_enable(h, 1 if on else 0), "qem_profile_enable")


def qem_profile_read(h, kind: int):
    ms, n = C.c_double(), C.c_int64()
    L.check(L.load().qem_profile_read(h, kind, C.byref(ms), C.byref(n)), "qem_profile_read")
    return ms.value, n.value


def qem_profile_name(kind: int) -> str:
    r = L.load().qem_profile_name(kind)
    return r.decode() if r else None


# ---------------------------------------------------------------------------- owner object
class Plan:
    """A libqem plan for one model: uploads the model's data to the device,
    builds the descriptor and owns the plan handle."""

    def __init__(self, model: S.Model, K: int, precision: str = "fp32", device: str = "cuda",
                 stream: torch.cuda.Stream | None = None, var_floor: float = 0.0, timeout_s: float = 0.0,
                 tile: int = 0):
        self.model = model
        self.K = K
        self.device = torch.device(device)
        self.stream = stream
        self._keep = []
        desc = L.ModelDesc()
        desc.n_levels = len(model.levels)
        for l, lv in enumerate(model.levels):
            d = desc.levels[l]
            d.n, d.dim, d.prior = lv.n, lv.dim, lv.prior
            d.prior_a, d.prior_b = float(lv.prior_a), float(lv.prior_b)
            d.lik, d.lik_var, d.n_obs, d.qfam = lv.lik, float(lv.lik_var), lv.n_obs if lv.lik else 0, lv.qfam
            d.chain = int(getattr(lv, "chain", 1) or 1)
            d.qcond = int(getattr(lv, "qcond", 0) or 0)
            if lv.parent is not None:
                par = np.ascontiguousarray(lv.parent, np.int64)
                self._keep.append(par)
                d.parent = par.ctypes.data
            if lv.lik and lv.n_obs:
                x = torch.as_tensor(np.ascontiguousarray(lv.x, np.float32)).to(self.device)
                y = torch.as_tensor(np.ascontiguousarray(lv.y, np.float32)).to(self.device)
                self._keep += [x, y]
                d.x, d.y = x.data_ptr(), y.data_ptr()
        opts = L.PlanOpts()
        opts.K, opts.precision, opts.tile = K, PREC[precision] if isinstance(precision, str) else precision, tile
        opts.stream = _stream_handle(stream)
        opts.var_floor, opts.timeout_s = var_floor, timeout_s
        torch.cuda.synchronize(self.device)
        self.h = qem_plan(desc, opts)
        q_len, eps_len, w_len, n_inst = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        L.check(L.load().qem_sizes(self.h, C.byref(q_len), C.byref(eps_len), C.byref(w_len), C.byref(n_inst)),
                "qem_sizes")
        self.q_len, self.eps_len, self.w_len, self.n_inst = q_len.value, eps_len.value, w_len.value, n_inst.value
        self.z_len = sum(lv.n * K * lv.dim for lv in model.levels)
        ws = C.c_size_t()
        L.check(L.load().qem_workspace_size(self.h, C.byref(ws)), "qem_workspace_size")
        self.workspace_bytes = ws.value

    # layout helpers -------------------------------------------------------
    def flat(self, arrays, dtype=torch.float32) -> torch.Tensor:
        a = np.concatenate([np.ascontiguousarray(x).reshape(-1) for x in arrays]) if arrays else np.zeros(0)
        return torch.as_tensor(a.astype({torch.float32: np.float32, torch.float64: np.float64}[dtype])).to(self.device)

    def split(self, t: torch.Tensor, per_elt) -> list:
        out, off = [], 0
        a = t.detach().cpu().numpy()
        for lv in self.model.levels:
            sz = lv.n * int(np.prod(per_elt(lv)))
            out.append(a[off:off + sz].reshape((lv.n,) + tuple(per_elt(lv))))
            off += sz
        return out

    def split_q(self, t):
        return self.split(t, lambda lv: (2, lv.dim))

    def split_w(self, t):
        return self.split(t, lambda lv: (self.K,))

    def split_z(self, t):
        return self.split(t, lambda lv: (self.K, lv.dim))

    # calls ----------------------------------------------------------------
    def estep(self, q, eps=None, seed: int = 0, it: int = 0, moments=None, log_pmp=None):
        if moments is None:
            moments = torch.empty(self.q_len, dtype=torch.float64, device=self.device)
        if log_pmp is None:
            log_pmp = torch.empty(self.n_inst, dtype=torch.float64, device=self.device)
        qem_estep(self.h, q, eps, seed, it, moments, log_pmp)
        return moments, log_pmp

    def estep_split_root(self, q, eps=None, seed: int = 0, it: int = 0, moments=None, log_pmp=None,
                         root_weights=None):
        """E-step with the root's mean and log-variance halves as separate latents
        (K^2 parent index pairs); returns (moments, log_pmp, root_weights [n_inst, 2, K])."""
        if moments is None:
            moments = torch.empty(self.q_len, dtype=torch.float64, device=self.device)
        if log_pmp is None:
            log_pmp = torch.empty(self.n_inst, dtype=torch.float64, device=self.device)
        if root_weights is None:
            root_weights = torch.empty((self.n_inst, 2, self.K), dtype=torch.float32, device=self.device)
        qem_estep_split_root(self.h, q, eps, seed, it, moments, log_pmp, root_weights)
        return moments, log_pmp, root_weights

    def set_perm(self, perm=None):
        """Parent-copy permutations of the qcond level (device int32 [n_1, K]) for the
        following E-steps, or None for the counter-based draw."""
        self._perm = None if perm is None else torch.as_tensor(perm, dtype=torch.int32).to(self.device).contiguous()
        L.check(L.load().qem_set_perm(self.h, _ptr(self._perm)), "qem_set_perm")

    def test_expire_wait(self, on: bool = True) -> None:
        """Test hook: make the tensor-core contractions' first wait run out
        (after timeout_s), so that the E-step reports QEM_ERR_TIMEOUT."""
        L.check(L.load().qem_test_expire_wait(self.h, 1 if on else 0), "qem_test_expire_wait")

    def set_elem_base(self, base) -> None:
        """Index of element 0 of each level in the counter-based noise streams
        (a shard passes its first element's index in the whole model)."""
        a = (C.c_int64 * len(self.model.levels))(*[int(b) for b in base])
        L.check(L.load().qem_set_elem_base(self.h, a), "qem_set_elem_base")

    def shard_forward(self, q, eps=None, seed: int = 0, it: int = 0, root_G=None) -> torch.Tensor:
        """Sampling and contraction up to the plate sums into the root; returns
        this shard's G [n_inst, K] (device double) for the caller's sum over shards."""
        if root_G is None:
            root_G = torch.empty((self.n_inst, self.K), dtype=torch.float64, device=self.device)
        L.check(L.load().qem_estep_shard_forward(self.h, _ptr(q), _ptr(eps), seed, it, _ptr(root_G)),
                "qem_estep_shard_forward")
        return root_G

    def shard_finish(self, root_G, moments=None, log_pmp=None):
        """Root step on the summed G, then this shard's adjoint and moments."""
        if moments is None:
            moments = torch.empty(self.q_len, dtype=torch.float64, device=self.device)
        if log_pmp is None:
            log_pmp = torch.empty(self.n_inst, dtype=torch.float64, device=self.device)
        L.check(L.load().qem_estep_shard_finish(self.h, _ptr(root_G), _ptr(moments), _ptr(log_pmp)),
                "qem_estep_shard_finish")
        return moments, log_pmp

    def log_pmp_fresh(self, q, seed: int, it: int, log_pmp=None):
        """log P_MP of q from a fresh draw of the samples (device double [n_inst])."""
        if log_pmp is None:
            log_pmp = torch.empty(self.n_inst, dtype=torch.float64, device=self.device)
        L.check(L.load().qem_log_pmp_fresh(self.h, _ptr(q), seed, it, _ptr(log_pmp)), "qem_log_pmp_fresh")
        return log_pmp

    def predictive(self, level: int, x_new, y_new):
        """Predictive log-likelihood of held-out (x_new [n, N, D], y_new [n, N]) per element."""
        out = torch.empty(self.model.levels[level].n, dtype=torch.float64, device=self.device)
        xd = None if x_new is None else torch.as_tensor(x_new, dtype=torch.float32).to(self.device).contiguous()
        yd = torch.as_tensor(y_new, dtype=torch.float32).to(self.device).contiguous()
        L.check(L.load().qem_predictive(self.h, level, _ptr(xd), _ptr(yd), yd.shape[1], _ptr(out)), "qem_predictive")
        torch.cuda.current_stream().synchronize()
        return out

    def moments_rescale(self, log_pmp_same, log_pmp_fresh, moments):
        L.check(L.load().qem_moments_rescale(self.h, _ptr(log_pmp_same), _ptr(log_pmp_fresh), _ptr(moments)),
                "qem_moments_rescale")
        return moments

    def mstep(self, moments, mean_params, q_params, lam: float, sched_p: float = 0.0, t: int = 1):
        qem_mstep(self.h, moments, mean_params, q_params, lam, sched_p, t)

    def mean_params(self, q):
        m = torch.empty(self.q_len, dtype=torch.float64, device=self.device)
        qem_mean_params(self.h, q, m)
        return m

    def log_pmp(self) -> np.ndarray:
        return qem_log_pmp(self.h, self.n_inst)

    def weights(self) -> torch.Tensor:
        w = torch.empty(self.w_len, dtype=torch.float32, device=self.device)
        qem_weights(self.h, w)
        return w

    def samples(self) -> torch.Tensor:
        z = torch.empty(self.z_len, dtype=torch.float32, device=self.device)
        qem_samples(self.h, z)
        return z

    def run(self, T: int, lam: float, mean_params, q_params, moments=None, sched_p: float = 0.0, seed: int = 0,
            trace=None, t0: int = 1):
        """Iterations t0 .. t0 + T - 1 of Alg. 1 as one graph launch (t0 > 1
        continues a run from its saved mean parameters)."""
        if moments is None:
            moments = torch.empty(self.q_len, dtype=torch.float64, device=self.device)
        qem_run(self.h, T, t0, lam, sched_p, seed, mean_params, q_params, moments, trace)
        return moments

    def run_kernels(self) -> tuple:
        """(kernels per iteration of the qem_run loop, kernels per qem_run call outside it)."""
        a, b = C.c_int64(), C.c_int64()
        L.check(L.load().qem_run_kernels(self.h, C.byref(a), C.byref(b)), "qem_run_kernels")
        return a.value, b.value

    def tune(self, q_params, force: bool = False) -> dict:
        qem_tune(self.h, q_params, L.QEM_TUNE_FORCE if force else 0)
        return qem_tune_get(self.h)

    def tuning(self) -> dict:
        return qem_tune_get(self.h)

    def set_tuning(self, **kw) -> dict:
        """Apply launch shapes (keys of tuning()); unspecified ones keep their value."""
        cur = qem_tune_get(self.h)
        cur.update(kw)
        keys = ["sample_threads", "mom_threads", "fwd_rows", "fwd_chunk", "tc_sched"]
        a = (C.c_int * 5)(*[int(cur[k]) for k in keys])
        L.check(L.load().qem_tune_set(self.h, a), "qem_tune_set")
        return qem_tune_get(self.h)

    def adjoint_pairs(self) -> tuple:
        """(kept pairs on the tensor-core adjoint, all kept pairs) of the last E-step."""
        a, b = C.c_double(), C.c_double()
        L.check(L.load().qem_adjoint_pairs(self.h, C.byref(a), C.byref(b)), "qem_adjoint_pairs")
        return a.value, b.value

    def profile(self, on: bool = True) -> None:
        qem_profile_enable(self.h, on)

    def profile_read(self) -> dict:
        """{kernel class: (total ms, launches)} since profiling was enabled."""
        return {L.QEM_K_NAMES[k]: qem_profile_read(self.h, k) for k in range(len(L.QEM_K_NAMES))}

    def close(self):
        if getattr(self, "h", None):
            qem_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
