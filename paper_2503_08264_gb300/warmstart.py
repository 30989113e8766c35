"""Learned warm start: the proposal network of the qem_mlp_* calls.

Argument marshalling only: features, forward, loss and gradient, Adam and
the proposal parameters all run in libqem's kernels.  Training batches are
contiguous slices of a dataset the caller uploads already shuffled.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L
from . import synth as S


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class WarmStart:
    """Network parameters with their Adam state, on the current CUDA device."""

    D = L.QEM_MLP_DIM
    N_IN = 2 * L.QEM_MLP_DIM + 1
    N_OUT = 2 * L.QEM_MLP_DIM

    def __init__(self, seed: int = 0, params: np.ndarray | None = None):
        p = S.mlp_init(seed) if params is None else np.asarray(params, np.float32)
        assert p.size == L.QEM_MLP_PARAMS
        self.params = torch.as_tensor(p).cuda()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.t = 0
        self._ws = None

    def features(self, x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
        """x [n, N, D], y [n, N] (device) -> features [n, 2D+1]."""
        n, N = y.shape
        f = torch.empty(n, self.N_IN, dtype=torch.float32, device=x.device)
        L.check(L.load().qem_mlp_features(_ptr(x), _ptr(y), n, N, x.shape[-1], _ptr(f), _stream()),
                "qem_mlp_features")
        return f

    def forward(self, feats: torch.Tensor) -> torch.Tensor:
        out = torch.empty(feats.shape[0], self.N_OUT, dtype=torch.float32, device=feats.device)
        L.check(L.load().qem_mlp_forward(_ptr(self.params), _ptr(feats), feats.shape[0], _ptr(out), _stream()),
                "qem_mlp_forward")
        return out

    def predict_q(self, feats: torch.Tensor) -> torch.Tensor:
        """Proposal parameters [n, 2, D] (means, scales) of the users."""
        out = self.forward(feats)
        q = torch.empty(feats.shape[0], 2, self.D, dtype=torch.float32, device=feats.device)
        L.check(L.load().qem_mlp_to_q(_ptr(out), feats.shape[0], _ptr(q), _stream()), "qem_mlp_to_q")
        return q

    def _workspace(self, n: int) -> torch.Tensor:
        nb = C.c_size_t()
        L.check(L.load().qem_mlp_workspace_size(n, C.byref(nb)), "qem_mlp_workspace_size")
        if self._ws is None or self._ws.numel() * 4 < nb.value:
            self._ws = torch.empty((nb.value + 3) // 4, dtype=torch.float32, device="cuda")
        return self._ws

    def loss_grad(self, feats: torch.Tensor, target: torch.Tensor, loss: torch.Tensor | None = None):
        """Gradient (into self.grad) and mean KL (into loss, a device double [1])."""
        n = feats.shape[0]
        L.check(L.load().qem_mlp_backward(_ptr(self.params), _ptr(feats), _ptr(target), n, _ptr(self.grad),
                                          _ptr(loss), _ptr(self._workspace(n)), _stream()), "qem_mlp_backward")
        return self.grad

    def step(self, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        self.t += 1
        L.check(L.load().qem_mlp_step(_ptr(self.params), _ptr(self.grad), _ptr(self.m), _ptr(self.v), self.t, lr,
                                      beta1, beta2, eps, _stream()), "qem_mlp_step")

    def train(self, feats: torch.Tensor, target: torch.Tensor, epochs: int, batch: int = 4096,
              lr: float = 1e-3) -> list:
        """Adam over contiguous batches of (feats, target) [n, 2, D]; returns the
        loss of the last batch of every epoch."""
        n = feats.shape[0]
        loss = torch.zeros(1, dtype=torch.float64, device=feats.device)
        hist = []
        for _ in range(epochs):
            for b0 in range(0, n, batch):
                b1 = min(n, b0 + batch)
                self.loss_grad(feats[b0:b1], target[b0:b1], loss)
                self.step(lr)
            hist.append(float(loss.item()))
        return hist
