"""Learned scheduler: plain-miner traces -> an 8-64-64-2 bf16 MLP trained on
the GPU by libfim's own forward / backward / Adam kernels -> FIM_LEARNED.

Trace row of a prefix class (written by the DFS kernel under FIM_TRACE):
  features  |Y|/16, log2(1+S(Y))/32, S(Y)/n, log2(1+k)/16, S(Y)/S(X),
            mean_e S(X u e)/S(X), log2(1+nw)/32, minsup/S(Y)
            (each O(1) by construction, so the bf16 input rounding of the
            kernel's inference is harmless and no standardisation is needed)
  targets   log2(1 + candidate words ANDed in Y's subtree),
            1 if counting Y through its diffset touches fewer 32-byte sectors
The network only orders root classes (longest predicted subtree first) and
picks each class's representation; it never changes a support.  Training is
mixed precision: float32 master weights and Adam, bf16 forward/backward (the
precision the DFS kernel infers in).
"""
from __future__ import annotations

import numpy as np

from . import datagen, fim


def collect_traces(ctx, csr, minsup: int, flags: int = 0):
    """Mine with FIM_TRACE (plain schedule) and return (features, targets)."""
    fim.fim_build_bitmaps(ctx, csr.indptr, csr.indices, csr.m)
    fim.fim_mine(ctx, minsup, flags | fim.FIM_TRACE)
    return fim.fim_fetch_traces(ctx)


def train(ctx, x: np.ndarray, t: np.ndarray, steps: int = 2000, lr: float = 1e-3, batch: int = 4096,
          seed: int = 0, init: np.ndarray | None = None, bf16: bool = True):
    """Adam on mean loss over contiguous mini-batches of a seeded shuffle.
    Returns (weights float32 [4866], per-step loss list)."""
    import torch
    n = x.shape[0]
    if n == 0:
        raise ValueError("no training rows")
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    dx = torch.from_numpy(np.ascontiguousarray(x[perm], np.float32)).cuda()
    dt = torch.from_numpy(np.ascontiguousarray(t[perm], np.float32)).cuda()
    w0 = (init if init is not None else datagen.mlp_init_weights(seed)).astype(np.float32)
    dp = torch.from_numpy(w0.copy()).cuda()
    dm = torch.zeros_like(dp)
    dv = torch.zeros_like(dp)
    dg = torch.zeros_like(dp)
    B = min(batch, n)
    dy = torch.empty((B, 2), dtype=torch.float32, device="cuda")
    dc = torch.empty((B, 256), dtype=torch.float32, device="cuda")
    hist = []
    nb = max(1, n // B)
    for step in range(1, steps + 1):
        s0 = ((step - 1) % nb) * B
        xb, tb = dx[s0:s0 + B], dt[s0:s0 + B]
        fim.fim_mlp_forward(ctx, dp, xb, dy, dc, bf16=bf16)
        hist.append(fim.fim_mlp_backward(ctx, dp, xb, dy, tb, dc, dg, bf16=bf16))
        fim.fim_mlp_adam(ctx, dp, dg, dm, dv, step, lr)
    torch.cuda.synchronize()
    return dp.cpu().numpy(), hist


def fit(ctx, x: np.ndarray, t: np.ndarray, steps: int = 3000, lr: float = 2e-3, seed: int = 0):
    """Train on the kernel's features as written: weights for FIM_LEARNED."""
    return train(ctx, x, t, steps=steps, lr=lr, seed=seed)


def predict(ctx, w: np.ndarray, x: np.ndarray, bf16: bool = True) -> np.ndarray:
    """MLP outputs [n, 2] on the GPU (the inference arithmetic)."""
    import torch
    dp = torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda()
    dx = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
    dy = torch.empty((x.shape[0], 2), dtype=torch.float32, device="cuda")
    fim.fim_mlp_forward(ctx, dp, dx, dy, None, bf16=bf16)
    torch.cuda.synchronize()
    return dy.cpu().numpy()


def evaluate(ctx, w: np.ndarray, x: np.ndarray, t: np.ndarray) -> dict:
    """Prediction error against the plain miner's measured traces."""
    y = predict(ctx, w, x)
    resid = y[:, 0] - t[:, 0]
    var = float(np.var(t[:, 0])) or 1.0
    return {"work_mse": float(np.mean(resid ** 2)), "work_r2": 1.0 - float(np.mean(resid ** 2)) / var,
            "repr_accuracy": float(np.mean((y[:, 1] > 0) == (t[:, 1] > 0.5))),
            "rows": int(x.shape[0])}
