"""Learned initial guess of the forward solves: data generation with the
library's own forward solver, training and inference of the BF16 U-Net
(libqpat.so: qpat_unet_*), and the guessed solve.  Every numerical step runs
in the library's kernels; this module only sequences the calls.

Grids: Kuhn cubes with n nodes per side (n a multiple of 16), whose node
index is the voxel index of the network (the identity resampling)."""
from __future__ import annotations

import numpy as np

from . import qpat as Q


def grid_h(cfg) -> float:
    return cfg.L / (cfg.n - 1)


def sample(mesh, cfg, kappa, mu, flux, params=None):
    """Features (K, N, 3) float32 and forward solutions (K, N) float32 of one
    phantom, from the library's forward solve."""
    import torch
    dev = torch.device("cuda")
    k = torch.as_tensor(np.ascontiguousarray(kappa), device=dev)
    m = torch.as_tensor(np.ascontiguousarray(mu), device=dev)
    f = torch.as_tensor(np.ascontiguousarray(flux), device=dev)
    K, N = flux.shape[0], mesh.N
    phi = torch.empty((K, N), dtype=torch.float64, device=dev)
    h = torch.empty_like(phi)
    Q.qpat_forward_dev(mesh, k, m, f, phi, h, params or Q.qpat_default_params(precision=1, fp32_operator=1))
    x = torch.empty((K, N, 3), dtype=torch.float32, device=dev)
    Q.qpat_unet_features_dev(mesh, k, m, f, grid_h(cfg), x)
    return x, phi.float()


def train(unet: Q.UNet, X, T, steps: int, lr: float = 2e-3, batch: int = 4, seed: int = 0):
    """Adam steps on random mini-batches of (X, T) (tensors (S, N, 3), (S, N));
    returns the loss history."""
    import torch
    rng = np.random.default_rng(seed)
    S = X.shape[0]
    losses = []
    for it in range(steps):
        idx = torch.as_tensor(rng.choice(S, size=min(batch, S), replace=False), device=X.device)
        xb = X.index_select(0, idx).contiguous()
        tb = T.index_select(0, idx).contiguous()
        step_lr = lr * (0.5 * (1 + np.cos(np.pi * it / max(steps, 1))) * 0.9 + 0.1)
        losses.append(unet.train_step(xb, tb, step_lr))
    return losses


def guess(unet: Q.UNet, x):
    """Predicted fluence (K, N) float64 for features x (K, N, 3)."""
    import torch
    y = torch.empty(x.shape[:2], dtype=torch.float32, device=x.device)
    unet.predict(x.contiguous(), y)
    out = torch.empty(y.shape, dtype=torch.float64, device=x.device)
    Q.qpat_unet_to_double_dev(y, out)
    return out
