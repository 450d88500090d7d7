"""Learned initial guess for the SMM iteration: features, targets and the
training / inference loop around the library's network (smm_guess_*).

The network maps per-element fields (log sigma_t, scattering ratio, source)
to the nodal scalar flux of the converged SMM solution.
All network arithmetic runs in libsmm.so; this module only arranges arrays
(element grid <-> channels) and normalizes them.  Its proposal enters
smm_iterate as the initial varphi with options.guess_check set, so a
harmful proposal falls back to the zero guess and the converged answer is
unchanged.
"""
from __future__ import annotations

import numpy as np


def features(sigma_t, sigma_s, q_elem, nx):
    """[3][nx][nx] float32: log sigma_t, scattering ratio, source."""
    f = np.stack([np.log(sigma_t), sigma_s / sigma_t, q_elem]).astype(np.float32)
    return f.reshape(3, nx, nx)


def targets(phi, nx, n):
    """[n][nx][nx]: the nodal varphi of each element as channels."""
    ne = nx * nx
    return np.asarray(phi).reshape(ne, n).T.reshape(n, nx, nx).astype(np.float32)


class Normalizer:
    """Per-channel affine normalization fitted on the training set."""

    def __init__(self, data):
        self.mean = data.mean(axis=(0, 2, 3), keepdims=True)
        self.std = data.std(axis=(0, 2, 3), keepdims=True) + 1e-6

    def fwd(self, x):
        return ((x - self.mean) / self.std).astype(np.float32)

    def inv(self, y):
        return y * self.std + self.mean


def train(net, X, Y, steps, batch, lr, seed=0, log_every=0):
    """Adam steps on random mini-batches (inputs and targets already normalized,
    CUDA float32 tensors [N][C][H][W]); returns the loss history."""
    import torch

    rng = np.random.default_rng(seed)
    losses = []
    N = X.shape[0]
    for s in range(steps):
        idx = torch.as_tensor(rng.choice(N, size=min(batch, N), replace=False), device=X.device)
        xb = X.index_select(0, idx).contiguous()
        yb = Y.index_select(0, idx).contiguous()
        cur_lr = lr * (0.1 ** (s / max(steps, 1)))
        losses.append(net.train_step(xb, yb, cur_lr))
        if log_every and s % log_every == 0:
            print(f"step {s} loss {losses[-1]:.4e}")
    return losses


def predict_phi(net, x_norm, ynorm: Normalizer, nx, n):
    """Nodal varphi [nx*nx*n] (float64) proposed by the network for one input."""
    import torch

    out = torch.zeros((1, n, nx, nx), dtype=torch.float32, device=x_norm.device)
    net.forward(x_norm.reshape(1, 3, nx, nx).contiguous(), out)
    y = ynorm.inv(out.cpu().numpy())[0]
    phi = y[:n].reshape(n, nx * nx).T
    return np.ascontiguousarray(phi.ravel(), dtype=np.float64)
