"""Training the learned CG warm start with the library's own kernels.

Data are the method's own inner-CG solutions: for atoms of one or more systems,
`mka_warm_start_features` gives the inputs and patch, `mka_cg_patch_targets` runs
the inner CG (x0 = 0) and writes s_j on the patch. Training is mini-batch Adam
through `mka_mlp_train_step` (forward, backward and update all in the library's
kernels); PyTorch only holds the device buffers and draws the batch order.
"""
from __future__ import annotations

import numpy as np

from . import mka


def collect(sysh, atoms: np.ndarray, arith: str = "mixed", cg_tol: float = 1e-7):
    """Inputs X [4n][132], targets Y [4n][68] and CG iterations [4n] (device tensors) for the atoms."""
    import torch
    n = len(atoms)
    X = torch.empty((4 * n, 132), dtype=torch.float32, device="cuda")
    Y = torch.empty((4 * n, 68), dtype=torch.float32, device="cuda")
    patch = torch.empty((n, 17), dtype=torch.int32, device="cuda")
    iters = torch.empty(4 * n, dtype=torch.int32, device="cuda")
    mka.mka_warm_start_features(sysh, atoms, X.data_ptr(), patch.data_ptr())
    mka.mka_cg_patch_targets(sysh, atoms, arith, cg_tol, patch.data_ptr(), Y.data_ptr(), iters.data_ptr())
    torch.cuda.synchronize()
    return X, Y, iters


def train(net, X, Y, epochs: int = 20, batch: int = 1024, lr: float = 1e-3, seed: int = 0) -> list[float]:
    """Mini-batch Adam over (X, Y); returns the mean loss of each epoch."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    n = X.shape[0]
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    for _ in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=g)
        tot, steps = 0.0, 0
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            xb = X.index_select(0, idx).contiguous()
            yb = Y.index_select(0, idx).contiguous()
            mka.mka_mlp_train_step(net, xb.data_ptr(), yb.data_ptr(), batch, lr, loss.data_ptr())
            tot += float(loss.item())
            steps += 1
        hist.append(tot / max(steps, 1))
    return hist


def mse(net, X, Y) -> float:
    """Mean squared error of the network on (X, Y), from the library's loss kernel."""
    import torch
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    mka.mka_mlp_gradients(net, X.data_ptr(), Y.data_ptr(), X.shape[0], None, loss.data_ptr())
    return float(loss.item())
