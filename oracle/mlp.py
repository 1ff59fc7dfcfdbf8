"""Oracle: the warm-start network and its inputs, in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The inner CG for s_j = S^{-1} e_j (Sec. 2) may start from any x0; a network
predicts x0 on the 17-atom patch around j's atom (the atom and its 16 nearest
neighbours, distance order, ties by atom id, 4 orbitals each = 68 values).
Inputs (132): for the 32 nearest neighbours within 3 A (distance order, ties by
id, the atom itself excluded) their distance d and direction cosines (l, m, n)
of r_b - r_a, zeros beyond; then a one-hot of j's orbital (s, px, py, pz).

Network: 132 -> 128 -> 128 -> 68, SiLU after the two hidden layers,
parameters packed as W1 [128x132], b1, W2 [128x128], b2, W3 [68x128], b3.
Loss: mean over the batch and the 68 outputs of (y - t)^2. Optimiser: Adam
(Kingma & Ba 2015) with bias correction.
"""
from __future__ import annotations

import numpy as np

from .sk import min_image

SIZES = (132, 128, 128, 68)
N_NEIGH = 32
R_NEIGH = 3.0
N_PATCH = 17


def n_params() -> int:
    return sum(SIZES[i + 1] * SIZES[i] + SIZES[i + 1] for i in range(3))


def unpack(theta: np.ndarray) -> list[tuple[np.ndarray, np.ndarray]]:
    out, k = [], 0
    for i in range(3):
        o, n = SIZES[i + 1], SIZES[i]
        W = theta[k:k + o * n].reshape(o, n)
        k += o * n
        b = theta[k:k + o]
        k += o
        out.append((W, b))
    return out


def silu(x):
    return x / (1.0 + np.exp(-x))


def dsilu(x):
    s = 1.0 / (1.0 + np.exp(-x))
    return s * (1.0 + x * (1.0 - s))


def forward(theta: np.ndarray, X: np.ndarray):
    (W1, b1), (W2, b2), (W3, b3) = unpack(theta)
    Z1 = X @ W1.T + b1
    H1 = silu(Z1)
    Z2 = H1 @ W2.T + b2
    H2 = silu(Z2)
    Y = H2 @ W3.T + b3
    return Y, (X, Z1, H1, Z2, H2)


def loss_and_grad(theta: np.ndarray, X: np.ndarray, T: np.ndarray) -> tuple[float, np.ndarray]:
    """MSE loss and its gradient with respect to the packed parameters (backpropagation)."""
    (W1, b1), (W2, b2), (W3, b3) = unpack(theta)
    Y, (X, Z1, H1, Z2, H2) = forward(theta, X)
    B, K = Y.shape
    L = float(np.sum((Y - T) ** 2) / (B * K))
    dY = 2.0 * (Y - T) / (B * K)
    gW3, gb3 = dY.T @ H2, dY.sum(0)
    dZ2 = (dY @ W3) * dsilu(Z2)
    gW2, gb2 = dZ2.T @ H1, dZ2.sum(0)
    dZ1 = (dZ2 @ W2) * dsilu(Z1)
    gW1, gb1 = dZ1.T @ X, dZ1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return L, g


def adam_step(theta, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def neighbours_sorted(pos: np.ndarray, box: np.ndarray, a: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """All other atoms by increasing minimum-image distance (ties by id): ids, distances, displacements."""
    d = min_image(pos - pos[a], box)
    r = np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2])
    order = np.lexsort((np.arange(len(r)), r))
    order = order[order != a]
    return order, r[order], d[order]


def features(pos: np.ndarray, box: np.ndarray, a: int) -> tuple[np.ndarray, np.ndarray]:
    """The 4 input rows (one per orbital of atom a) and the 17 patch atom ids."""
    ids, r, d = neighbours_sorted(pos, box, a)
    geo = np.zeros((N_NEIGH, 4))
    k = min(N_NEIGH, int(np.sum(r <= R_NEIGH)))
    geo[:k, 0] = r[:k]
    geo[:k, 1:] = d[:k] / r[:k, None]
    X = np.zeros((4, 132))
    X[:, :128] = geo.ravel()
    X[np.arange(4), 128 + np.arange(4)] = 1.0
    patch = np.concatenate([[a], ids[:N_PATCH - 1]]).astype(np.int64)
    return X, patch
