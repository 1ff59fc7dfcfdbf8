"""Pins for the oracle's warm-start network: backpropagation against central finite
differences, Adam against torch.optim.Adam, SiLU' against a difference quotient, and the
input features against a perfect diamond lattice (first shell: 4 atoms at a*sqrt(3)/4
along (+-1, +-1, +-1)/sqrt(3); second shell: 12 at a/sqrt(2))."""
import numpy as np
import pytest

from oracle import mlp
from synth import lattice_positions


def test_silu_derivative():
    x = np.linspace(-6, 6, 25)
    h = 1e-6
    np.testing.assert_allclose(mlp.dsilu(x), (mlp.silu(x + h) - mlp.silu(x - h)) / (2 * h), rtol=1e-7, atol=1e-9)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = rng.normal(size=mlp.n_params()) * 0.1
    X = rng.normal(size=(5, 132))
    T = rng.normal(size=(5, 68)) * 0.1
    L, g = mlp.loss_and_grad(theta, X, T)
    idx = rng.choice(mlp.n_params(), 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (mlp.loss_and_grad(theta + e, X, T)[0] - mlp.loss_and_grad(theta - e, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)) + 1e-10, (i, fd, g[i])


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    theta = rng.normal(size=50)
    p = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(50)
    v = np.zeros(50)
    for t in range(1, 6):
        g = rng.normal(size=50)
        p.grad = torch.tensor(g)
        opt.step()
        theta, m, v = mlp.adam_step(theta, g, m, v, t)
    np.testing.assert_allclose(theta, p.detach().numpy(), rtol=0, atol=1e-12)


def test_features_on_perfect_diamond():
    a = 3.567
    pos, box = lattice_positions("diamond", a, 3, 0.0, 0.0, 0)
    X, patch = mlp.features(pos, box, 0)
    geo = X[0, :128].reshape(32, 4)
    nn = a * np.sqrt(3) / 4
    np.testing.assert_allclose(geo[:4, 0], nn, atol=1e-12)
    np.testing.assert_allclose(np.abs(geo[:4, 1:]), 1 / np.sqrt(3), atol=1e-12)
    np.testing.assert_allclose(geo[4:16, 0], a / np.sqrt(2), atol=1e-12)
    assert np.all(geo[28:] == 0)                            # 4 + 12 + 12 atoms lie within 3 A
    np.testing.assert_allclose(np.linalg.norm(geo[:28, 1:], axis=1), 1.0, atol=1e-12)
    assert patch[0] == 0 and len(set(patch.tolist())) == 17
    np.testing.assert_array_equal(X[:, 128:], np.eye(4))


def test_silu_closed_values():
    """SiLU(x) = x sigma(x): SiLU(0) = 0, SiLU(1) = 1 / (1 + e^-1), SiLU(-x) = SiLU(x) - x."""
    assert mlp.silu(0.0) == 0.0
    assert abs(mlp.silu(1.0) - 1.0 / (1.0 + np.exp(-1.0))) < 1e-16
    x = np.linspace(-5, 5, 11)
    np.testing.assert_allclose(mlp.silu(-x), mlp.silu(x) - x, rtol=0, atol=1e-14)


def test_forward_matches_torch_layers():
    """The packed parameters unpacked as W [out][in] row-major and b, run through torch's own linear
    and SiLU in FP64: a transposed weight, a swapped layer or a wrong activation would differ."""
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    rng = np.random.default_rng(7)
    theta = rng.normal(size=mlp.n_params()) * 0.2
    X = rng.normal(size=(9, 132))
    Y, _ = mlp.forward(theta, X)
    t = torch.tensor(theta)
    k, h = 0, torch.tensor(X)
    for i, act in enumerate((True, True, False)):
        o, n = mlp.SIZES[i + 1], mlp.SIZES[i]
        W = t[k:k + o * n].reshape(o, n)
        k += o * n
        b = t[k:k + o]
        k += o
        h = F.linear(h, W, b)
        if act:
            h = F.silu(h)
    assert k == mlp.n_params()
    np.testing.assert_allclose(Y, h.numpy(), rtol=0, atol=1e-12)


def test_forward_matches_scalar_loop():
    """A one-row forward pass written as scalar loops over the packed vector (offsets counted by hand)."""
    rng = np.random.default_rng(8)
    theta = rng.normal(size=mlp.n_params()) * 0.2
    x = rng.normal(size=132)
    Y, _ = mlp.forward(theta, x[None, :])
    h, off = list(x), 0
    for i in range(3):
        n_in, n_out = mlp.SIZES[i], mlp.SIZES[i + 1]
        wofs, bofs = off, off + n_out * n_in
        out = []
        for r in range(n_out):
            s = theta[bofs + r]
            for c in range(n_in):
                s += theta[wofs + r * n_in + c] * h[c]
            out.append(s / (1.0 + np.exp(-s)) if i < 2 else s)
        h, off = out, bofs + n_out
    np.testing.assert_allclose(Y[0], h, rtol=0, atol=1e-12)
