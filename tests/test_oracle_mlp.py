"""Pins of the FP64 surrogate oracle: gradients against central finite
differences and torch float64 autograd, Adam against torch.optim.Adam."""
import numpy as np
import pytest

from oracle import mlp

N = 12  # members (small for finite differences)


def batch(seed, B=5):
    rng = np.random.default_rng(seed)
    zi = rng.standard_normal((B, N))
    zj = rng.standard_normal((B, N))
    off = rng.uniform(-1, 1, (B, 3))
    t = rng.standard_normal(B)
    return zi, zj, off, t


def test_param_count():
    assert mlp.n_params(100) == 46401


def test_gradient_finite_differences():
    zi, zj, off, t = batch(1)
    w = mlp.init(N, 3)
    _, g = mlp.loss_and_grad(w, zi, zj, off, t, N)
    rng = np.random.default_rng(4)
    idx = rng.choice(len(w), 60, replace=False)
    for i in idx:
        h = 1e-6
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss_and_grad(wp, zi, zj, off, t, N)[0] -
              mlp.loss_and_grad(wm, zi, zj, off, t, N)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def torch_model(w):
    torch = pytest.importorskip("torch")
    P = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True)
         for k, v in mlp.unpack(w, N).items()}

    def f(zi, zj, off):
        def enc(z):
            h = torch.nn.functional.gelu(z @ P["W1"].T + P["b1"])
            return h @ P["W2"].T + P["b2"]
        ei, ej = enc(zi), enc(zj)
        x = torch.cat([ei, ej, (ei - ej).abs(), off], 1)
        h3 = torch.nn.functional.gelu(x @ P["W3"].T + P["b3"])
        return h3 @ P["w4"] + P["b4"][0]
    return P, f


def test_gradient_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    zi, zj, off, t = batch(2, B=16)
    w = mlp.init(N, 5)
    P, f = torch_model(w)
    T = lambda a: torch.tensor(a, dtype=torch.float64)
    y = f(T(zi), T(zj), T(off))
    loss = ((y - T(t)) ** 2).mean()
    loss.backward()
    ref = np.concatenate([P[k].grad.numpy().ravel() for k, _ in mlp.shapes(N)])
    l2, g = mlp.loss_and_grad(w, zi, zj, off, t, N)
    assert abs(l2 - loss.item()) < 1e-12
    assert np.abs(g - ref).max() < 1e-10
    y2, _ = mlp.forward(w, zi, zj, off, N)
    assert np.abs(y2 - y.detach().numpy()).max() < 1e-12


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    w = rng.standard_normal(50)
    p = torch.tensor(w.copy(), requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(50)
    v = np.zeros(50)
    for step in range(1, 6):
        g = rng.standard_normal(50)
        p.grad = torch.tensor(g.copy())
        opt.step()
        w, m, v = mlp.adam(w, g, m, v, step, 1e-3)
    assert np.abs(w - p.detach().numpy()).max() < 1e-12
