"""FP64 oracle of the learned pairwise surrogate (test infrastructure).

The paper proposes, as future work (Section 7), training a neural network to
predict MI values so that sampling gets faster. The surrogate here is that
network (a project addition): a per-point encoder maps a point's standardized
member vector to an embedding, a pair head maps two embeddings and their
relative position to a predicted measure value.

  encoder  z (n) -> h1 = GELU(W1 z + b1) (128) -> e = W2 h1 + b2 (64)
  head     x = [e_i, e_j, |e_i - e_j|, off] (195) -> h3 = GELU(W3 x + b3) (128)
           -> y = w4 . h3 + b4
  loss     mean squared error against standardized targets
  Adam     beta1 0.9, beta2 0.999, eps 1e-8 (Kingma and Ba 2015)

READINGS: z is the z-score of the member vector ((v - mean) / sample std);
off = (position_j - position_i) / (X, Y, Z); GELU is the exact erf form
0.5 x (1 + erf(x / sqrt 2)); d|u|/du is sign(u) (0 at 0).

Parameters travel as one flat FP64 vector in the order W1 (128 x n, row-major),
b1, W2 (64 x 128), b2, W3 (128 x 195), b3, w4 (128), b4 (1); the CUDA library
uses the same layout (as fp32 master weights). Plain numpy; only tests and the
benchmark's CPU leg may import this module.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

H1, E, H3 = 128, 64, 128
HEAD_IN = 3 * E + 3


def shapes(n: int):
    return [("W1", (H1, n)), ("b1", (H1,)), ("W2", (E, H1)), ("b2", (E,)),
            ("W3", (H3, HEAD_IN)), ("b3", (H3,)), ("w4", (H3,)), ("b4", (1,))]


def n_params(n: int) -> int:
    return sum(int(np.prod(s)) for _, s in shapes(n))


def unpack(flat, n):
    out, o = {}, 0
    for name, s in shapes(n):
        size = int(np.prod(s))
        out[name] = np.asarray(flat[o:o + size], np.float64).reshape(s)
        o += size
    return out


def pack(d, n):
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in shapes(n)])


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)


def zscore(F, pts):
    """Standardized member vectors of points pts of a [n][...] field: [len][n]."""
    V = np.asarray(F, np.float64).reshape(F.shape[0], -1)[:, pts].T
    m = V.mean(1, keepdims=True)
    s = V.std(1, ddof=1, keepdims=True)
    return np.where(s > 0, (V - m) / np.where(s > 0, s, 1.0), 0.0)


def offsets(X, Y, Z, pi, pj):
    def pos(p):
        p = np.asarray(p, np.int64)
        return np.stack([p % X, (p // X) % Y, p // (X * Y)], 1).astype(np.float64)
    return (pos(pj) - pos(pi)) / np.array([X, Y, Z], np.float64)


def forward(flat, zi, zj, off, n):
    P = unpack(flat, n)
    cache = {}
    for tag, z in (("i", zi), ("j", zj)):
        a1 = z @ P["W1"].T + P["b1"]
        h1 = gelu(a1)
        e = h1 @ P["W2"].T + P["b2"]
        cache[tag] = (z, a1, h1, e)
    ei, ej = cache["i"][3], cache["j"][3]
    x = np.concatenate([ei, ej, np.abs(ei - ej), off], 1)
    a3 = x @ P["W3"].T + P["b3"]
    h3 = gelu(a3)
    y = h3 @ P["w4"] + P["b4"][0]
    cache["head"] = (x, a3, h3)
    return y, cache


def loss_and_grad(flat, zi, zj, off, t, n):
    """MSE loss (mean over the batch) and its gradient w.r.t. the flat parameters."""
    P = unpack(flat, n)
    y, c = forward(flat, zi, zj, off, n)
    B = len(t)
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / B
    x, a3, h3 = c["head"]
    G = {}
    G["w4"] = h3.T @ dy
    G["b4"] = np.array([dy.sum()])
    da3 = np.outer(dy, P["w4"]) * gelu_grad(a3)
    G["W3"] = da3.T @ x
    G["b3"] = da3.sum(0)
    dx = da3 @ P["W3"]
    ei, ej = c["i"][3], c["j"][3]
    sg = np.sign(ei - ej)
    de = {"i": dx[:, :E] + dx[:, 2 * E:3 * E] * sg, "j": dx[:, E:2 * E] - dx[:, 2 * E:3 * E] * sg}
    G["W2"] = np.zeros_like(P["W2"])
    G["b2"] = np.zeros_like(P["b2"])
    G["W1"] = np.zeros_like(P["W1"])
    G["b1"] = np.zeros_like(P["b1"])
    for tag in ("i", "j"):
        z, a1, h1, _ = c[tag]
        G["W2"] += de[tag].T @ h1
        G["b2"] += de[tag].sum(0)
        da1 = (de[tag] @ P["W2"]) * gelu_grad(a1)
        G["W1"] += da1.T @ z
        G["b1"] += da1.sum(0)
    return loss, pack(G, n)


def adam(flat, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (step counts from 1); returns new (params, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v


def init(n, seed):
    """Seeded initial parameters: normal(0, 1/fan_in) weights, zero biases."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, s in shapes(n):
        if name.startswith("b"):
            d[name] = np.zeros(s)
        else:
            fan_in = s[1] if len(s) == 2 else s[0]
            d[name] = rng.standard_normal(s) / math.sqrt(fan_in)
    return pack(d, n)
