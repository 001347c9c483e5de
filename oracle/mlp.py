"""Oracle: the surrogate network in FP64 (forward, backward, Adam).

Test infrastructure only (see ``oracle/__init__.py``).

The surrogate maps an encoded lens vector to the standardised pair
(log chi2 at the L-curve corner, log10 lambda at the corner).  It is a
plain multilayer perceptron: hidden layers z = W a + b, a = silu(z) with
silu(z) = z / (1 + exp(-z)), a linear output layer, mean-squared-error loss
over the batch and outputs, and the Adam update (Kingma & Ba 2015):

    m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
    w <- w - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

The GPU path runs its matrix products on BF16 operands; the oracle takes
the BF16-rounded weights it is handed and computes everything else in FP64.
"""
from __future__ import annotations

import numpy as np


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def bf16_round(x):
    """Round FP32/FP64 values to the nearest BF16 value (ties to even)."""
    x = np.asarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32)
    return np.where(np.isfinite(x), out, x).astype(np.float64)


def encode_lens(lens):
    """Continuous encoding of (b, q, phi, x0, y0, gamma, theta_g): the SIE is
    pi-periodic in phi and the shear pi-periodic in theta_g, so angles enter
    through doubled-angle components."""
    L = np.atleast_2d(np.asarray(lens, dtype=np.float64))
    b, q, phi, x0, y0, g, tg = L.T
    return np.stack([b, (1 - q) * np.cos(2 * phi), (1 - q) * np.sin(2 * phi), x0, y0,
                     g * np.cos(2 * tg), g * np.sin(2 * tg)], axis=1)


def forward(params, X):
    """params: list of (W [out, in], b [out]).  Returns (Y, cache)."""
    a = np.asarray(X, dtype=np.float64)
    acts, pres = [a], []
    for li, (W, b) in enumerate(params):
        z = a @ W.T + b
        pres.append(z)
        a = z if li == len(params) - 1 else silu(z)
        acts.append(a)
    return a, (acts, pres)


def loss(params, X, T):
    Y, _ = forward(params, X)
    return float(np.mean((Y - np.asarray(T, dtype=np.float64)) ** 2))


def backward(params, X, T):
    """Gradients of the mean-squared error: list of (dW, db)."""
    Y, (acts, pres) = forward(params, X)
    n = Y.size
    d = 2.0 * (Y - np.asarray(T, dtype=np.float64)) / n
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        dz = d if li == len(params) - 1 else d * silu_grad(pres[li])
        grads[li] = (dz.T @ acts[li], dz.sum(axis=0))
        d = dz @ W
    return grads


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.t = 0
        self.m = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.v = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]

    def step(self, params, grads):
        self.t += 1
        out = []
        for i, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
            new = []
            for j, (p, g) in enumerate(((W, gW), (b, gb))):
                m = self.b1 * self.m[i][j] + (1 - self.b1) * g
                v = self.b2 * self.v[i][j] + (1 - self.b2) * g * g
                self.m[i] = tuple(m if jj == j else self.m[i][jj] for jj in range(2))
                self.v[i] = tuple(v if jj == j else self.v[i][jj] for jj in range(2))
                mh = m / (1 - self.b1 ** self.t)
                vh = v / (1 - self.b2 ** self.t)
                new.append(p - self.lr * mh / (np.sqrt(vh) + self.eps))
            out.append(tuple(new))
        return out
