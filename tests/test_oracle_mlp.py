"""Pins for the oracle's surrogate network (forward, backward, Adam).

Gradients are pinned by central finite differences of the loss; SiLU by
its closed form; Adam by its first step (which moves every weight by
-lr sign(g)) and by convergence to the least-squares solution when the
network is a single linear layer; BF16 rounding by hand-made cases.
"""
import math

import numpy as np

from oracle.mlp import Adam, backward, bf16_round, encode_lens, forward, loss, silu, silu_grad


def _params(rng, sizes):
    return [(rng.standard_normal((o, i)) / math.sqrt(i), 0.1 * rng.standard_normal(o))
            for i, o in zip(sizes[:-1], sizes[1:])]


def test_silu_closed_form():
    z = np.array([-3.0, -0.5, 0.0, 0.7, 4.0])
    np.testing.assert_allclose(silu(z), z * (1 / (1 + np.exp(-z))), rtol=1e-15)
    h = 1e-6
    np.testing.assert_allclose(silu_grad(z), (silu(z + h) - silu(z - h)) / (2 * h), rtol=1e-8)
    assert silu(0.0) == 0.0 and abs(silu_grad(0.0) - 0.5) < 1e-15


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    params = _params(rng, [7, 16, 12, 2])
    X = rng.standard_normal((9, 7))
    T = rng.standard_normal((9, 2))
    grads = backward(params, X, T)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for (idx, arr, g) in ((np.unravel_index(rng.integers(W.size), W.shape), W, grads[li][0]),
                              ((rng.integers(b.size),), b, grads[li][1])):
            old = arr[idx]
            arr[idx] = old + h
            lp = loss(params, X, T)
            arr[idx] = old - h
            lm = loss(params, X, T)
            arr[idx] = old
            assert abs((lp - lm) / (2 * h) - g[idx]) <= 1e-7 * max(1.0, abs(g[idx]))


def test_adam_first_step_is_sign_step():
    rng = np.random.default_rng(1)
    params = _params(rng, [7, 8, 2])
    X, T = rng.standard_normal((5, 7)), rng.standard_normal((5, 2))
    g = backward(params, X, T)
    opt = Adam(params, lr=0.01, eps=0.0)
    new = opt.step(params, g)
    for (W, b), (W2, b2), (gW, gb) in zip(params, new, g):
        np.testing.assert_allclose(W2 - W, -0.01 * np.sign(gW), atol=1e-15)
        np.testing.assert_allclose(b2 - b, -0.01 * np.sign(gb), atol=1e-15)


def test_linear_network_reaches_least_squares():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((64, 7))
    Wt = rng.standard_normal((2, 7))
    T = X @ Wt.T + 0.3 + 0.01 * rng.standard_normal((64, 2))
    params = [(np.zeros((2, 7)), np.zeros(2))]
    opt = Adam(params, lr=0.05)
    for it in range(5000):
        if it == 3000:
            opt.lr = 0.002  # constant-step Adam rattles around the optimum; settle it
        params = opt.step(params, backward(params, X, T))
    A = np.hstack([X, np.ones((64, 1))])
    sol, *_ = np.linalg.lstsq(A, T, rcond=None)
    np.testing.assert_allclose(params[0][0], sol[:7].T, atol=5e-4)
    np.testing.assert_allclose(params[0][1], sol[7], atol=5e-4)


def test_forward_shapes_and_output_layer_linear():
    rng = np.random.default_rng(3)
    params = _params(rng, [7, 4, 2])
    X = rng.standard_normal((3, 7))
    Y, (acts, pres) = forward(params, X)
    np.testing.assert_allclose(Y, pres[-1])
    np.testing.assert_allclose(acts[1], silu(X @ params[0][0].T + params[0][1]))


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 0.0])
    # bf16 keeps 8 significant bits: 1 + 2^-8 is a tie -> even (1.0); 1 + 3*2^-8 -> 1 + 2^-6
    np.testing.assert_array_equal(bf16_round(x), [1.0, 1.0, 1.0 + 2 ** -7, 1.0 + 2 ** -6, -2.5, 0.0])


def test_lens_encoding_is_pi_periodic():
    l1 = np.array([1.0, 0.7, 0.4, 0.01, -0.02, 0.05, 0.3])
    l2 = l1.copy()
    l2[2] += math.pi
    l2[6] += math.pi
    np.testing.assert_allclose(encode_lens(l1), encode_lens(l2), atol=1e-12)
    # a round lens has no orientation
    l3 = l1.copy()
    l3[1] = 1.0
    l4 = l3.copy()
    l4[2] = 1.1
    np.testing.assert_allclose(encode_lens(l3), encode_lens(l4), atol=1e-15)
