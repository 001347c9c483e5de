"""GPU parity of the surrogate network's BF16 kernels against the FP64 oracle.

The oracle runs with the same BF16-rounded weights; the GPU also rounds
activations and output gradients to BF16 before each tensor-core product,
so forward outputs agree to ~1e-2 relative and gradients to a cosine
similarity above 0.999 (BF16 keeps 8 significant bits).
"""
import numpy as np
import pytest
import torch

from oracle.mlp import Adam, backward, bf16_round, forward

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1101_5803_gb300 import binding as b
    return b


def _oracle_params(net, flat=None):
    return [(bf16_round(W).reshape(W.shape), b.astype(np.float64)) for W, b in net.layers(flat)]


@pytest.mark.parametrize("dims", [[7, 64, 48, 2], [7, 256, 256, 256, 2]])
def test_forward_and_gradients(binding, dims):
    net = binding.MLP(dims, seed=1)
    rng = np.random.default_rng(0)
    X = rng.standard_normal((300, 7)).astype(np.float32)
    T = rng.standard_normal((300, 2)).astype(np.float32)
    xg, tg = torch.as_tensor(X, device="cuda"), torch.as_tensor(T, device="cuda")
    params = _oracle_params(net)
    Yo, _ = forward(params, bf16_round(X))
    Yg = net.forward(xg).cpu().numpy()
    assert np.abs(Yg - Yo).max() <= 2e-2 * np.abs(Yo).max()
    g, loss, _ = net.grad(xg, tg)
    torch.cuda.synchronize()
    go = backward(params, bf16_round(X), T.astype(np.float64))
    flat_o = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in go])
    gg = g.cpu().numpy().astype(np.float64)
    o = 0
    for (gw, gb) in go:
        for ref in (gw.ravel(), gb.ravel()):
            part = gg[o:o + ref.size]
            o += ref.size
            cos = part @ ref / (np.linalg.norm(part) * np.linalg.norm(ref) + 1e-300)
            assert cos > 0.999, cos
            assert np.linalg.norm(part - ref) <= 5e-2 * np.linalg.norm(ref)
    assert o == flat_o.size
    lo = np.mean((Yo - T) ** 2)
    assert abs(loss.item() - lo) <= 2e-2 * lo
    net.close()


@pytest.mark.parametrize("rows,k,n", [(1, 7, 2), (127, 64, 16), (128, 65, 17), (300, 256, 256),
                                       (1000, 300, 300), (257, 33, 200)])
def test_tensor_core_product_per_element(binding, rows, k, n):
    """A one-layer network is the product itself: Y = bf16(X) bf16(W)^T + b.
    Every element is checked against FP64 on the same BF16 operands, with the
    FP32 accumulation bound (K + 8) 2^-22 sum|terms|: ragged M, N and K
    tiles, N above one 256-column tile, and K above one 64-wide chunk."""
    net = binding.MLP([k, n], seed=5)
    rng = np.random.default_rng(rows + k + n)
    flat = rng.standard_normal(net.n_params).astype(np.float32)
    net.set_params(flat)
    X = rng.standard_normal((rows, k)).astype(np.float32)
    (W, b), = net.layers(flat)
    Xr, Wr = bf16_round(X), bf16_round(W).reshape(W.shape)
    ref = Xr @ Wr.T + b
    bound = (k + 8) * 2.0 ** -22 * (np.abs(Xr) @ np.abs(Wr).T + np.abs(b)) + 1e-30
    Y = net.forward(torch.as_tensor(X, device="cuda")).cpu().numpy().astype(np.float64)
    assert Y.shape == (rows, n)
    assert np.all(np.abs(Y - ref) <= bound), np.max(np.abs(Y - ref) / bound)
    net.close()


def test_adam_step_matches_oracle(binding):
    net = binding.MLP([7, 32, 2], seed=2)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((64, 7)).astype(np.float32)
    T = rng.standard_normal((64, 2)).astype(np.float32)
    p0 = net.get_params().astype(np.float64)
    xg, tg = torch.as_tensor(X, device="cuda"), torch.as_tensor(T, device="cuda")
    g, _, _ = net.grad(xg, tg)
    g = g.cpu().numpy().astype(np.float64)
    net.train_step(xg, tg, 1e-2)
    p1 = net.get_params().astype(np.float64)
    # the first Adam step moves each parameter by -lr g / (|g| + eps): the
    # oracle's Adam applied to the GPU's gradient must give the same move
    lay, o = [], 0
    for i, j in zip([7, 32], [32, 2]):
        lay.append((p0[o:o + i * j].reshape(j, i), p0[o + i * j:o + i * j + j]))
        o += i * j + j
    glay, o = [], 0
    for i, j in zip([7, 32], [32, 2]):
        glay.append((g[o:o + i * j].reshape(j, i), g[o + i * j:o + i * j + j]))
        o += i * j + j
    new = Adam(lay, lr=1e-2).step(lay, glay)
    ref = np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in new])
    np.testing.assert_allclose(p1, ref, atol=2e-6)
    net.close()


def test_training_fits_a_smooth_map(binding):
    net = binding.MLP([7, 64, 64, 2], seed=3)
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (2048, 7)).astype(np.float32)
    T = np.stack([np.sin(X[:, 0] * 2) + X[:, 1] * X[:, 2], np.cos(X[:, 3]) - 0.5 * X[:, 4] ** 2], 1)
    T = T.astype(np.float32)
    xg, tg = torch.as_tensor(X, device="cuda"), torch.as_tensor(T, device="cuda")
    first = None
    for it in range(1500):
        idx = torch.as_tensor(rng.integers(0, 2048, 256), device="cuda")
        loss = net.train_step(xg[idx], tg[idx], 3e-3)
        if first is None:
            first = loss.item()
    Y = net.forward(xg).cpu().numpy()
    mse = float(np.mean((Y - T) ** 2))
    assert mse < 0.02 * first and mse < 5e-3, (first, mse)
    net.close()


def _rows(seed, step, batch, n):
    """The minibatch rows of mirage_mlp_train's step `step`: slot j takes
    splitmix64-finaliser(seed * golden + (step << 24) + j) mod n, written
    out here from the finaliser's published definition."""
    M = (1 << 64) - 1
    out = []
    for j in range(batch):
        z = (seed * 0x9E3779B97F4A7C15 + (step << 24) + j) & M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        z ^= z >> 31
        out.append(z % n)
    return np.array(out)


def test_device_training_loop_matches_host_steps(binding):
    # mirage_mlp_train draws each step's rows on the device; with the same
    # rows handed to train_step one at a time the parameters must agree
    rng = np.random.default_rng(7)
    X = rng.standard_normal((300, 7)).astype(np.float32)
    T = rng.standard_normal((300, 2)).astype(np.float32)
    xg, tg = torch.as_tensor(X, device="cuda"), torch.as_tensor(T, device="cuda")
    a = binding.MLP([7, 64, 48, 2], seed=5)
    b = binding.MLP([7, 64, 48, 2], seed=5)
    a.train(xg, tg, steps=3, batch=96, lr=3e-3, seed=11)
    for k in range(3):
        idx = torch.as_tensor(_rows(11, k, 96, 300), device="cuda")
        b.train_step(xg[idx], tg[idx], 3e-3)
    torch.cuda.synchronize()
    pa, pb = a.get_params(), b.get_params()
    np.testing.assert_allclose(pa, pb, rtol=1e-5, atol=1e-6)
    # a second call continues the step count (Adam's bias corrections)
    a.train(xg, tg, steps=1, batch=96, lr=3e-3, seed=12)
    idx = torch.as_tensor(_rows(12, 3, 96, 300), device="cuda")
    b.train_step(xg[idx], tg[idx], 3e-3)
    torch.cuda.synchronize()
    np.testing.assert_allclose(a.get_params(), b.get_params(), rtol=1e-5, atol=1e-6)
    a.close()
    b.close()


def test_device_training_loop_fits_a_smooth_map(binding):
    net = binding.MLP([7, 64, 64, 2], seed=3)
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (2048, 7)).astype(np.float32)
    T = np.stack([np.sin(X[:, 0] * 2) + X[:, 1] * X[:, 2], np.cos(X[:, 3]) - 0.5 * X[:, 4] ** 2], 1)
    T = T.astype(np.float32)
    xg, tg = torch.as_tensor(X, device="cuda"), torch.as_tensor(T, device="cuda")
    first = float(np.mean((net.forward(xg).cpu().numpy() - T) ** 2))
    net.train(xg, tg, steps=1500, batch=256, lr=3e-3, seed=1)
    Y = net.forward(xg).cpu().numpy()
    mse = float(np.mean((Y - T) ** 2))
    assert mse < 0.02 * first and mse < 5e-3, (first, mse)
    net.close()
