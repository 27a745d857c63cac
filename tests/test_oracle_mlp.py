"""Pins of the FP64 MLP oracle used for the learned stress closure.

GELU against values of the normal CDF, a single affine layer against a
numpy matmul, backward against central finite differences of the forward,
and AdamW against torch's independent CPU implementation."""
import math

import numpy as np
import pytest

import oracle as O


def test_gelu_values_and_identities():
    assert O.gelu(0.0) == 0.0
    assert abs(O.gelu(1.0) - 0.8413447460685429) < 1e-15  # Phi(1)
    for x in (-3.0, -0.4, 0.7, 2.5):
        assert abs(O.gelu(-x) - (O.gelu(x) - x)) < 1e-14  # Phi(-x) = 1 - Phi(x)
    assert abs(O.gelu(12.0) - 12.0) < 1e-12 and abs(O.gelu(-12.0)) < 1e-12


def test_single_affine_layer_is_matmul():
    rng = np.random.default_rng(0)
    dims = [4, 3]
    W = rng.normal(size=(3, 4))
    b = rng.normal(size=3)
    params = np.concatenate([W.ravel(), b])
    x = rng.normal(size=(5, 4))
    y = O.mlp_forward(dims, params, x)
    assert np.allclose(y, x @ W.T + b, rtol=0, atol=1e-14)


def _init(dims, rng):
    ps = []
    for a, b in zip(dims[:-1], dims[1:]):
        ps.append(rng.normal(size=(b, a)).ravel() / math.sqrt(a))
        ps.append(rng.normal(size=b) * 0.1)
    return np.concatenate(ps)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    dims = [6, 9, 8, 3]
    params = _init(dims, rng)
    assert params.size == O.mlp_n_params(dims)
    x = rng.normal(size=(7, 6))
    t = rng.normal(size=(7, 3))
    loss, g = O.mlp_loss_grad(dims, params, x, t)
    eps = 1e-6
    idx = rng.choice(params.size, size=60, replace=False)
    for k in idx:
        pp = params.copy()
        pp[k] += eps
        lp, _ = O.mlp_loss_grad(dims, pp, x, t)
        pp[k] -= 2 * eps
        lm, _ = O.mlp_loss_grad(dims, pp, x, t)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (k, fd, g[k])
    # the loss itself is the mean squared error of the forward pass
    y = O.mlp_forward(dims, params, x)
    assert abs(loss - np.mean((y - t) ** 2)) < 1e-14


def test_adamw_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    n = 50
    p0 = rng.normal(size=n)
    grads = [rng.normal(size=n) for _ in range(4)]
    lr, b1, b2, eps, wd = 1e-3, 0.9, 0.999, 1e-8, 0.01
    p = p0.copy()
    m = np.zeros(n)
    v = np.zeros(n)
    for t, g in enumerate(grads, start=1):
        O.adamw_step(p, g, m, v, lr, b1, b2, eps, wd, t)
    tp = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.AdamW([tp], lr=lr, betas=(b1, b2), eps=eps, weight_decay=wd)
    for g in grads:
        opt.zero_grad()
        tp.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
    assert np.allclose(p, tp.detach().numpy(), rtol=0, atol=1e-15)
