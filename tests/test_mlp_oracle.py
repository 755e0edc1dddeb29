"""Pins of the learned-stencil network's CPU oracle (no GPU): chain-rule gradients against
central finite differences, hard-swish against its closed form, a hand-computed tiny network,
and the patch layout."""

import numpy as np
import pytest

from oracle import mlp_oracle as M


def test_hswish_closed_form_and_derivative():
    z = np.linspace(-6, 6, 101) + 0.0123  # off the kinks at -3 and 3
    ref = np.where(z < -3, 0.0, np.where(z > 3, z, z * (z + 3) / 6))
    assert np.allclose(M.hswish(z), ref, rtol=0, atol=1e-15)
    h = 1e-6
    fd = (M.hswish(z + h) - M.hswish(z - h)) / (2 * h)
    assert np.abs(fd - M.hswish_grad(z)).max() < 1e-8
    assert M.hswish(0.0) == 0.0 and abs(M.hswish_grad(0.0) - 0.5) < 1e-15


def test_tiny_network_by_hand():
    # one input, one hidden unit, one output: y = w2 * hswish(w1 x + b1) + b2
    x = np.array([[0.5]])
    W = [np.array([[2.0]]), np.array([[-3.0]])]
    b = [np.array([0.25]), np.array([1.0])]
    y, _ = M.mlp_forward(x, W, b)
    z = 2.0 * 0.5 + 0.25
    assert abs(y[0, 0] - (-3.0 * z * (z + 3) / 6 + 1.0)) < 1e-15


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    sizes = [7, 11, 9, 5]
    W = [rng.standard_normal((sizes[i + 1], sizes[i])) * 0.5 for i in range(3)]
    b = [rng.standard_normal(sizes[i + 1]) * 0.1 for i in range(3)]
    x = rng.standard_normal((6, sizes[0]))
    t = rng.standard_normal((6, sizes[-1]))
    loss, dW, db = M.mlp_backward(x, t, W, b)
    y, _ = M.mlp_forward(x, W, b)
    assert abs(loss - np.mean((y - t) ** 2)) < 1e-15
    for layer in range(3):
        for idx in [(0, 0), (sizes[layer + 1] - 1, sizes[layer] - 1), (2, 3)]:
            fd = M.finite_difference(x, t, W, b, layer, idx)
            assert abs(fd - dW[layer][idx]) <= 1e-7 * max(1.0, abs(fd)), (layer, idx)
    # bias gradient of the last layer: d loss / d b = mean over batch of 2 (y - t) / n_out
    assert np.allclose(db[2], (2 * (y - t) / y.size).sum(axis=0), rtol=1e-12, atol=0)


def test_patch_layout():
    rng = np.random.default_rng(3)
    n = 8
    v = rng.standard_normal((n, n))
    P = M.patches(v, radius=2)
    j = (3, 6)
    flat = j[0] * n + j[1]
    k = 0
    for o0 in range(-2, 3):
        for o1 in range(-2, 3):
            assert P[flat, k] == v[(j[0] + o0) % n, (j[1] + o1) % n] / (n * n)
            k += 1
