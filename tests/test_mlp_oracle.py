"""Pins of the learned-stencil network's CPU oracle (no GPU): chain-rule gradients against
central finite differences, ReLU against its closed form, a hand-computed tiny network, and
the patch layout."""

import numpy as np
import pytest

from oracle import mlp_oracle as M


def test_relu_closed_form_and_derivative():
    z = np.linspace(-6, 6, 101) + 0.0123  # off the kink at 0
    assert np.array_equal(M.relu(z), np.where(z > 0, z, 0.0))
    h = 1e-6
    fd = (M.relu(z + h) - M.relu(z - h)) / (2 * h)
    assert np.abs(fd - M.relu_grad(z)).max() < 1e-8
    assert M.relu(0.0) == 0.0 and M.relu_grad(0.0) == 0.0 and M.relu_grad(1e-300) == 1.0


def test_tiny_network_by_hand():
    # one input, two hidden units (one active, one not), one output:
    # y = w2 . relu(W1 x + b1) + b2
    x = np.array([[0.5]])
    W = [np.array([[2.0], [-4.0]]), np.array([[-3.0, 5.0]])]
    b = [np.array([0.25, 1.0]), np.array([1.0])]
    y, _ = M.mlp_forward(x, W, b)
    # z = (1.25, -1.0): relu -> (1.25, 0); y = -3 * 1.25 + 5 * 0 + 1
    assert abs(y[0, 0] - (-3.0 * 1.25 + 1.0)) < 1e-15
    loss, dW, db = M.mlp_backward(x, np.array([[0.0]]), W, b)
    g = 2.0 * y[0, 0]  # d loss / d y for one sample, one output
    assert abs(dW[1][0, 0] - g * 1.25) < 1e-14 and dW[1][0, 1] == 0.0
    assert abs(dW[0][0, 0] - g * -3.0 * 0.5) < 1e-14 and dW[0][1, 0] == 0.0


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
