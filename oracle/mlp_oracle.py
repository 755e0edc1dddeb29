"""Plain FP64 oracle of the learned-stencil network (the surrogate for steps a3-a6).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline of the benchmark); the library never
imports it. The paper has no learned component: this network is a surrogate trained on the
paper's own stencils (Sec. 4.1, 4.2), so its oracle is the textbook definition of a
multilayer perceptron, written out in numpy:

    z_l = a_{l-1} W_l^T + b_l,   a_l = relu(z_l) = max(z_l, 0)   (hidden),
    y   = a_{L-1} W_L^T + b_L,   loss = mean over the batch and the outputs of (y - t)^2,

with the gradients of that loss by the chain rule. Weights enter as float64 copies of the
values the GPU uses (bf16 weights, fp32 biases); the comparison tolerance reflects bf16
activations on the GPU.

Input of the network for a point j: the (2r+1)^d patch of h^2 v around j (periodic), in
lexicographic offset order (last axis fastest), then h^2 s_j with s_j the point's snapped shift;
normalised by (x - mean) / std of the training set. Output: alpha (|mu| values) and c (|mu|
values), normalised per output.
"""

from __future__ import annotations

import numpy as np

__all__ = ["relu", "relu_grad", "mlp_forward", "mlp_backward", "patches",
           "finite_difference"]


def relu(z):
    """The ReLU activation max(z, 0)."""
    return np.maximum(z, 0.0)


def relu_grad(z):
    """Its derivative: 1 where z > 0, else 0 (0 at z = 0)."""
    z = np.asarray(z, dtype=np.float64)
    return (z > 0.0).astype(np.float64)


def mlp_forward(x: np.ndarray, weights: list, biases: list):
    """Returns (y, cache). x: [B, K0]; weights[l]: [N_l, K_l]; biases[l]: [N_l]."""
    a = np.asarray(x, dtype=np.float64)
    zs, acts = [], [a]
    L = len(weights)
    for li, (W, b) in enumerate(zip(weights, biases)):
        z = a @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        zs.append(z)
        a = relu(z) if li < L - 1 else z
        acts.append(a)
    return a, (zs, acts)


def mlp_backward(x, t, weights, biases):
    """Loss and its gradients (dW_l, db_l) for loss = mean((y - t)^2)."""
    y, (zs, acts) = mlp_forward(x, weights, biases)
    t = np.asarray(t, np.float64)
    loss = float(np.mean((y - t) ** 2))
    g = 2.0 * (y - t) / y.size
    L = len(weights)
    dWs, dbs = [None] * L, [None] * L
    for li in range(L - 1, -1, -1):
        dz = g if li == L - 1 else g * relu_grad(zs[li])
        dWs[li] = dz.T @ acts[li]
        dbs[li] = dz.sum(axis=0)
        g = dz @ np.asarray(weights[li], np.float64)
    return loss, dWs, dbs


def finite_difference(x, t, weights, biases, which, index, h=1e-6):
    """Central difference of the loss with respect to one weight (which = layer, index)."""
    def loss_with(delta):
        ws = [np.array(W, dtype=np.float64, copy=True) for W in weights]
        ws[which][index] += delta
        y, _ = mlp_forward(x, ws, biases)
        return float(np.mean((y - np.asarray(t, np.float64)) ** 2))
    return (loss_with(h) - loss_with(-h)) / (2 * h)


def patches(v: np.ndarray, radius: int = 2) -> np.ndarray:
    """h^2 v over the (2r+1)^d neighbourhood of every point, [N, (2r+1)^d], periodic."""
    n, d = v.shape[0], v.ndim
    h2v = v / float(n * n)
    rng = range(-radius, radius + 1)
    offs = np.array(np.meshgrid(*([list(rng)] * d), indexing="ij")).reshape(d, -1).T
    cols = [np.roll(h2v, tuple(-o for o in off), axis=tuple(range(d))).reshape(-1) for off in offs]
    return np.stack(cols, axis=1)
