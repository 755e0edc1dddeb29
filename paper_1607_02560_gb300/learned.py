"""Training driver of the learned-stencil network (argument marshalling around liblsp.so).

The training data are the stencils the eigen path itself produces: for every training potential
the library builds all stencils (FP64), then samples (patch, stencil) pairs from that build on
the device. Pairs from different potentials are interleaved in chunks so that every batch mixes
several potentials. All arithmetic (pair sampling, normalisation statistics, forward, backward,
Adam) runs in the library's kernels; torch only holds the device buffers.
"""

from __future__ import annotations

import time

import numpy as np

from .lsp import Context, Mlp

CHUNK = 1024


def make_pool(mlp: Mlp, potentials, samples_per_potential: int, stream, seed: int = 0):
    """Device pool of raw training pairs, interleaved by chunks of CHUNK samples."""
    import torch

    P = len(potentials)
    per = (samples_per_potential // CHUNK) * CHUNK
    total = P * per
    X = torch.empty((total, mlp.nf), dtype=torch.float32, device="cuda")
    T = torch.empty((total, mlp.out), dtype=torch.float32, device="cuda")
    nch = per // CHUNK
    ctx = None
    for pi, v in enumerate(potentials):
        if ctx is None or ctx.n != v.shape[0]:
            ctx = Context(v.ndim, v.shape[0], stream=stream)
        ctx.set_potential(v)
        ctx.build_stencils(policy="local")
        for c in range(nch):
            row = (c * P + pi) * CHUNK
            mlp.training_pairs(ctx, CHUNK, seed * 1000003 + pi * 7919 + c, X[row:row + CHUNK],
                               T[row:row + CHUNK])
    return X, T


def train(mlp: Mlp, X, T, steps: int, batch: int = 4096, lr: float = 2e-3, lr_final: float = 1e-4,
          log_every: int = 0):
    """Adam on contiguous batches of the interleaved pool, cosine-decayed learning rate."""
    n = X.shape[0]
    nb = n // batch
    losses = []
    t0 = time.time()
    for s in range(steps):
        b = s % nb
        rate = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * s / max(steps - 1, 1)))
        loss = mlp.train_step(X[b * batch:(b + 1) * batch], T[b * batch:(b + 1) * batch], batch,
                              float(rate))
        losses.append(loss)
        if log_every and s % log_every == 0:
            print(f"step {s} loss {loss:.3e} ({time.time() - t0:.1f}s)")
    return losses


def train_surrogate(d: int, potentials, samples_per_potential: int = 65536, steps: int = 3000,
                    batch: int = 4096, lr: float = 2e-3, seed: int = 0, stream=None,
                    log_every: int = 0):
    """A network trained on the eigen-path stencils of `potentials`."""
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    mlp = Mlp(d, seed=seed, stream=stream)
    X, T = make_pool(mlp, potentials, samples_per_potential, stream, seed)
    torch.cuda.synchronize()
    mlp.fit_normalization(X, T, X.shape[0])
    losses = train(mlp, X, T, steps, batch=batch, lr=lr, log_every=log_every)
    return mlp, losses
