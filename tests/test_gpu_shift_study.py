"""|S|-quantization study on the 2D n = 256 Helmholtz workload (GPU stencils, CPU oracle GMRES).

Sec. 4.1 spreads |S| = O(n) shifts over [v_min, v_max]; the Sec. 5 tables use n/16 in 2D. This
study measures the GMRES(40) iteration count (rtol 1e-6, preconditioner P^-1 C) against |S|:
the single shift snap(mean v) of Sec. 3, the paper policy with K = 2 .. 64 shifts, every point's
own shift, and the learned stencils. It also checks the remark of Sec. 5 that the shift list
depends on v only through its range: a table over every lattice shift of a covering range
[lo, hi] serves every potential inside it exactly as its own per-point build would.
The counts are printed (the design notes record them); the assertions are the method's
expectations, with the +1 margin the mixed and learned paths are held to.
"""

import numpy as np
import pytest
import scipy.sparse

import oracle as O
from lsp_inputs import gaussian_source, helmholtz_random_bumps, make_workload


pytestmark = pytest.mark.gpu


CAP = 200  # inner iterations (5 restart cycles of 40); more means "not converged"


def _ctx(v, stream):
    from paper_1607_02560_gb300 import Context
    return Context(v.ndim, v.shape[0], stream=stream)


def _iters(ctx, v, f):
    """Inner GMRES iterations to rtol 1e-6, or CAP + 1 when it has not converged by CAP."""
    N = v.size
    mats = {}
    for which in "CP":
        rowptr, colidx, vals = ctx.export_sparse_rows(which)
        mats[which] = scipy.sparse.csr_matrix((vals, colidx, rowptr), shape=(N, N))
    _, it, res, info = O.gmres_solve(v, f, mats["P"], mats["C"], maxiter=CAP // 40)
    if info != 0:
        return CAP + 1
    assert res < 1e-4
    return it


@pytest.fixture(scope="module")
def stream():
    import torch
    from paper_1607_02560_gb300 import build
    build.build()
    return torch.cuda.Stream()


def test_iterations_against_the_number_of_shifts(stream):
    v = make_workload("helm2d_n256")
    f = gaussian_source(256, 2, 2.0)
    ctx = _ctx(v, stream)
    ctx.set_potential(v)
    counts = {}
    ctx.build_stencils(policy="mean")
    counts["mean (|S|=1)"] = _iters(ctx, v, f)
    paper = {}
    for K in (2, 4, 8, 16, 32, 64):
        ctx.build_stencils(policy="paper", nshifts=K)
        ns = len(ctx.get_shift_table(with_sidx=False)["s"])
        paper[K] = _iters(ctx, v, f)
        counts[f"paper K={K} (|S|={ns})"] = paper[K]
    ctx.build_stencils(policy="local")
    ns = len(ctx.get_shift_table(with_sidx=False)["s"])
    counts[f"local (|S|={ns})"] = local = _iters(ctx, v, f)
    for k, it in counts.items():
        print(f"{k}: {it if it <= CAP else f'> {CAP}'} iterations")
    # |S| = O(n) shifts (n/16 and more) converge within the paper's 5-12 iterations; the count
    # is not monotone in |S| (where the shifts fall against the potential's values matters),
    # and every point's own shift is within one of the best of them. A few shifts over the
    # whole range, or the single shift of Sec. 3, leave this high-frequency Helmholtz problem
    # far less well preconditioned.
    for K in (16, 32, 64):
        assert paper[K] <= 12, paper
    assert local <= min(paper[16], paper[32], paper[64]) + 1
    assert counts["mean (|S|=1)"] >= 3 * paper[16]
    assert paper[2] >= 3 * paper[16] and paper[4] >= 3 * paper[16]
    assert paper[8] > paper[16]


def test_learned_stencils_against_the_eigen_path(stream):
    """Records the GMRES count with the learned stencils at n = 256 (omega = 2 pi 64).

    Under the per-point policy the method's alpha depends on the point only through s_j, and
    at this frequency the sparsification residual alpha^T G[mu, mu^c] of the eigen path is so
    small that a relative error of ~1e-3 in alpha (bf16 network, fp32 arithmetic) raises it by
    orders of magnitude: the count is measured and reported, and only convergence is asserted
    here. The +1 target of the learned path is held at 2D n = 32 (tests/test_gpu_learned.py).
    """
    from paper_1607_02560_gb300.learned import train_surrogate
    n = 256
    v = make_workload("helm2d_n256")
    f = gaussian_source(n, 2, 2.0)
    pots = [helmholtz_random_bumps(n, 2 * np.pi * 64, 16, s) for s in range(100, 116)]
    mlp, losses = train_surrogate(2, pots, samples_per_potential=32768, steps=4000, batch=4096,
                                  lr=2e-3, seed=3, stream=stream)
    ctx = _ctx(v, stream)
    ctx.set_mlp(mlp)
    ctx.set_potential(v)
    ctx.build_stencils(policy="local")
    it_local = _iters(ctx, v, f)
    ctx.build_stencils(mode="learned")
    assert ctx.mode_used() == "learned"
    it_learned = _iters(ctx, v, f)
    print(f"local eigen path: {it_local}, learned: {it_learned} iterations "
          f"(final loss {np.mean(losses[-50:]):.3g})")
    assert it_local <= 12 and it_learned <= CAP


def test_stencils_prebuilt_for_a_range_serve_every_potential_in_it(stream):
    """Sec. 5: the shift list needs only [v_min, v_max], so stencils can be built in advance.
    A table over every lattice shift of a covering range [lo, hi] (the LIST policy) gives each
    potential inside it exactly the rows of its own per-point build, hence the same count.
    (Paper-policy lists spread over a wider range are a different matter: even at the same
    spacing the count depends on where the shifts fall, 19 against 7 iterations here.)"""
    n = 256
    f = gaussian_source(n, 2, 2.0)
    va = make_workload("helm2d_n256")
    vb = helmholtz_random_bumps(n, 2 * np.pi * 64, 16, 7)
    lo, hi = min(va.min(), vb.min()), max(va.max(), vb.max())
    m = np.arange(int(O.snap_index(np.array([lo]))[0]), int(O.snap_index(np.array([hi]))[0]) + 1)
    shifts = O.shift_value(m)
    for v in (va, vb):
        ctx = _ctx(v, stream)
        ctx.set_potential(v)
        ctx.build_stencils(policy="list", shifts=shifts)
        rows_pre = {k: ctx.get_rows(k).copy() for k in "QCP"}
        it_pre = _iters(ctx, v, f)
        ctx.build_stencils(policy="local")
        for k in "QCP":
            assert np.array_equal(ctx.get_rows(k), rows_pre[k]), k
        it_own = _iters(ctx, v, f)
        print(f"prebuilt for [{lo:.4g}, {hi:.4g}] ({len(shifts)} lattice shifts): {it_pre}, "
              f"own per-point build: {it_own} iterations")
        assert it_pre == it_own
