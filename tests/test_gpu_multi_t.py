"""Multi-t stencils on the GPU (Sec. 4.2) against the CPU oracle.

* t = 2 (5 x 5 neighbourhoods in 2D, 5 x 5 x 5 in 3D) at every point: per-shift alpha, c,
  lambda_1 and the rows;
* per-point t_j from the nested-dissection geometry (leaf width 8, t_max = 2): the CSR export
  has the oracle's exact pattern (rows of 9 or 25 entries) and its values within the
  tolerances of the FP64 path;
* the oracle GMRES counts with the GPU's multi-t P and C equal the stored golden counts;
* the unsupported combinations fail cleanly.
"""

import json
import os

import numpy as np
import pytest
import scipy.sparse

import oracle as O
from lsp_inputs import gaussian_source, make_workload

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U = 2.0 ** -53
_STREAM = []


def ctx_for(v):
    import torch
    from paper_1607_02560_gb300 import Context, build
    build.build()
    if not _STREAM:
        _STREAM.append(torch.cuda.Stream())
    return Context(v.ndim, v.shape[0], stream=_STREAM[0])


def tols(n, d, s, t):
    """tol_alpha = max(1e-10, 16 u kappa_gap) and its propagation to c (as for t = 1)."""
    st = O.stencil_for_shift(n, d, float(s), t)
    w = np.linalg.eigvalsh(st["A"])
    kappa = np.abs(w).max() / max(w[1] - w[0], 1e-300)
    ta = max(1e-10, 16 * U * kappa)
    Gm = O.gather_offsets(st["g"], O.neighbourhood_offsets(d, t), n)
    tc = ta * np.abs(Gm).sum(axis=0).max() + 1e-13 * np.abs(st["c"]).max()
    return st, ta, tc


def csr(ctx, which, N):
    rowptr, colidx, vals = ctx.export_sparse_rows(which)
    return scipy.sparse.csr_matrix((vals, colidx, rowptr), shape=(N, N))


@pytest.mark.parametrize("policy", ["paper", "local"])
def test_t2_everywhere_matches_oracle(policy):
    v = make_workload("helm2d_n32")
    n, d = 32, 2
    ctx = ctx_for(v)
    ctx.set_potential(v)
    ctx.build_stencils(policy=policy, t=2)
    assert ctx.mu == 25
    tab = ctx.get_shift_table()
    ref = O.build_stencils(v, policy, t=2)
    assert np.array_equal(tab["s"], ref["S"])
    worst = {}
    for i, s in enumerate(ref["S"]):
        st, ta, tc = tols(n, d, s, 2)
        assert np.abs(tab["alpha"][i] - st["alpha"]).max() <= ta, i
        assert np.abs(tab["c"][i] - st["c"]).max() <= tc, i
        assert abs(tab["lam"][i, 0] - st["lam1"]) <= 1e-9 * np.abs(st["A"]).max()
        assert not (tab["flags"][i] & 4)
        worst[i] = (ta, tc)
    # rows: Q, C exactly the table entries of each point's shift, P by the formula
    Q, C, P = (ctx.get_rows(k) for k in "QCP")
    sidx = tab["s_idx"].astype(np.int64)
    assert np.array_equal(Q, tab["alpha"][sidx]) and np.array_equal(C, tab["c"][sidx])
    ta_max = max(a for a, _ in worst.values())
    tc_max = max(c for _, c in worst.values())
    assert np.abs(Q - ref["Q"]).max() <= ta_max
    assert np.abs(C - ref["C"]).max() <= tc_max
    vmax = np.abs(v).max() + np.abs(ref["S"]).max()
    assert np.abs(P - ref["P"]).max() <= ta_max + tc_max * vmax + 1e-13 * np.abs(ref["P"]).max()


@pytest.mark.parametrize("policy,n", [("paper", 32), ("local", 32), ("paper", 64)])
def test_multi_t_rows_match_oracle(policy, n):
    v = make_workload("helm2d_n32", n=n)
    d = 2
    ctx = ctx_for(v)
    ctx.set_potential(v)
    ctx.build_stencils(policy=policy, t=2, nd_leaf=8)
    ref = O.build_stencils_multi(v, policy, leaf=8, t_max=2)
    N = n * n
    ta_max = tc_max = 0.0
    for s in ref["S"]:
        for t in (1, 2):
            _, ta, tc = tols(n, d, s, t)
            ta_max, tc_max = max(ta_max, ta), max(tc_max, tc)
    vmax = np.abs(v).max() + np.abs(ref["S"]).max()
    for which, tol in (("Q", ta_max), ("C", tc_max),
                       ("P", ta_max + tc_max * vmax + 1e-13 * np.abs(ref["P"].data).max())):
        got, want = csr(ctx, which, N), ref[which]
        # the same sparsity pattern, entry by entry (rows of 9 or 25 entries, offset order)
        assert np.array_equal(got.indptr, want.indptr), which
        assert np.array_equal(got.indices, want.indices), which
        assert np.abs(got.data - want.data).max() <= tol, which
    lens = np.diff(csr(ctx, "Q", N).indptr)
    assert set(lens.tolist()) == {9, 25}


def test_multi_t_gmres_counts_match_golden():
    with open(os.path.join(GOLDEN, "gmres_multi_t_helm2d_n32.json")) as fh:
        gold = json.load(fh)["iterations"]
    v = make_workload("helm2d_n32")
    f = gaussian_source(32, 2, 2.0)
    ctx = ctx_for(v)
    ctx.set_potential(v)
    for key, want in gold.items():
        pol, label = key.split("/")
        ctx.build_stencils(policy=pol, t=2, nd_leaf=8 if label == "nd8" else 0)
        P, C = csr(ctx, "P", 1024), csr(ctx, "C", 1024)
        _, it, res, info = O.gmres_solve(v, f, P, C)
        assert info == 0 and it == want and res < 1e-4, (key, it, want)


def test_t2_switches_back_to_t1_and_graph_replay():
    from paper_1607_02560_gb300 import LspError  # noqa: F401
    v = make_workload("helm2d_n32")
    ctx = ctx_for(v)
    ctx.set_potential(v)
    ctx.build_stencils(policy="paper", t=1)
    q1 = ctx.get_rows("Q").copy()
    for _ in range(2):
        ctx.build_stencils(policy="paper", t=2, nd_leaf=8, use_graph=True)
    ctx.synchronize()
    assert ctx.mu == 25
    q2 = ctx.get_rows("Q").copy()
    ctx.build_stencils(policy="paper", t=2, nd_leaf=8)
    assert np.array_equal(ctx.get_rows("Q"), q2)
    ctx.build_stencils(policy="paper", t=1, use_graph=True)
    ctx.synchronize()
    assert ctx.mu == 9 and np.array_equal(ctx.get_rows("Q"), q1)


@pytest.mark.parametrize("policy", ["paper", "local"])
def test_t2_3d_everywhere_matches_oracle(policy):
    """3D t = 2 (125-point neighbourhoods, 35 classes): per-shift alpha, c and lambda_1 of the
    dense near-null solve, and the rows, against the oracle."""
    n, d = 16, 3
    v = make_workload("schr3d_n64", n=n)
    ctx = ctx_for(v)
    ctx.set_potential(v)
    ctx.build_stencils(policy=policy, t=2)
    assert ctx.mu == 125
    tab = ctx.get_shift_table()
    ref = O.build_stencils(v, policy, t=2)
    assert np.array_equal(tab["s"], ref["S"])
    ta_max = tc_max = 0.0
    for i, s in enumerate(ref["S"]):
        st, ta, tc = tols(n, d, s, 2)
        assert np.abs(tab["alpha"][i] - st["alpha"]).max() <= ta, i
        assert np.abs(tab["c"][i] - st["c"]).max() <= tc, i
        assert abs(tab["lam"][i, 0] - st["lam1"]) <= 1e-9 * np.abs(st["A"]).max()
        assert not (tab["flags"][i] & 4)
        ta_max, tc_max = max(ta_max, ta), max(tc_max, tc)
    Q, C, P = (ctx.get_rows(k) for k in "QCP")
    sidx = tab["s_idx"].astype(np.int64)
    assert np.array_equal(Q, tab["alpha"][sidx]) and np.array_equal(C, tab["c"][sidx])
    assert np.abs(Q - ref["Q"]).max() <= ta_max
    assert np.abs(C - ref["C"]).max() <= tc_max
    vmax = np.abs(v).max() + np.abs(ref["S"]).max()
    assert np.abs(P - ref["P"]).max() <= ta_max + tc_max * vmax + 1e-13 * np.abs(ref["P"]).max()


def test_multi_t_3d_rows_nd_and_gmres_match_oracle():
    """3D multi-t (t_j from leaf-8 boxes, rows of 27 or 125 entries): the CSR export against the
    oracle, the nested dissection of these rows, and the GMRES count with them."""
    n, d = 16, 3
    v = make_workload("schr3d_n64", n=n)
    N = n ** d
    ctx = ctx_for(v)
    ctx.set_potential(v)
    ctx.build_stencils(policy="paper", t=2, nd_leaf=8)
    ref = O.build_stencils_multi(v, "paper", leaf=8, t_max=2)
    ta_max = tc_max = 0.0
    for s in ref["S"]:
        for t in (1, 2):
            _, ta, tc = tols(n, d, s, t)
            ta_max, tc_max = max(ta_max, ta), max(tc_max, tc)
    vmax = np.abs(v).max() + np.abs(ref["S"]).max()
    for which, tol in (("Q", ta_max), ("C", tc_max),
                       ("P", ta_max + tc_max * vmax + 1e-13 * np.abs(ref["P"].data).max())):
        got, want = csr(ctx, which, N), ref[which]
        assert np.array_equal(got.indptr, want.indptr), which
        assert np.array_equal(got.indices, want.indices), which
        assert np.abs(got.data - want.data).max() <= tol, which
    assert set(np.diff(csr(ctx, "Q", N).indptr).tolist()) == {27, 125}
    ctx.nd_factor()
    f = gaussian_source(n, d, 2.0)
    _, res = ctx.gmres(f.reshape(-1))
    _, it, _, info = O.gmres_solve(v, f, csr(ctx, "P", N), csr(ctx, "C", N), maxiter=5)
    print(f"3D multi-t n=16: GPU {res}, oracle {it} iterations")
    assert info == 0 and res["converged"] == 1 and res["iterations"] == it


def test_unsupported_combinations_fail_cleanly():
    from paper_1607_02560_gb300 import LspError
    v1 = make_workload("helm1d_n256", n=64)
    ctx1 = ctx_for(v1)
    ctx1.set_potential(v1)
    with pytest.raises(LspError, match="UNSUPPORTED"):
        ctx1.build_stencils(t=2)
    v = make_workload("helm2d_n32")
    ctx = ctx_for(v)
    ctx.set_potential(v)
    for kw in ({"t": 3}, {"t": 2, "nd_leaf": 3}, {"t": 2, "nd_leaf": -1}):
        with pytest.raises(LspError, match="ARG"):
            ctx.build_stencils(**kw)
    ctx.build_stencils(policy="paper", t=2, nd_leaf=8)  # still usable after the errors
    assert ctx.mu == 25


def test_full_size_2d_n1024_multi_t_sampled():
    """Paper policy, t_j from leaf-8 boxes at n = 1024: sampled shifts against the oracle, and
    every row of the export equal to its shift's stencil (by t_j) by the formula of Sec. 4.1."""
    v = make_workload("helm2d_n1024")
    n, d = 1024, 2
    ctx = ctx_for(v)
    ctx.set_potential(v)
    ctx.build_stencils(policy="paper", t=2, nd_leaf=8)
    tab = ctx.get_shift_table()
    rng = np.random.default_rng(0)
    for i in rng.choice(len(tab["s"]), size=3, replace=False):
        st, ta, tc = tols(n, d, tab["s"][i], 2)
        assert np.abs(tab["alpha"][i] - st["alpha"]).max() <= ta
        assert np.abs(tab["c"][i] - st["c"]).max() <= tc
    # rows of the t_j = 2 points are the table's alpha/c at the point's shift
    T = O.t_choice(n, d, 8, 2).reshape(-1)
    Q = ctx.get_rows("Q")
    sidx = tab["s_idx"].astype(np.int64)
    two = np.nonzero(T == 2)[0]
    assert np.array_equal(Q[two], tab["alpha"][sidx[two]])
    one = np.nonzero(T == 1)[0]
    inner = [(a + 2) * 5 + (b + 2) for a in (-1, 0, 1) for b in (-1, 0, 1)]
    outer = sorted(set(range(25)) - set(inner))
    assert np.all(Q[np.ix_(one, outer)] == 0.0)
    assert np.allclose(np.linalg.norm(Q[np.ix_(one, inner)], axis=1), 1.0, atol=1e-12)
