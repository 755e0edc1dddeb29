"""The 1D path on the GPU: the one-dimensional example of Sec. 4.1 (the decay of (QG)[j, :]
away from j) and the single shift of Sec. 3 as a baseline, against the CPU oracle."""

import numpy as np
import pytest
import scipy.sparse

import oracle as O
from lsp_inputs import gaussian_source, make_workload

pytestmark = pytest.mark.gpu
U = 2.0 ** -53
_STREAM = []


def ctx_for(v):
    import torch
    from paper_1607_02560_gb300 import Context, build
    build.build()
    if not _STREAM:
        _STREAM.append(torch.cuda.Stream())
    return Context(v.ndim, v.shape[0], stream=_STREAM[0])


def tols(n, s):
    st = O.stencil_for_shift(n, 1, float(s))
    w = np.linalg.eigvalsh(st["A"])
    kappa = np.abs(w).max() / max(w[1] - w[0], 1e-300)
    ta = max(1e-10, 16 * U * kappa)
    Gm = O.gather_offsets(st["g"], O.neighbourhood_offsets(1), n)
    tc = ta * np.abs(Gm).sum(axis=0).max() + 1e-13 * np.abs(st["c"]).max()
    return st, ta, tc


@pytest.mark.parametrize("policy", ["local", "paper", "mean"])
@pytest.mark.parametrize("n", [64, 256])
def test_1d_stencils_match_oracle(policy, n):
    v = make_workload("helm1d_n256", n=n)
    ctx = ctx_for(v)
    ctx.set_potential(v)
    ctx.build_stencils(policy=policy)
    assert ctx.mu == 3
    tab = ctx.get_shift_table()
    ref = O.build_stencils(v, policy)
    assert np.array_equal(tab["s"], ref["S"])
    assert np.array_equal(tab["s_idx"], ref["s_idx"].reshape(-1))
    ta_max = tc_max = 0.0
    for i, s in enumerate(ref["S"]):
        st, ta, tc = tols(n, s)
        assert np.abs(tab["alpha"][i] - st["alpha"]).max() <= ta
        assert np.abs(tab["c"][i] - st["c"]).max() <= tc
        ta_max, tc_max = max(ta_max, ta), max(tc_max, tc)
    Q, C, P = (ctx.get_rows(k) for k in "QCP")
    assert np.abs(Q - ref["Q"]).max() <= ta_max
    assert np.abs(C - ref["C"]).max() <= tc_max
    vm = np.abs(v).max() + np.abs(ref["S"]).max()
    assert np.abs(P - ref["P"]).max() <= ta_max + tc_max * vm + 1e-13 * np.abs(ref["P"]).max()


def test_qg_row_decays_away_from_j():
    """The 1D example of Sec. 4.1: n = 32, s = -62 pi^2 (lattice index m = -16), j = 16.
    With the GPU's alpha, (QG)[j, :] = sum_a alpha_a G_s[j + o_a, :] is large only at the
    three columns of mu_j and decays away from them, and equals the oracle's row."""
    n, j = 32, 16
    s = -62 * O.PI2
    v = np.full(n, s)
    ctx = ctx_for(v)
    ctx.set_potential(v)
    ctx.build_stencils(policy="local")
    tab = ctx.get_shift_table()
    assert len(tab["s"]) == 1 and tab["s"][0] == s
    G = O.dense_green_matrix(n, 1, s)
    offs = O.neighbourhood_offsets(1)

    def qg_row(alpha):
        row = np.zeros(n)
        for a, o in enumerate(offs):
            row += alpha[a] * G[int((j + o[0]) % n)]
        return row

    gpu = qg_row(tab["alpha"][0])
    ref = qg_row(O.stencil_for_shift(n, 1, s)["alpha"])
    assert np.abs(gpu - ref).max() <= 1e-10 * np.abs(ref).max()
    dist = np.abs(np.arange(n) - j)
    prof = np.abs(gpu)
    print("|QG[16, j]|:", " ".join(f"{x:.2e}" for x in prof))
    assert prof[dist <= 1].max() > prof[dist >= 2].max()
    assert prof[dist >= 8].max() < prof[dist == 2].max()


def test_apply_operator_1d_plane_waves():
    import torch
    n = 64
    v = np.full(n, 3.5)
    ctx = ctx_for(v)
    ctx.set_potential(v)
    x = np.arange(n) / n
    for k in (1, 5, n // 2 - 1):
        u = np.cos(2 * np.pi * k * x)
        ud = torch.from_numpy(u).cuda()
        yd = torch.empty_like(ud)
        ctx.apply_operator(ud, yd)
        ctx.synchronize()
        lam = 4 * O.PI2 * k * k + 3.5
        assert np.abs(yd.cpu().numpy() - lam * u).max() <= 1e-12 * lam


def test_single_shift_of_section3_is_the_weaker_baseline():
    """|S| = 1 (snap(mean v), Sec. 3) against every point's own shift (Sec. 4.1) in 1D."""
    v = make_workload("helm1d_n256")
    n = 256
    f = gaussian_source(n, 1, 2.0)
    ctx = ctx_for(v)
    ctx.set_potential(v)
    counts = {}
    for pol in ("mean", "local"):
        ctx.build_stencils(policy=pol)
        mats = {}
        for which in "CP":
            rowptr, colidx, vals = ctx.export_sparse_rows(which)
            mats[which] = scipy.sparse.csr_matrix((vals, colidx, rowptr), shape=(n, n))
        _, it, res, info = O.gmres_solve(v, f, mats["P"], mats["C"], maxiter=5)
        counts[pol] = it if info == 0 else 201
    print("1D GMRES iterations:", counts)
    assert counts["local"] <= 12
    assert counts["mean"] >= counts["local"]
