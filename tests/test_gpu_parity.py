"""GPU path (liblsp.so through the C ABI) against the CPU oracle.

Tolerances. The near-null vector alpha of A = A1 - A2 (Eq. A) moves by about u * kappa under
a rounding-level change of A, with kappa = max|lambda| / (lambda_2 - lambda_1) and u = 2^-53;
the oracle itself shows this spread when its inverse-FFT kernel vectors are replaced by
long-double direct sums. So alpha is compared entrywise with
    tol_alpha = max(1e-10, 16 u kappa)
(kappa <= ~600 in 2D, so 1e-10 there; ~2e6 in 3D), and c = G alpha and the P rows inherit
the bound through their formulas:
    tol_c = tol_alpha * max_b sum_a |G[a, b]| + 1e-13 max|c|,
    tol_P = tol_alpha + tol_c * max|v[mu_j] - s_j| + 1e-13 max|P|.
Shift lists, per-point shift indices and CSR patterns are integer results: compared exactly.
"""

import numpy as np
import pytest

import oracle as O
from lsp_inputs import gaussian_source, make_workload

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1607_02560_gb300 import build as B
    B.build()


_STREAM = []


def ctx_for(v):
    """A context on a dedicated (non-default) stream, as the benchmark uses."""
    import torch
    from paper_1607_02560_gb300 import Context
    if not _STREAM:
        _STREAM.append(torch.cuda.Stream())
    return Context(v.ndim, v.shape[0], stream=_STREAM[0])


def shift_tols(n, d, s):
    st = O.stencil_for_shift(n, d, float(s))
    w = np.linalg.eigvalsh(st["A"])
    kappa = np.abs(w).max() / max(w[1] - w[0], 1e-300)
    ta = max(1e-10, 16 * U * kappa)
    offs = O.neighbourhood_offsets(d)
    Gm = O.gather_offsets(st["g"], offs, n)
    tc = ta * np.abs(Gm).sum(axis=0).max() + 1e-13 * np.abs(st["c"]).max()
    return st, ta, tc


def check_shift_table(tab, v, policy, nshifts=None, m_list=None, sample=None):
    n, d = v.shape[0], v.ndim
    ref = O.build_stencils(v, policy, nshifts=nshifts, m_list=m_list, shift_subset=[])
    assert np.array_equal(tab["s"], ref["S"]), "shift list differs"
    assert np.array_equal(tab["s_idx"].reshape(v.shape), ref["s_idx"]), "s_j differs"
    idx = range(len(ref["S"])) if sample is None else sample
    tols = {}
    for i in idx:
        st, ta, tc = shift_tols(n, d, ref["S"][i])
        ea = np.abs(tab["alpha"][i] - st["alpha"]).max()
        ec = np.abs(tab["c"][i] - st["c"]).max()
        assert ea <= ta, (i, ea, ta)
        assert ec <= tc, (i, ec, tc)
        assert abs(tab["lam"][i, 0] - st["lam1"]) <= 1e-9 * np.abs(st["A"]).max()
        tols[i] = (ta, tc)
    return ref, tols


def check_rows(ctx, v, ref, tols):
    """Rows at every point whose shift has an oracle stencil in `tols`."""
    d = v.ndim
    offs = O.neighbourhood_offsets(d)
    Q, C, P = (ctx.get_rows(k) for k in "QCP")
    sidx = ref["s_idx"].reshape(-1)
    vnb = np.stack([np.roll(v, tuple(-o for o in off), axis=tuple(range(d))) for off in offs],
                   axis=-1).reshape(-1, len(offs))
    checked = 0
    for i, (ta, tc) in tols.items():
        pts = np.nonzero(sidx == i)[0]
        if len(pts) == 0:
            continue
        st = O.stencil_for_shift(v.shape[0], d, float(ref["S"][i]))
        s = ref["S"][i]
        eP = st["alpha"][None, :] + st["c"][None, :] * (vnb[pts] - s)
        tp = ta + tc * np.abs(vnb[pts] - s).max() + 1e-13 * np.abs(eP).max()
        assert np.abs(Q[pts] - st["alpha"]).max() <= ta
        assert np.abs(C[pts] - st["c"]).max() <= tc
        assert np.abs(P[pts] - eP).max() <= tp
        checked += len(pts)
    return checked


def rows_consistent_with_table(ctx, v, tab):
    """Every row equals the formula of Sec. 4.1 applied to the GPU's own shift table."""
    d = v.ndim
    offs = O.neighbourhood_offsets(d)
    Q, C, P = (ctx.get_rows(k) for k in "QCP")
    sidx = tab["s_idx"].astype(np.int64)
    assert np.array_equal(Q, tab["alpha"][sidx])
    assert np.array_equal(C, tab["c"][sidx])
    vnb = np.stack([np.roll(v, tuple(-o for o in off), axis=tuple(range(d))) for off in offs],
                   axis=-1).reshape(-1, len(offs))
    eP = tab["alpha"][sidx] + tab["c"][sidx] * (vnb - tab["s"][sidx][:, None])
    assert np.abs(P - eP).max() <= 4e-16 * (np.abs(eP).max() + np.abs(tab["c"]).max()
                                             * np.abs(vnb).max())


SMALL = [("helm2d_n32", 8), ("helm2d_n32", 16), ("helm2d_n32", 32), ("helm2d_n256", 64),
         ("schr3d_n64", 8), ("schr3d_n64", 16)]


@pytest.mark.parametrize("name,n", SMALL)
@pytest.mark.parametrize("policy", ["local", "paper", "mean"])
def test_small_parity(name, n, policy):
    v = make_workload(name, n=n)
    ctx = ctx_for(v)
    ctx.set_potential(v)
    ctx.build_stencils(policy=policy)
    tab = ctx.get_shift_table()
    ref, tols = check_shift_table(tab, v, policy)
    assert check_rows(ctx, v, ref, tols) == v.size
    rows_consistent_with_table(ctx, v, tab)


@pytest.mark.parametrize("name,n", [("helm2d_n256", 64), ("schr3d_n64", 16)])
def test_full_jacobi_and_refinement_match(name, n):
    v = make_workload(name, n=n)
    ctx = ctx_for(v)
    ctx.set_potential(v)
    for kw in (dict(eig_method="full"), dict(refine_steps=1),
               dict(eig_method="full", refine_steps=1)):
        ctx.build_stencils(policy="local", **kw)
        tab = ctx.get_shift_table()
        check_shift_table(tab, v, "local")
        assert not np.any(tab["flags"] & 4)


def test_list_policy_and_errors():
    import torch
    from paper_1607_02560_gb300 import LspError
    v = make_workload("helm2d_n32", n=16)
    ctx = ctx_for(v)
    with pytest.raises(LspError) as e:
        ctx.build_stencils()
    assert e.value.status == 2  # build before set_potential
    bad = v.copy()
    bad[3, 4] = np.nan
    with pytest.raises(LspError) as e:
        ctx.set_potential(bad)
    assert e.value.status == 1
    ctx.set_potential(torch.from_numpy(v).cuda())
    m = np.array([-20, -15, -9])
    ctx.build_stencils(policy="list", shifts=O.shift_value(m))
    tab = ctx.get_shift_table()
    ref, tols = check_shift_table(tab, v, "list", m_list=m)
    assert check_rows(ctx, v, ref, tols) == v.size
    with pytest.raises(LspError) as e:  # -4 pi^2 * 5 = -4 pi^2 |(1, 2)|^2: resonant
        ctx.build_stencils(policy="list", shifts=[-20 * O.PI2])
    assert e.value.status == 3
    with pytest.raises(LspError) as e:
        ctx.build_stencils(policy="list", shifts=[-21.5 * O.PI2])
    assert e.value.status == 1


def test_graph_replay_is_bit_identical():
    v = make_workload("helm2d_n256", n=64)
    ctx = ctx_for(v)
    ctx.set_potential(v)
    ctx.build_stencils(policy="local")
    ref = [ctx.get_rows(k).copy() for k in "QCP"]
    for _ in range(3):
        ctx.build_stencils(policy="local", use_graph=True)
        for k, r in zip("QCP", ref):
            assert np.array_equal(ctx.get_rows(k), r)
    # switching precision in between must not leave a stale reciprocal table behind
    ctx.build_stencils(policy="local", mode="mixed", use_graph=True)
    mixed = ctx.get_rows("Q").copy()
    ctx.build_stencils(policy="local", use_graph=True)
    for k, r in zip("QCP", ref):
        assert np.array_equal(ctx.get_rows(k), r)
    ctx.build_stencils(policy="local", mode="mixed")
    assert np.array_equal(ctx.get_rows("Q"), mixed)


@pytest.mark.parametrize("name,n", [("helm2d_n32", 32), ("helm2d_n256", 256),
                                    ("schr3d_n64", 16), ("schr3d_n64", 32)])
def test_apply_operator(name, n):
    import torch
    v = make_workload(name, n=n)
    d = v.ndim
    ctx = ctx_for(v)
    ctx.set_potential(v)
    rng = np.random.default_rng(7)
    u = rng.standard_normal(v.shape)
    y = torch.empty(v.shape, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    ctx.apply_operator(torch.from_numpy(u).cuda(), y)
    ctx.synchronize()  # the context works on its own stream
    ref = O.apply_operator(v, u)
    scale = (4 * O.PI2 * d * (n / 2) ** 2 + np.abs(v).max()) * np.abs(u).max()
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-13 * scale
    # plane wave with constant v: eigenvalue 4 pi^2 |k|^2 + v
    vc = np.full(v.shape, -321.5)
    ctx.set_potential(vc)
    x = np.meshgrid(*([np.arange(n) / n] * d), indexing="ij")
    k = np.arange(1, d + 1) * max(1, n // 16)  # |k_i| <= n/2: no aliasing
    uw = np.cos(2 * np.pi * sum(ki * xi for ki, xi in zip(k, x)))
    torch.cuda.synchronize()
    ctx.apply_operator(torch.from_numpy(uw).cuda(), y)
    ctx.synchronize()
    lam = 4 * O.PI2 * float((k ** 2).sum()) - 321.5
    # FFT rounding is amplified by the largest symbol value, as for the random input above
    scale_c = (4 * O.PI2 * d * (n / 2) ** 2 + 321.5) * np.abs(uw).max()
    assert np.abs(y.cpu().numpy() - lam * uw).max() <= 1e-13 * scale_c


@pytest.mark.parametrize("name,n,policy", [("helm2d_n32", 32, "local"), ("schr3d_n64", 8, "paper")])
def test_export_csr(name, n, policy):
    v = make_workload(name, n=n)
    ctx = ctx_for(v)
    ctx.set_potential(v)
    ctx.build_stencils(policy=policy)
    for which in "QCP":
        rowptr, colidx, vals = ctx.export_sparse_rows(which)
        rows = ctx.get_rows(which)
        ref = O.rows_to_csr(rows, n, v.ndim)
        assert np.array_equal(rowptr, ref.indptr)
        assert np.array_equal(colidx, ref.indices)
        assert np.array_equal(vals, rows.reshape(-1))


def test_gmres_counts_unchanged_with_gpu_stencils():
    import json
    import os
    import scipy.sparse
    with open(os.path.join(os.path.dirname(__file__), "golden", "gmres_helm2d_n32.json")) as fh:
        gold = json.load(fh)["iterations"]
    v = make_workload("helm2d_n32")
    n = 32
    ctx = ctx_for(v)
    ctx.set_potential(v)
    for pol in ("local", "paper", "mean"):
        ctx.build_stencils(policy=pol)
        mats = {}
        for which in "CP":
            rowptr, colidx, vals = ctx.export_sparse_rows(which)
            mats[which] = scipy.sparse.csr_matrix((vals, colidx, rowptr), shape=(n * n, n * n))
        _, it, res, info = O.gmres_solve(v, gaussian_source(n, 2, 2.0), mats["P"], mats["C"])
        assert info == 0 and it == gold[f"{pol}/2.0"], (pol, it)


# ---- full sizes, in the launch configuration of the benchmark (graph replay) -------------

def test_full_size_2d_n1024_sampled():
    v = make_workload("helm2d_n1024")
    ctx = ctx_for(v)
    ctx.set_potential(v)
    for _ in range(2):
        ctx.build_stencils(policy="local", use_graph=True)
    tab = ctx.get_shift_table()
    # the shifts at v_min and v_max (the ends of the sorted list) and 40 seeded others
    rng = np.random.default_rng(11)
    ns = len(tab["s"])
    sample = sorted(set(rng.choice(np.arange(1, ns - 1), 40, replace=False).tolist())
                    | {0, ns - 1})
    ref, tols = check_shift_table(tab, v, "local", sample=sample)
    assert check_rows(ctx, v, ref, tols) > 0
    rows_consistent_with_table(ctx, v, tab)
    assert not np.any(tab["flags"] & 4)


def test_full_size_2d_n1024_paper_policy():
    v = make_workload("helm2d_n1024")
    ctx = ctx_for(v)
    ctx.set_potential(v)
    ctx.build_stencils(policy="paper", use_graph=True)
    tab = ctx.get_shift_table()
    sample = [0, len(tab["s"]) // 2, len(tab["s"]) - 1]
    ref, tols = check_shift_table(tab, v, "paper", sample=sample)
    assert check_rows(ctx, v, ref, tols) > 0
    rows_consistent_with_table(ctx, v, tab)


def test_full_size_3d_n64_all_shifts():
    v = make_workload("schr3d_n64")
    ctx = ctx_for(v)
    ctx.set_potential(v)
    ctx.build_stencils(policy="local", use_graph=True)
    tab = ctx.get_shift_table()
    ref, tols = check_shift_table(tab, v, "local")
    assert check_rows(ctx, v, ref, tols) == v.size


# ---- mixed precision (FP32 contractions and Gram, FP64 near-null solve) ------------------

U32 = 2.0 ** -24


@pytest.mark.parametrize("name,n", [("helm2d_n256", 64), ("helm2d_n32", 32), ("schr3d_n64", 16)])
def test_mixed_mode_error_bound(name, n):
    """The mixed path's alpha error against the FP64 oracle stays within the bound that FP32
    kernel vectors imply: |d alpha| <~ u32 * C * kappa, with C = sum|terms| / |g| of the
    frequency sums (below 1e3 on these workloads)."""
    v = make_workload(name, n=n)
    ctx = ctx_for(v)
    ctx.set_potential(v)
    ctx.build_stencils(policy="local", mode="mixed")
    tab = ctx.get_shift_table()
    ref = O.build_stencils(v, "local", shift_subset=[])
    assert np.array_equal(tab["s"], ref["S"])
    assert np.array_equal(tab["s_idx"].reshape(v.shape), ref["s_idx"])
    worst = 0.0
    for i in range(len(ref["S"])):
        st = O.stencil_for_shift(n, v.ndim, float(ref["S"][i]))
        w = np.linalg.eigvalsh(st["A"])
        kappa = np.abs(w).max() / (w[1] - w[0])
        err = np.abs(tab["alpha"][i] - st["alpha"]).max()
        worst = max(worst, err / (U32 * kappa))
        assert err <= max(1e-6, 1e3 * U32 * kappa), (i, err, kappa)
    print(f"mixed {name} n={n}: max |d alpha| / (u32 kappa) = {worst:.3g}")


def test_mixed_mode_gmres_within_one():
    import json
    import os
    import scipy.sparse
    with open(os.path.join(os.path.dirname(__file__), "golden", "gmres_helm2d_n32.json")) as fh:
        gold = json.load(fh)["iterations"]
    v = make_workload("helm2d_n32")
    n = 32
    ctx = ctx_for(v)
    ctx.set_potential(v)
    for pol in ("local", "paper"):
        ctx.build_stencils(policy=pol, mode="mixed")
        mats = {}
        for which in "CP":
            rowptr, colidx, vals = ctx.export_sparse_rows(which)
            mats[which] = scipy.sparse.csr_matrix((vals, colidx, rowptr), shape=(n * n, n * n))
        _, it, res, info = O.gmres_solve(v, gaussian_source(n, 2, 2.0), mats["P"], mats["C"])
        assert info == 0 and it <= gold[f"{pol}/2.0"] + 1, (pol, it)


def test_mixed_mode_full_size_gmres_proxy():
    """At 2D n=1024 the mixed stencils of sampled shifts stay close to the FP64 path's."""
    v = make_workload("helm2d_n1024")
    ctx = ctx_for(v)
    ctx.set_potential(v)
    ctx.build_stencils(policy="local", use_graph=True)
    t64 = ctx.get_shift_table(with_sidx=False)
    ctx.build_stencils(policy="local", mode="mixed", use_graph=True)
    t32 = ctx.get_shift_table(with_sidx=False)
    assert np.array_equal(t64["s"], t32["s"])
    err = np.abs(t64["alpha"] - t32["alpha"]).max()
    kap = np.abs(t64["lam"]).max()  # noqa: F841 (kept for the printout)
    print(f"mixed vs fp64 at n=1024: max |d alpha| = {err:.3g}")
    assert err < 1e-2


@pytest.mark.parametrize("name,nsample", [("helm2d_n256", 200), ("helm2d_n1024", 24),
                                          ("schr3d_n64", 0)])
def test_mixed_mode_full_size_against_the_oracle(name, nsample):
    """The mixed path at the full sizes of the 2D n = 256, 2D n = 1024 and 3D n = 64
    workloads, against the FP64 oracle: per shift |d alpha| <= 1e3 u32 kappa (the bound of
    test_mixed_mode_error_bound), on the shifts at v_min and v_max and a seeded sample of the
    others (every shift when nsample = 0). Prints the largest |d alpha| / (u32 kappa)."""
    v = make_workload(name)
    n, d = v.shape[0], v.ndim
    ctx = ctx_for(v)
    ctx.set_potential(v)
    ctx.build_stencils(policy="local", mode="mixed", use_graph=True)
    tab = ctx.get_shift_table()
    ref = O.build_stencils(v, "local", shift_subset=[])
    assert np.array_equal(tab["s"], ref["S"])
    assert np.array_equal(tab["s_idx"].reshape(v.shape), ref["s_idx"])
    ns = len(ref["S"])
    if nsample and nsample < ns - 2:
        rng = np.random.default_rng(12)
        idx = sorted(set(rng.choice(np.arange(1, ns - 1), nsample, replace=False).tolist())
                     | {0, ns - 1})
    else:
        idx = range(ns)
    worst, worst_abs = 0.0, 0.0
    for i in idx:
        st = O.stencil_for_shift(n, d, float(ref["S"][i]))
        w = np.linalg.eigvalsh(st["A"])
        kappa = np.abs(w).max() / (w[1] - w[0])
        err = np.abs(tab["alpha"][i] - st["alpha"]).max()
        worst = max(worst, err / (U32 * kappa))
        worst_abs = max(worst_abs, err)
        assert err <= max(1e-6, 1e3 * U32 * kappa), (i, err, kappa)
    print(f"mixed {name} full size: {len(idx)} shifts, max |d alpha| = {worst_abs:.3g}, "
          f"max |d alpha| / (u32 kappa) = {worst:.3g}")


# ---- double-word stages (FP32 pairs on the FP32 pipe), held to the FP64 tolerance --------

def dword_margin(tab, v, policy, sample=None):
    """Largest |d alpha| / tol_alpha over the checked shifts (tol_alpha of the FP64 path)."""
    n, d = v.shape[0], v.ndim
    ref = O.build_stencils(v, policy, shift_subset=[])
    idx = range(len(ref["S"])) if sample is None else sample
    worst = 0.0
    for i in idx:
        st, ta, tc = shift_tols(n, d, ref["S"][i])
        worst = max(worst, np.abs(tab["alpha"][i] - st["alpha"]).max() / ta)
    return worst


@pytest.mark.parametrize("name,n", [("helm2d_n32", 8), ("helm2d_n32", 16), ("helm2d_n32", 32),
                                    ("helm2d_n256", 64), ("helm2d_n256", 128)])
@pytest.mark.parametrize("policy", ["local", "paper", "mean"])
def test_dword_small_parity(name, n, policy):
    v = make_workload(name, n=n)
    ctx = ctx_for(v)
    ctx.set_potential(v)
    ctx.build_stencils(policy=policy, mode="dword")
    assert ctx.mode_used() == "dword"
    tab = ctx.get_shift_table()
    ref, tols = check_shift_table(tab, v, policy)
    assert check_rows(ctx, v, ref, tols) == v.size
    rows_consistent_with_table(ctx, v, tab)
    print(f"dword {name} n={n} {policy}: max |d alpha| / tol = {dword_margin(tab, v, policy):.3g}")


def test_dword_in_3d_runs_the_fp64_stages():
    v = make_workload("schr3d_n64", n=16)
    ctx = ctx_for(v)
    ctx.set_potential(v)
    ctx.build_stencils(policy="local", mode="dword")
    assert ctx.mode_used() == "fp64"
    q = ctx.get_rows("Q").copy()
    ctx.build_stencils(policy="local", mode="fp64")
    assert np.array_equal(ctx.get_rows("Q"), q)


@pytest.mark.parametrize("name,nsample", [("helm2d_n256", 200), ("helm2d_n1024", 40)])
def test_dword_full_size_sampled(name, nsample):
    v = make_workload(name)
    ctx = ctx_for(v)
    ctx.set_potential(v)
    for _ in range(2):
        ctx.build_stencils(policy="local", mode="dword", use_graph=True)
    tab = ctx.get_shift_table()
    ns = len(tab["s"])
    rng = np.random.default_rng(13)
    sample = sorted(set(rng.choice(np.arange(1, ns - 1), nsample, replace=False).tolist())
                    | {0, ns - 1})
    ref, tols = check_shift_table(tab, v, "local", sample=sample)
    assert check_rows(ctx, v, ref, tols) > 0
    rows_consistent_with_table(ctx, v, tab)
    print(f"dword {name} full size: {len(sample)} shifts, max |d alpha| / tol = "
          f"{dword_margin(tab, v, 'local', sample):.3g}")


def test_dword_graph_replay_is_bit_identical_and_gmres_unchanged():
    import json
    import os
    import scipy.sparse
    v = make_workload("helm2d_n32")
    n = 32
    ctx = ctx_for(v)
    ctx.set_potential(v)
    ctx.build_stencils(policy="local", mode="dword")
    first = [ctx.get_rows(k).copy() for k in "QCP"]
    for _ in range(2):
        ctx.build_stencils(policy="local", mode="dword", use_graph=True)
        for k, r in zip("QCP", first):
            assert np.array_equal(ctx.get_rows(k), r)
    with open(os.path.join(os.path.dirname(__file__), "golden", "gmres_helm2d_n32.json")) as fh:
        gold = json.load(fh)["iterations"]
    for pol in ("local", "paper"):
        ctx.build_stencils(policy=pol, mode="dword")
        mats = {}
        for which in "CP":
            rowptr, colidx, vals = ctx.export_sparse_rows(which)
            mats[which] = scipy.sparse.csr_matrix((vals, colidx, rowptr), shape=(n * n, n * n))
        _, it, res, info = O.gmres_solve(v, gaussian_source(n, 2, 2.0), mats["P"], mats["C"])
        assert info == 0 and it == gold[f"{pol}/2.0"], (pol, it)


# ---- launch-shape autotuner ------------------------------------------------------------------

@pytest.mark.parametrize("name,n,mode", [("helm2d_n256", 256, "fp64"), ("helm2d_n256", 256, "dword"),
                                         ("helm2d_n256", 256, "mixed"), ("schr3d_n64", 32, "fp64")])
def test_autotuned_builds_are_bit_identical(name, n, mode):
    v = make_workload(name, n=n)
    ref = ctx_for(v)
    ref.set_potential(v)
    ref.build_stencils(policy="local", mode=mode, use_graph=True)
    want = [ref.get_rows(k).copy() for k in "QCP"]
    ctx = ctx_for(v)
    ctx.set_autotune(True)
    ctx.set_potential(v)
    for _ in range(3):  # the tuning pass, then graph record and replay with the tuned shapes
        ctx.build_stencils(policy="local", mode=mode, use_graph=True)
        for k, r in zip("QCP", want):
            assert np.array_equal(ctx.get_rows(k), r)
    tun = ctx.tuning()
    assert any(k.startswith("stage1") for k in tun) and any(k.startswith("rows") for k in tun)
    for key, (th, ps, md, mb) in tun.items():
        assert th in (64, 128, 256) and ps in (2, 4, 8, 16, 32) and 0 < mb <= md * 1.0001, key
    print(f"autotune {name} n={n} {mode}: " + ", ".join(
        f"{k}={th}x{ps} ({md:.4f}->{mb:.4f} ms)" for k, (th, ps, md, mb) in tun.items()))
