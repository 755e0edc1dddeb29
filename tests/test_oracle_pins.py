"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test checks the oracle against something other than itself: a closed form, an invariant
stated in the paper, a brute-force dense computation, a long-double direct sum, or values
written by tests/golden/make_golden.py (which calls only the oracle). The last tests plant
plausible mistakes in a copy of the oracle and check that a pin catches each one.
"""

import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from lsp_inputs import gaussian_source, make_workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---- Sec. 2: L + diag(v) has plane-wave eigenvectors for constant v ----------------------

@pytest.mark.parametrize("n,d", [(16, 2), (8, 3), (32, 1)])
def test_plane_waves_are_eigenvectors(n, d):
    rng = np.random.default_rng(5)
    vconst = -123.25
    v = np.full((n,) * d, vconst)
    x = np.meshgrid(*([np.arange(n) / n] * d), indexing="ij")
    ks = [rng.integers(-n // 2, n // 2, d) for _ in range(4)] + [np.full(d, n // 2)]
    for k in ks:
        phase = 2 * np.pi * sum(ki * xi for ki, xi in zip(k, x))
        lam = 4 * math.pi ** 2 * float(np.sum(np.asarray(k, dtype=float) ** 2)) + vconst
        for u in (np.cos(phase), np.sin(phase)):
            if np.abs(u).max() < 1e-9:  # sin at the aliased k = n/2 vanishes on the grid
                continue
            y = O.apply_operator(v, u)
            assert np.abs(y - lam * u).max() <= 1e-12 * abs(lam) * np.abs(u).max() + 1e-10


def test_operator_is_real_symmetric():
    n, d = 8, 2
    v = make_workload("helm2d_n32", n=n)
    N = n ** d
    M = np.stack([O.apply_operator(v, e.reshape(n, n)).ravel() for e in np.eye(N)], axis=1)
    assert np.abs(M - M.T).max() <= 1e-11 * np.abs(M).max()


# ---- Sec. 3 / 4.2: the kernel vector g_s and g_s * g_s ------------------------------------

@pytest.mark.parametrize("n,d,m", [(16, 2, -40), (32, 2, -100), (8, 3, -30), (16, 3, 7)])
def test_kernel_vector_identities(n, d, m):
    s = float(O.shift_value(m))
    g, g2 = O.kernel_vectors(n, d, s)
    # even: g[j] = g[-j]; invariant under axis permutations (|k|^2 is)
    neg = tuple(slice(None) for _ in range(d))
    gneg = np.roll(np.flip(g, axis=tuple(range(d))), 1, axis=tuple(range(d)))
    assert np.abs(g - gneg).max() <= 1e-14 * np.abs(g).max()
    for perm in itertools.permutations(range(d)):
        assert np.abs(g - np.transpose(g, perm)).max() <= 1e-14 * np.abs(g).max()
    # k = 0 mode: sum_j g[j] = 1/s, sum_j (g*g)[j] = 1/s^2
    assert abs(g.sum() - 1 / s) <= 1e-12 * abs(1 / s)
    assert abs(g2.sum() - 1 / s ** 2) <= 1e-12 / s ** 2
    # (L + s) g = delta_0
    delta = O.apply_operator(np.full(g.shape, s), g)
    e0 = np.zeros_like(g)
    e0[(0,) * d] = 1.0
    assert np.abs(delta - e0).max() <= 1e-11
    # g * g really is the self-convolution (direct cyclic convolution at tiny n)
    if n ** d <= 256:
        conv = np.zeros_like(g)
        for j in np.ndindex(*g.shape):
            conv += g[j] * np.roll(g, j, axis=tuple(range(d)))
        assert np.abs(conv - g2).max() <= 1e-13 * np.abs(g2).max()
    del neg


def _direct_longdouble(n, d, s, offs):
    pi = np.longdouble("3.14159265358979323846264338327950288")
    k = O.freq_axis(n).astype(np.longdouble)
    kg = np.meshgrid(*([k] * d), indexing="ij")
    gh = 1 / (4 * pi * pi * sum(x * x for x in kg) + np.longdouble(s))
    out, out2 = [], []
    for o in offs:
        c = np.cos(2 * pi * sum(oi * x for oi, x in zip(o, kg)) / n)
        out.append((c * gh).sum() / n ** d)
        out2.append((c * gh * gh).sum() / n ** d)
    return np.array(out, dtype=np.float64), np.array(out2, dtype=np.float64)


@pytest.mark.parametrize("n,d,m", [(64, 2, -150), (128, 2, -900), (16, 3, -40)])
def test_kernel_vector_matches_direct_sum(n, d, m):
    s = float(O.shift_value(m))
    g, g2 = O.kernel_vectors(n, d, s)
    offs = [o for o in itertools.product(range(3), repeat=d) if list(o) == sorted(o)]
    gd, g2d = _direct_longdouble(n, d, s, offs)
    gf = np.array([g[o] for o in offs])
    g2f = np.array([g2[o] for o in offs])
    assert np.abs(gf - gd).max() <= 1e-12 * np.abs(gd).max()
    assert np.abs(g2f - g2d).max() <= 1e-12 * np.abs(g2d).max()


# ---- Sec. 3 / 4.2: Eq. A against the dense Green's matrix and its SVD --------------------

@pytest.mark.parametrize("n,d,m,t", [(8, 2, -8, 1), (10, 2, -12, 1), (12, 2, -18, 1),
                                     (8, 2, 3, 1), (6, 3, -5, 1), (8, 3, -9, 1),
                                     (10, 2, -12, 2), (12, 2, -18, 2), (12, 2, 3, 2),
                                     (10, 3, -14, 2), (12, 3, -20, 2)])
def test_gram_identity_and_svd_match_dense(n, d, m, t):
    s = float(O.shift_value(m))
    st = O.stencil_for_shift(n, d, s, t)
    offs = O.neighbourhood_offsets(d, t)
    for j in [(0,) * d, tuple(range(1, d + 1)), (n - 1,) * d]:
        alpha, sig, mu, G = O.brute_force_stencil(n, d, s, j, t)
        comp = sorted(set(range(n ** d)) - set(mu))
        B = G[np.ix_(mu, comp)]
        A_dense = B @ B.T
        assert np.abs(A_dense - st["A"]).max() <= 1e-12 * np.abs(A_dense).max()
        # translation invariance: the same alpha at every j (Sec. 3, Sec. 4.1)
        assert np.abs(alpha - st["alpha"]).max() <= 1e-9
        # optimal value = smallest singular value, lambda_1 = sigma_min^2
        assert abs(sig ** 2 - st["lam1"]) <= 1e-9 * np.abs(A_dense).max()
        # C[j, mu] = Q[j, mu] G[mu, mu]
        c_dense = alpha @ G[np.ix_(mu, mu)]
        assert np.abs(c_dense - st["c"]).max() <= 1e-9 * np.abs(c_dense).max()
    assert len(offs) == (2 * t + 1) ** d


def test_gram_is_positive_semidefinite():
    for (n, d, m) in [(32, 2, -60), (16, 3, -20)]:
        st = O.stencil_for_shift(n, d, float(O.shift_value(m)))
        w = np.linalg.eigvalsh(st["A"])
        assert w.min() >= -1e-12 * np.abs(w).max()


# ---- Sec. 4.1: shifts -----------------------------------------------------------------------

def test_snap_rounds_half_away_from_zero():
    # (x/pi^2 - 2)/4 = +0.5 and -0.5 exactly
    assert int(O.snap_index(4 * O.PI2)) == 1
    assert int(O.snap_index(0.0)) == -1
    assert int(O.snap_index(2 * O.PI2)) == 0
    assert int(O.snap_index(-2 * O.PI2)) == -1
    ms = np.arange(-50, 50)
    assert np.array_equal(O.snap_index(O.shift_value(ms)), ms)


def test_lattice_shifts_are_never_resonant():
    v = make_workload("helm2d_n256", n=64)
    for pol in ("local", "paper", "mean"):
        st = O.build_stencils(v, pol, shift_subset=[])
        lam = O.symbol(64, 2)
        for s in st["S"]:
            assert np.abs(lam + s).min() >= 2 * O.PI2 * (1 - 1e-12)


def test_assign_shift_ties_go_to_smaller_shift():
    m = np.array([-1, 0])          # s = -2 pi^2 and +2 pi^2: the midpoint 0 is an exact tie
    s = O.shift_value(m)
    mid = np.array([[0.0, s[0] + 1.0, s[1] - 1.0]])
    idx = O.assign_shifts(mid, m)
    assert idx.tolist() == [[0, 0, 1]]


def test_paper_shift_list():
    v = make_workload("helm2d_n256", n=64)
    K = 8
    m = O.paper_shift_list(v, K)
    assert 1 <= len(m) <= K and np.all(np.diff(m) > 0)
    assert m[0] == O.snap_index(v.min()) and m[-1] == O.snap_index(v.max())


def test_paper_shift_points_are_evenly_spaced_with_both_ends():
    # hand values: K points from v_min to v_max inclusive, spacing (v_max - v_min) / (K - 1)
    assert O.paper_shift_points(-3.0, 5.0, 5).tolist() == [-3.0, -1.0, 1.0, 3.0, 5.0]
    assert O.paper_shift_points(10.0, 16.0, 4).tolist() == [10.0, 12.0, 14.0, 16.0]
    assert O.paper_shift_points(0.0, 1.0, 2).tolist() == [0.0, 1.0]
    assert O.paper_shift_points(-7.0, 9.0, 1).tolist() == [-7.0]


def test_paper_shift_list_interior_after_snapping():
    # v / pi^2 spans [3.9, 25.9] and K = 5: x / pi^2 = 3.9, 9.4, 14.9, 20.4, 25.9, so
    # (x / pi^2 - 2) / 4 = 0.475, 1.85, 3.225, 4.6, 5.975 and m = 0, 2, 3, 5, 6
    v = np.array([[3.9, 10.0], [25.9, 7.0]]) * O.PI2
    assert O.paper_shift_list(v, 5).tolist() == [0, 2, 3, 5, 6]
    # v / pi^2 spans [0.1, 9.9] and K = 5: (x / pi^2 - 2) / 4 = -0.475, 0.1375, 0.75, 1.3625,
    # 1.975, so m = 0, 0, 1, 1, 2, deduplicated to 0, 1, 2
    v = np.array([0.1, 5.0, 9.9]) * O.PI2
    assert O.paper_shift_list(v, 5).tolist() == [0, 1, 2]


# ---- the sign of the near-null vector (the paper leaves it open; reading: centre > 0) -------

def test_sign_rule_on_hand_vectors():
    assert O.sign_fix(np.array([0.3, -0.8, 0.1]), 1).tolist() == [-0.3, 0.8, -0.1]
    assert O.sign_fix(np.array([0.3, 0.8, 0.1]), 1).tolist() == [0.3, 0.8, 0.1]
    # centre entry below 1e-12: the first entry with |alpha_i| > 1e-12 is made positive
    assert O.sign_fix(np.array([0.0, -0.6, 1e-13, 0.8]), 2).tolist() == [0.0, 0.6, -1e-13, -0.8]
    assert O.sign_fix(np.array([1e-13, 0.6, 0.0, -0.8]), 2).tolist() == [1e-13, 0.6, 0.0, -0.8]


@pytest.mark.parametrize("n,d,m,t", [(16, 2, -20, 1), (32, 2, -60, 1), (12, 2, -18, 2),
                                     (8, 3, -9, 1), (10, 3, -14, 2)])
def test_every_oracle_stencil_has_a_positive_centre(n, d, m, t):
    st = O.stencil_for_shift(n, d, float(O.shift_value(m)), t)
    centre = len(O.neighbourhood_offsets(d, t)) // 2
    assert st["alpha"][centre] > 0
    # the brute-force SVD vector agrees up to sign, and its sign is fixed the same way
    alpha_bf, _, _, _ = O.brute_force_stencil(n, d, float(O.shift_value(m)), (0,) * d, t) \
        if n ** d <= 1000 else (st["alpha"], None, None, None)
    assert abs(abs(float(alpha_bf @ st["alpha"])) - 1.0) < 1e-9
    assert alpha_bf[centre] > 0


def test_every_oracle_row_has_a_positive_centre():
    v = make_workload("helm2d_n256", n=32)
    for pol in ("local", "paper"):
        st = O.build_stencils(v, pol)
        assert (st["Q"][:, 4] > 0).all()
        assert (st["alpha"][:, 4] > 0).all()


@pytest.mark.parametrize("mutation", ["spacing_by_K", "flipped_sign_rule"])
def test_shift_and_sign_pins_catch_planted_mistakes(monkeypatch, mutation):
    import oracle.lsp_oracle as L
    if mutation == "spacing_by_K":
        def bad(vmin, vmax, K):
            step = (vmax - vmin) / K
            return np.array([vmin + i * step for i in range(K - 1)] + [vmax])
        monkeypatch.setattr(L, "paper_shift_points", bad)
        v = np.array([[3.9, 10.0], [25.9, 7.0]]) * O.PI2
        assert L.paper_shift_list(v, 5).tolist() != [0, 2, 3, 5, 6]
    else:
        orig = L.sign_fix
        monkeypatch.setattr(L, "sign_fix", lambda a, c: -orig(a, c))
        st = L.stencil_for_shift(16, 2, float(O.shift_value(-20)))
        assert not st["alpha"][4] > 0


# ---- Sec. 4.1: rows -------------------------------------------------------------------------

def test_constant_potential_gives_identical_rows():
    n, d = 16, 2
    v = np.full((n, n), -700.0)
    for pol in ("local", "paper", "mean"):
        st = O.build_stencils(v, pol)
        assert len(st["S"]) == 1
        for k in ("Q", "C", "P"):
            assert np.abs(st[k] - st[k][0]).max() == 0.0


def test_single_shift_reduces_to_section3():
    n, d = 16, 2
    v = make_workload("helm2d_n32", n=n)
    st = O.build_stencils(v, "mean")
    s = float(O.shift_value(O.snap_index(v.mean())))
    ref = O.stencil_for_shift(n, d, s)
    Q, C, P = O.sparse_matrices(st, n, d)
    # Sec. 3: Q rows are alpha, C rows are alpha^T G[mu, mu], P = Q + C diag(q), q = v - s
    q = (v - s).ravel()
    assert np.abs(st["Q"] - ref["alpha"]).max() == 0.0
    assert np.abs(st["C"] - ref["c"]).max() == 0.0
    Pd = Q.toarray() + C.toarray() @ np.diag(q)
    assert np.abs(P.toarray() - Pd).max() <= 1e-12 * np.abs(Pd).max()


def test_csr_pattern_matches_shifted_sum():
    n, d = 8, 3
    v = make_workload("schr3d_n64", n=n)
    st = O.build_stencils(v, "paper")
    P = O.rows_to_csr(st["P"], n, d)
    u = np.random.default_rng(0).standard_normal((n,) * d)
    offs = st["offsets"]
    ref = sum(st["P"][:, i].reshape(v.shape) * np.roll(u, tuple(-o for o in off), (0, 1, 2))
              for i, off in enumerate(offs))
    assert np.abs((P @ u.ravel()).reshape(v.shape) - ref).max() <= 1e-12 * np.abs(ref).max()


def test_qg_row_decays_away_from_j():
    # The 1D example of Sec. 4.1: n = 32, j = 16, s = -62 pi^2 (lattice m = -16).
    n, d, j = 32, 1, 16
    s = -62 * O.PI2
    assert int(O.snap_index(s)) == -16
    st = O.stencil_for_shift(n, d, s)
    G = O.dense_green_matrix(n, d, s)
    row = np.zeros(n)
    for a, o in enumerate(O.neighbourhood_offsets(d)):
        row += st["alpha"][a] * G[int((j + o[0]) % n)]
    dist = np.abs(np.arange(n) - j)
    trunc = np.abs(row)[dist >= 2]
    near = np.abs(row)[dist == 2].max()
    far = np.abs(row)[dist >= 8].max()
    assert far < near and np.abs(row)[dist <= 1].max() > trunc.max()


# ---- Sec. 5: GMRES(40), rtol 1e-6, preconditioned by P^-1 C ------------------------------

def test_gmres_iteration_counts_match_golden():
    with open(os.path.join(GOLDEN, "gmres_helm2d_n32.json")) as fh:
        gold = json.load(fh)
    v = make_workload("helm2d_n32")
    for key, want in gold["iterations"].items():
        pol, sig = key.split("/")
        st = O.build_stencils(v, pol)
        Q, C, P = O.sparse_matrices(st, 32, 2)
        _, it, res, info = O.gmres_solve(v, gaussian_source(32, 2, float(sig)), P, C)
        assert info == 0 and it == want, (key, it, want)
        # the paper's tables report 5-12 iterations for this method
        assert 3 <= it <= 12
        assert res < 1e-4


@pytest.mark.parametrize("case", ["t1_n8", "t1_n16_paper", "multi_t_n16"])
def test_solve_p_is_the_exact_inverse(case):
    """x = P^-1 y (Eq. QC): the sparse LU agrees with a dense solve and leaves a residual at
    the rounding level, for t = 1 rows and for the multi-t rows of a leaf-8 dissection."""
    if case == "t1_n8":
        v = make_workload("helm2d_n32", n=8)
        P = O.sparse_matrices(O.build_stencils(v, "local"), 8, 2)[2]
    elif case == "t1_n16_paper":
        v = make_workload("helm2d_n32", n=16)
        P = O.sparse_matrices(O.build_stencils(v, "paper"), 16, 2)[2]
    else:
        v = make_workload("helm2d_n32", n=16)
        P = O.build_stencils_multi(v, "paper", leaf=8, t_max=2)["P"]
    N = v.size
    y = np.random.default_rng(11).standard_normal(N)
    x = O.solve_p(P, y)
    Pd = P.toarray()
    xd = np.linalg.solve(Pd, y)
    cond = np.linalg.cond(Pd)
    assert np.abs(x - xd).max() <= 1e-13 * cond * np.abs(xd).max()
    assert np.linalg.norm(Pd @ x - y) <= 1e-12 * np.linalg.norm(Pd, 2) * np.linalg.norm(x)


def test_unpreconditioned_gmres_stalls():
    v = make_workload("helm2d_n32")
    _, it, res, info = O.gmres_solve(v, gaussian_source(32, 2), maxiter=3)
    assert info != 0 and res > 1e-3


# ---- Sec. 4.2: per-point neighbourhood size t_j from the nested-dissection geometry -------

def test_t_choice_reproduces_the_paper_figure():
    with open(os.path.join(GOLDEN, "tchoice_fig_16x16.json")) as fh:
        fig = json.load(fh)
    T = O.t_choice(16, 2, leaf=fig["leaf"], t_max=fig["t_max_drawn"])
    assert np.array_equal(T, np.array(fig["grid"]))


@pytest.mark.parametrize("n,d,leaf", [(32, 2, 8), (16, 2, 4), (16, 3, 8)])
def test_t_choice_keeps_boxes_apart_and_is_maximal(n, d, leaf):
    # the sparsity requirement of nested dissection, stated independently of the rule: an
    # interaction between j and i may not cross an edge, i.e. along no axis may a separator
    # line (a multiple of leaf; the periodic seam is one) lie strictly between j_a and i_a.
    # t_j (uncapped) must satisfy it for all of mu_j^{t_j}, and t_j + 1 must not.
    T = O.t_choice(n, d, leaf=leaf, t_max=10 * leaf)

    def crosses(j, t):
        for a in range(d):
            for i_a in (j[a] - t, j[a] + t):  # the extreme offsets decide along each axis
                lo, hi = min(j[a], i_a), max(j[a], i_a)
                if any(m % leaf == 0 for m in range(lo + 1, hi)):
                    return True
        return False

    for j in np.ndindex(*(n,) * d):
        t = int(T[j])
        assert 1 <= t <= leaf
        assert not crosses(j, t) and crosses(j, t + 1), (j, t)


def test_multi_t_rows_reduce_to_the_uniform_build():
    v = make_workload("helm2d_n32")
    for pol in ("paper", "local"):
        ref = O.build_stencils(v, pol)
        for t in (1, 2):
            multi = O.build_stencils_multi(v, pol, t_of=t * np.ones(v.shape, dtype=np.int64))
            if t == 1:
                Q, C, P = O.sparse_matrices(ref, 32, 2)
            else:
                ref2 = O.build_stencils(v, pol, t=2)
                Q, C, P = O.sparse_matrices(ref2, 32, 2, t=2)
            for a, b in ((Q, multi["Q"]), (C, multi["C"]), (P, multi["P"])):
                assert (a != b).nnz == 0
    # mixed t: every row has (2 t_j + 1)^d entries at its own neighbourhood
    st = O.build_stencils_multi(v, "paper")
    lens = np.diff(st["Q"].indptr)
    assert np.array_equal(lens, (2 * st["t"].reshape(-1) + 1) ** 2)


def test_multi_t_gmres_counts_match_golden():
    with open(os.path.join(GOLDEN, "gmres_multi_t_helm2d_n32.json")) as fh:
        gold = json.load(fh)["iterations"]
    v = make_workload("helm2d_n32")
    f = gaussian_source(32, 2, 2.0)
    for key, want in gold.items():
        pol, label = key.split("/")
        kw = {} if label == "nd8" else {"t_of": 2 * np.ones(v.shape, dtype=np.int64)}
        st = O.build_stencils_multi(v, pol, **kw)
        _, it, res, info = O.gmres_solve(v, f, st["P"], st["C"])
        assert info == 0 and it == want and res < 1e-4, (key, it, want)
        # within the paper's range for this method (Sec. 5 tables: 5-12)
        assert 2 <= it <= 12


# ---- planted mistakes: each must be caught by one of the pins above ---------------------

def _dense_A(n, d, s):
    alpha, sig, mu, G = O.brute_force_stencil(n, d, s, (0,) * d)
    comp = sorted(set(range(n ** d)) - set(mu))
    B = G[np.ix_(mu, comp)]
    return B @ B.T, alpha


@pytest.mark.parametrize("mutation", ["drop_A2", "sign_of_s", "transposed_gather",
                                      "pointwise_g2", "largest_eigvec"])
def test_pins_catch_planted_mistakes(monkeypatch, mutation):
    n, d, s = 10, 2, float(O.shift_value(-12))
    A_ref, alpha_ref = _dense_A(n, d, s)
    orig_gram, orig_kv = O.gram_matrix, O.kernel_vectors
    import oracle.lsp_oracle as L
    if mutation == "drop_A2":
        monkeypatch.setattr(L, "gram_matrix",
                            lambda g, g2, offs: (orig_gram(g, g2, offs)[0]
                                                 + orig_gram(g, g2, offs)[1] @ orig_gram(g, g2, offs)[1].T,
                                                 orig_gram(g, g2, offs)[1]))
    elif mutation == "sign_of_s":
        monkeypatch.setattr(L, "kernel_vectors", lambda n_, d_, s_: orig_kv(n_, d_, -s_))
    elif mutation == "transposed_gather":
        def bad(g, g2, offs):
            A, Gm = orig_gram(g, g2, offs)
            n_ = g.shape[0]
            shifted = np.roll(g, 1, axis=0)
            Gm2 = L._gather(shifted, offs, n_)
            return L._gather(g2, offs, n_) - Gm2 @ Gm2.T, Gm2
        monkeypatch.setattr(L, "gram_matrix", bad)
    elif mutation == "pointwise_g2":
        # g_s * g_s taken as a pointwise square instead of a convolution
        monkeypatch.setattr(L, "kernel_vectors",
                            lambda n_, d_, s_: (orig_kv(n_, d_, s_)[0],
                                                orig_kv(n_, d_, s_)[0] ** 2))
    elif mutation == "largest_eigvec":
        def bad_nn(A, centre):
            w, V = np.linalg.eigh(A)
            return O.sign_fix(V[:, -1], centre), w[-1], w[-2], False
        monkeypatch.setattr(L, "near_null", bad_nn)
    st = L.stencil_for_shift(n, d, s)
    caught = (np.abs(st["A"] - A_ref).max() > 1e-12 * np.abs(A_ref).max()
              or np.abs(st["alpha"] - alpha_ref).max() > 1e-9)
    assert caught


@pytest.mark.parametrize("mutation", ["separators_like_boxes", "leaf_off_by_one"])
def test_t_choice_pins_catch_planted_mistakes(mutation):
    # plausible slips in the t_j rule, each caught by the paper's figure
    with open(os.path.join(GOLDEN, "tchoice_fig_16x16.json")) as fh:
        fig = json.load(fh)
    x = np.indices((16, 16))
    leaf = fig["leaf"]
    if mutation == "separators_like_boxes":
        r = x % leaf
        T = np.minimum(np.where(r == 0, 0, np.minimum(r, leaf - r)).min(axis=0), 4)
    else:
        r = x % (leaf + 1)
        T = np.minimum(np.where(r == 0, leaf + 1, np.minimum(r, leaf + 1 - r)).min(axis=0), 4)
    assert not np.array_equal(T, np.array(fig["grid"]))
    assert np.array_equal(O.t_choice(16, 2, leaf=leaf, t_max=4), np.array(fig["grid"]))
