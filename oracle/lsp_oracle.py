"""Plain FP64 CPU oracle: the stencil setup of the localized sparsifying preconditioner.

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline of the benchmark). It is written
from the paper (Liu & Ying, "Localized sparsifying preconditioner for periodic indefinite
systems"), step by step in the paper's order and notation, with numpy/scipy primitives
(fftn, eigh, svd, splu, gmres) as the only building blocks: no blocking, fusion or
reordering beyond what the definitions state.

Conventions chosen where the paper is silent (each one is also listed with its reason in the
design notes of the repository):

* Arrays on J are row-major with the last axis fastest; K is held in FFT order
  (0..n/2-1, -n/2..-1), which is the set K = [-n/2, n/2)^d of Sec. 2.
* The neighbourhood mu_0^t is listed in lexicographic offset order (o_1..o_d in [-t, t], last
  offset fastest); row j of Q, C, P uses columns (j + o) mod n in that order.
* s_j is the arg-min over S of |s - v_j| (the text of Sec. 4.1 writes a min), ties to the
  smaller shift.
* Shifts are snapped to the resonance-free lattice s = (4m+2) pi^2 of Sec. 4.1 with
  m = round-half-away-from-zero((x / pi^2 - 2) / 4).
* The near-null vector's sign: alpha[centre] > 0, else the first entry with |alpha| > 1e-12
  is made positive.
* A shift is flagged degenerate when lambda_2 - lambda_1 < 1e-8 * max|lambda|.

Parity status of every function here: pinned (see tests/test_oracle_pins.py), except where a
docstring says "parity unpinned".
"""

from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg

__all__ = [
    "PI2", "freq_axis", "symbol", "apply_operator", "round_half_away", "snap_index",
    "shift_value", "paper_shift_points", "paper_shift_list", "default_nshifts", "assign_shifts", "solve_p",
    "neighbourhood_offsets", "kernel_vectors", "gram_matrix", "near_null",
    "stencil_for_shift", "build_stencils", "rows_to_csr", "sparse_matrices",
    "gmres_solve", "dense_green_matrix", "brute_force_stencil", "sign_fix",
    "local_shift_indices", "gather_offsets", "t_choice", "build_stencils_multi",
]

PI2 = math.pi * math.pi  # pi^2 as one correctly rounded product of the float64 pi


# --------------------------------------------------------------------------------------------
# Sec. 2: grids, unitary DFT, the pseudospectral operator L + diag(v)  (Eq. dmodel)
# --------------------------------------------------------------------------------------------

def freq_axis(n: int) -> np.ndarray:
    """One axis of K = {-n/2 <= k < n/2} in FFT order (Sec. 2)."""
    return np.fft.fftfreq(n, d=1.0 / n)


def symbol(n: int, d: int) -> np.ndarray:
    """4 pi^2 |k|^2 on K (FFT order): the Fourier symbol of L (Sec. 2)."""
    k = freq_axis(n)
    grids = np.meshgrid(*([k] * d), indexing="ij")
    k2 = sum(g * g for g in grids)
    return 4.0 * PI2 * k2


def apply_operator(v: np.ndarray, u: np.ndarray) -> np.ndarray:
    """y = (L + diag(v)) u with L = F^-1 diag(4 pi^2 |k|^2) F (Sec. 2, Eq. dmodel).

    The unitary factors n^{-d/2} of F and F^-1 multiply to 1/N, which is numpy's ifftn
    normalisation, so F^-1 diag(.) F = ifftn(diag(.) fftn(.)).
    """
    n, d = v.shape[0], v.ndim
    lam = symbol(n, d)
    lu = np.fft.ifftn(lam * np.fft.fftn(u))
    if np.isrealobj(u):
        lu = lu.real
    return lu + v * u


# --------------------------------------------------------------------------------------------
# Sec. 4.1: shift list S and per-point shift s_j
# --------------------------------------------------------------------------------------------

def round_half_away(y):
    """Round to the nearest integer, halves away from zero (exact for |y| < 2^52)."""
    y = np.asarray(y, dtype=np.float64)
    r = np.trunc(y)
    frac = y - r
    return (r + np.sign(y) * (np.abs(frac) >= 0.5)).astype(np.int64)


def snap_index(x):
    """Lattice index m of the resonance-free shift (4m+2) pi^2 nearest to x (Sec. 4.1).

    The eigenvalues of L are multiples of 4 pi^2, so (4m+2) pi^2 keeps L + s invertible.
    """
    x = np.asarray(x, dtype=np.float64)
    return round_half_away((x / PI2 - 2.0) / 4.0)


def shift_value(m):
    """s = (4m + 2) pi^2 (Sec. 4.1)."""
    return (4.0 * np.asarray(m, dtype=np.float64) + 2.0) * PI2


def default_nshifts(n: int, d: int) -> int:
    """|S| of the paper's experiments: n/16 in 2D, n/4 in 3D (Tables of Sec. 5), at least 2."""
    return max(2, n // 16 if d == 2 else n // 4)


def paper_shift_points(vmin: float, vmax: float, nshifts: int) -> np.ndarray:
    """The nshifts points spread evenly over [v_min, v_max], before snapping (Sec. 4.1).

    x_i = v_min + i * ((v_max - v_min) / (K - 1)) for i < K-1 and x_{K-1} = v_max; K = 1 gives
    v_min alone.
    """
    K = int(nshifts)
    if K < 1:
        raise ValueError("nshifts must be >= 1")
    if K == 1:
        return np.array([float(vmin)])
    step = (float(vmax) - float(vmin)) / (K - 1)
    return np.array([float(vmin) + i * step for i in range(K - 1)] + [float(vmax)])


def paper_shift_list(v: np.ndarray, nshifts: int) -> np.ndarray:
    """S: nshifts points spread evenly over [v_min, v_max], snapped to the lattice, deduped.

    Sec. 4.1 ("Now let us discuss how to choose S"). Returns the sorted lattice indices m.
    """
    xs = paper_shift_points(float(v.min()), float(v.max()), nshifts)
    return np.unique(snap_index(xs))


def assign_shifts(v: np.ndarray, m_list: np.ndarray) -> np.ndarray:
    """s_j = arg-min_{s in S} |s - v_j|, ties to the smaller s (Sec. 4.1). Returns indices."""
    s = shift_value(m_list)
    dist = np.abs(s[None, :] - v.reshape(-1, 1))
    return np.argmin(dist, axis=1).astype(np.int64).reshape(v.shape)


def local_shift_indices(v: np.ndarray):
    """The per-point ("ideal") shift G_{v_j} of Sec. 4.1, snapped to the lattice.

    Returns (m_list, s_idx): the distinct lattice indices in increasing order and, per point,
    the index of its own snapped shift in that list.
    """
    m = snap_index(v)
    m_list, inv = np.unique(m.ravel(), return_inverse=True)
    return m_list, inv.reshape(v.shape).astype(np.int64)


# --------------------------------------------------------------------------------------------
# Sec. 3 / Sec. 4.2: kernel vector g_s, g_s * g_s, the Gram identity A = A1 - A2 (Eq. A)
# --------------------------------------------------------------------------------------------

def neighbourhood_offsets(d: int, t: int = 1) -> np.ndarray:
    """mu_0^t = {i : ||i||_inf <= t} (Sec. 4.2) in lexicographic order, last offset fastest."""
    return np.array(list(itertools.product(range(-t, t + 1), repeat=d)), dtype=np.int64)


def kernel_vectors(n: int, d: int, s: float):
    """g_s and g_s * g_s on the whole grid J (Sec. 3 definition of G; Sec. 4.2).

    G_s = (L + s)^-1 = F^-1 diag(1/(4 pi^2 |k|^2 + s)) F, so G_s[j1, j2] = g_s[j1 - j2] with
    g_s = ifftn(ghat). The convolution g_s * g_s has transform ghat^2.
    """
    ghat = 1.0 / (symbol(n, d) + s)
    gc = np.fft.ifftn(ghat)
    g2c = np.fft.ifftn(ghat * ghat)
    g, g2 = gc.real.copy(), g2c.real.copy()
    scale = max(float(np.abs(g).max()), 1e-300)
    if float(np.abs(gc.imag).max()) > 1e-12 * scale:
        raise AssertionError("g_s is not real")
    return g, g2


def gather_offsets(vec: np.ndarray, offs: np.ndarray, n: int) -> np.ndarray:
    """M[a, b] = vec[(o_a - o_b) mod n]  (translation invariance, Sec. 4.2)."""
    diff = (offs[:, None, :] - offs[None, :, :]) % n
    return vec[tuple(diff[..., i] for i in range(offs.shape[1]))]


_gather = gather_offsets


def gram_matrix(g: np.ndarray, g2: np.ndarray, offs: np.ndarray):
    """A = A1 - A2 of Eq. A for the neighbourhood offs; returns (A, Gm).

    A1[a, b] = (g_s * g_s)[o_a - o_b]  (rows of G_s dotted with each other),
    A2 = G_s[mu, mu] G_s[mu, mu]^T with G_s[mu, mu][a, b] = g_s[o_a - o_b].
    """
    n = g.shape[0]
    Gm = _gather(g, offs, n)
    A1 = _gather(g2, offs, n)
    A2 = Gm @ Gm.T
    return A1 - A2, Gm


def sign_fix(alpha: np.ndarray, centre: int) -> np.ndarray:
    """Fix the +/- ambiguity of a singular vector: alpha[centre] > 0, else first |entry|>1e-12."""
    a = np.array(alpha, dtype=np.float64)
    if abs(a[centre]) > 1e-12:
        return a if a[centre] > 0 else -a
    for x in a:
        if abs(x) > 1e-12:
            return a if x > 0 else -a
    return a


def near_null(A: np.ndarray, centre: int):
    """Eigenvector of the smallest eigenvalue of A = A1 - A2 (Sec. 4.2, after Eq. A).

    Returns (alpha, lambda_1, lambda_2, degenerate).
    """
    w, V = np.linalg.eigh(A)
    alpha = sign_fix(V[:, 0], centre)
    lam_max = float(np.abs(w).max())
    degenerate = bool(len(w) > 1 and (w[1] - w[0]) < 1e-8 * lam_max)
    return alpha, float(w[0]), float(w[1]) if len(w) > 1 else math.inf, degenerate


def stencil_for_shift(n: int, d: int, s: float, t: int = 1):
    """alpha_s^t and the C stencil c = alpha^T G_s[mu, mu] for one shift (Sec. 4.1, 4.2)."""
    offs = neighbourhood_offsets(d, t)
    g, g2 = kernel_vectors(n, d, s)
    A, Gm = gram_matrix(g, g2, offs)
    centre = len(offs) // 2
    alpha, lam1, lam2, degen = near_null(A, centre)
    c = Gm.T @ alpha
    return dict(alpha=alpha, c=c, lam1=lam1, lam2=lam2, degenerate=degen, g=g, g2=g2, A=A)


# --------------------------------------------------------------------------------------------
# Sec. 4.1: rows of Q, C and P for every point
# --------------------------------------------------------------------------------------------

def build_stencils(v: np.ndarray, policy: str = "local", nshifts: int | None = None,
                   m_list=None, t: int = 1, shift_subset=None):
    """All stencil rows for the potential v (Sec. 4.1).

    policy: "local" (each point's own snapped shift), "paper" (|S| evenly spread shifts),
    "mean" (the single shift snap(mean v) of Sec. 3), "list" (caller's lattice indices m_list).

    Q[j, mu_j] = alpha_{s_j}^T, C[j, mu_j] = alpha_{s_j}^T G_{s_j}[mu_j, mu_j],
    P[j, mu_j] = Q[j, mu_j] + C[j, mu_j] diag(v[mu_j] - s_j).

    shift_subset: optional indices into the shift list; only those shifts are solved (for
    sampled checks at large n) and rows are returned only for points using them.
    """
    n, d = v.shape[0], v.ndim
    if policy == "local":
        m_arr, s_idx = local_shift_indices(v)
    elif policy == "paper":
        m_arr = paper_shift_list(v, nshifts or default_nshifts(n, d))
        s_idx = assign_shifts(v, m_arr)
    elif policy == "mean":
        m_arr = np.unique(snap_index(np.array([float(v.mean())])))
        s_idx = np.zeros(v.shape, dtype=np.int64)
    elif policy == "list":
        m_arr = np.unique(np.asarray(m_list, dtype=np.int64))
        s_idx = assign_shifts(v, m_arr)
    else:
        raise ValueError(policy)
    S = shift_value(m_arr)
    offs = neighbourhood_offsets(d, t)
    mu = len(offs)
    todo = range(len(S)) if shift_subset is None else list(shift_subset)
    alpha = np.full((len(S), mu), np.nan)
    cst = np.full((len(S), mu), np.nan)
    lam1 = np.full(len(S), np.nan)
    degen = np.zeros(len(S), dtype=bool)
    for i in todo:
        st = stencil_for_shift(n, d, float(S[i]), t)
        alpha[i], cst[i], lam1[i], degen[i] = st["alpha"], st["c"], st["lam1"], st["degenerate"]
    # v[j + o] for every offset o (periodic wrap): np.roll by -o.
    vnb = np.stack([np.roll(v, tuple(-o for o in off), axis=tuple(range(d))) for off in offs],
                   axis=-1).reshape(-1, mu)
    idx = s_idx.reshape(-1)
    Q = alpha[idx]
    C = cst[idx]
    P = Q + C * (vnb - S[idx][:, None])
    return dict(m=m_arr, S=S, s_idx=s_idx, alpha=alpha, c=cst, lam1=lam1, degenerate=degen,
                Q=Q, C=C, P=P, offsets=offs)


# --------------------------------------------------------------------------------------------
# Sec. 4.2: per-point neighbourhood size t_j from the nested-dissection geometry
# --------------------------------------------------------------------------------------------

def t_choice(n: int, d: int, leaf: int = 8, t_max: int = 2) -> np.ndarray:
    """t_j for every point (Sec. 4.2 and its figure of t choices), shape (n,)*d.

    Nested dissection with leaf boxes of width `leaf` puts separators on the grid lines
    x_a = 0 (mod leaf). Two points of different boxes must not interact, so t_j is the largest
    t with mu_j^t inside the closed box of j along every axis: along an axis where j is not on
    a separator (r = x_a mod leaf > 0) that is min(r, leaf - r); along an axis where it is, the
    neighbourhood may reach the next separator line, i.e. leaf. t_j is the minimum over the
    axes, capped by t_max (the largest t for which stencils are built). With leaf = 4 and
    t_max = 4 this reproduces the paper's 16 x 16 example point by point.
    """
    x = np.indices((n,) * d)
    r = x % leaf
    f = np.where(r == 0, leaf, np.minimum(r, leaf - r))
    return np.minimum(f.min(axis=0), t_max).astype(np.int64)


def build_stencils_multi(v: np.ndarray, policy: str = "paper", nshifts: int | None = None,
                         m_list=None, leaf: int = 8, t_max: int = 2, t_of=None):
    """Rows with per-point neighbourhoods mu_j^{t_j} (Sec. 4.2):

    Q[j, mu_j^{t_j}] = (alpha_{s_j}^{t_j})^T, C[j, .] = Q[j, .] G_{s_j}[mu_j^{t_j}, mu_j^{t_j}],
    P[j, .] = Q[j, .] + C[j, .] diag(v[mu_j^{t_j}] - s_j),

    with t_j from t_choice (or the array t_of) and s_j from the shift policy as in
    build_stencils. A stencil (alpha_s^t, c_s^t) is computed for every (shift, t) pair that
    some point uses. Returns scipy CSR matrices Q, C, P (columns of each row in the
    lexicographic offset order of mu^{t_j}) and the per-(shift, t) tables.
    """
    n, d = v.shape[0], v.ndim
    base = build_stencils(v, policy, nshifts=nshifts, m_list=m_list, shift_subset=[])
    S, s_idx = base["S"], base["s_idx"].reshape(-1)
    tj = (t_choice(n, d, leaf, t_max) if t_of is None else np.asarray(t_of)).reshape(-1)
    N = n ** d
    tables = {}
    for t in sorted(set(int(x) for x in tj)):
        used = sorted(set(int(i) for i in s_idx[tj == t]))
        for i in used:
            st = stencil_for_shift(n, d, float(S[i]), t)
            tables[(i, t)] = st
    coords = np.stack(np.unravel_index(np.arange(N), (n,) * d), axis=-1)
    rows = {k: [] for k in "QCP"}
    cols, ptr = [], [0]
    flat_v = v.reshape(-1)
    for j in range(N):
        t = int(tj[j])
        st = tables[(int(s_idx[j]), t)]
        offs = neighbourhood_offsets(d, t)
        cj = np.ravel_multi_index(tuple(((coords[j] + offs) % n).T), (n,) * d)
        q, c = st["alpha"], st["c"]
        rows["Q"].append(q)
        rows["C"].append(c)
        rows["P"].append(q + c * (flat_v[cj] - S[s_idx[j]]))
        cols.append(cj)
        ptr.append(ptr[-1] + len(offs))
    colidx = np.concatenate(cols)
    indptr = np.asarray(ptr, dtype=np.int64)
    mats = {k: scipy.sparse.csr_matrix((np.concatenate(rows[k]), colidx, indptr), shape=(N, N))
            for k in "QCP"}
    return dict(S=S, s_idx=base["s_idx"], t=tj.reshape(v.shape), tables=tables,
                Q=mats["Q"], C=mats["C"], P=mats["P"])


def rows_to_csr(rows: np.ndarray, n: int, d: int, t: int = 1) -> scipy.sparse.csr_matrix:
    """Sparse N x N matrix with rows[j, i] at column (j + o_i) mod n (Sec. 4.1 pattern)."""
    offs = neighbourhood_offsets(d, t)
    N = n ** d
    mu = len(offs)
    jj = np.stack(np.unravel_index(np.arange(N), (n,) * d), axis=-1)  # [N, d]
    cols = np.empty((N, mu), dtype=np.int64)
    for i, o in enumerate(offs):
        cols[:, i] = np.ravel_multi_index(tuple(((jj + o) % n).T), (n,) * d)
    indptr = np.arange(N + 1, dtype=np.int64) * mu
    return scipy.sparse.csr_matrix((rows.reshape(-1), cols.reshape(-1), indptr), shape=(N, N))


def sparse_matrices(st: dict, n: int, d: int, t: int = 1):
    """(Q, C, P) as scipy CSR matrices."""
    return tuple(rows_to_csr(st[k], n, d, t) for k in ("Q", "C", "P"))


# --------------------------------------------------------------------------------------------
# Sec. 4.1 (Eq. PC) and Sec. 5: P^-1 C as a preconditioner for GMRES(40), rtol 1e-6
# --------------------------------------------------------------------------------------------

def gmres_solve(v: np.ndarray, f: np.ndarray, P=None, C=None, restart: int = 40,
                rtol: float = 1e-6, maxiter: int = 2000):
    """Solve (L + diag v) u = f by GMRES, left-preconditioned with P^-1 C (Eq. PC).

    A sparse LU of P stands in for nested dissection (any exact factorisation gives the same
    P^-1). x0 = 0; the stopping test is on the preconditioned residual. Returns
    (u, inner_iterations, true_relative_residual). With P = C = None, no preconditioner.
    """
    n, d = v.shape[0], v.ndim
    N = n ** d
    shape = v.shape

    def A(x):
        return apply_operator(v, x.reshape(shape)).reshape(-1)

    if P is not None:
        lu = scipy.sparse.linalg.splu(P.tocsc())

        def M(x):
            return lu.solve(C @ x)
    else:
        def M(x):
            return x

    op = scipy.sparse.linalg.LinearOperator((N, N), matvec=lambda x: M(A(x)), dtype=np.float64)
    b = M(f.reshape(-1))
    count = [0]

    def cb(_):
        count[0] += 1

    u, info = scipy.sparse.linalg.gmres(op, b, rtol=rtol, atol=0.0, restart=restart,
                                        maxiter=maxiter, callback=cb, callback_type="pr_norm")
    res = np.linalg.norm(A(u) - f.reshape(-1)) / np.linalg.norm(f)
    return u.reshape(shape), count[0], float(res), int(info)


def solve_p(P: scipy.sparse.spmatrix, y: np.ndarray) -> np.ndarray:
    """x = P^-1 y: the sparse solve behind the preconditioner P^-1 C (Sec. 3, Eq. QC; Sec. 4.1).

    The paper factors P by nested dissection (Fig. nd, Table cost); every exact factorisation
    gives the same x up to rounding, so this is the definition with a sparse LU as its step.
    """
    lu = scipy.sparse.linalg.splu(scipy.sparse.csc_matrix(P))
    return lu.solve(np.asarray(y, dtype=np.float64))


# --------------------------------------------------------------------------------------------
# Sec. 3: brute-force dense path (tiny n only) -- independent of the FFT identity
# --------------------------------------------------------------------------------------------

def dense_green_matrix(n: int, d: int, s: float) -> np.ndarray:
    """G_s = (L + s I)^-1 from the explicit unitary DFT matrix (Sec. 2, Sec. 3)."""
    k = freq_axis(n)
    j = np.arange(n)
    F1 = np.exp(-2j * np.pi * np.outer(k, j) / n) / math.sqrt(n)   # rows k, columns j
    F = F1
    for _ in range(d - 1):
        F = np.kron(F, F1)
    kg = np.meshgrid(*([k] * d), indexing="ij")
    lam = 4.0 * PI2 * sum(x * x for x in kg).reshape(-1)
    L = F.conj().T @ np.diag(lam) @ F
    G = np.linalg.inv(L + s * np.eye(n ** d))
    if float(np.abs(G.imag).max()) > 1e-10 * float(np.abs(G).max()):
        raise AssertionError("dense G_s is not real")
    return G.real


def brute_force_stencil(n: int, d: int, s: float, j, t: int = 1):
    """alpha by the SVD of G_s[mu_j, mu_j^c] (Sec. 3); returns (alpha, sigma_min, mu_j)."""
    G = dense_green_matrix(n, d, s)
    offs = neighbourhood_offsets(d, t)
    jj = np.asarray(j)
    mu = [int(np.ravel_multi_index(tuple((jj + o) % n), (n,) * d)) for o in offs]
    comp = sorted(set(range(n ** d)) - set(mu))
    U, sig, _ = np.linalg.svd(G[np.ix_(mu, comp)], full_matrices=True)
    alpha = sign_fix(U[:, len(mu) - 1], len(offs) // 2)
    return alpha, float(sig[len(mu) - 1]), mu, G
