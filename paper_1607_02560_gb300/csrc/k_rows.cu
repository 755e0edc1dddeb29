// Step a7: the rows of Q, C and P for every grid point (Sec. 4.1):
//   Q[j, mu_j] = alpha_{s_j},  C[j, mu_j] = c_{s_j},  P[j, mu_j] = alpha_{s_j} + c_{s_j} .* (v[mu_j] - s_j),
// with s_j the shift of S nearest to v_j (ties to the smaller shift) and mu_j = j + mu_0 taken
// periodically. Also the per-point shift index alone (for the shift table) and the CSR column
// indices of the common sparsity pattern.
//
// HBM-bound: per point 8 bytes of v are read and 3 |mu| doubles are written. A block handles
// 256 consecutive points, whose rows form one contiguous span of every output array, so
// consecutive threads store consecutive doubles (fully coalesced, streaming stores).
#include "lsp_internal.h"

namespace lsp {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int64_t snap_m(double x) {
  // Fast path: fma(x, 1/(4 pi^2), -1/2) is within a few ulp of the exact (x/pi^2 - 2)/4, so
  // its nearest integer is the exact one unless it lies next to a half-integer.
  const double yf = fma(x, kQuarterInvPi2, -0.5);
  const double r = rint(yf);
  if (0.5 - fabs(yf - r) > 1e-14 * fabs(yf) + 1e-14) return (int64_t)r;
  const double y = __dmul_rn(__dsub_rn(__ddiv_rn(x, kPi2), 2.0), 0.25);
  return (int64_t)round(y);
}
__device__ __forceinline__ double shift_of(int64_t m) { return lattice_shift(m); }

// Index in the sorted list S (given by lattice indices) of the shift nearest to x; ties go to
// the smaller shift. |s - x| is monotone on each side of x, so only the two shifts around the
// insertion point can win.
__device__ __forceinline__ int nearest_shift(const int32_t* __restrict__ m, int ns, double x) {
  int lo = 0, hi = ns;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (shift_of(__ldg(m + mid)) < x)
      lo = mid + 1;
    else
      hi = mid;
  }
  if (lo == 0) return 0;
  if (lo == ns) return ns - 1;
  const double d1 = fabs(__dsub_rn(shift_of(__ldg(m + lo - 1)), x));
  const double d2 = fabs(__dsub_rn(shift_of(__ldg(m + lo)), x));
  return d1 <= d2 ? lo - 1 : lo;
}

template <int D>
__device__ __forceinline__ int64_t neighbour(int64_t j, int o, int logn, int64_t mask) {
  if (D == 1) {
    return (j + o - 1) & mask;
  } else if (D == 2) {
    const int64_t x1 = j & mask, x0 = j >> logn;
    const int64_t y0 = (x0 + (o / 3) - 1) & mask, y1 = (x1 + (o % 3) - 1) & mask;
    return (y0 << logn) | y1;
  } else {
    const int64_t x2 = j & mask, x1 = (j >> logn) & mask, x0 = j >> (2 * logn);
    const int64_t y0 = (x0 + (o / 9) - 1) & mask, y1 = (x1 + ((o / 3) % 3) - 1) & mask,
                  y2 = (x2 + (o % 3) - 1) & mask;
    return (y0 << (2 * logn)) | (y1 << logn) | y2;
  }
}

// P[j, o] = alpha[o] + c[o] (v[j + o] - s) is formed as fma(c[o], v[j + o], ap[o]) from the
// per-shift table ap = alpha - c s (written by the eigen kernels with alpha and c): one FP64
// operation per element instead of two,
// which halves the FP64-pipe work of this kernel (the FP64 pipe, not HBM, held it back). c s
// is of the order of alpha here, so the two roundings cost a few ulp of P.
template <int D, bool LOCAL, bool ROWS, bool SIDX>
__global__ void __launch_bounds__(kThreads) k_rows(
    const double* __restrict__ v, int64_t N, int logn, const int32_t* __restrict__ idx_of,
    int64_t mlo, int64_t R, int32_t* __restrict__ err, const int32_t* __restrict__ shift_m,
    const int32_t* __restrict__ count,
    const double* __restrict__ alpha, const double* __restrict__ cst,
    const double* __restrict__ ap, double* __restrict__ Q,
    double* __restrict__ C, double* __restrict__ P, int32_t* __restrict__ sidx_out) {
  constexpr int MU = D == 1 ? 3 : (D == 2 ? 9 : 27);
  __shared__ int s_idx[kThreads];
  const int64_t mask = ((int64_t)1 << logn) - 1;
  const int ns = *count;
  for (int64_t j0 = (int64_t)blockIdx.x * kThreads; j0 < N; j0 += (int64_t)gridDim.x * kThreads) {
    const int npts = (int)min((int64_t)kThreads, N - j0);
    const int t = threadIdx.x;
    if (t < npts) {
      const double x = __ldg(v + j0 + t);
      int idx;
      if (LOCAL) {
        const int64_t r = snap_m(x) - mlo;
        idx = (r >= 0 && r < R) ? __ldg(idx_of + r) : -1;
        if (idx < 0) {  // cannot happen when host and device snap alike; recorded, row set to 0
          atomicOr(err, 2);
          idx = 0;
        }
      } else
        idx = nearest_shift(shift_m, ns, x);
      idx = (int)checked(idx, ns, err);
      s_idx[t] = idx;
      if (SIDX) sidx_out[j0 + t] = idx;
    }
    __syncthreads();
    if (ROWS) {
      const int64_t obase = j0 * MU;
      for (int e = t; e < npts * MU; e += kThreads) {
        const int p = e / MU, o = e - p * MU;
        const int idx = s_idx[p];
        const double a = __ldg(alpha + (int64_t)idx * MU + o);
        const double cc = __ldg(cst + (int64_t)idx * MU + o);
        const double aff = __ldg(ap + (int64_t)idx * MU + o);
        const double vn = __ldg(v + checked(neighbour<D>(j0 + p, o, logn, mask), N, err));
        __stcs(Q + obase + e, a);
        __stcs(C + obase + e, cc);
        __stcs(P + obase + e, fma(cc, vn, aff));
      }
    }
    __syncthreads();
  }
}

template <int D>
__global__ void __launch_bounds__(kThreads) k_colidx(int64_t N, int logn, int32_t* __restrict__ col,
                                                     int64_t* __restrict__ rowptr) {
  constexpr int MU = D == 1 ? 3 : (D == 2 ? 9 : 27);
  const int64_t mask = ((int64_t)1 << logn) - 1;
  for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < N * MU;
       e += (int64_t)gridDim.x * kThreads) {
    const int64_t j = e / MU;
    const int o = (int)(e - j * MU);
    col[e] = (int32_t)neighbour<D>(j, o, logn, mask);
  }
  for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j <= N;
       j += (int64_t)gridDim.x * kThreads)
    rowptr[j] = j * MU;
}

// ---- t = 2 rows (2D and 3D): 5^d columns per point in the lexicographic offset order ------
// t_j at a point: 2 without a leaf; else min(2, min_a f(x_a mod leaf)) with f(0) = leaf,
// f(r) = min(r, leaf - r): the largest t whose neighbourhood crosses no separator line (plane)
// of a nested dissection with leaf boxes of width `leaf` (Sec. 4.2).
template <int D>
__device__ __forceinline__ int t_of_point(const int64_t* x, int leaf) {
  if (leaf <= 0) return 2;
  int t = 2;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int r = (int)(x[a] % leaf);
    t = min(t, r == 0 ? leaf : min(r, leaf - r));
  }
  return t;
}

template <int D>
__device__ __forceinline__ void coords_of(int64_t j, int logn, int64_t mask, int64_t* x) {
#pragma unroll
  for (int a = D - 1; a >= 0; --a) {
    x[a] = j & mask;
    j >>= logn;
  }
}

// offsets of the o-th column of a 5^D row, and the index of the same offset in a 3^D row (or
// -1 when it lies outside [-1, 1]^D)
template <int D>
__device__ __forceinline__ int decode5(int o, int* off) {
  int inner = 0, in3 = 1;
#pragma unroll
  for (int a = D - 1; a >= 0; --a) {
    off[a] = o % 5 - 2;
    o /= 5;
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    in3 = in3 && off[a] >= -1 && off[a] <= 1;
    inner = inner * 3 + (off[a] + 1);
  }
  return in3 ? inner : -1;
}

template <int D>
__device__ __forceinline__ int64_t wrap_index(const int64_t* x, const int* off, int logn,
                                              int64_t mask) {
  int64_t g = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) g = (g << logn) | ((x[a] + off[a]) & mask);
  return g;
}

// A t_j = 2 point writes alpha2/c2 of its shift in all 5^D columns; a t_j = 1 point writes
// alpha/c of the 3^D stencil in the inner columns (|o_a| <= 1) and zeros elsewhere.
template <int D, bool LOCAL>
__global__ void __launch_bounds__(kThreads) k_rows_t2(
    const double* __restrict__ v, int64_t N, int logn, int leaf,
    const int32_t* __restrict__ idx_of, int64_t mlo, int64_t R, int32_t* __restrict__ err,
    const int32_t* __restrict__ shift_m, const int32_t* __restrict__ count,
    const double* __restrict__ alpha1, const double* __restrict__ c1,
    const double* __restrict__ alpha2, const double* __restrict__ c2, double* __restrict__ Q,
    double* __restrict__ C, double* __restrict__ P) {
  constexpr int MU = D == 2 ? 25 : 125, MU1 = D == 2 ? 9 : 27;
  __shared__ int s_idx[kThreads];
  __shared__ int s_t[kThreads];
  __shared__ double s_val[kThreads];
  const int64_t mask = ((int64_t)1 << logn) - 1;
  const int ns = *count;
  for (int64_t j0 = (int64_t)blockIdx.x * kThreads; j0 < N; j0 += (int64_t)gridDim.x * kThreads) {
    const int npts = (int)min((int64_t)kThreads, N - j0);
    const int t = threadIdx.x;
    if (t < npts) {
      const int64_t j = j0 + t;
      const double x = __ldg(v + j);
      int idx;
      if (LOCAL) {
        const int64_t r = snap_m(x) - mlo;
        idx = (r >= 0 && r < R) ? __ldg(idx_of + r) : -1;
        if (idx < 0) {
          atomicOr(err, 2);
          idx = 0;
        }
      } else {
        idx = nearest_shift(shift_m, ns, x);
      }
      idx = (int)checked(idx, ns, err);
      int64_t xc[D];
      coords_of<D>(j, logn, mask, xc);
      s_idx[t] = idx;
      s_t[t] = t_of_point<D>(xc, leaf);
      s_val[t] = shift_of(__ldg(shift_m + idx));
    }
    __syncthreads();
    const int64_t obase = j0 * MU;
    for (int e = t; e < npts * MU; e += kThreads) {
      const int p = e / MU, o = e - p * MU;
      int off[D];
      const int inner = decode5<D>(o, off);
      const int idx = s_idx[p];
      double a = 0.0, cc = 0.0;
      if (s_t[p] == 2) {
        a = __ldg(alpha2 + (int64_t)idx * MU + o);
        cc = __ldg(c2 + (int64_t)idx * MU + o);
      } else if (inner >= 0) {
        a = __ldg(alpha1 + (int64_t)idx * MU1 + inner);
        cc = __ldg(c1 + (int64_t)idx * MU1 + inner);
      }
      int64_t xc[D];
      coords_of<D>(j0 + p, logn, mask, xc);
      const double vn = __ldg(v + wrap_index<D>(xc, off, logn, mask));
      __stcs(Q + obase + e, a);
      __stcs(C + obase + e, cc);
      __stcs(P + obase + e, fma(cc, vn - s_val[p], a));
    }
    __syncthreads();
  }
}

// CSR export of a t = 2 build: row j keeps the (2 t_j + 1)^D columns of mu_j^{t_j}, in the
// lexicographic order of its own offsets (the inner 3^D of the 5^D-wide row when t_j = 1).
// rowptr holds the prefix sums of the row lengths.
template <int D>
__global__ void __launch_bounds__(kThreads) k_export_t2(const double* __restrict__ rows,
                                                        int64_t N, int logn, int leaf,
                                                        const int64_t* __restrict__ rowptr,
                                                        int32_t* __restrict__ col,
                                                        double* __restrict__ val) {
  constexpr int MU = D == 2 ? 25 : 125;
  const int64_t mask = ((int64_t)1 << logn) - 1;
  for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < N * MU;
       e += (int64_t)gridDim.x * kThreads) {
    const int64_t j = e / MU;
    const int o = (int)(e - j * MU);
    int off[D];
    const int inner = decode5<D>(o, off);
    int64_t xc[D];
    coords_of<D>(j, logn, mask, xc);
    const int tj = t_of_point<D>(xc, leaf);
    if (tj == 1 && inner < 0) continue;
    const int k = tj == 2 ? o : inner;
    const int64_t pos = rowptr[j] + k;
    col[pos] = (int32_t)wrap_index<D>(xc, off, logn, mask);
    val[pos] = rows[e];
  }
}

// ---- the learned-stencil gate (a9) --------------------------------------------------------
// Class of o_a - o_b for offsets a, b of mu_0^1 (lexicographic, last axis fastest): the sorted
// |components|, numbered as the stage tables number them (1D: 0 1 2; 2D: 00 01 02 11 12 22;
// 3D: 000 001 002 011 012 022 111 112 122 222). Compile-time, so that fully unrolled loops
// index the class values held in registers.
template <int D>
__host__ __device__ constexpr int cls1(int a, int b) {
  if (D == 1) return a - b < 0 ? b - a : a - b;
  if (D == 2) {
    const int x0 = a / 3 - b / 3, y0 = a % 3 - b % 3;
    const int x = x0 < 0 ? -x0 : x0, y = y0 < 0 ? -y0 : y0;
    const int lo = x < y ? x : y, hi = x < y ? y : x;
    return lo == 0 ? hi : (lo == 1 ? 2 + hi : 5);
  }
  const int p0 = a / 9 - b / 9, q0 = (a / 3) % 3 - (b / 3) % 3, r0 = a % 3 - b % 3;
  int x = p0 < 0 ? -p0 : p0, y = q0 < 0 ? -q0 : q0, z = r0 < 0 ? -r0 : r0;
  if (x > y) { const int t = x; x = y; y = t; }
  if (y > z) { const int t = y; y = z; z = t; }
  if (x > y) { const int t = x; x = y; y = t; }
  if (x == 0) return y == 0 ? z : (y == 1 ? 2 + z : 5);
  if (x == 1) return 6 + (y - 1) + (z - 1);
  return 9;
}

// Per point j, with alpha the learned Q row (normalised, sign matched to the eigen path's
// alpha* of the point's shift s_j) and delta = alpha - alpha*:
//   ||alpha^T G_s[mu, mu^c]||^2 = alpha^T A alpha = lambda_1 + delta^T (A - lambda_1 I) delta,
// since A alpha* = lambda_1 alpha* and |alpha| = |alpha*| = 1 (Sec. 3: the optimum of the
// sparsification problem is the smallest singular value, lambda_1 = sigma_min^2). The ratio
//   rho_j = ||alpha^T G[mu, mu^c]|| / sigma_min = sqrt(1 + delta^T (A - lambda_1 I) delta / lambda_1)
// has no cancellation in this form (A - lambda_1 I is positive semidefinite and delta small),
// so the quadratic form is evaluated in FP32 from the class values of g_s and g_s * g_s
// (A = A1 - Gm Gm^T, Eq. A). A point with rho_j > tau (or an unusable lambda_1) falls back to
// the eigen path: its Q, C and P rows are rewritten from alpha*, c* of its shift (a7). A point
// that passes keeps its learned Q row, and its C and P rows are formed from it in FP64.
template <int D, bool LOCAL>
__global__ void __launch_bounds__(kThreads) k_learned_gate(
    const double* __restrict__ v, int64_t N, int logn, const int32_t* __restrict__ idx_of,
    int64_t mlo, int64_t R, const int32_t* __restrict__ shift_m,
    const int32_t* __restrict__ count, int64_t cap, const double* __restrict__ gvals,
    const double* __restrict__ alpha, const double* __restrict__ cst,
    const double* __restrict__ ap, const double* __restrict__ lam, double tau2,
    double* __restrict__ Q, double* __restrict__ C, double* __restrict__ P,
    float* __restrict__ rho, int32_t* __restrict__ nfall, int32_t* __restrict__ err) {
  constexpr int MU = D == 1 ? 3 : (D == 2 ? 9 : 27);
  constexpr int NC = D == 1 ? 3 : (D == 2 ? 6 : 10);
  const int64_t mask = ((int64_t)1 << logn) - 1;
  const int ns = *count;
  for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * kThreads) {
    const double x = __ldg(v + j);
    int idx;
    if (LOCAL) {
      const int64_t r = snap_m(x) - mlo;
      idx = (r >= 0 && r < R) ? __ldg(idx_of + r) : -1;
      if (idx < 0) {
        atomicOr(err, 2);
        idx = 0;
      }
    } else {
      idx = nearest_shift(shift_m, ns, x);
    }
    idx = (int)checked(idx, ns, err);
    double al[MU], as[MU];
    double nrm2 = 0.0, dot = 0.0;
#pragma unroll
    for (int a = 0; a < MU; ++a) {
      al[a] = Q[j * MU + a];
      as[a] = __ldg(alpha + (int64_t)idx * MU + a);
      nrm2 = fma(al[a], al[a], nrm2);
      dot = fma(al[a], as[a], dot);
    }
    // the residual does not depend on the row's sign: match it to alpha*
    const double scl = (nrm2 > 0.0 ? 1.0 / sqrt(nrm2) : 0.0) * (dot < 0.0 ? -1.0 : 1.0);
    float dl[MU];
    float dd = 0.0f;
#pragma unroll
    for (int a = 0; a < MU; ++a) {
      dl[a] = (float)(fma(al[a], scl, -as[a]));
      dd = fmaf(dl[a], dl[a], dd);
    }
    float g[NC], g2[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      g[c] = (float)__ldg(gvals + (int64_t)(2 * c) * cap + idx);
      g2[c] = (float)__ldg(gvals + (int64_t)(2 * c + 1) * cap + idx);
    }
    float q1 = 0.0f, q2 = 0.0f;  // delta^T A1 delta and |Gm delta|^2
#pragma unroll
    for (int b = 0; b < MU; ++b) {
      float w = 0.0f, u = 0.0f;
#pragma unroll
      for (int a = 0; a < MU; ++a) {
        w = fmaf(g[cls1<D>(a, b)], dl[a], w);
        u = fmaf(g2[cls1<D>(a, b)], dl[a], u);
      }
      q1 = fmaf(dl[b], u, q1);
      q2 = fmaf(w, w, q2);
    }
    const double l1 = __ldg(lam + 2 * (int64_t)idx);
    const double r2 = 1.0 + ((double)q1 - (double)q2 - l1 * (double)dd) / l1;
    const bool ok = nrm2 > 0.0 && l1 > 0.0 && r2 <= tau2;  // false for NaN as well
    rho[j] = (l1 > 0.0 && nrm2 > 0.0 && r2 == r2) ? (float)sqrt(fmax(r2, 1.0)) : INFINITY;
    if (ok) {
      // the network supplies alpha only: C and P follow from it by the method's formulas,
      // C[j, mu_j] = Q[j, mu_j] G_s[mu_j, mu_j] and P = Q + C diag(v - s) (Sec. 4.1), in FP64
      double gd[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) gd[c] = __ldg(gvals + (int64_t)(2 * c) * cap + idx);
      const double s = shift_of(__ldg(shift_m + idx));
#pragma unroll
      for (int b = 0; b < MU; ++b) {
        double cb = 0.0;
#pragma unroll
        for (int a = 0; a < MU; ++a) cb = fma(al[a], gd[cls1<D>(a, b)], cb);
        const double vn = __ldg(v + neighbour<D>(j, b, logn, mask));
        C[j * MU + b] = cb;
        P[j * MU + b] = fma(cb, vn - s, al[b]);
      }
    } else {
      // the eigen path's rows, formed exactly as k_rows forms them
      atomicAdd(nfall, 1);
#pragma unroll 1
      for (int a = 0; a < MU; ++a) {
        const double aa = __ldg(alpha + (int64_t)idx * MU + a);
        const double cc = __ldg(cst + (int64_t)idx * MU + a);
        const double aff = __ldg(ap + (int64_t)idx * MU + a);
        const double vn = __ldg(v + neighbour<D>(j, a, logn, mask));
        Q[j * MU + a] = aa;
        C[j * MU + a] = cc;
        P[j * MU + a] = fma(cc, vn, aff);
      }
    }
  }
}

int log2i(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

template <int D, bool LOCAL, bool ROWS, bool SIDX>
void launch_rows_t(lsp_ctx* c, const int32_t* count) {
  const int64_t N = c->geo.N;
  auto go = [&](LaunchShape sh) {
    int64_t b = (N + kThreads - 1) / kThreads;
    if (b > 152 * (int64_t)sh.per_sm) b = 152 * (int64_t)sh.per_sm;
    k_rows<D, LOCAL, ROWS, SIDX><<<(int)b, kThreads, 0, c->stream>>>(
        (const double*)c->v.p, N, log2i(c->geo.n), (const int32_t*)c->idx_of.p, c->mrange.lo,
        c->mrange.size(), (int32_t*)c->counts.p + kErrWord, (const int32_t*)c->shift_m.p,
        count, (const double*)c->alpha.p, (const double*)c->cst.p, (const double*)c->ap.p,
        (double*)c->Q.p, (double*)c->C.p, (double*)c->P.p, (int32_t*)c->sidx.p);
    return cudaGetLastError();
  };
  if (!ROWS) {  // the shift-index export is not tuned
    go({kThreads, 16});
    return;
  }
  // one block per 256 points (shared tables are sized for it): only the grid cap is tuned
  tuned_launch(c, std::string("rows/d") + std::to_string(D) + (LOCAL ? "/local" : "/list") + "/w" +
                      work_bucket(N),
               {kThreads, 16}, kThreads, kThreads, go);
}

template <bool ROWS, bool SIDX>
void dispatch_rows(lsp_ctx* c, int policy, const int32_t* count) {
  const bool local = policy == LSP_SHIFT_LOCAL;
  if (c->geo.d == 1) {
    if (local)
      launch_rows_t<1, true, ROWS, SIDX>(c, count);
    else
      launch_rows_t<1, false, ROWS, SIDX>(c, count);
  } else if (c->geo.d == 2) {
    if (local)
      launch_rows_t<2, true, ROWS, SIDX>(c, count);
    else
      launch_rows_t<2, false, ROWS, SIDX>(c, count);
  } else {
    if (local)
      launch_rows_t<3, true, ROWS, SIDX>(c, count);
    else
      launch_rows_t<3, false, ROWS, SIDX>(c, count);
  }
}

}  // namespace

cudaError_t launch_rows(lsp_ctx* c, int policy, const int32_t* count) {
  int t = timer_begin(c, "rows");
  dispatch_rows<true, false>(c, policy, count);
  timer_end(c, t);
  return cudaGetLastError();
}

cudaError_t launch_learned_gate(lsp_ctx* c, int policy, const int32_t* count, int64_t cap,
                                double tau, float* rho, int32_t* nfall) {
  const int64_t N = c->geo.N;
  int64_t b = (N + kThreads - 1) / kThreads;
  if (b > 152 * 16) b = 152 * 16;
  int t = timer_begin(c, "gate");
  auto args = [&](auto kern) {
    kern<<<(int)b, kThreads, 0, c->stream>>>(
        (const double*)c->v.p, N, log2i(c->geo.n), (const int32_t*)c->idx_of.p, c->mrange.lo,
        c->mrange.size(), (const int32_t*)c->shift_m.p, count, cap, (const double*)c->gvals.p,
        (const double*)c->alpha.p, (const double*)c->cst.p, (const double*)c->ap.p,
        (const double*)c->lam.p, tau * tau,
        (double*)c->Q.p, (double*)c->C.p, (double*)c->P.p, rho, nfall,
        (int32_t*)c->counts.p + kErrWord);
  };
  const bool local = policy == LSP_SHIFT_LOCAL;
  if (c->geo.d == 1) {
    if (local) args(k_learned_gate<1, true>); else args(k_learned_gate<1, false>);
  } else if (c->geo.d == 2) {
    if (local) args(k_learned_gate<2, true>); else args(k_learned_gate<2, false>);
  } else {
    if (local) args(k_learned_gate<3, true>); else args(k_learned_gate<3, false>);
  }
  timer_end(c, t);
  return cudaGetLastError();
}

cudaError_t launch_sidx(lsp_ctx* c, int policy, const int32_t* count) {
  int t = timer_begin(c, "sidx");
  dispatch_rows<false, true>(c, policy, count);
  timer_end(c, t);
  return cudaGetLastError();
}

cudaError_t launch_rows_t2(lsp_ctx* c, int policy, const int32_t* count, int leaf) {
  const int64_t N = c->geo.N;
  int64_t b = (N + kThreads - 1) / kThreads;
  if (b > 152 * 16) b = 152 * 16;
  int t = timer_begin(c, "rows");
  auto args = [&](auto kern) {
    kern<<<(int)b, kThreads, 0, c->stream>>>(
        (const double*)c->v.p, N, log2i(c->geo.n), leaf, (const int32_t*)c->idx_of.p,
        c->mrange.lo, c->mrange.size(), (int32_t*)c->counts.p + kErrWord,
        (const int32_t*)c->shift_m.p, count, (const double*)c->alpha.p, (const double*)c->cst.p,
        (const double*)c->alpha2.p, (const double*)c->cst2.p, (double*)c->Q.p, (double*)c->C.p,
        (double*)c->P.p);
  };
  const bool local = policy == LSP_SHIFT_LOCAL;
  if (c->geo.d == 2) {
    if (local)
      args(k_rows_t2<2, true>);
    else
      args(k_rows_t2<2, false>);
  } else {
    if (local)
      args(k_rows_t2<3, true>);
    else
      args(k_rows_t2<3, false>);
  }
  timer_end(c, t);
  return cudaGetLastError();
}

cudaError_t launch_export_t2(lsp_ctx* c, const double* rows, int leaf, const int64_t* rowptr,
                             int32_t* colidx, double* vals) {
  const int64_t work = c->geo.N * (c->geo.d == 2 ? 25 : 125);
  int64_t b = (work + kThreads - 1) / kThreads;
  if (b > 152 * 16) b = 152 * 16;
  if (c->geo.d == 2)
    k_export_t2<2><<<(int)b, kThreads, 0, c->stream>>>(rows, c->geo.N, log2i(c->geo.n), leaf,
                                                       rowptr, colidx, vals);
  else
    k_export_t2<3><<<(int)b, kThreads, 0, c->stream>>>(rows, c->geo.N, log2i(c->geo.n), leaf,
                                                       rowptr, colidx, vals);
  return cudaGetLastError();
}

cudaError_t launch_colidx(lsp_ctx* c) {
  const int64_t work = c->geo.N * c->geo.mu;
  int64_t b = (work + kThreads - 1) / kThreads;
  if (b > 152 * 16) b = 152 * 16;
  int t = timer_begin(c, "colidx");
  if (c->geo.d == 1)
    k_colidx<1><<<(int)b, kThreads, 0, c->stream>>>(c->geo.N, log2i(c->geo.n),
                                                     (int32_t*)c->colidx.p, (int64_t*)c->rowptr.p);
  else if (c->geo.d == 2)
    k_colidx<2><<<(int)b, kThreads, 0, c->stream>>>(c->geo.N, log2i(c->geo.n),
                                                     (int32_t*)c->colidx.p, (int64_t*)c->rowptr.p);
  else
    k_colidx<3><<<(int)b, kThreads, 0, c->stream>>>(c->geo.N, log2i(c->geo.n),
                                                     (int32_t*)c->colidx.p, (int64_t*)c->rowptr.p);
  timer_end(c, t);
  return cudaGetLastError();
}

}  // namespace lsp
