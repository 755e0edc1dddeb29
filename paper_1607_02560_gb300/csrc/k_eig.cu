// Steps a4-a6 for every shift, one warp per shift, FP64:
//   a4  A = A1 - A2 (Eq. A): A1[a,b] = (g_s*g_s)[o_a - o_b], A2 = G_s[mu,mu] G_s[mu,mu]^T with
//       G_s[mu,mu][a,b] = g_s[o_a - o_b]  (translation invariance, Sec. 4.2);
//   a5  alpha = eigenvector of the smallest eigenvalue of A (Sec. 4.2), ||alpha|| = 1,
//       alpha[centre] > 0 (else the first entry above 1e-12 in magnitude is made positive);
//   a6  c = alpha^T G_s[mu, mu]  (C[j, mu_j] of Sec. 4.1).
//
// A commutes with the signed permutations of the axes acting on mu_0, because g_s[o] depends
// on o only through the multiset {|o_i|}. In a symmetry-adapted basis (one row of every
// irreducible representation occurring in mu_0) A is block diagonal, so its spectrum is the
// union of the spectra of a few blocks of size <= 4 (3 + 1 + 1 + 2x2 in 2D; 4 + 3x3 + 2x2 +
// 3x2 + 3x1 + 1 in 3D). LSP_EIG_SYMMETRIC solves those blocks; LSP_EIG_FULL runs cyclic Jacobi
// on the whole |mu| x |mu| matrix. Both give every eigenvalue, so lambda_2 and the degeneracy
// flag are exact in either method.
#include <float.h>
#include <string.h>

#include "lsp_internal.h"

namespace lsp {
namespace {

__constant__ uint8_t c_cls[kMaxMu][kMaxMu];
__constant__ SymBasis c_sym;
// Projection entries (block, i, j), i <= j, for the symmetric method.
__constant__ int8_t c_ent[64][3];
__constant__ int c_nent;

// Cyclic Jacobi on a small symmetric matrix held by one thread. a is dim x dim (row-major,
// leading dimension 4) and is overwritten; v receives the eigenvectors as columns.
// Rotations follow the standard choice tan(phi) = sign(theta) / (|theta| + sqrt(theta^2 + 1)),
// theta = (a_qq - a_pp) / (2 a_pq); off-diagonal entries at or below 1e-17 sqrt|a_pp a_qq| are
// treated as converged (relative criterion, accurate for positive semidefinite matrices).
template <int NM>
__device__ int jacobi_nm(double (&a)[NM][NM], double (&v)[NM][NM], int dim) {
  for (int i = 0; i < NM; ++i)
    for (int j = 0; j < NM; ++j) v[i][j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 40; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < dim - 1; ++p) {
      for (int q = p + 1; q < dim; ++q) {
        const double apq = a[p][q];
        if (fabs(apq) <= 1e-17 * sqrt(fabs(a[p][p] * a[q][q])) || apq == 0.0) {
          a[p][q] = a[q][p] = 0.0;
          continue;
        }
        rotated = true;
        const double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
        double t;
        if (fabs(theta) > 1e150)
          t = 0.5 / theta;
        else
          t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < dim; ++k) {
          const double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < dim; ++k) {
          const double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
        a[p][q] = a[q][p] = 0.0;
        for (int k = 0; k < dim; ++k) {
          const double vkp = v[k][p], vkq = v[k][q];
          v[k][p] = c * vkp - s * vkq;
          v[k][q] = s * vkp + c * vkq;
        }
      }
    }
    if (!rotated) return 1;
  }
  return 0;
}
__device__ int jacobi_small(double a[4][4], double v[4][4], int dim) {
  return jacobi_nm<4>(*reinterpret_cast<double(*)[4][4]>(a), *reinterpret_cast<double(*)[4][4]>(v),
                      dim);
}

// Per-block copies of the class table and the symmetry-adapted vectors: the warp kernel
// indexes them with lane-dependent indices, which constant memory would serialise.

// 2^-e for the exponent of |x| (exact scaling without FP64 arithmetic on the exponent).
__device__ __forceinline__ double pow2_inv_exp(double x) {
  const long long bits = __double_as_longlong(x) & 0x7ff0000000000000LL;
  if (bits == 0 || bits == 0x7ff0000000000000LL) return 1.0;
  return __longlong_as_double(0x7fe0000000000000LL - bits);  // 2^(1023 - e) * 2^... = 2^-e
}

// LDL^T factorisation (no pivoting) of a symmetric positive definite dim x dim matrix; returns
// false if a pivot is not positive. L unit lower triangular, id = 1 / D.
__device__ __forceinline__ bool ldlt(const double s[4][4], int dim, double L[4][4],
                                     double id[4]) {
  double d[4];
  for (int j = 0; j < dim; ++j) {
    double dj = s[j][j];
    for (int k = 0; k < j; ++k) dj -= L[j][k] * L[j][k] * d[k];
    if (!(dj > 0.0)) return false;
    d[j] = dj;
    id[j] = 1.0 / dj;
    for (int i = j + 1; i < dim; ++i) {
      double a = s[i][j];
      for (int k = 0; k < j; ++k) a -= L[i][k] * L[j][k] * d[k];
      L[i][j] = a * id[j];
    }
  }
  return true;
}

// x <- (L D L^T)^-1 x, renormalised by a power of two.
__device__ __forceinline__ void ldlt_solve(const double L[4][4], const double id[4], int dim,
                                           double x[4]) {
  for (int i = 0; i < dim; ++i)
    for (int k = 0; k < i; ++k) x[i] -= L[i][k] * x[k];
  for (int i = 0; i < dim; ++i) x[i] *= id[i];
  for (int i = dim - 1; i >= 0; --i)
    for (int k = i + 1; k < dim; ++k) x[i] -= L[k][i] * x[k];
  double mx = 0.0;
  for (int i = 0; i < dim; ++i) mx = fmax(mx, fabs(x[i]));
  const double p2 = pow2_inv_exp(mx);
  for (int i = 0; i < dim; ++i) x[i] *= p2;
}

// Smallest eigenpair of a small symmetric positive semidefinite block (dim <= 4) by inverse
// iteration with one LDL^T factorisation, checked by its residual; cyclic Jacobi when the
// factorisation fails or the iteration has not converged. *lam2 receives the block's next
// eigenvalue (inverse iteration on the block deflated by the first pair; used for the
// degeneracy flag only). Far fewer FP64 instructions than Jacobi's divide/square-root chains.
__device__ int block_min_eig(const double b[4][4], int dim, double y[4], double* lam_min,
                             double* lam2) {
  y[0] = y[1] = y[2] = y[3] = 0.0;
  if (dim == 1) {
    y[0] = 1.0;
    *lam_min = b[0][0];
    *lam2 = DBL_MAX;
    return 1;
  }
  double sc = 0.0;
  for (int i = 0; i < dim; ++i)
    for (int j = 0; j < dim; ++j) sc = fmax(sc, fabs(b[i][j]));
  const double isc = sc > 0 ? 1.0 / sc : 0.0;
  double s[4][4], L[4][4], id[4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      s[i][j] = (i < dim && j < dim) ? b[i][j] * isc : 0.0;
      L[i][j] = 0.0;
    }
  bool ok = ldlt(s, dim, L, id);
  double x[4] = {1.0, 0.5, 0.25, 0.125};
  double ls = 0.0;
  if (ok) {
    for (int it = 0; it < 40; ++it) ldlt_solve(L, id, dim, x);
    double nrm = 0.0;
    for (int i = 0; i < dim; ++i) nrm = fma(x[i], x[i], nrm);
    const double inv = rsqrt(nrm);
    double r[4] = {0, 0, 0, 0}, res = 0.0;
    for (int i = 0; i < dim; ++i) x[i] *= inv;
    for (int i = 0; i < dim; ++i) {
      for (int j = 0; j < dim; ++j) r[i] = fma(s[i][j], x[j], r[i]);
      ls = fma(x[i], r[i], ls);
    }
    for (int i = 0; i < dim; ++i) res = fmax(res, fabs(r[i] - ls * x[i]));
    ok = res <= 64 * 2.2e-16 && isfinite(ls);
  }
  if (!ok) {
    double a[4][4], vv[4][4];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) a[i][j] = s[i][j];
    const int conv = jacobi_small(a, vv, dim);
    int kk = 0;
    for (int i = 1; i < dim; ++i)
      if (a[i][i] < a[kk][kk]) kk = i;
    double second = DBL_MAX;
    for (int i = 0; i < dim; ++i)
      if (i != kk) second = fmin(second, a[i][i]);
    for (int i = 0; i < dim; ++i) y[i] = vv[i][kk];
    *lam_min = a[kk][kk] * sc;
    *lam2 = second * sc;
    return conv;
  }
  for (int i = 0; i < dim; ++i) y[i] = x[i];
  *lam_min = ls * sc;
  // second eigenvalue: move the found one above the others, iterate again
  double tr = 0.0;
  for (int i = 0; i < dim; ++i) tr += s[i][i];
  const double shift = fabs(tr) + 1.0;
  for (int i = 0; i < dim; ++i)
    for (int j = 0; j < dim; ++j) s[i][j] = fma(shift * y[i], y[j], s[i][j]);
  double z[4] = {0.125, 0.25, 0.5, 1.0};
  if (ldlt(s, dim, L, id)) {
    for (int it = 0; it < 12; ++it) ldlt_solve(L, id, dim, z);
    double nrm = 0.0, q = 0.0;
    for (int i = 0; i < dim; ++i) nrm = fma(z[i], z[i], nrm);
    for (int i = 0; i < dim; ++i) {
      double r = 0.0;
      for (int j = 0; j < dim; ++j) r = fma(s[i][j], z[j], r);
      q = fma(z[i], r, q);
    }
    *lam2 = (q / nrm) * sc;
  } else {
    *lam2 = *lam_min;  // degenerate
  }
  return 1;
}

template <int MU>
struct __align__(16) BlockTables {
  double u[kMaxSymVec][MU];
  uint8_t cls[MU][MU];
};

template <int MU>
struct __align__(16) WarpSmem {
  double A[MU * MU];
  double V[MU * MU];
  double g[2 * kMaxCls];
  double B[kMaxSymBlk][16];
  double lam[kMaxSymBlk][4];
  double y[kMaxSymBlk][4];
  double alpha[MU];
  double work[MU + 1];
  int conv[kMaxSymBlk];
};

// Sign convention: alpha[centre] > 0, else the first entry with |alpha| > 1e-12.
template <int MU>
__device__ void sign_fix(double* alpha, int centre) {
  double ref = alpha[centre];
  if (!(fabs(ref) > 1e-12)) {
    ref = 0.0;
    for (int a = 0; a < MU; ++a)
      if (fabs(alpha[a]) > 1e-12) {
        ref = alpha[a];
        break;
      }
  }
  if (ref < 0)
    for (int a = 0; a < MU; ++a) alpha[a] = -alpha[a];
}

// Lane-parallel cyclic Jacobi on the whole MU x MU matrix in shared memory (lane k owns row
// and column k in each update). Returns 1 when converged.
template <int MU>
__device__ int jacobi_full(WarpSmem<MU>& sm, int lane) {
  double* A = sm.A;
  double* V = sm.V;
  for (int e = lane; e < MU * MU; e += 32) V[e] = (e / MU == e % MU) ? 1.0 : 0.0;
  __syncwarp();
  for (int sweep = 0; sweep < 40; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < MU - 1; ++p) {
      for (int q = p + 1; q < MU; ++q) {
        const double apq = A[p * MU + q], app = A[p * MU + p], aqq = A[q * MU + q];
        __syncwarp();
        if (fabs(apq) <= 1e-17 * sqrt(fabs(app * aqq)) || apq == 0.0) continue;
        rotated = true;
        const double theta = (aqq - app) / (2.0 * apq);
        double t;
        if (fabs(theta) > 1e150)
          t = 0.5 / theta;
        else
          t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        if (lane < MU) {
          const double akp = A[lane * MU + p], akq = A[lane * MU + q];
          A[lane * MU + p] = c * akp - s * akq;
          A[lane * MU + q] = s * akp + c * akq;
        }
        __syncwarp();
        if (lane < MU) {
          const double apk = A[p * MU + lane], aqk = A[q * MU + lane];
          A[p * MU + lane] = c * apk - s * aqk;
          A[q * MU + lane] = s * apk + c * aqk;
          const double vkp = V[lane * MU + p], vkq = V[lane * MU + q];
          V[lane * MU + p] = c * vkp - s * vkq;
          V[lane * MU + q] = s * vkp + c * vkq;
        }
        __syncwarp();
        if (lane == 0) A[p * MU + q] = A[q * MU + p] = 0.0;
        __syncwarp();
      }
    }
    if (!rotated) return 1;
  }
  return 0;
}

// One inverse-iteration step in FP64: alpha <- (A0 - sigma I)^-1 alpha / ||.||, sigma the
// Rayleigh quotient of alpha. A0 is rebuilt from g (A may have been overwritten). Gaussian
// elimination with partial pivoting, lanes own columns. A zero pivot leaves alpha unchanged.
template <int MU>
__device__ void refine_step(WarpSmem<MU>& sm, const BlockTables<MU>& tb, int lane, int centre) {
  double* M = sm.V;  // the matrix (A0 - sigma I); the right-hand side lives in sm.work
  for (int e = lane; e < MU * MU; e += 32) {
    const int a = e / MU, b = e % MU;
    double s = 0.0;
    for (int k = 0; k < MU; ++k) s = fma(sm.g[2 * tb.cls[a][k]], sm.g[2 * tb.cls[b][k]], s);
    M[e] = sm.g[2 * tb.cls[a][b] + 1] - s;
  }
  __syncwarp();
  // Rayleigh quotient
  double part = 0.0;
  if (lane < MU) {
    double r = 0.0;
    for (int b = 0; b < MU; ++b) r = fma(M[lane * MU + b], sm.alpha[b], r);
    part = r * sm.alpha[lane];
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  const double sigma = part;
  if (lane < MU) {
    M[lane * MU + lane] -= sigma;
    sm.work[lane] = sm.alpha[lane];
  }
  __syncwarp();
  bool ok = true;
  for (int k = 0; k < MU; ++k) {
    // pivot search (every lane reads the same shared data and picks the same row)
    int piv = k;
    double best = fabs(M[k * MU + k]);
    for (int r = k + 1; r < MU; ++r) {
      const double x = fabs(M[r * MU + k]);
      if (x > best) {
        best = x;
        piv = r;
      }
    }
    if (best == 0.0) {
      ok = false;
      break;
    }
    __syncwarp();
    if (piv != k && lane < MU) {
      const double t0 = M[k * MU + lane];
      M[k * MU + lane] = M[piv * MU + lane];
      M[piv * MU + lane] = t0;
    }
    if (piv != k && lane == 0) {
      const double t1 = sm.work[k];
      sm.work[k] = sm.work[piv];
      sm.work[piv] = t1;
    }
    __syncwarp();
    const double dkk = M[k * MU + k];
    const double bk = sm.work[k];
    // lane r > k eliminates row r
    if (lane > k && lane < MU) {
      const double f = M[lane * MU + k] / dkk;
      for (int cidx = k; cidx < MU; ++cidx) M[lane * MU + cidx] -= f * M[k * MU + cidx];
      sm.work[lane] -= f * bk;
    }
    __syncwarp();
  }
  if (!ok) return;
  if (lane == 0) {
    for (int r = MU - 1; r >= 0; --r) {
      double s = sm.work[r];
      for (int cidx = r + 1; cidx < MU; ++cidx) s -= M[r * MU + cidx] * sm.work[cidx];
      sm.work[r] = s / M[r * MU + r];
    }
    double nrm = 0.0;
    for (int r = 0; r < MU; ++r) nrm = fma(sm.work[r], sm.work[r], nrm);
    nrm = sqrt(nrm);
    if (nrm > 0 && isfinite(nrm)) {
      for (int r = 0; r < MU; ++r) sm.alpha[r] = sm.work[r] / nrm;
      sign_fix<MU>(sm.alpha, centre);
    }
  }
  __syncwarp();
}

template <int MU, int NCLS, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_eig(const double* __restrict__ gvals,
                                                    int64_t cap, const int32_t* __restrict__ count,
                                                    int method, int refine,
                                                    double* __restrict__ alpha_out,
                                                    double* __restrict__ c_out,
                                                    double* __restrict__ lam_out,
                                                    int32_t* __restrict__ flags_out,
                                                    const int32_t* __restrict__ shift_m,
                                                    double* __restrict__ ap_out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  BlockTables<MU>& tb = *reinterpret_cast<BlockTables<MU>*>(smraw);
  WarpSmem<MU>& sm =
      reinterpret_cast<WarpSmem<MU>*>(smraw + ((sizeof(BlockTables<MU>) + 15) / 16) * 16)[w];
  for (int e = threadIdx.x; e < kMaxSymVec * MU; e += WARPS * 32)
    tb.u[e / MU][e % MU] = c_sym.u[e / MU][e % MU];
  for (int e = threadIdx.x; e < MU * MU; e += WARPS * 32) tb.cls[e / MU][e % MU] = c_cls[e / MU][e % MU];
  __syncthreads();
  const int64_t cnt = *count;
  const int centre = MU / 2;
  for (int64_t i = (int64_t)blockIdx.x * WARPS + w; i < cnt; i += (int64_t)gridDim.x * WARPS) {
    if (lane < 2 * NCLS) sm.g[lane] = gvals[(int64_t)lane * cap + i];
    __syncwarp();
    // a4: A = A1 - G G^T
    for (int e = lane; e < MU * MU; e += 32) {
      const int a = e / MU, b = e % MU;
      double s = 0.0;
      for (int k = 0; k < MU; ++k) s = fma(sm.g[2 * tb.cls[a][k]], sm.g[2 * tb.cls[b][k]], s);
      sm.A[e] = sm.g[2 * tb.cls[a][b] + 1] - s;
    }
    __syncwarp();
    double lam1 = 0, lam2 = 0, lmax = 0;
    int flags = 0;
    if (method == LSP_EIG_FULL) {
      const int conv = jacobi_full<MU>(sm, lane);
      if (lane == 0) {
        int best = 0;
        for (int a = 1; a < MU; ++a)
          if (sm.A[a * MU + a] < sm.A[best * MU + best]) best = a;
        lam1 = sm.A[best * MU + best];
        lam2 = DBL_MAX;
        for (int a = 0; a < MU; ++a) {
          const double x = sm.A[a * MU + a];
          lmax = fmax(lmax, fabs(x));
          if (a != best) lam2 = fmin(lam2, x);
        }
        for (int a = 0; a < MU; ++a) sm.alpha[a] = sm.V[a * MU + best];
        if (!conv) flags |= LSP_FLAG_NOT_CONVERGED;
      }
    } else {
      // projections B_b[i][j] = u_i^T A u_j
      for (int ent = lane; ent < c_nent; ent += 32) {
        const int b = c_ent[ent][0], ii = c_ent[ent][1], jj = c_ent[ent][2];
        const double* ui = tb.u[c_sym.first[b] + ii];
        const double* uj = tb.u[c_sym.first[b] + jj];
        double s = 0.0;
        for (int a = 0; a < MU; ++a) {
          if (ui[a] == 0.0) continue;
          double r = 0.0;
          for (int cc = 0; cc < MU; ++cc)
            if (uj[cc] != 0.0) r = fma(sm.A[a * MU + cc], uj[cc], r);
          s = fma(ui[a], r, s);
        }
        sm.B[b][ii * 4 + jj] = s;
        sm.B[b][jj * 4 + ii] = s;
      }
      __syncwarp();
      if (lane < c_sym.nblk) {
        const int dim = c_sym.dim[lane];
        double a[4][4], y[4], lmin, l2;
        for (int r = 0; r < 4; ++r)
          for (int q = 0; q < 4; ++q) a[r][q] = (r < dim && q < dim) ? sm.B[lane][r * 4 + q] : 0.0;
        if (dim == 2) {
          // closed form for 2 x 2 blocks
          const double m = 0.5 * (a[0][0] + a[1][1]), h = 0.5 * (a[0][0] - a[1][1]);
          const double rr = sqrt(fma(h, h, a[0][1] * a[0][1]));
          const double hi = m + rr;
          lmin = hi != 0.0 ? (a[0][0] * a[1][1] - a[0][1] * a[0][1]) / hi : m - rr;
          l2 = hi;
          double p = a[0][1], q = lmin - a[0][0];
          if (fabs(a[0][0] - lmin) < fabs(a[1][1] - lmin)) {
            p = lmin - a[1][1];
            q = a[0][1];
          }
          double nr = sqrt(p * p + q * q);
          if (nr == 0) { p = 1; q = 0; nr = 1; }
          y[0] = p / nr;
          y[1] = q / nr;
          y[2] = y[3] = 0.0;
          sm.conv[lane] = 1;
        } else {
          sm.conv[lane] = block_min_eig(a, dim, y, &lmin, &l2);
        }
        sm.lam[lane][0] = lmin;
        sm.lam[lane][1] = dim > 1 ? l2 : DBL_MAX;
        sm.lam[lane][2] = DBL_MAX;
        sm.lam[lane][3] = DBL_MAX;
        double tr = 0.0;
        for (int r = 0; r < dim; ++r) tr += a[r][r];
        sm.work[lane] = tr;  // bound of the block's largest eigenvalue (PSD blocks)
        for (int r = 0; r < 4; ++r) sm.y[lane][r] = y[r];
      }
      __syncwarp();
      if (lane == 0) {
        int bstar = 0;
        for (int b = 1; b < c_sym.nblk; ++b)
          if (sm.lam[b][0] < sm.lam[bstar][0]) bstar = b;
        lam1 = sm.lam[bstar][0];
        lam2 = DBL_MAX;
        for (int b = 0; b < c_sym.nblk; ++b) lmax = fmax(lmax, fabs(sm.work[b]));
        for (int b = 0; b < c_sym.nblk; ++b) {
          for (int r = 0; r < c_sym.dim[b] && r < 2; ++r) {
            if (b == bstar && r == 0) {
              if (c_sym.copies[b] > 1) lam2 = fmin(lam2, sm.lam[b][r]);
              continue;
            }
            lam2 = fmin(lam2, sm.lam[b][r]);
          }
          if (!sm.conv[b]) flags |= LSP_FLAG_NOT_CONVERGED;
        }
        if (bstar != 0) flags |= LSP_FLAG_NONSYMMETRIC;
        for (int a = 0; a < MU; ++a) {
          double s = 0.0;
          for (int r = 0; r < c_sym.dim[bstar]; ++r)
            s = fma(sm.y[bstar][r], tb.u[c_sym.first[bstar] + r][a], s);
          sm.alpha[a] = s;
        }
      }
    }
    if (lane == 0) {
      if (lam2 - lam1 < 1e-8 * lmax) flags |= LSP_FLAG_DEGENERATE;
      sign_fix<MU>(sm.alpha, centre);
    }
    __syncwarp();
    for (int r = 0; r < refine; ++r) refine_step<MU>(sm, tb, lane, centre);
    // a6: c[b] = sum_a alpha[a] G[a, b]
    if (lane < MU) {
      double s = 0.0;
      for (int a = 0; a < MU; ++a) s = fma(sm.g[2 * tb.cls[a][lane]], sm.alpha[a], s);
      alpha_out[i * MU + lane] = sm.alpha[lane];
      c_out[i * MU + lane] = s;
      // P rows are fma(c, v, alpha - c s_i) (see k_rows)
      ap_out[i * MU + lane] = fma(-s, lattice_shift(__ldg(shift_m + i)), sm.alpha[lane]);
    }
    if (lane == 0) {
      lam_out[2 * i + 0] = lam1;
      lam_out[2 * i + 1] = lam2;
      flags_out[i] = flags;
    }
    __syncwarp();
  }
}

// ---- 3D, one warp per shift, blocks formed from the class values --------------------------
// The blocks of A in 3D are A1g (4 x 4), T1u (3 x 3), Eg and T2g (2 x 2), T2u and A2u (1 x 1),
// each on the vectors U_b of one partner of an irreducible representation. G = G_s[mu, mu]
// commutes with the symmetry group, so it maps span(U_b) into itself: G U_b = U_b G_b with
// G_b = U_b^T G U_b, and the block of A = A1 - G G^T is B_b = U_b^T A1 U_b - G_b G_b. Both
// U_b^T A1 U_b and G_b are linear in the class values, X_b[i][j] = sum_k coef[e][k] x[k] with
// coef[e][k] = sum of u_i[a] u_j[c] over the pairs (a, c) of class k (e = (b, i, j), i <= j):
// 20 terms per entry instead of forming the 27 x 27 matrix A and projecting it.
//
// The 4 x 4 and 3 x 3 blocks are solved side by side on the two 16-lane halves of the warp
// (lane (r, c) of a half holds entry (r, c)): M = (B + delta I)^-1 from an LDL^T factorisation
// (delta = 1e-13 tr B keeps the factorisation positive definite without moving eigenvectors),
// then seven squarings M <- M^2, scaled by a power of two, so M^128 is dominated by the
// eigenvector of the smallest eigenvalue (inverse iteration with exponent 128). Its Rayleigh
// quotient and residual are taken with B; a block whose residual fails the check is solved
// again by block_min_eig. The next eigenvalue of the block (for the degeneracy flag) comes from
// three squarings of M deflated by the found pair. The 2 x 2 blocks use the closed form.
__constant__ double c_coef3[24][kMaxCls];

struct Eig3Warp {
  double g[2 * kMaxCls];
  double Gb[6][16];
  double B[6][16];
  double M[2][16];
  double v[6][4];    // eigenvector (block coordinates) of each block's smallest eigenvalue
  double lam[6][2];  // each block's smallest and next eigenvalue
  double tr[6];      // each block's trace (bound of its largest eigenvalue)
  int conv[2];
};

// 2^-2e for the exponent e of x: squares of entries scaled by the square of the trace's scale.
__device__ __forceinline__ double pow2_inv_exp_sq(double x) {
  const double p = pow2_inv_exp(x);
  return p * p;
}

// Scaled squaring of the symmetric 4 x 4 matrix M of a 16-lane half; lane (r, c) gets the new
// entry (r, c). Reads before the caller's __syncwarp, writes after it.
__device__ __forceinline__ double sq_entry(const double* M, int r, int c) {
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) s = fma(M[r * 4 + k], M[k * 4 + c], s);
  return s * pow2_inv_exp_sq(M[0] + M[5] + M[10] + M[15]);
}

// Dominant column of the matrix of a half after the squarings, normalised.
__device__ __forceinline__ void dominant_column(const double* M, double v[4]) {
  int jm = 0;
#pragma unroll
  for (int j = 1; j < 4; ++j)
    if (M[j * 5] > M[jm * 5]) jm = j;
  double n2 = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = M[k * 4 + jm];
    n2 = fma(v[k], v[k], n2);
  }
  const double inv = n2 > 0.0 ? rsqrt(n2) : 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] *= inv;
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_eig3d(const double* __restrict__ gvals,
                                                      int64_t cap,
                                                      const int32_t* __restrict__ count,
                                                      double* __restrict__ alpha_out,
                                                      double* __restrict__ c_out,
                                                      double* __restrict__ lam_out,
                                                      int32_t* __restrict__ flags_out,
                                                      const int32_t* __restrict__ shift_m,
                                                      double* __restrict__ ap_out) {
  constexpr int MU = 27, NCLS = 10, NENT = 24, CENTRE = 13;
  __shared__ double s_coef[NENT][NCLS];
  __shared__ double s_u[kMaxSymVec][MU];
  __shared__ int8_t s_ent[NENT][3];
  __shared__ Eig3Warp sw[WARPS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < NENT * NCLS; e += WARPS * 32)
    s_coef[e / NCLS][e % NCLS] = c_coef3[e / NCLS][e % NCLS];
  for (int e = threadIdx.x; e < kMaxSymVec * MU; e += WARPS * 32)
    s_u[e / MU][e % MU] = c_sym.u[e / MU][e % MU];
  for (int e = threadIdx.x; e < NENT * 3; e += WARPS * 32) s_ent[e / 3][e % 3] = c_ent[e / 3][e % 3];
  __syncthreads();
  Eig3Warp& sm = sw[w];
  const int64_t cnt = *count;
  const int h = lane >> 4, q = lane & 15, r = q >> 2, cc = q & 3;  // half h solves block h
  for (int64_t i = (int64_t)blockIdx.x * WARPS + w; i < cnt; i += (int64_t)gridDim.x * WARPS) {
    if (lane < 2 * NCLS) sm.g[lane] = gvals[(int64_t)lane * cap + i];
    for (int e = lane; e < 6 * 16; e += 32) {
      (&sm.Gb[0][0])[e] = 0.0;
      (&sm.B[0][0])[e] = 0.0;
    }
    __syncwarp();
    // ---- a4: G_b and U_b^T A1 U_b entries, then B_b = U_b^T A1 U_b - G_b G_b ----
    int eb = 0, ei = 0, ej = 0;
    double a1 = 0.0;
    if (lane < NENT) {
      eb = s_ent[lane][0];
      ei = s_ent[lane][1];
      ej = s_ent[lane][2];
      double gg = 0.0;
#pragma unroll
      for (int k = 0; k < NCLS; ++k) {
        gg = fma(s_coef[lane][k], sm.g[2 * k], gg);
        a1 = fma(s_coef[lane][k], sm.g[2 * k + 1], a1);
      }
      sm.Gb[eb][ei * 4 + ej] = gg;
      sm.Gb[eb][ej * 4 + ei] = gg;
    }
    __syncwarp();
    if (lane < NENT) {
      double s = a1;
#pragma unroll
      for (int k = 0; k < 4; ++k) s = fma(-sm.Gb[eb][ei * 4 + k], sm.Gb[eb][k * 4 + ej], s);
      sm.B[eb][ei * 4 + ej] = s;
      sm.B[eb][ej * 4 + ei] = s;
    }
    __syncwarp();
    // ---- a5 for blocks 0 and 1 (one per half) ----
    double b[4][4], scale = 0.0, tr = 0.0;
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        b[x][y] = sm.B[h][x * 4 + y];
        scale = fmax(scale, fabs(b[x][y]));
      }
#pragma unroll
    for (int x = 0; x < 4; ++x) tr += b[x][x];
    if (h == 1) b[3][3] = 4.0 * scale + 1.0;  // decoupled pad above every eigenvalue of the 3 x 3
    double s4[4][4], L[4][4], id[4];
    const double delta = 1e-13 * fabs(tr);
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        s4[x][y] = b[x][y] + (x == y ? delta : 0.0);
        L[x][y] = 0.0;
      }
    const bool fact = ldlt(s4, 4, L, id);
    // entry (r, cc) of M0 = (B + delta I)^-1: column cc by forward and back substitution
    double xv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) xv[k] = k == cc ? 1.0 : 0.0;
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int k = 0; k < x; ++k) xv[x] = fma(-L[x][k], xv[k], xv[x]);
#pragma unroll
    for (int x = 0; x < 4; ++x) xv[x] *= id[x];
#pragma unroll
    for (int x = 3; x >= 0; --x)
#pragma unroll
      for (int k = x + 1; k < 4; ++k) xv[x] = fma(-L[k][x], xv[k], xv[x]);
    double m0 = xv[0];
#pragma unroll
    for (int k = 1; k < 4; ++k)
      if (r == k) m0 = xv[k];
    if (!fact) m0 = r == cc ? 1.0 : 0.0;
    sm.M[h][q] = m0;
    __syncwarp();
#pragma unroll 1
    for (int k = 0; k < 7; ++k) {
      const double nv = sq_entry(sm.M[h], r, cc);
      __syncwarp();
      sm.M[h][q] = nv;
      __syncwarp();
    }
    double v1[4];
    dominant_column(sm.M[h], v1);
    if (h == 1) v1[3] = 0.0;
    double lam = 0.0, res = 0.0, bv[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      bv[x] = 0.0;
#pragma unroll
      for (int y = 0; y < 4; ++y) bv[x] = fma(b[x][y], v1[y], bv[x]);
      lam = fma(v1[x], bv[x], lam);
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) res = fmax(res, fabs(fma(-lam, v1[x], bv[x])));
    const int conv = fact && isfinite(lam) && res <= 64.0 * DBL_EPSILON * scale;
    // next eigenvalue of the block: M0 deflated by (v1, mu1), three squarings, Rayleigh quotient
    double part = v1[r] * m0 * v1[cc];
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    __syncwarp();
    sm.M[h][q] = fma(-part * v1[r], v1[cc], m0);
    __syncwarp();
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
      const double nv = sq_entry(sm.M[h], r, cc);
      __syncwarp();
      sm.M[h][q] = nv;
      __syncwarp();
    }
    double v2[4];
    dominant_column(sm.M[h], v2);
    double lam2b = 0.0;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      double t = 0.0;
#pragma unroll
      for (int y = 0; y < 4; ++y) t = fma(b[x][y], v2[y], t);
      lam2b = fma(v2[x], t, lam2b);
    }
    if (!(v2[0] != 0.0 || v2[1] != 0.0 || v2[2] != 0.0 || v2[3] != 0.0)) lam2b = lam;
    if (q == 0) {
      sm.lam[h][0] = lam;
      sm.lam[h][1] = lam2b;
      sm.tr[h] = tr;
      sm.conv[h] = conv;
#pragma unroll
      for (int x = 0; x < 4; ++x) sm.v[h][x] = v1[x];
    }
    // ---- the 2 x 2 (Eg, T2g) and 1 x 1 (T2u, A2u) blocks ----
    if (lane < 4) {
      const int bb = 2 + lane;
      const double a00 = sm.B[bb][0], a01 = sm.B[bb][1], a11 = sm.B[bb][5];
      double lo, hi, y0 = 1.0, y1 = 0.0;
      if (bb < 4) {
        const double mm = 0.5 * (a00 + a11), hh = 0.5 * (a00 - a11);
        const double rr = sqrt(fma(hh, hh, a01 * a01));
        hi = mm + rr;
        lo = hi != 0.0 ? (a00 * a11 - a01 * a01) / hi : mm - rr;
        double pp = a01, qq = lo - a00;
        if (fabs(a00 - lo) < fabs(a11 - lo)) {
          pp = lo - a11;
          qq = a01;
        }
        double nr = sqrt(pp * pp + qq * qq);
        if (nr == 0.0) {
          pp = 1.0;
          qq = 0.0;
          nr = 1.0;
        }
        y0 = pp / nr;
        y1 = qq / nr;
        sm.tr[bb] = a00 + a11;
      } else {
        lo = a00;
        hi = DBL_MAX;
        sm.tr[bb] = a00;
      }
      sm.lam[bb][0] = lo;
      sm.lam[bb][1] = hi;
      sm.v[bb][0] = y0;
      sm.v[bb][1] = y1;
      sm.v[bb][2] = 0.0;
      sm.v[bb][3] = 0.0;
    }
    __syncwarp();
    // ---- fallback for a 4 x 4 or 3 x 3 block whose residual check failed ----
    if (lane < 2 && !sm.conv[lane]) {
      const int dim = lane == 0 ? 4 : 3;
      double a[4][4], y[4], lmin, l2;
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int z = 0; z < 4; ++z) a[x][z] = sm.B[lane][x * 4 + z];
      sm.conv[lane] = block_min_eig(a, dim, y, &lmin, &l2) ? 2 : 0;
      sm.lam[lane][0] = lmin;
      sm.lam[lane][1] = l2;
#pragma unroll
      for (int x = 0; x < 4; ++x) sm.v[lane][x] = y[x];
    }
    __syncwarp();
    // ---- selection (every lane, uniform) ----
    int bstar = 0;
#pragma unroll
    for (int bb = 1; bb < 6; ++bb)
      if (sm.lam[bb][0] < sm.lam[bstar][0]) bstar = bb;
    const double lam1 = sm.lam[bstar][0];
    double lam2 = DBL_MAX, lmax = 0.0;
#pragma unroll
    for (int bb = 0; bb < 6; ++bb) {
      lmax = fmax(lmax, fabs(sm.tr[bb]));
      if (bb == bstar) {
        lam2 = fmin(lam2, sm.lam[bb][1]);
        if (c_sym.copies[bb] > 1) lam2 = fmin(lam2, sm.lam[bb][0]);
      } else {
        lam2 = fmin(lam2, sm.lam[bb][0]);
      }
    }
    int flags = 0;
    if (!sm.conv[0] || !sm.conv[1]) flags |= LSP_FLAG_NOT_CONVERGED;
    if (bstar != 0) flags |= LSP_FLAG_NONSYMMETRIC;
    if (lam2 - lam1 < 1e-8 * lmax) flags |= LSP_FLAG_DEGENERATE;
    // ---- alpha = U_b y and (a6) c = G alpha = U_b (G_b y) ----
    const int first = c_sym.first[bstar];
    double y[4], gy[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) y[x] = sm.v[bstar][x];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      gy[x] = 0.0;
#pragma unroll
      for (int z = 0; z < 4; ++z) gy[x] = fma(sm.Gb[bstar][x * 4 + z], y[z], gy[x]);
    }
    double av = 0.0, cv = 0.0;
    if (lane < MU) {
      const int dimb = c_sym.dim[bstar];
#pragma unroll
      for (int x = 0; x < 4; ++x)
        if (x < dimb) {
          av = fma(y[x], s_u[first + x][lane], av);
          cv = fma(gy[x], s_u[first + x][lane], cv);
        }
    }
    // sign: alpha[centre] > 0, else the first entry above 1e-12 in magnitude
    const double acen = __shfl_sync(0xffffffffu, av, CENTRE);
    const unsigned big = __ballot_sync(0xffffffffu, lane < MU && fabs(av) > 1e-12);
    const double afirst = __shfl_sync(0xffffffffu, av, big ? __ffs(big) - 1 : 0);
    const double ref = fabs(acen) > 1e-12 ? acen : (big ? afirst : 0.0);
    if (ref < 0.0) {
      av = -av;
      cv = -cv;
    }
    if (lane < MU) {
      alpha_out[i * MU + lane] = av;
      c_out[i * MU + lane] = cv;
      ap_out[i * MU + lane] = fma(-cv, lattice_shift(__ldg(shift_m + i)), av);
    }
    if (lane == 0) {
      lam_out[2 * i + 0] = lam1;
      lam_out[2 * i + 1] = lam2;
      flags_out[i] = flags;
    }
    __syncwarp();
  }
}

// ---- 2D, t = 2: one warp per shift, blocks of mu_0^2 formed from the class values ----------
// mu_0^2 is the 5 x 5 neighbourhood; its symmetry blocks (host-built basis, see build_sym_t2)
// are A1 (6 x 6), E (6 x 6, two partners), B1 (3 x 3), B2 (3 x 3) and A2 (1 x 1). As in 3D,
// G maps every block's span into itself, so B_b = U_b^T A1 U_b - G_b G_b with both terms linear
// in the 15 class values through one coefficient table (55 entries). The 6 x 6 blocks are
// solved one after the other on the whole warp as 8 x 8 matrices (two entries per lane, the
// padding decoupled on the diagonal above the block's spectrum): LDL^T of B + delta I column by
// column, the inverse by lanes 0-7 (one column each), seven scaled squarings, Rayleigh quotient
// and residual; the next eigenvalue from three squarings of the deflated inverse. The 3 x 3
// blocks run side by side on the two half-warps (4 x 4 padded, as in 3D); A2 is 1 x 1.
constexpr int kT2Ent = 55;
__constant__ double c_coef2[kT2Ent][kMaxCls];
__constant__ int8_t c_ent2[kT2Ent][3];
__constant__ SymBasis c_sym2;

struct EigT2Warp {
  double g[2 * 15];
  double Gb[5][64];   // 8 x 8 padded blocks (row stride 8)
  double B[5][64];
  double L[64], dd[8], dinv[8];
  double M[64], M0[64];
  double M4[2][16];   // the two half-warps' 4 x 4 matrices
  double v[5][8];     // eigenvector (block coordinates) of each block's smallest eigenvalue
  double lam[5][2];
  double tr[5];
  int conv[5];
};

// Smallest eigenpair (and next eigenvalue) of the block b (dim <= 6) held in sm.B[b], on the
// whole warp. Writes sm.v[b], sm.lam[b], sm.tr[b], sm.conv[b].
__device__ void warp_block_eig8(EigT2Warp& sm, int b, int dim, int lane) {
  const double* Bb = sm.B[b];
  const int r0 = lane >> 3, r1 = r0 + 4, cc = lane & 7;
  // scale and trace of the block
  double sc = fmax(fabs(Bb[r0 * 8 + cc]), fabs(Bb[r1 * 8 + cc]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sc = fmax(sc, __shfl_xor_sync(0xffffffffu, sc, o));
  double tr = 0.0;
  for (int k = 0; k < dim; ++k) tr += Bb[k * 9];
  const double pad = 4.0 * sc * dim + 1.0;  // above every eigenvalue of the block
  const double delta = 1e-13 * fabs(tr);
  // S = B + delta I with the padding, into M (lane-parallel)
  auto S_at = [&](int r, int c) {
    const double x = (r < dim && c < dim) ? Bb[r * 8 + c] : (r == c ? pad : 0.0);
    return r == c ? x + delta : x;
  };
  sm.M[r0 * 8 + cc] = S_at(r0, cc);
  sm.M[r1 * 8 + cc] = S_at(r1, cc);
  __syncwarp();
  // LDL^T, one column at a time; lane i (j < i < 8) forms L[i][j]
  bool fact = true;
  for (int j = 0; j < 8; ++j) {
    double dj = sm.M[j * 9];
    for (int k = 0; k < j; ++k) dj -= sm.L[j * 8 + k] * sm.L[j * 8 + k] * sm.dd[k];
    if (!(dj > 0.0)) fact = false;
    const double idj = 1.0 / dj;
    if (lane > j && lane < 8) {
      double a = sm.M[lane * 8 + j];
      for (int k = 0; k < j; ++k) a -= sm.L[lane * 8 + k] * sm.L[j * 8 + k] * sm.dd[k];
      sm.L[lane * 8 + j] = a * idj;
    }
    if (lane == 0) {
      sm.dd[j] = dj;
      sm.dinv[j] = idj;
    }
    __syncwarp();
  }
  // M0 = (L D L^T)^-1: lane c < 8 forms column c
  if (lane < 8) {
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = k == lane ? 1.0 : 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int k = 0; k < i; ++k) x[i] = fma(-sm.L[i * 8 + k], x[k], x[i]);
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] *= sm.dinv[i];
#pragma unroll
    for (int i = 7; i >= 0; --i)
#pragma unroll
      for (int k = i + 1; k < 8; ++k) x[i] = fma(-sm.L[k * 8 + i], x[k], x[i]);
#pragma unroll
    for (int i = 0; i < 8; ++i) sm.M0[i * 8 + lane] = fact ? x[i] : (i == lane ? 1.0 : 0.0);
  }
  __syncwarp();
  const double m00 = sm.M0[r0 * 8 + cc], m01 = sm.M0[r1 * 8 + cc];
  sm.M[r0 * 8 + cc] = m00;
  sm.M[r1 * 8 + cc] = m01;
  __syncwarp();
  auto square = [&](int rounds) {
    for (int k = 0; k < rounds; ++k) {
      double s0 = 0.0, s1 = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        s0 = fma(sm.M[r0 * 8 + q], sm.M[q * 8 + cc], s0);
        s1 = fma(sm.M[r1 * 8 + q], sm.M[q * 8 + cc], s1);
      }
      double t8 = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) t8 += sm.M[q * 9];
      const double p2 = pow2_inv_exp_sq(t8);
      __syncwarp();
      sm.M[r0 * 8 + cc] = s0 * p2;
      sm.M[r1 * 8 + cc] = s1 * p2;
      __syncwarp();
    }
  };
  auto dominant = [&](double (&vv)[8]) {
    int jm = 0;
    for (int q = 1; q < 8; ++q)
      if (sm.M[q * 9] > sm.M[jm * 9]) jm = q;
    double n2 = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      vv[q] = q < dim ? sm.M[q * 8 + jm] : 0.0;
      n2 = fma(vv[q], vv[q], n2);
    }
    const double inv = n2 > 0.0 ? rsqrt(n2) : 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) vv[q] *= inv;
  };
  // Rayleigh quotient v^T B v and residual max |B v - lambda v| (lanes 0-7 form one row each)
  auto rayleigh = [&](const double (&vv)[8], double* res) {
    double row = 0.0;
    if (lane < dim)
      for (int q = 0; q < dim; ++q) row = fma(Bb[lane * 8 + q], vv[q], row);
    double bv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) bv[q] = __shfl_sync(0xffffffffu, row, q);
    double lam = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) lam = fma(vv[q], bv[q], lam);
    double rr = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < dim) rr = fmax(rr, fabs(fma(-lam, vv[q], bv[q])));
    *res = rr;
    return lam;
  };
  square(7);
  double v1[8], res1;
  dominant(v1);
  const double lam1 = rayleigh(v1, &res1);
  const int conv = fact && isfinite(lam1) && res1 <= 64.0 * DBL_EPSILON * sc;
  // next eigenvalue: M0 deflated by (v1, mu1), three squarings
  double part = v1[r0] * m00 * v1[cc] + v1[r1] * m01 * v1[cc];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  __syncwarp();
  sm.M[r0 * 8 + cc] = fma(-part * v1[r0], v1[cc], m00);
  sm.M[r1 * 8 + cc] = fma(-part * v1[r1], v1[cc], m01);
  __syncwarp();
  square(3);
  double v2[8], res2;
  dominant(v2);
  double lam2 = dim > 1 ? rayleigh(v2, &res2) : DBL_MAX;
  if (dim > 1 && !(v2[0] != 0.0 || v2[1] != 0.0 || v2[2] != 0.0 || v2[3] != 0.0 ||
                   v2[4] != 0.0 || v2[5] != 0.0))
    lam2 = lam1;
  if (lane == 0) {
    sm.lam[b][0] = lam1;
    sm.lam[b][1] = lam2;
    sm.tr[b] = tr;
    sm.conv[b] = conv;
#pragma unroll
    for (int q = 0; q < 8; ++q) sm.v[b][q] = v1[q];
  }
  __syncwarp();
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_eig2d_t2(const double* __restrict__ gvals,
                                                         int64_t cap,
                                                         const int32_t* __restrict__ count,
                                                         double* __restrict__ alpha_out,
                                                         double* __restrict__ c_out,
                                                         double* __restrict__ lam_out,
                                                         int32_t* __restrict__ flags_out) {
  constexpr int MU = 25, NCLS = 15, CENTRE = 12;
  __shared__ double s_coef[kT2Ent][NCLS];
  __shared__ double s_u[kMaxSymVec][MU];
  __shared__ int8_t s_ent[kT2Ent][3];
  __shared__ EigT2Warp sw[WARPS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < kT2Ent * NCLS; e += WARPS * 32)
    s_coef[e / NCLS][e % NCLS] = c_coef2[e / NCLS][e % NCLS];
  for (int e = threadIdx.x; e < kMaxSymVec * MU; e += WARPS * 32)
    s_u[e / MU][e % MU] = c_sym2.u[e / MU][e % MU];
  for (int e = threadIdx.x; e < kT2Ent * 3; e += WARPS * 32) s_ent[e / 3][e % 3] = c_ent2[e / 3][e % 3];
  __syncthreads();
  EigT2Warp& sm = sw[w];
  const int64_t cnt = *count;
  const int h = lane >> 4, q = lane & 15, r = q >> 2, cc = q & 3;
  for (int64_t i = (int64_t)blockIdx.x * WARPS + w; i < cnt; i += (int64_t)gridDim.x * WARPS) {
    if (lane < 2 * NCLS) sm.g[lane] = gvals[(int64_t)lane * cap + i];
    for (int e = lane; e < 5 * 64; e += 32) {
      (&sm.Gb[0][0])[e] = 0.0;
      (&sm.B[0][0])[e] = 0.0;
    }
    __syncwarp();
    // ---- a4: G_b and U_b^T A1 U_b, then B_b = U_b^T A1 U_b - G_b G_b (entries e, e + 32) ----
    double a1v[2] = {0.0, 0.0};
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
      const int e = lane + 32 * pass;
      if (e < kT2Ent) {
        const int eb = s_ent[e][0], ei = s_ent[e][1], ej = s_ent[e][2];
        double gg = 0.0, aa = 0.0;
#pragma unroll
        for (int k = 0; k < NCLS; ++k) {
          gg = fma(s_coef[e][k], sm.g[2 * k], gg);
          aa = fma(s_coef[e][k], sm.g[2 * k + 1], aa);
        }
        sm.Gb[eb][ei * 8 + ej] = gg;
        sm.Gb[eb][ej * 8 + ei] = gg;
        a1v[pass] = aa;
      }
    }
    __syncwarp();
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
      const int e = lane + 32 * pass;
      if (e < kT2Ent) {
        const int eb = s_ent[e][0], ei = s_ent[e][1], ej = s_ent[e][2];
        double sv = a1v[pass];
#pragma unroll
        for (int k = 0; k < 8; ++k) sv = fma(-sm.Gb[eb][ei * 8 + k], sm.Gb[eb][k * 8 + ej], sv);
        sm.B[eb][ei * 8 + ej] = sv;
        sm.B[eb][ej * 8 + ei] = sv;
      }
    }
    __syncwarp();
    // ---- a5: the two 6 x 6 blocks (A1, E) on the whole warp ----
    warp_block_eig8(sm, 0, 6, lane);
    warp_block_eig8(sm, 1, 6, lane);
    // ---- the 3 x 3 blocks (B1, B2) on the two half-warps, padded to 4 x 4 ----
    {
      const int bb = 2 + h;
      double b4[4][4], scale = 0.0, tr = 0.0;
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          b4[x][y] = (x < 3 && y < 3) ? sm.B[bb][x * 8 + y] : 0.0;
          scale = fmax(scale, fabs(b4[x][y]));
        }
#pragma unroll
      for (int x = 0; x < 3; ++x) tr += b4[x][x];
      b4[3][3] = 4.0 * scale * 3 + 1.0;
      double s4[4][4], L4[4][4], id4[4];
      const double delta = 1e-13 * fabs(tr);
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          s4[x][y] = b4[x][y] + (x == y ? delta : 0.0);
          L4[x][y] = 0.0;
        }
      const bool fact = ldlt(s4, 4, L4, id4);
      double xv[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) xv[k] = k == cc ? 1.0 : 0.0;
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int k = 0; k < x; ++k) xv[x] = fma(-L4[x][k], xv[k], xv[x]);
#pragma unroll
      for (int x = 0; x < 4; ++x) xv[x] *= id4[x];
#pragma unroll
      for (int x = 3; x >= 0; --x)
#pragma unroll
        for (int k = x + 1; k < 4; ++k) xv[x] = fma(-L4[k][x], xv[k], xv[x]);
      double m0 = xv[0];
#pragma unroll
      for (int k = 1; k < 4; ++k)
        if (r == k) m0 = xv[k];
      if (!fact) m0 = r == cc ? 1.0 : 0.0;
      sm.M4[h][q] = m0;
      __syncwarp();
#pragma unroll 1
      for (int k = 0; k < 7; ++k) {
        const double nv = sq_entry(sm.M4[h], r, cc);
        __syncwarp();
        sm.M4[h][q] = nv;
        __syncwarp();
      }
      double v1[4];
      dominant_column(sm.M4[h], v1);
      v1[3] = 0.0;
      double lam = 0.0, res = 0.0, bv[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        bv[x] = 0.0;
#pragma unroll
        for (int y = 0; y < 4; ++y) bv[x] = fma(b4[x][y], v1[y], bv[x]);
        lam = fma(v1[x], bv[x], lam);
      }
#pragma unroll
      for (int x = 0; x < 4; ++x) res = fmax(res, fabs(fma(-lam, v1[x], bv[x])));
      const int conv = fact && isfinite(lam) && res <= 64.0 * DBL_EPSILON * scale;
      double part = v1[r] * m0 * v1[cc];
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      __syncwarp();
      sm.M4[h][q] = fma(-part * v1[r], v1[cc], m0);
      __syncwarp();
#pragma unroll 1
      for (int k = 0; k < 3; ++k) {
        const double nv = sq_entry(sm.M4[h], r, cc);
        __syncwarp();
        sm.M4[h][q] = nv;
        __syncwarp();
      }
      double v2[4];
      dominant_column(sm.M4[h], v2);
      double lam2b = 0.0;
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        double t = 0.0;
#pragma unroll
        for (int y = 0; y < 4; ++y) t = fma(b4[x][y], v2[y], t);
        lam2b = fma(v2[x], t, lam2b);
      }
      if (!(v2[0] != 0.0 || v2[1] != 0.0 || v2[2] != 0.0)) lam2b = lam;
      if (q == 0) {
        sm.lam[bb][0] = lam;
        sm.lam[bb][1] = lam2b;
        sm.tr[bb] = tr;
        sm.conv[bb] = conv;
#pragma unroll
        for (int x = 0; x < 8; ++x) sm.v[bb][x] = x < 4 ? v1[x] : 0.0;
      }
    }
    // ---- A2 (1 x 1) ----
    if (lane == 0) {
      sm.lam[4][0] = sm.B[4][0];
      sm.lam[4][1] = DBL_MAX;
      sm.tr[4] = sm.B[4][0];
      sm.conv[4] = 1;
#pragma unroll
      for (int x = 0; x < 8; ++x) sm.v[4][x] = x == 0 ? 1.0 : 0.0;
    }
    __syncwarp();
    // ---- fallback: cyclic Jacobi for a block whose residual check failed (one lane each) ----
    if (lane < 4 && !sm.conv[lane]) {
      const int dim = lane < 2 ? 6 : 3;
      double a[8][8], vv[8][8];
      for (int x = 0; x < 8; ++x)
        for (int y = 0; y < 8; ++y) a[x][y] = (x < dim && y < dim) ? sm.B[lane][x * 8 + y] : 0.0;
      const int ok = jacobi_nm<8>(a, vv, dim);
      int kk = 0;
      for (int x = 1; x < dim; ++x)
        if (a[x][x] < a[kk][kk]) kk = x;
      double second = DBL_MAX;
      for (int x = 0; x < dim; ++x)
        if (x != kk) second = fmin(second, a[x][x]);
      sm.lam[lane][0] = a[kk][kk];
      sm.lam[lane][1] = second;
      for (int x = 0; x < 8; ++x) sm.v[lane][x] = x < dim ? vv[x][kk] : 0.0;
      sm.conv[lane] = ok ? 2 : 0;
    }
    __syncwarp();
    // ---- selection (uniform) ----
    int bstar = 0;
#pragma unroll
    for (int bb = 1; bb < 5; ++bb)
      if (sm.lam[bb][0] < sm.lam[bstar][0]) bstar = bb;
    const double lam1 = sm.lam[bstar][0];
    double lam2 = DBL_MAX, lmax = 0.0;
    int flags = 0;
#pragma unroll
    for (int bb = 0; bb < 5; ++bb) {
      lmax = fmax(lmax, fabs(sm.tr[bb]));
      if (!sm.conv[bb]) flags |= LSP_FLAG_NOT_CONVERGED;
      if (bb == bstar) {
        lam2 = fmin(lam2, sm.lam[bb][1]);
        if (c_sym2.copies[bb] > 1) lam2 = fmin(lam2, sm.lam[bb][0]);
      } else {
        lam2 = fmin(lam2, sm.lam[bb][0]);
      }
    }
    if (bstar != 0) flags |= LSP_FLAG_NONSYMMETRIC;
    if (lam2 - lam1 < 1e-8 * lmax) flags |= LSP_FLAG_DEGENERATE;
    // ---- alpha = U_b y and (a6) c = G alpha = U_b (G_b y) ----
    const int first = c_sym2.first[bstar], dimb = c_sym2.dim[bstar];
    double y[8], gy[8];
#pragma unroll
    for (int x = 0; x < 8; ++x) y[x] = sm.v[bstar][x];
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      gy[x] = 0.0;
#pragma unroll
      for (int z = 0; z < 8; ++z) gy[x] = fma(sm.Gb[bstar][x * 8 + z], y[z], gy[x]);
    }
    double av = 0.0, cv = 0.0;
    if (lane < MU) {
#pragma unroll
      for (int x = 0; x < 8; ++x)
        if (x < dimb) {
          av = fma(y[x], s_u[first + x][lane], av);
          cv = fma(gy[x], s_u[first + x][lane], cv);
        }
    }
    const double acen = __shfl_sync(0xffffffffu, av, CENTRE);
    const unsigned big = __ballot_sync(0xffffffffu, lane < MU && fabs(av) > 1e-12);
    const double afirst = __shfl_sync(0xffffffffu, av, big ? __ffs(big) - 1 : 0);
    const double ref = fabs(acen) > 1e-12 ? acen : (big ? afirst : 0.0);
    if (ref < 0.0) {
      av = -av;
      cv = -cv;
    }
    if (lane < MU) {
      alpha_out[i * MU + lane] = av;
      c_out[i * MU + lane] = cv;
    }
    if (lane == 0) {
      lam_out[2 * i + 0] = lam1;
      lam_out[2 * i + 1] = lam2;
      flags_out[i] = flags;
    }
    __syncwarp();
  }
}

// ---- 2D, one thread per shift ------------------------------------------------------------
// In 2D the symmetry-adapted vectors are u_0..u_2 (fully symmetric: centre, edges, corners),
// u_3 (edges, x^2 - y^2), u_4 (corners, xy) and u_5, u_6 (x-odd on edges and corners). With
// W_i = G_s[mu, mu] u_i (linear in g) and the A1 part u_i^T A1 u_j (linear in g * g), every
// block entry is  B_ij = u_i^T A1 u_j - W_i . W_j, so the 9 x 9 matrix A is never formed.
__constant__ double c_W2[7][9][6];   // W_i[k] = sum_c c_W2[i][k][c] g[c]
__constant__ double c_B2[7][7][6];   // u_i^T A1 u_j = sum_c c_B2[i][j][c] (g*g)[c]
__constant__ float c_W2f[7][9][6];   // the same tables in FP32 (mixed mode)
__constant__ float c_B2f[7][7][6];

template <typename GT>
__device__ __forceinline__ GT coefW(int i, int k, int c);
template <>
__device__ __forceinline__ double coefW<double>(int i, int k, int c) { return c_W2[i][k][c]; }
template <>
__device__ __forceinline__ float coefW<float>(int i, int k, int c) { return c_W2f[i][k][c]; }
template <typename GT>
__device__ __forceinline__ GT coefB(int i, int j, int c);
template <>
__device__ __forceinline__ double coefB<double>(int i, int j, int c) { return c_B2[i][j][c]; }
template <>
__device__ __forceinline__ float coefB<float>(int i, int j, int c) { return c_B2f[i][j][c]; }

// GT is the arithmetic of the Gram assembly: double (FP64 mode) or float (mixed mode).
template <int I, typename GT>
__device__ __forceinline__ void w_vec(const GT (&g)[6], GT (&w)[9]) {
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    GT s = GT(0);
#pragma unroll
    for (int c = 0; c < 6; ++c) s = fma(coefW<GT>(I, k, c), g[c], s);
    w[k] = s;
  }
}
template <int I, int J, typename GT>
__device__ __forceinline__ GT b_entry(const GT (&g2)[6], const GT (&wi)[9], const GT (&wj)[9]) {
  GT s = GT(0);
#pragma unroll
  for (int c = 0; c < 6; ++c) s = fma(coefB<GT>(I, J, c), g2[c], s);
  GT t = GT(0);
#pragma unroll
  for (int k = 0; k < 9; ++k) t = fma(wi[k], wj[k], t);
  return s - t;
}

// 2^-ilogb(x) for x > 0: the power of two that scales x into [1, 2). For a normal x whose
// reciprocal power is normal (biased exponent field ef in 1..2045) it is built from the
// exponent field with integer operations, 2^(1023 - ef + 1023) as a bit pattern, which keeps
// the FP64 pipe (narrow on this GPU) free; other x take the library functions.
__device__ __forceinline__ double pow2_neg_ilogb(double x) {
  const int ef = (int)((__double_as_longlong(x) >> 52) & 0x7FF);
  if (ef >= 1 && ef <= 2045) return __longlong_as_double((long long)(2046 - ef) << 52);
  return exp2((double)(-ilogb(x)));
}

// Eigenvalues of the symmetric 2 x 2 [[a, b], [b, c]], smaller one first; the small one as
// det / large avoids cancellation.
__device__ __forceinline__ void eig2(double a, double b, double c, double& lo, double& hi) {
  const double m = 0.5 * (a + c), h = 0.5 * (a - c);
  const double r = sqrt(fma(h, h, b * b));
  hi = m + r;
  lo = (hi != 0.0) ? (a * c - b * b) / hi : m - r;
  if (lo > hi) {
    const double t = lo;
    lo = hi;
    hi = t;
  }
}

template <typename GT>
__global__ void __launch_bounds__(128) k_eig2d(const double* __restrict__ gvals, int64_t cap,
                                               const int32_t* __restrict__ count,
                                               double* __restrict__ alpha_out,
                                               double* __restrict__ c_out,
                                               double* __restrict__ lam_out,
                                               int32_t* __restrict__ flags_out,
                                               const int32_t* __restrict__ shift_m,
                                               double* __restrict__ ap_out) {
  const int64_t cnt = *count;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x) {
    GT g[6], g2[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      g[c] = (GT)__ldg(gvals + (int64_t)(2 * c) * cap + i);
      g2[c] = (GT)__ldg(gvals + (int64_t)(2 * c + 1) * cap + i);
    }
    // fully symmetric block (3 x 3)
    GT w0[9], w1[9], w2[9];
    w_vec<0>(g, w0);
    w_vec<1>(g, w1);
    w_vec<2>(g, w2);
    double b00 = b_entry<0, 0>(g2, w0, w0), b01 = b_entry<0, 1>(g2, w0, w1),
           b02 = b_entry<0, 2>(g2, w0, w2), b11 = b_entry<1, 1>(g2, w1, w1),
           b12 = b_entry<1, 2>(g2, w1, w2), b22 = b_entry<2, 2>(g2, w2, w2);
    // the other blocks: two 1 x 1 and one 2 x 2 (two copies)
    double e00, e01, e11, bb1, bb2;
    {
      GT u[9], v[9];
      w_vec<3>(g, u);
      bb1 = b_entry<3, 3>(g2, u, u);
      w_vec<4>(g, u);
      bb2 = b_entry<4, 4>(g2, u, u);
      w_vec<5>(g, u);
      w_vec<6>(g, v);
      e00 = b_entry<5, 5>(g2, u, u);
      e01 = b_entry<5, 6>(g2, u, v);
      e11 = b_entry<6, 6>(g2, v, v);
    }
    // smallest eigenpair of the 3 x 3 block: scale to unit max entry, then repeated products
    // with the adjugate (= det * inverse: inverse iteration without divisions), starting from
    // the adjugate column with the largest diagonal entry.
    const double sc = fmax(fmax(fmax(fabs(b00), fabs(b01)), fmax(fabs(b02), fabs(b11))),
                           fmax(fabs(b12), fabs(b22)));
    const double isc = sc > 0 ? 1.0 / sc : 0.0;
    const double s00 = b00 * isc, s01 = b01 * isc, s02 = b02 * isc, s11 = b11 * isc,
                 s12 = b12 * isc, s22 = b22 * isc;
    const double a00 = s11 * s22 - s12 * s12, a01 = s02 * s12 - s01 * s22,
                 a02 = s01 * s12 - s02 * s11, a11 = s00 * s22 - s02 * s02,
                 a12 = s01 * s02 - s00 * s12, a22 = s00 * s11 - s01 * s01;
    double x0, x1, x2;
    if (a00 >= a11 && a00 >= a22) {
      x0 = a00; x1 = a01; x2 = a02;
    } else if (a11 >= a22) {
      x0 = a01; x1 = a11; x2 = a12;
    } else {
      x0 = a02; x1 = a12; x2 = a22;
    }
#pragma unroll
    for (int it = 0; it < 5; ++it) {
      const double y0 = a00 * x0 + a01 * x1 + a02 * x2;
      const double y1 = a01 * x0 + a11 * x1 + a12 * x2;
      const double y2 = a02 * x0 + a12 * x1 + a22 * x2;
      // renormalise by a power of two (exact) to stay clear of under/overflow
      const double mx = fmax(fabs(y0), fmax(fabs(y1), fabs(y2)));
      const double p2 = mx > 0 ? pow2_neg_ilogb(mx) : 1.0;
      x0 = y0 * p2;
      x1 = y1 * p2;
      x2 = y2 * p2;
    }
    const double inrm = rsqrt(x0 * x0 + x1 * x1 + x2 * x2);
    double y[3] = {x0 * inrm, x1 * inrm, x2 * inrm};
    // one Newton correction of the normalisation (rsqrt is approximate)
    {
      const double n2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
      const double f = 1.5 - 0.5 * n2;
      y[0] *= f;
      y[1] *= f;
      y[2] *= f;
    }
    const double r0 = s00 * y[0] + s01 * y[1] + s02 * y[2];
    const double r1 = s01 * y[0] + s11 * y[1] + s12 * y[2];
    const double r2 = s02 * y[0] + s12 * y[1] + s22 * y[2];
    const double ls = y[0] * r0 + y[1] * r1 + y[2] * r2;  // Rayleigh quotient (scaled)
    const double res = fmax(fabs(r0 - ls * y[0]), fmax(fabs(r1 - ls * y[1]), fabs(r2 - ls * y[2])));
    int flags = 0;
    double l1s = ls;
    // remaining eigenvalues of the 3 x 3 block from its trace and principal minors
    const double tr = s00 + s11 + s22, m2 = a00 + a11 + a22;
    double S = tr - l1s, Pp = m2 - l1s * S;
    double disc = fmax(0.25 * S * S - Pp, 0.0);
    double l3s = 0.5 * S + sqrt(disc);
    double l2s = l3s > 0 ? Pp / l3s : 0.0;
    // The adjugate iteration converges to the eigenvalue of smallest magnitude. Accept it when
    // the residual is at rounding level and it is also the algebraically smallest (it can be
    // slightly negative when the block was assembled in FP32); otherwise run cyclic Jacobi.
    if (!(res <= 64 * 2.2e-16) || !(l1s <= l2s)) {
      double a[4][4] = {{s00, s01, s02, 0}, {s01, s11, s12, 0}, {s02, s12, s22, 0}, {0, 0, 0, 0}};
      double vv[4][4];
      if (!jacobi_small(a, vv, 3)) flags |= LSP_FLAG_NOT_CONVERGED;
      int k = 0;
      if (a[1][1] < a[k][k]) k = 1;
      if (a[2][2] < a[k][k]) k = 2;
      l1s = a[k][k];
      y[0] = vv[0][k];
      y[1] = vv[1][k];
      y[2] = vv[2][k];
      S = tr - l1s;
      Pp = m2 - l1s * S;
      disc = fmax(0.25 * S * S - Pp, 0.0);
      l3s = 0.5 * S + sqrt(disc);
      l2s = l3s > 0 ? Pp / l3s : 0.0;
    }
    double lam1 = l1s * sc, lamA2 = l2s * sc, lamA3 = l3s * sc;
    double eLo, eHi;
    eig2(e00, e01, e11, eLo, eHi);
    // winner over the blocks; lambda_2 counts the 2 x 2 block twice (two irrep copies)
    int win = 0;
    double best = lam1;
    if (bb1 < best) { best = bb1; win = 1; }
    if (bb2 < best) { best = bb2; win = 2; }
    if (eLo < best) { best = eLo; win = 3; }
    double lam2;
    if (win == 0)
      lam2 = fmin(fmin(lamA2, bb1), fmin(bb2, eLo));
    else if (win == 3)
      lam2 = eLo;  // second copy of the same eigenvalue
    else
      lam2 = fmin(fmin(lam1, win == 1 ? bb2 : bb1), eLo);
    const double lmax = fmax(fmax(fabs(lamA3), fabs(eHi)), fmax(fabs(bb1), fabs(bb2)));
    if (lam2 - best < 1e-8 * lmax) flags |= LSP_FLAG_DEGENERATE;
    if (win != 0) flags |= LSP_FLAG_NONSYMMETRIC;
    double al[9], cv[9];
    if (win == 0) {
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        al[a] = y[0] * c_sym.u[0][a] + y[1] * c_sym.u[1][a] + y[2] * c_sym.u[2][a];
        cv[a] = y[0] * w0[a] + y[1] * w1[a] + y[2] * w2[a];
      }
    } else if (win == 1 || win == 2) {
      const int vi = win == 1 ? 3 : 4;
      GT u[9];
      if (win == 1) w_vec<3>(g, u); else w_vec<4>(g, u);
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        al[a] = c_sym.u[vi][a];
        cv[a] = u[a];
      }
    } else {
      // eigenvector of the 2 x 2 block for eLo
      double p = e01, q = eLo - e00;
      if (fabs(e00 - eLo) < fabs(e11 - eLo)) {
        p = eLo - e11;
        q = e01;
      }
      double nr = sqrt(p * p + q * q);
      if (nr == 0) { p = 1; q = 0; nr = 1; }
      p /= nr;
      q /= nr;
      GT u[9], v[9];
      w_vec<5>(g, u);
      w_vec<6>(g, v);
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        al[a] = p * c_sym.u[5][a] + q * c_sym.u[6][a];
        cv[a] = p * u[a] + q * v[a];
      }
    }
    // sign: alpha[centre] > 0, else the first entry above 1e-12 in magnitude
    double ref = al[4];
    if (!(fabs(ref) > 1e-12)) {
      ref = 0.0;
#pragma unroll
      for (int a = 0; a < 9; ++a)
        if (ref == 0.0 && fabs(al[a]) > 1e-12) ref = al[a];
    }
    const double sg = ref < 0 ? -1.0 : 1.0;
    const double si = lattice_shift(__ldg(shift_m + i));
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const double aa = sg * al[a], ca = sg * cv[a];
      alpha_out[i * 9 + a] = aa;
      c_out[i * 9 + a] = ca;
      ap_out[i * 9 + a] = fma(-ca, si, aa);  // P rows are fma(c, v, alpha - c s_i)
    }
    lam_out[2 * i + 0] = best;
    lam_out[2 * i + 1] = lam2;
    flags_out[i] = flags;
  }
}

template <int MU, int NCLS, int WARPS>
cudaError_t launch_eig_t(lsp_ctx* c, const int32_t* count, int64_t cap, int method, int refine) {
  const size_t smem =
      ((sizeof(BlockTables<MU>) + 15) / 16) * 16 + sizeof(WarpSmem<MU>) * WARPS;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_eig<MU, NCLS, WARPS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int64_t b = (cap + WARPS - 1) / WARPS;
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  k_eig<MU, NCLS, WARPS><<<(int)b, WARPS * 32, smem, c->stream>>>(
      (const double*)c->gvals.p, cap, count, method, refine, (double*)c->alpha.p,
      (double*)c->cst.p, (double*)c->lam.p, (int32_t*)c->sflags.p,
      (const int32_t*)c->shift_m.p, (double*)c->ap.p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t upload_sym(lsp_ctx* c) {
  uint8_t cls[kMaxMu][kMaxMu];  // the t = 1 classes (the geometry holds up to 125 offsets)
  for (int a = 0; a < kMaxMu; ++a)
    for (int b = 0; b < kMaxMu; ++b) cls[a][b] = c->geo.cls_of[a][b];
  cudaError_t e = cudaMemcpyToSymbol(c_cls, cls, sizeof cls);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_sym, &c->sym, sizeof(SymBasis));
  if (e != cudaSuccess) return e;
  int8_t ent[64][3];
  int n = 0;
  for (int b = 0; b < c->sym.nblk; ++b)
    for (int i = 0; i < c->sym.dim[b]; ++i)
      for (int j = i; j < c->sym.dim[b]; ++j) {
        ent[n][0] = (int8_t)b;
        ent[n][1] = (int8_t)i;
        ent[n][2] = (int8_t)j;
        ++n;
      }
  e = cudaMemcpyToSymbol(c_ent, ent, sizeof(ent));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_nent, &n, sizeof(int));
  if (e != cudaSuccess) return e;
  if (c->geo.d == 3) {
    // coef[e][k] = sum of u_i[a] u_j[b] over the pairs (a, b) of class k, e = (block, i, j)
    static double coef[24][kMaxCls];
    memset(coef, 0, sizeof coef);
    if (n != 24) return cudaErrorInvalidValue;
    for (int q = 0; q < n; ++q) {
      const int b = ent[q][0], i = ent[q][1], j = ent[q][2];
      const double* ui = c->sym.u[c->sym.first[b] + i];
      const double* uj = c->sym.u[c->sym.first[b] + j];
      for (int a = 0; a < c->geo.mu; ++a)
        for (int bb = 0; bb < c->geo.mu; ++bb) coef[q][c->geo.cls_of[a][bb]] += ui[a] * uj[bb];
    }
    return cudaMemcpyToSymbol(c_coef3, coef, sizeof coef);
  }
  if (c->geo.d != 2) return cudaSuccess;  // the tables below are for the 2D kernels
  // W_i[k] = sum_a G[k, a] u_i[a] = sum_a g[cls(k, a)] u_i[a];  u_i^T A1 u_j = sum g2[cls(a,b)] u_i[a] u_j[b]
  static double W2[7][9][6], B2[7][7][6];
  memset(W2, 0, sizeof W2);
  memset(B2, 0, sizeof B2);
  for (int i = 0; i < 7; ++i)
    for (int k = 0; k < 9; ++k)
      for (int a = 0; a < 9; ++a) W2[i][k][c->geo.cls_of[k][a]] += c->sym.u[i][a];
  for (int i = 0; i < 7; ++i)
    for (int j = 0; j < 7; ++j)
      for (int a = 0; a < 9; ++a)
        for (int b = 0; b < 9; ++b)
          B2[i][j][c->geo.cls_of[a][b]] += c->sym.u[i][a] * c->sym.u[j][b];
  static float W2f[7][9][6], B2f[7][7][6];
  for (int i = 0; i < 7; ++i)
    for (int k = 0; k < 9; ++k)
      for (int q = 0; q < 6; ++q) W2f[i][k][q] = (float)W2[i][k][q];
  for (int i = 0; i < 7; ++i)
    for (int j = 0; j < 7; ++j)
      for (int q = 0; q < 6; ++q) B2f[i][j][q] = (float)B2[i][j][q];
  e = cudaMemcpyToSymbol(c_W2, W2, sizeof W2);
  if (e != cudaSuccess) return e;
  {
    // t = 2 (2D): block entries (b, i <= j) of mu_0^2 and their class coefficients
    const SymBasis& s2 = c->sym2;
    const Geometry& g2 = c->geo2;
    static double coef2[kT2Ent][kMaxCls];
    int8_t ent2[kT2Ent][3];
    memset(coef2, 0, sizeof coef2);
    int q = 0;
    for (int b = 0; b < s2.nblk; ++b)
      for (int i = 0; i < s2.dim[b]; ++i)
        for (int j = i; j < s2.dim[b]; ++j) {
          if (q >= kT2Ent) return cudaErrorInvalidValue;
          ent2[q][0] = (int8_t)b;
          ent2[q][1] = (int8_t)i;
          ent2[q][2] = (int8_t)j;
          const double* ui = s2.u[s2.first[b] + i];
          const double* uj = s2.u[s2.first[b] + j];
          for (int a = 0; a < g2.mu; ++a)
            for (int bb = 0; bb < g2.mu; ++bb) coef2[q][g2.cls_of[a][bb]] += ui[a] * uj[bb];
          ++q;
        }
    if (q != kT2Ent) return cudaErrorInvalidValue;
    e = cudaMemcpyToSymbol(c_coef2, coef2, sizeof coef2);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyToSymbol(c_ent2, ent2, sizeof ent2);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyToSymbol(c_sym2, &s2, sizeof(SymBasis));
    if (e != cudaSuccess) return e;
  }
  e = cudaMemcpyToSymbol(c_W2f, W2f, sizeof W2f);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_B2f, B2f, sizeof B2f);
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_B2, B2, sizeof B2);
}

cudaError_t launch_eig_t2(lsp_ctx* c, const int32_t* count, int64_t cap) {
  int t = timer_begin(c, "eig_t2");
  constexpr int kW = 2;
  int64_t b = (cap + kW - 1) / kW;
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  k_eig2d_t2<kW><<<(int)b, kW * 32, 0, c->stream>>>(
      (const double*)c->gvals.p, cap, count, (double*)c->alpha2.p, (double*)c->cst2.p,
      (double*)c->lam2.p, (int32_t*)c->sflags2.p);
  timer_end(c, t);
  return cudaGetLastError();
}

cudaError_t launch_eig(lsp_ctx* c, const int32_t* count, int64_t cap, int method, int refine,
                       bool fp32_gram) {
  int t = timer_begin(c, "eig");
  cudaError_t e;
  if (c->geo.d == 2 && method == LSP_EIG_SYMMETRIC && refine == 0) {
    // one thread per shift; the block size (<= 128) and grid cap come from the autotuner
    e = tuned_launch(c, std::string("eig2d/") + (fp32_gram ? "f32" : "f64") + "/w" +
                            work_bucket(cap),
                     {128, 16}, 128, 0, [&](LaunchShape sh) {
      int64_t b = (cap + sh.threads - 1) / sh.threads;
      if (b > 152 * (int64_t)sh.per_sm) b = 152 * (int64_t)sh.per_sm;
      if (b < 1) b = 1;
      if (fp32_gram)
        k_eig2d<float><<<(int)b, sh.threads, 0, c->stream>>>(
            (const double*)c->gvals.p, cap, count, (double*)c->alpha.p, (double*)c->cst.p,
            (double*)c->lam.p, (int32_t*)c->sflags.p, (const int32_t*)c->shift_m.p,
            (double*)c->ap.p);
      else
        k_eig2d<double><<<(int)b, sh.threads, 0, c->stream>>>(
            (const double*)c->gvals.p, cap, count, (double*)c->alpha.p, (double*)c->cst.p,
            (double*)c->lam.p, (int32_t*)c->sflags.p, (const int32_t*)c->shift_m.p,
            (double*)c->ap.p);
      return cudaGetLastError();
    });
  } else if (c->geo.d == 3 && method == LSP_EIG_SYMMETRIC && refine == 0) {
    constexpr int kW = 4;
    int64_t b = (cap + kW - 1) / kW;
    if (b > 152 * 8) b = 152 * 8;
    if (b < 1) b = 1;
    k_eig3d<kW><<<(int)b, kW * 32, 0, c->stream>>>((const double*)c->gvals.p, cap, count,
                                                   (double*)c->alpha.p, (double*)c->cst.p,
                                                   (double*)c->lam.p, (int32_t*)c->sflags.p,
                                                   (const int32_t*)c->shift_m.p,
                                                   (double*)c->ap.p);
    e = cudaGetLastError();
  } else {
    e = c->geo.d == 1   ? launch_eig_t<3, 3, 8>(c, count, cap, method, refine)
        : c->geo.d == 2 ? launch_eig_t<9, 6, 8>(c, count, cap, method, refine)
                        : launch_eig_t<27, 10, 2>(c, count, cap, method, refine);
  }
  timer_end(c, t);
  return e;
}

}  // namespace lsp
