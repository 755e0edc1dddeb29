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
__device__ int jacobi_small(double a[4][4], double v[4][4], int dim) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) v[i][j] = (i == j) ? 1.0 : 0.0;
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
__device__ void refine_step(WarpSmem<MU>& sm, int lane, int centre) {
  double* M = sm.V;  // the matrix (A0 - sigma I); the right-hand side lives in sm.work
  for (int e = lane; e < MU * MU; e += 32) {
    const int a = e / MU, b = e % MU;
    double s = 0.0;
    for (int k = 0; k < MU; ++k) s = fma(sm.g[2 * c_cls[a][k]], sm.g[2 * c_cls[b][k]], s);
    M[e] = sm.g[2 * c_cls[a][b] + 1] - s;
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
                                                    int32_t* __restrict__ flags_out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  WarpSmem<MU>& sm = reinterpret_cast<WarpSmem<MU>*>(smraw)[w];
  const int64_t cnt = *count;
  const int centre = MU / 2;
  for (int64_t i = (int64_t)blockIdx.x * WARPS + w; i < cnt; i += (int64_t)gridDim.x * WARPS) {
    if (lane < 2 * NCLS) sm.g[lane] = gvals[(int64_t)lane * cap + i];
    __syncwarp();
    // a4: A = A1 - G G^T
    for (int e = lane; e < MU * MU; e += 32) {
      const int a = e / MU, b = e % MU;
      double s = 0.0;
      for (int k = 0; k < MU; ++k) s = fma(sm.g[2 * c_cls[a][k]], sm.g[2 * c_cls[b][k]], s);
      sm.A[e] = sm.g[2 * c_cls[a][b] + 1] - s;
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
        const double* ui = c_sym.u[c_sym.first[b] + ii];
        const double* uj = c_sym.u[c_sym.first[b] + jj];
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
        double a[4][4], v[4][4];
        for (int r = 0; r < 4; ++r)
          for (int q = 0; q < 4; ++q) a[r][q] = (r < dim && q < dim) ? sm.B[lane][r * 4 + q] : 0.0;
        sm.conv[lane] = jacobi_small(a, v, dim);
        // sort eigenvalues ascending, keep the eigenvector of the smallest
        int order[4] = {0, 1, 2, 3};
        for (int r = 0; r < dim; ++r)
          for (int q = r + 1; q < dim; ++q)
            if (a[order[q]][order[q]] < a[order[r]][order[r]]) {
              int tmp = order[r];
              order[r] = order[q];
              order[q] = tmp;
            }
        for (int r = 0; r < 4; ++r) sm.lam[lane][r] = r < dim ? a[order[r]][order[r]] : DBL_MAX;
        for (int r = 0; r < 4; ++r) sm.y[lane][r] = r < dim ? v[r][order[0]] : 0.0;
      }
      __syncwarp();
      if (lane == 0) {
        int bstar = 0;
        for (int b = 1; b < c_sym.nblk; ++b)
          if (sm.lam[b][0] < sm.lam[bstar][0]) bstar = b;
        lam1 = sm.lam[bstar][0];
        lam2 = DBL_MAX;
        for (int b = 0; b < c_sym.nblk; ++b) {
          for (int r = 0; r < c_sym.dim[b]; ++r) {
            lmax = fmax(lmax, fabs(sm.lam[b][r]));
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
            s = fma(sm.y[bstar][r], c_sym.u[c_sym.first[bstar] + r][a], s);
          sm.alpha[a] = s;
        }
      }
    }
    if (lane == 0) {
      if (lam2 - lam1 < 1e-8 * lmax) flags |= LSP_FLAG_DEGENERATE;
      sign_fix<MU>(sm.alpha, centre);
    }
    __syncwarp();
    for (int r = 0; r < refine; ++r) refine_step<MU>(sm, lane, centre);
    // a6: c[b] = sum_a alpha[a] G[a, b]
    if (lane < MU) {
      double s = 0.0;
      for (int a = 0; a < MU; ++a) s = fma(sm.g[2 * c_cls[a][lane]], sm.alpha[a], s);
      alpha_out[i * MU + lane] = sm.alpha[lane];
      c_out[i * MU + lane] = s;
    }
    if (lane == 0) {
      lam_out[2 * i + 0] = lam1;
      lam_out[2 * i + 1] = lam2;
      flags_out[i] = flags;
    }
    __syncwarp();
  }
}

template <int MU, int NCLS, int WARPS>
cudaError_t launch_eig_t(lsp_ctx* c, const int32_t* count, int64_t cap, int method, int refine) {
  const size_t smem = sizeof(WarpSmem<MU>) * WARPS;
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
      (double*)c->cst.p, (double*)c->lam.p, (int32_t*)c->sflags.p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t upload_sym(lsp_ctx* c) {
  cudaError_t e = cudaMemcpyToSymbol(c_cls, c->geo.cls_of, sizeof(c->geo.cls_of));
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
  return cudaMemcpyToSymbol(c_nent, &n, sizeof(int));
}

cudaError_t launch_eig(lsp_ctx* c, const int32_t* count, int64_t cap, int method, int refine) {
  int t = timer_begin(c, "eig");
  cudaError_t e = c->geo.d == 2 ? launch_eig_t<9, 6, 8>(c, count, cap, method, refine)
                                : launch_eig_t<27, 10, 2>(c, count, cap, method, refine);
  timer_end(c, t);
  return e;
}

}  // namespace lsp
