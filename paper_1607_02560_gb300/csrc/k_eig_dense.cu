// Steps a4-a6 for t = 2 in 3D (Sec. 4.2, Eq. A): the neighbourhood mu_0^2 = [-2, 2]^3 has
// 125 offsets and the kernel vectors enter through 35 classes (sorted |offset| triples over
// {0..4}). Few shifts occur in 3D (tens), so each shift gets one CTA and a dense solve:
//   A = A1 - Gm Gm^T, A1[a][b] = (g*g)[cls(a, b)], Gm[a][b] = g[cls(a, b)]   (Gm symmetric),
//   B = (A + delta I)^-1 by an in-place Gauss-Jordan sweep (A is positive semidefinite, so
//       A + delta I is positive definite and needs no pivoting), delta = 1e-13 trace(A),
//   alpha = the dominant eigenvector of B by power iteration (inverse iteration on A),
//   lambda_1 = alpha^T A alpha with A alpha = A1 alpha - Gm (Gm alpha) from the class values,
//   lambda_2 by the same iteration on B deflated by alpha (for the degeneracy flag),
//   c = Gm alpha (Sec. 4.1: C[j, mu_j] = Q[j, mu_j] G[mu_j, mu_j]).
// Sign: alpha[centre] > 0, else the first entry above 1e-12 in magnitude.
#include <float.h>
#include <math.h>

#include "lsp_internal.h"

namespace lsp {
namespace {

constexpr int kM = 125;    // |mu_0^2| in 3D
constexpr int kNC = 35;    // classes
constexpr int kT = 256;    // threads
constexpr int kPowerIters = 80;
constexpr int kDeflIters = 16;  // lambda_2 only decides the degeneracy flag

// the class table of mu_0^2 - mu_0^2 (uint8 [125][125]), copied into shared memory per CTA
__constant__ uint8_t c_cls125[kM * kM];

// y = M x for the 125 x 125 matrix M (row-major, shared), one warp per row, fixed order
__device__ __forceinline__ void matvec(const double* __restrict__ M, const double* __restrict__ x,
                                       double* __restrict__ y) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = warp; r < kM; r += kT / 32) {
    double acc = 0.0;
    for (int k = lane; k < kM; k += 32) acc = fma(M[r * kM + k], x[k], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y[r] = acc;
  }
}

// y = K x with K[a][b] = kv[cls(a, b)] (a class-valued symmetric matrix)
__device__ __forceinline__ void cls_matvec(const uint8_t* __restrict__ cls,
                                           const double* __restrict__ kv,
                                           const double* __restrict__ x, double* __restrict__ y) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = warp; r < kM; r += kT / 32) {
    double acc = 0.0;
    for (int k = lane; k < kM; k += 32) acc = fma(kv[cls[r * kM + k]], x[k], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y[r] = acc;
  }
}

// sum of x[i] y[i] over the CTA in a fixed order; every thread gets the result
__device__ __forceinline__ double dot(const double* x, const double* y, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc = 0.0;
  for (int i = threadIdx.x; i < kM; i += kT) acc = fma(x[i], y[i], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __syncthreads();
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < kT / 32; ++w) s += red[w];
  return s;
}

// 1 / sqrt(x . x): one reciprocal by one thread, shared with the CTA
__device__ __forceinline__ double inv_norm(const double* x, double* red, double* slot) {
  const double s = dot(x, x, red);
  if (threadIdx.x == 0) *slot = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  __syncthreads();
  return *slot;
}

__global__ void __launch_bounds__(kT) k_eig_dense3(const double* __restrict__ gvals, int64_t cap,
                                                   const int32_t* __restrict__ count,
                                                   double* __restrict__ alpha_out,
                                                   double* __restrict__ c_out,
                                                   double* __restrict__ lam_out,
                                                   int32_t* __restrict__ flags_out) {
  extern __shared__ double smd[];
  double* A = smd;                                          // 125 x 125
  uint8_t* cls = reinterpret_cast<uint8_t*>(A + kM * kM);  // 125 x 125
  __shared__ double g[2][kNC];
  __shared__ double x[kM], y[kM], u[kM], w[kM];
  __shared__ double red[kT / 32];
  __shared__ double sd;
  const int tid = threadIdx.x;
  for (int e = tid; e < kM * kM; e += kT) cls[e] = c_cls125[e];
  const int64_t ns = *count;
  for (int64_t i = blockIdx.x; i < ns; i += gridDim.x) {
    __syncthreads();
    for (int e = tid; e < 2 * kNC; e += kT)
      g[e % 2][e / 2] = gvals[(int64_t)e * cap + i];  // SoA [cls * 2 + f][cap]
    __syncthreads();
    // ---- A = A1 - Gm Gm^T: row a of Gm in registers of one warp's lanes, entries a <= b ----
    for (int a = tid >> 5; a < kM; a += kT / 32) {
      const uint8_t* ca = cls + a * kM;
      for (int b = a + (tid & 31); b < kM; b += 32) {
        const uint8_t* cb = cls + b * kM;
        double acc = g[1][ca[b]];
        for (int k = 0; k < kM; ++k) acc = fma(-g[0][ca[k]], g[0][cb[k]], acc);
        A[a * kM + b] = acc;
        A[b * kM + a] = acc;
      }
    }
    __syncthreads();
    double tr = 0.0;
    for (int a = 0; a < kM; ++a) tr += A[a * kM + a];
    const double delta = 1e-13 * fabs(tr);
    for (int a = tid; a < kM; a += kT) A[a * kM + a] += delta;
    __syncthreads();
    // ---- B = (A + delta I)^-1, Gauss-Jordan sweep in place (no pivoting) ----
    for (int k = 0; k < kM; ++k) {
      if (tid == 0) sd = 1.0 / A[k * kM + k];  // the one division of this pivot
      __syncthreads();
      const double dinv = sd;
      for (int j = tid; j < kM; j += kT) {
        u[j] = A[k * kM + j] * dinv;  // row k, scaled
        w[j] = A[j * kM + k];         // column k
      }
      __syncthreads();
      // one warp per row, lanes over the columns
      for (int r = tid >> 5; r < kM; r += kT / 32) {
        double* Ar = A + r * kM;
        const double wr = w[r];
        if (r == k) {
          for (int j = tid & 31; j < kM; j += 32) Ar[j] = j == k ? dinv : u[j];
        } else {
          for (int j = tid & 31; j < kM; j += 32) Ar[j] = j == k ? -wr * dinv : fma(-wr, u[j], Ar[j]);
        }
      }
      __syncthreads();
    }
    // ---- power iteration on B: alpha (the near-null vector of A) ----
    for (int a = tid; a < kM; a += kT) x[a] = 1.0 + 0.03125 * (double)((a * 37) % 17);
    __syncthreads();
    double inv = inv_norm(x, red, &sd);
    for (int a = tid; a < kM; a += kT) x[a] *= inv;
    __syncthreads();
    int flags = LSP_FLAG_NOT_CONVERGED;
    for (int it = 0; it < kPowerIters; ++it) {
      matvec(A, x, y);
      __syncthreads();
      inv = inv_norm(y, red, &sd);
      double chg = 0.0;
      for (int a = tid; a < kM; a += kT) {
        const double v = y[a] * inv;
        chg = fmax(chg, fabs(v - x[a]));
      }
      for (int o = 16; o > 0; o >>= 1) chg = fmax(chg, __shfl_xor_sync(0xffffffffu, chg, o));
      __syncthreads();
      if ((tid & 31) == 0) red[tid >> 5] = chg;
      __syncthreads();
      double cmax = 0.0;
      for (int q = 0; q < kT / 32; ++q) cmax = fmax(cmax, red[q]);
      for (int a = tid; a < kM; a += kT) x[a] = y[a] * inv;
      __syncthreads();
      if (cmax < 4e-15) {  // uniform: every thread reduced the same values
        flags = 0;
        break;
      }
    }
    // ---- lambda_1 = alpha^T A alpha; c = Gm alpha ----
    cls_matvec(cls, g[0], x, u);  // u = Gm alpha = c
    cls_matvec(cls, g[1], x, w);  // w = A1 alpha
    __syncthreads();
    cls_matvec(cls, g[0], u, y);  // y = Gm (Gm alpha)
    __syncthreads();
    for (int a = tid; a < kM; a += kT) w[a] -= y[a];  // A alpha
    __syncthreads();
    const double lam1 = dot(x, w, red);
    // ---- lambda_2: power iteration on B deflated by alpha ----
    for (int a = tid; a < kM; a += kT) y[a] = 1.0 - 0.0625 * (double)((a * 11) % 7);
    __syncthreads();
    double iw_last = 0.0;  // 1 / |B y| of the last step: lambda_2 + delta
    {
      const double pr = dot(x, y, red);
      for (int a = tid; a < kM; a += kT) y[a] -= pr * x[a];
      __syncthreads();
      const double iy = inv_norm(y, red, &sd);
      for (int a = tid; a < kM; a += kT) y[a] *= iy;
      __syncthreads();
    }
    for (int it = 0; it < kDeflIters; ++it) {  // w = B y, projected off alpha before and after
      matvec(A, y, w);
      __syncthreads();
      const double pr = dot(x, w, red);
      for (int a = tid; a < kM; a += kT) w[a] -= pr * x[a];
      __syncthreads();
      const double iw = inv_norm(w, red, &sd);
      if (!(iw > 0.0)) break;  // uniform
      iw_last = iw;
      for (int a = tid; a < kM; a += kT) y[a] = w[a] * iw;
      __syncthreads();
    }
    const double lam2 = iw_last > 0.0 ? iw_last - delta : DBL_MAX;
    if (lam2 - lam1 < 1e-8 * fabs(tr)) flags |= LSP_FLAG_DEGENERATE;
    // ---- sign and output ----
    double ref = x[kM / 2];
    if (!(fabs(ref) > 1e-12)) {
      ref = 0.0;
      for (int a = 0; a < kM; ++a)
        if (fabs(x[a]) > 1e-12) {
          ref = x[a];
          break;
        }
    }
    const double sg = ref < 0.0 ? -1.0 : 1.0;
    for (int a = tid; a < kM; a += kT) {
      alpha_out[i * kM + a] = sg * x[a];
      c_out[i * kM + a] = sg * u[a];
    }
    if (tid == 0) {
      lam_out[2 * i + 0] = lam1;
      lam_out[2 * i + 1] = lam2;
      flags_out[i] = flags;
    }
  }
}

}  // namespace

cudaError_t upload_cls125(const Geometry& g) {
  static uint8_t t[kM * kM];
  for (int a = 0; a < kM; ++a)
    for (int b = 0; b < kM; ++b) t[a * kM + b] = g.cls_of[a][b];
  return cudaMemcpyToSymbol(c_cls125, t, sizeof t);
}

cudaError_t launch_eig_dense3(lsp_ctx* c, const int32_t* count, int64_t cap) {
  if (c->geo2.mu != kM) return cudaErrorInvalidValue;
  const size_t smem = sizeof(double) * kM * kM + kM * kM;
  cudaError_t e = cudaFuncSetAttribute(k_eig_dense3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int t = timer_begin(c, "eig_t2");
  int64_t b = cap < 152 ? cap : 152;
  if (b < 1) b = 1;
  k_eig_dense3<<<(int)b, kT, smem, c->stream>>>(
      (const double*)c->gvals.p, cap, count, (double*)c->alpha2.p, (double*)c->cst2.p,
      (double*)c->lam2.p, (int32_t*)c->sflags2.p);
  timer_end(c, t);
  return cudaGetLastError();
}

}  // namespace lsp
