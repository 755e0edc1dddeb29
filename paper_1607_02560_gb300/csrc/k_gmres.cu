// Device side of restarted GMRES (Sec. 5: restart 40, relative tolerance 1e-6) for
// (L + diag v) u = f, left-preconditioned by P^-1 C (Eq. PC). The Arnoldi basis V, the
// Hessenberg matrix H (column-major, leading dimension ld = restart + 1), the Givens rotations
// and the least-squares right-hand side S all stay on the device; the host loop reads back one
// residual estimate per inner iteration. Reductions use a fixed grid and a fixed summation
// order, so two runs on the same data take the same decisions.
#include <math.h>

#include "nd.h"

namespace lsp {
namespace {

constexpr int kRedBlocks = 1024;  // <= the partial-sum slots of GmresSlot
constexpr int kRedThreads = 256;

int red_grid(int64_t N) {
  const int64_t b = (N + kRedThreads - 1) / kRedThreads;
  return (int)(b < kRedBlocks ? (b > 0 ? b : 1) : kRedBlocks);
}

// w -= h_prev * v_prev (when v_prev), then *h_out = sum_i v_next[i] w[i] (or w[i]^2).
// The last block to finish adds the block partials in block order.
__global__ void __launch_bounds__(kRedThreads) k_mgs(double* __restrict__ w,
                                                     const double* __restrict__ v_prev,
                                                     const double* __restrict__ h_prev,
                                                     const double* __restrict__ v_next,
                                                     double* __restrict__ gs,
                                                     double* __restrict__ h_out, int64_t N) {
  __shared__ double wsum[kRedThreads / 32];
  __shared__ bool last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double h = v_prev ? *h_prev : 0.0;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kRedThreads + tid; i < N;
       i += (int64_t)gridDim.x * kRedThreads) {
    double wi = w[i];
    if (v_prev) {
      wi = fma(-h, v_prev[i], wi);
      w[i] = wi;
    }
    acc = fma(v_next ? v_next[i] : wi, wi, acc);
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) wsum[warp] = acc;
  __syncthreads();
  if (tid == 0) {
    double b = 0.0;
    for (int k = 0; k < kRedThreads / 32; ++k) b += wsum[k];
    gs[kGsPartial + blockIdx.x] = b;
    __threadfence();
    const unsigned t = atomicAdd((unsigned*)(gs + kGsTicket), 1u);
    last = t == gridDim.x - 1;
  }
  __syncthreads();
  if (last && warp == 0) {
    __threadfence();
    double b = 0.0;
    for (int k = lane; k < (int)gridDim.x; k += 32) b += __ldcg(gs + kGsPartial + k);
    for (int off = 16; off > 0; off >>= 1) b += __shfl_xor_sync(0xffffffffu, b, off);
    if (lane == 0) {
      *h_out = b;
      *(unsigned*)(gs + kGsTicket) = 0u;
    }
  }
}

// y[i] = (a ? a[i] : 0) + sign * (scale ? *scale : 1) * x[i]
__global__ void k_axpby(double* __restrict__ y, const double* a, const double* x,
                        const double* __restrict__ scale, double sign, int64_t N) {
  const double sc = sign * (scale ? *scale : 1.0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(sc, x[i], a ? a[i] : 0.0);
}

// v0 = r / beta with beta = sqrt(gs[kGsNorm]); S = (beta, 0, ...).
__global__ void k_gmres_start(double* __restrict__ gs, int ld, int restart,
                              const double* __restrict__ r, double* __restrict__ v0, int64_t N) {
  __shared__ double sinv;
  const double beta = sqrt(gs[kGsNorm]);
  if (threadIdx.x == 0) sinv = beta > 0.0 ? 1.0 / beta : 0.0;  // one division per block
  __syncthreads();
  const double inv = sinv;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    v0[i] = r[i] * inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double* S = gs + kGsArrays + (int64_t)ld * restart + 2 * restart;
    for (int k = 0; k < ld; ++k) S[k] = 0.0;
    S[0] = beta;
    gs[kGsBeta] = beta;
  }
}

// Column col of H holds <v_k, w> (k <= col) from the MGS steps; complete it with |w|, apply
// the previous rotations, make the rotation that zeroes H[col + 1][col], rotate S.
__global__ void k_gmres_givens(double* __restrict__ gs, int col, int ld, int restart) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double* H = gs + kGsArrays;
  double* cs = H + (int64_t)ld * restart;
  double* sn = cs + restart;
  double* S = sn + restart;
  double* hc = H + (int64_t)col * ld;
  const double h0 = sqrt(gs[kGsH0]), h1 = sqrt(gs[kGsH1]);
  const bool brk = !(h1 > 2.220446049250313e-16 * h0);
  gs[kGsBreak] = brk ? 1.0 : 0.0;
  gs[kGsInvH1] = brk ? 0.0 : 1.0 / h1;
  hc[col + 1] = brk ? 0.0 : h1;
  for (int k = 0; k < col; ++k) {
    const double a = hc[k], b = hc[k + 1];
    hc[k] = cs[k] * a + sn[k] * b;
    hc[k + 1] = -sn[k] * a + cs[k] * b;
  }
  const double a = hc[col], b = hc[col + 1];
  const double rr = hypot(a, b);
  double c = 1.0, s = 0.0;
  if (rr > 0.0) {
    c = a / rr;
    s = b / rr;
  }
  cs[col] = c;
  sn[col] = s;
  hc[col] = rr;
  hc[col + 1] = 0.0;
  S[col + 1] = -s * S[col];
  S[col] = c * S[col];
  gs[kGsPresid] = fabs(S[col + 1]);
}

// y = H[0..col, 0..col]^-1 S[0..col] (back substitution, in every block), x += V[:, 0..col] y.
__global__ void k_gmres_update(const double* __restrict__ gs, int col, int ld, int restart,
                               const double* __restrict__ V, double* __restrict__ x, int64_t N) {
  __shared__ double y[64];
  if (threadIdx.x == 0) {
    const double* H = gs + kGsArrays;
    const double* S = H + (int64_t)ld * restart + 2 * restart;
    for (int k = col; k >= 0; --k) {
      double v = S[k];
      for (int j = k + 1; j <= col; ++j) v -= H[(int64_t)j * ld + k] * y[j];
      const double d = H[(int64_t)k * ld + k];
      y[k] = d != 0.0 ? v / d : 0.0;
    }
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = x[i];
    for (int k = 0; k <= col; ++k) acc = fma(y[k], V[(int64_t)k * N + i], acc);
    x[i] = acc;
  }
}

int ew_grid(int64_t N) {
  const int64_t b = (N + 255) / 256;
  return (int)(b < 152 * 8 ? (b > 0 ? b : 1) : 152 * 8);
}

}  // namespace

cudaError_t launch_mgs(lsp_ctx* c, double* w, const double* v_prev, const double* h_prev,
                       const double* v_next, double* h_out, int64_t N) {
  double* gs = (double*)c->nd->gs.p;
  k_mgs<<<red_grid(N), kRedThreads, 0, c->stream>>>(w, v_prev, h_prev, v_next, gs, h_out, N);
  return cudaGetLastError();
}

cudaError_t launch_axpby(lsp_ctx* c, double* y, const double* a, const double* x,
                         const double* scale, double sign, int64_t N) {
  k_axpby<<<ew_grid(N), 256, 0, c->stream>>>(y, a, x, scale, sign, N);
  return cudaGetLastError();
}

cudaError_t launch_gmres_start(lsp_ctx* c, double* gs, int ld, const double* r, double* v0,
                               int64_t N) {
  k_gmres_start<<<ew_grid(N), 256, 0, c->stream>>>(gs, ld, ld - 1, r, v0, N);
  return cudaGetLastError();
}

cudaError_t launch_gmres_givens(lsp_ctx* c, double* gs, int col, int ld) {
  k_gmres_givens<<<1, 32, 0, c->stream>>>(gs, col, ld, ld - 1);
  return cudaGetLastError();
}

cudaError_t launch_gmres_update(lsp_ctx* c, double* gs, int col, int ld, const double* V,
                                double* x, int64_t N) {
  k_gmres_update<<<ew_grid(N), 256, 0, c->stream>>>(gs, col, ld, ld - 1, V, x, N);
  return cudaGetLastError();
}

}  // namespace lsp
