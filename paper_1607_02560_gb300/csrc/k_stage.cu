// Step a3: kernel vectors g_s and g_s * g_s at the offsets of mu_0 - mu_0, for every shift.
//
// Definition (Sec. 3 and Sec. 4.2): G_s = F^-1 diag(1/(4 pi^2 |k|^2 + s)) F, so
//   g_s[o]       = N^-1 sum_{k in K} e^{2 pi i o.k / n} / (4 pi^2 |k|^2 + s),
//   (g_s*g_s)[o] = N^-1 sum_{k in K} e^{2 pi i o.k / n} / (4 pi^2 |k|^2 + s)^2.
// The summand depends on k only through |k_1|, ..., |k_d|, so folding the signs of k gives
//   g_f[o](s) = N^-1 sum_{p in [0, n/2]^d} prod_i X_{|o_i|}(p_i) w_f(|p|^2 + m),
// with X_a(p) = w_p cos(2 pi a p / n) (w_p = 1 at p = 0, n/2, else 2) and, because every shift
// lies on the lattice s = (4m+2) pi^2 (Sec. 4.1), 4 pi^2 |k|^2 + s = pi^2 (4 (|k|^2 + m) + 2):
// the denominator is a function of the integer |p|^2 + m alone, w_f(l) = (pi^2 (4 l + 2))^-f.
//
// The d-fold sum is evaluated one axis at a time, each stage shared by all shifts:
//   T_0,f(l) = w_f(l)                                   (table over E_0),
//   T_k,f[a, rest](l) = sum_p X_a(p) T_{k-1},f[rest](p^2 + l)   for l in E_k,
//   g_f[a_1..a_d](m) = N^-1 T_d,f[a_1..a_d](m)          (E_d = the shift list).
// T_k is symmetric in its class tuple, so only sorted tuples (a <= rest) are formed. This is
// the exact sum of the definition with the terms grouped by axis; no approximation is made.
#include "lsp_internal.h"

namespace lsp {
namespace {

constexpr int kThreads = 256;

// Output class c of stage k: (first index a, class of the remaining tuple in stage k-1).
// Stage 2 pairs (a<=b): 00 01 02 11 12 22. Stage 3 triples (a<=b<=c): 000 001 002 011 012 022
// 111 112 122 222, remaining pair indexed as in stage 2. Compile-time tables, so the register
// arrays below are indexed by constants after unrolling.
template <int K>
struct StageMap;
template <>
struct StageMap<1> {
  static constexpr int NCP = 1, NCO = 3;
  __host__ __device__ static constexpr int a(int c) { return c; }
  __host__ __device__ static constexpr int r(int) { return 0; }
};
template <>
struct StageMap<2> {
  static constexpr int NCP = 3, NCO = 6;
  __host__ __device__ static constexpr int a(int c) {
    return c < 3 ? 0 : (c < 5 ? 1 : 2);
  }
  __host__ __device__ static constexpr int r(int c) {
    return c < 3 ? c : (c < 5 ? c - 2 : 2);
  }
};
template <>
struct StageMap<3> {
  static constexpr int NCP = 6, NCO = 10;
  __host__ __device__ static constexpr int a(int c) {
    return c < 6 ? 0 : (c < 9 ? 1 : 2);
  }
  __host__ __device__ static constexpr int r(int c) {
    return c < 6 ? c : (c < 9 ? c - 3 : 5);
  }
};

// One thread per domain point l. For stage 1 the input is the w table and w^2 is formed in
// registers; later stages read both functions of every input class. Output layout is
// structure-of-arrays: Tout[(c * 2 + f) * stride_out + pos].
template <int K>
__global__ void __launch_bounds__(kThreads) k_stage(const int32_t* __restrict__ list,
                                                    const int32_t* __restrict__ count_ptr, int P,
                                                    const double* __restrict__ X,
                                                    const double* __restrict__ Tprev,
                                                    int64_t lo_prev, int64_t stride_prev,
                                                    double* __restrict__ Tout, int64_t lo_out,
                                                    int64_t stride_out, int by_index,
                                                    double scale) {
  using M = StageMap<K>;
  extern __shared__ double xs[];  // [3][P]
  for (int i = threadIdx.x; i < 3 * P; i += kThreads) xs[i] = X[i];
  __syncthreads();
  // list == nullptr: the domain is the whole range [lo_out, lo_out + stride_out)
  const int64_t cnt = list ? (int64_t)*count_ptr : stride_out;
  for (int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x; idx < cnt;
       idx += (int64_t)gridDim.x * kThreads) {
    const int64_t l = list ? (int64_t)__ldg(list + idx) : lo_out + idx;
    double acc[M::NCO][2];
#pragma unroll
    for (int c = 0; c < M::NCO; ++c) acc[c][0] = acc[c][1] = 0.0;
    const double* base = Tprev + (l - lo_prev);
    for (int p = 0; p < P; ++p) {
      const int64_t off = (int64_t)p * p;
      double in[M::NCP][2];
      if (K == 1) {
        const double w = __ldg(base + off);
        in[0][0] = w;
        in[0][1] = w * w;
      } else {
#pragma unroll
        for (int c = 0; c < M::NCP; ++c) {
          in[c][0] = __ldg(base + (2 * c + 0) * stride_prev + off);
          in[c][1] = __ldg(base + (2 * c + 1) * stride_prev + off);
        }
      }
      const double x[3] = {xs[p], xs[P + p], xs[2 * P + p]};
#pragma unroll
      for (int c = 0; c < M::NCO; ++c) {
        acc[c][0] = fma(x[M::a(c)], in[M::r(c)][0], acc[c][0]);
        acc[c][1] = fma(x[M::a(c)], in[M::r(c)][1], acc[c][1]);
      }
    }
    const int64_t pos = by_index ? idx : (l - lo_out);
#pragma unroll
    for (int c = 0; c < M::NCO; ++c) {
      Tout[(2 * c + 0) * stride_out + pos] = acc[c][0] * scale;
      Tout[(2 * c + 1) * stride_out + pos] = acc[c][1] * scale;
    }
  }
}

template <int K>
cudaError_t launch_k(lsp_ctx* c, const int32_t* list, const int32_t* count, int64_t cap,
                     const double* Tprev, int64_t lo_prev, int64_t stride_prev, double* Tout,
                     int64_t lo_out, int64_t stride_out, bool by_index, double scale) {
  const int P = c->geo.P;
  const size_t smem = sizeof(double) * 3 * P;
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k_stage<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int64_t b = (cap + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > 152 * 16) b = 152 * 16;
  k_stage<K><<<(int)b, kThreads, smem, c->stream>>>(list, count, P, (const double*)c->xtab.p,
                                                     Tprev, lo_prev, stride_prev, Tout, lo_out,
                                                     stride_out, by_index ? 1 : 0, scale);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_stage(lsp_ctx* c, int d, int k, const int32_t* list, const int32_t* count,
                         int64_t cap, const double* Tprev, int64_t lo_prev, int64_t stride_prev,
                         double* Tout, int64_t lo_out, int64_t stride_out, bool by_index) {
  // The final stage carries the 1/N of the inverse transform (N a power of two: exact).
  const double scale = (k == d) ? 1.0 / (double)c->geo.N : 1.0;
  static const char* names[4] = {"", "stage1", "stage2", "stage3"};
  int t = timer_begin(c, names[k]);
  cudaError_t e;
  if (k == 1)
    e = launch_k<1>(c, list, count, cap, Tprev, lo_prev, stride_prev, Tout, lo_out, stride_out,
                    by_index, scale);
  else if (k == 2)
    e = launch_k<2>(c, list, count, cap, Tprev, lo_prev, stride_prev, Tout, lo_out, stride_out,
                    by_index, scale);
  else
    e = launch_k<3>(c, list, count, cap, Tprev, lo_prev, stride_prev, Tout, lo_out, stride_out,
                    by_index, scale);
  timer_end(c, t);
  (void)d;
  return e;
}

}  // namespace lsp
