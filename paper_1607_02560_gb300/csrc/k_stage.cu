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

// Output class c of stage k: (first index a, class of the remaining tuple in stage k-1), for
// A cosine rows X_0..X_{A-1} (A = 2t + 1: offsets up to 2t are needed for mu^t). Stage 1 has A
// classes (a). Stage 2 pairs (a <= b): for A = 3 in the order 00 01 02 11 12 22; for A = 5
// the same six first, then the pairs with b = 3 (03 13 23 33) and b = 4 (04 14 24 34 44), so
// the classes of t = 1 keep their indices in a t = 2 table. Stage 3 triples (a <= b <= c, A = 3):
// 000 001 002 011 012 022 111 112 122 222, remaining pair indexed as in stage 2. Compile-time
// tables, so the register arrays below are indexed by constants after unrolling.
template <int K, int A>
struct StageMap;
template <int A>
struct StageMap<1, A> {
  static constexpr int NCP = 1, NCO = A;
  __host__ __device__ static constexpr int a(int c) { return c; }
  __host__ __device__ static constexpr int r(int) { return 0; }
};
template <>
struct StageMap<2, 3> {
  static constexpr int NCP = 3, NCO = 6;
  __host__ __device__ static constexpr int a(int c) {
    return c < 3 ? 0 : (c < 5 ? 1 : 2);
  }
  __host__ __device__ static constexpr int r(int c) {
    return c < 3 ? c : (c < 5 ? c - 2 : 2);
  }
};
template <>
struct StageMap<2, 5> {
  static constexpr int NCP = 5, NCO = 15;
  __host__ __device__ static constexpr int a(int c) {
    return c < 6 ? StageMap<2, 3>::a(c) : (c < 10 ? c - 6 : c - 10);
  }
  __host__ __device__ static constexpr int r(int c) {
    return c < 6 ? StageMap<2, 3>::r(c) : (c < 10 ? 3 : 4);
  }
};
template <>
struct StageMap<3, 3> {
  static constexpr int NCP = 6, NCO = 10;
  __host__ __device__ static constexpr int a(int c) {
    return c < 6 ? 0 : (c < 9 ? 1 : 2);
  }
  __host__ __device__ static constexpr int r(int c) {
    return c < 6 ? c : (c < 9 ? c - 3 : 5);
  }
};

// Stage 3 for A = 5 (t = 2 in 3D): the 35 sorted triples over {0..4}, the ten of A = 3 first
// in their order, then those with largest component 3, then 4, each group lexicographic; a
// triple (a <= b <= c) is (a, class of the pair (b, c) in the stage-2 order of A = 5).
template <>
struct StageMap<3, 5> {
  static constexpr int NCP = 15, NCO = 35;
  __host__ __device__ static constexpr int a(int c) {
    constexpr int t[35] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 2, 0, 0, 0, 0, 1, 1, 1, 2,
                           2, 3, 0, 0, 0, 0, 0, 1, 1, 1, 1, 2, 2, 2, 3, 3, 4};
    return t[c];
  }
  __host__ __device__ static constexpr int r(int c) {
    constexpr int t[35] = {0, 1, 2, 3, 4,  5,  3,  4,  5,  5,  6,  7,  8,  9,  7,  8,  9, 8,
                           9, 9, 10, 11, 12, 13, 14, 11, 12, 13, 14, 12, 13, 14, 13, 14, 14};
    return t[c];
  }
};

// R is the arithmetic type: double for the FP64 mode, float for the mixed mode. OUT is the
// type of the output table (the last stage always writes double g values).
template <typename R>
struct Vec2;
template <>
struct Vec2<double> { using type = double2; };
template <>
struct Vec2<float> { using type = float2; };

// Accumulate the stage-K sums of one domain point l over the frequencies p = first, first +
// step, ... (all of them for step = 1). Structure-of-arrays tables: Tprev[(c * 2 + f) *
// stride_prev + (l + p^2 - lo_prev)].
//
// Stage 1 reads the w table and pairs every p < n/4 with its mirror q = n/2 - p:
// X_a(q) = (-1)^a X_a(p) (w_q = w_p, cos(pi a - t) = (-1)^a cos t), so
//   sum_p X_a(p) w(p^2 + l) = sum_{p < n/4} X_a(p) [w(p^2 + l) + (-1)^a w(q^2 + l)] + X_a(n/4) w(n^2/16 + l),
// 5 arithmetic operations per frequency instead of 7 (the host table satisfies the mirror
// identity exactly). In FP64 the table interleaves (w, w^2) and is read with one 16-byte load
// (the FP64 pipe is the bound); in FP32 it holds w alone and the square is formed in registers
// (the L2 bandwidth is the bound).
template <int K, int A, typename R>
__device__ __forceinline__ void stage_accumulate(const R* __restrict__ xs, int P, int64_t l,
                                                 const R* __restrict__ Tprev, int64_t lo_prev,
                                                 int64_t stride_prev, int first, int step,
                                                 R (&acc)[StageMap<K, A>::NCO][2]) {
  using M = StageMap<K, A>;
  using R2 = typename Vec2<R>::type;
  const int half = P - 1;  // n/2
  if (K == 1) {
    const R2* tab = reinterpret_cast<const R2*>(Tprev) + (l - lo_prev);
    const R* tab1 = Tprev + (l - lo_prev);
    constexpr bool kPair = sizeof(R) == 8;
    const int quarter = half / 2;  // n/4
#pragma unroll 4
    for (int p = first; p < quarter; p += step) {
      const int q = half - p;
      R2 wa, wb;
      if (kPair) {
        wa = __ldg(tab + (int64_t)p * p);
        wb = __ldg(tab + (int64_t)q * q);
      } else {
        wa.x = __ldg(tab1 + (int64_t)p * p);
        wb.x = __ldg(tab1 + (int64_t)q * q);
        wa.y = wa.x * wa.x;
        wb.y = wb.x * wb.x;
      }
      const R s1 = wa.x + wb.x, d1 = wa.x - wb.x;
      const R s2 = wa.y + wb.y, d2 = wa.y - wb.y;
#pragma unroll
      for (int a = 0; a < A; ++a) {  // even a: X_a(q) = X_a(p); odd a: X_a(q) = -X_a(p)
        const R xa = xs[a * P + p];
        acc[a][0] = fma(xa, (a & 1) ? d1 : s1, acc[a][0]);
        acc[a][1] = fma(xa, (a & 1) ? d2 : s2, acc[a][1]);
      }
    }
    if (first == 0) {
      R2 wm;
      if (kPair) {
        wm = __ldg(tab + (int64_t)quarter * quarter);
      } else {
        wm.x = __ldg(tab1 + (int64_t)quarter * quarter);
        wm.y = wm.x * wm.x;
      }
#pragma unroll
      for (int c = 0; c < A; ++c) {
        acc[c][0] = fma(xs[c * P + quarter], wm.x, acc[c][0]);
        acc[c][1] = fma(xs[c * P + quarter], wm.y, acc[c][1]);
      }
    }
  } else {
    const R* base = Tprev + (l - lo_prev);
    for (int p = first; p < P; p += step) {
      const int64_t off = (int64_t)p * p;
      R in[M::NCP][2];
#pragma unroll
      for (int c = 0; c < M::NCP; ++c) {
        in[c][0] = __ldg(base + (2 * c + 0) * stride_prev + off);
        in[c][1] = __ldg(base + (2 * c + 1) * stride_prev + off);
      }
      R x[A];
#pragma unroll
      for (int a = 0; a < A; ++a) x[a] = xs[a * P + p];
#pragma unroll
      for (int c = 0; c < M::NCO; ++c) {
        acc[c][0] = fma(x[M::a(c)], in[M::r(c)][0], acc[c][0]);
        acc[c][1] = fma(x[M::a(c)], in[M::r(c)][1], acc[c][1]);
      }
    }
  }
}

// One thread per domain point (SPLIT = false), or one warp per domain point with the lanes
// splitting the frequencies and a shuffle reduction at the end (SPLIT = true, used when the
// domain is too small to fill the GPU, e.g. a few dozen shifts). Output: Tout[(c * 2 + f) *
// stride_out + pos], pos = index in the list (by_index) or l - lo_out.
template <int K, int A, typename R, typename OUT, bool SPLIT>
__global__ void __launch_bounds__(kThreads) k_stage(const int32_t* __restrict__ list,
                                                    const int32_t* __restrict__ count_ptr, int P,
                                                    const R* __restrict__ X,
                                                    const R* __restrict__ Tprev,
                                                    int64_t lo_prev, int64_t stride_prev,
                                                    OUT* __restrict__ Tout, int64_t lo_out,
                                                    int64_t stride_out, int by_index,
                                                    double scale, int32_t* __restrict__ err) {
  using M = StageMap<K, A>;
  extern __shared__ __align__(16) unsigned char xs_raw[];
  R* xs = reinterpret_cast<R*>(xs_raw);  // [A][P]
  for (int i = threadIdx.x; i < A * P; i += kThreads) xs[i] = X[i];
  __syncthreads();
  // list == nullptr: the domain is the whole range [lo_out, lo_out + stride_out)
  const int64_t cnt = list ? (int64_t)*count_ptr : stride_out;
  const int lane = threadIdx.x & 31;
  const int64_t per_block = SPLIT ? kThreads / 32 : kThreads;
  const int64_t sub = SPLIT ? (threadIdx.x >> 5) : threadIdx.x;
  for (int64_t idx = (int64_t)blockIdx.x * per_block + sub; idx < cnt;
       idx += (int64_t)gridDim.x * per_block) {
    const int64_t l = list ? (int64_t)__ldg(list + idx) : lo_out + idx;
    const int64_t pos = by_index ? idx : (l - lo_out);
    // the previous table is read at l + p^2, p in [0, n/2]; the output at pos
    if (!checked_range(l - lo_prev, l - lo_prev + (int64_t)(P - 1) * (P - 1), stride_prev, err) ||
        !checked_range(pos, pos, stride_out, err))
      continue;
    R acc[M::NCO][2];
#pragma unroll
    for (int c = 0; c < M::NCO; ++c) acc[c][0] = acc[c][1] = R(0);
    stage_accumulate<K, A, R>(xs, P, l, Tprev, lo_prev, stride_prev, SPLIT ? lane : 0,
                           SPLIT ? 32 : 1, acc);
    if (SPLIT) {
#pragma unroll
      for (int c = 0; c < M::NCO; ++c)
#pragma unroll
        for (int f = 0; f < 2; ++f)
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) acc[c][f] += __shfl_xor_sync(0xffffffffu, acc[c][f], o);
      if (lane != 0) continue;
    }
#pragma unroll
    for (int c = 0; c < M::NCO; ++c) {
      Tout[(2 * c + 0) * stride_out + pos] = (OUT)((double)acc[c][0] * scale);
      Tout[(2 * c + 1) * stride_out + pos] = (OUT)((double)acc[c][1] * scale);
    }
  }
}

template <int K, int A, typename R, typename OUT, bool SPLIT>
cudaError_t launch_kk(lsp_ctx* c, const int32_t* list, const int32_t* count, int64_t cap,
                      const R* X, const R* Tprev, int64_t lo_prev, int64_t stride_prev, OUT* Tout,
                      int64_t lo_out, int64_t stride_out, bool by_index, double scale) {
  const int P = c->geo.P;
  const size_t smem = sizeof(R) * A * P;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_stage<K, A, R, OUT, SPLIT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t per_block = SPLIT ? kThreads / 32 : kThreads;
  int64_t b = (cap + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > 152 * 16) b = 152 * 16;
  k_stage<K, A, R, OUT, SPLIT><<<(int)b, kThreads, smem, c->stream>>>(
      list, count, P, X, Tprev, lo_prev, stride_prev, Tout, lo_out, stride_out, by_index ? 1 : 0,
      scale, (int32_t*)c->counts.p + kErrWord);
  return cudaGetLastError();
}

// Domains below about two threads per SM-lane slot are spread over warps instead.
constexpr int64_t kSplitBelow = 152 * 256;

template <int K, int A, typename R, typename OUT>
cudaError_t launch_k(lsp_ctx* c, const int32_t* list, const int32_t* count, int64_t cap,
                     const R* X, const R* Tprev, int64_t lo_prev, int64_t stride_prev, OUT* Tout,
                     int64_t lo_out, int64_t stride_out, bool by_index, double scale) {
  if (cap < kSplitBelow)
    return launch_kk<K, A, R, OUT, true>(c, list, count, cap, X, Tprev, lo_prev, stride_prev,
                                         Tout, lo_out, stride_out, by_index, scale);
  return launch_kk<K, A, R, OUT, false>(c, list, count, cap, X, Tprev, lo_prev, stride_prev, Tout,
                                        lo_out, stride_out, by_index, scale);
}

template <typename R>
cudaError_t launch_typed(lsp_ctx* c, int d, int k, int t, const int32_t* list,
                         const int32_t* count, int64_t cap, const void* Tprev, int64_t lo_prev,
                         int64_t stride_prev, void* Tout, int64_t lo_out, int64_t stride_out,
                         bool by_index, double scale, const R* X) {
  const R* prev = (const R*)Tprev;
  if (t == 2) {  // five cosine rows (2D and 3D)
    if (k == 1)
      return launch_k<1, 5, R, R>(c, list, count, cap, X, prev, lo_prev, stride_prev, (R*)Tout,
                                  lo_out, stride_out, by_index, scale);
    if (k == 2 && d == 3)
      return launch_k<2, 5, R, R>(c, list, count, cap, X, prev, lo_prev, stride_prev, (R*)Tout,
                                  lo_out, stride_out, by_index, scale);
    if (k == 2)
      return launch_k<2, 5, R, double>(c, list, count, cap, X, prev, lo_prev, stride_prev,
                                       (double*)Tout, lo_out, stride_out, by_index, scale);
    return launch_k<3, 5, R, double>(c, list, count, cap, X, prev, lo_prev, stride_prev,
                                     (double*)Tout, lo_out, stride_out, by_index, scale);
  }
  if (k == d) {  // last stage: double g values for the eigen step
    double* out = (double*)Tout;
    if (k == 1)  // 1D: the single stage
      return launch_k<1, 3, R, double>(c, list, count, cap, X, prev, lo_prev, stride_prev, out,
                                       lo_out, stride_out, by_index, scale);
    if (k == 2)
      return launch_k<2, 3, R, double>(c, list, count, cap, X, prev, lo_prev, stride_prev, out,
                                       lo_out, stride_out, by_index, scale);
    return launch_k<3, 3, R, double>(c, list, count, cap, X, prev, lo_prev, stride_prev, out,
                                     lo_out, stride_out, by_index, scale);
  }
  R* out = (R*)Tout;
  if (k == 1)
    return launch_k<1, 3, R, R>(c, list, count, cap, X, prev, lo_prev, stride_prev, out, lo_out,
                                stride_out, by_index, scale);
  return launch_k<2, 3, R, R>(c, list, count, cap, X, prev, lo_prev, stride_prev, out, lo_out,
                              stride_out, by_index, scale);
}

}  // namespace

cudaError_t launch_stage(lsp_ctx* c, int d, int k, int t, const int32_t* list,
                         const int32_t* count, int64_t cap, const void* Tprev, int64_t lo_prev,
                         int64_t stride_prev, void* Tout, int64_t lo_out, int64_t stride_out,
                         bool by_index, bool fp32) {
  // The final stage carries the 1/N of the inverse transform (N a power of two: exact).
  const double scale = (k == d) ? 1.0 / (double)c->geo.N : 1.0;
  static const char* names[4] = {"", "stage1", "stage2", "stage3"};
  int tm = timer_begin(c, names[k]);
  cudaError_t e =
      fp32 ? launch_typed<float>(c, d, k, t, list, count, cap, Tprev, lo_prev, stride_prev, Tout,
                                 lo_out, stride_out, by_index, scale, (const float*)c->xtab32.p)
           : launch_typed<double>(c, d, k, t, list, count, cap, Tprev, lo_prev, stride_prev, Tout,
                                  lo_out, stride_out, by_index, scale, (const double*)c->xtab.p);
  timer_end(c, tm);
  return e;
}

}  // namespace lsp
