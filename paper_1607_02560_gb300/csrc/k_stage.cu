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
#include <type_traits>

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

// ---- double-word arithmetic on the FP32 pipe ----------------------------------------------
// A double word is an unevaluated sum h + l of two floats with |l| <= ulp(h) / 2, which carries
// about 48 significant bits. GB300 issues FP32 at 64 times its FP64 rate, so a stage evaluated
// in double words (about ten FP32 operations per multiply-add) costs a fraction of the FP64
// form. The building blocks are the classical error-free transformations: the exact sum of two
// floats with its rounding error (Knuth's two-sum, six operations) and the exact product with
// its error from one fused multiply-add. Explicit _rn intrinsics keep the compiler from
// contracting or reassociating them.
struct dword {
  float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e with |e| well below ulp(s) after the exact sum of a and b (|a| >= |b| or a = 0).
__device__ __forceinline__ dword fast_renorm(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// a + b and a - b of double words: the highs summed exactly, the lows and the error added.
__device__ __forceinline__ dword dw_add(dword a, dword b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return fast_renorm(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ dword dw_sub(dword a, dword b) {
  float s, e;
  two_sum(a.h, -b.h, s, e);
  return fast_renorm(s, __fadd_rn(e, __fsub_rn(a.l, b.l)));
}
// acc += x * y. The product of the highs is exact with its error term; the cross terms of
// the lows enter that error term; the high of the sum is formed exactly and its error, with
// the product's, goes into the low word. The low word is folded back by dw_norm every few
// steps, so that its own rounding stays at the level of the double-word precision.
__device__ __forceinline__ void dw_mac(dword& acc, dword x, dword y) {
  const float p = __fmul_rn(x.h, y.h);
  float pe = __fmaf_rn(x.h, y.h, -p);
  pe = __fmaf_rn(x.h, y.l, pe);
  pe = __fmaf_rn(x.l, y.h, pe);
  float s, e;
  two_sum(acc.h, p, s, e);
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(e, pe));
}
__device__ __forceinline__ void dw_norm(dword& a) { a = fast_renorm(a.h, a.l); }
__device__ __forceinline__ dword dw_shfl_xor(dword a, int o) {
  return {__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o)};
}

template <typename R>
__device__ __forceinline__ R zero_of() { return R(0); }
template <>
__device__ __forceinline__ dword zero_of<dword>() { return {0.0f, 0.0f}; }

// Output conversion: intermediate stages keep their type; the last stage writes FP64 g values
// (the final 1/N scale is a power of two, exact in every type).
__device__ __forceinline__ void store_out(double* p, double v, double scale) { *p = v * scale; }
__device__ __forceinline__ void store_out(float* p, float v, double scale) { *p = (float)((double)v * scale); }
__device__ __forceinline__ void store_out(double* p, float v, double scale) { *p = (double)v * scale; }
__device__ __forceinline__ void store_out(double* p, dword v, double scale) {
  *p = ((double)v.h + (double)v.l) * scale;
}
__device__ __forceinline__ void store_out(dword* p, dword v, double) {
  dw_norm(v);
  *p = v;
}

// Double-word form of stage_accumulate (below): the same sums in the same order, with the
// w table holding (w, w^2) as two double words per l (16 bytes, one load) and the stage tables
// holding double words. The accumulators are renormalised every four frequencies.
template <int K, int A>
__device__ __forceinline__ void stage_accumulate_dw(const dword* __restrict__ xs, int P,
                                                    int64_t l, const dword* __restrict__ Tprev,
                                                    int64_t lo_prev, int64_t stride_prev,
                                                    int first, int step,
                                                    dword (&acc)[StageMap<K, A>::NCO][2]) {
  using M = StageMap<K, A>;
  const int half = P - 1;  // n/2
  if (K == 1) {
    const float4* tab = reinterpret_cast<const float4*>(Tprev) + (l - lo_prev);
    const int quarter = half / 2;  // n/4
    int cnt = 0;
#pragma unroll 4
    for (int p = first; p < quarter; p += step) {
      const int q = half - p;
      const float4 wa = __ldg(tab + (int64_t)p * p);
      const float4 wb = __ldg(tab + (int64_t)q * q);
      const dword a1 = {wa.x, wa.y}, b1 = {wb.x, wb.y}, a2 = {wa.z, wa.w}, b2 = {wb.z, wb.w};
      const dword s1 = dw_add(a1, b1), d1 = dw_sub(a1, b1);
      const dword s2 = dw_add(a2, b2), d2 = dw_sub(a2, b2);
#pragma unroll
      for (int a = 0; a < A; ++a) {  // even a: X_a(q) = X_a(p); odd a: X_a(q) = -X_a(p)
        const dword xa = xs[a * P + p];
        dw_mac(acc[a][0], xa, (a & 1) ? d1 : s1);
        dw_mac(acc[a][1], xa, (a & 1) ? d2 : s2);
      }
      if ((++cnt & 3) == 0) {
#pragma unroll
        for (int a = 0; a < A; ++a) {
          dw_norm(acc[a][0]);
          dw_norm(acc[a][1]);
        }
      }
    }
    if (first == 0) {
      const float4 wm = __ldg(tab + (int64_t)quarter * quarter);
#pragma unroll
      for (int c = 0; c < A; ++c) {
        dw_mac(acc[c][0], xs[c * P + quarter], dword{wm.x, wm.y});
        dw_mac(acc[c][1], xs[c * P + quarter], dword{wm.z, wm.w});
      }
    }
  } else {
    const dword* base = Tprev + (l - lo_prev);
    int cnt = 0;
#pragma unroll 4
    for (int p = first; p < P; p += step) {
      const int64_t off = (int64_t)p * p;
      dword in[M::NCP][2];
#pragma unroll
      for (int c = 0; c < M::NCP; ++c) {
        const float2 v0 = __ldg(reinterpret_cast<const float2*>(base + (2 * c + 0) * stride_prev + off));
        const float2 v1 = __ldg(reinterpret_cast<const float2*>(base + (2 * c + 1) * stride_prev + off));
        in[c][0] = {v0.x, v0.y};
        in[c][1] = {v1.x, v1.y};
      }
      dword x[A];
#pragma unroll
      for (int a = 0; a < A; ++a) x[a] = xs[a * P + p];
#pragma unroll
      for (int c = 0; c < M::NCO; ++c) {
        dw_mac(acc[c][0], x[M::a(c)], in[M::r(c)][0]);
        dw_mac(acc[c][1], x[M::a(c)], in[M::r(c)][1]);
      }
      if ((++cnt & 3) == 0) {
#pragma unroll
        for (int c = 0; c < M::NCO; ++c) {
          dw_norm(acc[c][0]);
          dw_norm(acc[c][1]);
        }
      }
    }
  }
}

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
    // eight frequencies per trip: up to 48 gathers in flight per thread (the loop is bound by
    // their latency in FP32; measured 0.172 -> 0.165 ms FP32, 1.010 -> 0.999 ms FP64 at 2D
    // n = 1024); the order of the sum is unchanged
#pragma unroll 8
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

// LANES threads per domain point: one (a large domain fills the GPU by itself), four (a
// domain of a few hundred thousand points, e.g. the shift list of the per-point policy at 2D
// n = 1024, which one thread per point would leave at a third of the SM's thread slots), or a
// whole warp (a few dozen shifts). The lanes of a group split the frequencies (lane r takes
// p = r, r + LANES, ...) and a shuffle reduction combines them; the order of every sum depends
// only on LANES, which the domain size fixes, not on the launch shape. Output:
// Tout[(c * 2 + f) * stride_out + pos], pos = index in the list (by_index) or l - lo_out.
template <int K, int A, typename R, typename OUT, int LANES>
__device__ __forceinline__ void stage_body(const int32_t* __restrict__ list,
                                           const int32_t* __restrict__ count_ptr, int P,
                                           const R* __restrict__ X, const R* __restrict__ Tprev,
                                           int64_t lo_prev, int64_t stride_prev,
                                           OUT* __restrict__ Tout, int64_t lo_out,
                                           int64_t stride_out, int by_index, double scale,
                                           int32_t* __restrict__ err) {
  using M = StageMap<K, A>;
  extern __shared__ __align__(16) unsigned char xs_raw[];
  R* xs = reinterpret_cast<R*>(xs_raw);  // [A][P]
  for (int i = threadIdx.x; i < A * P; i += blockDim.x) xs[i] = X[i];
  __syncthreads();
  // list == nullptr: the domain is the whole range [lo_out, lo_out + stride_out)
  const int64_t cnt = list ? (int64_t)*count_ptr : stride_out;
  const int lane = threadIdx.x % LANES;
  const int64_t per_block = blockDim.x / LANES;
  const int64_t sub = threadIdx.x / LANES;
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
    for (int c = 0; c < M::NCO; ++c) acc[c][0] = acc[c][1] = zero_of<R>();
    if constexpr (std::is_same<R, dword>::value)
      stage_accumulate_dw<K, A>(xs, P, l, Tprev, lo_prev, stride_prev, lane, LANES, acc);
    else
      stage_accumulate<K, A, R>(xs, P, l, Tprev, lo_prev, stride_prev, lane, LANES, acc);
    if (LANES > 1) {
      // the LANES consecutive lanes of a group hold one point; xor offsets below LANES stay
      // inside the group (LANES divides 32 and every lane of the warp takes part)
#pragma unroll
      for (int c = 0; c < M::NCO; ++c)
#pragma unroll
        for (int f = 0; f < 2; ++f)
#pragma unroll
          for (int o = LANES / 2; o > 0; o >>= 1) {
            if constexpr (std::is_same<R, dword>::value) {
              dw_norm(acc[c][f]);
              acc[c][f] = dw_add(acc[c][f], dw_shfl_xor(acc[c][f], o));
            } else {
              acc[c][f] += __shfl_xor_sync(0xffffffffu, acc[c][f], o);
            }
          }
      if (lane != 0) continue;
    }
#pragma unroll
    for (int c = 0; c < M::NCO; ++c) {
      store_out(Tout + (2 * c + 0) * stride_out + pos, acc[c][0], scale);
      store_out(Tout + (2 * c + 1) * stride_out + pos, acc[c][1], scale);
    }
  }
}

#define LSP_STAGE_PARAMS                                                                     \
  const int32_t *__restrict__ list, const int32_t *__restrict__ count_ptr, int P,              \
      const R *__restrict__ X, const R *__restrict__ Tprev, int64_t lo_prev,                   \
      int64_t stride_prev, OUT *__restrict__ Tout, int64_t lo_out, int64_t stride_out,         \
      int by_index, double scale, int32_t *__restrict__ err
#define LSP_STAGE_ARGS \
  list, count_ptr, P, X, Tprev, lo_prev, stride_prev, Tout, lo_out, stride_out, by_index, scale, err

// Register budgets, measured at 2D n = 1024 and 3D n = 64. Four resident blocks of 256 threads
// (at most 64 registers) suit the stages whose gathers the unrolled loops keep in flight:
// FP32 stage 2 0.165 -> 0.159 ms, FP32 stage 1 -3%, double-word stages 1 and 2 -4% and -3%,
// the FP64 3D stage 3 0.020 -> 0.014 ms. The FP64 stage 1 (no gather: consecutive reads, FP64
// pipe bound) is 2% faster with the compiler's own choice (48 registers, five blocks).
template <int K, int A, typename R, typename OUT, int LANES>
__global__ void __launch_bounds__(kThreads) k_stage(LSP_STAGE_PARAMS) {
  stage_body<K, A, R, OUT, LANES>(LSP_STAGE_ARGS);
}
template <int K, int A, typename R, typename OUT, int LANES>
__global__ void __launch_bounds__(kThreads, 4) k_stage_b4(LSP_STAGE_PARAMS) {
  stage_body<K, A, R, OUT, LANES>(LSP_STAGE_ARGS);
}
#undef LSP_STAGE_PARAMS
#undef LSP_STAGE_ARGS

template <int K, int A, typename R, typename OUT, int LANES>
constexpr auto stage_kernel() {
  if constexpr (K == 1 && std::is_same<R, double>::value)
    return k_stage<K, A, R, OUT, LANES>;
  else
    return k_stage_b4<K, A, R, OUT, LANES>;
}

template <int K, int A, typename R, typename OUT, int LANES>
cudaError_t launch_kk(lsp_ctx* c, const int32_t* list, const int32_t* count, int64_t cap,
                      const R* X, const R* Tprev, int64_t lo_prev, int64_t stride_prev, OUT* Tout,
                      int64_t lo_out, int64_t stride_out, bool by_index, double scale) {
  const int P = c->geo.P;
  const size_t smem = sizeof(R) * A * P;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(stage_kernel<K, A, R, OUT, LANES>(),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  // launch shape: 256 threads and at most 16 CTAs per SM unless the autotuner found better
  // (the per-point order of the sums does not depend on it, so the results do not either)
  const std::string key = std::string("stage") + std::to_string(K) + "/A" + std::to_string(A) +
                          "/" + (sizeof(R) == 4 ? "f32" : (std::is_same<R, dword>::value ? "dw" : "f64")) +
                          "/lanes" + std::to_string(LANES) + "/w" + work_bucket(cap);
  return tuned_launch(c, key, {kThreads, 16}, kThreads, 0, [&](LaunchShape sh) {
    const int64_t per_block = sh.threads / LANES;
    int64_t b = (cap + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 152 * (int64_t)sh.per_sm) b = 152 * (int64_t)sh.per_sm;
    stage_kernel<K, A, R, OUT, LANES>()<<<(int)b, sh.threads, smem, c->stream>>>(
        list, count, P, X, Tprev, lo_prev, stride_prev, Tout, lo_out, stride_out,
        by_index ? 1 : 0, scale, (int32_t*)c->counts.p + kErrWord);
    return cudaGetLastError();
  });
}

// A domain below two threads per SM thread slot of the GPU (152 x 2048) shares each point
// among lanes: a warp per point below 152 x 256 points, four lanes per point above.
constexpr int64_t kWarpBelow = 152 * 256, kQuadBelow = 152 * 2048;

template <int K, int A, typename R, typename OUT>
cudaError_t launch_k(lsp_ctx* c, const int32_t* list, const int32_t* count, int64_t cap,
                     const R* X, const R* Tprev, int64_t lo_prev, int64_t stride_prev, OUT* Tout,
                     int64_t lo_out, int64_t stride_out, bool by_index, double scale) {
  if (cap < kWarpBelow)
    return launch_kk<K, A, R, OUT, 32>(c, list, count, cap, X, Tprev, lo_prev, stride_prev,
                                       Tout, lo_out, stride_out, by_index, scale);
  if (cap < kQuadBelow)
    return launch_kk<K, A, R, OUT, 4>(c, list, count, cap, X, Tprev, lo_prev, stride_prev, Tout,
                                      lo_out, stride_out, by_index, scale);
  return launch_kk<K, A, R, OUT, 1>(c, list, count, cap, X, Tprev, lo_prev, stride_prev, Tout,
                                    lo_out, stride_out, by_index, scale);
}

template <typename R>
cudaError_t launch_typed(lsp_ctx* c, int d, int k, int t, const int32_t* list,
                         const int32_t* count, int64_t cap, const void* Tprev, int64_t lo_prev,
                         int64_t stride_prev, void* Tout, int64_t lo_out, int64_t stride_out,
                         bool by_index, double scale, const R* X) {
  const R* prev = (const R*)Tprev;
  if constexpr (std::is_same<R, dword>::value) {
    if (t == 2) return cudaErrorInvalidValue;  // double-word stages serve t = 1 builds only
  } else if (t == 2) {  // five cosine rows (2D and 3D)
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
                         bool by_index, int prec) {
  // The final stage carries the 1/N of the inverse transform (N a power of two: exact).
  const double scale = (k == d) ? 1.0 / (double)c->geo.N : 1.0;
  static const char* names[4] = {"", "stage1", "stage2", "stage3"};
  int tm = timer_begin(c, names[k]);
  cudaError_t e;
  if (prec == kPrecFP32)
    e = launch_typed<float>(c, d, k, t, list, count, cap, Tprev, lo_prev, stride_prev, Tout,
                            lo_out, stride_out, by_index, scale, (const float*)c->xtab32.p);
  else if (prec == kPrecDword)
    e = launch_typed<dword>(c, d, k, t, list, count, cap, Tprev, lo_prev, stride_prev, Tout,
                            lo_out, stride_out, by_index, scale, (const dword*)c->xtabdw.p);
  else
    e = launch_typed<double>(c, d, k, t, list, count, cap, Tprev, lo_prev, stride_prev, Tout,
                             lo_out, stride_out, by_index, scale, (const double*)c->xtab.p);
  timer_end(c, tm);
  return e;
}

}  // namespace lsp
