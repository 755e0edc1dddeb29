// Learned stencils (a surrogate for steps a3-a6): a multilayer perceptron maps the patch of
// h^2 v around a point to its stencil coefficients (alpha, c). The paper has no learned
// component; the network is trained on the stencils of Sec. 4.1-4.2 that the FP64 path
// produces, and the eigen-solve remains its fallback and its judge.
//
//   x  = (h^2 v[j + o] - mu_x) / sigma_x  for the (2r+1)^d offsets o (r = 2), then
//        (h^2 s_j - mu_x) / sigma_x with s_j = snap(v_j), zero-padded to K0. The stencil of the
//        method depends on v_j only through the snapped shift s_j (a step function of v_j), so
//        s_j is given to the network directly; the patch lets it use the neighbourhood too.
//   z1 = x W1^T + b1, h1 = a(z1);  z2, h2;  z3, h3 (hidden width 256), a = hard-swish
//   y  = h3 W4^T + b4;  (alpha, c) = y * sigma_y + mu_y;  alpha /= |alpha|, c scaled alike
//   rows: Q = alpha, C = c, P = alpha + c .* (v[mu_j] - s_j), s_j = snap(v_j)   (Sec. 4.1)
//
// Tensor cores: every layer is a BF16 x BF16 -> FP32 tcgen05 MMA with the accumulator in
// tensor memory (M = 128 rows per tile, N = 256). A single elected thread issues the MMAs and
// the bulk copies of the weight chunks (double-buffered); the epilogue (bias, activation, bf16
// pack into the canonical shared-memory layout of the next layer's A operand) runs on eight
// warps from tcgen05.ld. Training uses the same fused forward (saving z and h),
// a generic tcgen05 TN GEMM for the backward products, and Adam.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "lsp_internal.h"
#include "tc_common.cuh"

using namespace lsp;

namespace {

constexpr int kH = 256;         // hidden width
constexpr int kTile = 128;      // rows per tile (MMA M)
constexpr int kChunkK = 64;     // K width of a GEMM staging chunk (training)
constexpr int kChunkBytes = 16384;  // bytes of a streamed weight chunk (fused kernel)
constexpr int kThreads = 128;   // GEMM kernel: 4 warps, one TMEM lane quarter each
constexpr int kFusedThreads = 288;  // fused kernel: 8 epilogue warps + 1 producer warp

struct Dims {
  int d, mu, nf, K0, OUT, OUTP;
};
Dims dims_for(int d) {
  Dims m;
  m.d = d;
  m.mu = d == 2 ? 9 : 27;
  m.nf = d == 2 ? 26 : 126;  // 5^d patch features + the snapped shift h^2 s_j
  m.K0 = d == 2 ? 32 : 128;
  m.OUT = 2 * m.mu;
  m.OUTP = d == 2 ? 32 : 64;
  return m;
}

// Flat parameter vector layout (fp32): W1 [256 x K0], b1 [256], W2 [256 x 256], b2, W3, b3,
// W4 [OUTP x 256], b4 [OUTP]; then the normalisation mu_x, sigma_x, mu_y[OUTP], sigma_y[OUTP],
// and the input range [lo, hi] of h^2 v seen in training.
struct Layout {
  int64_t w[4], b[4], wn[4], nN[4], nK[4], norm, range, total, nparams;
};
Layout layout_for(const Dims& m) {
  Layout L;
  const int N[4] = {kH, kH, kH, m.OUTP}, K[4] = {m.K0, kH, kH, kH};
  int64_t off = 0;
  for (int l = 0; l < 4; ++l) {
    L.nN[l] = N[l];
    L.nK[l] = K[l];
    L.w[l] = off;
    L.wn[l] = (int64_t)N[l] * K[l];
    off += L.wn[l];
    L.b[l] = off;
    off += N[l];
  }
  L.nparams = off;
  L.norm = off;
  off += 2 + 2 * m.OUTP;
  L.range = off;
  off += 2;
  L.total = off;
  return L;
}

// Streamed weight chunks: every layer's W [N x K] in K-slices of 16 KiB (N x kw bf16,
// canonical K-major layout), in layer order; the fused kernel double-buffers them.
struct ChunkPlan {
  int n;
  int64_t off[40];   // bytes into the tile buffer
  int kw[40];        // K width of the chunk
  int nrows[40];     // N of the chunk (= the layer's output width)
  int layer[40];
  int k0[40];
  int64_t total_bytes;
};
ChunkPlan plan_for(const Dims& m) {
  ChunkPlan p;
  p.n = 0;
  int64_t off = 0;
  const int K[4] = {m.K0, kH, kH, kH}, N[4] = {kH, kH, kH, m.OUTP};
  for (int l = 0; l < 4; ++l) {
    const int kw_max = kChunkBytes / (N[l] * 2);
    for (int k0 = 0; k0 < K[l]; k0 += kw_max) {
      const int kw = K[l] - k0 < kw_max ? K[l] - k0 : kw_max;
      p.off[p.n] = off;
      p.kw[p.n] = kw;
      p.nrows[p.n] = N[l];
      p.layer[p.n] = l;
      p.k0[p.n] = k0;
      ++p.n;
      off += (int64_t)N[l] * kw * 2;
    }
  }
  p.total_bytes = off;
  return p;
}

__device__ __forceinline__ float act(float z) {
  return z * fminf(fmaxf(z + 3.0f, 0.0f), 6.0f) * (1.0f / 6.0f);
}
__device__ __forceinline__ float act_grad(float z) {
  return z < -3.0f ? 0.0f : (z > 3.0f ? 1.0f : (2.0f * z + 3.0f) * (1.0f / 6.0f));
}

__device__ __forceinline__ int64_t snap_m(double x) {
  const double yf = fma(x, kQuarterInvPi2, -0.5);
  const double r = rint(yf);
  if (0.5 - fabs(yf - r) > 1e-14 * fabs(yf) + 1e-14) return (int64_t)r;
  const double y = __dmul_rn(__dsub_rn(__ddiv_rn(x, kPi2), 2.0), 0.25);
  return (int64_t)round(y);
}

// Linear index of j + o (periodic) for an offset o with components in [-R, R], given as
// a lexicographic index into (2R+1)^D.
template <int D, int R>
__device__ __forceinline__ int64_t nb_index(int64_t j, int o, int logn, int64_t mask) {
  constexpr int W = 2 * R + 1;
  int64_t out = 0;
  int rem = o;
  int offs[3] = {0, 0, 0};
#pragma unroll
  for (int a = D - 1; a >= 0; --a) {
    offs[a] = rem % W - R;
    rem /= W;
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int64_t xa = (j >> ((D - 1 - a) * logn)) & mask;
    out = (out << logn) | ((xa + offs[a]) & mask);
  }
  return out;
}

struct FusedParams {
  const uint8_t* tiles;  // chunk stream + W4
  const float* bias;     // flat params (fp32): biases read from here
  const float* params;
  int64_t M;
  // rows mode
  const double* v;
  const float* h2v;  // h^2 v (fp32), per point
  const float* h2s;  // h^2 s_j (fp32), per point
  int logn;
  double h2;
  double* Q;
  double* C;
  double* P;
  // batch mode
  const float* Xraw;  // [M x nf] raw features (h^2 v)
  float* Y;           // [M x OUTP] normalised outputs
  __nv_bfloat16* Hs[3];
  float* Zs[3];
  __nv_bfloat16* X16;  // [M x K0] normalised inputs (bf16), saved for the backward pass
  int* err;
  ChunkPlan plan;
  int64_t bias_off[4], norm_off;
};

constexpr int kModeRows = 0, kModeBatch = 1;

// The weight chunks are prefetched NBUF - 1 deep (6 buffers in 2D, 4 in 3D), so their L2
// latency hides behind the MMAs of earlier chunks. Warps 0-7 are the epilogue warps: warp w reads tensor-memory lanes 32 (w % 4) .. (one tile row
// per lane) and the column half w / 4; warps 0-3 also build the input tile. Warp 8 is the
// producer: its elected lane issues the weight bulk copies and the MMAs while the rest of that
// warp waits at __syncwarp, so no issuing thread shares a warp with spinning threads.
template <int D, int MODE>
__global__ void __launch_bounds__(kFusedThreads, 1) k_mlp_fused(FusedParams p) {
  constexpr int MU = D == 2 ? 9 : 27;
  constexpr int NF = D == 2 ? 26 : 126;  // patch + snapped shift
  constexpr int NP = NF - 1;
  constexpr int K0 = D == 2 ? 32 : 128;
  constexpr int OUTP = D == 2 ? 32 : 64;
  constexpr int NBUF = D == 2 ? 6 : 4;  // weight-chunk buffers (prefetch depth NBUF - 1)
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* Xs = smem;                               // 128 x K0 bf16
  uint8_t* Hs = Xs + kTile * K0 * 2;                // 128 x 256 bf16
  uint8_t* Wb = Hs + kTile * kH * 2;                // NBUF x 16 KiB
  float* bs = reinterpret_cast<float*>(Wb + NBUF * kChunkBytes);  // b1 b2 b3 (3 x 256) + b4
  float* nrm = bs + 3 * kH + OUTP;                  // mu_x sig_x mu_y[OUTP] sig_y[OUTP]
  __shared__ __align__(8) uint64_t bar_mma, bar_w[6], bar_f[6];
  __shared__ uint32_t tslot;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool producer = warp == 8;
  const int quarter_w = warp & 3;  // tensor-memory lane quarter of an epilogue warp
  const int colhalf = warp >> 2;   // 0 or 1: which half of the 256 columns
  const bool leader = producer && lane == 0;

  for (int i = tid; i < kH; i += kFusedThreads) {
    bs[i] = p.params[p.bias_off[0] + i];
    bs[kH + i] = p.params[p.bias_off[1] + i];
    bs[2 * kH + i] = p.params[p.bias_off[2] + i];
  }
  for (int i = tid; i < OUTP; i += kFusedThreads) bs[3 * kH + i] = p.params[p.bias_off[3] + i];
  for (int i = tid; i < 2 + 2 * OUTP; i += kFusedThreads) nrm[i] = p.params[p.norm_off + i];
  if (leader) {
    tc::mbar_init(&bar_mma, 1);
    for (int b = 0; b < NBUF; ++b) {
      tc::mbar_init(&bar_w[b], 1);
      tc::mbar_init(&bar_f[b], 1);
    }
    s_abort = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tslot, kH);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  // the leader's pipeline state
  uint32_t ph_w[6] = {0, 0, 0, 0, 0, 0}, ph_f[6] = {0, 0, 0, 0, 0, 0};
  bool f_pending[6] = {false, false, false, false, false, false};
  uint32_t ph_mma = 0;
  const int64_t mask = ((int64_t)1 << p.logn) - 1;
  const float mu_x = nrm[0], isig_x = 1.0f / nrm[1];

  auto issue = [&](int gi) {  // leader: bulk copy of chunk gi into buffer gi % NBUF
    const int b = gi % NBUF;
    if (f_pending[b]) {
      if (!tc::mbar_wait(&bar_f[b], ph_f[b], p.err, 2)) s_abort = 1;
      ph_f[b] ^= 1;
      f_pending[b] = false;
    }
    const uint32_t bytes = (uint32_t)p.plan.nrows[gi] * p.plan.kw[gi] * 2;
    tc::mbar_expect_tx(&bar_w[b], bytes);
    tc::bulk_g2s(Wb + b * kChunkBytes, p.tiles + p.plan.off[gi], bytes, &bar_w[b]);
  };
  // leader: MMAs of chunk gi against A = (layer 0 ? X : H) columns [k0, k0 + kw)
  auto consume = [&](int gi) {
    const int b = gi % NBUF;
    if (!tc::mbar_wait(&bar_w[b], ph_w[b], p.err, 4)) s_abort = 1;
    ph_w[b] ^= 1;
    tc::fence_after();
    const int kw = p.plan.kw[gi], k0 = p.plan.k0[gi];
    const bool first = p.plan.layer[gi] == 0;
    const uint8_t* A = first ? Xs : Hs;
    const int KA = first ? K0 : kH;
    const uint32_t sboA = (uint32_t)(KA / 8) * 128, sboB = (uint32_t)(kw / 8) * 128;
    const uint32_t aBase = tc::smem_u32(A) + (uint32_t)(k0 / 8) * 128;
    const uint32_t bBase = tc::smem_u32(Wb + b * kChunkBytes);
    const uint32_t idesc = tc::idesc_bf16(kTile, p.plan.nrows[gi]);
    for (int s = 0; s < kw / 16; ++s) {
      const uint64_t ad = tc::desc_kmajor(aBase + s * 256, 128, sboA);
      const uint64_t bd = tc::desc_kmajor(bBase + s * 256, 128, sboB);
      tc::mma_bf16(tmem, ad, bd, idesc, (k0 > 0 || s > 0) ? 1u : 0u);
    }
    tc::commit(&bar_f[b]);
    f_pending[b] = true;
  };

  const int64_t ntiles = (p.M + kTile - 1) / kTile;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    if (s_abort) break;
    const int64_t r0 = tile * kTile;
    const int64_t row = r0 + tid;  // this thread's row in the input stage
    // ---- input stage (warps 0-3): normalised features, bf16, canonical layout ----
    if (warp < 4) {
      float f[K0];
#pragma unroll
      for (int k = 0; k < K0; ++k) f[k] = 0.0f;
      if (row < p.M) {
        if (MODE == kModeRows) {
#pragma unroll 5
          for (int k = 0; k < NP; ++k)
            f[k] = (__ldg(p.h2v + nb_index<D, 2>(row, k, p.logn, mask)) - mu_x) * isig_x;
          f[NP] = (__ldg(p.h2s + row) - mu_x) * isig_x;
        } else {
          for (int k = 0; k < NF; ++k) f[k] = (p.Xraw[row * NF + k] - mu_x) * isig_x;
        }
      }
#pragma unroll
      for (int k8 = 0; k8 < K0; k8 += 8) {
        uint4 q;
        q.x = tc::pack_bf16(f[k8 + 0], f[k8 + 1]);
        q.y = tc::pack_bf16(f[k8 + 2], f[k8 + 3]);
        q.z = tc::pack_bf16(f[k8 + 4], f[k8 + 5]);
        q.w = tc::pack_bf16(f[k8 + 6], f[k8 + 7]);
        *reinterpret_cast<uint4*>(Xs + tc::kmajor_off(tid, k8, K0)) = q;
        if (MODE == kModeBatch && row < p.M)
          *reinterpret_cast<uint4*>(p.X16 + row * K0 + k8) = q;
      }
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    for (int layer = 0; layer < 4; ++layer) {
      if (leader && !s_abort) {
        if (layer == 0)
          for (int gi = 0; gi < NBUF - 1 && gi < p.plan.n; ++gi) issue(gi);
        // issue-ahead distance NBUF - 1: the buffer refilled after chunk gi is the one chunk
        // gi - 1 used, whose MMAs were committed one step earlier
        for (int gi = 0; gi < p.plan.n; ++gi) {
          if (p.plan.layer[gi] != layer) continue;
          consume(gi);
          if (gi + NBUF - 1 < p.plan.n) issue(gi + NBUF - 1);
        }
        tc::commit(&bar_mma);
      }
      if (producer) {
        __syncwarp();
      } else {
        // the epilogue warps wait for the layer's accumulator (bounded)
        if (!tc::mbar_wait(&bar_mma, ph_mma, p.err, 8)) s_abort = 1;
      }
      ph_mma ^= 1;
      tc::fence_after();
      const int trow = quarter_w * 32 + lane;  // TMEM lane = tile row
      const int64_t myrow = r0 + trow;
      const uint32_t taddr = tmem + ((uint32_t)(quarter_w * 32) << 16);
      if (producer) {
        // nothing: the producer warp waits at the barrier below
      } else if (layer < 3) {
        const float* bl = bs + layer * kH;
        for (int c0 = colhalf * (kH / 2); c0 < (colhalf + 1) * (kH / 2); c0 += 64) {
          uint32_t ra[32], rb[32];
          tc::tmem_ld32_nowait(taddr + c0, ra);
          tc::tmem_ld32_nowait(taddr + c0 + 32, rb);
          tc::ld_wait();
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            const uint32_t* r = half ? rb : ra;
            const int cb = c0 + 32 * half;
            float h[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              const float z = __uint_as_float(r[i]) + bl[cb + i];
              h[i] = act(z);
              if (MODE == kModeBatch && myrow < p.M) p.Zs[layer][myrow * kH + cb + i] = z;
            }
#pragma unroll
            for (int q8 = 0; q8 < 4; ++q8) {
              uint4 q;
              q.x = tc::pack_bf16(h[8 * q8 + 0], h[8 * q8 + 1]);
              q.y = tc::pack_bf16(h[8 * q8 + 2], h[8 * q8 + 3]);
              q.z = tc::pack_bf16(h[8 * q8 + 4], h[8 * q8 + 5]);
              q.w = tc::pack_bf16(h[8 * q8 + 6], h[8 * q8 + 7]);
              *reinterpret_cast<uint4*>(Hs + tc::kmajor_off(trow, cb + 8 * q8, kH)) = q;
              if (MODE == kModeBatch && myrow < p.M)
                *reinterpret_cast<uint4*>(p.Hs[layer] + myrow * kH + cb + 8 * q8) = q;
            }
          }
        }
      } else if (colhalf == 0) {
        float y[OUTP];
#pragma unroll
        for (int c0 = 0; c0 < OUTP; c0 += 16) {
          float a[16];
          tc::tmem_ld16(taddr + c0, a);
#pragma unroll
          for (int i = 0; i < 16; ++i) y[c0 + i] = a[i] + bs[3 * kH + c0 + i];
        }
        if (myrow < p.M) {
          if (MODE == kModeBatch) {
#pragma unroll
            for (int o = 0; o < OUTP; ++o) p.Y[myrow * OUTP + o] = y[o];
          } else {
            // de-normalise, unit-normalise alpha (c scaled alike: P^-1 C is invariant); the
            // network's precision is fp32, the difference v - s_j is taken in fp64
            float al[MU], cc[MU], nrm2 = 0.0f;
#pragma unroll
            for (int i = 0; i < MU; ++i) {
              al[i] = y[i] * nrm[2 + OUTP + i] + nrm[2 + i];
              cc[i] = y[MU + i] * nrm[2 + OUTP + MU + i] + nrm[2 + MU + i];
              nrm2 = fmaf(al[i], al[i], nrm2);
            }
            const float sc = nrm2 > 0.0f ? rsqrtf(nrm2) : 1.0f;
            const double s = __dmul_rn((double)(4 * snap_m(__ldg(p.v + myrow)) + 2), kPi2);
#pragma unroll
            for (int i = 0; i < MU; ++i) {
              constexpr int R = 1;
              const double vn = __ldg(p.v + nb_index<D, R>(myrow, i, p.logn, mask));
              const float a_ = al[i] * sc, c_ = cc[i] * sc;
              __stcs(p.Q + myrow * MU + i, (double)a_);
              __stcs(p.C + myrow * MU + i, (double)c_);
              __stcs(p.P + myrow * MU + i, (double)fmaf(c_, (float)(vn - s), a_));
            }
          }
        }
      }
      tc::fence_async_smem();
      tc::fence_before();
      __syncthreads();
      tc::fence_after();
    }
  }
  // drain: the last chunks' completion barriers (already complete unless aborted)
  if (leader && !s_abort) {
    for (int b = 0; b < NBUF; ++b)
      if (f_pending[b]) tc::mbar_wait(&bar_f[b], ph_f[b], p.err, 2);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kH);
}

// ---- generic C[M x N] (fp32) = A[M x K] B[N x K]^T, bf16 row-major operands ---------------
// M % 128 == 0, N % 16 == 0, K % 16 == 0. One CTA per 128 x min(N, 256) tile; K in chunks of
// up to 64 staged in the canonical layout; one elected thread issues the MMAs.
__global__ void __launch_bounds__(128, 1) k_gemm_tn(const __nv_bfloat16* __restrict__ A,
                                                    const __nv_bfloat16* __restrict__ B,
                                                    float* __restrict__ Cm, int M, int N, int K,
                                                    int* err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int NT_MAX = 256;
  uint8_t* As = smem;                    // 128 x 64
  uint8_t* Bs = smem + 128 * kChunkK * 2;  // 256 x 64
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * NT_MAX;
  const int NT = (N - n0) < NT_MAX ? (N - n0) : NT_MAX;
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    s_abort = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tslot, NT_MAX);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  uint32_t ph = 0;
  for (int k0 = 0; k0 < K; k0 += kChunkK) {
    const int kw = (K - k0) < kChunkK ? (K - k0) : kChunkK;
    const int seg = kw / 8;  // 16-byte segments per row
    for (int e = tid; e < 128 * seg; e += 128) {
      const int r = e / seg, s8 = (e % seg) * 8;
      const uint4 q = *reinterpret_cast<const uint4*>(A + (int64_t)(m0 + r) * K + k0 + s8);
      *reinterpret_cast<uint4*>(As + tc::kmajor_off(r, s8, kw)) = q;
    }
    for (int e = tid; e < NT * seg; e += 128) {
      const int r = e / seg, s8 = (e % seg) * 8;
      const uint4 q = *reinterpret_cast<const uint4*>(B + (int64_t)(n0 + r) * K + k0 + s8);
      *reinterpret_cast<uint4*>(Bs + tc::kmajor_off(r, s8, kw)) = q;
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0 && !s_abort) {
      const uint32_t sbo = (uint32_t)(kw / 8) * 128;
      for (int s = 0; s < kw / 16; ++s) {
        const uint64_t ad = tc::desc_kmajor(tc::smem_u32(As) + s * 256, 128, sbo);
        const uint64_t bd = tc::desc_kmajor(tc::smem_u32(Bs) + s * 256, 128, sbo);
        tc::mma_bf16(tmem, ad, bd, tc::idesc_bf16(128, NT), (k0 > 0 || s > 0) ? 1u : 0u);
      }
      tc::commit(&bar);
      if (!tc::mbar_wait(&bar, ph, err, 16)) s_abort = 1;
    }
    ph ^= 1;
    tc::fence_before();
    __syncthreads();  // the staging buffers are free again
    tc::fence_after();
    if (s_abort) break;
  }
  if (!s_abort) {
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    const int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < NT; c0 += 16) {
      float a[16];
      tc::tmem_ld16(taddr + c0, a);
#pragma unroll
      for (int i = 0; i < 16; ++i) Cm[(int64_t)row * N + n0 + c0 + i] = a[i];
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, NT_MAX);
}

// ---- elementwise kernels of the training step ----------------------------------------------
// dY = 2 (y - t_norm) / (B * OUT) on the OUT real outputs (0 on padding), bf16 row-major and
// transposed ([128 x B], rows >= OUT zero); loss partial sums in double.
__global__ void k_loss_grad(const float* __restrict__ Y, const float* __restrict__ Traw,
                            const float* __restrict__ params, int64_t norm_off, int64_t B,
                            int OUT, int OUTP, __nv_bfloat16* __restrict__ dY,
                            __nv_bfloat16* __restrict__ dYT, float* __restrict__ dY32,
                            double* __restrict__ loss) {
  double acc = 0.0;
  const double scale = 2.0 / ((double)B * OUT);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < B * OUTP;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / OUTP;
    const int o = (int)(e - b * OUTP);
    float g = 0.0f;
    if (o < OUT) {
      const float mu = params[norm_off + 2 + o], sg = params[norm_off + 2 + OUTP + o];
      const float t = (Traw[b * OUT + o] - mu) / sg;
      const float r = Y[e] - t;
      acc += (double)r * r;
      g = (float)(scale * r);
    }
    dY[e] = __float2bfloat16(g);
    dY32[e] = g;
    dYT[(int64_t)o * B + b] = __float2bfloat16(g);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// dZ = dH * a'(Z) (fp32 in), bf16 row-major and transposed copies.
__global__ void k_silu_back(const float* __restrict__ dH, const float* __restrict__ Z, int64_t B,
                            __nv_bfloat16* __restrict__ dZ, __nv_bfloat16* __restrict__ dZT,
                            float* __restrict__ dZ32) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < B * kH;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / kH;
    const int k = (int)(e - b * kH);
    const float g = dH[e] * act_grad(Z[e]);
    dZ[e] = __float2bfloat16(g);
    dZ32[e] = g;
    dZT[(int64_t)k * B + b] = __float2bfloat16(g);
  }
}

// Column sums of a [B x N] fp32 matrix (bias gradients), one thread per column.
__global__ void k_colsum(const float* __restrict__ G, int64_t B, int N, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  double s = 0.0;
  for (int64_t b = 0; b < B; ++b) s += G[b * N + c];
  out[c] = (float)s;
}

// out[c][r] = in[r][c] for a [R x Cn] bf16 matrix.
__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ in, int64_t R, int Cn,
                                 __nv_bfloat16* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < R * Cn;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / Cn;
    const int c = (int)(e - r * Cn);
    out[(int64_t)c * R + r] = in[e];
  }
}

// Adam on the flat parameter vector (gradients already in g).
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// bf16 copies of the weights: the chunk stream of the fused kernel (canonical K-major tiles)
// and transposed row-major copies W^T [K x N] for the backward products.
__global__ void k_retile(const float* __restrict__ params, Layout L, ChunkPlan plan, int OUTP,
                         uint8_t* __restrict__ tiles, __nv_bfloat16* __restrict__ WT0,
                         __nv_bfloat16* __restrict__ WT1, __nv_bfloat16* __restrict__ WT2,
                         __nv_bfloat16* __restrict__ WT3, __nv_bfloat16* __restrict__ W16_0,
                         __nv_bfloat16* __restrict__ W16_1, __nv_bfloat16* __restrict__ W16_2,
                         __nv_bfloat16* __restrict__ W16_3) {
  __nv_bfloat16* WT[4] = {WT0, WT1, WT2, WT3};
  __nv_bfloat16* W16[4] = {W16_0, W16_1, W16_2, W16_3};
  for (int l = 0; l < 4; ++l) {
    const int N = (int)L.nN[l], K = (int)L.nK[l];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)N * K;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int n = (int)(e / K), k = (int)(e % K);
      const __nv_bfloat16 x = __float2bfloat16(params[L.w[l] + e]);
      WT[l][(int64_t)k * N + n] = x;
      W16[l][e] = x;
      int gi = 0;
      for (int q = 0; q < plan.n; ++q)
        if (plan.layer[q] == l && k >= plan.k0[q] && k < plan.k0[q] + plan.kw[q]) gi = q;
      *reinterpret_cast<__nv_bfloat16*>(tiles + plan.off[gi] +
                                        tc::kmajor_off(n, k - plan.k0[gi], plan.kw[gi])) = x;
    }
  }
}

// Normalisation statistics: mean and standard deviation of all raw features (one pair) and of
// every output column.
__global__ void k_norm_stats(const float* __restrict__ X, const float* __restrict__ T, int64_t B,
                             int NF, int OUT, int OUTP, float* __restrict__ params,
                             int64_t norm_off, int64_t range_off) {
  // one block: thread 0..OUT-1 columns of T, the last warp does X
  const int t = threadIdx.x;
  if (t < OUT) {
    double s = 0, s2 = 0;
    for (int64_t b = 0; b < B; ++b) {
      const double x = T[b * OUT + t];
      s += x;
      s2 += x * x;
    }
    const double mu = s / B, var = fmax(s2 / B - mu * mu, 0.0);
    params[norm_off + 2 + t] = (float)mu;
    params[norm_off + 2 + OUTP + t] = (float)fmax(sqrt(var), 1e-30);
  } else if (t < OUTP) {
    params[norm_off + 2 + t] = 0.0f;
    params[norm_off + 2 + OUTP + t] = 1.0f;
  }
  if (t == blockDim.x - 1) {
    double s = 0, s2 = 0, lo = 1e300, hi = -1e300;
    for (int64_t e = 0; e < B * NF; ++e) {
      const double x = X[e];
      s += x;
      s2 += x * x;
      lo = fmin(lo, x);
      hi = fmax(hi, x);
    }
    const double n = (double)B * NF;
    const double mu = s / n, var = fmax(s2 / n - mu * mu, 0.0);
    params[norm_off + 0] = (float)mu;
    params[norm_off + 1] = (float)fmax(sqrt(var), 1e-30);
    params[range_off + 0] = (float)lo;
    params[range_off + 1] = (float)hi;
  }
}

// Per point, fp32 h^2 v and h^2 s_j (s_j = snap(v_j)): the learned build's inputs.
__global__ void k_prep_inputs(const double* __restrict__ v, int64_t N, double h2,
                              float* __restrict__ h2v, float* __restrict__ h2s) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x) {
    const double x = v[j];
    h2v[j] = (float)(x * h2);
    h2s[j] = (float)(__dmul_rn((double)(4 * snap_m(x) + 2), kPi2) * h2);
  }
}

// Training pairs from a context's last eigen-path build: raw patch features of random points
// and their (alpha, c) targets. The random point of sample i is a hash of (seed, i).
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdULL;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ULL;
  x ^= x >> 33;
  return x;
}
template <int D>
__global__ void k_pairs(const double* __restrict__ v, int64_t N, int logn, double h2,
                        const double* __restrict__ Qr, const double* __restrict__ Cr,
                        int64_t nsamples, uint64_t seed, float* __restrict__ X,
                        float* __restrict__ T) {
  constexpr int MU = D == 2 ? 9 : 27;
  constexpr int NF = D == 2 ? 26 : 126;
  const int64_t mask = ((int64_t)1 << logn) - 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nsamples;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = (int64_t)(mix64(seed * 0x9E3779B97F4A7C15ULL + (uint64_t)i) % (uint64_t)N);
    for (int k = 0; k < NF - 1; ++k)
      X[i * NF + k] = (float)(v[nb_index<D, 2>(j, k, logn, mask)] * h2);
    const double sj = __dmul_rn((double)(4 * snap_m(v[j]) + 2), kPi2);
    X[i * NF + NF - 1] = (float)(sj * h2);
    for (int a = 0; a < MU; ++a) {
      T[i * 2 * MU + a] = (float)Qr[j * MU + a];
      T[i * 2 * MU + MU + a] = (float)Cr[j * MU + a];
    }
  }
}

}  // namespace

// ---- host side ------------------------------------------------------------------------------

struct lsp_mlp {
  Dims dm;
  Layout L;
  ChunkPlan plan;
  cudaStream_t stream = nullptr;
  std::string err;
  lsp::DevBuf params, grads, adam_m, adam_v, tiles, WT[4], W16[4], errflag, loss;
  // training workspace
  int64_t cap = 0;
  lsp::DevBuf X16, XT, Zs[3], Hs[3], HT[3], Y, dY16, dYT, dY32, G, dZ16, dZT, dZ32;
  int64_t step = 0;
};

namespace {

lsp_status mfail(lsp_mlp* m, lsp_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (m) m->err = buf;
  return st;
}
#define MCUDA(m, expr)                                                                    \
  do {                                                                                    \
    cudaError_t _e = (expr);                                                              \
    if (_e != cudaSuccess)                                                                \
      return mfail(m, _e == cudaErrorMemoryAllocation ? LSP_ERR_OOM : LSP_ERR_CUDA,       \
                   "%s failed: %s", #expr, cudaGetErrorString(_e));                       \
  } while (0)

bool grow(lsp::DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes) return true;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  b.bytes = bytes;
  return true;
}

size_t fused_smem(int d) {
  const Dims m = dims_for(d);
  const int nbuf = d == 2 ? 6 : 4;
  return (size_t)kTile * m.K0 * 2 + kTile * kH * 2 + (size_t)nbuf * kChunkBytes +
         sizeof(float) * (3 * kH + m.OUTP + 2 + 2 * m.OUTP) + 64;
}

FusedParams fused_params(lsp_mlp* m) {
  FusedParams p;
  memset(&p, 0, sizeof p);
  p.tiles = (const uint8_t*)m->tiles.p;
  p.params = (const float*)m->params.p;
  p.plan = m->plan;
  for (int l = 0; l < 4; ++l) p.bias_off[l] = m->L.b[l];
  p.norm_off = m->L.norm;
  p.err = (int*)m->errflag.p;
  return p;
}

template <int D, int MODE>
cudaError_t launch_fused(lsp_mlp* m, const FusedParams& p, int64_t rows) {
  const size_t smem = fused_smem(D);
  cudaError_t e = cudaFuncSetAttribute(k_mlp_fused<D, MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int64_t tiles = (rows + kTile - 1) / kTile;
  // two CTAs per SM where the shared memory allows (2D)
  const int per_sm = smem <= 110 * 1024 ? 2 : 1;
  int grid = (int)(tiles < 152 * per_sm ? tiles : 152 * per_sm);
  if (grid < 1) grid = 1;
  k_mlp_fused<D, MODE><<<grid, kFusedThreads, smem, m->stream>>>(p);
  return cudaGetLastError();
}

lsp_status retile(lsp_mlp* m) {
  k_retile<<<152 * 4, 256, 0, m->stream>>>(
      (const float*)m->params.p, m->L, m->plan, m->dm.OUTP, (uint8_t*)m->tiles.p,
      (__nv_bfloat16*)m->WT[0].p, (__nv_bfloat16*)m->WT[1].p, (__nv_bfloat16*)m->WT[2].p,
      (__nv_bfloat16*)m->WT[3].p, (__nv_bfloat16*)m->W16[0].p, (__nv_bfloat16*)m->W16[1].p,
      (__nv_bfloat16*)m->W16[2].p, (__nv_bfloat16*)m->W16[3].p);
  MCUDA(m, cudaGetLastError());
  return LSP_OK;
}

lsp_status check_err(lsp_mlp* m) {
  int e = 0;
  MCUDA(m, cudaMemcpyAsync(&e, m->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  MCUDA(m, cudaStreamSynchronize(m->stream));
  if (e) return mfail(m, LSP_ERR_TIMEOUT, "a tensor-core wait gave up (bits %d)", e);
  return LSP_OK;
}

lsp_status ensure_workspace(lsp_mlp* m, int64_t B) {
  if (m->cap >= B) return LSP_OK;
  const Dims& d = m->dm;
  bool ok = grow(m->X16, sizeof(__nv_bfloat16) * B * d.K0) &&
            grow(m->XT, sizeof(__nv_bfloat16) * B * d.K0) && grow(m->Y, sizeof(float) * B * d.OUTP) &&
            grow(m->dY16, sizeof(__nv_bfloat16) * B * d.OUTP) &&
            grow(m->dYT, sizeof(__nv_bfloat16) * B * 128) &&
            grow(m->dY32, sizeof(float) * B * d.OUTP) && grow(m->G, sizeof(float) * B * kH) &&
            grow(m->dZ16, sizeof(__nv_bfloat16) * B * kH) &&
            grow(m->dZT, sizeof(__nv_bfloat16) * B * kH) && grow(m->dZ32, sizeof(float) * B * kH);
  for (int l = 0; ok && l < 3; ++l)
    ok = grow(m->Zs[l], sizeof(float) * B * kH) && grow(m->Hs[l], sizeof(__nv_bfloat16) * B * kH) &&
         grow(m->HT[l], sizeof(__nv_bfloat16) * B * kH);
  if (!ok) return mfail(m, LSP_ERR_OOM, "training workspace allocation failed");
  m->cap = B;
  return LSP_OK;
}

cudaError_t gemm(lsp_mlp* m, const void* A, const void* B, float* C, int M, int N, int K) {
  // 48 KiB of staging is enough; asking for 100 KiB keeps at most two CTAs per SM, so their two
  // 256-column tensor-memory allocations always fit in the SM's 512 columns.
  const size_t smem = 100 * 1024;
  cudaError_t e =
      cudaFuncSetAttribute(k_gemm_tn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(M / 128, (N + 255) / 256);
  k_gemm_tn<<<grid, 128, smem, m->stream>>>((const __nv_bfloat16*)A, (const __nv_bfloat16*)B, C, M,
                                            N, K, (int*)m->errflag.p);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

lsp_status lsp_mlp_create(int d, uint64_t seed, void* cuda_stream, lsp_mlp** out) {
  if (!out || (d != 2 && d != 3)) return LSP_ERR_ARG;
  *out = nullptr;
  lsp_mlp* m = new (std::nothrow) lsp_mlp();
  if (!m) return LSP_ERR_OOM;
  m->dm = dims_for(d);
  m->L = layout_for(m->dm);
  m->plan = plan_for(m->dm);
  m->stream = (cudaStream_t)cuda_stream;
  const int64_t P = m->L.total;
  bool ok = grow(m->params, sizeof(float) * P) && grow(m->grads, sizeof(float) * P) &&
            grow(m->adam_m, sizeof(float) * P) && grow(m->adam_v, sizeof(float) * P) &&
            grow(m->tiles, (size_t)m->plan.total_bytes) && grow(m->errflag, 64) &&
            grow(m->loss, 64);
  for (int l = 0; ok && l < 4; ++l)
    ok = grow(m->WT[l], sizeof(__nv_bfloat16) * m->L.wn[l]) &&
         grow(m->W16[l], sizeof(__nv_bfloat16) * m->L.wn[l]);
  if (!ok) {
    lsp_mlp_destroy(m);
    return LSP_ERR_OOM;
  }
  // He-style initialisation (uniform, scale sqrt(6 / fan_in) / 2), zero biases, identity
  // normalisation; padded outputs and padded inputs get zero weights.
  std::vector<float> h(P, 0.0f);
  uint64_t s = seed * 0x9E3779B97F4A7C15ULL + 12345;
  auto uni = [&]() {
    s ^= s << 13;
    s ^= s >> 7;
    s ^= s << 17;
    return (double)(s >> 11) / 9007199254740992.0;
  };
  const Dims& dm = m->dm;
  for (int l = 0; l < 4; ++l) {
    const int N = (int)m->L.nN[l], K = (int)m->L.nK[l];
    const int fan_in = l == 0 ? dm.nf : K;
    const double a = sqrt(6.0 / fan_in) * (l == 3 ? 0.25 : 1.0);
    for (int n = 0; n < N; ++n)
      for (int k = 0; k < K; ++k) {
        const bool live = !(l == 0 && k >= dm.nf) && !(l == 3 && n >= dm.OUT);
        h[m->L.w[l] + (int64_t)n * K + k] = live ? (float)((2 * uni() - 1) * a) : 0.0f;
      }
  }
  h[m->L.norm + 1] = 1.0f;
  for (int o = 0; o < dm.OUTP; ++o) h[m->L.norm + 2 + dm.OUTP + o] = 1.0f;
  h[m->L.range + 0] = -1e30f;
  h[m->L.range + 1] = 1e30f;
  lsp_status st = LSP_OK;
  if (cudaMemcpy(m->params.p, h.data(), sizeof(float) * P, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(m->adam_m.p, 0, sizeof(float) * P) != cudaSuccess ||
      cudaMemset(m->adam_v.p, 0, sizeof(float) * P) != cudaSuccess ||
      cudaMemset(m->tiles.p, 0, m->plan.total_bytes) != cudaSuccess ||
      cudaMemset(m->errflag.p, 0, 64) != cudaSuccess)
    st = LSP_ERR_CUDA;
  if (st == LSP_OK) st = retile(m);
  if (st == LSP_OK && cudaStreamSynchronize(m->stream) != cudaSuccess) st = LSP_ERR_CUDA;
  if (st != LSP_OK) {
    lsp_mlp_destroy(m);
    return st;
  }
  *out = m;
  return LSP_OK;
}

lsp_status lsp_mlp_destroy(lsp_mlp* m) {
  if (!m) return LSP_OK;
  cudaStreamSynchronize(m->stream);
  lsp::DevBuf* bufs[] = {&m->params, &m->grads, &m->adam_m, &m->adam_v, &m->tiles, &m->errflag,
                         &m->loss, &m->X16, &m->XT, &m->Y, &m->dY16, &m->dYT, &m->dY32, &m->G,
                         &m->dZ16, &m->dZT, &m->dZ32};
  for (auto* b : bufs)
    if (b->p) cudaFree(b->p);
  for (int l = 0; l < 4; ++l) {
    if (m->WT[l].p) cudaFree(m->WT[l].p);
    if (m->W16[l].p) cudaFree(m->W16[l].p);
  }
  for (int l = 0; l < 3; ++l) {
    if (m->Zs[l].p) cudaFree(m->Zs[l].p);
    if (m->Hs[l].p) cudaFree(m->Hs[l].p);
    if (m->HT[l].p) cudaFree(m->HT[l].p);
  }
  delete m;
  return LSP_OK;
}

lsp_status lsp_mlp_param_count(const lsp_mlp* m, int64_t* total, int64_t* nweights) {
  if (!m) return LSP_ERR_ARG;
  if (total) *total = m->L.total;
  if (nweights) *nweights = m->L.nparams;
  return LSP_OK;
}

lsp_status lsp_mlp_get_params(lsp_mlp* m, float* host) {
  if (!m || !host) return LSP_ERR_ARG;
  MCUDA(m, cudaMemcpyAsync(host, m->params.p, sizeof(float) * m->L.total, cudaMemcpyDeviceToHost,
                           m->stream));
  MCUDA(m, cudaStreamSynchronize(m->stream));
  return LSP_OK;
}

lsp_status lsp_mlp_set_params(lsp_mlp* m, const float* host) {
  if (!m || !host) return LSP_ERR_ARG;
  MCUDA(m, cudaMemcpyAsync(m->params.p, host, sizeof(float) * m->L.total, cudaMemcpyHostToDevice,
                           m->stream));
  lsp_status st = retile(m);
  if (st != LSP_OK) return st;
  MCUDA(m, cudaStreamSynchronize(m->stream));
  return LSP_OK;
}

lsp_status lsp_mlp_fit_normalization(lsp_mlp* m, const float* X_dev, const float* T_dev,
                                     int64_t n) {
  if (!m || !X_dev || !T_dev || n < 2) return LSP_ERR_ARG;
  cudaGetLastError();
  k_norm_stats<<<1, 128, 0, m->stream>>>(X_dev, T_dev, n, m->dm.nf, m->dm.OUT, m->dm.OUTP,
                                         (float*)m->params.p, m->L.norm, m->L.range);
  MCUDA(m, cudaGetLastError());
  MCUDA(m, cudaStreamSynchronize(m->stream));
  return LSP_OK;
}

lsp_status lsp_mlp_forward(lsp_mlp* m, const float* X_dev, int64_t batch, float* Y_dev) {
  if (!m || !X_dev || !Y_dev || batch < 1) return LSP_ERR_ARG;
  cudaGetLastError();
  const int64_t B = (batch + 127) / 128 * 128;
  lsp_status st = ensure_workspace(m, B);
  if (st != LSP_OK) return st;
  FusedParams p = fused_params(m);
  p.M = batch;
  p.Xraw = X_dev;
  p.Y = Y_dev;
  p.X16 = (__nv_bfloat16*)m->X16.p;
  for (int l = 0; l < 3; ++l) {
    p.Zs[l] = (float*)m->Zs[l].p;
    p.Hs[l] = (__nv_bfloat16*)m->Hs[l].p;
  }
  {
    const cudaError_t e = m->dm.d == 2 ? launch_fused<2, kModeBatch>(m, p, batch)
                                       : launch_fused<3, kModeBatch>(m, p, batch);
    MCUDA(m, e);
  }
  return check_err(m);
}

lsp_status lsp_mlp_train_step(lsp_mlp* m, const float* X_dev, const float* T_dev, int64_t batch,
                              float lr, int apply, float* loss_out, float* grads_host) {
  if (!m || !X_dev || !T_dev || batch < 128 || batch % 128 != 0) return LSP_ERR_ARG;
  cudaGetLastError();
  const Dims& d = m->dm;
  const Layout& L = m->L;
  lsp_status st = ensure_workspace(m, batch);
  if (st != LSP_OK) return st;
  // forward (saves z, h, and the normalised bf16 inputs)
  FusedParams p = fused_params(m);
  p.M = batch;
  p.Xraw = X_dev;
  p.Y = (float*)m->Y.p;
  p.X16 = (__nv_bfloat16*)m->X16.p;
  for (int l = 0; l < 3; ++l) {
    p.Zs[l] = (float*)m->Zs[l].p;
    p.Hs[l] = (__nv_bfloat16*)m->Hs[l].p;
  }
  {
    const cudaError_t e = d.d == 2 ? launch_fused<2, kModeBatch>(m, p, batch)
                                   : launch_fused<3, kModeBatch>(m, p, batch);
    MCUDA(m, e);
  }
  // loss and dY
  MCUDA(m, cudaMemsetAsync(m->loss.p, 0, sizeof(double), m->stream));
  MCUDA(m, cudaMemsetAsync(m->dYT.p, 0, sizeof(__nv_bfloat16) * 128 * batch, m->stream));
  k_loss_grad<<<152 * 4, 256, 0, m->stream>>>(
      (const float*)m->Y.p, T_dev, (const float*)m->params.p, L.norm, batch, d.OUT, d.OUTP,
      (__nv_bfloat16*)m->dY16.p, (__nv_bfloat16*)m->dYT.p, (float*)m->dY32.p,
      (double*)m->loss.p);
  MCUDA(m, cudaGetLastError());
  float* g = (float*)m->grads.p;
  MCUDA(m, cudaMemsetAsync(g, 0, sizeof(float) * L.total, m->stream));
  // layer 4: dW4 = dY^T h3 (M padded to 128), db4 = colsum(dY), dH3 = dY W4
  for (int l = 0; l < 3; ++l)
    k_transpose_bf16<<<152 * 4, 256, 0, m->stream>>>((const __nv_bfloat16*)m->Hs[l].p, batch, kH,
                                                     (__nv_bfloat16*)m->HT[l].p);
  k_transpose_bf16<<<152 * 4, 256, 0, m->stream>>>((const __nv_bfloat16*)m->X16.p, batch, d.K0,
                                                   (__nv_bfloat16*)m->XT.p);
  float* G = (float*)m->G.p;  // [>= 128 x 256] scratch for weight gradients / [B x 256] for dH
  MCUDA(m, gemm(m, m->dYT.p, m->HT[2].p, G, 128, kH, (int)batch));
  MCUDA(m, cudaMemcpyAsync(g + L.w[3], G, sizeof(float) * d.OUTP * kH, cudaMemcpyDeviceToDevice,
                           m->stream));
  k_colsum<<<1, 128, 0, m->stream>>>((const float*)m->dY32.p, batch, d.OUTP, g + L.b[3]);
  // dH3 = dY W4: A = dY [B x OUTP], B-operand = W4^T [256 x OUTP]
  MCUDA(m, gemm(m, m->dY16.p, m->WT[3].p, G, (int)batch, kH, d.OUTP));
  for (int l = 2; l >= 0; --l) {
    k_silu_back<<<152 * 4, 256, 0, m->stream>>>(G, (const float*)m->Zs[l].p, batch,
                                                (__nv_bfloat16*)m->dZ16.p,
                                                (__nv_bfloat16*)m->dZT.p, (float*)m->dZ32.p);
    MCUDA(m, cudaGetLastError());
    k_colsum<<<2, 128, 0, m->stream>>>((const float*)m->dZ32.p, batch, kH, g + L.b[l]);
    // dW_l = dZ^T a_{l-1}: A = dZ^T [256 x B], B-operand = a_{l-1}^T [K_l x B]
    const void* prevT = l == 0 ? m->XT.p : m->HT[l - 1].p;
    const int Kl = (int)L.nK[l];
    MCUDA(m, gemm(m, m->dZT.p, prevT, g + L.w[l], kH, Kl, (int)batch));
    if (l > 0) {
      // dH_{l-1} = dZ W_l: A = dZ [B x 256], B-operand = W_l^T [256 x 256]
      MCUDA(m, gemm(m, m->dZ16.p, m->WT[l].p, G, (int)batch, kH, kH));
    }
  }
  double loss = 0;
  MCUDA(m, cudaMemcpyAsync(&loss, m->loss.p, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  st = check_err(m);
  if (st != LSP_OK) return st;
  if (loss_out) *loss_out = (float)(loss / ((double)batch * d.OUT));
  if (grads_host)
    MCUDA(m, cudaMemcpy(grads_host, g, sizeof(float) * L.nparams, cudaMemcpyDeviceToHost));
  if (apply) {
    ++m->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)m->step), c2 = 1.0f - powf(b2, (float)m->step);
    k_adam<<<152 * 4, 256, 0, m->stream>>>((float*)m->params.p, g, (float*)m->adam_m.p,
                                           (float*)m->adam_v.p, L.nparams, lr, b1, b2, 1e-8f, c1,
                                           c2);
    MCUDA(m, cudaGetLastError());
    st = retile(m);
    if (st != LSP_OK) return st;
  }
  return LSP_OK;
}

lsp_status lsp_mlp_training_pairs(lsp_ctx* c, lsp_mlp* m, int64_t nsamples, uint64_t seed,
                                  float* X_dev, float* T_dev) {
  if (!c || !m || !X_dev || !T_dev || nsamples < 1) return LSP_ERR_ARG;
  if (!c->built || c->built_learned) return mfail(m, LSP_ERR_STATE, "no eigen-path build in ctx");
  if (c->geo.d != m->dm.d) return mfail(m, LSP_ERR_ARG, "dimension mismatch");
  cudaGetLastError();
  int logn = 0;
  while ((1 << logn) < c->geo.n) ++logn;
  const double h2 = 1.0 / ((double)c->geo.n * c->geo.n);
  if (c->geo.d == 2)
    k_pairs<2><<<152 * 4, 256, 0, c->stream>>>((const double*)c->v.p, c->geo.N, logn, h2,
                                                (const double*)c->Q.p, (const double*)c->C.p,
                                                nsamples, seed, X_dev, T_dev);
  else
    k_pairs<3><<<152 * 4, 256, 0, c->stream>>>((const double*)c->v.p, c->geo.N, logn, h2,
                                                (const double*)c->Q.p, (const double*)c->C.p,
                                                nsamples, seed, X_dev, T_dev);
  MCUDA(m, cudaGetLastError());
  MCUDA(m, cudaStreamSynchronize(c->stream));
  return LSP_OK;
}

const char* lsp_mlp_last_error(const lsp_mlp* m) { return m ? m->err.c_str() : "null network"; }

}  // extern "C"

namespace lsp {

// Learned build: the fused network over every point writes Q, C and P directly.
cudaError_t launch_learned_rows(lsp_ctx* c, lsp_mlp* m) {
  // the weights may still be written by the network's own stream (training, set_params)
  cudaError_t se = cudaStreamSynchronize(m->stream);
  if (se != cudaSuccess) return se;
  FusedParams p = fused_params(m);
  p.M = c->geo.N;
  p.v = (const double*)c->v.p;
  int logn = 0;
  while ((1 << logn) < c->geo.n) ++logn;
  p.logn = logn;
  p.h2 = 1.0 / ((double)c->geo.n * c->geo.n);
  p.Q = (double*)c->Q.p;
  p.C = (double*)c->C.p;
  p.P = (double*)c->P.p;
  p.err = (int*)c->counts.p + kErrWord;
  if (!ensure(c, c->learn_in, sizeof(float) * 2 * c->geo.N)) return cudaErrorMemoryAllocation;
  p.h2v = (const float*)c->learn_in.p;
  p.h2s = (const float*)c->learn_in.p + c->geo.N;
  cudaStream_t saved = m->stream;
  m->stream = c->stream;
  int t0 = timer_begin(c, "mlp_prep");
  k_prep_inputs<<<152 * 8, 256, 0, c->stream>>>((const double*)c->v.p, c->geo.N, p.h2,
                                                (float*)c->learn_in.p,
                                                (float*)c->learn_in.p + c->geo.N);
  timer_end(c, t0);
  int t = timer_begin(c, "mlp_rows");
  cudaError_t e = c->geo.d == 2 ? launch_fused<2, kModeRows>(m, p, c->geo.N)
                                : launch_fused<3, kModeRows>(m, p, c->geo.N);
  timer_end(c, t);
  m->stream = saved;
  return e;
}

bool mlp_input_range(lsp_mlp* m, float* lo, float* hi) {
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return false;
  float r[2];
  if (cudaMemcpy(r, (const float*)m->params.p + m->L.range, sizeof r, cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return false;
  *lo = r[0];
  *hi = r[1];
  return true;
}

int mlp_dim(const lsp_mlp* m) { return m->dm.d; }

cudaError_t mlp_sync(lsp_mlp* m) { return cudaStreamSynchronize(m->stream); }

}  // namespace lsp
