// Learned stencils (a surrogate for steps a3-a6): a multilayer perceptron maps the patch of
// h^2 v around a point to its stencil coefficients (alpha, c). The paper has no learned
// component; the network is trained on the stencils of Sec. 4.1-4.2 that the FP64 path
// produces, and the eigen-solve remains its fallback and its judge.
//
//   x  = (h^2 v[j + o] - mu_x) / sigma_x  for the (2r+1)^d offsets o (r = 2), then
//        (h^2 s_j - mu_x) / sigma_x with s_j = snap(v_j), zero-padded to K0. The stencil of the
//        method depends on v_j only through the snapped shift s_j (a step function of v_j), so
//        s_j is given to the network directly; the patch lets it use the neighbourhood too.
//   z1 = x W1^T + b1, h1 = a(z1);  z2, h2;  z3, h3 (hidden width 256), a = ReLU
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
// Largest streamed weight chunk of the inference kernels. The weights are packed chunk by chunk
// (plan_for); a chunk of an N-wide layer covers K = kChunkBytes / (2 N) inputs.
#ifndef LSP_MLP_CHUNK_BYTES
#define LSP_MLP_CHUNK_BYTES 32768
#endif
constexpr int kChunkBytes = LSP_MLP_CHUNK_BYTES;
static_assert(kChunkBytes >= 8192 && (kChunkBytes & (kChunkBytes - 1)) == 0,
              "a chunk holds at least one K step of 16 of a 256-wide layer");
// shared memory for weight chunks: one tile in flight (2D, 3D), two tiles in flight (2D)
constexpr int kWBuf2D = 131072, kWBuf3D = 98304, kWBufPP = 65536;
constexpr int kMaxChunks = 64;
constexpr int kFusedThreads = 320;  // fused kernel: 8 epilogue warps, MMA warp, loader warp

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

// Streamed weight chunks: every layer's W [N x K] in K-slices of at most 32 KiB (N x kw bf16,
// kw = min(K, 32 KiB / 2N), canonical K-major layout), in layer order. The fused kernel walks
// the same plan at compile time (FusedCfg).
struct ChunkPlan {
  int n;
  int64_t off[kMaxChunks];   // bytes into the tile buffer
  int kw[kMaxChunks];        // K width of the chunk
  int nrows[kMaxChunks];     // N of the chunk (= the layer's output width)
  int layer[kMaxChunks];
  int k0[kMaxChunks];
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

// Derivative of the ReLU activation max(z, 0) (0 at z = 0).
__device__ __forceinline__ float act_grad(float z) { return z > 0.0f ? 1.0f : 0.0f; }

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
  const uint8_t* tiles;  // the weight chunk stream
  const float* params;   // flat params (fp32): biases and normalisation read from here
  const uint8_t* Xt;     // normalised bf16 inputs, one canonical 128 x K0 tile after another
  int64_t M;
  // rows mode: v = vh + vl and s_j = sh + sl per point (fp32 pairs, see k_point_features)
  const float* vh;
  const float* vl;
  const float* sh;
  const float* sl;
  int logn;
  double* Q;
  double* C;
  double* P;
  // batch mode
  float* Y;  // [M x OUTP] normalised outputs
  __nv_bfloat16* Hs[3];
  float* Zs[3];
  int* err;
  // limit of the pipeline's operand waits (the drain at the end always waits up to 1 s, so
  // that no copy or MMA is still in flight when the CTA exits)
  uint64_t wait_ns;
  ChunkPlan plan;
  int64_t bias_off[4], norm_off;
};

constexpr int kModeRows = 0, kModeBatch = 1;
constexpr int kPassCols = 64;            // columns of H per epilogue pass / ready signal
constexpr int kNPass = kH / kPassCols;   // 4
constexpr int kEpiWarps = 8;

template <int D>
struct FusedCfg {
  static constexpr int MU = D == 2 ? 9 : 27;
  static constexpr int K0 = D == 2 ? 32 : 128;
  static constexpr int OUTP = D == 2 ? 32 : 64;
  static constexpr int XBUF = D == 2 ? 2 : 1;  // input-tile buffers
  static constexpr int NBUF = (D == 2 ? kWBuf2D : kWBuf3D) / kChunkBytes;  // weight buffers
  static constexpr int XBYTES = kTile * K0 * 2;
  // the chunk plan of plan_for(), at compile time
  __host__ __device__ static constexpr int N(int l) { return l < 3 ? kH : OUTP; }
  __host__ __device__ static constexpr int K(int l) { return l == 0 ? K0 : kH; }
  __host__ __device__ static constexpr int KW(int l) {
    return K(l) < kChunkBytes / (2 * N(l)) ? K(l) : kChunkBytes / (2 * N(l));
  }
  __host__ __device__ static constexpr int NCH(int l) { return K(l) / KW(l); }
  __host__ __device__ static constexpr int CHUNK_BYTES(int l) { return N(l) * KW(l) * 2; }
  __host__ __device__ static constexpr int64_t OFF(int l) {
    return l == 0 ? 0 : OFF(l - 1) + (int64_t)N(l - 1) * K(l - 1) * 2;
  }
  // normalisation block (mu_x sig_x mu_y[OUTP] sig_y[OUTP]) padded to 16 bytes, so that the
  // arrays behind it keep their 16-byte alignment
  static constexpr int NRM = (2 + 2 * OUTP + 3) & ~3;
  static constexpr size_t smem = (size_t)XBUF * XBYTES + kTile * kH * 2 +
                                 (size_t)NBUF * kChunkBytes +
                                 sizeof(float) * (3 * kH + OUTP + NRM) + 64;
};
template <int D>
constexpr int chunk_count() {
  return FusedCfg<D>::NCH(0) + FusedCfg<D>::NCH(1) + FusedCfg<D>::NCH(2) + FusedCfg<D>::NCH(3);
}
static_assert(chunk_count<2>() <= kMaxChunks && chunk_count<3>() <= kMaxChunks,
              "the chunk plan must fit ChunkPlan");

// float -> double on the integer pipe (the FP64 pipe, which the hardware conversion uses, is
// narrow on this GPU): the 8-bit exponent is rebased from bias 127 to bias 1023 (255 to 2047
// for infinities and NaN, whose payload moves along) and the 23-bit fraction becomes the top
// of the 52-bit one. Exact for normal numbers, zeros, infinities and NaN; subnormal inputs
// (|x| < 2^-126) give a zero of the same sign.
__device__ __forceinline__ double f2d_int(float x) {
  const uint32_t f = __float_as_uint(x), a = f & 0x7FFFFFFFu;
  const uint32_t bias = a >= 0x7F800000u ? (1792u << 20) : (896u << 20);
  const bool sub = a < 0x00800000u;
  const uint32_t hi = (sub ? 0u : (a >> 3) + bias) | (f & 0x80000000u);
  const uint32_t lo = sub ? 0u : f << 29;
  return __hiloint2double((int)hi, (int)lo);
}

// Fused forward over tiles of 128 rows, persistent (one CTA per SM, tiles strided by the grid).
//
// Loader warp 9 (one lane): bulk-copies the input tiles (XBUF buffers, the next tile's as early
// as a buffer is free) and the 32 KiB weight chunks (NBUF buffers, across layer and tile
// boundaries); a buffer is refilled once the MMAs that read it have completed (bar_f, bar_xf).
// Both producer threads walk the chunk plan at compile time (FusedCfg), so their loops carry
// no index arithmetic beyond a buffer counter.
// MMA warp 8 (one lane): issues every MMA and never waits for MMA completion, only for its
// operands: layer l accumulates into tensor-memory accumulator l % 2 (columns 256 (l % 2) ..),
// so layer l + 1 can run while the epilogue still reads layer l. A chunk of layer l > 0 reads
// the columns [k0, k0 + kw) of H and is issued as soon as the epilogue has signalled those
// 64-column passes (bar_h); after the layer's last chunk it commits bar_acc.
// Epilogue warps 0-7: warp w reads tensor-memory lanes 32 (w % 4) .. (one tile row per lane);
// for layers 0-2 it handles columns 32 (w / 4) .. + 31 of each 64-column pass (bias,
// activation, bf16 into H), then arrives once on that pass's barrier (8 arrivals). Layer 3: warps 0-3 write Q and C (or Y), warps
// 4-7 write P.
//
// Ordering: the MMAs of layer l + 1 into accumulator (l + 1) % 2 are issued only after every
// slice of epilogue l has been signalled, which follows the epilogue's reads of accumulator
// (l + 1) % 2 for layer l - 1; epilogue l overwrites H only after the MMAs of layer l (the
// readers of the previous H) completed. Every wait is bounded (1 s); a timed-out wait sets the
// error word and makes every thread skip the remaining waits.
// Two columns of the hidden-layer epilogue: z = acc + b with one packed FP32 addition (it
// rounds like the scalar one), then ReLU and the conversion to bf16 in one instruction,
// packed as the next layer's operand wants it (column 2i in the low half). Returns the packed
// pair; z0, z1 receive z (kept for the backward pass in batch mode).
__device__ __forceinline__ uint32_t relu_bf16x2(uint32_t a0, uint32_t a1, float b0, float b1,
                                                float& z0, float& z1) {
  uint32_t h, r0, r1;
  asm("{\n\t.reg .b64 a, b, z;\n\t"
      "mov.b64 a, {%3, %4};\n\t"
      "mov.b64 b, {%5, %6};\n\t"
      "add.rn.f32x2 z, a, b;\n\t"
      "mov.b64 {%1, %2}, z;\n\t"
      "cvt.rn.relu.bf16x2.f32 %0, %2, %1;\n\t}"
      : "=r"(h), "=r"(r0), "=r"(r1)
      : "r"(a0), "r"(a1), "r"(__float_as_uint(b0)), "r"(__float_as_uint(b1)));
  z0 = __uint_as_float(r0);
  z1 = __uint_as_float(r1);
  return h;
}

template <int D, int MODE>
__global__ void __launch_bounds__(kFusedThreads, 1) k_mlp_fused(FusedParams p) {
  using Cfg = FusedCfg<D>;
  constexpr int MU = Cfg::MU, OUTP = Cfg::OUTP, NBUF = Cfg::NBUF;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* Xs = smem;                                // XBUF x (128 x K0) bf16
  uint8_t* Hs = Xs + Cfg::XBUF * Cfg::XBYTES;        // 128 x 256 bf16
  uint8_t* Wb = Hs + kTile * kH * 2;                 // NBUF x 16 KiB
  float* bs = reinterpret_cast<float*>(Wb + NBUF * kChunkBytes);  // b1 b2 b3 (3 x 256) + b4
  float* nrm = bs + 3 * kH + OUTP;                   // mu_x sig_x mu_y[OUTP] sig_y[OUTP]
  __shared__ __align__(8) uint64_t bar_w[NBUF], bar_f[NBUF], bar_x[2], bar_xf[2], bar_acc[2],
      bar_h[kNPass], bar_done;
  __shared__ uint32_t tslot;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool producer = warp == kEpiWarps;
  const bool leader = producer && lane == 0;

  for (int i = tid; i < kH; i += kFusedThreads) {
    bs[i] = p.params[p.bias_off[0] + i];
    bs[kH + i] = p.params[p.bias_off[1] + i];
    bs[2 * kH + i] = p.params[p.bias_off[2] + i];
  }
  for (int i = tid; i < OUTP; i += kFusedThreads) bs[3 * kH + i] = p.params[p.bias_off[3] + i];
  for (int i = tid; i < 2 + 2 * OUTP; i += kFusedThreads) nrm[i] = p.params[p.norm_off + i];
  if (leader) {
    for (int b = 0; b < NBUF; ++b) {
      tc::mbar_init(&bar_w[b], 1);
      tc::mbar_init(&bar_f[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&bar_x[b], 1);
      tc::mbar_init(&bar_xf[b], 1);
      tc::mbar_init(&bar_acc[b], 1);
    }
    for (int s = 0; s < kNPass; ++s) tc::mbar_init(&bar_h[s], kEpiWarps);
    tc::mbar_init(&bar_done, 1);
    s_abort = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tslot, 2 * kH);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  volatile int* abort_flag = &s_abort;
  // a bounded wait that is skipped once any wait of the CTA has given up
  auto wait = [&](uint64_t* bar, uint32_t parity, int bit) {
    if (tc::mbar_test(bar, parity)) return true;  // fast path: already complete
    if (*abort_flag) return false;
    if (tc::mbar_wait(bar, parity, p.err, bit, p.wait_ns)) return true;
    *abort_flag = 1;
    return false;
  };
  // the same for a whole warp: lane 0 waits, the warp reconverges behind it
  auto wait_warp = [&](uint64_t* bar, uint32_t parity, int bit) {
    if (lane == 0) wait(bar, parity, bit);
    __syncwarp();
  };
  const int64_t ntiles = (p.M + kTile - 1) / kTile;
  const int64_t my_tiles =
      blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (warp == kEpiWarps + 1) {
    // ---- loader: input tiles and weight chunks, in the order the MMA warp consumes them ----
    if (lane == 0) {
      uint32_t slot = 0, ph_f = 0, ph_xf = 0;  // next buffer; phase parities (bit masks)
      uint32_t issued = 0, cnt_x = 0;
      auto load_x = [&](int64_t it) {
        const int xb = Cfg::XBUF == 2 ? (int)(it & 1) : 0;
        const int64_t tile = blockIdx.x + it * gridDim.x;
        tc::mbar_expect_tx(&bar_x[xb], Cfg::XBYTES);
        tc::bulk_g2s(Xs + xb * Cfg::XBYTES, p.Xt + tile * Cfg::XBYTES, Cfg::XBYTES, &bar_x[xb]);
        ++cnt_x;
      };
      if (my_tiles > 0) load_x(0);
      for (int64_t it = 0; it < my_tiles && !*abort_flag; ++it) {
        if (Cfg::XBUF == 2 && it + 1 < my_tiles) {
          if (it + 1 >= 2) {
            // buffer (it + 1) % 2 is free once tile it - 1's first-layer MMAs completed
            const int xb = (int)((it + 1) & 1);
            wait(&bar_xf[xb], ph_xf >> xb & 1, 1);
            ph_xf ^= 1u << xb;
          }
          if (!*abort_flag) load_x(it + 1);
        }
#pragma unroll
        for (int l = 0; l < 4; ++l) {
#pragma unroll
          for (int c = 0; c < Cfg::NCH(l); ++c) {
            if (issued >= (uint32_t)NBUF) {
              // the MMAs of the chunk NBUF jobs earlier (same buffer) must have completed
              wait(&bar_f[slot], ph_f >> slot & 1, 2);
              ph_f ^= 1u << slot;
            }
            if (*abort_flag) break;
            tc::mbar_expect_tx(&bar_w[slot], Cfg::CHUNK_BYTES(l));
            tc::bulk_g2s(Wb + slot * kChunkBytes,
                         p.tiles + Cfg::OFF(l) + (int64_t)c * Cfg::CHUNK_BYTES(l),
                         Cfg::CHUNK_BYTES(l), &bar_w[slot]);
            ++issued;
            slot = slot + 1 == (uint32_t)NBUF ? 0 : slot + 1;
          }
          if (Cfg::XBUF == 1 && l == 0 && it + 1 < my_tiles && !*abort_flag) {
            // the single input buffer is free once this tile's first-layer MMAs completed
            wait(&bar_xf[0], ph_xf & 1, 1);
            ph_xf ^= 1u;
            if (!*abort_flag) load_x(it + 1);
          }
        }
      }
      // drain: every copy issued has landed (bounded; complete unless aborted). The copies of
      // buffer b are its uses number 0, 1, ...; the last one completed phase (uses - 1) % 2.
      for (int b = 0; b < NBUF; ++b) {
        const uint32_t uses = issued / NBUF + ((uint32_t)b < issued % NBUF ? 1u : 0u);
        if (uses) tc::mbar_wait(&bar_w[b], (uses - 1) & 1, p.err, 0);
      }
      if (Cfg::XBUF == 2) {
        for (int b = 0; b < 2; ++b) {
          const uint32_t uses = cnt_x / 2 + ((uint32_t)b < cnt_x % 2 ? 1u : 0u);
          if (uses) tc::mbar_wait(&bar_x[b], (uses - 1) & 1, p.err, 0);
        }
      } else if (cnt_x) {
        tc::mbar_wait(&bar_x[0], (cnt_x - 1) & 1, p.err, 0);
      }
    }
    __syncwarp();
  } else if (producer) {
    // ---- MMA issuer: never waits for MMA completion, only for its operands ----
    if (lane == 0) {
      uint32_t slot = 0, ph_w = 0, ph_h = 0, ph_x = 0;
      for (int64_t it = 0; it < my_tiles && !*abort_flag; ++it) {
        const int xb = Cfg::XBUF == 2 ? (int)(it & 1) : 0;
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const uint32_t acc = tmem + (uint32_t)((l & 1) * kH);
          int waited = 0;  // slices of H signalled for this layer
#pragma unroll
          for (int c = 0; c < Cfg::NCH(l); ++c) {
            const int k0 = c * Cfg::KW(l);
            if (l == 0) {
              if (c == 0) {
                wait(&bar_x[xb], ph_x >> xb & 1, 1);
                ph_x ^= 1u << xb;
              }
            } else {
              // the passes that cover this chunk's K columns (a chunk may end inside a pass)
              const int need = (k0 + Cfg::KW(l) + kPassCols - 1) / kPassCols;
              for (; waited < need; ++waited) {
                wait(&bar_h[waited], ph_h >> waited & 1, 32);
                ph_h ^= 1u << waited;
              }
            }
            wait(&bar_w[slot], ph_w >> slot & 1, 4);
            ph_w ^= 1u << slot;
            if (*abort_flag) break;
            tc::fence_after();
            const uint32_t aBase = l == 0 ? tc::smem_u32(Xs + xb * Cfg::XBYTES) + (k0 / 8) * 128
                                          : tc::smem_u32(Hs) + (k0 / 8) * 128;
            const uint32_t sboA = (uint32_t)((l == 0 ? Cfg::K0 : kH) / 8) * 128;
            const uint32_t sboB = (uint32_t)(Cfg::KW(l) / 8) * 128;
            const uint32_t bBase = tc::smem_u32(Wb + slot * kChunkBytes);
            constexpr uint32_t idesc_h = tc::idesc_bf16(kTile, kH);
            const uint32_t idesc = l < 3 ? idesc_h : tc::idesc_bf16(kTile, Cfg::OUTP);
            // the start-address field (address / 16, 14 bits) of a descriptor advances by
            // 256 / 16 per K step of 16; shared addresses stay below 2^18, so no carry
            const uint64_t ad0 = tc::desc_kmajor(aBase, 128, sboA);
            const uint64_t bd0 = tc::desc_kmajor(bBase, 128, sboB);
#pragma unroll
            for (int s = 0; s < Cfg::KW(l) / 16; ++s)
              tc::mma_bf16(acc, ad0 + (uint64_t)(16 * s), bd0 + (uint64_t)(16 * s), idesc,
                           (c == 0 && s == 0) ? 0u : 1u);
            tc::commit(&bar_f[slot]);
            slot = slot + 1 == (uint32_t)NBUF ? 0 : slot + 1;
          }
          if (*abort_flag) break;
          tc::commit(&bar_acc[l & 1]);
          if (l == 0) tc::commit(&bar_xf[xb]);
        }
      }
      // every MMA of this thread has completed before the tensor memory is released
      tc::commit(&bar_done);
      tc::mbar_wait(&bar_done, 0, p.err, 0);
    }
    __syncwarp();
  } else {
    // ---- epilogue warps ----
    const int quarter = warp & 3, grp = warp >> 2;
    const int trow = quarter * 32 + lane;  // tensor-memory lane = tile row
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    uint32_t ph_acc[2] = {0, 0};
    const int64_t mask = ((int64_t)1 << p.logn) - 1;
    for (int64_t it = 0; it < my_tiles; ++it) {
      if (__shfl_sync(0xffffffffu, *abort_flag, 0)) break;  // warp-uniform
      const int64_t r0 = (blockIdx.x + it * gridDim.x) * kTile;
      const int64_t myrow = r0 + trow;
      for (int layer = 0; layer < 3; ++layer) {
        const int a = layer & 1;
        wait_warp(&bar_acc[a], ph_acc[a], 8);
        ph_acc[a] ^= 1;
        tc::fence_after();
        const uint32_t taddr = tmem + lane_off + (uint32_t)(a * kH);
        const float* bl = bs + layer * kH;
        uint32_t r[2][32];
        tc::tmem_ld32_nowait(taddr + grp * 32, r[0]);
#pragma unroll
        for (int pass = 0; pass < kNPass; ++pass) {
          const int cb = pass * kPassCols + grp * 32;  // this warp's 32 columns of the pass
          tc::ld_wait(r[pass & 1]);
          if (pass + 1 < kNPass)
            tc::tmem_ld32_nowait(taddr + cb + kPassCols, r[(pass + 1) & 1]);
          const uint32_t* rr = r[pass & 1];
#pragma unroll
          for (int q8 = 0; q8 < 4; ++q8) {
            // ReLU of z = acc + b, eight columns: two bias loads, four packed additions, four
            // converting ReLUs into bf16 pairs, one 16-byte store
            const int i = 8 * q8;
            const float4 b0 = *reinterpret_cast<const float4*>(bl + cb + i);
            const float4 b1 = *reinterpret_cast<const float4*>(bl + cb + i + 4);
            float z[8];
            uint4 q;
            q.x = relu_bf16x2(rr[i + 0], rr[i + 1], b0.x, b0.y, z[0], z[1]);
            q.y = relu_bf16x2(rr[i + 2], rr[i + 3], b0.z, b0.w, z[2], z[3]);
            q.z = relu_bf16x2(rr[i + 4], rr[i + 5], b1.x, b1.y, z[4], z[5]);
            q.w = relu_bf16x2(rr[i + 6], rr[i + 7], b1.z, b1.w, z[6], z[7]);
            *reinterpret_cast<uint4*>(Hs + tc::kmajor_off(trow, cb + i, kH)) = q;
            if (MODE == kModeBatch && myrow < p.M) {
#pragma unroll
              for (int u = 0; u < 8; ++u) p.Zs[layer][myrow * kH + cb + i + u] = z[u];
              *reinterpret_cast<uint4*>(p.Hs[layer] + myrow * kH + cb + i) = q;
            }
          }
          // this warp's part of the pass is written: make it visible to the tensor cores
          tc::fence_async_smem();
          tc::fence_before();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&bar_h[pass]);
        }
      }
      // ---- layer 3: the outputs (accumulator 1) ----
      // rows mode, group 1, 2D: the fp32 pairs of s_j and of v at the stencil offsets, loaded
      // while the layer-3 MMAs run (in 3D the 56 values cost more registers than they save)
      float pf_sh = 0.f, pf_sl = 0.f, pf_vh[MU], pf_vl[MU];
#pragma unroll
      for (int i = 0; i < MU; ++i) pf_vh[i] = pf_vl[i] = 0.f;
      if (D == 2 && MODE == kModeRows && grp == 1 && myrow < p.M) {
        pf_sh = __ldg(p.sh + myrow);
        pf_sl = __ldg(p.sl + myrow);
#pragma unroll
        for (int i = 0; i < MU; ++i) {
          const int64_t nb = nb_index<D, 1>(myrow, i, p.logn, mask);
          pf_vh[i] = __ldg(p.vh + nb);
          pf_vl[i] = __ldg(p.vl + nb);
        }
      }
      wait_warp(&bar_acc[1], ph_acc[1], 8);
      ph_acc[1] ^= 1;
      tc::fence_after();
      if (__shfl_sync(0xffffffffu, *abort_flag, 0)) break;
      float y[OUTP];
      {
        const uint32_t taddr = tmem + lane_off + (uint32_t)kH;
        uint32_t r[32];
#pragma unroll
        for (int c0 = 0; c0 < OUTP; c0 += 32) {
          tc::tmem_ld32_nowait(taddr + c0, r);
          tc::ld_wait(r);
#pragma unroll
          for (int i = 0; i < 32; ++i) y[c0 + i] = __uint_as_float(r[i]) + bs[3 * kH + c0 + i];
        }
      }
      tc::fence_before();
      if (myrow < p.M) {
        if (MODE == kModeBatch) {
          if (grp == 0) {
#pragma unroll
            for (int o = 0; o < OUTP; ++o) p.Y[myrow * OUTP + o] = y[o];
          }
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
          if (grp == 0) {
#pragma unroll
            for (int i = 0; i < MU; ++i) {
              __stcs(p.Q + myrow * MU + i, (double)(al[i] * sc));
              __stcs(p.C + myrow * MU + i, (double)(cc[i] * sc));
            }
          } else {
            // v[mu_j] - s_j from the fp32 pairs: the difference of the high parts is exact
            // when v and s_j are within a factor of two of each other (the usual case)
            if (D == 3 && myrow < p.M) {
              pf_sh = __ldg(p.sh + myrow);
              pf_sl = __ldg(p.sl + myrow);
#pragma unroll
              for (int i = 0; i < MU; ++i) {
                const int64_t nb = nb_index<D, 1>(myrow, i, p.logn, mask);
                pf_vh[i] = __ldg(p.vh + nb);
                pf_vl[i] = __ldg(p.vl + nb);
              }
            }
#pragma unroll
            for (int i = 0; i < MU; ++i) {
              const float dv = (pf_vh[i] - pf_sh) + (pf_vl[i] - pf_sl);
              __stcs(p.P + myrow * MU + i, (double)(fmaf(cc[i] * sc, dv, al[i] * sc)));
            }
          }
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 2 * kH);
}

// ---- two tiles in flight (2D) -----------------------------------------------------------
// The fused kernel above runs one tile's layers back to back, so the tensor cores wait while
// the epilogue converts a layer and the epilogue waits while the next layer multiplies. Here a
// CTA takes its tiles in pairs (A, B), each with its own accumulator (tensor-memory columns
// 256 t ..) and its own activation buffer H_t, and interleaves them: the MMAs of B's layer l run
// while the epilogue converts A's layer l, and the MMAs of A's layer l + 1 run while it converts
// B's, so that the epilogue warps always have a layer to convert.
//
// Order of work, per pair: for l = 0..3, for t = A, B: MMAs (t, l), then epilogue (t, l).
// MMA (t, l) waits for epilogue (t, l - 1) (its accumulator read out, H_t written; for l = 0
// the output layer of the previous pair's tile t) and, for l = 0, for the input tile X_t.
// Epilogue (t, l) waits for the MMAs (t, l) (bar_acc[t]). The loader streams the weight chunks
// in the MMA warp's order (every tile reads all of them; two 32 KiB buffers), and the next
// pair's input tile t once the layer-0 MMAs of tile t have completed. Every wait is bounded as
// in the fused kernel; a wait that gives up stops the CTA after its copies and MMAs drain.
constexpr int kPPThreads = 320;  // 8 epilogue warps, the MMA warp, the loader warp

struct PPCfg {
  static constexpr int MU = 9, K0 = 32, OUTP = 32, NBUF = kWBufPP / kChunkBytes;
  static constexpr int XBYTES = kTile * K0 * 2;  // 8 KiB per input tile
  static constexpr int HBYTES = kTile * kH * 2;  // 64 KiB per activation buffer
  static constexpr int NRM = (2 + 2 * OUTP + 3) & ~3;
  static constexpr size_t smem = 2 * (size_t)XBYTES + 2 * (size_t)HBYTES +
                                 (size_t)NBUF * kChunkBytes +
                                 sizeof(float) * (3 * kH + OUTP + NRM) + 64;
};

template <int MODE>
__global__ void __launch_bounds__(kPPThreads, 1) k_mlp_pp(FusedParams p) {
  using Cfg = FusedCfg<2>;  // the chunk plan of the 2D network
  constexpr int MU = PPCfg::MU, OUTP = PPCfg::OUTP, NBUF = PPCfg::NBUF;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* Xs = smem;                                   // 2 x (128 x 32) bf16
  uint8_t* Hs = Xs + 2 * PPCfg::XBYTES;                 // 2 x (128 x 256) bf16
  uint8_t* Wb = Hs + 2 * PPCfg::HBYTES;                 // NBUF x 32 KiB
  float* bs = reinterpret_cast<float*>(Wb + NBUF * kChunkBytes);
  float* nrm = bs + 3 * kH + OUTP;
  __shared__ __align__(8) uint64_t bar_w[NBUF], bar_f[NBUF], bar_x[2], bar_xf[2], bar_acc[2],
      bar_e[2], bar_done;
  __shared__ uint32_t tslot;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool mma_warp = warp == kEpiWarps;
  const bool loader = warp == kEpiWarps + 1;

  for (int i = tid; i < kH; i += kPPThreads) {
    bs[i] = p.params[p.bias_off[0] + i];
    bs[kH + i] = p.params[p.bias_off[1] + i];
    bs[2 * kH + i] = p.params[p.bias_off[2] + i];
  }
  for (int i = tid; i < OUTP; i += kPPThreads) bs[3 * kH + i] = p.params[p.bias_off[3] + i];
  for (int i = tid; i < 2 + 2 * OUTP; i += kPPThreads) nrm[i] = p.params[p.norm_off + i];
  if (mma_warp && lane == 0) {
    for (int b = 0; b < NBUF; ++b) {
      tc::mbar_init(&bar_w[b], 1);
      tc::mbar_init(&bar_f[b], 1);
    }
    for (int t = 0; t < 2; ++t) {
      tc::mbar_init(&bar_x[t], 1);
      tc::mbar_init(&bar_xf[t], 1);
      tc::mbar_init(&bar_acc[t], 1);
      tc::mbar_init(&bar_e[t], kEpiWarps);
    }
    tc::mbar_init(&bar_done, 1);
    s_abort = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tslot, 2 * kH);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  volatile int* abort_flag = &s_abort;
  auto wait = [&](uint64_t* bar, uint32_t parity, int bit) {
    if (tc::mbar_test(bar, parity)) return true;
    if (*abort_flag) return false;
    if (tc::mbar_wait(bar, parity, p.err, bit, p.wait_ns)) return true;
    *abort_flag = 1;
    return false;
  };
  auto wait_warp = [&](uint64_t* bar, uint32_t parity, int bit) {
    if (lane == 0) wait(bar, parity, bit);
    __syncwarp();
  };
  // this CTA's tiles: blockIdx.x + i * gridDim.x, i < my_tiles; pairs (2k, 2k + 1)
  const int64_t ntiles = (p.M + kTile - 1) / kTile;
  const int64_t my_tiles =
      blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t my_pairs = (my_tiles + 1) / 2;
  auto tile_of = [&](int64_t pair, int t) { return (int64_t)blockIdx.x + (2 * pair + t) * gridDim.x; };
  auto has = [&](int64_t pair, int t) { return 2 * pair + t < my_tiles; };

  if (loader) {
    if (lane == 0) {
      uint32_t slot = 0, ph_f = 0, ph_xf = 0, issued = 0, cnt_x[2] = {0, 0};
      auto load_x = [&](int64_t pair, int t) {
        tc::mbar_expect_tx(&bar_x[t], PPCfg::XBYTES);
        tc::bulk_g2s(Xs + t * PPCfg::XBYTES, p.Xt + tile_of(pair, t) * PPCfg::XBYTES,
                     PPCfg::XBYTES, &bar_x[t]);
        ++cnt_x[t];
      };
      if (my_pairs > 0) {
        load_x(0, 0);
        if (has(0, 1)) load_x(0, 1);
      }
      for (int64_t pr = 0; pr < my_pairs && !*abort_flag; ++pr) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          for (int t = 0; t < 2; ++t) {
            if (!has(pr, t) || *abort_flag) continue;
#pragma unroll
            for (int c = 0; c < Cfg::NCH(l); ++c) {
              if (issued >= (uint32_t)NBUF) {
                wait(&bar_f[slot], ph_f >> slot & 1, 2);  // the MMAs that read this buffer
                ph_f ^= 1u << slot;
              }
              if (*abort_flag) break;
              tc::mbar_expect_tx(&bar_w[slot], Cfg::CHUNK_BYTES(l));
              tc::bulk_g2s(Wb + slot * kChunkBytes,
                           p.tiles + Cfg::OFF(l) + (int64_t)c * Cfg::CHUNK_BYTES(l),
                           Cfg::CHUNK_BYTES(l), &bar_w[slot]);
              ++issued;
              slot = slot + 1 == (uint32_t)NBUF ? 0 : slot + 1;
            }
            // after tile t's layer-1 chunks: its input buffer is free once its layer-0 MMAs
            // completed; bring in the next pair's tile t
            if (l == 1 && has(pr + 1, t) && !*abort_flag) {
              wait(&bar_xf[t], ph_xf >> t & 1, 1);
              ph_xf ^= 1u << t;
              if (!*abort_flag) load_x(pr + 1, t);
            }
          }
        }
      }
      // drain: every copy issued has landed (1 s limit; complete unless aborted)
      for (int b = 0; b < NBUF; ++b) {
        const uint32_t uses = issued / NBUF + ((uint32_t)b < issued % NBUF ? 1u : 0u);
        if (uses) tc::mbar_wait(&bar_w[b], (uses - 1) & 1, p.err, 0);
      }
      for (int t = 0; t < 2; ++t)
        if (cnt_x[t]) tc::mbar_wait(&bar_x[t], (cnt_x[t] - 1) & 1, p.err, 0);
    }
    __syncwarp();
  } else if (mma_warp) {
    if (lane == 0) {
      uint32_t slot = 0, ph_w = 0, ph_x = 0, ph_e = 0;
      uint32_t e_done[2] = {0, 0};  // epilogues of tile slot t completed so far (expected)
      for (int64_t pr = 0; pr < my_pairs && !*abort_flag; ++pr) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          for (int t = 0; t < 2; ++t) {
            if (!has(pr, t) || *abort_flag) continue;
            if (l == 0) {
              wait(&bar_x[t], ph_x >> t & 1, 1);
              ph_x ^= 1u << t;
            }
            if (e_done[t] > 0) {  // the previous epilogue of this slot: H_t written, acc read
              wait(&bar_e[t], ph_e >> t & 1, 32);
              ph_e ^= 1u << t;
            }
            const uint32_t acc = tmem + (uint32_t)(t * kH);
#pragma unroll
            for (int c = 0; c < Cfg::NCH(l); ++c) {
              wait(&bar_w[slot], ph_w >> slot & 1, 4);
              ph_w ^= 1u << slot;
              if (*abort_flag) break;
              tc::fence_after();
              const int k0 = c * Cfg::KW(l);
              const uint32_t aBase = l == 0 ? tc::smem_u32(Xs + t * PPCfg::XBYTES) + (k0 / 8) * 128
                                            : tc::smem_u32(Hs + t * PPCfg::HBYTES) + (k0 / 8) * 128;
              const uint32_t sboA = (uint32_t)((l == 0 ? Cfg::K0 : kH) / 8) * 128;
              const uint32_t sboB = (uint32_t)(Cfg::KW(l) / 8) * 128;
              const uint32_t bBase = tc::smem_u32(Wb + slot * kChunkBytes);
              constexpr uint32_t idesc_h = tc::idesc_bf16(kTile, kH);
              const uint32_t idesc = l < 3 ? idesc_h : tc::idesc_bf16(kTile, OUTP);
              const uint64_t ad0 = tc::desc_kmajor(aBase, 128, sboA);
              const uint64_t bd0 = tc::desc_kmajor(bBase, 128, sboB);
#pragma unroll
              for (int s = 0; s < Cfg::KW(l) / 16; ++s)
                tc::mma_bf16(acc, ad0 + (uint64_t)(16 * s), bd0 + (uint64_t)(16 * s), idesc,
                             (c == 0 && s == 0) ? 0u : 1u);
              tc::commit(&bar_f[slot]);
              slot = slot + 1 == (uint32_t)NBUF ? 0 : slot + 1;
            }
            if (*abort_flag) break;
            tc::commit(&bar_acc[t]);
            if (l == 0) tc::commit(&bar_xf[t]);
            ++e_done[t];
          }
        }
      }
      // every MMA of this thread has completed before the tensor memory is released
      tc::commit(&bar_done);
      tc::mbar_wait(&bar_done, 0, p.err, 0);
    }
    __syncwarp();
  } else {
    // ---- epilogue warps: (A, l), (B, l), (A, l + 1), ... ----
    const int quarter = warp & 3, grp = warp >> 2;
    const int trow = quarter * 32 + lane;  // tensor-memory lane = tile row
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    uint32_t ph_acc = 0;
    const int64_t mask = ((int64_t)1 << p.logn) - 1;
    // rows mode, warps of group 1: the fp32 pairs of s_j and of v at the stencil offsets that
    // P = alpha + c (v - s_j) needs, loaded one layer ahead (set a: tile A, set b: tile B)
    float a_sh = 0.f, a_sl = 0.f, a_vh[MU], a_vl[MU], b_sh = 0.f, b_sl = 0.f, b_vh[MU], b_vl[MU];
#pragma unroll
    for (int i = 0; i < MU; ++i) a_vh[i] = a_vl[i] = b_vh[i] = b_vl[i] = 0.f;
    auto prefetch = [&](int64_t row, float& sh, float& sl, float (&vh)[MU], float (&vl)[MU]) {
      if (row >= p.M) return;
      sh = __ldg(p.sh + row);
      sl = __ldg(p.sl + row);
#pragma unroll
      for (int i = 0; i < MU; ++i) {
        const int64_t nb = nb_index<2, 1>(row, i, p.logn, mask);
        vh[i] = __ldg(p.vh + nb);
        vl[i] = __ldg(p.vl + nb);
      }
    };
    for (int64_t pr = 0; pr < my_pairs; ++pr) {
      if (__shfl_sync(0xffffffffu, *abort_flag, 0)) break;
      for (int l = 0; l < 4; ++l) {
        for (int t = 0; t < 2; ++t) {
          if (!has(pr, t)) continue;
          if (MODE == kModeRows && grp == 1) {
            if (l == 2 && t == 1) {
              prefetch(tile_of(pr, 0) * kTile + trow, a_sh, a_sl, a_vh, a_vl);
            } else if (l == 3 && t == 0) {
              if (has(pr, 1))
                prefetch(tile_of(pr, 1) * kTile + trow, b_sh, b_sl, b_vh, b_vl);
              else
                prefetch(tile_of(pr, 0) * kTile + trow, a_sh, a_sl, a_vh, a_vl);
            }
          }
          wait_warp(&bar_acc[t], ph_acc >> t & 1, 8);
          ph_acc ^= 1u << t;
          tc::fence_after();
          const bool stop = __shfl_sync(0xffffffffu, *abort_flag, 0);
          const uint32_t taddr = tmem + lane_off + (uint32_t)(t * kH);
          const int64_t myrow = tile_of(pr, t) * kTile + trow;
          uint8_t* Ht = Hs + t * PPCfg::HBYTES;
          if (l < 3 && !stop) {
            const float* bl = bs + l * kH;
            uint32_t r[2][32];
            tc::tmem_ld32_nowait(taddr + grp * 32, r[0]);
#pragma unroll
            for (int pass = 0; pass < kNPass; ++pass) {
              const int cb = pass * kPassCols + grp * 32;
              tc::ld_wait(r[pass & 1]);
              if (pass + 1 < kNPass)
                tc::tmem_ld32_nowait(taddr + cb + kPassCols, r[(pass + 1) & 1]);
              const uint32_t* rr = r[pass & 1];
#pragma unroll
              for (int q8 = 0; q8 < 4; ++q8) {
                const int i = 8 * q8;
                const float4 b0 = *reinterpret_cast<const float4*>(bl + cb + i);
                const float4 b1 = *reinterpret_cast<const float4*>(bl + cb + i + 4);
                float z[8];
                uint4 q;
                q.x = relu_bf16x2(rr[i + 0], rr[i + 1], b0.x, b0.y, z[0], z[1]);
                q.y = relu_bf16x2(rr[i + 2], rr[i + 3], b0.z, b0.w, z[2], z[3]);
                q.z = relu_bf16x2(rr[i + 4], rr[i + 5], b1.x, b1.y, z[4], z[5]);
                q.w = relu_bf16x2(rr[i + 6], rr[i + 7], b1.z, b1.w, z[6], z[7]);
                *reinterpret_cast<uint4*>(Ht + tc::kmajor_off(trow, cb + i, kH)) = q;
                if (MODE == kModeBatch && myrow < p.M) {
#pragma unroll
                  for (int u = 0; u < 8; ++u) p.Zs[l][myrow * kH + cb + i + u] = z[u];
                  *reinterpret_cast<uint4*>(p.Hs[l] + myrow * kH + cb + i) = q;
                }
              }
            }
            // H_t is written and the accumulator read: the MMAs of (t, l + 1) may go
            tc::fence_async_smem();
          } else if (!stop) {
            // output layer: (alpha, c) and the rows, or the normalised outputs Y
            float y[OUTP];
            {
              uint32_t r[32];
              tc::tmem_ld32_nowait(taddr, r);
              tc::ld_wait(r);
#pragma unroll
              for (int i = 0; i < 32; ++i) y[i] = __uint_as_float(r[i]) + bs[3 * kH + i];
            }
            if (MODE == kModeBatch) {
              if (grp == 0 && myrow < p.M) {
#pragma unroll
                for (int o = 0; o < OUTP; ++o) p.Y[myrow * OUTP + o] = y[o];
              }
            } else {
              // de-normalise, unit-normalise alpha (c scaled alike: P^-1 C is invariant)
              float al[MU], cc[MU], nrm2 = 0.0f;
#pragma unroll
              for (int i = 0; i < MU; ++i) {
                al[i] = y[i] * nrm[2 + OUTP + i] + nrm[2 + i];
                cc[i] = y[MU + i] * nrm[2 + OUTP + MU + i] + nrm[2 + MU + i];
                nrm2 = fmaf(al[i], al[i], nrm2);
              }
              const float sc = nrm2 > 0.0f ? rsqrtf(nrm2) : 1.0f;
              // This warp's 32 rows of Q and C (group 0) or of P (group 1) are contiguous
              // blocks of 32 x MU doubles in global memory. When all 32 rows exist they are
              // staged in H_t (free: the layer-3 MMAs that read it have completed, and the
              // next writes to it follow this epilogue's arrival) and leave by one bulk copy
              // per block; otherwise each row is stored directly.
              constexpr int BLK = 32 * MU * 8;
              const int64_t wrow0 = tile_of(pr, t) * kTile + quarter * 32;
              const bool full = wrow0 + 32 <= p.M;
              double* stg = reinterpret_cast<double*>(Ht + (grp == 0 ? quarter : 8 + quarter) * BLK);
              if (grp == 0) {
#pragma unroll
                for (int i = 0; i < MU; ++i) {
                  // Q and C convert on the integer pipe while group 1 converts P on the FP64
                  // pipe: the two pipes run side by side
                  const double qv = f2d_int(al[i] * sc), cv = f2d_int(cc[i] * sc);
                  if (full) {
                    stg[lane * MU + i] = qv;
                    stg[4 * BLK / 8 + lane * MU + i] = cv;
                  } else if (myrow < p.M) {
                    __stcs(p.Q + myrow * MU + i, qv);
                    __stcs(p.C + myrow * MU + i, cv);
                  }
                }
              } else {
                // v[mu_j] - s_j from the fp32 pairs: the difference of the high parts is exact
                // when v and s_j are within a factor of two of each other (the usual case)
                const float sh = t == 0 ? a_sh : b_sh, sl = t == 0 ? a_sl : b_sl;
#pragma unroll
                for (int i = 0; i < MU; ++i) {
                  const float dv = ((t == 0 ? a_vh[i] : b_vh[i]) - sh) +
                                   ((t == 0 ? a_vl[i] : b_vl[i]) - sl);
                  const double pv = (double)(fmaf(cc[i] * sc, dv, al[i] * sc));
                  if (full)
                    stg[lane * MU + i] = pv;
                  else if (myrow < p.M)
                    __stcs(p.P + myrow * MU + i, pv);
                }
              }
              if (full) {
                tc::fence_async_smem();
                __syncwarp();
                if (lane == 0) {
                  if (grp == 0) {
                    tc::bulk_s2g(p.Q + wrow0 * MU, stg, BLK);
                    tc::bulk_s2g(p.C + wrow0 * MU, stg + 4 * BLK / 8, BLK);
                  } else {
                    tc::bulk_s2g(p.P + wrow0 * MU, stg, BLK);
                  }
                  tc::bulk_commit();
                  tc::bulk_wait_read();  // H_t may be written again once every warp arrived
                }
              }
            }
          }
          tc::fence_before();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&bar_e[t]);
        }
      }
    }
    if (lane == 0) tc::bulk_wait_all();  // this warp's row stores have landed
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 2 * kH);
}

// ---- two tiles in flight on a CTA pair (2D, cta_group::2) ----------------------------------
// The two-tile schedule above streams every weight chunk into every CTA through two 32 KiB
// buffers, and a chunk takes ~1.1k cycles from its copy to its arrival, against ~0.5k cycles of
// MMA for the chunk before it, so the MMAs stall at every buffer reuse. Here a cluster of two
// CTAs (one TPC) runs the same schedule on super-tiles of 256 rows with M = 256 MMAs: each CTA
// holds its 128 rows (input tile, activations, accumulator rows) and HALF of every weight chunk
// (N/2 rows of the K-major chunk, 16 KiB), so the same 64 KiB give four chunk buffers (three
// chunks of lead) and each SM streams half the weight bytes.
//
// The even CTA (rank 0) issues every MMA and commit; commits arrive in both CTAs (bar_f: a
// buffer may be refilled; bar_acc: an accumulator is ready; bar_xf: an input buffer is free;
// bar_done). Operands of the odd CTA are reported to the even one: its MMA warp forwards the
// arrival of each of its weight halves (bar_wp) and input tiles (bar_xp), and every epilogue
// warp of both CTAs arrives on the even CTA's bar_e (16 arrivals). Both CTAs walk the same
// sequence of super-tiles, so the weight stream stays in step. Every wait is bounded; a CTA
// that gives up stops arriving, and its partner's waits then run out too.
//
// Measured on GB300 (2D n = 1024): 0.47 ms against 0.36 ms for the one-CTA two-tile kernel, with
// bit-identical rows. The weight stalls are gone, but the pair MMAs of a chunk take ~700 cycles
// instead of ~500, and the cluster-scope arrivals lengthen every epilogue by ~1k cycles
// (forwarding them through one thread instead made it 0.50 ms). Selectable as schedule 2.
constexpr int kPP2Half = kChunkBytes / 2;

struct PP2Cfg {
  static constexpr int NBUF = kWBufPP / kPP2Half;  // half-chunk buffers
};

template <int MODE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kPPThreads, 1) k_mlp_pp2(FusedParams p) {
  using Cfg = FusedCfg<2>;
  constexpr int MU = PPCfg::MU, OUTP = PPCfg::OUTP, NBUF = PP2Cfg::NBUF;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* Xs = smem;                    // 2 x (128 x 32) bf16: this CTA's rows of tiles A, B
  uint8_t* Hs = Xs + 2 * PPCfg::XBYTES;  // 2 x (128 x 256) bf16
  uint8_t* Wb = Hs + 2 * PPCfg::HBYTES;  // NBUF x 16 KiB: this CTA's half of each chunk
  float* bs = reinterpret_cast<float*>(Wb + NBUF * kPP2Half);
  float* nrm = bs + 3 * kH + OUTP;
  __shared__ __align__(8) uint64_t bar_w[NBUF], bar_wp[NBUF], bar_f[NBUF], bar_x[2], bar_xp[2],
      bar_xf[2], bar_acc[2], bar_e[2], bar_done;
  __shared__ uint32_t tslot;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool mma_warp = warp == kEpiWarps;
  const bool loader = warp == kEpiWarps + 1;
  const uint32_t rank = tc::cluster_rank();

  for (int i = tid; i < kH; i += kPPThreads) {
    bs[i] = p.params[p.bias_off[0] + i];
    bs[kH + i] = p.params[p.bias_off[1] + i];
    bs[2 * kH + i] = p.params[p.bias_off[2] + i];
  }
  for (int i = tid; i < OUTP; i += kPPThreads) bs[3 * kH + i] = p.params[p.bias_off[3] + i];
  for (int i = tid; i < 2 + 2 * OUTP; i += kPPThreads) nrm[i] = p.params[p.norm_off + i];
  if (mma_warp && lane == 0) {
    for (int b = 0; b < NBUF; ++b) {
      tc::mbar_init(&bar_w[b], 1);
      tc::mbar_init(&bar_wp[b], 1);
      tc::mbar_init(&bar_f[b], 1);
    }
    for (int t = 0; t < 2; ++t) {
      tc::mbar_init(&bar_x[t], 1);
      tc::mbar_init(&bar_xp[t], 1);
      tc::mbar_init(&bar_xf[t], 1);
      tc::mbar_init(&bar_acc[t], 1);
      tc::mbar_init(&bar_e[t], 2 * kEpiWarps);
    }
    tc::mbar_init(&bar_done, 1);
    s_abort = 0;
  }
  if (warp == 0) tc::tmem_alloc_pair(&tslot, 2 * kH);
  tc::fence_before();
  __syncthreads();
  // both CTAs' barriers are initialised before either CTA arrives on the other's
  tc::cluster_sync();
  tc::fence_after();
  const uint32_t tmem = tslot;
  volatile int* abort_flag = &s_abort;
  auto wait = [&](uint64_t* bar, uint32_t parity, int bit) {
    if (tc::mbar_test_cluster(bar, parity)) return true;
    if (*abort_flag) return false;
    if (tc::mbar_wait_cluster(bar, parity, p.err, bit, p.wait_ns)) return true;
    *abort_flag = 1;
    return false;
  };
  auto wait_warp = [&](uint64_t* bar, uint32_t parity, int bit) {
    if (lane == 0) wait(bar, parity, bit);
    __syncwarp();
  };
  // super-tiles of 256 rows: the pair handles cl + i * ncl, i < my_super, in pairs (A, B);
  // this CTA's rows of super-tile s are the 128-row tile 2 s + rank
  const int64_t ntiles = (p.M + kTile - 1) / kTile;
  const int64_t nsuper = (ntiles + 1) / 2;
  const int64_t cl = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  const int64_t my_super = cl < nsuper ? (nsuper - 1 - cl) / ncl + 1 : 0;
  const int64_t my_pairs = (my_super + 1) / 2;
  auto tile_of = [&](int64_t pair, int t) {
    return 2 * (cl + (2 * pair + t) * ncl) + (int64_t)rank;
  };
  auto has = [&](int64_t pair, int t) { return 2 * pair + t < my_super; };

  if (loader) {
    if (lane == 0) {
      uint32_t slot = 0, ph_f = 0, ph_xf = 0, issued = 0, cnt_x[2] = {0, 0};
      auto load_x = [&](int64_t pair, int t) {
        tc::mbar_expect_tx(&bar_x[t], PPCfg::XBYTES);
        tc::bulk_g2s(Xs + t * PPCfg::XBYTES, p.Xt + tile_of(pair, t) * PPCfg::XBYTES,
                     PPCfg::XBYTES, &bar_x[t]);
        ++cnt_x[t];
      };
      if (my_pairs > 0) {
        load_x(0, 0);
        if (has(0, 1)) load_x(0, 1);
      }
      for (int64_t pr = 0; pr < my_pairs && !*abort_flag; ++pr) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          for (int t = 0; t < 2; ++t) {
            if (!has(pr, t) || *abort_flag) continue;
#pragma unroll
            for (int c = 0; c < Cfg::NCH(l); ++c) {
              if (issued >= (uint32_t)NBUF) {
                wait(&bar_f[slot], ph_f >> slot & 1, 2);  // the pair MMAs that read it
                ph_f ^= 1u << slot;
              }
              if (*abort_flag) break;
              const int half = Cfg::CHUNK_BYTES(l) / 2;
              tc::mbar_expect_tx(&bar_w[slot], half);
              tc::bulk_g2s(Wb + slot * kPP2Half,
                           p.tiles + Cfg::OFF(l) + (int64_t)c * Cfg::CHUNK_BYTES(l) +
                               (int64_t)rank * half,
                           half, &bar_w[slot]);
              ++issued;
              slot = slot + 1 == (uint32_t)NBUF ? 0 : slot + 1;
            }
            if (l == 1 && has(pr + 1, t) && !*abort_flag) {
              wait(&bar_xf[t], ph_xf >> t & 1, 1);
              ph_xf ^= 1u << t;
              if (!*abort_flag) load_x(pr + 1, t);
            }
          }
        }
      }
      for (int b = 0; b < NBUF; ++b) {
        const uint32_t uses = issued / NBUF + ((uint32_t)b < issued % NBUF ? 1u : 0u);
        if (uses) tc::mbar_wait(&bar_w[b], (uses - 1) & 1, p.err, 0);
      }
      for (int t = 0; t < 2; ++t)
        if (cnt_x[t]) tc::mbar_wait(&bar_x[t], (cnt_x[t] - 1) & 1, p.err, 0);
    }
    __syncwarp();
  } else if (mma_warp && rank != 0) {
    // ---- odd CTA: forward the arrival of its operands to the even CTA ----
    if (lane == 0) {
      uint32_t slot = 0, ph_w = 0, ph_x = 0;
      for (int64_t pr = 0; pr < my_pairs && !*abort_flag; ++pr) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          for (int t = 0; t < 2; ++t) {
            if (!has(pr, t) || *abort_flag) continue;
            if (l == 0) {
              if (!wait(&bar_x[t], ph_x >> t & 1, 1)) break;
              ph_x ^= 1u << t;
              tc::mbar_arrive_cluster(&bar_xp[t], 0);
            }
#pragma unroll
            for (int c = 0; c < Cfg::NCH(l); ++c) {
              if (!wait(&bar_w[slot], ph_w >> slot & 1, 4)) break;
              ph_w ^= 1u << slot;
              tc::mbar_arrive_cluster(&bar_wp[slot], 0);
              slot = slot + 1 == (uint32_t)NBUF ? 0 : slot + 1;
            }
          }
        }
      }
      // the even CTA's last commit: every pair MMA (which reads this CTA's shared memory and
      // writes its tensor memory) has completed
      tc::mbar_wait(&bar_done, 0, p.err, 0);
    }
    __syncwarp();
  } else if (mma_warp) {
    // ---- even CTA: every MMA of the pair ----
    if (lane == 0) {
      uint32_t slot = 0, ph_w = 0, ph_x = 0, ph_e = 0;
      uint32_t e_done[2] = {0, 0};
      for (int64_t pr = 0; pr < my_pairs && !*abort_flag; ++pr) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          for (int t = 0; t < 2; ++t) {
            if (!has(pr, t) || *abort_flag) continue;
            if (l == 0) {
              wait(&bar_x[t], ph_x >> t & 1, 1);
              wait(&bar_xp[t], ph_x >> t & 1, 1);
              ph_x ^= 1u << t;
            }
            if (e_done[t] > 0) {  // both CTAs' epilogues of this slot: H_t written, acc read
              wait(&bar_e[t], ph_e >> t & 1, 32);
              ph_e ^= 1u << t;
            }
            const uint32_t acc = tmem + (uint32_t)(t * kH);
#pragma unroll
            for (int c = 0; c < Cfg::NCH(l); ++c) {
              wait(&bar_w[slot], ph_w >> slot & 1, 4);
              wait(&bar_wp[slot], ph_w >> slot & 1, 4);
              ph_w ^= 1u << slot;
              if (*abort_flag) break;
              tc::fence_after();
              const int k0 = c * Cfg::KW(l);
              const uint32_t aBase = l == 0 ? tc::smem_u32(Xs + t * PPCfg::XBYTES) + (k0 / 8) * 128
                                            : tc::smem_u32(Hs + t * PPCfg::HBYTES) + (k0 / 8) * 128;
              const uint32_t sboA = (uint32_t)((l == 0 ? Cfg::K0 : kH) / 8) * 128;
              const uint32_t sboB = (uint32_t)(Cfg::KW(l) / 8) * 128;
              const uint32_t bBase = tc::smem_u32(Wb + slot * kPP2Half);
              constexpr uint32_t idesc_h = tc::idesc_bf16(2 * kTile, kH);
              const uint32_t idesc = l < 3 ? idesc_h : tc::idesc_bf16(2 * kTile, OUTP);
              const uint64_t ad0 = tc::desc_kmajor(aBase, 128, sboA);
              const uint64_t bd0 = tc::desc_kmajor(bBase, 128, sboB);
#pragma unroll
              for (int s = 0; s < Cfg::KW(l) / 16; ++s)
                tc::mma_bf16_pair(acc, ad0 + (uint64_t)(16 * s), bd0 + (uint64_t)(16 * s), idesc,
                                  (c == 0 && s == 0) ? 0u : 1u);
              tc::commit_pair(&bar_f[slot]);
              slot = slot + 1 == (uint32_t)NBUF ? 0 : slot + 1;
            }
            if (*abort_flag) break;
            tc::commit_pair(&bar_acc[t]);
            if (l == 0) tc::commit_pair(&bar_xf[t]);
            ++e_done[t];
          }
        }
      }
      tc::commit_pair(&bar_done);
      tc::mbar_wait(&bar_done, 0, p.err, 0);
    }
    __syncwarp();
  } else {
    // ---- epilogue warps: (A, l), (B, l), (A, l + 1), ... ----
    const int quarter = warp & 3, grp = warp >> 2;
    const int trow = quarter * 32 + lane;  // tensor-memory lane = tile row
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    uint32_t ph_acc = 0;
    const int64_t mask = ((int64_t)1 << p.logn) - 1;
    // rows mode, warps of group 1: the fp32 pairs of s_j and of v at the stencil offsets that
    // P = alpha + c (v - s_j) needs, loaded one layer ahead (set a: tile A, set b: tile B)
    float a_sh = 0.f, a_sl = 0.f, a_vh[MU], a_vl[MU], b_sh = 0.f, b_sl = 0.f, b_vh[MU], b_vl[MU];
#pragma unroll
    for (int i = 0; i < MU; ++i) a_vh[i] = a_vl[i] = b_vh[i] = b_vl[i] = 0.f;
    auto prefetch = [&](int64_t row, float& sh, float& sl, float (&vh)[MU], float (&vl)[MU]) {
      if (row >= p.M) return;
      sh = __ldg(p.sh + row);
      sl = __ldg(p.sl + row);
#pragma unroll
      for (int i = 0; i < MU; ++i) {
        const int64_t nb = nb_index<2, 1>(row, i, p.logn, mask);
        vh[i] = __ldg(p.vh + nb);
        vl[i] = __ldg(p.vl + nb);
      }
    };
    for (int64_t pr = 0; pr < my_pairs; ++pr) {
      if (__shfl_sync(0xffffffffu, *abort_flag, 0)) break;
      for (int l = 0; l < 4; ++l) {
        for (int t = 0; t < 2; ++t) {
          if (!has(pr, t)) continue;
          if (MODE == kModeRows && grp == 1) {
            if (l == 2 && t == 1) {
              prefetch(tile_of(pr, 0) * kTile + trow, a_sh, a_sl, a_vh, a_vl);
            } else if (l == 3 && t == 0) {
              if (has(pr, 1))
                prefetch(tile_of(pr, 1) * kTile + trow, b_sh, b_sl, b_vh, b_vl);
              else
                prefetch(tile_of(pr, 0) * kTile + trow, a_sh, a_sl, a_vh, a_vl);
            }
          }
          wait_warp(&bar_acc[t], ph_acc >> t & 1, 8);
          ph_acc ^= 1u << t;
          tc::fence_after();
          const bool stop = __shfl_sync(0xffffffffu, *abort_flag, 0);
          const uint32_t taddr = tmem + lane_off + (uint32_t)(t * kH);
          const int64_t myrow = tile_of(pr, t) * kTile + trow;
          uint8_t* Ht = Hs + t * PPCfg::HBYTES;
          if (l < 3 && !stop) {
            const float* bl = bs + l * kH;
            uint32_t r[2][32];
            tc::tmem_ld32_nowait(taddr + grp * 32, r[0]);
#pragma unroll
            for (int pass = 0; pass < kNPass; ++pass) {
              const int cb = pass * kPassCols + grp * 32;
              tc::ld_wait(r[pass & 1]);
              if (pass + 1 < kNPass)
                tc::tmem_ld32_nowait(taddr + cb + kPassCols, r[(pass + 1) & 1]);
              const uint32_t* rr = r[pass & 1];
#pragma unroll
              for (int q8 = 0; q8 < 4; ++q8) {
                const int i = 8 * q8;
                const float4 b0 = *reinterpret_cast<const float4*>(bl + cb + i);
                const float4 b1 = *reinterpret_cast<const float4*>(bl + cb + i + 4);
                float z[8];
                uint4 q;
                q.x = relu_bf16x2(rr[i + 0], rr[i + 1], b0.x, b0.y, z[0], z[1]);
                q.y = relu_bf16x2(rr[i + 2], rr[i + 3], b0.z, b0.w, z[2], z[3]);
                q.z = relu_bf16x2(rr[i + 4], rr[i + 5], b1.x, b1.y, z[4], z[5]);
                q.w = relu_bf16x2(rr[i + 6], rr[i + 7], b1.z, b1.w, z[6], z[7]);
                *reinterpret_cast<uint4*>(Ht + tc::kmajor_off(trow, cb + i, kH)) = q;
                if (MODE == kModeBatch && myrow < p.M) {
#pragma unroll
                  for (int u = 0; u < 8; ++u) p.Zs[l][myrow * kH + cb + i + u] = z[u];
                  *reinterpret_cast<uint4*>(p.Hs[l] + myrow * kH + cb + i) = q;
                }
              }
            }
            // H_t is written and the accumulator read: the MMAs of (t, l + 1) may go
            tc::fence_async_smem();
          } else if (!stop) {
            // output layer: (alpha, c) and the rows, or the normalised outputs Y
            float y[OUTP];
            {
              uint32_t r[32];
              tc::tmem_ld32_nowait(taddr, r);
              tc::ld_wait(r);
#pragma unroll
              for (int i = 0; i < 32; ++i) y[i] = __uint_as_float(r[i]) + bs[3 * kH + i];
            }
            if (MODE == kModeBatch) {
              if (grp == 0 && myrow < p.M) {
#pragma unroll
                for (int o = 0; o < OUTP; ++o) p.Y[myrow * OUTP + o] = y[o];
              }
            } else {
              // de-normalise, unit-normalise alpha (c scaled alike: P^-1 C is invariant)
              float al[MU], cc[MU], nrm2 = 0.0f;
#pragma unroll
              for (int i = 0; i < MU; ++i) {
                al[i] = y[i] * nrm[2 + OUTP + i] + nrm[2 + i];
                cc[i] = y[MU + i] * nrm[2 + OUTP + MU + i] + nrm[2 + MU + i];
                nrm2 = fmaf(al[i], al[i], nrm2);
              }
              const float sc = nrm2 > 0.0f ? rsqrtf(nrm2) : 1.0f;
              // This warp's 32 rows of Q and C (group 0) or of P (group 1) are contiguous
              // blocks of 32 x MU doubles in global memory. When all 32 rows exist they are
              // staged in H_t (free: the layer-3 MMAs that read it have completed, and the
              // next writes to it follow this epilogue's arrival) and leave by one bulk copy
              // per block; otherwise each row is stored directly.
              constexpr int BLK = 32 * MU * 8;
              const int64_t wrow0 = tile_of(pr, t) * kTile + quarter * 32;
              const bool full = wrow0 + 32 <= p.M;
              double* stg = reinterpret_cast<double*>(Ht + (grp == 0 ? quarter : 8 + quarter) * BLK);
              if (grp == 0) {
#pragma unroll
                for (int i = 0; i < MU; ++i) {
                  // Q and C convert on the integer pipe while group 1 converts P on the FP64
                  // pipe: the two pipes run side by side
                  const double qv = f2d_int(al[i] * sc), cv = f2d_int(cc[i] * sc);
                  if (full) {
                    stg[lane * MU + i] = qv;
                    stg[4 * BLK / 8 + lane * MU + i] = cv;
                  } else if (myrow < p.M) {
                    __stcs(p.Q + myrow * MU + i, qv);
                    __stcs(p.C + myrow * MU + i, cv);
                  }
                }
              } else {
                // v[mu_j] - s_j from the fp32 pairs: the difference of the high parts is exact
                // when v and s_j are within a factor of two of each other (the usual case)
                const float sh = t == 0 ? a_sh : b_sh, sl = t == 0 ? a_sl : b_sl;
#pragma unroll
                for (int i = 0; i < MU; ++i) {
                  const float dv = ((t == 0 ? a_vh[i] : b_vh[i]) - sh) +
                                   ((t == 0 ? a_vl[i] : b_vl[i]) - sl);
                  const double pv = (double)(fmaf(cc[i] * sc, dv, al[i] * sc));
                  if (full)
                    stg[lane * MU + i] = pv;
                  else if (myrow < p.M)
                    __stcs(p.P + myrow * MU + i, pv);
                }
              }
              if (full) {
                tc::fence_async_smem();
                __syncwarp();
                if (lane == 0) {
                  if (grp == 0) {
                    tc::bulk_s2g(p.Q + wrow0 * MU, stg, BLK);
                    tc::bulk_s2g(p.C + wrow0 * MU, stg + 4 * BLK / 8, BLK);
                  } else {
                    tc::bulk_s2g(p.P + wrow0 * MU, stg, BLK);
                  }
                  tc::bulk_commit();
                  tc::bulk_wait_read();  // H_t may be written again once every warp arrived
                }
              }
            }
          }
          tc::fence_before();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive_cluster(&bar_e[t], 0);  // on the even CTA's bar_e
        }
      }
    }
    if (lane == 0) tc::bulk_wait_all();  // this warp's row stores have landed
  }
  tc::fence_before();
  __syncthreads();
  // neither CTA leaves (or releases the pair's tensor memory) while the other may still arrive
  // on its barriers or its MMAs read the other's shared memory
  tc::cluster_sync();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc_pair(tmem, 2 * kH);
}


// Per point j of a learned build: the normalised features of h^2 v_j and of h^2 s_j (bf16,
// s_j = snap(v_j)), and fp32 pairs v_j = vh + vl, s_j = sh + sl for the P epilogue. Since
// h^2 = 1/n^2 is a power of two, (float)(v h^2) = (float)v * h^2 exactly.
__global__ void k_point_features(const double* __restrict__ v, int64_t N, float h2f,
                                 const float* __restrict__ params, int64_t norm_off,
                                 __nv_bfloat16* __restrict__ xb, __nv_bfloat16* __restrict__ sb,
                                 float* __restrict__ vh, float* __restrict__ vl,
                                 float* __restrict__ sh, float* __restrict__ sl) {
  const float mu_x = params[norm_off], isig_x = 1.0f / params[norm_off + 1];
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x) {
    const double x = v[j];
    const float xf = (float)x;
    const double s = __dmul_rn((double)(4 * snap_m(x) + 2), kPi2);
    const float sf = (float)s;
    xb[j] = __float2bfloat16((xf * h2f - mu_x) * isig_x);
    sb[j] = __float2bfloat16(((float)(s * (double)h2f) - mu_x) * isig_x);
    vh[j] = xf;
    vl[j] = (float)(x - (double)xf);
    sh[j] = sf;
    sl[j] = (float)(s - (double)sf);
  }
}

// Learned-build inputs in the canonical K-major tile layout of the fused kernel, one thread per
// row (grid point j): the features xb over the 5^d patch of j (lexicographic offsets), then
// sb[j], zero-padded to K0. Consecutive threads are consecutive points along the last axis,
// so every patch offset is one coalesced load per warp. Rows beyond M (the last tile's tail)
// are zero.
template <int D>
__global__ void k_inputs_rows(const __nv_bfloat16* __restrict__ xb,
                              const __nv_bfloat16* __restrict__ sb, int logn, int64_t M,
                              uint8_t* __restrict__ Xt) {
  constexpr int NF = D == 2 ? 26 : 126, NP = NF - 1;
  constexpr int K0 = D == 2 ? 32 : 128;
  const int64_t mask = ((int64_t)1 << logn) - 1;
  const int64_t rows = (M + 2 * kTile - 1) / (2 * kTile) * (2 * kTile);  // whole tile pairs
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < rows;
       row += (int64_t)gridDim.x * blockDim.x) {
    const bool live = row < M;
    uint8_t* tile = Xt + (row / kTile) * (int64_t)(kTile * K0 * 2);
    const int r = (int)(row % kTile);
    // the five wrapped coordinates of each axis at offsets -2..2, already shifted into place:
    // the index of patch offset k (lexicographic, as nb_index<D, 2>) is then two ORs
    int64_t Y[D][5];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int sh = (D - 1 - a) * logn;
      const int64_t xa = (row >> sh) & mask;
#pragma unroll
      for (int o = 0; o < 5; ++o) Y[a][o] = ((xa + o - 2) & mask) << sh;
    }
#pragma unroll
    for (int k8 = 0; k8 < K0; k8 += 8) {
      __nv_bfloat16 f[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = k8 + i;
        __nv_bfloat16 x = __float2bfloat16(0.0f);
        if (live && k < NP) {
          const int64_t nb = D == 2 ? (Y[0][(k / 5) % 5] | Y[D - 1][k % 5])
                                    : (Y[0][(k / 25) % 5] | Y[D - 2][(k / 5) % 5] | Y[D - 1][k % 5]);
          x = xb[nb];
        }
        if (live && k == NP) x = sb[row];
        f[i] = x;
      }
      *reinterpret_cast<uint4*>(tile + tc::kmajor_off(r, k8, K0)) =
          *reinterpret_cast<const uint4*>(f);
    }
  }
}

// Training-batch inputs: the raw features Xraw[j][0..NF) normalised, bf16, written in the
// canonical K-major tile layout of the fused kernel (16 bytes = 8 features of one row per
// thread, consecutive threads writing consecutive 16-byte units) and row-major (X16) for the
// backward pass. Rows beyond M (the last tile's tail) are zero.
template <int D>
__global__ void k_inputs_batch(const float* __restrict__ Xraw, const float* __restrict__ params,
                               int64_t norm_off, int64_t M, uint8_t* __restrict__ Xt,
                               __nv_bfloat16* __restrict__ X16) {
  constexpr int NF = D == 2 ? 26 : 126;
  constexpr int K0 = D == 2 ? 32 : 128, KG = K0 / 8;
  const float mu_x = params[norm_off], isig_x = 1.0f / params[norm_off + 1];
  const int64_t units = (M + kTile - 1) / kTile * kTile * KG;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < units;
       e += (int64_t)gridDim.x * blockDim.x) {
    // e = ((tile * 16 + row / 8) * KG + kg) * 8 + row % 8
    const int64_t qv = e >> 3;
    const int kg = (int)(qv % KG);
    const int64_t row = (qv / KG) * 8 + (e & 7);
    __nv_bfloat16 f[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = kg * 8 + i;
      f[i] = __float2bfloat16(row < M && k < NF ? (Xraw[row * NF + k] - mu_x) * isig_x : 0.0f);
    }
    const uint4 q = *reinterpret_cast<const uint4*>(f);
    reinterpret_cast<uint4*>(Xt)[e] = q;
    if (row < M) reinterpret_cast<uint4*>(X16 + row * K0)[kg] = q;
  }
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
  uint64_t wait_ns = lsp::tc::kWaitLimitNs;  // operand-wait limit of the fused kernel
  int schedule = 1;  // 2D: 1 = two tiles in flight (k_mlp_pp), 0 = one tile at a time,
                     // 2 = two 256-row tiles in flight on a CTA pair (k_mlp_pp2, rows mode)
  // training workspace
  int64_t cap = 0;
  lsp::DevBuf X16, XT, Xt, Zs[3], Hs[3], HT[3], Y, dY16, dYT, dY32, G, dZ16, dZT, dZ32;
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
  if (lsp::alloc_should_fail() || cudaMalloc(&b.p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  b.bytes = bytes;
  return true;
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
  p.wait_ns = m->wait_ns;
  return p;
}

// Bytes of the canonical input tiles for `rows` rows (whole tiles).
// Whole pairs of 128-row tiles (the CTA-pair kernel reads both tiles of a 256-row super-tile;
// rows beyond M are zero).
size_t input_tile_bytes(int d, int64_t rows) {
  return (size_t)((rows + 2 * kTile - 1) / (2 * kTile)) * 2 * kTile * dims_for(d).K0 * 2;
}

template <int D, int MODE>
cudaError_t launch_fused(lsp_mlp* m, const FusedParams& p, int64_t rows) {
  if constexpr (D == 2 && MODE == kModeRows) {
    if (m->schedule == 2) {
      const size_t smem = PPCfg::smem;
      cudaError_t e = cudaFuncSetAttribute(k_mlp_pp2<MODE>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      const int64_t super = ((rows + kTile - 1) / kTile + 1) / 2;
      const int pairs = (int)(super < 76 ? super : 76);  // one CTA pair per TPC
      k_mlp_pp2<MODE><<<2 * (pairs < 1 ? 1 : pairs), kPPThreads, smem, m->stream>>>(p);
      return cudaGetLastError();
    }
  }
  if (D == 2 && m->schedule >= 1) {  // batch mode of schedule 2 runs the one-CTA kernel
    const size_t smem = PPCfg::smem;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_pp<MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (rows + kTile - 1) / kTile;
    int grid = (int)(tiles < 152 ? tiles : 152);
    if (grid < 1) grid = 1;
    k_mlp_pp<MODE><<<grid, kPPThreads, smem, m->stream>>>(p);
    return cudaGetLastError();
  }
  const size_t smem = FusedCfg<D>::smem;
  cudaError_t e = cudaFuncSetAttribute(k_mlp_fused<D, MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (rows + kTile - 1) / kTile;
  // persistent: one CTA per SM (its tensor memory takes all 512 columns)
  int grid = (int)(tiles < 152 ? tiles : 152);
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
            grow(m->Xt, input_tile_bytes(d.d, B)) &&
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

// Training-mode forward: normalised bf16 inputs (canonical tiles and row-major), then the fused
// network, saving z and h of every hidden layer.
cudaError_t batch_forward(lsp_mlp* m, const float* X_dev, int64_t batch, float* Y_dev) {
  FusedParams p = fused_params(m);
  p.M = batch;
  p.Xt = (const uint8_t*)m->Xt.p;
  p.Y = Y_dev;
  for (int l = 0; l < 3; ++l) {
    p.Zs[l] = (float*)m->Zs[l].p;
    p.Hs[l] = (__nv_bfloat16*)m->Hs[l].p;
  }
  __nv_bfloat16* X16 = (__nv_bfloat16*)m->X16.p;
  if (m->dm.d == 2)
    k_inputs_batch<2><<<152 * 8, 256, 0, m->stream>>>(X_dev, p.params, p.norm_off, batch,
                                                      (uint8_t*)p.Xt, X16);
  else
    k_inputs_batch<3><<<152 * 8, 256, 0, m->stream>>>(X_dev, p.params, p.norm_off, batch,
                                                      (uint8_t*)p.Xt, X16);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return m->dm.d == 2 ? launch_fused<2, kModeBatch>(m, p, batch)
                      : launch_fused<3, kModeBatch>(m, p, batch);
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
                         &m->loss, &m->X16, &m->XT, &m->Xt, &m->Y, &m->dY16, &m->dYT, &m->dY32, &m->G,
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
  MCUDA(m, batch_forward(m, X_dev, batch, Y_dev));
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
  MCUDA(m, batch_forward(m, X_dev, batch, (float*)m->Y.p));
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

lsp_status lsp_mlp_set_schedule(lsp_mlp* m, int schedule) {
  if (!m || schedule < 0 || schedule > 2) return LSP_ERR_ARG;
  m->schedule = schedule;
  return LSP_OK;
}

lsp_status lsp_mlp_set_wait_limit(lsp_mlp* m, uint64_t ns) {
  if (!m) return LSP_ERR_ARG;
  m->wait_ns = ns ? ns : lsp::tc::kWaitLimitNs;
  return LSP_OK;
}

}  // extern "C"

namespace lsp {

// Learned build: the fused network over every point writes Q, C and P directly.
cudaError_t launch_learned_rows(lsp_ctx* c, lsp_mlp* m) {
  // the weights may still be written by the network's own stream (training, set_params)
  cudaError_t se = cudaStreamSynchronize(m->stream);
  if (se != cudaSuccess) return se;
  FusedParams p = fused_params(m);
  const int64_t N = c->geo.N;
  p.M = N;
  int logn = 0;
  while ((1 << logn) < c->geo.n) ++logn;
  p.logn = logn;
  p.Q = (double*)c->Q.p;
  p.C = (double*)c->C.p;
  p.P = (double*)c->P.p;
  p.err = (int*)c->counts.p + kErrWord;
  // learn_in: the input tiles, then per point xb, sb (bf16) and vh, vl, sh, sl (fp32)
  const size_t xt_bytes = input_tile_bytes(c->geo.d, N);
  const size_t pts = ((size_t)N * 2 + 255) / 256 * 256, ptf = ((size_t)N * 4 + 255) / 256 * 256;
  if (!ensure(c, c->learn_in, xt_bytes + 2 * pts + 4 * ptf)) return cudaErrorMemoryAllocation;
  uint8_t* base = (uint8_t*)c->learn_in.p;
  p.Xt = base;
  __nv_bfloat16* xb = (__nv_bfloat16*)(base + xt_bytes);
  __nv_bfloat16* sb = (__nv_bfloat16*)(base + xt_bytes + pts);
  float* f32 = (float*)(base + xt_bytes + 2 * pts);
  float* vh = f32;
  float* vl = (float*)((uint8_t*)f32 + ptf);
  float* sh = (float*)((uint8_t*)f32 + 2 * ptf);
  float* sl = (float*)((uint8_t*)f32 + 3 * ptf);
  p.vh = vh;
  p.vl = vl;
  p.sh = sh;
  p.sl = sl;
  const float h2f = (float)(1.0 / ((double)c->geo.n * c->geo.n));
  cudaStream_t saved = m->stream;
  m->stream = c->stream;
  int t0 = timer_begin(c, "mlp_features");
  k_point_features<<<152 * 8, 256, 0, c->stream>>>((const double*)c->v.p, N, h2f, p.params,
                                                   p.norm_off, xb, sb, vh, vl, sh, sl);
  cudaError_t e = cudaGetLastError();
  timer_end(c, t0);
  int t1 = timer_begin(c, "mlp_inputs");
  if (e == cudaSuccess) {
    if (c->geo.d == 2)
      k_inputs_rows<2><<<152 * 8, 256, 0, c->stream>>>(xb, sb, logn, N, base);
    else
      k_inputs_rows<3><<<152 * 8, 256, 0, c->stream>>>(xb, sb, logn, N, base);
    e = cudaGetLastError();
  }
  timer_end(c, t1);
  if (e == cudaSuccess) {
    int t = timer_begin(c, "mlp_rows");
    e = c->geo.d == 2 ? launch_fused<2, kModeRows>(m, p, c->geo.N)
                      : launch_fused<3, kModeRows>(m, p, c->geo.N);
    timer_end(c, t);
  }
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
