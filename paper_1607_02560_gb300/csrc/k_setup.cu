// Steps a1-a2 and the domain bookkeeping of a3:
//  * potential statistics v_min, v_max, mean (Sec. 3 mean shift; Sec. 4.1 range of S),
//  * per-point lattice shift m_j = snap(v_j) for the per-point policy (Sec. 4.1, G_{v_j}),
//  * stream compaction of flag arrays into sorted index lists,
//  * marking of the integer domains E_k of the lattice-separable kernel-vector stages,
//  * the reciprocal table w(l) = 1 / (pi^2 (4 l + 2)) (Sec. 3 definition of G_s on the lattice).
#include <float.h>

#include "lsp_internal.h"

namespace lsp {
namespace {

constexpr int kThreads = 256;
constexpr int kTileFlags = kThreads * 16;  // flags per compaction tile (one uint4 per thread)

__device__ __forceinline__ double warp_min(double x) {
  for (int o = 16; o > 0; o >>= 1) x = fmin(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}
__device__ __forceinline__ double warp_max(double x) {
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}
__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Per-block partial min / max / sum / count of non-finite values, 4 doubles per block. With
// vcopy, v is also stored there (v read from page-locked host memory over the host link, so
// the upload and the statistics take one pass and no copy engine).
__device__ void stats_partial(const double* __restrict__ v, int64_t N, double* __restrict__ part,
                              double* __restrict__ vcopy) {
  double mn = DBL_MAX, mx = -DBL_MAX, sm = 0.0, bad = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * kThreads) {
    const double x = v[j];
    if (vcopy) vcopy[j] = x;
    if (!isfinite(x)) {
      bad += 1.0;
      continue;
    }
    mn = fmin(mn, x);
    mx = fmax(mx, x);
    sm += x;
  }
  __shared__ double red[4][kThreads / 32];
  mn = warp_min(mn);
  mx = warp_max(mx);
  sm = warp_sum(sm);
  bad = warp_sum(bad);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    red[0][w] = mn;
    red[1][w] = mx;
    red[2][w] = sm;
    red[3][w] = bad;
  }
  __syncthreads();
  if (w == 0) {
    mn = l < kThreads / 32 ? red[0][l] : DBL_MAX;
    mx = l < kThreads / 32 ? red[1][l] : -DBL_MAX;
    sm = l < kThreads / 32 ? red[2][l] : 0.0;
    bad = l < kThreads / 32 ? red[3][l] : 0.0;
    mn = warp_min(mn);
    mx = warp_max(mx);
    sm = warp_sum(sm);
    bad = warp_sum(bad);
    if (l == 0) {
      part[4 * blockIdx.x + 0] = mn;
      part[4 * blockIdx.x + 1] = mx;
      part[4 * blockIdx.x + 2] = sm;
      part[4 * blockIdx.x + 3] = bad;
    }
  }
}

// Reduces the partials to (min, max, sum, non-finite count) in out[0..3], and also in
// host_out[0..3] (page-locked host memory, device address) when given, so that the host reads
// them without a copy. The partials are taken in block order, so the sum does not depend on
// which block finished last.
__device__ void stats_final(const double* part, int nb, double* out, double* host_out) {
  double mn = DBL_MAX, mx = -DBL_MAX, sm = 0.0, bad = 0.0;
  for (int b = threadIdx.x; b < nb; b += kThreads) {
    mn = fmin(mn, part[4 * b + 0]);
    mx = fmax(mx, part[4 * b + 1]);
    sm += part[4 * b + 2];
    bad += part[4 * b + 3];
  }
  __shared__ double red[4][kThreads / 32];
  mn = warp_min(mn);
  mx = warp_max(mx);
  sm = warp_sum(sm);
  bad = warp_sum(bad);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    red[0][w] = mn;
    red[1][w] = mx;
    red[2][w] = sm;
    red[3][w] = bad;
  }
  __syncthreads();
  if (w == 0) {
    mn = l < kThreads / 32 ? red[0][l] : DBL_MAX;
    mx = l < kThreads / 32 ? red[1][l] : -DBL_MAX;
    sm = l < kThreads / 32 ? red[2][l] : 0.0;
    bad = l < kThreads / 32 ? red[3][l] : 0.0;
    mn = warp_min(mn);
    mx = warp_max(mx);
    sm = warp_sum(sm);
    bad = warp_sum(bad);
    if (l == 0) {
      out[0] = mn;
      out[1] = mx;
      out[2] = sm;
      out[3] = bad;
      if (host_out) {
        host_out[0] = mn;
        host_out[1] = mx;
        host_out[2] = sm;
        host_out[3] = bad;
      }
    }
  }
}

// One launch: every block writes its partial, and the block that finishes last (a ticket
// counter, reset by that block for the next call) reduces them all.
__global__ void __launch_bounds__(kThreads) k_stats(const double* __restrict__ v, int64_t N,
                                                    double* __restrict__ part,
                                                    double* __restrict__ vcopy,
                                                    double* __restrict__ out,
                                                    double* __restrict__ host_out,
                                                    unsigned int* __restrict__ ticket) {
  stats_partial(v, N, part, vcopy);
  __shared__ bool last;
  __threadfence();  // this block's partial is visible before its ticket is taken
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  stats_final(part, gridDim.x, out, host_out);
  if (threadIdx.x == 0) *ticket = 0u;
}

// Lattice index of the resonance-free shift (4m+2) pi^2 nearest to x (Sec. 4.1); halves away
// from zero. Explicit round-to-nearest intrinsics keep the decision identical to a plain
// IEEE evaluation of (x / pi^2 - 2) / 4 (no contraction into fused operations).
__device__ __forceinline__ int64_t snap_m(double x) {
  // Fast path: fma(x, 1/(4 pi^2), -1/2) is within a few ulp of the exact (x/pi^2 - 2)/4, so
  // its nearest integer is the exact one unless it lies next to a half-integer.
  const double yf = fma(x, kQuarterInvPi2, -0.5);
  const double r = rint(yf);
  if (0.5 - fabs(yf - r) > 1e-14 * fabs(yf) + 1e-14) return (int64_t)r;
  const double y = __dmul_rn(__dsub_rn(__ddiv_rn(x, kPi2), 2.0), 0.25);
  return (int64_t)round(y);
}

// The host derived [mlo, mlo + R) from snap(v_min) and snap(v_max) with the same IEEE
// operations; an index outside it would mean the two disagree, and is recorded in *err.
__global__ void __launch_bounds__(kThreads) k_mark_local(const double* __restrict__ v, int64_t N,
                                                         int64_t mlo, int64_t R,
                                                         uint8_t* __restrict__ flag,
                                                         int32_t* __restrict__ err) {
  for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * kThreads) {
    const int64_t r = snap_m(__ldg(v + j)) - mlo;
    if (r >= 0 && r < R)
      flag[r] = 1;
    else
      atomicOr(err, 1);
  }
}

// E_{k-1} gets every l + p^2 for l in the list of E_k and p in [0, P).
__global__ void __launch_bounds__(kThreads) k_mark_stage(const int32_t* __restrict__ list,
                                                         const int32_t* __restrict__ count, int P,
                                                         int64_t lo_prev,
                                                         uint8_t* __restrict__ flag_prev) {
  const int64_t cnt = *count;
  for (int p = blockIdx.y; p < P; p += gridDim.y) {
    const int64_t p2 = (int64_t)p * p;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * kThreads) {
      flag_prev[(int64_t)__ldg(list + i) + p2 - lo_prev] = 1;
    }
  }
}

__device__ __forceinline__ int count16(uint4 q) {
  return __popc(q.x & 0x01010101u) + __popc(q.y & 0x01010101u) + __popc(q.z & 0x01010101u) +
         __popc(q.w & 0x01010101u);
}

// Compaction pass 1: number of set flags in each tile of kTileFlags.
__global__ void __launch_bounds__(kThreads) k_compact_count(const uint8_t* __restrict__ flag,
                                                            int32_t* __restrict__ tilecnt) {
  const uint4 q = reinterpret_cast<const uint4*>(flag)[(int64_t)blockIdx.x * kThreads + threadIdx.x];
  int c = count16(q);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  __shared__ int red[kThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    tilecnt[blockIdx.x] = s;
  }
}

// Compaction pass 2: exclusive scan of the tile counts (one block), total into *count.
__global__ void __launch_bounds__(1024) k_compact_scan(int32_t* __restrict__ tilecnt, int ntiles,
                                                       int32_t* __restrict__ count) {
  __shared__ int part[1024];
  const int per = (ntiles + 1023) / 1024;
  const int b0 = threadIdx.x * per;
  int s = 0;
  for (int i = 0; i < per; ++i)
    if (b0 + i < ntiles) s += tilecnt[b0 + i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int add = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += add;
    __syncthreads();
  }
  int run = part[threadIdx.x] - s;  // exclusive
  for (int i = 0; i < per; ++i) {
    if (b0 + i < ntiles) {
      int c = tilecnt[b0 + i];
      tilecnt[b0 + i] = run;
      run += c;
    }
  }
  if (threadIdx.x == 1023) *count = part[1023];
}

// Compaction pass 3: write list[pos] = lo + r for every set flag r (in increasing r), and
// idx_of[r] = pos (or -1) when idx_of is given.
__global__ void __launch_bounds__(kThreads) k_compact_write(const uint8_t* __restrict__ flag,
                                                            const int32_t* __restrict__ tileoff,
                                                            int64_t lo, int64_t range,
                                                            int32_t* __restrict__ list,
                                                            int32_t* __restrict__ idx_of) {
  const int64_t base = (int64_t)blockIdx.x * kTileFlags + (int64_t)threadIdx.x * 16;
  const uint4 q = reinterpret_cast<const uint4*>(flag)[(int64_t)blockIdx.x * kThreads + threadIdx.x];
  const int c = count16(q);
  int incl = c;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  __shared__ int wsum[kThreads / 32];
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  int woff = 0;
  for (int i = 0; i < w; ++i) woff += wsum[i];
  int pos = tileoff[blockIdx.x] + woff + incl - c;
  const uint32_t words[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int64_t r = base + k;
    const bool set = (words[k >> 2] >> (8 * (k & 3))) & 1u;
    if (r < range) {
      if (set) {
        list[pos] = (int32_t)(lo + r);
        if (idx_of) idx_of[r] = pos;
        ++pos;
      } else if (idx_of) {
        idx_of[r] = -1;
      }
    }
  }
}

// w(l) = 1 / (pi^2 (4 l + 2)): FP64 interleaved with w^2, or w alone rounded to FP32.
__global__ void __launch_bounds__(kThreads) k_wtable64(int64_t lo, int64_t range,
                                                       double2* __restrict__ w) {
  for (int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x; r < range;
       r += (int64_t)gridDim.x * kThreads) {
    const double l4 = (double)(4 * (lo + r) + 2);  // exact integer
    const double x = 1.0 / __dmul_rn(kPi2, l4);
    w[r] = make_double2(x, x * x);
  }
}
__global__ void __launch_bounds__(kThreads) k_wtable32(int64_t lo, int64_t range,
                                                       float* __restrict__ w) {
  for (int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x; r < range;
       r += (int64_t)gridDim.x * kThreads) {
    const double l4 = (double)(4 * (lo + r) + 2);
    w[r] = (float)(1.0 / __dmul_rn(kPi2, l4));
  }
}

// Double words (hi, lo floats) of w and w^2 from their FP64 values, interleaved per l.
__global__ void __launch_bounds__(kThreads) k_wtable_dw(int64_t lo, int64_t range,
                                                        float4* __restrict__ w) {
  for (int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x; r < range;
       r += (int64_t)gridDim.x * kThreads) {
    const double l4 = (double)(4 * (lo + r) + 2);
    const double x = 1.0 / __dmul_rn(kPi2, l4), x2 = x * x;
    const float xh = (float)x, x2h = (float)x2;
    w[r] = make_float4(xh, (float)(x - (double)xh), x2h, (float)(x2 - (double)x2h));
  }
}

int grid_for(int64_t work, int per_block = kThreads) {
  int64_t b = (work + per_block - 1) / per_block;
  const int64_t cap = 152 * 32;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// Zeroes n 32-bit words. A kernel rather than a memset, so that the build never waits behind
// host copies queued on the copy engines.
__global__ void __launch_bounds__(kThreads) k_zero_u32(uint32_t* __restrict__ p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads)
    p[i] = 0u;
}

// dst[0, n) = src[0, n) (doubles; both 16-byte aligned): pairs by every thread, an odd last
// element by thread 0.
__global__ void __launch_bounds__(kThreads) k_copy_f64(const double* __restrict__ src,
                                                       double* __restrict__ dst, int64_t n) {
  const int64_t n2 = n / 2;
  const double2* s2 = reinterpret_cast<const double2*>(src);
  double2* d2 = reinterpret_cast<double2*>(dst);
  const int64_t t0 = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  for (int64_t i = t0; i < n2; i += (int64_t)gridDim.x * kThreads) d2[i] = s2[i];
  if (t0 == 0 && (n & 1)) dst[n - 1] = src[n - 1];
}

}  // namespace

cudaError_t launch_stats(lsp_ctx* c, int nblocks, const double* src) {
  int t = timer_begin(c, "stats");
  double* vd = (double*)c->v.p;
  double* st = (double*)c->stats.p;
  k_stats<<<nblocks, kThreads, 0, c->stream>>>(src, c->geo.N, (double*)c->stats_part.p,
                                               src == vd ? nullptr : vd, st, c->h_stats_dev,
                                               (unsigned int*)(st + 4));
  timer_end(c, t);
  return cudaGetLastError();
}

cudaError_t launch_zero(lsp_ctx* c, void* p, size_t bytes) {
  const int64_t n = (int64_t)(bytes / 4);
  int t = timer_begin(c, "zero");
  k_zero_u32<<<grid_for(n), kThreads, 0, c->stream>>>((uint32_t*)p, n);
  timer_end(c, t);
  return cudaGetLastError();
}

cudaError_t launch_copy_f64(lsp_ctx* c, const double* src, double* dst, int64_t n) {
  int t = timer_begin(c, "copy_rows");
  k_copy_f64<<<grid_for((n + 1) / 2), kThreads, 0, c->stream>>>(src, dst, n);
  timer_end(c, t);
  return cudaGetLastError();
}

cudaError_t launch_mark_local(lsp_ctx* c) {
  int t = timer_begin(c, "mark_local");
  k_mark_local<<<grid_for(c->geo.N), kThreads, 0, c->stream>>>(
      (const double*)c->v.p, c->geo.N, c->mrange.lo, c->mrange.size(), (uint8_t*)c->shift_flag.p,
      (int32_t*)c->counts.p + kErrWord);
  timer_end(c, t);
  return cudaGetLastError();
}

// flags must hold a multiple of kTileFlags bytes (zero beyond `range`); tile scratch lives in
// the context's `counts` buffer after its first 16 entries.
cudaError_t launch_compact(lsp_ctx* c, const uint8_t* flags, int64_t lo, int64_t range,
                           int32_t* list, int32_t* count, int32_t* idx_of) {
  const int ntiles = (int)((range + kTileFlags - 1) / kTileFlags);
  int32_t* tiles = (int32_t*)c->counts.p + 16;
  int t = timer_begin(c, "compact");
  k_compact_count<<<ntiles, kThreads, 0, c->stream>>>(flags, tiles);
  k_compact_scan<<<1, 1024, 0, c->stream>>>(tiles, ntiles, count);
  k_compact_write<<<ntiles, kThreads, 0, c->stream>>>(flags, tiles, lo, range, list, idx_of);
  timer_end(c, t);
  return cudaGetLastError();
}

cudaError_t launch_mark_stage(lsp_ctx* c, const int32_t* list, const int32_t* count, int64_t cap,
                              int64_t lo_prev, uint8_t* flag_prev) {
  const int P = c->geo.P;
  int gx = (int)((cap + kThreads - 1) / kThreads);
  if (gx > 1024) gx = 1024;
  if (gx < 1) gx = 1;
  dim3 grid(gx, P < 4096 ? P : 4096);
  int t = timer_begin(c, "mark_stage");
  k_mark_stage<<<grid, kThreads, 0, c->stream>>>(list, count, P, lo_prev, flag_prev);
  timer_end(c, t);
  return cudaGetLastError();
}

cudaError_t launch_wtable(lsp_ctx* c, int64_t lo, int64_t range, void* w, int prec) {
  int t = timer_begin(c, "wtable");
  if (prec == kPrecFP32)
    k_wtable32<<<grid_for(range), kThreads, 0, c->stream>>>(lo, range, (float*)w);
  else if (prec == kPrecDword)
    k_wtable_dw<<<grid_for(range), kThreads, 0, c->stream>>>(lo, range, (float4*)w);
  else
    k_wtable64<<<grid_for(range), kThreads, 0, c->stream>>>(lo, range, (double2*)w);
  timer_end(c, t);
  return cudaGetLastError();
}

}  // namespace lsp
