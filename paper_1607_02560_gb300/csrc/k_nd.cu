// Numeric phases of the nested dissection of P (Sec. 3, Eq. QC; Fig. nd; Table cost), see
// nd.h for the tree and the front layout:
//  - assembly: a front = its children's Schur complements (extend-add through the ring maps)
//    plus P's entries listed for it;
//  - partial inversion of each front on its eliminated set E with row pivoting inside E
//    (Gauss-Jordan sweep): in shared memory for small fronts, else in blocked steps of
//    kNdPanel pivots (panel choice, row block, rank-kNdPanel update of the whole front);
//  - the solve: one matrix-vector product per front going up the tree, one coming down.
// Every reduction runs in a fixed order, so a factorisation and a solve are deterministic.
#include <math.h>
#include <stdio.h>

#include "nd.h"

namespace lsp {
namespace {

constexpr int NP = kNdPanel;

__global__ void k_nd_extend(double* __restrict__ F, const double* __restrict__ Fc,
                            const int32_t* __restrict__ inv, int count, int f, int nchild,
                            int fc, int sc) {
  const int64_t ff = (int64_t)f * f, total = (int64_t)count * ff;
  const int64_t fcc = (int64_t)fc * fc;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = idx / ff;
    const int rem = (int)(idx - p * ff);
    const int i = rem / f, j = rem - i * f;
    const int32_t* iv = inv + p * f * 2;
    double acc = 0.0;
    for (int c = 0; c < nchild; ++c) {
      const int ai = iv[i * 2 + c], aj = iv[j * 2 + c];
      if (ai >= 0 && aj >= 0) {
        const int64_t child = nchild == 1 ? p : 2 * p + c;
        acc += Fc[child * fcc + (int64_t)(sc + ai) * fc + sc + aj];
      }
    }
    F[idx] = acc;
  }
}

__global__ void k_nd_scatter(double* __restrict__ F, const double* __restrict__ rows,
                             const int32_t* __restrict__ dst, const int32_t* __restrict__ src,
                             int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    F[dst[e]] += rows[src[e]];
}

// argmax of |value| over a warp with ties to the smaller index
__device__ __forceinline__ void warp_argmax_f(float& best, int& bi) {
  for (int off = 16; off > 0; off >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, off);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
    if (ob > best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
  }
}
__device__ __forceinline__ void warp_argmax(double& best, int& bi) {
  for (int off = 16; off > 0; off >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, off);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
    if (ob > best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
  }
}

// Partial inversion of one front (f <= kNdSmallFront) in shared memory, one pivot at a time.
// Pivot k: the row of largest |F[i][k]| among the rows k..s-1 still unpivoted; then
//   F[k][k] <- 1/F[k][k], F[k][j] <- F[k][j]/F[k][k], F[i][k] <- -F[i][k]/F[k][k],
//   F[i][j] <- F[i][j] - F[i][k] F[k][j]/F[k][k]   (i, j != k).
__global__ void __launch_bounds__(256) k_nd_sweep_small(double* __restrict__ fronts, int f, int s,
                                                        int32_t* __restrict__ perm,
                                                        int32_t* __restrict__ err) {
  extern __shared__ double sm[];
  double* F = sm;
  double* colk = F + f * f;
  double* rowk = colk + f;
  __shared__ int sperm[kNdSmallFront];
  __shared__ int piv, bad;
  __shared__ double spiv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
  double* G = fronts + (int64_t)blockIdx.x * f * f;
  for (int e = tid; e < f * f; e += nt) F[e] = G[e];
  for (int e = tid; e < s; e += nt) sperm[e] = e;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < s; ++k) {
    if (warp == 0) {
      double best = -1.0;
      int bi = s;
      for (int i = k + lane; i < s; i += 32) {
        const double a = fabs(F[i * f + k]);
        if (a > best) {
          best = a;
          bi = i;
        }
      }
      warp_argmax(best, bi);
      if (lane == 0) {
        if (!(best > 0.0) || !isfinite(best)) {
          bad = 1;
          atomicOr(err, 1);
        }
        piv = bi < s ? bi : k;
        spiv = 1.0 / F[piv * f + k];  // the one FP64 division of this pivot
      }
    }
    __syncthreads();
    if (bad) break;
    const int p = piv;
    if (p != k) {
      for (int j = tid; j < f; j += nt) {
        const double a = F[k * f + j];
        F[k * f + j] = F[p * f + j];
        F[p * f + j] = a;
      }
      if (tid == 0) {
        const int t = sperm[k];
        sperm[k] = sperm[p];
        sperm[p] = t;
      }
      __syncthreads();
    }
    const double dinv = spiv;
    for (int j = tid; j < f; j += nt) {
      rowk[j] = F[k * f + j] * dinv;
      colk[j] = F[j * f + k];
    }
    __syncthreads();
    for (int i = warp; i < f; i += nt / 32) {
      double* Fi = F + i * f;
      if (i == k) {
        for (int j = lane; j < f; j += 32) Fi[j] = j == k ? dinv : rowk[j];
      } else {
        const double ci = colk[i];
        for (int j = lane; j < f; j += 32) Fi[j] = j == k ? -ci * dinv : fma(-ci, rowk[j], Fi[j]);
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < f * f; e += nt) G[e] = F[e];
  for (int e = tid; e < s; e += nt) perm[(int64_t)blockIdx.x * s + e] = sperm[e];
}

// ---- blocked partial inversion: one step eliminates the pivot columns K = [k, k + nb) ----
// swaps layout per front: [0] = number of entries q, then dst[q] at 1 + q, src[q] at
// 1 + 2 NP + q: after the step, position dst holds the row that was at position src.
constexpr int kSwapInts = 1 + 4 * NP;

// FP32 value of x for ranking pivot candidates, from the high word of the IEEE double: sign,
// exponent rebased from 1023 to 127, the top 20 fraction bits (relative error < 2^-20);
// magnitudes below the FP32 normal range give 0, above it infinity. Integer operations only.
__device__ __forceinline__ float rank_f32(double x) {
  const int hi = __double2hiint(x);
  const int e = ((hi >> 20) & 0x7ff) - (1023 - 127);
  const unsigned sign = (unsigned)hi & 0x80000000u;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned)e << 23) | (((unsigned)hi & 0xfffffu) << 3));
}

// Part 1, one CTA per front: choose nb pivot rows among positions k..s-1 by partial pivoting
// on the panel F[k.., K]; record the row exchanges, update perm, write the column block
// cbuf[x][c] = F[src(x)][k + c] of the exchanged rows x, and the inverse of the pivot block.
// The pivot rows come from a trial elimination of the panel in FP32: it only ranks candidate
// rows by magnitude, while every value the factorisation keeps is FP64, computed from the
// original entries (the pivot-block inverse here, the row block and the update in parts 2 and
// 3). Each thread keeps its panel rows (row tid + t * 256, t < kPanelRows) in registers and
// publishes its best candidate row to shared memory, so a pivot costs one block barrier.
// Common end of part 1 (after the pivot rows sel[0..nb) are known, block-synchronised):
// row exchanges, the column block of the exchanged rows, the FP64 pivot-block inverse.
__device__ __forceinline__ void panel_tail(const double* __restrict__ F, int f, int s, int k,
                                           int nb, int64_t fid, const int* sel,
                                           int32_t* __restrict__ perm, double* __restrict__ cbuf,
                                           double* __restrict__ pinv,
                                           int32_t* __restrict__ swaps, int32_t* __restrict__ err) {
  constexpr int NT = 256;
  __shared__ int nq;
  __shared__ int dstp[2 * NP], srcp[2 * NP];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // row exchanges (warp 0): position k + j takes the row chosen j-th; the rows of K that were
  // not chosen move, in increasing position order, to the positions the chosen rows left
  // outside K (taken in choice order)
  if (warp == 0) {
    const bool act = lane < nb;
    const int ps = act ? k + sel[lane] : 0;
    const bool inK = act && ps < k + nb;
    const unsigned selK = __reduce_or_sync(0xffffffffu, inK ? 1u << (ps - k) : 0u);
    const unsigned full = nb >= 32 ? 0xffffffffu : (1u << nb) - 1u;
    const unsigned displaced = ~selK & full;  // K positions whose rows were not chosen
    const unsigned outb = __ballot_sync(0xffffffffu, act && !inK);
    const int rank = __popc(outb & ((1u << lane) - 1u));  // among the chosen rows outside K
    int dpos = -1;
    if (act && !inK) {  // the rank-th displaced position of K
      unsigned mk = displaced;
      for (int t = 0; t < rank; ++t) mk &= mk - 1u;
      dpos = k + __ffs(mk) - 1;
    }
    const int nout = __popc(outb);
    int32_t* pf = perm + fid * s;
    int32_t* sw = swaps + fid * kSwapInts;
    const int old_sel = act ? pf[ps] : 0;
    const int old_dis = dpos >= 0 ? pf[dpos] : 0;
    __syncwarp();
    if (act) {
      dstp[lane] = k + lane;
      srcp[lane] = ps;
      pf[k + lane] = old_sel;
    }
    if (dpos >= 0) {
      dstp[nb + rank] = ps;
      srcp[nb + rank] = dpos;
      pf[ps] = old_dis;
    }
    __syncwarp();
    const int qq = nb + nout;
    if (lane == 0) {
      nq = qq;
      sw[0] = qq;
    }
    for (int a = lane; a < qq; a += 32) {
      sw[1 + a] = dstp[a];
      sw[1 + 2 * NP + a] = srcp[a];
    }
  }
  __syncthreads();
  const int q = nq;
  // the column block of the exchanged rows (the other rows are read in place by part 2)
  double* cb = cbuf + fid * (int64_t)f * NP;
  for (int e = tid; e < q * NP; e += NT) {
    const int a = e / NP, c = e % NP;
    cb[(int64_t)dstp[a] * NP + c] = c < nb ? F[(int64_t)srcp[a] * f + k + c] : 0.0;
  }
  // inverse of the pivot block A (FP64): Gauss-Jordan on [A | I], one element per thread in
  // each half (rows r = tid / 16, columns c and c + 16), no row exchanges: pivot j is taken in
  // the unpivoted row p_j of largest |a_pj,j| (integer comparison of magnitude bits), row p_j
  // is scaled by one reciprocal, column j is eliminated from the other rows. The left block
  // ends as a permutation with a 1 at (p_j, j), so row j of A^-1 is the right block's row p_j.
  __shared__ double aug[NP][2 * NP + 1];
  __shared__ double gd;
  __shared__ int gp, rowpiv[NP];
  const int gr = tid / NP, gc = tid % NP;  // 256 threads = 16 rows x 16 column pairs
  {
    int src = k + gr;
    for (int e = 0; e < q; ++e)
      if (dstp[e] == k + gr) src = srcp[e];
    aug[gr][gc] = (gr < nb && gc < nb) ? F[(int64_t)src * f + k + gc] : 0.0;
    aug[gr][NP + gc] = (gr < nb && gc == gr) ? 1.0 : 0.0;
    if (gc == 0) rowpiv[gr] = gr < nb ? -1 : NP;  // pivot index of the row, -1 while unpivoted
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (warp == 0) {
      const bool cand_ok = lane < nb && rowpiv[lane] < 0;
      unsigned long long key =
          cand_ok ? ((unsigned long long)__double_as_longlong(aug[lane][j]) & 0x7fffffffffffffffull)
                  : 0ull;
      int p = lane;
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, off);
        const int op = __shfl_xor_sync(0xffffffffu, p, off);
        if (ok > key || (ok == key && op < p)) {
          key = ok;
          p = op;
        }
      }
      if (lane == 0) {
        if (key == 0ull || key >= 0x7ff0000000000000ull) atomicOr(err, 4);  // zero, Inf or NaN
        gp = p;
        rowpiv[p] = j;
        gd = 1.0 / aug[p][j];  // the one FP64 division of this pivot
      }
    }
    __syncthreads();
    const int p = gp;
    const double d = gd;
    const double lr = gr == p ? 0.0 : aug[gr][j];  // multipliers, read before any update
    const double p0 = aug[p][gc] * d, p1 = aug[p][NP + gc] * d;
    __syncthreads();
    if (gr == p) {
      aug[gr][gc] = p0;
      aug[gr][NP + gc] = p1;
    } else {
      aug[gr][gc] = fma(-lr, p0, aug[gr][gc]);
      aug[gr][NP + gc] = fma(-lr, p1, aug[gr][NP + gc]);
    }
    __syncthreads();
  }
  {
    const int jr = rowpiv[gr];
    if (jr >= 0 && jr < NP) pinv[fid * NP * NP + jr * NP + gc] = gc < nb ? aug[gr][NP + gc] : 0.0;
    else if (gr >= nb) pinv[fid * NP * NP + gr * NP + gc] = 0.0;
  }
}

constexpr int kPanelRows = 8;  // rows per thread: panels of up to 2048 rows (the cross, n = 1024)
__global__ void __launch_bounds__(256) k_nd_panel(const double* __restrict__ fronts, int f, int s,
                                                  int k, int nb, int32_t* __restrict__ perm,
                                                  double* __restrict__ cbuf,
                                                  double* __restrict__ pinv,
                                                  int32_t* __restrict__ swaps,
                                                  int32_t* __restrict__ err) {
  constexpr int NT = 256;
  __shared__ float cand[2][NT][NP + 1];  // each thread's best remaining row, double-buffered
  __shared__ float wbest[2][8];
  __shared__ int wbi[2][8];
  __shared__ int sel[NP];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = s - k;
  const int64_t fid = blockIdx.x;
  const double* F = fronts + fid * f * f;
  float rv[kPanelRows][NP];
#pragma unroll
  for (int t = 0; t < kPanelRows; ++t) {
    const int i = tid + t * NT;
    const double* Fi = F + (int64_t)(k + (i < m ? i : 0)) * f + k;
    double v[NP];
#pragma unroll
    for (int c = 0; c < NP; ++c) v[c] = (i < m && c < nb) ? Fi[c] : 0.0;
#pragma unroll
    for (int c = 0; c < NP; ++c) rv[t][c] = rank_f32(v[c]);
  }
  unsigned used = 0;  // bit t: row tid + t NT is a pivot row (or does not exist)
#pragma unroll
  for (int t = 0; t < kPanelRows; ++t)
    if (tid + t * NT >= m) used |= 1u << t;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    if (j >= nb) break;
    // this thread's candidate for pivot j
    float best = -1.0f;
    int bt = 0;
#pragma unroll
    for (int t = 0; t < kPanelRows; ++t) {
      const float a = fabsf(rv[t][j]);
      if (!(used >> t & 1u) && a > best) {
        best = a;
        bt = t;
      }
    }
    int bi = best >= 0.0f ? tid + bt * NT : m;
#pragma unroll
    for (int c = 0; c < NP; ++c) {
      if (c < j) continue;
      float val = rv[0][c];
#pragma unroll
      for (int t = 1; t < kPanelRows; ++t)
        if (t == bt) val = rv[t][c];
      cand[j & 1][tid][c] = val;
    }
    warp_argmax_f(best, bi);
    if (lane == 0) {
      wbest[j & 1][warp] = best;
      wbi[j & 1][warp] = bi;
    }
    __syncthreads();
    float b = wbest[j & 1][0];
    int pr = wbi[j & 1][0];
#pragma unroll
    for (int w = 1; w < NT / 32; ++w) {
      const float bw = wbest[j & 1][w];
      const int iw = wbi[j & 1][w];
      if (bw > b || (bw == b && iw < pr)) {
        b = bw;
        pr = iw;
      }
    }
    if (!(b > 0.0f) || !isfinite(b) || pr >= m) {  // uniform: every thread read the same values
      if (tid == 0) {
        atomicOr(err, 2);
        swaps[fid * kSwapInts] = 0;  // the next kernels of the step then exchange nothing
      }
      return;
    }
    if (tid == 0) sel[j] = pr;
    const int owner = pr % NT, ot = pr / NT;
    float pv[NP];  // the pivot row from column j on
#pragma unroll
    for (int c = 0; c < NP; ++c) pv[c] = c >= j ? cand[j & 1][owner][c] : 0.0f;
    if (owner == tid) used |= 1u << ot;
    const float ipv = 1.0f / pv[j];
#pragma unroll
    for (int t = 0; t < kPanelRows; ++t) {
      if (used >> t & 1u) continue;
      const float l = rv[t][j] * ipv;
#pragma unroll
      for (int c = 0; c < NP; ++c)
        if (c > j) rv[t][c] = fmaf(-l, pv[c], rv[t][c]);
    }
  }
  __syncthreads();  // sel complete
  panel_tail(F, f, s, k, nb, fid, sel, perm, cbuf, pinv, swaps, err);
}

// Part 1 for panels of more than kPanelRows * 256 rows (the root planes of 3D grids): the same
// FP32 trial elimination with the ranking rows in a global scratch (L2-resident) instead of
// registers; each thread handles rows tid + t * 256, t < 64 (up to 16 384 rows).
__global__ void __launch_bounds__(256) k_nd_panel_big(const double* __restrict__ fronts, int f,
                                                      int s, int k, int nb,
                                                      int32_t* __restrict__ perm,
                                                      double* __restrict__ cbuf,
                                                      double* __restrict__ pinv,
                                                      int32_t* __restrict__ swaps,
                                                      int32_t* __restrict__ err,
                                                      float* __restrict__ scratch) {
  constexpr int NT = 256, PS = NP + 1;
  __shared__ float cand[2][NT][PS];
  __shared__ float wbest[2][8];
  __shared__ int wbi[2][8];
  __shared__ int sel[NP];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = s - k;
  const int64_t fid = blockIdx.x;
  const double* F = fronts + fid * f * f;
  float* pan = scratch + fid * (int64_t)s * PS;
  const int nrows = (m - tid + NT - 1) / NT;  // rows of this thread (<= 64)
  float best = -1.0f;
  int bt = 0;
  for (int t = 0; t < nrows; ++t) {
    const int i = tid + t * NT;
    const double* Fi = F + (int64_t)(k + i) * f + k;
    double v[NP];
#pragma unroll
    for (int c = 0; c < NP; ++c) v[c] = c < nb ? Fi[c] : 0.0;
#pragma unroll
    for (int c = 0; c < NP; ++c) pan[(int64_t)i * PS + c] = rank_f32(v[c]);
    const float a = fabsf(rank_f32(v[0]));
    if (a > best) {
      best = a;
      bt = t;
    }
  }
  unsigned long long used = 0;
  for (int j = 0; j < nb; ++j) {
    int bi = best >= 0.0f ? tid + bt * NT : m;
    if (best >= 0.0f) {
      const float* rowc = pan + (int64_t)bi * PS;
#pragma unroll
      for (int c = 0; c < NP; ++c)
        if (c >= j) cand[j & 1][tid][c] = rowc[c];
    }
    warp_argmax_f(best, bi);
    if (lane == 0) {
      wbest[j & 1][warp] = best;
      wbi[j & 1][warp] = bi;
    }
    __syncthreads();
    float b = wbest[j & 1][0];
    int pr = wbi[j & 1][0];
#pragma unroll
    for (int w = 1; w < NT / 32; ++w) {
      const float bw = wbest[j & 1][w];
      const int iw = wbi[j & 1][w];
      if (bw > b || (bw == b && iw < pr)) {
        b = bw;
        pr = iw;
      }
    }
    if (!(b > 0.0f) || !isfinite(b) || pr >= m) {  // uniform
      if (tid == 0) {
        atomicOr(err, 2);
        swaps[fid * kSwapInts] = 0;
      }
      return;
    }
    if (tid == 0) sel[j] = pr;
    const int owner = pr % NT;
    if (owner == tid) used |= 1ull << (pr / NT);
    float pv[NP];
#pragma unroll
    for (int c = 0; c < NP; ++c) pv[c] = c >= j ? cand[j & 1][owner][c] : 0.0f;
    const float ipv = 1.0f / pv[j];
    best = -1.0f;
    bt = 0;
    for (int t = 0; t < nrows; ++t) {
      if (used >> t & 1ull) continue;
      float* row = pan + (int64_t)(tid + t * NT) * PS;
      float x[NP];
#pragma unroll
      for (int c = 0; c < NP; ++c) x[c] = row[c];
      const float l = x[j] * ipv;
#pragma unroll
      for (int c = 0; c < NP; ++c)
        if (c > j) x[c] = fmaf(-l, pv[c], x[c]);
#pragma unroll
      for (int c = 0; c < NP; ++c)
        if (c > j) row[c] = x[c];
      if (j + 1 < nb) {
        float a = 0.0f;
#pragma unroll
        for (int c = 0; c < NP; ++c)
          if (c == j + 1) a = fabsf(x[c]);
        if (a > best) {
          best = a;
          bt = t;
        }
      }
    }
  }
  __syncthreads();  // sel complete
  panel_tail(F, f, s, k, nb, fid, sel, perm, cbuf, pinv, swaps, err);
}

// Part 2: rows K become A_KK^-1 F[K, j] for the columns j outside K (after applying the row
// exchanges to those columns), and the column block becomes [A_KK^-1 on K; -cbuf A_KK^-1 off K];
// the column tiles also complete cbuf with the rows that the exchanges did not move.
constexpr int kRowThreads = 64;  // one column (or row) per thread; small CTAs spread the step
__global__ void __launch_bounds__(kRowThreads) k_nd_rowblock(double* __restrict__ fronts, int f, int k,
                                                     int nb, int tiles_w,
                                                     double* __restrict__ cbuf,
                                                     const double* __restrict__ pinv,
                                                     const int32_t* __restrict__ swaps) {
  __shared__ double pi[NP][NP];
  __shared__ int dstp[2 * NP], srcp[2 * NP], kq[NP];
  __shared__ int nq;
  const int tid = threadIdx.x;
  const int64_t fid = blockIdx.y;
  double* F = fronts + fid * f * f;
  const int32_t* sw = swaps + fid * kSwapInts;
  for (int e = tid; e < NP * NP; e += blockDim.x) pi[e / NP][e % NP] = pinv[fid * NP * NP + e];
  if (tid == 0) {
    int q0 = sw[0];
    q0 = q0 < 0 || q0 > 2 * NP ? 0 : q0;
    for (int a = 0; a < q0; ++a) {
      const int dp = sw[1 + a], sp = sw[1 + 2 * NP + a];
      if (dp < 0 || dp >= f || sp < 0 || sp >= f) q0 = 0;
    }
    nq = q0;
  }
  __syncthreads();
  const int q = nq;
  if (tid < q) {
    dstp[tid] = sw[1 + tid];
    srcp[tid] = sw[1 + 2 * NP + tid];
  }
  __syncthreads();
  if (tid < nb) {
    int a0 = -1;
    for (int a = 0; a < q; ++a)
      if (dstp[a] == k + tid) a0 = a;
    kq[tid] = a0;
  }
  __syncthreads();
  if ((int)blockIdx.x < tiles_w) {
    const int j = blockIdx.x * blockDim.x + tid;
    if (j >= f || (j >= k && j < k + nb)) return;
    double val[2 * NP];
    for (int a = 0; a < 2 * NP; ++a)
      if (a < q) val[a] = F[(int64_t)srcp[a] * f + j];
    double rv[NP];
    for (int c = 0; c < NP; ++c) {
      double v = 0.0;
      if (c < nb) {
        v = F[(int64_t)(k + c) * f + j];
        for (int a = 0; a < 2 * NP; ++a)
          if (a == kq[c]) v = val[a];
      }
      rv[c] = v;
    }
    for (int c = 0; c < nb; ++c) {
      double w = 0.0;
      for (int mm = 0; mm < NP; ++mm) w = fma(pi[c][mm], rv[mm], w);
      F[(int64_t)(k + c) * f + j] = w;
    }
    for (int a = 0; a < 2 * NP; ++a)
      if (a < q && (dstp[a] < k || dstp[a] >= k + nb)) F[(int64_t)dstp[a] * f + j] = val[a];
  } else {
    const int x = (blockIdx.x - tiles_w) * blockDim.x + tid;
    if (x >= f) return;
    bool moved = false;
    for (int a = 0; a < q; ++a)
      if (dstp[a] == x) moved = true;
    double* cx = cbuf + fid * (int64_t)f * NP + (int64_t)x * NP;
    double* Fx = F + (int64_t)x * f + k;
    double cr[NP];
    if (moved) {  // written by part 1 from the row's source position
#pragma unroll
      for (int mm = 0; mm < NP; ++mm) cr[mm] = cx[mm];
    } else {      // still in place: this thread is the only reader and writer of F[x][K]
#pragma unroll
      for (int mm = 0; mm < NP; ++mm) cr[mm] = mm < nb ? Fx[mm] : 0.0;
#pragma unroll
      for (int mm = 0; mm < NP; ++mm) cx[mm] = cr[mm];
    }
    if (x >= k && x < k + nb) {
      for (int c = 0; c < nb; ++c) Fx[c] = pi[x - k][c];
    } else {
      for (int c = 0; c < nb; ++c) {
        double acc = 0.0;
#pragma unroll
        for (int mm = 0; mm < NP; ++mm) acc = fma(cr[mm], pi[mm][c], acc);
        Fx[c] = -acc;
      }
    }
  }
}

// Part 3: F[i][j] -= cbuf[i][:] . F[K][j] for every i, j outside K (64 x 64 tiles).
constexpr int kUT = 64;
// Columns updated: [col_lo, col_hi) without [skip_lo, skip_hi) (which holds K); the tiles
// start at col_lo. With look-ahead a step is split into the next panel's columns and the rest.
__global__ void __launch_bounds__(256) k_nd_update(double* __restrict__ fronts, int f, int k,
                                                   int nb, int tiles_j, int col_lo, int col_hi,
                                                   int skip_lo, int skip_hi,
                                                   const double* __restrict__ cbuf) {
  __shared__ double cs[kUT][NP + 1];
  __shared__ double ws[NP][kUT];
  const int tid = threadIdx.x;
  const int64_t fid = blockIdx.y;
  double* F = fronts + fid * f * f;
  const int ti = blockIdx.x / tiles_j, tj = blockIdx.x % tiles_j;
  const int i0 = ti * kUT, j0 = col_lo + tj * kUT;
  const double* cb = cbuf + fid * (int64_t)f * NP;
  for (int e = tid; e < kUT * NP; e += blockDim.x) {
    const int r = e / NP, c = e % NP;
    cs[r][c] = (i0 + r < f) ? cb[(int64_t)(i0 + r) * NP + c] : 0.0;
    const int c2 = e / kUT, col = e % kUT;
    ws[c2][col] = (c2 < nb && j0 + col < col_hi) ? F[(int64_t)(k + c2) * f + j0 + col] : 0.0;
  }
  __syncthreads();
  const int ty = tid / 16, tx = tid % 16;
  double acc[4][4];
  bool rok[4], cok[4];
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * a;
    rok[a] = i < f && (i < k || i >= k + nb);
    cok[a] = j < col_hi && (j < skip_lo || j >= skip_hi);
  }
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      acc[a][b] = (rok[a] && cok[b]) ? F[(int64_t)(i0 + ty + 16 * a) * f + j0 + tx + 16 * b] : 0.0;
#pragma unroll
  for (int c = 0; c < NP; ++c) {
    double cr[4], wr[4];
    for (int a = 0; a < 4; ++a) cr[a] = cs[ty + 16 * a][c];
    for (int b = 0; b < 4; ++b) wr[b] = ws[c][tx + 16 * b];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(-cr[a], wr[b], acc[a][b]);
  }
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      if (rok[a] && cok[b]) F[(int64_t)(i0 + ty + 16 * a) * f + j0 + tx + 16 * b] = acc[a][b];
}

// ---- solve ----
// Going up: w = [y_E; 0] + children's u (through the ring maps), w'_E = w_E[perm];
// z = A^-1 w_E = F[E, E] w'_E; u = w_R + F[R, E] w'_E. 64 rows of one front per CTA.
__global__ void __launch_bounds__(256) k_nd_fwd(const double* __restrict__ F, int f, int s, int r,
                                                const int32_t* __restrict__ E,
                                                const int32_t* __restrict__ perm,
                                                const int32_t* __restrict__ inv, int nchild,
                                                const double* __restrict__ uc, int rc,
                                                const double* __restrict__ y,
                                                double* __restrict__ z, double* __restrict__ u,
                                                int rows) {
  extern __shared__ double wE[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t p = blockIdx.y;
  const double* Fp = F + p * f * f;
  const int32_t* iv = nchild ? inv + p * f * 2 : nullptr;
  auto wsum = [&](int i) -> double {
    double v = i < s ? y[E[p * s + i]] : 0.0;
    for (int c = 0; c < nchild; ++c) {
      const int a = iv[i * 2 + c];
      if (a >= 0) v += uc[(nchild == 1 ? p : 2 * p + c) * rc + a];
    }
    return v;
  };
  for (int m = tid; m < s; m += blockDim.x) wE[m] = wsum(perm[p * s + m]);
  __syncthreads();
  const int row0 = blockIdx.x * rows;
  for (int rr = warp; rr < rows; rr += blockDim.x / 32) {
    const int i = row0 + rr;
    if (i >= f) break;
    const double* Fi = Fp + (int64_t)i * f;
    double acc = 0.0;
    for (int m = lane; m < s; m += 32) acc = fma(Fi[m], wE[m], acc);
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) {
      if (i < s)
        z[p * s + i] = acc;
      else
        u[p * r + (i - s)] = wsum(i) + acc;
    }
  }
}

// Coming down: x_E = z - F[E, R] x_R, x_R read from the ancestors' results.
__global__ void __launch_bounds__(256) k_nd_bwd(const double* __restrict__ F, int f, int s, int r,
                                                const int32_t* __restrict__ E,
                                                const int32_t* __restrict__ R,
                                                const double* __restrict__ z,
                                                double* __restrict__ x, int rows) {
  extern __shared__ double xR[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t p = blockIdx.y;
  const double* Fp = F + p * f * f;
  for (int m = tid; m < r; m += blockDim.x) xR[m] = x[R[p * r + m]];
  __syncthreads();
  const int row0 = blockIdx.x * rows;
  for (int rr = warp; rr < rows; rr += blockDim.x / 32) {
    const int i = row0 + rr;
    if (i >= s) break;
    const double* Fi = Fp + (int64_t)i * f + s;
    double acc = 0.0;
    for (int m = lane; m < r; m += 32) acc = fma(Fi[m], xR[m], acc);
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) x[E[p * s + i]] = z[p * s + i] - acc;
  }
}

// Copies rows 0..nr-1, columns c0..c0+nc-1 of the f x f front Fp into dst (row stride ld),
// eight independent loads in flight per thread.
__device__ __forceinline__ void stage_block(const double* __restrict__ Fp, int f, int c0, int nr,
                                            int nc, double* __restrict__ dst, int ld) {
  const int total = nr * nc, nt = blockDim.x;
  for (int e0 = threadIdx.x; e0 < total; e0 += 8 * nt) {
    double v[8];
    int at[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = e0 + q * nt;
      at[q] = -1;
      if (e < total) {
        const int i = e / nc, m = e - i * nc;
        v[q] = Fp[(int64_t)i * f + c0 + m];
        at[q] = i * ld + m;
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (at[q] >= 0) dst[at[q]] = v[q];
  }
}

// Fronts whose block fits in shared memory, one CTA per front: the block the product reads is staged
// in shared memory with an odd row stride (conflict-free column access), then one thread per
// row. Same sums in the same order as the warp-per-row kernels would not give; each kernel is
// deterministic on its own.
__global__ void __launch_bounds__(256) k_nd_fwd_small(const double* __restrict__ F, int f, int s,
                                                      int r, const int32_t* __restrict__ E,
                                                      const int32_t* __restrict__ perm,
                                                      const int32_t* __restrict__ inv,
                                                      int nchild, const double* __restrict__ uc,
                                                      int rc, const double* __restrict__ y,
                                                      double* __restrict__ z,
                                                      double* __restrict__ u) {
  extern __shared__ double sh[];
  const int ld = s | 1;
  double* wE = sh;           // s
  double* Ms = sh + ld;      // f rows of stride ld: F[i][0..s)
  const int tid = threadIdx.x;
  const int64_t p = blockIdx.x;
  const double* Fp = F + p * f * f;
  const int32_t* iv = nchild ? inv + p * f * 2 : nullptr;
  auto wsum = [&](int i) -> double {
    double v = i < s ? y[E[p * s + i]] : 0.0;
    for (int c = 0; c < nchild; ++c) {
      const int a = iv[i * 2 + c];
      if (a >= 0) v += uc[(nchild == 1 ? p : 2 * p + c) * rc + a];
    }
    return v;
  };
  for (int m = tid; m < s; m += blockDim.x) wE[m] = wsum(perm[p * s + m]);
  stage_block(Fp, f, 0, f, s, Ms, ld);
  __syncthreads();
  for (int i = tid; i < f; i += blockDim.x) {
    const double* Mi = Ms + i * ld;
    double a0 = 0.0, a1 = 0.0;
    int m = 0;
    for (; m + 1 < s; m += 2) {
      a0 = fma(Mi[m], wE[m], a0);
      a1 = fma(Mi[m + 1], wE[m + 1], a1);
    }
    if (m < s) a0 = fma(Mi[m], wE[m], a0);
    const double acc = a0 + a1;
    if (i < s)
      z[p * s + i] = acc;
    else
      u[p * r + (i - s)] = wsum(i) + acc;
  }
}

__global__ void __launch_bounds__(256) k_nd_bwd_small(const double* __restrict__ F, int f, int s,
                                                      int r, const int32_t* __restrict__ E,
                                                      const int32_t* __restrict__ R,
                                                      const double* __restrict__ z,
                                                      double* __restrict__ x) {
  extern __shared__ double sh[];
  const int ld = r | 1;
  double* xR = sh;          // r
  double* Mb = sh + ld;     // s rows of stride ld: F[i][s..f)
  const int tid = threadIdx.x;
  const int64_t p = blockIdx.x;
  const double* Fp = F + p * f * f;
  for (int m = tid; m < r; m += blockDim.x) xR[m] = x[R[p * r + m]];
  stage_block(Fp, f, s, s, r, Mb, ld);
  __syncthreads();
  for (int i = tid; i < s; i += blockDim.x) {
    const double* Mi = Mb + i * ld;
    double a0 = 0.0, a1 = 0.0;
    int m = 0;
    for (; m + 1 < r; m += 2) {
      a0 = fma(Mi[m], xR[m], a0);
      a1 = fma(Mi[m + 1], xR[m + 1], a1);
    }
    if (m < r) a0 = fma(Mi[m], xR[m], a0);
    x[E[p * s + i]] = z[p * s + i] - (a0 + a1);
  }
}

// y_j = sum_a rows[j][a] u[(j + o_a) mod n], o_a in [-t, t]^d lexicographic (last fastest).
__global__ void k_apply_rows(const double* __restrict__ rows, int mu, int d, int n, int t,
                             const double* __restrict__ u, double* __restrict__ y, int64_t N) {
  const int w = 2 * t + 1;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x) {
    int x[3] = {0, 0, 0};
    int64_t rem = j;
    for (int a = d - 1; a >= 0; --a) {
      x[a] = (int)(rem % n);
      rem /= n;
    }
    const double* rj = rows + j * mu;
    double acc = 0.0;
    for (int a = 0; a < mu; ++a) {
      int o = a;
      int64_t col = 0;
      int64_t stride = 1;
      for (int b = d - 1; b >= 0; --b) {
        const int ob = o % w - t;
        o /= w;
        col += (int64_t)((x[b] + ob + n) % n) * stride;
        stride *= n;
      }
      acc = fma(rj[a], u[col], acc);
    }
    y[j] = acc;
  }
}

__global__ void k_nd_iota(int32_t* __restrict__ perm, int count, int s) {
  const int64_t total = (int64_t)count * s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    perm[e] = (int32_t)(e % s);
}

// "<stem>@<depth>": per-depth timer names (stable storage for the timer table)
const char* level_name(const char* stem, int depth) {
  static char names[7][32][24];
  const int k = stem[3] == 'f' ? 0 : stem[3] == 'b' ? 1 : stem[3] == 's' ? 2 : stem[3] == 'a' ? 3
              : stem[3] == 'p' ? 4 : stem[3] == 'r' ? 5 : 6;
  if (depth < 0 || depth >= 32) return stem;
  snprintf(names[k][depth], sizeof names[k][depth], "%s@%d", stem, depth);
  return names[k][depth];
}

int grid_for(int64_t n, int threads) {
  const int64_t b = (n + threads - 1) / threads;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

}  // namespace

cudaError_t launch_nd_assemble(lsp_ctx* c, int depth, const double* rows) {
  NdState& S = *c->nd;
  const NdLevel& lv = S.plan.lv[depth];
  double* F = (double*)S.fronts.p + lv.front_off;
  const int64_t total = (int64_t)lv.count * lv.f * lv.f;
  int t = timer_begin(c, level_name("nd_asm", depth));
  if (lv.nchild == 0) {
    cudaError_t e = cudaMemsetAsync(F, 0, sizeof(double) * total, c->stream);
    if (e != cudaSuccess) return e;
  } else {
    const NdLevel& cl = S.plan.lv[depth + 1];
    k_nd_extend<<<grid_for(total, 256), 256, 0, c->stream>>>(
        F, (const double*)S.fronts.p + cl.front_off, (const int32_t*)S.inv.p + lv.inv_off,
        lv.count, lv.f, lv.nchild, cl.f, cl.s);
  }
  if (lv.asm_n > 0)
    k_nd_scatter<<<grid_for(lv.asm_n, 256), 256, 0, c->stream>>>(
        F, rows, (const int32_t*)S.asm_dst.p + lv.asm_off, (const int32_t*)S.asm_src.p + lv.asm_off,
        lv.asm_n);
  timer_end(c, t);
  return cudaGetLastError();
}

cudaError_t launch_nd_sweep(lsp_ctx* c, int depth) {
  NdState& S = *c->nd;
  const NdLevel& lv = S.plan.lv[depth];
  double* F = (double*)S.fronts.p + lv.front_off;
  int32_t* perm = (int32_t*)S.perm.p + lv.perm_off;
  int32_t* err = (int32_t*)S.err.p;
  if (lv.s == 0) return cudaSuccess;
  int t = timer_begin(c, level_name("nd_sweep", depth));
  if (lv.f <= kNdSmallFront) {
    const size_t smem = sizeof(double) * ((size_t)lv.f * lv.f + 2 * lv.f);
    cudaError_t e = cudaFuncSetAttribute(k_nd_sweep_small,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_nd_sweep_small<<<lv.count, 256, smem, c->stream>>>(F, lv.f, lv.s, perm, err);
    timer_end(c, t);
    return cudaGetLastError();
  }
  // blocked steps; perm starts as the identity
  k_nd_iota<<<grid_for((int64_t)lv.count * lv.s, 256), 256, 0, c->stream>>>(perm, lv.count, lv.s);
  const bool big = lv.s > kPanelRows * 256;
  if (big && !S.pscratch.p) return cudaErrorInvalidValue;
  const int tiles_w = (lv.f + kRowThreads - 1) / kRowThreads;
  const int tiles_c = (lv.f + kRowThreads - 1) / kRowThreads;
  const int tiles_u = (lv.f + kUT - 1) / kUT;
  // Look-ahead: once a step's update has reached the next panel's columns, that panel runs on
  // the side stream while the rest of the update runs here (disjoint columns). The step
  // buffers (cbuf, pinv, swaps) alternate between two copies. Per-kernel timing keeps one
  // stream so that every launch is bracketed by its own events.
  const bool ahead = S.side != nullptr && !c->timing;
  auto buf = [&](int par, double** cb, double** pv, int32_t** sw) {
    *cb = (double*)S.cbuf.p + (int64_t)par * S.cbuf_half;
    *pv = (double*)S.pinv.p + (int64_t)par * S.pinv_half;
    *sw = (int32_t*)S.swaps.p + (int64_t)par * S.swaps_half;
  };
  auto panel = [&](int k, int par, cudaStream_t st) {
    double *cb, *pv;
    int32_t* sw;
    buf(par, &cb, &pv, &sw);
    const int nb = lv.s - k < NP ? lv.s - k : NP;
    const int t1 = c->timing ? timer_begin(c, level_name("nd_pnl", depth)) : -1;
    if (big)
      k_nd_panel_big<<<lv.count, 256, 0, st>>>(F, lv.f, lv.s, k, nb, perm, cb, pv, sw, err,
                                               (float*)S.pscratch.p);
    else
      k_nd_panel<<<lv.count, 256, 0, st>>>(F, lv.f, lv.s, k, nb, perm, cb, pv, sw, err);
    timer_end(c, t1);
  };
  auto update = [&](int k, int nb, const double* cb, int col_lo, int col_hi, int skip_lo,
                    int skip_hi) {
    const int tj = (col_hi - col_lo + kUT - 1) / kUT;
    const int t3 = c->timing ? timer_begin(c, level_name("nd_upd", depth)) : -1;
    k_nd_update<<<dim3(tiles_u * tj, lv.count), 256, 0, c->stream>>>(
        F, lv.f, k, nb, tj, col_lo, col_hi, skip_lo, skip_hi, cb);
    timer_end(c, t3);
  };
  panel(0, 0, c->stream);
  for (int k = 0, step = 0; k < lv.s; k += NP, ++step) {
    const int nb = lv.s - k < NP ? lv.s - k : NP;
    const int par = step & 1;
    double *cb, *pv;
    int32_t* sw;
    buf(par, &cb, &pv, &sw);
    if (ahead && step > 0) {
      cudaError_t e = cudaStreamWaitEvent(c->stream, S.ev_panel, 0);
      if (e != cudaSuccess) return e;
    }
    const int t2 = c->timing ? timer_begin(c, level_name("nd_row", depth)) : -1;
    k_nd_rowblock<<<dim3(tiles_w + tiles_c, lv.count), kRowThreads, 0, c->stream>>>(
        F, lv.f, k, nb, tiles_w, cb, pv, sw);
    timer_end(c, t2);
    const int kn = k + nb;
    if (kn >= lv.s) {  // last step: the whole update
      update(k, nb, cb, 0, lv.f, k, kn);
    } else if (ahead) {
      const int nbn = lv.s - kn < NP ? lv.s - kn : NP;
      update(k, nb, cb, kn, kn + nbn, k, kn);  // the next panel's columns first
      cudaError_t e = cudaEventRecord(S.ev_cols, c->stream);
      if (e != cudaSuccess) return e;
      e = cudaStreamWaitEvent(S.side, S.ev_cols, 0);
      if (e != cudaSuccess) return e;
      panel(kn, par ^ 1, S.side);
      e = cudaEventRecord(S.ev_panel, S.side);
      if (e != cudaSuccess) return e;
      update(k, nb, cb, 0, lv.f, k, kn + nbn);  // the rest, beside the panel
    } else {
      update(k, nb, cb, 0, lv.f, k, kn);
      panel(kn, par ^ 1, c->stream);
    }
  }
  timer_end(c, t);
  return cudaGetLastError();
}

cudaError_t launch_nd_solve(lsp_ctx* c, const double* y, double* x) {
  NdState& S = *c->nd;
  const NdPlan& P = S.plan;
  const int L = (int)P.lv.size();
  const double* Fb = (const double*)S.fronts.p;
  double* z = (double*)S.z.p;
  double* u = (double*)S.u.p;
  const int32_t* E = (const int32_t*)S.E.p;
  const int32_t* R = (const int32_t*)S.R.p;
  // rows of one front per CTA: 64 where the level has fronts enough to fill the GPU, else 8
  // (one row per warp) so that the few large fronts near the root still spread over the SMs
  auto rows_for = [](int count, int nrows) {
    return (int64_t)count * ((nrows + 63) / 64) >= 8 * 152 ? 64 : 8;
  };
  for (int d = L - 1; d >= 0; --d) {
    const NdLevel& lv = P.lv[d];
    const NdLevel* cl = lv.nchild ? &P.lv[d + 1] : nullptr;
    const int rows = rows_for(lv.count, lv.f);
    dim3 grid((lv.f + rows - 1) / rows, lv.count);
    int t = timer_begin(c, level_name("nd_fwd", d));
    // one CTA per front with the block staged in shared memory: small fronts, or larger ones
    // when the depth has fronts enough to fill the GPU (else rows spread over many CTAs)
    const size_t smf = sizeof(double) * ((size_t)(lv.s | 1) * (lv.f + 1));
    const bool many = lv.count >= 2 * 152;
    if (lv.f <= kNdSmallFront || (many && smf <= kNdStagedBytes)) {
      k_nd_fwd_small<<<lv.count, lv.f <= kNdSmallFront ? 128 : 256, smf, c->stream>>>(
          Fb + lv.front_off, lv.f, lv.s, lv.r, E + lv.E_off,
          (const int32_t*)S.perm.p + lv.perm_off,
          lv.nchild ? (const int32_t*)S.inv.p + lv.inv_off : nullptr, lv.nchild,
          cl ? u + cl->u_off : nullptr, cl ? cl->r : 0, y, z + lv.z_off, u + lv.u_off);
    } else {
      k_nd_fwd<<<grid, 256, sizeof(double) * (lv.s > 0 ? lv.s : 1), c->stream>>>(
          Fb + lv.front_off, lv.f, lv.s, lv.r, E + lv.E_off,
          (const int32_t*)S.perm.p + lv.perm_off,
          lv.nchild ? (const int32_t*)S.inv.p + lv.inv_off : nullptr, lv.nchild,
          cl ? u + cl->u_off : nullptr, cl ? cl->r : 0, y, z + lv.z_off, u + lv.u_off, rows);
    }
    timer_end(c, t);
  }
  for (int d = 0; d < L; ++d) {
    const NdLevel& lv = P.lv[d];
    const int rows = rows_for(lv.count, lv.s);
    dim3 grid((lv.s + rows - 1) / rows, lv.count);
    int t = timer_begin(c, level_name("nd_bwd", d));
    const size_t smb = sizeof(double) * ((size_t)(lv.r | 1) * (lv.s + 1));
    const bool many = lv.count >= 2 * 152;
    if (lv.f <= kNdSmallFront || (many && smb <= kNdStagedBytes)) {
      k_nd_bwd_small<<<lv.count, lv.s <= kNdSmallFront ? 128 : 256, smb, c->stream>>>(
          Fb + lv.front_off, lv.f, lv.s, lv.r,
                                                       E + lv.E_off, R + lv.R_off,
                                                       z + lv.z_off, x);
    } else {
      k_nd_bwd<<<grid, 256, sizeof(double) * (lv.r > 0 ? lv.r : 1), c->stream>>>(
          Fb + lv.front_off, lv.f, lv.s, lv.r, E + lv.E_off, R + lv.R_off, z + lv.z_off, x,
          rows);
    }
    timer_end(c, t);
  }
  return cudaGetLastError();
}

cudaError_t nd_prepare_kernels(int max_smem) {
  // staged solve kernels: (s | 1) (f + 1) or (r | 1) (s + 1) doubles, with s, r <= f <= 160
  // for small fronts, and at most kNdStagedBytes for the larger ones
  const int small_front = (int)sizeof(double) * ((kNdSmallFront | 1) + 1) * (kNdSmallFront + 1);
  const int small = small_front > (int)kNdStagedBytes ? small_front : (int)kNdStagedBytes;
  cudaError_t e = cudaFuncSetAttribute(k_nd_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       max_smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_nd_fwd_small, cudaFuncAttributeMaxDynamicSharedMemorySize, small);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_nd_bwd_small, cudaFuncAttributeMaxDynamicSharedMemorySize, small);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_nd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

cudaError_t launch_apply_rows(lsp_ctx* c, const double* rows, int mu, int t, const double* u,
                              double* y) {
  const int64_t N = c->geo.N;
  int tm = timer_begin(c, "apply_rows");
  k_apply_rows<<<grid_for(N, 256), 256, 0, c->stream>>>(rows, mu, c->geo.d, c->geo.n, t, u, y, N);
  timer_end(c, tm);
  return cudaGetLastError();
}

}  // namespace lsp
