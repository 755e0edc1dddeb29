// y = (L + diag(v)) u with L = F^-1 diag(4 pi^2 |k|^2) F (Sec. 2, Eq. dmodel).
//
// A d-dimensional complex FP64 FFT done one axis at a time: every block transforms whole
// lines of the chosen axis in shared memory (iterative radix-2, bit-reversed load, twiddles
// from a table computed on the host in extended precision). Passes:
//   1D: [fwd from real u, * 4 pi^2 k^2, inv, y = Re/n + v u] in one pass
//   2D: [fwd axis0 from real u] -> [fwd axis1, * 4 pi^2 |k|^2, inv axis1] -> [inv axis0, y = Re/N + v u]
//   3D: [fwd 0] -> [fwd 1] -> [fwd 2, * symbol, inv 2] -> [inv 1] -> [inv 0, output]
// The unitary factors n^{-d/2} of F and F^-1 combine into the single 1/N of the output pass.
#include "lsp_internal.h"

namespace lsp {
namespace {

// kAll (d = 1): load the real input, transform, apply the symbol, transform back and output.
enum Mode { kPlain = 0, kLoadReal = 1, kSymbol = 2, kOutput = 3, kAll = 4 };

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ void fft_line(double2* x, int n, int logn, const double2* __restrict__ tw,
                                         bool inverse) {
  for (int s = 1; s <= logn; ++s) {
    const int m = 1 << s, half = m >> 1, tstride = n >> s;
    for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
      const int grp = b / half, k = b - grp * half;
      const int i = grp * m + k, j = i + half;
      double2 w = __ldg(tw + k * tstride);
      if (inverse) w.y = -w.y;
      const double2 a = x[i], t = cmul(x[j], w);
      x[i] = make_double2(a.x + t.x, a.y + t.y);
      x[j] = make_double2(a.x - t.x, a.y - t.y);
    }
    __syncthreads();
  }
}

// Lines along `axis` (stride S = n^(d-1-axis) between elements); one line per block.
// u and y may be the same array (y = (L + diag v) u in place): the output pass reads u[g]
// before it writes y[g], element by element in the same thread, and no other pass reads u
// after the first one, so neither pointer is declared __restrict__.
__global__ void k_fft_axis(double2* __restrict__ Z, const double* u,
                           const double* __restrict__ v, double* y, int d, int n,
                           int logn, int axis, int64_t nlines, const double2* __restrict__ tw,
                           int mode, int fwd_first) {
  extern __shared__ double2 line[];
  int64_t S = 1;
  for (int a = axis + 1; a < d; ++a) S *= n;
  for (int64_t l = blockIdx.x; l < nlines; l += gridDim.x) {
    const int64_t inner = l % S, outer = l / S;
    const int64_t base = outer * S * n + inner;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int r = __brev(i) >> (32 - logn);
      const int64_t g = base + (int64_t)i * S;
      line[r] = (mode == kLoadReal || mode == kAll) ? make_double2(u[g], 0.0) : Z[g];
    }
    __syncthreads();
    fft_line(line, n, logn, tw, !fwd_first);
    if (mode == kSymbol || mode == kAll) {
      // multiply by 4 pi^2 |k|^2 (k in FFT order), then transform back along this axis
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int64_t g = base + (int64_t)i * S;
        double k2 = 0.0;
        for (int a = d - 1; a >= 0; --a) {
          const int ka = (int)(g % n);
          g /= n;
          const double kk = ka < n / 2 ? (double)ka : (double)(ka - n);
          k2 += kk * kk;
        }
        const double lam = 4.0 * kPi2 * k2;
        line[i].x *= lam;
        line[i].y *= lam;
      }
      __syncthreads();
      // bit-reverse again in place for the inverse transform
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int r = __brev(i) >> (32 - logn);
        if (r > i) {
          const double2 t = line[i];
          line[i] = line[r];
          line[r] = t;
        }
      }
      __syncthreads();
      fft_line(line, n, logn, tw, true);
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int64_t g = base + (int64_t)i * S;
      if (mode == kOutput || mode == kAll) {
        const double inv_n = 1.0 / (double)nlines / (double)n;  // 1/N (exact, power of two)
        const double ug = u[g];
        y[g] = fma(v[g], ug, line[i].x * inv_n);
      } else {
        Z[g] = line[i];
      }
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_apply(lsp_ctx* c, const double* u, double* y) {
  const int d = c->geo.d, n = c->geo.n;
  int logn = 0;
  while ((1 << logn) < n) ++logn;
  const int64_t nlines = c->geo.N / n;
  const size_t smem = sizeof(double2) * n;
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k_fft_axis, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int threads = n / 2 < 256 ? (n / 2 < 32 ? 32 : n / 2) : 256;
  int64_t blocks = nlines < 152 * 32 ? nlines : 152 * 32;
  double2* Z = (double2*)c->fftbuf.p;
  const double2* tw = (const double2*)c->twiddle.p;
  const double* v = (const double*)c->v.p;
  int t = timer_begin(c, "apply_fft");
  if (d == 1) {  // one pass: forward, symbol, inverse, output
    k_fft_axis<<<(int)blocks, threads, smem, c->stream>>>(Z, u, v, y, 1, n, logn, 0, nlines, tw,
                                                          kAll, 1);
    timer_end(c, t);
    return cudaGetLastError();
  }
  // forward passes on axes 0..d-2
  for (int axis = 0; axis < d - 1; ++axis)
    k_fft_axis<<<(int)blocks, threads, smem, c->stream>>>(Z, u, v, y, d, n, logn, axis, nlines, tw,
                                                          axis == 0 ? kLoadReal : kPlain, 1);
  // last axis: forward, symbol, inverse
  k_fft_axis<<<(int)blocks, threads, smem, c->stream>>>(Z, u, v, y, d, n, logn, d - 1, nlines, tw,
                                                        kSymbol, 1);
  // inverse passes on axes d-2..0; the last one writes y
  for (int axis = d - 2; axis >= 0; --axis)
    k_fft_axis<<<(int)blocks, threads, smem, c->stream>>>(Z, u, v, y, d, n, logn, axis, nlines, tw,
                                                          axis == 0 ? kOutput : kPlain, 0);
  timer_end(c, t);
  return cudaGetLastError();
}

}  // namespace lsp

// ---- y = (L + diag v) u without any device allocation -------------------------------------
// Some callers cannot allocate device memory at the moment they need the operator: code that
// runs while a CUDA stream is being captured into a graph (where cudaMalloc is not permitted),
// and code whose device memory is owned by a pool or framework allocator that forbids extra
// allocations, or that cannot afford the device-wide synchronisation a cudaMalloc may cause.
// For them the complex work array of the transform lives in a fixed, file-scope device array
// instead of a context buffer. Every GPU that loads this library holds that array (16 MiB for
// the work array plus 32 KiB of twiddles) until the process exits.
namespace lsp {
namespace {

constexpr int64_t kNoAllocMaxPoints = (int64_t)1 << 20;  // must match LSP_NOALLOC_MAX_POINTS
constexpr int kNoAllocMaxHalfN = 2048;
static __device__ __align__(256) double2 g_noalloc_work[kNoAllocMaxPoints];
static __device__ __align__(256) double2 g_noalloc_twiddle[kNoAllocMaxHalfN];

// exp(-2 pi i j / n), j < n/2, with the CUDA math library's sincospi.
__global__ void k_noalloc_twiddles(double2* __restrict__ tw, int n) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n / 2; j += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)j / (double)n, &s, &c);
    tw[j] = make_double2(c, -s);
  }
}

}  // namespace
}  // namespace lsp

extern "C" lsp_status lsp_apply_operator_noalloc(int d, int n, const double* v_dev,
                                                 const double* u_dev, double* y_dev,
                                                 void* cuda_stream) {
  using namespace lsp;
  if (d != 2 && d != 3) return LSP_ERR_ARG;
  if (n < 8 || (n & (n - 1)) != 0 || n / 2 > kNoAllocMaxHalfN) return LSP_ERR_ARG;
  int64_t N = 1;
  for (int i = 0; i < d; ++i) N *= n;
  if (N > kNoAllocMaxPoints) return LSP_ERR_ARG;  // larger grids need the context path
  if (!v_dev || !u_dev || !y_dev) return LSP_ERR_ARG;
  // The symbol names are host-side stand-ins, not device addresses, so they are never passed
  // to a kernel. Their device addresses are looked up on every call, in the current device's
  // current context: the lookup allocates nothing, and a cached address could outlive a
  // context that was torn down and created again. The first call in a context loads the
  // library's device code there, so make it before any stream capture.
  double2* Z = nullptr;
  double2* tw = nullptr;
  if (cudaGetSymbolAddress((void**)&Z, g_noalloc_work) != cudaSuccess ||
      cudaGetSymbolAddress((void**)&tw, g_noalloc_twiddle) != cudaSuccess) {
    cudaGetLastError();
    return LSP_ERR_CUDA;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int logn = 0;
  while ((1 << logn) < n) ++logn;
  const int64_t nlines = N / n;
  const size_t smem = sizeof(double2) * n;  // <= 16 KiB for n <= 1024
  const int threads = n / 2 < 256 ? (n / 2 < 32 ? 32 : n / 2) : 256;
  const int blocks = (int)(nlines < 152 * 32 ? nlines : 152 * 32);
  cudaGetLastError();
  k_noalloc_twiddles<<<(n / 2 + 255) / 256, 256, 0, st>>>(tw, n);
  // The first pass writes every element of Z before any pass reads it, so the work array
  // needs no clearing between calls.
  for (int axis = 0; axis < d - 1; ++axis)
    k_fft_axis<<<blocks, threads, smem, st>>>(Z, u_dev, v_dev, y_dev, d, n, logn, axis, nlines, tw,
                                              axis == 0 ? kLoadReal : kPlain, 1);
  k_fft_axis<<<blocks, threads, smem, st>>>(Z, u_dev, v_dev, y_dev, d, n, logn, d - 1, nlines, tw,
                                            kSymbol, 1);
  for (int axis = d - 2; axis >= 0; --axis)
    k_fft_axis<<<blocks, threads, smem, st>>>(Z, u_dev, v_dev, y_dev, d, n, logn, axis, nlines, tw,
                                              axis == 0 ? kOutput : kPlain, 0);
  return cudaGetLastError() == cudaSuccess ? LSP_OK : LSP_ERR_CUDA;
}
