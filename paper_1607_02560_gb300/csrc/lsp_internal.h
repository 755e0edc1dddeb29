// Internal declarations shared by the translation units of liblsp.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <map>
#include <string>
#include <vector>

#include "../../include/lsp.h"

struct lsp_mlp;
namespace lsp {
struct NdState;
}

namespace lsp {

// pi^2 as the correctly rounded product of the double nearest pi. Kept identical on host and
// device so that lattice snapping takes bit-identical decisions everywhere.
constexpr double kPi = 3.141592653589793;
constexpr double kPi2 = kPi * kPi;
constexpr double kQuarterInvPi2 = 0.25 / kPi2;  // for the fast path of the lattice snap

constexpr int kMaxD = 3;
constexpr int kMaxMu = 27;      // (2t+1)^d of the symmetry-reduced paths: 27 (t = 1, 3D), 25 (t = 2, 2D)
constexpr int kMaxMuGeo = 125;  // (2t+1)^d of any neighbourhood: 125 for t = 2 in 3D
constexpr int kMaxCls = 15;     // sorted |offset| tuples: 10 over {0,1,2}^3, 15 over {0..4}^2
constexpr int kMaxSymVec = 19;  // symmetry-adapted basis vectors (19 for t = 2, d = 2)
constexpr int kMaxSymBlk = 6;
// counts[] layout: [0] |S|, [1], [2] sizes of the compacted stage domains, [kErrWord] device
// error bits, [16...] compaction tile scratch.
constexpr int kErrWord = 15;
// Arithmetic of the lattice-separable stages (a3): FP64, FP32 (mixed mode), double words of
// FP32 (the dword mode: about 48 significant bits on the FP32 pipe).
constexpr int kPrecFP64 = 0, kPrecFP32 = 1, kPrecDword = 2;
constexpr int kGateWord = 14;  // points the learned-stencil gate sent back to the eigen path
// Bit of the error word set by a checked build (-DLSP_CHECKS) when an index left its array.
constexpr int kErrBounds = 1 << 10;

#ifdef __CUDACC__
// The lattice shift s = (4m + 2) pi^2 (Sec. 4.1), evaluated identically wherever a kernel needs
// it (round-to-nearest product, no contraction).
__device__ __forceinline__ double lattice_shift(int64_t m) {
  return __dmul_rn((double)(4 * m + 2), kPi2);
}
// Checked builds (-DLSP_CHECKS): an index outside [0, n) is recorded in the error word and
// replaced by 0, so the access stays inside the array; plain builds compile this away.
__device__ __forceinline__ int64_t checked(int64_t i, int64_t n, int32_t* err) {
#ifdef LSP_CHECKS
  if (i < 0 || i >= n) {
    atomicOr(err, kErrBounds);
    return 0;
  }
#endif
  return i;
}
// True when [lo, hi] lies inside [0, n) (always true in plain builds); records otherwise.
__device__ __forceinline__ bool checked_range(int64_t lo, int64_t hi, int64_t n, int32_t* err) {
#ifdef LSP_CHECKS
  if (lo < 0 || hi >= n) {
    atomicOr(err, kErrBounds);
    return false;
  }
#endif
  return true;
}
#endif

// Symmetry-adapted basis of R^{|mu|} for the hyperoctahedral group acting on mu_0^t:
// one row of every irreducible representation that occurs. Block b has `dim` basis vectors
// (its multiplicity in mu_0) and stands for `copies` identical blocks (the irrep dimension).
struct SymBasis {
  int nblk;
  int dim[kMaxSymBlk];
  int copies[kMaxSymBlk];
  int first[kMaxSymBlk];          // index of its first vector
  int nvec;
  double u[kMaxSymVec][kMaxMu];   // orthonormal vectors, dense over mu_0
};

// Offset tables of mu_0^t.
struct Geometry {
  int d, n, t, mu, ncls, centre;
  int64_t N;
  int P;                           // n/2 + 1 frequencies per axis in [0, n/2]
  int off[kMaxMuGeo][kMaxD];             // mu_0 offsets, lexicographic
  uint8_t cls_of[kMaxMuGeo][kMaxMuGeo];  // class of o_a - o_b (sorted |components|)
};

// Launch shape of a tunable kernel: threads per block and the grid cap in CTAs per SM.
struct LaunchShape {
  int threads, per_sm;
};
struct TuneRecord {
  LaunchShape best;
  float ms_default, ms_best;
  int candidates;
};

struct Range {
  int64_t lo = 0, hi = -1;  // inclusive
  int64_t size() const { return hi >= lo ? hi - lo + 1 : 0; }
};

// Device buffer that only grows.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct KernelTimer {
  std::string name;
  double ms = 0;
  int64_t launches = 0;
};

}  // namespace lsp

struct lsp_ctx {
  lsp::Geometry geo;
  lsp::SymBasis sym;
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;

  // potential and its statistics (a1)
  bool have_v = false;
  double vmin = 0, vmax = 0, vmean = 0;
  lsp::DevBuf v, stats_part, stats;
  double* h_stats = nullptr;  // pinned
  double* h_stats_dev = nullptr;  // its device address (null: read back with a copy)

  // cos table X_a(p) = w_p cos(2 pi a p / n), a = 0..4, p = 0..n/2 (FP64 and FP32 copies;
  // t = 1 reads rows 0..2)
  lsp::DevBuf xtab, xtab32, xtabdw;

  // t = 2 neighbourhoods (2D): offsets, classes and symmetry basis of mu_0^2, and the build's
  // choice: rows of a t = 2 build are (2t+1)^d = 25 wide; with nd_leaf > 0 a point uses
  // t_j = min(2, largest t whose neighbourhood crosses no separator x_a = 0 mod nd_leaf) and
  // its inner 3 x 3 columns when t_j = 1
  lsp::Geometry geo2;
  lsp::SymBasis sym2;
  int t_built = 1, leaf_built = 0;

  // shift list (a2)
  bool built = false;
  int last_policy = -1;
  int64_t ns_host = -1;          // |S| when known on the host, else -1
  lsp::Range mrange;             // lattice index range covering S
  lsp::DevBuf shift_m, shift_flag, idx_of, counts;
  int32_t* h_list = nullptr;     // pinned staging for host-made shift lists
  int64_t h_list_cap = 0;

  // lattice-separable stages (a3)
  lsp::Range erange[lsp::kMaxD + 1];  // E_k ranges; E_d = shifts, E_0 = table domain
  lsp::DevBuf eflag[lsp::kMaxD], elist[lsp::kMaxD], T[lsp::kMaxD], wtab;
  bool edense[lsp::kMaxD] = {false, false, false};  // E_k evaluated over its whole range
  int64_t wtab_lo = 0, wtab_size = -1;  // range held by wtab (-1: none)
  int wtab_prec = -1;
  int64_t alloc_gen = 0;  // bumped whenever a device buffer is (re)allocated

  // per-shift results (a3-a6); *2: the t = 2 stencils
  lsp::DevBuf gvals, alpha, cst, lam, sflags, alpha2, cst2, lam2, sflags2;
  lsp::DevBuf ap;  // alpha - c s per shift and offset (t = 1): the P rows are fma(c, v, ap)
  // launch-shape autotuner (lsp_set_autotune): the first build of a configuration times
  // candidate shapes of the stage, eigen and row kernels eagerly; the winners are kept here
  bool autotune = false, tuning = false;
  std::map<std::string, lsp::TuneRecord> tune;
  std::vector<std::vector<int64_t>> tuned_configs;
  int64_t tune_gen = 0;  // bumped when a tuning pass changes shapes (invalidates the graph)
  // learned-stencil gate: per-point residual ratio of the last gated learned build
  lsp::DevBuf gate_rho;
  bool built_gated = false;

  // rows (a7) and export
  lsp::DevBuf Q, C, P, sidx, colidx, rowptr, expvals;
  // asynchronous host copies of the rows (lsp_get_rows_async): a device staging copy per block
  // (Q, C, P), taken on the context stream, is sent to the host on copy_stream, so that the next
  // build may overwrite the rows while the host copy is still in flight
  lsp::DevBuf stage[3];
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_staged[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_copied[3] = {nullptr, nullptr, nullptr};

  // FFT (apply_operator)
  lsp::DevBuf fftbuf, twiddle;

  // timing
  bool timing = false;
  std::vector<lsp::KernelTimer> timers;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  size_t ev_next = 0;

  // learned surrogate (LSP_LEARNED builds)
  lsp_mlp* mlp = nullptr;
  lsp::DevBuf learn_in;  // the network inputs (bf16, canonical tiles) of a learned build
  bool built_learned = false;
  int mode_used = -1;

  // nested dissection of P and the GMRES workspace (lsp_nd_factor, lsp_gmres); build_gen
  // counts successful builds so that a factorisation of older rows is never used
  lsp::NdState* nd = nullptr;
  int64_t build_gen = 0;

  // graph cache
  cudaGraphExec_t graph = nullptr;
  std::vector<int64_t> graph_key;
};

namespace lsp {

// ---- host helpers (lsp_api.cu) ----
bool ensure(lsp_ctx* ctx, DevBuf& b, size_t bytes);
// True when an injected allocation failure is due (lsp_inject_alloc_failure).
bool alloc_should_fail();
int timer_begin(lsp_ctx* ctx, const char* name);
void timer_end(lsp_ctx* ctx, int slot);

// ---- launchers; each returns cudaGetLastError() after the launch ----
// src: c->v itself, or page-locked host memory (device address) that is copied into c->v
// v_min, v_max, sum and the count of non-finite values of v in stats[0..3] (one launch; the
// ticket of its last block lives in stats[4] and is zero between calls).
cudaError_t launch_stats(lsp_ctx* c, int nblocks, const double* src);
// bytes / 4 words of p set to zero (bytes a multiple of 4, p 4-byte aligned)
cudaError_t launch_zero(lsp_ctx* c, void* p, size_t bytes);
// n doubles from src to dst (device, 16-byte aligned)
cudaError_t launch_copy_f64(lsp_ctx* c, const double* src, double* dst, int64_t n);
cudaError_t launch_mark_local(lsp_ctx* c);
cudaError_t launch_compact(lsp_ctx* c, const uint8_t* flags, int64_t lo, int64_t range,
                           int32_t* list, int32_t* count, int32_t* idx_of);
cudaError_t launch_mark_stage(lsp_ctx* c, const int32_t* list, const int32_t* count,
                              int64_t cap, int64_t lo_prev, uint8_t* flag_prev);
cudaError_t launch_wtable(lsp_ctx* c, int64_t lo, int64_t range, void* w, int prec);
cudaError_t launch_stage(lsp_ctx* c, int d, int k, int t, const int32_t* list,
                         const int32_t* count, int64_t cap, const void* Tprev, int64_t lo_prev,
                         int64_t stride_prev, void* Tout, int64_t lo_out, int64_t stride_out,
                         bool by_index, int prec);
cudaError_t launch_eig_t2(lsp_ctx* c, const int32_t* count, int64_t cap);
cudaError_t launch_eig_dense3(lsp_ctx* c, const int32_t* count, int64_t cap);
cudaError_t upload_cls125(const Geometry& g);
cudaError_t launch_rows_t2(lsp_ctx* c, int policy, const int32_t* count, int leaf);
cudaError_t launch_export_t2(lsp_ctx* c, const double* rows, int leaf, const int64_t* rowptr,
                             int32_t* colidx, double* vals);
cudaError_t launch_eig(lsp_ctx* c, const int32_t* count, int64_t cap, int eig_method,
                       int refine_steps, bool fp32_gram);
cudaError_t launch_rows(lsp_ctx* c, int policy, const int32_t* count);
cudaError_t launch_sidx(lsp_ctx* c, int policy, const int32_t* count);
// Launch through the autotuner: the tuned shape of `key` if there is one; during a tuning pass
// (ctx->tuning) each candidate shape is timed (side-effect-free kernels only: the launch must
// be repeatable) and the fastest kept; otherwise `def`. threads_max bounds the block size (the
// kernel's launch bound); fixed_threads > 0 tunes only the grid cap.
cudaError_t tuned_launch(lsp_ctx* c, const std::string& key, LaunchShape def, int threads_max,
                         int fixed_threads, const std::function<cudaError_t(LaunchShape)>& launch);
std::string work_bucket(int64_t work);
cudaError_t launch_learned_gate(lsp_ctx* c, int policy, const int32_t* count, int64_t cap,
                                double tau, float* rho, int32_t* nfall);
cudaError_t launch_colidx(lsp_ctx* c);
cudaError_t launch_apply(lsp_ctx* c, const double* u, double* y);
void nd_free(NdState* s);
cudaError_t upload_sym(lsp_ctx* c);
cudaError_t launch_learned_rows(lsp_ctx* c, lsp_mlp* m);
bool mlp_input_range(lsp_mlp* m, float* lo, float* hi);
int mlp_dim(const lsp_mlp* m);
cudaError_t mlp_sync(lsp_mlp* m);

}  // namespace lsp
