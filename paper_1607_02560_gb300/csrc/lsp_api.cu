// Host side of the C ABI declared in include/lsp.h: context life cycle, buffer management,
// the launch sequence of build_stencils (steps a1-a7), CUDA-graph replay, per-kernel timing,
// and the copy-out calls.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <atomic>

#include "lsp_internal.h"

using namespace lsp;

namespace {

lsp_status fail(lsp_ctx* c, lsp_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return st;
}

#define CUDA_OK(ctx, expr)                                                               \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess)                                                               \
      return fail(ctx, _e == cudaErrorMemoryAllocation ? LSP_ERR_OOM : LSP_ERR_CUDA,     \
                  "%s failed: %s", #expr, cudaGetErrorString(_e));                       \
  } while (0)

// Lattice index of the shift (4m+2) pi^2 nearest to x, halves away from zero (Sec. 4.1).
// Host code is compiled without floating-point contraction, so this is the plain IEEE
// evaluation, identical to the device version.
int64_t snap_host(double x) {
  volatile double q = x / kPi2;
  volatile double r = (q - 2.0) * 0.25;
  return (int64_t)round(r);
}
double shift_host(int64_t m) {
  volatile double a = (double)(4 * m + 2);
  return a * kPi2;
}

// Classes of the stage-k table: sorted k-tuples over {0..2t} (t = 1: 3, 6, 10; t = 2: 5, 15, 35).
int ncls_stage(int k, int t = 1) {
  return t == 1 ? (k == 1 ? 3 : (k == 2 ? 6 : 10)) : (k == 1 ? 5 : (k == 2 ? 15 : 35));
}

// Is r = |k|^2 for some k in K = [-n/2, n/2)^d ?  (the eigenvalues of L are 4 pi^2 |k|^2)
bool is_norm(int64_t r, int d, int half) {
  for (int64_t a = 0; a <= half; ++a) {
    const int64_t ra = r - a * a;
    if (ra < 0) break;
    if (d == 1) {
      if (ra == 0) return true;
      continue;
    }
    for (int64_t b = 0; b <= half; ++b) {
      const int64_t rb = ra - b * b;
      if (rb < 0) break;
      if (d == 2) {
        if (rb == 0) return true;
        continue;
      }
      const int64_t c = (int64_t)llround(sqrt((double)rb));
      if (c <= half && c * c == rb) return true;
    }
  }
  return false;
}

// ---- geometry and symmetry basis ------------------------------------------------------

// Class of a sorted pair a <= b of |offset| components: the six pairs over {0,1,2} in the order
// 00 01 02 11 12 22, then (t = 2) the pairs with b = 3 (03 13 23 33) and b = 4 (04 .. 44), so
// the classes of t = 1 keep their indices in a t = 2 table (the stage kernels use this order).
int pair_index(int a, int b) {
  static const int t[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  return b <= 2 ? t[a][b] : b * (b + 1) / 2 + a;
}
// Class of a sorted triple a <= b <= c of |offset| components: the ten triples over {0,1,2}
// in the order 000 001 002 011 012 022 111 112 122 222, then (t = 2) the triples with largest
// component 3 and then 4, each group in lexicographic order, so the classes of t = 1 keep
// their indices in a t = 2 table (the stage kernels use this order).
int triple_index(int a, int b, int c) {  // a <= b <= c
  int idx = 0;
  for (int top = 2; top <= 4; ++top)
    for (int x = 0; x <= top; ++x)
      for (int y = x; y <= top; ++y)
        for (int z = y; z <= top; ++z) {
          if (top > 2 && z != top) continue;  // groups: max <= 2, then max = 3, max = 4
          if (x == a && y == b && z == c) return idx;
          ++idx;
        }
  return -1;
}

// mu_0^t = [-t, t]^d (t = 1 in 2D and 3D, t = 2 in 2D), lexicographic, last axis fastest.
void build_geometry(Geometry& g, int d, int n, int t = 1) {
  memset(&g, 0, sizeof g);
  g.d = d;
  g.n = n;
  g.t = t;
  const int w = 2 * t + 1;
  g.mu = d == 1 ? w : (d == 2 ? w * w : w * w * w);
  g.ncls = d == 1 ? 2 * t + 1 : (d == 2 ? w * (w + 1) / 2 : w * (w + 1) * (w + 2) / 6);
  g.centre = g.mu / 2;
  g.N = 1;
  for (int i = 0; i < d; ++i) g.N *= n;
  g.P = n / 2 + 1;
  for (int a = 0; a < g.mu; ++a) {
    int rem = a;
    for (int i = d - 1; i >= 0; --i) {
      g.off[a][i] = rem % w - t;
      rem /= w;
    }
  }
  for (int a = 0; a < g.mu; ++a)
    for (int b = 0; b < g.mu; ++b) {
      int v[3] = {0, 0, 0};
      for (int i = 0; i < d; ++i) v[i] = abs(g.off[a][i] - g.off[b][i]);
      std::sort(v, v + d);
      g.cls_of[a][b] = (uint8_t)(d == 1 ? v[0]
                                        : d == 2 ? pair_index(v[0], v[1])
                                                 : triple_index(v[0], v[1], v[2]));
    }
}

// Symmetry-adapted vectors: block = one row of an irreducible representation of the signed
// permutation group; vector = a polynomial pattern restricted to one orbit of mu_0 (the points
// with exactly k nonzero offsets).
enum Pat { kOne, kX, kX2mY2, kXY, kXY2mZ2, kXYZ };
double pattern(int kind, const int* o) {
  const double x = o[0], y = o[1], z = o[2];
  switch (kind) {
    case kOne: return 1.0;
    case kX: return x;
    case kX2mY2: return x * x - y * y;
    case kXY: return x * y;
    case kXY2mZ2: return x * (y * y - z * z);
    default: return x * y * z;
  }
}

bool build_sym(SymBasis& s, const Geometry& g) {
  memset(&s, 0, sizeof s);
  struct Blk { int copies; int nv; int orbit[4]; int kind[4]; };
  std::vector<Blk> blks;
  if (g.d == 1) {  // the reflection o -> -o: even (centre, the pair) and odd (the pair)
    blks = {{1, 2, {0, 1}, {kOne, kOne}}, {1, 1, {1}, {kX}}};
  } else if (g.d == 2) {
    blks = {{1, 3, {0, 1, 2}, {kOne, kOne, kOne}},
            {1, 1, {1}, {kX2mY2}},
            {1, 1, {2}, {kXY}},
            {2, 2, {1, 2}, {kX, kX}}};
  } else {
    blks = {{1, 4, {0, 1, 2, 3}, {kOne, kOne, kOne, kOne}},
            {3, 3, {1, 2, 3}, {kX, kX, kX}},
            {2, 2, {1, 2}, {kX2mY2, kX2mY2}},
            {3, 2, {2, 3}, {kXY, kXY}},
            {3, 1, {2}, {kXY2mZ2}},
            {1, 1, {3}, {kXYZ}}};
  }
  s.nblk = (int)blks.size();
  int total = 0;
  for (int b = 0; b < s.nblk; ++b) {
    s.dim[b] = blks[b].nv;
    s.copies[b] = blks[b].copies;
    s.first[b] = s.nvec;
    total += blks[b].nv * blks[b].copies;
    for (int i = 0; i < blks[b].nv; ++i) {
      double* u = s.u[s.nvec++];
      double nrm = 0.0;
      for (int a = 0; a < g.mu; ++a) {
        int o[3] = {0, 0, 0}, nz = 0;
        for (int k = 0; k < g.d; ++k) {
          o[k] = g.off[a][k];
          nz += o[k] != 0;
        }
        u[a] = nz == blks[b].orbit[i] ? pattern(blks[b].kind[i], o) : 0.0;
        nrm += u[a] * u[a];
      }
      if (nrm == 0.0) return false;
      nrm = sqrt(nrm);
      for (int a = 0; a < g.mu; ++a) u[a] /= nrm;
    }
  }
  if (total != g.mu) return false;
  for (int i = 0; i < s.nvec; ++i)
    for (int j = 0; j < s.nvec; ++j) {
      double dot = 0.0;
      for (int a = 0; a < g.mu; ++a) dot += s.u[i][a] * s.u[j][a];
      if (fabs(dot - (i == j ? 1.0 : 0.0)) > 1e-14) return false;
    }
  return true;
}

// Symmetry-adapted basis of mu_0^2 in 2D (25 points, orbits of the signed permutations of the
// axes: |o| = (0,0), (0,1), (1,1), (0,2), (1,2), (2,2) of sizes 1, 4, 4, 4, 8, 4). Blocks:
// A1 (the constant on each orbit, 6), A2 (xy(x^2 - y^2) on (1,2)), B1 (x^2 - y^2 on (0,1),
// (0,2), (1,2)), B2 (xy on (1,1), (2,2), (1,2)) and E (partner x: x on (0,1), (1,1), (0,2),
// (2,2), (1,2), and x y^2 on (1,2); 2 copies). Vectors of a block are orthonormalised in
// order (Gram-Schmidt: x and x y^2 share the 8-point orbit).
bool build_sym_t2(SymBasis& s, const Geometry& g) {
  memset(&s, 0, sizeof s);
  if (g.d != 2 || g.t != 2) return false;
  enum { kOne, kX, kX2mY2, kXY, kXYx2mY2, kXY2 };
  struct Vec { int o0, o1, kind; };
  struct Blk { int copies; int nv; Vec v[6]; };
  const Blk blks[5] = {
      {1, 6, {{0, 0, kOne}, {0, 1, kOne}, {1, 1, kOne}, {0, 2, kOne}, {1, 2, kOne}, {2, 2, kOne}}},
      {2, 6, {{0, 1, kX}, {1, 1, kX}, {0, 2, kX}, {2, 2, kX}, {1, 2, kX}, {1, 2, kXY2}}},
      {1, 3, {{0, 1, kX2mY2}, {0, 2, kX2mY2}, {1, 2, kX2mY2}}},
      {1, 3, {{1, 1, kXY}, {2, 2, kXY}, {1, 2, kXY}}},
      {1, 1, {{1, 2, kXYx2mY2}}}};
  s.nblk = 5;
  int total = 0;
  for (int b = 0; b < s.nblk; ++b) {
    s.dim[b] = blks[b].nv;
    s.copies[b] = blks[b].copies;
    s.first[b] = s.nvec;
    total += blks[b].nv * blks[b].copies;
    for (int i = 0; i < blks[b].nv; ++i) {
      double* u = s.u[s.nvec];
      for (int a = 0; a < g.mu; ++a) {
        const int x = g.off[a][0], y = g.off[a][1];
        int o[2] = {abs(x), abs(y)};
        if (o[0] > o[1]) std::swap(o[0], o[1]);
        double val = 0.0;
        if (o[0] == blks[b].v[i].o0 && o[1] == blks[b].v[i].o1) {
          switch (blks[b].v[i].kind) {
            case kOne: val = 1.0; break;
            case kX: val = x; break;
            case kX2mY2: val = x * x - y * y; break;
            case kXY: val = x * y; break;
            case kXYx2mY2: val = x * y * (x * x - y * y); break;
            default: val = x * y * y; break;
          }
        }
        u[a] = val;
      }
      for (int k = s.first[b]; k < s.nvec; ++k) {  // Gram-Schmidt within the block
        double dot = 0.0;
        for (int a = 0; a < g.mu; ++a) dot += s.u[k][a] * u[a];
        for (int a = 0; a < g.mu; ++a) u[a] -= dot * s.u[k][a];
      }
      double nrm = 0.0;
      for (int a = 0; a < g.mu; ++a) nrm += u[a] * u[a];
      if (nrm < 1e-12) return false;
      nrm = sqrt(nrm);
      for (int a = 0; a < g.mu; ++a) u[a] /= nrm;
      ++s.nvec;
    }
  }
  if (total != g.mu) return false;
  for (int i = 0; i < s.nvec; ++i)
    for (int j = 0; j < s.nvec; ++j) {
      double dot = 0.0;
      for (int a = 0; a < g.mu; ++a) dot += s.u[i][a] * s.u[j][a];
      if (fabs(dot - (i == j ? 1.0 : 0.0)) > 1e-13) return false;
    }
  return true;
}

size_t round_up(size_t x, size_t m) { return (x + m - 1) / m * m; }

}  // namespace

namespace lsp {
bool ensure(lsp_ctx* c, DevBuf& b, size_t bytes);
}
namespace {
// ensure() that also forgets a cached content key when the buffer is reallocated.
bool ensure_tracked(lsp_ctx* c, lsp::DevBuf& b, size_t bytes, int64_t* key) {
  void* before = b.p;
  if (!lsp::ensure(c, b, bytes)) return false;
  if (b.p != before) *key = -1;
  return true;
}
}  // namespace

namespace lsp {

// Allocation-failure injection (lsp_inject_alloc_failure): allocations left before the one
// that fails; -1 when off.
static std::atomic<int> g_alloc_fail_in{-1};

bool alloc_should_fail() {
  int k = g_alloc_fail_in.load();
  while (k >= 0) {
    if (g_alloc_fail_in.compare_exchange_weak(k, k - 1)) return k == 0;
  }
  return false;
}

bool ensure(lsp_ctx* c, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return true;
  ++c->alloc_gen;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  size_t want = round_up(bytes, 256);
  if (alloc_should_fail() || cudaMalloc(&b.p, want) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    c->err = "device allocation of " + std::to_string(want) + " bytes failed";
    return false;
  }
  b.bytes = want;
  return true;
}

std::string work_bucket(int64_t work) {
  int b = 0;
  while (b < 62 && ((int64_t)1 << b) < work) ++b;
  return std::to_string(b);
}

cudaError_t tuned_launch(lsp_ctx* c, const std::string& key, LaunchShape def, int threads_max,
                         int fixed_threads, const std::function<cudaError_t(LaunchShape)>& launch) {
  auto it = c->tune.find(key);
  if (it != c->tune.end()) return launch(it->second.best);
  if (!c->tuning) return launch(def);
  // candidates: the default first, then threads x grid caps (CTAs per SM)
  std::vector<LaunchShape> cand = {def};
  const int th_opts[3] = {64, 128, 256}, sm_opts[5] = {2, 4, 8, 16, 32};
  for (int th : th_opts) {
    if (th > threads_max || (fixed_threads > 0 && th != fixed_threads)) continue;
    for (int ps : sm_opts)
      if (!(th == def.threads && ps == def.per_sm)) cand.push_back({th, ps});
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cudaGetLastError();
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cudaGetLastError();
  }
  float best_ms = 1e30f, def_ms = 0.0f;
  LaunchShape best = def;
  cudaError_t err = cudaSuccess;
  for (size_t k = 0; k < cand.size() && err == cudaSuccess; ++k) {
    err = launch(cand[k]);  // warm
    float ms = 1e30f;
    for (int r = 0; r < 3 && err == cudaSuccess; ++r) {
      cudaEventRecord(e0, c->stream);
      err = launch(cand[k]);
      cudaEventRecord(e1, c->stream);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float t = 0.0f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
      if (t < ms) ms = t;
    }
    if (k == 0) def_ms = ms;
    if (ms < best_ms * 0.98f || k == 0) {  // a new shape must win by 2%
      best_ms = ms;
      best = cand[k];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return err;
  c->tune[key] = {best, def_ms, best_ms, (int)cand.size()};
  return launch(best);
}

int timer_begin(lsp_ctx* c, const char* name) {
  if (!c->timing) return -1;
  int slot = -1;
  for (size_t i = 0; i < c->timers.size(); ++i)
    if (c->timers[i].name == name) slot = (int)i;
  if (slot < 0) {
    c->timers.push_back({name, 0.0, 0});
    slot = (int)c->timers.size() - 1;
  }
  if (c->ev_next + 2 > c->ev_pool.size()) {
    for (int k = 0; k < 64; ++k) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      c->ev_pool.push_back(e);
    }
  }
  cudaEvent_t e0 = c->ev_pool[c->ev_next++], e1 = c->ev_pool[c->ev_next++];
  cudaEventRecord(e0, c->stream);
  c->ev_pending.push_back({slot, {e0, e1}});
  return (int)c->ev_pending.size() - 1;
}

void timer_end(lsp_ctx* c, int t) {
  if (t < 0 || !c->timing) return;
  cudaEventRecord(c->ev_pending[t].second.second, c->stream);
}

}  // namespace lsp

namespace {

lsp_status flush_timers(lsp_ctx* c) {
  if (c->ev_pending.empty()) return LSP_OK;
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  for (auto& pe : c->ev_pending) {
    float ms = 0;
    CUDA_OK(c, cudaEventElapsedTime(&ms, pe.second.first, pe.second.second));
    c->timers[pe.first].ms += ms;
    c->timers[pe.first].launches += 1;
  }
  c->ev_pending.clear();
  c->ev_next = 0;
  return LSP_OK;
}

// The launch sequence of steps a2-a7 for the sizes already prepared in the context.
// Arithmetic of the a3 stages for a build: FP32 in the mixed mode; double words in the dword
// mode for t = 1 in 1D and 2D (in 3D the stages are a small part of the build and the
// tolerance, set by the spectral gap, is tight, so they stay FP64); FP64 otherwise.
int stage_prec(const lsp_ctx* c, const lsp_stencil_opts& o) {
  if (o.mode == LSP_MIXED) return kPrecFP32;
  if (o.mode == LSP_DWORD && o.t == 1 && c->geo.d <= 2) return kPrecDword;
  return kPrecFP64;
}

lsp_status issue_build(lsp_ctx* c, const lsp_stencil_opts& o, int64_t cap_s, bool upload,
                       bool rows = true) {
  const int d = c->geo.d;
  int32_t* counts = (int32_t*)c->counts.p;
  // zeroing by kernels: a memset may be queued behind host copies on the copy engines
  CUDA_OK(c, launch_zero(c, counts + kErrWord, sizeof(int32_t)));
  if (o.policy == LSP_SHIFT_LOCAL) {
    const int64_t R = c->mrange.size();
    CUDA_OK(c, launch_zero(c, c->shift_flag.p, round_up(R, 4096)));
    CUDA_OK(c, launch_mark_local(c));
    CUDA_OK(c, launch_compact(c, (const uint8_t*)c->shift_flag.p, c->mrange.lo, R,
                              (int32_t*)c->shift_m.p, counts + 0, (int32_t*)c->idx_of.p));
  } else if (upload) {
    CUDA_OK(c, cudaMemcpyAsync(c->shift_m.p, c->h_list, sizeof(int32_t) * cap_s,
                               cudaMemcpyHostToDevice, c->stream));
    CUDA_OK(c, cudaMemcpyAsync(counts, c->h_list + cap_s, sizeof(int32_t),
                               cudaMemcpyHostToDevice, c->stream));
  }
  const int32_t* list = (const int32_t*)c->shift_m.p;
  const int32_t* count = counts + 0;
  int64_t cap = cap_s;
  for (int k = d - 1; k >= 1; --k) {
    const int64_t sz = c->erange[k].size();
    if (c->edense[k]) {
      // every l of the range is evaluated: no marking or compaction needed
      list = nullptr;
      count = nullptr;
      cap = sz;
      continue;
    }
    CUDA_OK(c, launch_zero(c, c->eflag[k].p, round_up(sz, 4096)));
    CUDA_OK(c, launch_mark_stage(c, list, count, cap, c->erange[k].lo, (uint8_t*)c->eflag[k].p));
    CUDA_OK(c, launch_compact(c, (const uint8_t*)c->eflag[k].p, c->erange[k].lo, sz,
                              (int32_t*)c->elist[k].p, counts + (d - k), nullptr));
    list = (const int32_t*)c->elist[k].p;
    count = counts + (d - k);
    cap = sz;
  }
  const int prec = stage_prec(c, o);  // the w table is refreshed by the caller
  const bool fp32 = prec == kPrecFP32;
  for (int k = 1; k <= d; ++k) {
    const void* prev = k == 1 ? c->wtab.p : c->T[k - 1].p;
    const int64_t lo_prev = c->erange[k - 1].lo, stride_prev = c->erange[k - 1].size();
    if (k < d) {
      const bool dense = c->edense[k];
      CUDA_OK(c, launch_stage(c, d, k, o.t, dense ? nullptr : (const int32_t*)c->elist[k].p,
                              dense ? nullptr : counts + (d - k), c->erange[k].size(), prev,
                              lo_prev, stride_prev, c->T[k].p, c->erange[k].lo,
                              c->erange[k].size(), false, prec));
    } else {
      CUDA_OK(c, launch_stage(c, d, k, o.t, (const int32_t*)c->shift_m.p, counts + 0, cap_s,
                              prev, lo_prev, stride_prev, c->gvals.p, 0, cap_s, true, prec));
    }
  }
  // t = 1 stencils read the first classes of a t = 2 table (same row stride cap_s)
  // the eigen kernels also write ap = alpha - c s per shift for the P rows
  if (o.t == 1 || o.nd_leaf > 0)
    CUDA_OK(c, launch_eig(c, counts + 0, cap_s, o.eig_method, o.refine_steps, fp32));
  if (o.t == 2) {
    if (d == 2)
      CUDA_OK(c, launch_eig_t2(c, counts + 0, cap_s));
    else
      CUDA_OK(c, launch_eig_dense3(c, counts + 0, cap_s));
    CUDA_OK(c, launch_rows_t2(c, o.policy, counts + 0, o.nd_leaf));
  } else if (rows) {
    CUDA_OK(c, launch_rows(c, o.policy, counts + 0));
  }
  return LSP_OK;
}

}  // namespace

extern "C" {

void lsp_inject_alloc_failure(int after) { lsp::g_alloc_fail_in.store(after < 0 ? -1 : after); }

void lsp_default_opts(lsp_stencil_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->t = 1;
  o->policy = LSP_SHIFT_LOCAL;
  o->mode = LSP_FP64;
  o->eig_method = LSP_EIG_SYMMETRIC;
  o->learned_gate = 0.0;
}

lsp_status lsp_create(int d, int n, void* cuda_stream, lsp_ctx** out) {
  if (!out) return LSP_ERR_ARG;
  *out = nullptr;
  if (d < 1 || d > 3) return LSP_ERR_ARG;
  if (n < 8 || (n & (n - 1)) != 0 || n > (d == 3 ? 256 : 4096)) return LSP_ERR_ARG;
  lsp_ctx* c = new (std::nothrow) lsp_ctx();
  if (!c) return LSP_ERR_OOM;
  c->stream = (cudaStream_t)cuda_stream;
  build_geometry(c->geo, d, n);
  if (!build_sym(c->sym, c->geo)) {
    delete c;
    return LSP_ERR_STATE;
  }
  if (d == 2) {  // t = 2 neighbourhoods (2D: symmetry-reduced eigen path)
    build_geometry(c->geo2, d, n, 2);
    if (!build_sym_t2(c->sym2, c->geo2)) {
      delete c;
      return LSP_ERR_STATE;
    }
  } else if (d == 3 && n >= 8) {  // t = 2 neighbourhoods (3D: dense eigen path)
    build_geometry(c->geo2, d, n, 2);
  }
  lsp_status st = LSP_OK;
  do {
    if (cudaGetDevice(&c->device) != cudaSuccess) {
      st = LSP_ERR_CUDA;
      break;
    }
    if (cudaMallocHost(&c->h_stats, 8 * sizeof(double)) != cudaSuccess) {
      st = LSP_ERR_OOM;
      break;
    }
    if (cudaHostGetDevicePointer((void**)&c->h_stats_dev, c->h_stats, 0) != cudaSuccess) {
      cudaGetLastError();
      c->h_stats_dev = nullptr;
    }
    if (upload_sym(c) != cudaSuccess) {
      st = LSP_ERR_CUDA;
      break;
    }
    if (d == 3 && n >= 8 && upload_cls125(c->geo2) != cudaSuccess) {
      st = LSP_ERR_CUDA;
      break;
    }
    // X_a(p) = w_p cos(2 pi a p / n), a = 0..4, w_p = 1 at p = 0 and p = n/2, else 2. The cosine of
    // 2 pi r / n is taken from the first octant by exact symmetries, so the table satisfies
    // cos(pi a - t) = (-1)^a cos(t) (used by the mirror pairing of stage 1) bit for bit.
    const int P = c->geo.P;
    std::vector<double> X(5 * P);
    const long double two_pi = 6.283185307179586476925286766559005768L;
    auto cos_r = [&](int r) -> long double {  // cos(2 pi r / n), r in [0, n)
      r %= n;
      int sign = 1;
      if (r > n / 2) r = n - r;            // cos(2 pi - t) = cos t
      if (r > n / 4) {                     // cos(pi - t) = -cos t
        r = n / 2 - r;
        sign = -1;
      }
      long double val;
      if (r == 0)
        val = 1.0L;
      else if (4 * r == n)
        val = 0.0L;
      else if (8 * r > n)                   // cos t = sin(pi/2 - t)
        val = sinl(two_pi * (long double)(n / 4 - r) / (long double)n);
      else
        val = cosl(two_pi * (long double)r / (long double)n);
      return sign * val;
    };
    for (int a = 0; a < 5; ++a)
      for (int p = 0; p < P; ++p) {
        const long double wgt = (p == 0 || p == n / 2) ? 1.0L : 2.0L;
        X[a * P + p] = (double)(wgt * cos_r(a * p));
      }
    // twiddles exp(-2 pi i j / n), j < n/2
    std::vector<double> tw(n);
    for (int j = 0; j < n / 2; ++j) {
      const long double ang = two_pi * (long double)j / (long double)n;
      tw[2 * j] = (double)cosl(ang);
      tw[2 * j + 1] = (double)(-sinl(ang));
    }
    std::vector<float> X32(X.begin(), X.end());
    // double words of the same values, split from the extended-precision cosines
    std::vector<float> Xdw(2 * 5 * P);
    for (int a = 0; a < 5; ++a)
      for (int p = 0; p < P; ++p) {
        const long double wgt = (p == 0 || p == n / 2) ? 1.0L : 2.0L;
        const long double x = wgt * cos_r(a * p);
        const float hi = (float)x;
        Xdw[2 * (a * P + p)] = hi;
        Xdw[2 * (a * P + p) + 1] = (float)(x - (long double)hi);
      }
    if (!ensure(c, c->xtabdw, sizeof(float) * Xdw.size()) ||
        cudaMemcpy(c->xtabdw.p, Xdw.data(), sizeof(float) * Xdw.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
      st = LSP_ERR_CUDA;
      break;
    }
    if (!ensure(c, c->xtab32, sizeof(float) * X32.size()) ||
        cudaMemcpy(c->xtab32.p, X32.data(), sizeof(float) * X32.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
      st = LSP_ERR_CUDA;
      break;
    }
    if (!ensure(c, c->xtab, sizeof(double) * X.size()) ||
        !ensure(c, c->twiddle, sizeof(double) * tw.size()) ||
        !ensure(c, c->stats, 8 * sizeof(double))) {
      st = LSP_ERR_OOM;
      break;
    }
    if (cudaMemset(c->stats.p, 0, 8 * sizeof(double)) != cudaSuccess ||  // zero ticket
        cudaMemcpy(c->xtab.p, X.data(), sizeof(double) * X.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(c->twiddle.p, tw.data(), sizeof(double) * tw.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
      st = LSP_ERR_CUDA;
      break;
    }
  } while (0);
  if (st != LSP_OK) {
    lsp_destroy(c);
    return st;
  }
  *out = c;
  return LSP_OK;
}

lsp_status lsp_destroy(lsp_ctx* c) {
  if (!c) return LSP_OK;
  cudaStreamSynchronize(c->stream);
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamDestroy(c->copy_stream);
  }
  for (int k = 0; k < 3; ++k) {
    if (c->stage[k].p) cudaFree(c->stage[k].p);
    if (c->ev_staged[k]) cudaEventDestroy(c->ev_staged[k]);
    if (c->ev_copied[k]) cudaEventDestroy(c->ev_copied[k]);
  }
  DevBuf* bufs[] = {&c->v, &c->stats_part, &c->stats, &c->xtab, &c->xtab32, &c->xtabdw, &c->shift_m, &c->shift_flag,
                    &c->idx_of, &c->counts, &c->wtab, &c->gvals, &c->alpha, &c->cst, &c->ap, &c->lam,
                    &c->sflags, &c->Q, &c->C, &c->P, &c->sidx, &c->colidx, &c->rowptr,
                    &c->fftbuf, &c->twiddle, &c->learn_in, &c->alpha2, &c->cst2, &c->lam2,
                    &c->sflags2, &c->expvals};
  for (DevBuf* b : bufs)
    if (b->p) cudaFree(b->p);
  for (int k = 0; k < kMaxD; ++k) {
    if (c->eflag[k].p) cudaFree(c->eflag[k].p);
    if (c->elist[k].p) cudaFree(c->elist[k].p);
    if (c->T[k].p) cudaFree(c->T[k].p);
  }
  if (c->h_stats) cudaFreeHost(c->h_stats);
  if (c->h_list) cudaFreeHost(c->h_list);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  nd_free(c->nd);
  delete c;
  return LSP_OK;
}

lsp_status lsp_set_potential(lsp_ctx* c, const double* v, int v_on_device) {
  if (!c) return LSP_ERR_ARG;
  cudaGetLastError();  // a launch check below must not report an earlier, unrelated error
  if (!v) return fail(c, LSP_ERR_ARG, "v is NULL");
  const int64_t N = c->geo.N;
  if (!ensure(c, c->v, sizeof(double) * N)) return LSP_ERR_OOM;
  // Page-locked host memory is read by the statistics kernel itself, which also stores v on
  // the device; pageable host memory and device memory are copied first. Neither the upload
  // nor the read-back of the statistics then waits behind host copies still in flight on the
  // copy engines (lsp_get_rows_async of the previous build).
  const double* src = nullptr;
  if (!v_on_device) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, v) == cudaSuccess && at.type == cudaMemoryTypeHost &&
        at.devicePointer)
      src = (const double*)at.devicePointer;
    cudaGetLastError();
  }
  if (!src) {
    CUDA_OK(c, cudaMemcpyAsync(c->v.p, v, sizeof(double) * N,
                               v_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                               c->stream));
    src = (const double*)c->v.p;
  }
  // one block per SM: fewer partials for the last block to reduce (measured 20 -> 16 us in 3D
  // n = 64, 29 -> 23 us in 2D n = 1024 against four per SM)
  int nb = (int)std::min<int64_t>(152, (N + 255) / 256);
  if (!ensure(c, c->stats_part, sizeof(double) * 4 * nb)) return LSP_ERR_OOM;
  CUDA_OK(c, launch_stats(c, nb, src));
  if (!c->h_stats_dev)
    CUDA_OK(c, cudaMemcpyAsync(c->h_stats, c->stats.p, 4 * sizeof(double),
                               cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  c->have_v = false;
  c->built = false;
  if (c->h_stats[3] > 0)
    return fail(c, LSP_ERR_ARG, "v holds %.0f NaN/Inf values", c->h_stats[3]);
  c->vmin = c->h_stats[0];
  c->vmax = c->h_stats[1];
  c->vmean = c->h_stats[2] / (double)N;
  const double half = (double)(c->geo.n / 2);
  const double lim = 1073741824.0 - c->geo.d * half * half - 16;
  if (fabs((double)snap_host(c->vmin)) > lim || fabs((double)snap_host(c->vmax)) > lim)
    return fail(c, LSP_ERR_ARG, "potential range [%g, %g] exceeds the lattice index range",
                c->vmin, c->vmax);
  c->have_v = true;
  return LSP_OK;
}

lsp_status lsp_build_stencils(lsp_ctx* c, const lsp_stencil_opts* opts) {
  if (!c) return LSP_ERR_ARG;
  cudaGetLastError();
  lsp_stencil_opts o;
  if (opts)
    o = *opts;
  else
    lsp_default_opts(&o);
  if (!c->have_v) return fail(c, LSP_ERR_STATE, "build_stencils before set_potential");
  if (o.t != 1 && o.t != 2) return fail(c, LSP_ERR_ARG, "t must be 1 or 2");
  if (o.t == 2 && c->geo.d == 1)
    return fail(c, LSP_ERR_UNSUPPORTED, "t = 2 neighbourhoods are built in 2D and 3D");
  if (o.t == 2 && c->geo.n < 8)
    return fail(c, LSP_ERR_UNSUPPORTED, "t = 2 neighbourhoods need n >= 8");
  if (o.nd_leaf < 0 || (o.nd_leaf > 0 && (o.nd_leaf < 2 || c->geo.n % o.nd_leaf != 0)))
    return fail(c, LSP_ERR_ARG, "nd_leaf must be 0 or an even divisor >= 2 of n");
  if (o.t == 2 && o.mode == LSP_LEARNED)
    return fail(c, LSP_ERR_UNSUPPORTED, "learned builds use t = 1 neighbourhoods");
  if (o.mode != LSP_FP64 && o.mode != LSP_MIXED && o.mode != LSP_LEARNED && o.mode != LSP_DWORD)
    return fail(c, LSP_ERR_ARG, "bad mode %d", o.mode);
  bool gated = false;
  if (o.mode == LSP_LEARNED) {
    if (!c->mlp) return fail(c, LSP_ERR_STATE, "LEARNED build without a network (lsp_set_mlp)");
    // Gate: the network answers only inside the h^2 v range it was trained on; outside it
    // the FP64 eigen path builds the stencils instead.
    float lo = 0, hi = 0;
    if (!mlp_input_range(c->mlp, &lo, &hi)) return fail(c, LSP_ERR_CUDA, "reading the network");
    const double h2 = 1.0 / ((double)c->geo.n * c->geo.n);
    const double margin = 0.02 * ((double)hi - (double)lo);
    const bool in_range = c->vmin * h2 >= (double)lo - margin && c->vmax * h2 <= (double)hi + margin;
    if (in_range && o.learned_gate > 0.0) {
      gated = true;  // the eigen path runs below without its rows, then the network and the gate
    } else if (in_range) {
      const int64_t N = c->geo.N;
      const int mu = c->geo.mu;
      if (!ensure(c, c->Q, sizeof(double) * mu * N) || !ensure(c, c->C, sizeof(double) * mu * N) ||
          !ensure(c, c->P, sizeof(double) * mu * N) ||
          !ensure(c, c->counts, sizeof(int32_t) * 64))
        return LSP_ERR_OOM;
      c->built = false;
      CUDA_OK(c, launch_zero(c, (int32_t*)c->counts.p + kErrWord, sizeof(int32_t)));
      CUDA_OK(c, launch_learned_rows(c, c->mlp));
      c->built = true;
      c->built_learned = true;
      c->built_gated = false;
      ++c->build_gen;
      c->mode_used = LSP_LEARNED;
      c->t_built = 1;
      c->leaf_built = 0;
      return LSP_OK;
    }
    o.mode = LSP_FP64;  // fallback (or the eigen path under the gate)
  }
  if (!(o.learned_gate >= 0.0)) return fail(c, LSP_ERR_ARG, "learned_gate must be >= 0");
  if (o.policy < 0 || o.policy > 3) return fail(c, LSP_ERR_ARG, "bad policy %d", o.policy);
  if (o.eig_method != LSP_EIG_SYMMETRIC && o.eig_method != LSP_EIG_FULL)
    return fail(c, LSP_ERR_ARG, "bad eig_method %d", o.eig_method);
  if (o.refine_steps < 0 || o.refine_steps > 4)
    return fail(c, LSP_ERR_ARG, "refine_steps must be in [0, 4]");
  const int d = c->geo.d, n = c->geo.n;
  const int64_t N = c->geo.N;
  const Geometry& G = o.t == 2 ? c->geo2 : c->geo;
  const int mu = G.mu;
  const bool need_t1 = o.t == 1 || o.nd_leaf > 0;  // some point uses the 3 x 3 stencil
  c->built = false;

  // ---- a2: the shift set ----
  std::vector<int64_t> ms;
  int64_t cap_s = 0;
  if (o.policy == LSP_SHIFT_LOCAL) {
    c->mrange.lo = snap_host(c->vmin);
    c->mrange.hi = snap_host(c->vmax);
    cap_s = c->mrange.size();
  } else {
    if (o.policy == LSP_SHIFT_PAPER) {
      // |S| of the Sec. 5 tables: n/16 in 2D, n/4 in 3D; 1D (no experiment) as 3D
      int K = o.nshifts > 0 ? o.nshifts : std::max(2, d == 2 ? n / 16 : n / 4);
      if (K == 1) {
        ms.push_back(snap_host(c->vmin));
      } else {
        volatile double step = (c->vmax - c->vmin) / (double)(K - 1);
        for (int i = 0; i < K - 1; ++i) {
          volatile double prod = (double)i * step;
          volatile double x = c->vmin + prod;
          ms.push_back(snap_host(x));
        }
        ms.push_back(snap_host(c->vmax));
      }
    } else if (o.policy == LSP_SHIFT_MEAN) {
      ms.push_back(snap_host(c->vmean));
    } else {
      if (!o.shifts || o.nshifts < 1) return fail(c, LSP_ERR_ARG, "LIST policy needs shifts");
      for (int i = 0; i < o.nshifts; ++i) {
        const double s = o.shifts[i];
        if (!isfinite(s)) return fail(c, LSP_ERR_ARG, "shift %d is not finite", i);
        // resonance: s = -4 pi^2 |k|^2 for some k in K makes L + s singular (Sec. 3)
        const double r = -s / (4.0 * kPi2);
        const double rr = round(r);
        if (rr >= 0 && rr <= d * (double)(n / 2) * (n / 2) && fabs(r - rr) < 1e-12 * (1 + rr) &&
            is_norm((int64_t)rr, d, n / 2))
          return fail(c, LSP_ERR_RESONANT_SHIFT, "shift %.17g is an eigenvalue of -L", s);
        const int64_t m = snap_host(s);
        if (shift_host(m) != s)
          return fail(c, LSP_ERR_ARG, "shift %.17g is not on the lattice (4m+2) pi^2", s);
        ms.push_back(m);
      }
    }
    std::sort(ms.begin(), ms.end());
    ms.erase(std::unique(ms.begin(), ms.end()), ms.end());
    c->mrange.lo = ms.front();
    c->mrange.hi = ms.back();
    cap_s = (int64_t)ms.size();
  }
  const int64_t half2 = (int64_t)(n / 2) * (n / 2);
  c->erange[d] = c->mrange;
  for (int k = d - 1; k >= 0; --k) {
    c->erange[k].lo = c->erange[k + 1].lo;
    c->erange[k].hi = c->erange[k + 1].hi + half2;
  }
  if (c->erange[0].hi > 2147483000LL || c->erange[0].lo < -2147483000LL)
    return fail(c, LSP_ERR_ARG, "shift range too large for 32-bit lattice indices");
  // A stage domain E_k = {l + p^2} is evaluated over its whole range when the list it is built
  // from could cover it (upper bound of its size times n/2+1 offsets >= twice the range):
  // marking and compacting would then cost more than the few extra points.
  {
    int64_t ub = cap_s;
    for (int k = d - 1; k >= 1; --k) {
      const int64_t sz = c->erange[k].size();
      c->edense[k] = (k < d - 1 && c->edense[k + 1]) || ub * (int64_t)c->geo.P >= 2 * sz;
      ub = c->edense[k] ? sz : std::min<int64_t>(sz, ub * (int64_t)c->geo.P);
    }
  }

  // ---- buffers (all allocation happens before any capture) ----
  const int64_t R = c->mrange.size();
  bool ok = ensure(c, c->shift_m, sizeof(int32_t) * cap_s) &&
            ensure(c, c->counts, sizeof(int32_t) * (16 + 2 + c->erange[0].size() / 4096 + 16)) &&
            ensure(c, c->gvals, sizeof(double) * 2 * G.ncls * cap_s) &&
            (!need_t1 || (ensure(c, c->alpha, sizeof(double) * c->geo.mu * cap_s) &&
                          ensure(c, c->cst, sizeof(double) * c->geo.mu * cap_s) &&
                          ensure(c, c->ap, sizeof(double) * c->geo.mu * cap_s) &&
                          ensure(c, c->lam, sizeof(double) * 2 * cap_s) &&
                          ensure(c, c->sflags, sizeof(int32_t) * cap_s))) &&
            (o.t != 2 || (ensure(c, c->alpha2, sizeof(double) * mu * cap_s) &&
                          ensure(c, c->cst2, sizeof(double) * mu * cap_s) &&
                          ensure(c, c->lam2, sizeof(double) * 2 * cap_s) &&
                          ensure(c, c->sflags2, sizeof(int32_t) * cap_s))) &&
            ensure_tracked(c, c->wtab, sizeof(double) * 2 * c->erange[0].size(), &c->wtab_size) &&
            ensure(c, c->Q, sizeof(double) * mu * N) && ensure(c, c->C, sizeof(double) * mu * N) &&
            ensure(c, c->P, sizeof(double) * mu * N);
  if (ok && o.policy == LSP_SHIFT_LOCAL)
    ok = ensure(c, c->shift_flag, round_up(R, 4096)) && ensure(c, c->idx_of, sizeof(int32_t) * R);
  for (int k = 1; ok && k < d; ++k) {
    const int64_t sz = c->erange[k].size();
    ok = ensure(c, c->eflag[k], round_up(sz, 4096)) && ensure(c, c->elist[k], sizeof(int32_t) * sz) &&
         ensure(c, c->T[k], sizeof(double) * 2 * ncls_stage(k, o.t) * sz);
  }
  if (!ok) return LSP_ERR_OOM;
  if (o.policy != LSP_SHIFT_LOCAL) {
    if (c->h_list_cap < cap_s + 1) {
      if (c->h_list) cudaFreeHost(c->h_list);
      c->h_list = nullptr;
      c->h_list_cap = 0;
      if (cudaMallocHost(&c->h_list, sizeof(int32_t) * (cap_s + 1)) != cudaSuccess)
        return fail(c, LSP_ERR_OOM, "pinned allocation failed");
      c->h_list_cap = cap_s + 1;
    }
    CUDA_OK(c, cudaStreamSynchronize(c->stream));  // the staging buffer may still be in use
    for (int64_t i = 0; i < cap_s; ++i) c->h_list[i] = (int32_t)ms[i];
    c->h_list[cap_s] = (int32_t)cap_s;
    CUDA_OK(c, cudaMemcpyAsync(c->shift_m.p, c->h_list, sizeof(int32_t) * cap_s,
                               cudaMemcpyHostToDevice, c->stream));
    CUDA_OK(c, cudaMemcpyAsync(c->counts.p, c->h_list + cap_s, sizeof(int32_t),
                               cudaMemcpyHostToDevice, c->stream));
  }
  c->ns_host = o.policy == LSP_SHIFT_LOCAL ? -1 : cap_s;
  c->last_policy = o.policy;

  // w depends only on its index range and precision: refreshed (outside any graph) only when
  // those change, so a replayed graph always finds the table it was recorded with.
  {
    const int prec = stage_prec(c, o);
    if (!(c->wtab_lo == c->erange[0].lo && c->wtab_size == c->erange[0].size() &&
          c->wtab_prec == prec)) {
      CUDA_OK(c, launch_wtable(c, c->erange[0].lo, c->erange[0].size(), c->wtab.p, prec));
      c->wtab_lo = c->erange[0].lo;
      c->wtab_size = c->erange[0].size();
      c->wtab_prec = prec;
    }
  }
  lsp_status st;
  if (c->autotune && !c->timing) {
    // the first build of a configuration times the candidate launch shapes eagerly (outside
    // any capture); the build it runs is a complete one, and later builds use the winners
    std::vector<int64_t> cfg = {o.policy, o.mode, o.eig_method, o.refine_steps, o.t, o.nd_leaf,
                                (int64_t)gated, (int64_t)std::stoi(work_bucket(cap_s))};
    if (std::find(c->tuned_configs.begin(), c->tuned_configs.end(), cfg) ==
        c->tuned_configs.end()) {
      c->tuning = true;
      st = issue_build(c, o, cap_s, false, !gated);
      c->tuning = false;
      if (st != LSP_OK) return st;
      CUDA_OK(c, cudaStreamSynchronize(c->stream));
      c->tuned_configs.push_back(cfg);
      ++c->tune_gen;
    }
  }
  const bool capturable = c->stream != nullptr && c->stream != cudaStreamLegacy &&
                          c->stream != cudaStreamPerThread;
  if (o.use_graph && !c->timing && capturable) {
    std::vector<int64_t> key = {o.policy, o.mode, o.eig_method, o.refine_steps, o.t, o.nd_leaf,
                                (int64_t)gated, cap_s, c->mrange.lo,
                                c->mrange.hi, (int64_t)(intptr_t)c->v.p,
                                (int64_t)(intptr_t)c->Q.p};
    for (int k = 0; k <= d; ++k) key.push_back(c->erange[k].lo);
    for (int k = 0; k < kMaxD; ++k) key.push_back(c->edense[k]);
    key.push_back(c->alloc_gen);  // any reallocation invalidates recorded pointers
    key.push_back(c->tune_gen);   // so does a tuning pass (new launch shapes)
    if (!c->graph || key != c->graph_key) {
      if (c->graph) cudaGraphExecDestroy(c->graph);
      c->graph = nullptr;
      cudaGraph_t g;
      CUDA_OK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      st = issue_build(c, o, cap_s, false, !gated);
      cudaError_t ce = cudaStreamEndCapture(c->stream, &g);
      if (st != LSP_OK) return st;
      CUDA_OK(c, ce);
      ce = cudaGraphInstantiate(&c->graph, g, 0);
      cudaGraphDestroy(g);
      CUDA_OK(c, ce);
      c->graph_key = key;
    }
    CUDA_OK(c, cudaGraphLaunch(c->graph, c->stream));
    st = LSP_OK;
  } else {
    st = issue_build(c, o, cap_s, false, !gated);
  }
  if (st == LSP_OK && gated) {
    // the network's rows, then the per-point residual gate against the eigen path's tables
    if (!ensure(c, c->gate_rho, sizeof(float) * N)) return LSP_ERR_OOM;
    int32_t* counts = (int32_t*)c->counts.p;
    CUDA_OK(c, launch_learned_rows(c, c->mlp));
    CUDA_OK(c, launch_zero(c, counts + kGateWord, sizeof(int32_t)));
    CUDA_OK(c, launch_learned_gate(c, o.policy, counts + 0, cap_s, o.learned_gate,
                                   (float*)c->gate_rho.p, counts + kGateWord));
  }
  if (st == LSP_OK) {
    c->built = true;
    ++c->build_gen;
    c->built_learned = false;
    c->built_gated = gated;
    c->mode_used = gated ? LSP_LEARNED
                         : (o.mode == LSP_DWORD && stage_prec(c, o) != kPrecDword ? LSP_FP64
                                                                                 : o.mode);
    c->t_built = o.t;
    c->leaf_built = o.t == 2 ? o.nd_leaf : 0;
  }
  return st;
}

lsp_status lsp_apply_operator(lsp_ctx* c, const double* u, double* y) {
  if (!c) return LSP_ERR_ARG;
  cudaGetLastError();
  if (!u || !y) return fail(c, LSP_ERR_ARG, "u or y is NULL");
  if (!c->have_v) return fail(c, LSP_ERR_STATE, "apply_operator before set_potential");
  if (!ensure(c, c->fftbuf, sizeof(double) * 2 * c->geo.N)) return LSP_ERR_OOM;
  CUDA_OK(c, launch_apply(c, u, y));
  return LSP_OK;
}

// Row width of the last build: (2t+1)^d.
static int built_mu(const lsp_ctx* c) { return c->t_built == 2 ? c->geo2.mu : c->geo.mu; }

// t_j of a t = 2 build at point j (2D): 2 everywhere without a leaf, else the largest t <= 2
// whose neighbourhood crosses no separator line x_a = 0 (mod leaf) (Sec. 4.2).
static int t_of_point(int64_t j, int n, int leaf, int d = 2) {
  if (leaf <= 0) return 2;
  int t = 2;
  int64_t x[3];
  for (int a = d - 1; a >= 0; --a) {
    x[a] = j % n;
    j /= n;
  }
  for (int a = 0; a < d; ++a) {
    const int r = (int)(x[a] % leaf);
    const int f = r == 0 ? leaf : std::min(r, leaf - r);
    t = std::min(t, f);
  }
  return t;
}

static lsp_status rows_of(lsp_ctx* c, char which, const double** out) {
  if (!c->built) return fail(c, LSP_ERR_STATE, "no stencils built");
  switch (which) {
    case 'Q': *out = (const double*)c->Q.p; return LSP_OK;
    case 'C': *out = (const double*)c->C.p; return LSP_OK;
    case 'P': *out = (const double*)c->P.p; return LSP_OK;
    default: return fail(c, LSP_ERR_ARG, "which must be 'Q', 'C' or 'P'");
  }
}

lsp_status lsp_get_rows(lsp_ctx* c, char which, double* rows, int on_device) {
  if (!c) return LSP_ERR_ARG;
  if (!rows) return fail(c, LSP_ERR_ARG, "rows is NULL");
  const double* src;
  lsp_status st = rows_of(c, which, &src);
  if (st != LSP_OK) return st;
  const size_t bytes = sizeof(double) * built_mu(c) * c->geo.N;
  CUDA_OK(c, cudaMemcpyAsync(rows, src, bytes,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             c->stream));
  if (!on_device) CUDA_OK(c, cudaStreamSynchronize(c->stream));
  return LSP_OK;
}

lsp_status lsp_get_rows_async(lsp_ctx* c, char which, double* rows) {
  if (!c) return LSP_ERR_ARG;
  if (!rows) return fail(c, LSP_ERR_ARG, "rows is NULL");
  const double* src;
  lsp_status st = rows_of(c, which, &src);
  if (st != LSP_OK) return st;
  const int w = which == 'Q' ? 0 : which == 'C' ? 1 : 2;
  const size_t bytes = sizeof(double) * built_mu(c) * c->geo.N;
  if (!c->copy_stream) {
    CUDA_OK(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    for (int k = 0; k < 3; ++k) {
      CUDA_OK(c, cudaEventCreateWithFlags(&c->ev_staged[k], cudaEventDisableTiming));
      CUDA_OK(c, cudaEventCreateWithFlags(&c->ev_copied[k], cudaEventDisableTiming));
    }
  }
  if (c->stage[w].bytes < bytes) {
    CUDA_OK(c, cudaStreamSynchronize(c->copy_stream));  // the old staging copy may be in use
    if (!ensure(c, c->stage[w], bytes)) return LSP_ERR_OOM;
  }
  // the staging copy of this block is free again once its previous host copy has landed
  CUDA_OK(c, cudaStreamWaitEvent(c->stream, c->ev_copied[w], 0));
  // the staging copy by a kernel: a device-to-device memcpy could queue on the copy engine
  // behind the host copy of the previous block
  CUDA_OK(c, launch_copy_f64(c, src, (double*)c->stage[w].p, (int64_t)(bytes / sizeof(double))));
  CUDA_OK(c, cudaEventRecord(c->ev_staged[w], c->stream));
  CUDA_OK(c, cudaStreamWaitEvent(c->copy_stream, c->ev_staged[w], 0));
  CUDA_OK(c, cudaMemcpyAsync(rows, c->stage[w].p, bytes, cudaMemcpyDeviceToHost,
                             c->copy_stream));
  CUDA_OK(c, cudaEventRecord(c->ev_copied[w], c->copy_stream));
  return LSP_OK;
}

lsp_status lsp_wait_rows(lsp_ctx* c) {
  if (!c) return LSP_ERR_ARG;
  if (c->copy_stream) CUDA_OK(c, cudaStreamSynchronize(c->copy_stream));
  return LSP_OK;
}

lsp_status lsp_export_sparse_rows(lsp_ctx* c, char which, int64_t* rowptr, int32_t* colidx,
                                  double* vals, int64_t* nnz_out) {
  if (!c) return LSP_ERR_ARG;
  cudaGetLastError();
  const int64_t N = c->geo.N;
  if (c->built && c->t_built == 2) {
    // rows of (2 t_j + 1)^d entries: the structural zeros of t_j = 1 rows are left out
    std::vector<int64_t> ptr(N + 1);
    ptr[0] = 0;
    const int d = c->geo.d;
    for (int64_t j = 0; j < N; ++j) {
      const int w = 2 * t_of_point(j, c->geo.n, c->leaf_built, d) + 1;
      ptr[j + 1] = ptr[j] + (d == 2 ? w * w : w * w * w);
    }
    const int64_t nnz = ptr[N];
    if (nnz_out) *nnz_out = nnz;
    if (!rowptr && !colidx && !vals) return LSP_OK;
    if (!rowptr || !colidx || !vals)
      return fail(c, LSP_ERR_ARG, "rowptr, colidx and vals must all be given");
    const double* src;
    lsp_status st = rows_of(c, which, &src);
    if (st != LSP_OK) return st;
    if (!ensure(c, c->colidx, sizeof(int32_t) * nnz) ||
        !ensure(c, c->rowptr, sizeof(int64_t) * (N + 1)) ||
        !ensure(c, c->expvals, sizeof(double) * nnz))
      return LSP_ERR_OOM;
    CUDA_OK(c, cudaMemcpyAsync(c->rowptr.p, ptr.data(), sizeof(int64_t) * (N + 1),
                               cudaMemcpyHostToDevice, c->stream));
    CUDA_OK(c, launch_export_t2(c, src, c->leaf_built, (const int64_t*)c->rowptr.p,
                                (int32_t*)c->colidx.p, (double*)c->expvals.p));
    CUDA_OK(c, cudaMemcpyAsync(colidx, c->colidx.p, sizeof(int32_t) * nnz,
                               cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(c, cudaMemcpyAsync(vals, c->expvals.p, sizeof(double) * nnz, cudaMemcpyDeviceToHost,
                               c->stream));
    CUDA_OK(c, cudaStreamSynchronize(c->stream));
    memcpy(rowptr, ptr.data(), sizeof(int64_t) * (N + 1));
    return LSP_OK;
  }
  const int64_t nnz = c->geo.N * c->geo.mu;
  if (nnz_out) *nnz_out = nnz;
  if (!rowptr && !colidx && !vals) return LSP_OK;
  if (!rowptr || !colidx || !vals)
    return fail(c, LSP_ERR_ARG, "rowptr, colidx and vals must all be given");
  const double* src;
  lsp_status st = rows_of(c, which, &src);
  if (st != LSP_OK) return st;
  if (!ensure(c, c->colidx, sizeof(int32_t) * nnz) ||
      !ensure(c, c->rowptr, sizeof(int64_t) * (c->geo.N + 1)))
    return LSP_ERR_OOM;
  CUDA_OK(c, launch_colidx(c));
  CUDA_OK(c, cudaMemcpyAsync(colidx, c->colidx.p, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost,
                             c->stream));
  CUDA_OK(c, cudaMemcpyAsync(rowptr, c->rowptr.p, sizeof(int64_t) * (c->geo.N + 1),
                             cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaMemcpyAsync(vals, src, sizeof(double) * nnz, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  return LSP_OK;
}

lsp_status lsp_get_shift_table(lsp_ctx* c, int64_t* nshifts_out, double* s, double* alpha,
                               double* cst, double* lam, int32_t* flags, int32_t* s_idx) {
  if (!c) return LSP_ERR_ARG;
  if (!c->built) return fail(c, LSP_ERR_STATE, "no stencils built");
  if (c->built_learned)
    return fail(c, LSP_ERR_STATE, "a learned build has no shift table (rows only)");
  cudaGetLastError();
  int32_t head[16];
  CUDA_OK(c, cudaMemcpyAsync(head, c->counts.p, sizeof(head), cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  const int32_t ns = head[0];
  if (head[kErrWord] != 0)
    return fail(c, LSP_ERR_STATE, "device lattice snap disagreed with the host (bits %d)",
                head[kErrWord]);
  if (nshifts_out) *nshifts_out = ns;
  const bool t2 = c->t_built == 2;  // the t = 2 stencils of a t = 2 build
  const int mu = built_mu(c);
  if (s) {
    std::vector<int32_t> m(ns);
    CUDA_OK(c, cudaMemcpy(m.data(), c->shift_m.p, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost));
    for (int i = 0; i < ns; ++i) s[i] = shift_host(m[i]);
  }
  if (alpha)
    CUDA_OK(c, cudaMemcpy(alpha, (t2 ? c->alpha2 : c->alpha).p, sizeof(double) * mu * ns,
                          cudaMemcpyDeviceToHost));
  if (cst)
    CUDA_OK(c, cudaMemcpy(cst, (t2 ? c->cst2 : c->cst).p, sizeof(double) * mu * ns,
                          cudaMemcpyDeviceToHost));
  if (lam)
    CUDA_OK(c, cudaMemcpy(lam, (t2 ? c->lam2 : c->lam).p, sizeof(double) * 2 * ns,
                          cudaMemcpyDeviceToHost));
  if (flags)
    CUDA_OK(c, cudaMemcpy(flags, (t2 ? c->sflags2 : c->sflags).p, sizeof(int32_t) * ns,
                          cudaMemcpyDeviceToHost));
  if (s_idx) {
    if (!ensure(c, c->sidx, sizeof(int32_t) * c->geo.N)) return LSP_ERR_OOM;
    CUDA_OK(c, launch_sidx(c, c->last_policy, (const int32_t*)c->counts.p));
    CUDA_OK(c, cudaMemcpyAsync(s_idx, c->sidx.p, sizeof(int32_t) * c->geo.N,
                               cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(c, cudaStreamSynchronize(c->stream));
  }
  return LSP_OK;
}

lsp_status lsp_get_sizes(const lsp_ctx* c, int64_t* npoints, int* mu) {
  if (!c) return LSP_ERR_ARG;
  if (npoints) *npoints = c->geo.N;
  if (mu) *mu = built_mu(c);
  return LSP_OK;
}

lsp_status lsp_synchronize(lsp_ctx* c) {
  if (!c) return LSP_ERR_ARG;
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  CUDA_OK(c, cudaGetLastError());
  if (c->built && c->counts.p) {
    int32_t e = 0;
    CUDA_OK(c, cudaMemcpy(&e, (int32_t*)c->counts.p + kErrWord, sizeof e, cudaMemcpyDeviceToHost));
    if (e & kErrBounds)
      return fail(c, LSP_ERR_STATE, "an index left its array (checked build, bits %d)", e);
    if (e && (c->built_learned || c->built_gated))
      return fail(c, LSP_ERR_TIMEOUT, "a tensor-core wait gave up (bits %d)", e);
    if (e) return fail(c, LSP_ERR_STATE, "device lattice snap disagreed with the host (bits %d)", e);
  }
  return LSP_OK;
}

lsp_status lsp_set_mlp(lsp_ctx* c, lsp_mlp* m) {
  if (!c) return LSP_ERR_ARG;
  if (m && mlp_dim(m) != c->geo.d) return fail(c, LSP_ERR_ARG, "network dimension mismatch");
  if (m) CUDA_OK(c, mlp_sync(m));
  c->mlp = m;
  return LSP_OK;
}

lsp_status lsp_set_autotune(lsp_ctx* c, int on) {
  if (!c) return LSP_ERR_ARG;
  c->autotune = on != 0;
  return LSP_OK;
}

lsp_status lsp_get_tuning(const lsp_ctx* c, char* buf, int64_t len) {
  if (!c || !buf || len < 1) return LSP_ERR_ARG;
  std::string out;
  for (const auto& kv : c->tune) {
    char line[256];
    snprintf(line, sizeof line, "%s %d %d %.5f %.5f %d\n", kv.first.c_str(), kv.second.best.threads,
             kv.second.best.per_sm, kv.second.ms_default, kv.second.ms_best,
             kv.second.candidates);
    out += line;
  }
  if ((int64_t)out.size() + 1 > len) return LSP_ERR_ARG;
  memcpy(buf, out.c_str(), out.size() + 1);
  return LSP_OK;
}

lsp_status lsp_get_gate_stats(lsp_ctx* c, int64_t* fallback_points, float* rho_host) {
  if (!c) return LSP_ERR_ARG;
  if (!c->built || !c->built_gated)
    return fail(c, LSP_ERR_STATE, "the last build was not a gated learned build");
  cudaGetLastError();
  int32_t head[16];
  CUDA_OK(c, cudaMemcpyAsync(head, c->counts.p, sizeof(head), cudaMemcpyDeviceToHost, c->stream));
  if (rho_host)
    CUDA_OK(c, cudaMemcpyAsync(rho_host, c->gate_rho.p, sizeof(float) * c->geo.N,
                               cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  if (head[kErrWord] != 0)
    return fail(c, LSP_ERR_TIMEOUT, "a device wait gave up or a snap disagreed (bits %d)",
                head[kErrWord]);
  if (fallback_points) *fallback_points = head[kGateWord];
  return LSP_OK;
}

lsp_status lsp_get_mode_used(const lsp_ctx* c, int* mode) {
  if (!c || !mode) return LSP_ERR_ARG;
  *mode = c->mode_used;
  return LSP_OK;
}

lsp_status lsp_kernel_timing(lsp_ctx* c, int enable) {
  if (!c) return LSP_ERR_ARG;
  lsp_status st = flush_timers(c);
  if (st != LSP_OK) return st;
  if (enable) c->timers.clear();
  c->timing = enable != 0;
  return LSP_OK;
}

lsp_status lsp_kernel_times(lsp_ctx* c, int cap, char (*names)[32], double* ms, int64_t* launches,
                            int* count) {
  if (!c) return LSP_ERR_ARG;
  lsp_status st = flush_timers(c);
  if (st != LSP_OK) return st;
  if (count) *count = (int)c->timers.size();
  for (int i = 0; i < cap && i < (int)c->timers.size(); ++i) {
    if (names) {
      strncpy(names[i], c->timers[i].name.c_str(), 31);
      names[i][31] = 0;
    }
    if (ms) ms[i] = c->timers[i].ms;
    if (launches) launches[i] = c->timers[i].launches;
  }
  return LSP_OK;
}

const char* lsp_last_error(const lsp_ctx* c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
