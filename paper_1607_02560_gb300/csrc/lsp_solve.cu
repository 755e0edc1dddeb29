// Host side of the solve calls of include/lsp.h: the nested-dissection factorisation of P and
// its solve (Sec. 3, Eq. QC; Fig. nd; Table cost), the row matrix-vector product, and the
// restarted GMRES solve of (L + diag v) u = f left-preconditioned by P^-1 C (Eq. PC; Sec. 5).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <string>

#include "nd.h"

using namespace lsp;

namespace {

lsp_status sfail(lsp_ctx* c, lsp_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return st;
}

#define SCUDA(ctx, expr)                                                                  \
  do {                                                                                    \
    cudaError_t _e = (expr);                                                              \
    if (_e != cudaSuccess)                                                                \
      return sfail(ctx, _e == cudaErrorMemoryAllocation ? LSP_ERR_OOM : LSP_ERR_CUDA,     \
                   "%s failed: %s", #expr, cudaGetErrorString(_e));                       \
  } while (0)

int rows_mu(const lsp_ctx* c) { return c->t_built == 2 ? c->geo2.mu : c->geo.mu; }

const double* rows_ptr(const lsp_ctx* c, char which) {
  switch (which) {
    case 'Q': return (const double*)c->Q.p;
    case 'C': return (const double*)c->C.p;
    case 'P': return (const double*)c->P.p;
    default: return nullptr;
  }
}

template <class T>
lsp_status upload(lsp_ctx* c, DevBuf& b, const std::vector<T>& v) {
  if (!ensure(c, b, sizeof(T) * (v.empty() ? 1 : v.size()))) return LSP_ERR_OOM;
  if (!v.empty())
    SCUDA(c, cudaMemcpyAsync(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice,
                             c->stream));
  return LSP_OK;
}

bool nd_ready(const lsp_ctx* c) {
  return c->nd && c->nd->factored && c->nd->factored_gen == c->build_gen && c->built;
}

// x = P^-1 y with the chosen refinement steps x += P^-1 (y - P x); x may equal y.
lsp_status nd_apply(lsp_ctx* c, const double* y, double* x) {
  NdState& S = *c->nd;
  if (S.refine_steps == 0) {
    SCUDA(c, launch_nd_solve(c, y, x));
    return LSP_OK;
  }
  const int64_t N = c->geo.N;
  if (!ensure(c, S.ry, sizeof(double) * N) || !ensure(c, S.rd, sizeof(double) * N))
    return sfail(c, LSP_ERR_OOM, "refinement scratch: %s", c->err.c_str());
  double* ry = (double*)S.ry.p;
  double* rd = (double*)S.rd.p;
  SCUDA(c, cudaMemcpyAsync(ry, y, sizeof(double) * N, cudaMemcpyDeviceToDevice, c->stream));
  SCUDA(c, launch_nd_solve(c, ry, x));
  for (int k = 0; k < S.refine_steps; ++k) {
    SCUDA(c, launch_apply_rows(c, (const double*)c->P.p, rows_mu(c), c->t_built, x, rd));
    SCUDA(c, launch_axpby(c, rd, ry, rd, nullptr, -1.0, N));
    SCUDA(c, launch_nd_solve(c, rd, rd));
    SCUDA(c, launch_axpby(c, x, x, rd, nullptr, 1.0, N));
  }
  return LSP_OK;
}

}  // namespace

namespace lsp {

void nd_free(NdState* s) {
  if (!s) return;
  DevBuf* bufs[] = {&s->fronts, &s->E, &s->R, &s->inv, &s->asm_dst, &s->asm_src, &s->perm,
                    &s->z, &s->u, &s->cbuf, &s->pinv, &s->swaps, &s->err, &s->V, &s->w,
                    &s->b, &s->x, &s->tmp, &s->gs, &s->fvec, &s->ry, &s->rd, &s->pscratch};
  for (DevBuf* b : bufs)
    if (b->p) cudaFree(b->p);
  if (s->h_gs) cudaFreeHost(s->h_gs);
  if (s->ev_cols) cudaEventDestroy(s->ev_cols);
  if (s->ev_panel) cudaEventDestroy(s->ev_panel);
  if (s->side) cudaStreamDestroy(s->side);
  delete s;
}

cudaError_t nd_prepare_kernels(int max_smem);

}  // namespace lsp

extern "C" {

void lsp_default_nd_opts(lsp_nd_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
}

void lsp_default_gmres_opts(lsp_gmres_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->rtol = 1e-6;
  o->restart = 40;
  o->max_cycles = 50;
  o->precond = 1;
}

lsp_status lsp_nd_factor(lsp_ctx* c, const lsp_nd_opts* opts) {
  if (!c) return LSP_ERR_ARG;
  cudaGetLastError();
  if (!c->built) return sfail(c, LSP_ERR_STATE, "nd_factor before build_stencils");
  if (c->geo.d == 1)
    return sfail(c, LSP_ERR_UNSUPPORTED, "the nested dissection is built for 2D and 3D grids");
  int leaf = opts && opts->leaf ? opts->leaf : (c->t_built == 2 ? c->leaf_built : 8);
  if (leaf <= 0) leaf = 8;
  if (leaf < 4 || (leaf & (leaf - 1)) || leaf > c->geo.n)
    return sfail(c, LSP_ERR_ARG, "leaf width %d: must be a power of two in [4, n]", leaf);
  const int refine = opts ? opts->refine_steps : 0;
  if (refine < 0 || refine > 4) return sfail(c, LSP_ERR_ARG, "refine_steps must be in [0, 4]");
  if (c->t_built == 2 && c->leaf_built > 0 && leaf != c->leaf_built)
    return sfail(c, LSP_ERR_ARG, "leaf width %d differs from the nd_leaf %d of the build", leaf,
                 c->leaf_built);
  if (!c->nd) c->nd = new NdState();
  NdState& S = *c->nd;
  const int mu = rows_mu(c);
  const NdPlan& P0 = S.plan;
  if (!S.have_plan || P0.d != c->geo.d || P0.n != c->geo.n || P0.leaf != leaf ||
      P0.t_built != c->t_built ||
      P0.leaf_t != (c->t_built == 2 ? c->leaf_built : 0) || P0.mu != mu) {
    S.have_plan = false;
    S.factored = false;
    const std::string why =
        build_nd_plan(S.plan, c->geo.d, c->geo.n, leaf, c->t_built,
                      c->t_built == 2 ? c->leaf_built : 0, mu);
    if (!why.empty()) return sfail(c, LSP_ERR_UNSUPPORTED, "nested dissection: %s", why.c_str());
    lsp_status st;
    if ((st = upload(c, S.E, S.plan.E)) != LSP_OK) return st;
    if ((st = upload(c, S.R, S.plan.R)) != LSP_OK) return st;
    if ((st = upload(c, S.inv, S.plan.inv)) != LSP_OK) return st;
    if ((st = upload(c, S.asm_dst, S.plan.asm_dst)) != LSP_OK) return st;
    if ((st = upload(c, S.asm_src, S.plan.asm_src)) != LSP_OK) return st;
    const NdPlan& P = S.plan;
    int64_t cb = 1, pv = 1, sw = 1, ps = 0;
    int max_sr = 1;
    for (const NdLevel& lv : P.lv) {
      if (lv.f > kNdSmallFront) {
        cb = std::max(cb, (int64_t)lv.count * lv.f * kNdPanel);
        pv = std::max(pv, (int64_t)lv.count * kNdPanel * kNdPanel);
        sw = std::max(sw, (int64_t)lv.count * (1 + 4 * kNdPanel));
        if (lv.s > kNdPanelRegRows) ps = std::max(ps, (int64_t)lv.count * lv.s * (kNdPanel + 1));
      }
      max_sr = std::max(max_sr, std::max(lv.s, lv.r));
    }
    if (ps > 0 && !ensure(c, S.pscratch, sizeof(float) * ps))
      return sfail(c, LSP_ERR_OOM, "nested dissection buffers: %s", c->err.c_str());
    if (!ensure(c, S.fronts, sizeof(double) * P.front_doubles) ||
        !ensure(c, S.perm, sizeof(int32_t) * P.perm_ints) ||
        !ensure(c, S.z, sizeof(double) * P.z_doubles) ||
        !ensure(c, S.u, sizeof(double) * (P.u_doubles > 0 ? P.u_doubles : 1)) ||
        !ensure(c, S.cbuf, sizeof(double) * 2 * cb) ||
        !ensure(c, S.pinv, sizeof(double) * 2 * pv) ||
        !ensure(c, S.swaps, sizeof(int32_t) * 2 * sw) || !ensure(c, S.err, sizeof(int32_t)))
      return sfail(c, LSP_ERR_OOM, "nested dissection buffers: %s", c->err.c_str());
    S.cbuf_half = cb;
    S.pinv_half = pv;
    S.swaps_half = sw;
    SCUDA(c, cudaMemsetAsync(S.swaps.p, 0, sizeof(int32_t) * 2 * sw, c->stream));
    if (!S.side) {
      int least = 0, greatest = 0;
      SCUDA(c, cudaDeviceGetStreamPriorityRange(&least, &greatest));
      SCUDA(c, cudaStreamCreateWithPriority(&S.side, cudaStreamNonBlocking, greatest));
      SCUDA(c, cudaEventCreateWithFlags(&S.ev_cols, cudaEventDisableTiming));
      SCUDA(c, cudaEventCreateWithFlags(&S.ev_panel, cudaEventDisableTiming));
    }
    SCUDA(c, nd_prepare_kernels((int)std::min<int64_t>(sizeof(double) * max_sr + 64, 220 * 1024)));
    S.have_plan = true;
  }
  S.factored = false;
  const NdPlan& P = S.plan;
  SCUDA(c, cudaMemsetAsync(S.err.p, 0, sizeof(int32_t), c->stream));
  const double* rows = (const double*)c->P.p;
  for (int d = (int)P.lv.size() - 1; d >= 0; --d) {
    SCUDA(c, launch_nd_assemble(c, d, rows));
    SCUDA(c, launch_nd_sweep(c, d));
  }
  int32_t herr = 0;
  SCUDA(c, cudaMemcpyAsync(&herr, S.err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  SCUDA(c, cudaStreamSynchronize(c->stream));
  if (herr)
    return sfail(c, LSP_ERR_DEGENERATE,
                 "a pivot of the nested dissection vanished (code %d): P is singular", herr);
  S.factored = true;
  S.factored_gen = c->build_gen;
  S.refine_steps = refine;
  return LSP_OK;
}

static void fill_info(const NdPlan& P, lsp_nd_info* info) {
  memset(info, 0, sizeof *info);
  info->levels = (int)P.lv.size();
  info->leaf = P.leaf;
  int64_t fronts = 0;
  for (const NdLevel& lv : P.lv) fronts += lv.count;
  info->fronts = fronts;
  info->max_front = P.max_f;
  info->front_bytes = P.front_doubles * (int64_t)sizeof(double);
  info->solve_bytes = P.solve_bytes;
  info->flops = P.flops_sweep;
  info->flops_lu = P.flops_lu;
}

lsp_status lsp_nd_plan_info(int d, int n, int leaf, int t, int nd_leaf, lsp_nd_info* info,
                            int cap, int* count, int* s, int* r, char* err, int errcap) {
  if (err && errcap > 0) err[0] = 0;
  if (!info || (t != 1 && t != 2) || (d != 2 && d != 3) || cap < 0) return LSP_ERR_ARG;
  NdPlan P;
  const int w = 2 * t + 1;
  const std::string why =
      build_nd_plan(P, d, n, leaf, t, t == 2 ? nd_leaf : 0, d == 2 ? w * w : w * w * w);
  if (!why.empty()) {
    if (err && errcap > 0) snprintf(err, (size_t)errcap, "%s", why.c_str());
    return LSP_ERR_UNSUPPORTED;
  }
  fill_info(P, info);
  for (int d = 0; d < (int)P.lv.size() && d < cap; ++d) {
    if (count) count[d] = P.lv[d].count;
    if (s) s[d] = P.lv[d].s;
    if (r) r[d] = P.lv[d].r;
  }
  return LSP_OK;
}

lsp_status lsp_nd_get_info(lsp_ctx* c, lsp_nd_info* info) {
  if (!c || !info) return LSP_ERR_ARG;
  if (!c->nd || !c->nd->have_plan) return sfail(c, LSP_ERR_STATE, "no nested dissection planned");
  fill_info(c->nd->plan, info);
  info->factored = nd_ready(c) ? 1 : 0;
  return LSP_OK;
}

lsp_status lsp_nd_solve(lsp_ctx* c, const double* y, double* x) {
  if (!c) return LSP_ERR_ARG;
  cudaGetLastError();
  if (!y || !x) return sfail(c, LSP_ERR_ARG, "y or x is NULL");
  if (!nd_ready(c))
    return sfail(c, LSP_ERR_STATE, "nd_solve needs lsp_nd_factor of the current stencils");
  return nd_apply(c, y, x);
}

lsp_status lsp_apply_rows(lsp_ctx* c, char which, const double* u, double* y) {
  if (!c) return LSP_ERR_ARG;
  cudaGetLastError();
  if (!u || !y) return sfail(c, LSP_ERR_ARG, "u or y is NULL");
  if (u == y) return sfail(c, LSP_ERR_ARG, "u and y must not alias");
  if (!c->built) return sfail(c, LSP_ERR_STATE, "no stencils built");
  const double* rows = rows_ptr(c, which);
  if (!rows) return sfail(c, LSP_ERR_ARG, "which must be 'Q', 'C' or 'P'");
  SCUDA(c, launch_apply_rows(c, rows, rows_mu(c), c->t_built, u, y));
  return LSP_OK;
}

lsp_status lsp_gmres(lsp_ctx* c, const lsp_gmres_opts* opts, const double* f, double* u,
                     int on_device, lsp_gmres_result* out) {
  if (!c) return LSP_ERR_ARG;
  cudaGetLastError();
  lsp_gmres_opts o;
  lsp_default_gmres_opts(&o);
  if (opts) o = *opts;
  if (!f || !u) return sfail(c, LSP_ERR_ARG, "f or u is NULL");
  if (!(o.rtol > 0.0) || o.restart < 1 || o.restart > 60 || o.max_cycles < 1)
    return sfail(c, LSP_ERR_ARG, "rtol > 0, 1 <= restart <= 60 and max_cycles >= 1 required");
  if (!c->have_v) return sfail(c, LSP_ERR_STATE, "gmres before set_potential");
  if (o.precond && !nd_ready(c))
    return sfail(c, LSP_ERR_STATE, "the preconditioner needs lsp_nd_factor of the current stencils");
  if (!c->nd) c->nd = new NdState();
  NdState& S = *c->nd;
  const int64_t N = c->geo.N;
  const int m = o.restart, ld = m + 1;
  const int64_t gs_n = kGsArrays + (int64_t)ld * m + 2 * m + ld + m;
  if (!ensure(c, S.V, sizeof(double) * N * ld) || !ensure(c, S.w, sizeof(double) * N) ||
      !ensure(c, S.b, sizeof(double) * N) || !ensure(c, S.x, sizeof(double) * N) ||
      !ensure(c, S.tmp, sizeof(double) * N) || !ensure(c, S.fvec, sizeof(double) * N) ||
      !ensure(c, S.gs, sizeof(double) * gs_n) ||
      !ensure(c, c->fftbuf, sizeof(double) * 2 * N))
    return sfail(c, LSP_ERR_OOM, "gmres workspace: %s", c->err.c_str());
  if (!S.h_gs && cudaMallocHost(&S.h_gs, sizeof(double) * kGsPartial) != cudaSuccess) {
    S.h_gs = nullptr;
    return sfail(c, LSP_ERR_OOM, "pinned allocation failed");
  }
  double* V = (double*)S.V.p;
  double* w = (double*)S.w.p;
  double* b = (double*)S.b.p;
  double* x = (double*)S.x.p;
  double* tmp = (double*)S.tmp.p;
  double* fv = (double*)S.fvec.p;
  double* gs = (double*)S.gs.p;
  double* H = gs + kGsArrays;
  const double* Crows = (const double*)c->C.p;
  const int mu = rows_mu(c);
  SCUDA(c, cudaMemsetAsync(gs, 0, sizeof(double) * gs_n, c->stream));
  SCUDA(c, cudaMemcpyAsync(fv, f, sizeof(double) * N,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           c->stream));
  auto readback = [&]() -> lsp_status {
    SCUDA(c, cudaMemcpyAsync(S.h_gs, gs, sizeof(double) * kGsPartial, cudaMemcpyDeviceToHost,
                             c->stream));
    SCUDA(c, cudaStreamSynchronize(c->stream));
    return LSP_OK;
  };
  // out = P^-1 C (L + diag v) in   (or (L + diag v) in without the preconditioner)
  auto op = [&](const double* in, double* outv) -> lsp_status {
    if (o.precond) {
      SCUDA(c, launch_apply(c, in, tmp));
      SCUDA(c, launch_apply_rows(c, Crows, mu, c->t_built, tmp, outv));
      lsp_status sa = nd_apply(c, outv, outv);
      if (sa != LSP_OK) return sa;
    } else {
      SCUDA(c, launch_apply(c, in, outv));
    }
    return LSP_OK;
  };
  lsp_status st;
  // b = P^-1 C f
  if (o.precond) {
    SCUDA(c, launch_apply_rows(c, Crows, mu, c->t_built, fv, b));
    if ((st = nd_apply(c, b, b)) != LSP_OK) return st;
  } else {
    SCUDA(c, cudaMemcpyAsync(b, fv, sizeof(double) * N, cudaMemcpyDeviceToDevice, c->stream));
  }
  SCUDA(c, launch_mgs(c, b, nullptr, nullptr, nullptr, gs + kGsNorm, N));
  if ((st = readback()) != LSP_OK) return st;
  const double bnorm = sqrt(S.h_gs[kGsNorm]);
  SCUDA(c, cudaMemsetAsync(x, 0, sizeof(double) * N, c->stream));
  int iters = 0;
  bool conv = bnorm == 0.0, brk = false;
  double rnorm = bnorm;
  const double atol = o.rtol * bnorm;
  const double* r = b;  // the residual of x = 0
  for (int cycle = 0; cycle < o.max_cycles && !conv; ++cycle) {
    // gs[kGsNorm] holds |r|^2
    SCUDA(c, launch_gmres_start(c, gs, ld, r, V, N));
    int col = 0;
    for (col = 0; col < m; ++col) {
      double* vc = V + (int64_t)col * N;
      double* hc = H + (int64_t)col * ld;
      if ((st = op(vc, w)) != LSP_OK) return st;
      SCUDA(c, launch_mgs(c, w, nullptr, nullptr, nullptr, gs + kGsH0, N));
      for (int k = 0; k <= col; ++k)
        SCUDA(c, launch_mgs(c, w, k ? V + (int64_t)(k - 1) * N : nullptr, k ? hc + k - 1 : nullptr,
                            V + (int64_t)k * N, hc + k, N));
      SCUDA(c, launch_mgs(c, w, vc, hc + col, nullptr, gs + kGsH1, N));
      SCUDA(c, launch_gmres_givens(c, gs, col, ld));
      SCUDA(c, launch_axpby(c, V + (int64_t)(col + 1) * N, nullptr, w, gs + kGsInvH1, 1.0, N));
      if ((st = readback()) != LSP_OK) return st;
      ++iters;
      brk = S.h_gs[kGsBreak] != 0.0;
      if (S.h_gs[kGsPresid] <= atol || brk) break;
    }
    if (col == m) col = m - 1;
    SCUDA(c, launch_gmres_update(c, gs, col, ld, V, x, N));
    // r = b - op(x)
    if ((st = op(x, w)) != LSP_OK) return st;
    SCUDA(c, launch_axpby(c, w, b, w, nullptr, -1.0, N));
    SCUDA(c, launch_mgs(c, w, nullptr, nullptr, nullptr, gs + kGsNorm, N));
    if ((st = readback()) != LSP_OK) return st;
    rnorm = sqrt(S.h_gs[kGsNorm]);
    r = w;
    if (rnorm <= atol) conv = true;
    if (brk) break;
  }
  // |f - (L + diag v) x| / |f|
  SCUDA(c, launch_apply(c, x, tmp));
  SCUDA(c, launch_axpby(c, tmp, fv, tmp, nullptr, -1.0, N));
  SCUDA(c, launch_mgs(c, tmp, nullptr, nullptr, nullptr, gs + kGsH0, N));
  SCUDA(c, launch_mgs(c, fv, nullptr, nullptr, nullptr, gs + kGsH1, N));
  if ((st = readback()) != LSP_OK) return st;
  const double fn = sqrt(S.h_gs[kGsH1]);
  SCUDA(c, cudaMemcpyAsync(u, x, sizeof(double) * N,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           c->stream));
  SCUDA(c, cudaStreamSynchronize(c->stream));
  if (out) {
    out->iterations = iters;
    out->converged = conv ? 1 : 0;
    out->resid_precond = bnorm > 0.0 ? rnorm / bnorm : 0.0;
    out->resid_true = fn > 0.0 ? sqrt(S.h_gs[kGsH0]) / fn : 0.0;
  }
  return LSP_OK;
}

}  // extern "C"
