// Nested-dissection factorisation and solve of P on the GPU (Sec. 3, Eq. QC: the sparse matrix
// P = Q + C diag(v - s) has the sparsity of Q, so P^-1 can be applied by nested dissection;
// Fig. nd; Table cost: T_NDsetup, T_NDapp), and the Krylov solve that uses it (Sec. 5: GMRES
// with restart 40, relative tolerance 1e-6, left-preconditioned by P^-1 C).
//
// Elimination tree of the periodic grid (n = 2^p, leaf width b = 2^q):
//  - 2D (and 3D with n < 2b): depth 0 is the cross {some x_a = 0}; removing it leaves the open
//    square (cube) [1, n)^d;
//  - 3D with n >= 2b: depths 0, 1, 2 open one axis each: a node's points on the plane pair
//    {x_a = 0} U {x_a = n/2} are its eliminated set, its children the two halves
//    [1, n/2) and [n/2 + 1, n) along that axis; after three depths the nodes are open cubes;
//  - then: open boxes of (2^k - 1) points per side, split through their middle line (plane),
//    the longest side first, into two halves; the separator is the node's eliminated set;
//  - leaves: boxes of at most (b - 1)^d points, all eliminated at once.
// Every separator lies on x_a = 0 (mod b), so rows whose neighbourhood crosses no such line
// (t = 1 everywhere, or t_j from the leaf-b rule of Sec. 4.2) keep the dissection exact.
//
// A front holds the eliminated set E (|E| = s) followed by the ring R of its box (|R| = r):
// the points of ancestors' separators adjacent to the box. Its f x f matrix (f = s + r,
// row-major) is assembled from the two children's Schur complements and P's entries, then
// replaced in place by the partial inverse on E (the principal pivot transform), with row
// pivoting among the rows of E:
//     [A B; C D]  ->  [A^-1, A^-1 B; -C A^-1, D - C A^-1 B]      (A = the permuted E x E block)
// The solve is then two matrix-vector products per front (forward: z = A^-1 w_E,
// u = w_R - C A^-1 w_E; backward: x_E = z - A^-1 B x_R).
#pragma once

#include <string>
#include <vector>

#include "lsp_internal.h"

namespace lsp {

constexpr int kNdPanel = 16;       // columns eliminated per step in the blocked path
constexpr int kNdSmallFront = 160; // fronts with f <= this are swept in shared memory
constexpr int kNdStagedBytes = 64 * 1024;  // solve blocks up to this size are staged
constexpr int kNdMaxN = 1024;      // 2D: the cross has 2n - 1 points
constexpr int kNdMaxN3 = 64;       // 3D: the slab fronts have 2 (n/2 - 1) n + 2 n^2 points (12 160 at 64)
constexpr int kNdPanelRegRows = 8 * 256;  // panels up to this many rows keep them in registers

struct NdLevel {
  int count = 0;       // fronts at this depth
  int s = 0, r = 0, f = 0;
  int nchild = 0;      // children per front: 2, 1 (the cross root), 0 (leaves)
  int64_t front_off = 0;          // doubles into the front buffer (count * f * f)
  int64_t E_off = 0, R_off = 0;   // int32 offsets into E (count * s) and R (count * r)
  int64_t inv_off = 0;            // int32 offset into inv (count * f * 2)
  int64_t asm_off = 0, asm_n = 0; // P entries assembled at this depth
  int64_t perm_off = 0;           // int32 offset into perm (count * s)
  int64_t z_off = 0, u_off = 0;   // doubles into the solve vectors z (count * s), u (count * r)
};

struct NdPlan {
  int d = 2, n = 0, leaf = 0, mu = 0, t_built = 1, leaf_t = 0;
  std::vector<NdLevel> lv;  // lv[0]: the root separator; lv.back(): the leaves
  // E, R: grid indices of every front's eliminated set and ring, front after front.
  // inv[(front * f + i) * 2 + c]: position of front position i in child c's ring, or -1.
  // asm_dst / asm_src: P entry rows[src] goes to element dst of its depth's front block.
  std::vector<int32_t> E, R, inv, asm_dst, asm_src;
  int64_t front_doubles = 0, perm_ints = 0, z_doubles = 0, u_doubles = 0;
  double flops_sweep = 0;  // FP64 flops of the partial inversions, 2 s f^2 per front
  double flops_lu = 0;     // multifrontal LU count, 2/3 s^3 + 2 s^2 r + 2 s r^2 per front
  int64_t solve_bytes = 0; // front bytes one solve reads: (f s + s r) * 8 per front
  int max_f = 0, max_s = 0;
};

// Builds the plan for rows of width mu on the periodic n^d grid (d = 2, 3; t_built = 1: 3^d
// rows; t_built = 2: 5^d rows, of which point j uses its core from the leaf-leaf_t rule).
// Returns "" or the reason the rows or sizes do not fit the dissection.
std::string build_nd_plan(NdPlan& p, int d, int n, int leaf, int t_built, int leaf_t, int mu);

struct NdState {
  NdPlan plan;
  bool have_plan = false;
  bool factored = false;
  int64_t factored_gen = -1;  // ctx->build_gen of the rows that were factored
  int refine_steps = 0;       // iterative-refinement steps after every solve
  DevBuf fronts, E, R, inv, asm_dst, asm_src, perm, z, u, cbuf, pinv, swaps, err;
  DevBuf ry, rd;              // refinement scratch: a copy of y, the correction
  DevBuf pscratch;            // FP32 pivot-ranking rows of panels over 2048 rows
  int64_t cbuf_half = 0, pinv_half = 0, swaps_half = 0;  // the two copies of the step buffers
  cudaStream_t side = nullptr;  // look-ahead panels (high priority)
  cudaEvent_t ev_cols = nullptr, ev_panel = nullptr;
  // GMRES workspace
  DevBuf V, w, b, x, tmp, gs, fvec;
  double* h_gs = nullptr;  // pinned mirror of the scalars the host loop reads
  int restart_cap = 0;
};

void nd_free(NdState* s);

// ---- launchers (k_nd.cu) ----
cudaError_t launch_nd_assemble(lsp_ctx* c, int depth, const double* rows);
cudaError_t launch_nd_sweep(lsp_ctx* c, int depth);
cudaError_t launch_nd_solve(lsp_ctx* c, const double* y, double* x);
cudaError_t launch_apply_rows(lsp_ctx* c, const double* rows, int mu, int t, const double* u,
                              double* y);

// ---- GMRES kernels (k_gmres.cu) ----
// MGS step: w -= h_prev * v_prev (if v_prev), then *h_out = <v_next, w> (or <w, w>).
cudaError_t launch_mgs(lsp_ctx* c, double* w, const double* v_prev, const double* h_prev,
                       const double* v_next, double* h_out, int64_t N);
cudaError_t launch_axpby(lsp_ctx* c, double* y, const double* a, const double* x,
                         const double* scale, double sign, int64_t N);
cudaError_t launch_gmres_givens(lsp_ctx* c, double* gs, int col, int ld);
cudaError_t launch_gmres_update(lsp_ctx* c, double* gs, int col, int ld, const double* V,
                                double* x, int64_t N);
cudaError_t launch_gmres_start(lsp_ctx* c, double* gs, int ld, const double* r, double* v0,
                               int64_t N);

// Layout of the GMRES scalars (doubles) in NdState::gs; H is column-major (ld = restart + 1).
enum GmresSlot {
  kGsNorm = 0,     // scratch: a squared norm
  kGsH0 = 1,       // |w|^2 before orthogonalisation
  kGsH1 = 2,       // |w|^2 after
  kGsPresid = 3,   // |S[col + 1]| after the rotation
  kGsBreak = 4,    // 1 when w vanished (exact solution in the subspace)
  kGsInvH1 = 5,    // 1 / |w| (0 on breakdown)
  kGsBeta = 6,     // |r| at the start of a cycle
  kGsTicket = 7,   // reduction ticket (as an unsigned int)
  kGsPartial = 8,  // 1024 block partial sums
  kGsArrays = 8 + 1024  // then H[(ld) * restart], cs[restart], sn[restart], S[ld], y[restart]
};

}  // namespace lsp
