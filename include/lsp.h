/*
 * lsp.h -- C ABI of the GB300 stencil-setup library for the localized sparsifying
 * preconditioner (Liu & Ying, "Localized sparsifying preconditioner for periodic indefinite
 * systems").
 *
 * Problem (Sec. 1, Eq. model; Sec. 2, Eq. dmodel): (-Laplace + v) u = f on the periodic unit
 * cube [0,1)^d, discretised pseudospectrally on the n^d grid hJ, h = 1/n:
 *     (L + diag(v)) u = f,   L = F^-1 diag(4 pi^2 |k|^2) F,  k in K = [-n/2, n/2)^d.
 * For every grid point j the library builds the sparse rows Q[j, mu_j], C[j, mu_j] and
 * P[j, mu_j] of the preconditioner P^-1 C (Sec. 4.1, Eq. PC), mu_j = {i : |i - j|_inf <= t}.
 *
 * Conventions shared by every call:
 *  - Grid arrays are float64, row-major, last axis fastest, n^d entries.
 *  - Offsets o of mu_0 are in lexicographic order (o_1..o_d in [-t, t], last fastest);
 *    row j of Q, C, P holds |mu| = (2t+1)^d values, column (j + o) mod n for the o-th value.
 *  - Shifts live on the resonance-free lattice s = (4m + 2) pi^2 (Sec. 4.1); m is an integer
 *    "lattice index".
 *  - Every call returns an lsp_status; no call throws or aborts. On failure the context keeps a
 *    message readable with lsp_last_error().
 *  - Device work is issued on the CUDA stream given to lsp_create() and is stream ordered.
 *    Calls that return data to host memory synchronise that stream before returning.
 *  - Pointers passed in are borrowed for the duration of the call; output buffers are owned
 *    by the caller. The context owns all device scratch it allocates.
 */
#ifndef LSP_H
#define LSP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lsp_ctx lsp_ctx;

typedef enum {
  LSP_OK = 0,
  LSP_ERR_ARG = 1,             /* invalid argument (sizes, NaN/Inf in v, off-lattice shift) */
  LSP_ERR_STATE = 2,           /* call out of order (e.g. build before set_potential)        */
  LSP_ERR_RESONANT_SHIFT = 3,  /* a requested shift makes L + s singular (s = -4 pi^2 |k|^2) */
  LSP_ERR_CUDA = 4,            /* a CUDA runtime call or kernel launch failed                */
  LSP_ERR_OOM = 5,             /* device or pinned host allocation failed                    */
  LSP_ERR_TIMEOUT = 6,         /* a bounded device-side wait gave up                         */
  LSP_ERR_DEGENERATE = 7,      /* reserved: degenerate near-null spaces are flagged per shift */
  LSP_ERR_UNSUPPORTED = 8      /* valid request that this build does not implement           */
} lsp_status;

/*
 * LSP_FP64: every step in FP64. LSP_MIXED: the a3 contractions and the Gram blocks in FP32,
 * the near-null solve in FP64. LSP_LEARNED: a trained network gives alpha and c (see lsp_mlp).
 * LSP_DWORD: the a3 contractions in double words (pairs of FP32 values, about 48 significant
 * bits, formed with exact two-sum and fused-multiply-add product errors on the FP32 pipe), the
 * rest in FP64; the stencils meet the FP64 path's tolerance. Double words serve t = 1 builds
 * in 1D and 2D; elsewhere a LSP_DWORD build runs the FP64 stages (lsp_get_mode_used says so).
 */
typedef enum { LSP_FP64 = 0, LSP_MIXED = 1, LSP_LEARNED = 2, LSP_DWORD = 3 } lsp_mode;

typedef enum {
  LSP_SHIFT_PAPER = 0,  /* |S| shifts spread evenly over [v_min, v_max], snapped (Sec. 4.1)   */
  LSP_SHIFT_LOCAL = 1,  /* each point's own shift G_{v_j} of Sec. 4.1, snapped to the lattice */
  LSP_SHIFT_LIST = 2,   /* caller-given shift values (must lie on the lattice)               */
  LSP_SHIFT_MEAN = 3    /* the single shift snap(mean v) of Sec. 3                           */
} lsp_shift_policy;

typedef enum {
  LSP_EIG_SYMMETRIC = 0, /* block-diagonalise A by the cube symmetry of mu_0, solve the blocks */
  LSP_EIG_FULL = 1       /* cyclic Jacobi on the whole |mu| x |mu| matrix A                    */
} lsp_eig_method;

/* Per-shift flag bits (lsp_get_shift_table). */
#define LSP_FLAG_DEGENERATE 1    /* lambda_2 - lambda_1 < 1e-8 max|lambda|                    */
#define LSP_FLAG_NONSYMMETRIC 2  /* the smallest eigenvalue is not in the fully symmetric block */
#define LSP_FLAG_NOT_CONVERGED 4 /* Jacobi hit its sweep limit                                 */

typedef struct {
  int t;               /* neighbourhood radius t of mu_j^t (Sec. 4.2): 1 (|mu| = 3^d), or 2    */
                       /* in 2D and 3D (|mu| = 5^d; rows are 5^d wide, see nd_leaf)           */
  int policy;          /* lsp_shift_policy                                                     */
  int nshifts;         /* PAPER: |S| before de-duplication; 0 selects n/16 (2D), n/4 (1D, 3D) */
  const double* shifts;/* LIST: nshifts shift values in host memory, each (4m+2) pi^2          */
  int mode;            /* lsp_mode: FP64, MIXED (FP32 contractions/Gram, FP64 solve), LEARNED  */
  int refine_steps;    /* inverse-iteration steps applied to each near-null vector (0 or 1)   */
  int eig_method;      /* lsp_eig_method                                                       */
  int use_graph;       /* 1: record the launch sequence once per configuration, replay it     */
  int nd_leaf;         /* t = 2 only. 0: every point uses mu_j^2. b > 0 (even, dividing n):   */
                       /* point j uses t_j = min(2, T_b(j)), the largest t whose neighbourhood */
                       /* crosses no separator line x_a = 0 (mod b) of a nested dissection    */
                       /* with leaf boxes of width b (Sec. 4.2, figure of t choices: along an */
                       /* axis with r = x_a mod b > 0 the bound is min(r, b - r), on a        */
                       /* separator it is b). Rows stay 5^d wide: a t_j = 1 row fills its     */
                       /* inner 3^d columns and holds zeros elsewhere; the CSR export omits   */
                       /* them.                                                                */
  double learned_gate; /* LEARNED builds only. tau > 0: per-point residual gate. The eigen    */
                       /* path (a2-a6, FP64) also runs, and every point whose learned alpha   */
                       /* has rho_j = ||alpha^T G_{s_j}[mu_j, mu_j^c]|| / sigma_min(s_j) > tau */
                       /* (Sec. 3: sigma_min is the optimum of the sparsification problem)   */
                       /* gets the eigen path's Q, C, P rows instead (lsp_get_gate_stats).    */
                       /* 0: no gate (the network's rows as they come).                       */
} lsp_stencil_opts;

/*
 * Launch-shape autotuner (the paper has no counterpart; GB300 launch tuning). With on != 0,
 * the first build of each configuration (policy, mode, t, size class of the shift count) runs
 * eagerly, outside any graph capture, and times candidate launch shapes (threads per block and
 * grid caps in CTAs per SM) of the stage, 2D eigen and row kernels on the real data; later
 * builds (and recorded graphs) use the fastest. The per-point order of every sum is the same
 * under every shape, so tuned builds are bit-identical to untuned ones. Off by default.
 * lsp_get_tuning writes one line per tuned kernel ("key threads per_sm ms_default ms_best
 * candidates") into buf (NUL-terminated); LSP_ERR_ARG if len is too small.
 */
lsp_status lsp_set_autotune(lsp_ctx* ctx, int on);
lsp_status lsp_get_tuning(const lsp_ctx* ctx, char* buf, int64_t len);

/* Fill *opts with the defaults: t=1, LOCAL policy, FP64, symmetric eigen-solve, no graph,
 * nd_leaf = 0, learned_gate = 0. */
void lsp_default_opts(lsp_stencil_opts* opts);

/*
 * Create a context for the d-dimensional n^d grid (Sec. 2). d in {1, 2, 3}; n a power of two,
 * 8 <= n <= 4096 (1D, 2D) or 8 <= n <= 256 (3D), so that the offsets of mu_0 - mu_0 stay
 * distinct mod n. The 1D form (|mu| = 3) serves the one-dimensional example of Sec. 4.1. cuda_stream is a cudaStream_t (NULL = the legacy default stream) that every device
 * operation of the context is issued on. The current CUDA device at this call is the one used.
 * On success *out receives the context; release it with lsp_destroy().
 */
lsp_status lsp_create(int d, int n, void* cuda_stream, lsp_ctx** out);

/* Release a context and all device memory it owns. NULL is accepted. */
lsp_status lsp_destroy(lsp_ctx* ctx);

/*
 * Step a1: ingest the potential v (Sec. 2: v_j = v(h j)), n^d float64 values, row-major.
 * v_on_device = 1: v is a device pointer (copied device-to-device); 0: host pointer (copied
 * host-to-device). The call computes v_min, v_max and the mean (Sec. 3, Sec. 4.1) on the
 * device and waits for them (one small device-to-host read). Fails with LSP_ERR_ARG if v holds
 * NaN or Inf, or if the shifts it implies fall outside the supported lattice range |m| < 2^30.
 */
lsp_status lsp_set_potential(lsp_ctx* ctx, const double* v, int v_on_device);

/*
 * Steps a2-a7: build every stencil row (Sec. 4.1, Sec. 4.2).
 *   a2 shift list S and per-point shift s_j (arg-min of |s - v_j|, ties to the smaller s);
 *   a3 kernel vectors g_s = G_s[:, 0] and g_s * g_s at the offsets mu_0 - mu_0 (Sec. 4.2);
 *   a4 Gram matrix A = A1 - A2 of Eq. A;  a5 eigenvector alpha_s of its smallest eigenvalue,
 *      ||alpha|| = 1, alpha[centre] > 0;  a6 c_s = alpha_s^T G_s[mu_0, mu_0];
 *   a7 Q[j, mu_j] = alpha_{s_j}, C[j, mu_j] = c_{s_j},
 *      P[j, mu_j] = alpha_{s_j} + c_{s_j} .* (v[mu_j] - s_j).
 * Asynchronous on the context stream (except LIST/PAPER/MEAN, which upload a small shift list
 * from pinned host memory). Results stay on the device until read with lsp_get_rows(),
 * lsp_export_sparse_rows() or lsp_get_shift_table(). opts = NULL uses lsp_default_opts().
 * With t = 2 the same steps run on mu^2 (5^d offsets; g_s at offsets up to 4) and, when
 * nd_leaf > 0, also on mu^1 for the points with t_j = 1 (Sec. 4.2).
 * Errors: LSP_ERR_STATE without a potential; LSP_ERR_ARG for bad options or an off-lattice
 * LIST shift; LSP_ERR_RESONANT_SHIFT for a LIST shift equal to -4 pi^2 |k|^2 for a k in K;
 * LSP_ERR_UNSUPPORTED for t = 2 in 1D, for n < 8, or with the LEARNED mode.
 */
lsp_status lsp_build_stencils(lsp_ctx* ctx, const lsp_stencil_opts* opts);

/*
 * y = (L + diag(v)) u (Sec. 2, Eq. dmodel) for the context's current potential. u and y are
 * device pointers to n^d float64 values (real input; L maps real arrays to real arrays);
 * they may alias. Asynchronous on the context stream. LSP_ERR_STATE without a potential.
 */
lsp_status lsp_apply_operator(lsp_ctx* ctx, const double* u_dev, double* y_dev);

/*
 * Copy the dense row block of Q, C or P (which = 'Q', 'C', 'P'): n^d x |mu| float64,
 * row j at rows[j * |mu| ...], in mu_0 offset order (|mu| = (2t+1)^d of the last build, as
 * lsp_get_sizes reports it). on_device = 1: rows is a device pointer
 * (asynchronous copy); 0: host pointer (the call waits for the copy).
 */
lsp_status lsp_get_rows(lsp_ctx* ctx, char which, double* rows, int on_device);

/*
 * Start copying the row block of Q, C or P of the last build (layout as lsp_get_rows) into
 * host memory rows_host, and return without waiting. The block is first copied on the device
 * (a staging copy, stream-ordered on the context stream after the build); the host copy then
 * runs on a second stream of the context, so the next set_potential and build may proceed
 * while it is in flight (a serving loop overlaps step k's host copy with step k + 1's build).
 * A later call for the same block waits for the previous one's host copy before reusing the
 * staging copy. rows_host must stay valid and untouched until lsp_wait_rows() returns; page-
 * locked memory (cudaHostAlloc or cudaHostRegister) is needed for the copy to be asynchronous.
 * The staging copies take 3 n^d |mu| doubles of device memory, allocated on first use.
 * Errors: LSP_ERR_ARG (NULL rows_host, bad which), LSP_ERR_STATE before a build,
 * LSP_ERR_OOM, LSP_ERR_CUDA.
 */
lsp_status lsp_get_rows_async(lsp_ctx* ctx, char which, double* rows_host);

/* Wait until every copy started by lsp_get_rows_async() has landed in host memory. */
lsp_status lsp_wait_rows(lsp_ctx* ctx);

/*
 * Export Q, C or P as CSR in host memory: rowptr[n^d + 1] (int64), colidx[nnz] (int32),
 * vals[nnz] (float64), nnz = n^d |mu| (t = 2 builds with nd_leaf > 0: the sum over points
 * of (2 t_j + 1)^d). Column indices of a row follow the mu_j^{t_j} offset order, so they are
 * not sorted where the neighbourhood wraps around the periodic boundary.
 * With rowptr, colidx and vals all NULL only *nnz_out is written (size query). Waits for the
 * copies before returning.
 */
lsp_status lsp_export_sparse_rows(lsp_ctx* ctx, char which, int64_t* rowptr, int32_t* colidx,
                                  double* vals, int64_t* nnz_out);

/*
 * Read the per-shift table of the last build into host memory (Sec. 4.1: one stencil per
 * shift, shared by every point that uses that shift). *nshifts_out receives |S|. For a t = 2
 * build the table holds the t = 2 stencils (|mu| = 5^d).
 * Any output pointer may be NULL. s[|S|] shift values (increasing), alpha[|S| x |mu|],
 * c[|S| x |mu|], lam[|S| x 2] = (lambda_1, lambda_2) of A, flags[|S|] (LSP_FLAG_* bits),
 * s_idx[n^d] = index into s of each point's shift s_j. Waits before returning.
 */
lsp_status lsp_get_shift_table(lsp_ctx* ctx, int64_t* nshifts_out, double* s, double* alpha,
                               double* c, double* lam, int32_t* flags, int32_t* s_idx);

/* |mu| = (2t+1)^d for t = 1 and the number of grid points n^d. */
lsp_status lsp_get_sizes(const lsp_ctx* ctx, int64_t* npoints, int* mu);

/* Block until all work issued by the context has finished. */
lsp_status lsp_synchronize(lsp_ctx* ctx);

/*
 * Per-kernel timing with CUDA events on the context stream. enable = 1 starts recording
 * (graph replay is bypassed while enabled), 0 stops. lsp_kernel_times() copies, for up to
 * cap kernels, the name (NUL-terminated, up to 31 chars), the summed milliseconds and the
 * launch count since the last enable, and returns the number of kernels seen in *count.
 */
lsp_status lsp_kernel_timing(lsp_ctx* ctx, int enable);
lsp_status lsp_kernel_times(lsp_ctx* ctx, int cap, char (*names)[32], double* ms,
                            int64_t* launches, int* count);

/*
 * ---- Learned stencils (no counterpart in the paper: a surrogate for steps a3-a6) ----
 * A multilayer perceptron maps the 5^d patch of h^2 v around a point and the point's snapped
 * shift h^2 s_j (normalised) to that point's (alpha, c); it is trained on the stencils the
 * eigen path (Sec. 4.1-4.2) produces.
 * Layers: (5^d+1 -> 256), (256 -> 256), (256 -> 256) with ReLU max(z, 0), then (256 -> 2|mu|);
 * bf16 weights and hidden activations,
 * fp32 accumulation on the tensor cores, fp32 master weights and Adam. In a LEARNED build the
 * rows are Q = alpha / |alpha|, C = c / |alpha|, P = Q + C .* (v[mu_j] - s_j), s_j = snap(v_j).
 */
typedef struct lsp_mlp lsp_mlp;

/* New network for d in {2, 3}, initialised from `seed`, working on cuda_stream. */
lsp_status lsp_mlp_create(int d, uint64_t seed, void* cuda_stream, lsp_mlp** out);
lsp_status lsp_mlp_destroy(lsp_mlp* m);
/* Length of the flat fp32 parameter vector (*total) and how many of them are trainable. */
lsp_status lsp_mlp_param_count(const lsp_mlp* m, int64_t* total, int64_t* nweights);
/*
 * Copy the flat fp32 parameter vector to / from host memory. Layout: W1 [256 x K0], b1 [256],
 * W2 [256 x 256], b2, W3, b3, W4 [OUTP x 256], b4 [OUTP], then mu_x, sigma_x, mu_y[OUTP],
 * sigma_y[OUTP], and the trained input range [lo, hi] of h^2 v. K0 = 32 (2D) / 128 (3D) with
 * the 5^d + 1 real inputs first; OUTP = 32 / 64 with the 2|mu| real outputs first (alpha, c).
 */
lsp_status lsp_mlp_get_params(lsp_mlp* m, float* host);
lsp_status lsp_mlp_set_params(lsp_mlp* m, const float* host);
/*
 * Training pairs from the context's last FP64 or MIXED build: for nsamples pseudo-random
 * points (a hash of (seed, i)), X_dev[i] = the 5^d raw h^2 v features and h^2 s_j (fp32) and
 * T_dev[i] = (alpha, c) of the point (fp32, 2|mu| values). Device pointers, caller-owned.
 */
lsp_status lsp_mlp_training_pairs(lsp_ctx* ctx, lsp_mlp* m, int64_t nsamples, uint64_t seed,
                                  float* X_dev, float* T_dev);
/* Set the input / output normalisation and the trained input range from n raw pairs. */
lsp_status lsp_mlp_fit_normalization(lsp_mlp* m, const float* X_dev, const float* T_dev, int64_t n);
/* Y_dev[i] (OUTP fp32, normalised output space) for raw inputs X_dev[i], i < batch. */
lsp_status lsp_mlp_forward(lsp_mlp* m, const float* X_dev, int64_t batch, float* Y_dev);
/*
 * One training step on raw pairs (batch a multiple of 128): loss = mean over the batch and
 * the 2|mu| outputs of (y - t_normalised)^2. apply = 1 takes an Adam step with rate lr.
 * *loss_out (host) receives the loss; grads_host (optional, host, nweights floats) receives
 * the gradient of the trainable parameters before the update.
 */
lsp_status lsp_mlp_train_step(lsp_mlp* m, const float* X_dev, const float* T_dev, int64_t batch,
                              float lr, int apply, float* loss_out, float* grads_host);
const char* lsp_mlp_last_error(const lsp_mlp* m);
/*
 * Wall-time limit (ns) of the operand waits inside the network's fused kernel (0: the default,
 * 1 s). A wait that runs out sets the error word; the kernel then drains its copies and tensor-
 * core work in flight (those waits keep the 1 s limit), frees its tensor memory and returns, and
 * lsp_synchronize reports LSP_ERR_TIMEOUT; the context stays usable. The paper has no
 * counterpart: this exists so that the timeout path can be exercised without a stuck GPU.
 */
lsp_status lsp_mlp_set_wait_limit(lsp_mlp* m, uint64_t ns);
/*
 * Schedule of the 2D network's fused inference kernel: 1 (the default) keeps two 128-row tiles
 * in flight per SM, so that one tile's tensor-core products overlap the other's epilogue;
 * 0 runs one tile at a time; 2 runs the two-tile schedule on pairs of SMs (a two-CTA cluster
 * with 256-row tensor-core products, each CTA holding half of every weight chunk) for the
 * rows of a build, and schedule 1 for training batches. All three compute the same rows bit
 * for bit; schedule 2 measured slower than 1 and is kept for comparison. 3D networks always
 * run one tile at a time (two tiles' buffers do not fit in shared memory). LSP_ERR_ARG for any
 * other value.
 */
lsp_status lsp_mlp_set_schedule(lsp_mlp* m, int schedule);
/* Attach a network to a context for LSP_LEARNED builds (NULL detaches). Same d required. */
lsp_status lsp_set_mlp(lsp_ctx* ctx, lsp_mlp* m);
/*
 * Mode the last build actually used: a LEARNED build whose potential leaves the network's
 * trained input range falls back to LSP_FP64 (the eigen path).
 */
lsp_status lsp_get_mode_used(const lsp_ctx* ctx, int* mode);
/*
 * Result of the per-point residual gate of the last LEARNED build with learned_gate > 0
 * (Sec. 3: the residual ||alpha^T G_s[mu, mu^c]|| of a stencil against its optimum, the
 * smallest singular value). *fallback_points (host) receives how many points took the eigen
 * path's rows. rho_host (host, N floats, optional) receives each point's ratio
 * rho_j = sqrt(1 + delta^T (A - lambda_1 I) delta / lambda_1), delta the learned alpha
 * normalised and sign-matched minus the eigen path's alpha of the point's shift (+inf where
 * lambda_1 <= 0). The ratio of a fallback point is the learned one that failed the gate.
 * Synchronises the context's stream. LSP_ERR_STATE if the last build was not gated.
 */
lsp_status lsp_get_gate_stats(lsp_ctx* ctx, int64_t* fallback_points, float* rho_host);

/*
 * Allocation-failure injection for tests of the out-of-memory path (the paper has no
 * counterpart). after >= 0: the library's next `after` device allocations succeed and the one
 * after them fails as if cudaMalloc had run out of memory, so the call that needed it returns
 * LSP_ERR_OOM with nothing half-built (the context stays usable once the injection is cleared);
 * after < 0 clears it. Process-wide; not thread-safe against concurrent library calls.
 */
void lsp_inject_alloc_failure(int after);

/*
 * y = (L + diag(v)) u, like lsp_apply_operator, for callers that cannot allocate device
 * memory when they need the operator: code running while a stream is being captured into a
 * CUDA graph (cudaMalloc is not permitted there), or code whose device memory belongs to a
 * pool or framework allocator that must not see extra allocations or device-wide syncs.
 * The paper has no counterpart; this is a deployment variant of the same operator.
 *
 * Nothing is allocated: the transform's complex work array is a fixed array inside the
 * library (16 MiB plus 32 KiB of twiddles, held on every GPU that loads the library until the
 * process exits). The caller passes all inputs and outputs as device pointers to n^d float64
 * values: the potential v, the input u and the output y (y may alias u). d in {2, 3}, n a power
 * of two >= 8, and n^d <= LSP_NOALLOC_MAX_POINTS; larger grids return LSP_ERR_ARG (use a
 * context). The work is issued on cuda_stream (a cudaStream_t; NULL = legacy default stream).
 * Every call looks up the array's device address (cudaGetSymbolAddress) in the current
 * device's current context; the lookup allocates nothing. The first call in a context also
 * loads the library's device code there, so make that first call before any stream capture.
 * Every call on a device shares the one array: calls whose GPU work may overlap (different streams, no ordering)
 * race and give wrong results. Each call overwrites the whole work array before reading it,
 * so nothing needs clearing. Errors: LSP_ERR_ARG for bad sizes or NULL pointers,
 * LSP_ERR_CUDA if the address lookup or a launch fails.
 */
#define LSP_NOALLOC_MAX_POINTS 1048576
lsp_status lsp_apply_operator_noalloc(int d, int n, const double* v_dev, const double* u_dev,
                                      double* y_dev, void* cuda_stream);

/* ---- Applying the preconditioner (Sec. 3, Eq. QC and Eq. PC; Fig. nd; Table cost; Sec. 5) ----
 *
 * P = Q + C diag(v - s) has the sparsity of Q, so P^-1 is applied through a nested-dissection
 * factorisation, and (L + diag v) u = f is solved by GMRES left-preconditioned with P^-1 C.
 * 2D grids (n a power of two, 4 <= n <= 1024) and 3D grids (4 <= n <= 64); rows of a t = 1
 * build, or of a t = 2 build with nd_leaf = b (the t_j rule keeps every row inside the
 * separators of that dissection).
 *
 * Elimination tree: in 2D (and in 3D with n < 2b) the root separator {x : some x_a = 0} last,
 * before it the boxes of the remaining open square (cube); in 3D with n >= 2b the plane pairs
 * {x_a = 0} U {x_a = n/2} of axes 0, 1, 2 at depths 0, 1, 2 (two children per node), before them
 * the eight open cubes. Each open box is split through the middle grid line (plane) of its
 * longest side down to leaf boxes of at most (b - 1)^d points. Every separator lies on
 * x_a = 0 (mod b).
 * Each front (eliminated set E, ring R of ancestors' points) is inverted on E in place with row
 * pivoting inside E; the figure of Sec. 3 groups the separators into edges and vertices
 * instead, with the same leaf boxes and the same separator lines. */
typedef struct {
  int leaf;          /* b: power of two in [4, n]. 0: the nd_leaf of a t = 2 build, else 8      */
                     /* (Sec. 5 fixes b = 8)                                                     */
  int refine_steps;  /* 0..4 steps x += P^-1 (y - P x) after each solve (lsp_nd_solve and the   */
                     /* preconditioner of lsp_gmres). Pivots are chosen inside each front's E, */
                     /* so a front whose E block is ill-conditioned (long separators of a      */
                     /* high-frequency problem) raises the backward error of a plain solve     */
                     /* (measured 1e-9 at 2D n = 1024, 4 points per wavelength); one step      */
                     /* brings it to the rounding level.                                       */
} lsp_nd_opts;

typedef struct {
  int levels;           /* depth of the elimination tree + 1                                  */
  int leaf;             /* b                                                                  */
  int max_front;        /* largest front |E| + |R|                                            */
  int factored;         /* 1 when a factorisation of the current stencils is held             */
  int64_t fronts;       /* number of fronts                                                   */
  int64_t front_bytes;  /* device bytes of the fronts (sum of (|E| + |R|)^2 * 8)              */
  int64_t solve_bytes;  /* front bytes one solve reads (sum of (|E| + |R|) |E| + |E| |R|, x 8) */
  double flops;         /* FP64 flops of the factorisation as run: 2 |E| (|E| + |R|)^2 a front  */
  double flops_lu;      /* the multifrontal LU count 2/3 |E|^3 + 2 |E|^2 |R| + 2 |E| |R|^2    */
} lsp_nd_info;

/* Zero-initialised options (leaf 0, no refinement). */
void lsp_default_nd_opts(lsp_nd_opts* opts);

/* Factorise the P rows of the last build (stream-ordered on the context stream; returns after
 * the stream has finished, so the call's duration is the setup time T_NDsetup of Sec. 5). The
 * symbolic plan of the dissection is made on the host once per (n, b, row pattern) and kept.
 * Errors: LSP_ERR_STATE before a build; LSP_ERR_UNSUPPORTED for 1D grids, n above the limits
 * or rows that cross the separators (t = 2 without nd_leaf); LSP_ERR_ARG for a bad b or
 * b != nd_leaf;
 * LSP_ERR_DEGENERATE when a pivot vanishes (P singular). A later build invalidates the factor. */
lsp_status lsp_nd_factor(lsp_ctx* ctx, const lsp_nd_opts* opts);

/* Host only (no context, no device): plan the dissection of the n^d grid (d = 2, 3) with leaf
 * b for the rows of a t = 1 build (t = 1) or of a t = 2 build with nd_leaf (t = 2) and report
 * its sizes; the first `cap` depths (0 = the root separator) also give their front count and
 * |E|, |R| in count[], s[], r[] (any may be NULL). LSP_ERR_UNSUPPORTED with the reason in err
 * (errcap bytes) when the rows or sizes do not fit; LSP_ERR_ARG for d outside {2, 3}, t outside
 * {1, 2} or a NULL info. */
lsp_status lsp_nd_plan_info(int d, int n, int leaf, int t, int nd_leaf, lsp_nd_info* info,
                            int cap, int* count, int* s, int* r, char* err, int errcap);

/* Sizes and flop counts of the planned dissection. LSP_ERR_STATE if none was planned. */
lsp_status lsp_nd_get_info(lsp_ctx* ctx, lsp_nd_info* info);

/* x = P^-1 y for device vectors of n^d float64 (x may equal y), followed by the refinement
 * steps chosen at lsp_nd_factor; stream-ordered, deterministic.
 * LSP_ERR_STATE unless lsp_nd_factor ran on the current stencils. */
lsp_status lsp_nd_solve(lsp_ctx* ctx, const double* y_dev, double* x_dev);

/* y = M u for M = Q, C or P of the last build (row j: sum over its neighbourhood columns,
 * periodic wrap), device vectors of n^d float64 that must not alias; stream-ordered. */
lsp_status lsp_apply_rows(lsp_ctx* ctx, char which, const double* u_dev, double* y_dev);

typedef struct {
  double rtol;     /* stop when |P^-1 C (f - A u)| <= rtol |P^-1 C f| (Sec. 5: 1e-6)              */
  int restart;     /* Krylov dimension per cycle, 1..60 (Sec. 5: 40)                             */
  int max_cycles;  /* restart cycles before giving up                                           */
  int precond;     /* 1: left preconditioner P^-1 C (needs lsp_nd_factor); 0: none              */
} lsp_gmres_opts;

typedef struct {
  int iterations;        /* inner (Arnoldi) iterations: N_iter of the tables of Sec. 5           */
  int converged;         /* 1 when the preconditioned residual met rtol                          */
  double resid_precond;  /* |P^-1 C (f - A u)| / |P^-1 C f| at exit (A = L + diag v)             */
  double resid_true;     /* |f - A u| / |f|                                                      */
} lsp_gmres_result;

/* rtol 1e-6, restart 40, max_cycles 50, precond 1. */
void lsp_default_gmres_opts(lsp_gmres_opts* opts);

/* Solve (L + diag v) u = f by restarted GMRES with x0 = 0, modified Gram-Schmidt Arnoldi and
 * Givens rotations; the inner loop stops when the least-squares residual reaches rtol |b|
 * (b = P^-1 C f), a cycle ends with the explicit residual of the preconditioned system, and the
 * next cycle restarts from it. f and u are n^d float64, both in device memory (on_device = 1)
 * or both in host memory (0); the call returns after the stream has finished. Every vector
 * operation runs on the device; the host reads one residual estimate per inner iteration.
 * Errors: LSP_ERR_STATE before set_potential or, with precond, without a current factor. */
lsp_status lsp_gmres(lsp_ctx* ctx, const lsp_gmres_opts* opts, const double* f, double* u,
                     int on_device, lsp_gmres_result* result);

/* Message of the last failed call on this context ("" if none). Never NULL. */
const char* lsp_last_error(const lsp_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LSP_H */
