/*
 * nmg.h -- C ABI of the GB300 neural multigrid solver.
 *
 * The library solves A u = f for many right-hand sides f with the neural
 * multigrid cycle of the paper "A level-wise training scheme for learning
 * neural multigrid smoothers with application to integral equations":
 * NMGF1d (Algorithm 3) in 1D and NMGF2d (Algorithm 4) in 2D, iterated as
 * x^tau = NMGF(x^{tau-1}, f) from x^0 = 0 (Section 3.2) until the relative
 * residual ||f - A u|| / ||f|| reaches a tolerance.  As in the paper's
 * statement of the problem (Section 5: the matrix is fixed, only the
 * right-hand sides vary), a hierarchy is set up once from the kernel, grid,
 * regularisation weight, level count and frozen smoother weights, and then
 * solves any number of batches.
 *
 * Conventions for every entry point:
 *  - All functions return an nmg_status; no C++ exception crosses the ABI.
 *    Argument errors are detected before any kernel launch and leave device
 *    buffers untouched.  The text of the last error of a context is kept
 *    in nmg_last_error().
 *  - "device" pointers are CUDA device pointers on the context's device;
 *    work is ordered on the context's stream.  Functions that report values
 *    to the host (nmg_solve's info, norms) synchronise that stream before
 *    they return; the others are asynchronous.
 *  - A batch holds 0 .. NMG_MAX_BATCH right-hand sides (larger batches:
 *    NMG_ERR_ARG).
 *  - The caller owns every pointer it passes.  The library owns contexts,
 *    hierarchies and their workspaces until the matching destroy call.
 *  - Layouts are row-major: a batch of 2D grids is [batch][n][n], a batch
 *    of 1D grids is [batch][n], contiguous.  In 2D the operator is
 *    symmetric in both axes, so row-major storage of X is the paper's
 *    column-major Vec(X) of Section 3.3 read transposed, with the same
 *    operator.
 *  - Element types follow the hierarchy's precision:
 *      NMG_FP64          f, u, every level vector: double
 *      NMG_FP32          f, u, every level vector: float
 *      NMG_BF16_REFINE,
 *      NMG_BF16TOP_REFINE,
 *      NMG_BF16X3_REFINE,
 *      NMG_BF16FAST_REFINE,
 *      NMG_FP16_REFINE   f: float, u: double; level vectors of the inner
 *                        cycle (step entry points): float.  The smoother
 *                        runs on 16-bit tensor cores with fp32 accumulation.
 */
#ifndef NMG_H
#define NMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nmg_ctx nmg_ctx;   /* opaque: device, stream, error text */
typedef struct nmg_hier nmg_hier; /* opaque: one operator's level hierarchy */

typedef enum {
  NMG_OK = 0,
  NMG_ERR_ARG = -1,        /* invalid argument (null pointer, size, level) */
  NMG_ERR_OOM = -2,        /* device allocation failed */
  NMG_ERR_NOT_SPD = -3,    /* coarsest operator not positive definite */
  NMG_ERR_CUDA = -4,       /* a CUDA call failed; see nmg_last_error */
  NMG_ERR_TIMEOUT = -5,    /* a bounded device wait gave up */
  NMG_ERR_WEIGHTS = -6,    /* smoother weights inconsistent with the desc */
  NMG_ERR_UNSUPPORTED = -7 /* valid request this build does not implement */
} nmg_status;

/* largest batch of one call (one grid row of blocks per right-hand side) */
#define NMG_MAX_BATCH 65535

/* per right-hand-side outcome, in nmg_solve_info.status */
enum { NMG_CONVERGED = 0, NMG_NOT_CONVERGED = 1, NMG_DIVERGED = 2 };

/* Precision forms.  The refinement forms run the cycle as an inner solve of
 * an outer iterative refinement (residual in compensated fp32, update in
 * fp64) with the smoother's hidden layers on 16-bit tensor cores and fp32
 * accumulation:
 *   NMG_BF16_REFINE      every hidden-layer operand (activation and
 *                        weight) is a sum of three bf16 values (fp32-level,
 *                        2^-24 relative); each product takes the six MMAs
 *                        of its terms down to order 2^-16 (three MMA
 *                        instructions, 6x the MMA work of one bf16
 *                        product); per-cycle iterates agree with fp64 to
 *                        about 1e-5 even for trained smoothers that amplify
 *                        rounding strongly.
 *   NMG_BF16TOP_REFINE   the three-term form of NMG_BF16_REFINE on the
 *                        finest level's smoother, the pair form of
 *                        NMG_BF16X3_REFINE on every coarser level.  The
 *                        rounding of the finest smoother reaches the
 *                        cycle's result undamped; a coarser level's
 *                        output reaches it only through the filter,
 *                        prolongation and the finer levels, and for the
 *                        trained smoothers of the 512x512 operators the
 *                        pairs there leave the cycle's error at the
 *                        three-term level (a product emulation shows
 *                        the same error as three terms everywhere).
 *                        Saves about half the MMA work of the coarser
 *                        levels (a quarter of the pixels).
 *   NMG_BF16X3_REFINE    every hidden-layer operand is a pair of bf16
 *                        values (hi + lo, 2^-16 relative), three products
 *                        a_hi*w_hi + a_hi*w_lo + a_lo*w_hi (2 MMA
 *                        instructions, 3x the MMA work); per-cycle iterates
 *                        agree with fp64 to 1e-4..2e-3 depending on how
 *                        strongly the trained smoother amplifies rounding.
 *   NMG_BF16FAST_REFINE  one bf16 value per operand, 1 MMA per product;
 *                        the cycle converges at the same rate but single
 *                        cycles differ from fp64 by percents.
 *   NMG_FP16_REFINE      as NMG_BF16X3_REFINE with fp16 pairs (2^-22
 *                        relative) at the same cost; the network runs on
 *                        power-of-two-scaled values to stay inside fp16's
 *                        range (activations above 65504 are clamped).
 * All of them take f: float, u: double, like NMG_BF16_REFINE above. */
typedef enum {
  NMG_FP64 = 0,
  NMG_FP32 = 1,
  NMG_BF16_REFINE = 2,
  NMG_BF16FAST_REFINE = 3,
  NMG_FP16_REFINE = 4,
  NMG_BF16X3_REFINE = 5,
  NMG_BF16TOP_REFINE = 6
} nmg_precision;

/*
 * Operator description (Section 2.1, Eq. (1); Eq. (10) in 1D; the
 * Kronecker form alpha I(x)I + K(x)K of Section 4.2 in 2D).
 *   dim      1 or 2
 *   n        fine grid side: a power of two (the output filter uses radix-2
 *            FFTs), so n % 2^(levels-1) == 0 as Section 2.3 requires.  The
 *            coarsest grid must have at most 1024 unknowns.
 *   levels   L, counting the coarsest level; smoothers run on levels
 *            1..L-1, the exact solve on level L.  levels >= 1.
 *   alpha    regularisation weight (> 0 is not required, but the coarsest
 *            Galerkin operator must be SPD or setup fails NMG_ERR_NOT_SPD)
 *   taps     host array, copied at setup:
 *              dim 1: ntaps == n, the first column t_0..t_{n-1} of the
 *                     symmetric Toeplitz matrix (the discretised h*K);
 *                     A_1 = Toeplitz(t) + alpha I
 *              dim 2: ntaps == w+1, symmetric PSF taps g_0..g_w with
 *                     K[i][j] = g_|i-j| for |i-j| <= w;
 *                     A_1 = alpha I(x)I + K(x)K, zero boundary
 *   precision  nmg_precision
 *   filter   1: NMGF with the output filter F'_l (Algorithms 3/4);
 *            0: no filter (Algorithm 2, x = x* + h)
 *   reg, nreg  dim 1 only, optional (NULL, 0: D = I, the Tikhonov term):
 *            the regularisation matrix D of the anisotropic case of
 *            Section 4.1 (A = alpha D + K), symmetric tridiagonal, given as
 *            its n diagonal entries followed by its n-1 off-diagonal
 *            entries (nreg == 2n-1), host, copied at setup;
 *            A_1 = Toeplitz(t) + alpha D.  NMG_ERR_ARG if given in 2D or
 *            with another length.
 * Coarse operators are Galerkin products A_{l+1} = R A_l P with linear
 * interpolation P (coarse node J at fine 2J) and full weighting R = P^T/2
 * per axis.
 */
typedef struct {
  int dim;
  int n;
  int levels;
  double alpha;
  int ntaps;
  const double* taps;
  int precision;
  int filter;
  const double* reg;
  int nreg;
} nmg_operator_desc;

/* smoother architectures (nmg_smoother_desc.arch) */
#define NMG_SMOOTHER_CNN 0
#define NMG_SMOOTHER_FNO 1

/*
 * Smoother description: a CNN per smoother level (the paper's smoothers
 * are neural operators, Section 3.1; here conv -> ReLU -> ... -> conv with
 * zero 'same' padding and a bias on every layer), or the FNO of Appendix A.
 *   layers   number of conv layers (>= 2); channels 1 -> width ->...-> 1
 *            (every level, unless level_layers is given)
 *   width    hidden channels (2D: 32; 1D: 16 in this build)
 *   ksize    kernel size (2D: 3; 1D: 5 in this build)
 *   nlevels  smoother levels present in `weights`; must be >= levels-1.
 *            Only the first levels-1 are used (a coarsest level chosen
 *            below the trained one, as in Section 4.3).
 *   weights  host doubles, copied at setup.  For each level, for each
 *            layer: W in PyTorch Conv layout [Cout][Cin][k] (1D) or
 *            [Cout][Cin][k][k] (2D), then bias [Cout].
 *   level_layers  CNN only, optional: nlevels layer counts, one per smoother
 *            level (2..16; 3..16 in the refinement precisions), read at
 *            setup; NULL = `layers` on every level.  The paper sizes each
 *            level's network separately (Appendix A, Table 6: more layers
 *            and wider kernels on some grids); a deeper net widens the
 *            receptive field where the level's operator needs it.
 *   nweights total number of doubles in `weights` (checked).
 *   arch     NMG_SMOOTHER_CNN (0, the above) or NMG_SMOOTHER_FNO (1).
 *   modes    FNO only: m, the retained modes per axis (the half spectrum of
 *            the real 2D DFT with k1 in [0, m) and [n-m, n), k2 in [0, m);
 *            1 <= m <= 32 and 2m <= the smallest smoother level's side).
 * FNO (2D, precisions NMG_FP64 / NMG_FP32): a pointwise lift 1 -> width,
 * `layers` Fourier layers z <- ReLU(W * z + B + DFT^-1(R . DFT(z))) with W a
 * ksize x ksize 'same' convolution (odd ksize <= 7), and a pointwise
 * projection width -> 1 (width <= 64).  Weights per level, in this order:
 * lift W [width], lift b [width]; per layer W [width][width][ksize][ksize],
 * b [width], Re R [2][width][width][m][m], Im R [2][width][width][m][m]
 * ([block][in][out][k1][k2], block 0: k1 = 0..m-1, block 1: k1 =
 * n-m..n-1); projection W [width], b [1].
 */
typedef struct {
  int layers;
  int width;
  int ksize;
  int nlevels;
  const double* weights;
  size_t nweights;
  int arch;
  int modes;
  const int* level_layers;
} nmg_smoother_desc;

typedef struct {
  int cycles;     /* cycles applied before the tolerance was met */
  int status;     /* NMG_CONVERGED / NMG_NOT_CONVERGED / NMG_DIVERGED */
  double relres;  /* final ||f - A u|| / ||f|| (fp64 norm) */
} nmg_solve_info;

/* Create a context on CUDA device `device`.  stream: a cudaStream_t to
 * order work on, or NULL for a library-owned stream that is ordered after
 * work queued on the legacy default stream. */
nmg_status nmg_create(nmg_ctx** ctx, int device, void* stream);
void nmg_destroy(nmg_ctx* ctx);

/* Build the hierarchy (host fp64 Galerkin products, device fp64 Cholesky
 * of the coarsest operator, filter twiddles, packed weights).  Errors:
 * NMG_ERR_ARG, NMG_ERR_WEIGHTS, NMG_ERR_NOT_SPD, NMG_ERR_OOM, NMG_ERR_CUDA. */
nmg_status nmg_setup(nmg_ctx* ctx, const nmg_operator_desc* op,
                     const nmg_smoother_desc* sm, nmg_hier** out);
void nmg_destroy_hier(nmg_hier* h);

/* Solve A u = f for `batch` right-hand sides on the device.  u holds the
 * initial guess on entry (zeros for the paper's x^0 = 0) and the solution on
 * return.  A right-hand side stops receiving cycles once its relative
 * residual is <= rtol.  info: host array [batch] or NULL.  Synchronous. */
nmg_status nmg_solve(nmg_ctx* ctx, nmg_hier* h, int batch, const void* f, void* u,
                     double rtol, int max_cycles, nmg_solve_info* info);

/* ---- classical comparators (the paper's comparison columns) -----------
 * Both run on a hierarchy of precision NMG_FP64 or NMG_FP32 (f and u in
 * that type; NMG_ERR_UNSUPPORTED otherwise), with its operators, transfers
 * and coarsest Cholesky solve, from the caller's u (zeros for x^0 = 0), and
 * stop a right-hand side once ||f - A u|| / ||f|| <= rtol.  Synchronous;
 * info as for nmg_solve (cycles = V-cycles or CG iterations).
 *
 * nmg_solve_mg_jacobi: x^tau = MG(x^{tau-1}, f) with the V-cycle of
 * Algorithm 1 (nu1 pre- and nu2 post-smoothing steps per level; the paper's
 * comparator is the backslash cycle nu1 = 5, nu2 = 0, Section 4.1) and the
 * weighted Jacobi smoother of Section 2.2, x <- x + omega_l D_l^{-1}
 * (y - A_l x).  The paper does not print omega for this comparator; each
 * level uses omega_l = 1 / max_i (sum_j |A_l[i][j]|) / A_l[i][i], the
 * reciprocal of a Gershgorin bound on the largest eigenvalue of
 * D_l^{-1} A_l (a fixed omega = 1/2 diverges on blur operators, whose
 * diagonal is small against their largest eigenvalue).  nu1 + nu2 <= 64.
 *
 * nmg_solve_cg: conjugate gradients on A_1 u = f (no preconditioner, as in
 * Section 4.2); the stopping test uses the recurred residual r_k.
 * max_iters bounds the iterations. */
nmg_status nmg_solve_mg_jacobi(nmg_ctx* ctx, nmg_hier* h, int batch, const void* f, void* u,
                               double rtol, int max_cycles, int nu1, int nu2,
                               nmg_solve_info* info);
nmg_status nmg_solve_cg(nmg_ctx* ctx, nmg_hier* h, int batch, const void* f, void* u, double rtol,
                        int max_iters, nmg_solve_info* info);

/* One batch of one hierarchy inside a multi-hierarchy solve. */
typedef struct {
  nmg_hier* hier;        /* hierarchy of this item (each at most once per call) */
  int batch;             /* right-hand sides of this item (0 = skip) */
  const void* f;         /* device, [batch][n][n] (or [batch][n]) of the hierarchy's f type */
  void* u;               /* device, in/out, the hierarchy's u type */
  nmg_solve_info* info;  /* host array [batch] or NULL */
} nmg_solve_item;

/* Solve several batches on different hierarchies (grid sizes, operators,
 * precisions) together: one outer loop in which every iteration runs one
 * cycle and one convergence test for every item still active.  With graphs
 * enabled an iteration of all items is one CUDA graph whose items are
 * parallel branches, so small grids share the device.  Each item gets the
 * same results as nmg_solve on it alone.  Synchronous. */
nmg_status nmg_solve_multi(nmg_ctx* ctx, int nitems, const nmg_solve_item* items, double rtol,
                           int max_cycles);

/* Same as nmg_solve with HOST f and u: the library copies f (and u) to its
 * own device buffers, solves, and copies u back.  Host buffers may be
 * pageable or pinned.  Synchronous. */
nmg_status nmg_solve_host(nmg_ctx* ctx, nmg_hier* h, int batch, const void* f_host,
                          void* u_host, double rtol, int max_cycles,
                          nmg_solve_info* info);

/* nmg_solve_host from the zero initial guess x^0 = 0 of the outer loop
 * (Section 3.2: x^0 = 0, then Algorithms 3/4): u_host is output only
 * ([batch][n][n] (2D) or [batch][n], fp64 in the FP64 and refinement
 * precisions, fp32 in FP32); it is not read, and only f is copied to the
 * device.  Errors as nmg_solve_host.  Synchronous. */
nmg_status nmg_solve_host_zero(nmg_ctx* ctx, nmg_hier* h, int batch, const void* f_host,
                               void* u_host, double rtol, int max_cycles,
                               nmg_solve_info* info);

/* Exactly one cycle u <- NMGF(u, f) at the finest level for every
 * right-hand side (no convergence test).  Asynchronous. */
nmg_status nmg_cycle(nmg_ctx* ctx, nmg_hier* h, int batch, const void* f, void* u);

/* ---- serving: continuous batching over resident hierarchies ---------------
 * A server keeps every added operator's hierarchy resident and gives it a
 * pool of `slots` right-hand-side positions.  Requests are queued on the
 * host; each nmg_server_step() admits queued requests (arrival order) into
 * free slots of their operator, runs one outer iteration (one cycle and one
 * convergence test) for every live request of every operator, and retires
 * requests that converged (relative residual <= rtol), diverged or used
 * max_cycles cycles, copying u to the caller's buffer.  Each slot is
 * computed independently: a request's result does not depend on the other
 * requests in flight.  The server does not own the hierarchies. */
typedef struct nmg_server nmg_server;
/* budget_bytes bounds the device memory of all slot pools and their
 * workspaces (0: no bound beyond the device's free memory). */
nmg_status nmg_server_create(nmg_ctx* ctx, size_t budget_bytes, double rtol, int max_cycles,
                             nmg_server** out);
void nmg_server_destroy(nmg_server* s);
/* Make hierarchy h servable with up to `slots` concurrent requests.  The
 * pool (slot buffers for f and u and the hierarchy's workspace) starts with
 * min(slots, 4) slots and grows by doubling, up to `slots`, when requests
 * wait for it at a scheduler step -- each growth only if the device's free
 * memory at that moment (cudaMemGetInfo, less a reserve of max(256 MiB,
 * 1/64 of the device)) and the budget allow it; otherwise the requests stay
 * queued until slots free up (admission bounded by free HBM).  Growth keeps
 * the live requests in their slots.  NMG_ERR_OOM if not even the first
 * slots fit.  op_id: returned handle. */
nmg_status nmg_server_add_operator(nmg_server* s, nmg_hier* h, int slots, int* op_id);
/* Queue one right-hand side (host, the operator's f type, copied now); u_host
 * (host, the operator's u type) receives the solution when the request is
 * retired and must stay valid until then.  req_id: returned handle. */
nmg_status nmg_server_submit(nmg_server* s, int op_id, const void* f_host, void* u_host,
                             long long* req_id);
/* One scheduler step (synchronous); completed: requests retired by it. */
nmg_status nmg_server_step(nmg_server* s, int* completed);
/* state: 0 queued, 1 running, 2 done; times in seconds since server creation. */
nmg_status nmg_server_query(nmg_server* s, long long req_id, nmg_solve_info* info, int* state,
                            double* t_submit, double* t_admit, double* t_done);
nmg_status nmg_server_stats(const nmg_server* s, int* queued, int* running, size_t* bytes_used);

/* ---- single steps of the cycle (level is 0-based: 0 is the paper's l=1) --
 * Vectors are the hierarchy's level type (see above).  Asynchronous unless
 * a host output is requested. */

/* r = y - A_l x.  norms: host double[batch] receiving ||r||_2, or NULL. */
nmg_status nmg_residual(nmg_ctx* ctx, nmg_hier* h, int level, int batch,
                        const void* x, const void* y, void* r, double* norms);
/* yc = I_l^{l+1} (y - A_l x), yc on level l+1 (Algorithm 4, restriction). */
nmg_status nmg_residual_restrict(nmg_ctx* ctx, nmg_hier* h, int level, int batch,
                                 const void* x, const void* y, void* yc);
/* h = N_l(b / ||b||) ||b||, h = 0 where ||b|| = 0 (level < levels-1). */
nmg_status nmg_smooth(nmg_ctx* ctx, nmg_hier* h, int level, int batch,
                      const void* b, void* hout);
/* x = x* + F'_l(h) (filter on) or x* + h (filter off); xstar may be NULL
 * (zero) and may alias x. */
nmg_status nmg_filter_update(nmg_ctx* ctx, nmg_hier* h, int level, int batch,
                             const void* xstar, const void* hin, void* x);
/* x = (A^(L))^{-1} y on the coarsest level (fp64 Cholesky solve). */
nmg_status nmg_coarse_solve(nmg_ctx* ctx, nmg_hier* h, int batch, const void* y, void* x);
/* x += I_{l+1}^l e, e on level l+1, x on level l. */
nmg_status nmg_prolong_correct(nmg_ctx* ctx, nmg_hier* h, int level, int batch,
                               const void* e, void* x);

/* ---- residual step without device allocation ---------------------------
 * The paper has no counterpart: this entry point serves callers that must
 * not allocate device memory at call time.  nmg_residual above may grow the
 * hierarchy's workspace with cudaMalloc the first time it sees a larger
 * batch, and cudaMalloc / cudaFree can stall every stream on the device or
 * fail outright in a process whose device memory has been reserved up front
 * by a pooling allocator (a framework's caching allocator, a serving arena
 * with a fixed, audited footprint).  Such callers use this variant.
 *
 * It computes exactly what nmg_residual computes, with the same kernels:
 * r = y - A_l x on `level` for `batch` right-hand sides (vectors of the
 * hierarchy's level type, device memory, x and y unchanged, r caller-owned)
 * and, if norms is not NULL, ||r||_2 per right-hand side into the host
 * array norms[batch] (the call then waits for the context's stream).
 *
 * Its scratch (per-tile partial sums of r^2, the norms before they are
 * copied out, and the active flags) lives in one array of
 * NMG_NOALLOC_SCRATCH_BYTES bytes compiled into the library, one per
 * device.  The call allocates no device memory, calls no cudaMalloc or
 * cudaFree, and is not recorded by the nmg_profile_* timing (which creates
 * events); nmg_launch_count counts its launches.
 *   - Size limit: the call needs 4 B per right-hand side for the flags,
 *     8 B per right-hand side and residual tile for the partial sums and
 *     8 B per right-hand side for the norms, each part rounded up to 256 B;
 *     beyond NMG_NOALLOC_SCRATCH_BYTES it returns NMG_ERR_ARG before any
 *     launch, and nmg_last_error states the bytes needed and the limit.
 *     (At 512 x 512 with 64 x 64 residual tiles, 64 per image, that is
 *     about 2,000 right-hand sides; nmg_autotune may pick other tiles.)
 *   - Set-up: the first call on a device, with the context's device made
 *     current, looks up the array's device address once; later calls reuse
 *     it for the life of the process (a cudaDeviceReset of that device,
 *     which also invalidates every context and hierarchy of this library,
 *     ends its use).  Make that first call before any stream capture.
 *   - Sharing: every call on a device uses the same array.  Each call writes
 *     everything it reads back from it (nothing has to start at zero), but
 *     calls whose work overlaps on the GPU (other streams, other contexts on
 *     the same device, other host threads) race on the array and corrupt
 *     each other's norms; serialise them.
 * Errors: NMG_ERR_ARG (null pointers, level, batch, size limit),
 * NMG_ERR_CUDA. */
#define NMG_NOALLOC_SCRATCH_BYTES (1u << 20)
nmg_status nmg_residual_noalloc(nmg_ctx* ctx, nmg_hier* h, int level, int batch,
                                const void* x, const void* y, void* r, double* norms);

/* ---- inspection ------------------------------------------------------- */
/* Level side length, band half-widths and precision. */
nmg_status nmg_hier_info(const nmg_hier* h, int level, int* n, int* wK, int* wM,
                         int* precision);
/* Copy the level operator's 1D factors to host in dense form:
 * 2D: K_l and M_l, each n_l x n_l row-major (M may be NULL);
 * 1D: A_l (n_l x n_l) into K (M unused). */
nmg_status nmg_hier_level_dense(const nmg_hier* h, int level, double* K, double* M);

/* The Galerkin hierarchy of an operator description built on the host only
 * (no context, no device memory, no GPU needed): the same fp64 banded
 * products nmg_setup uses (A_{l+1} = R A_l P with R = P^T / 2 per axis,
 * Algorithms 3/4; 2D as K_{l+1} = R K_l P and M_{l+1} = R M_l P, Section
 * 4.2).  Writes the side n_l of level `level` (0 = finest), the band
 * half-widths of K_l and M_l (2D; -1 in 1D), and, where K is not NULL,
 * the level's factors in dense row-major form exactly as
 * nmg_hier_level_dense does (2D: K_l and M_l, n_l x n_l each, M may be
 * NULL; 1D: A_l into K).  Host pointers; any of n, wK, wM may be NULL.
 * NMG_ERR_ARG for an invalid description (the checks of nmg_setup on the
 * operator) or a level outside [0, levels). */
nmg_status nmg_host_level_dense(const nmg_operator_desc* op, int level, int* n, int* wK,
                                int* wM, double* K, double* M);

/* Number of kernels the library launched on this context so far. */
long long nmg_launch_count(const nmg_ctx* ctx);

/* Per-kernel-class timing.  nmg_profile_enable(ctx, 1) clears previous
 * records and starts recording a pair of CUDA events on the context's stream
 * around every launch; 0 stops recording (records are kept).
 * nmg_profile_read synchronises the stream and reports, for one class, the
 * number of recorded launches, their summed device time in milliseconds and
 * the summed work units (grid points x active right-hand sides; 0 for
 * bookkeeping kernels).  Classes: */
enum {
  NMG_K_RESIDUAL = 0,         /* r = y - A x (banded 2D / dense 1D) */
  NMG_K_RESTRICT = 1,         /* R (y - A x) fused */
  NMG_K_CNN_FIRST = 2,        /* first conv layer (2D SIMT) */
  NMG_K_CNN_HIDDEN = 3,       /* hidden conv layers (2D SIMT) */
  NMG_K_CNN_LAST = 4,         /* last conv layer (2D SIMT) */
  NMG_K_FILTER = 5,           /* output filter passes */
  NMG_K_COARSE = 6,           /* coarsest triangular solves */
  NMG_K_PROLONG = 7,          /* prolongation + correction */
  NMG_K_REFINE_RESIDUAL = 8,  /* compensated outer residual */
  NMG_K_OTHER = 9,            /* norms, convergence flags, updates */
  NMG_K_CNN_FUSED = 10        /* fused smoother (bf16 tensor cores, 1D) */
};
nmg_status nmg_profile_enable(nmg_ctx* ctx, int enable);
nmg_status nmg_profile_read(nmg_ctx* ctx, int kind, long long* launches, double* ms,
                            double* units);
/* Autotuner: for every level of a 2D hierarchy, time the candidate launch
 * shapes (tile sides of the residual, the fused residual + restriction and
 * the compensated outer residual, and on levels with a wide Toeplitz
 * stencil the strip kernels with k row chunks per 64-column strip; output
 * filter as three passes (mode 0),
 * one block-synchronous kernel (1), one warp-level kernel for 64x64 and
 * 128x128 levels (2), or three warp-level passes for 256x256 and 512x512
 * levels (3)) on the hierarchy's workspace with `batch`
 * right-hand sides, and
 * keep the fastest for later solves.  cache_path (may be NULL): a text file
 * from which choices for the same operator shape, precision and batch are
 * read instead of timed, and to which new choices are appended.  No effect
 * on results beyond fp rounding order. */
nmg_status nmg_autotune(nmg_ctx* ctx, nmg_hier* h, int batch, const char* cache_path);
/* The launch choices of one level (0 / -1: built-in defaults).  A tile
 * choice t > 0 is a tile side; t <= 0 selects the strip kernel where the
 * level has one, with -t row chunks per strip (0: the kernel's own choice
 * from its occupancy model). */
nmg_status nmg_hier_tuning(const nmg_hier* h, int level, int* res_tile, int* rst_tile,
                           int* ref_tile, int* filt_mode);

/* Solve loops replay one captured CUDA graph per outer iteration (cycle +
 * convergence test; captured on first use for a given batch, f, u and
 * rtol).  enable = 0 launches every kernel eagerly instead.  Profiling
 * (nmg_profile_enable) always launches eagerly.  Default: enabled. */
nmg_status nmg_set_graphs(nmg_ctx* ctx, int enable);

/* Bound of every device-side wait of the tensor-core kernels (mbarrier
 * waits between their copy, MMA and epilogue roles), in nanoseconds; 2 s by
 * default.  A launch whose wait runs out stops its roles, lets the copies
 * and MMAs it already issued complete, releases its tensor memory and
 * returns; the solve that ran it stops after that iteration and returns
 * NMG_ERR_TIMEOUT (the context and hierarchy stay usable).  Read by the
 * kernels at launch, so it also applies to already captured graphs.
 * Synchronous.  NMG_ERR_ARG if ns <= 0. */
nmg_status nmg_set_wait_limit(nmg_ctx* ctx, long long ns);

/* Failure-injection hook for tests (the paper has no counterpart): while
 * enable != 0, the MMA issuers of every warp-specialised tensor-core
 * smoother launch on this context (levels of side >= 32 in the refinement
 * precisions) first wait on a barrier that nothing arrives at, so each
 * launch ends by the wait limit above and the solve reports NMG_ERR_TIMEOUT.
 * No fault is raised on the device.  Synchronous. */
nmg_status nmg_inject_stall(nmg_ctx* ctx, int enable);

/* Wait for the context's stream. */
nmg_status nmg_sync(nmg_ctx* ctx);
const char* nmg_status_str(nmg_status s);
const char* nmg_last_error(const nmg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* NMG_H */
