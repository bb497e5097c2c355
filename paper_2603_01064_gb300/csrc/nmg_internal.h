// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/nmg.h"

namespace nmg {

// ---------------------------------------------------------------------------
// host-side hierarchy (fp64), built once per operator
// ---------------------------------------------------------------------------

// One level's operator.  2D: A_l = alpha M_l (x) M_l + K_l (x) K_l with K_l,
// M_l banded and stored as DIA rows: Kd[i*(2wK+1) + d] = K_l[i][i+d-wK]
// (zero where the column is outside [0, n)).  1D: dense A_l (n x n).
struct HostLevel {
  int n = 0;
  int wK = 0;
  int wM = 0;
  std::vector<double> Kd, Md;  // 2D
  std::vector<double> A;       // 1D dense
};

struct HostHierarchy {
  int dim = 0, n = 0, levels = 0;
  double alpha = 0;
  std::vector<HostLevel> lv;
  std::vector<double> coarse;  // dense nc x nc coarsest operator
  int nc = 0;
};

// Builds the Galerkin hierarchy; returns false with a message on bad input.
bool build_host_hierarchy(const nmg_operator_desc& op, HostHierarchy& H, std::string& err);

// Filter helpers (fp64, host): sqrt(2k/n) for folded bin k = 0..n/2 and the
// first column of the 1D circulant filter Re(IDFT(m' . DFT(.))).
std::vector<double> filter_mask_table(int n);
std::vector<double> filter_circulant_1d(int n);
// twiddles exp(-2 pi i k / n), k = 0..n/2-1, interleaved (re, im)
std::vector<double> fft_twiddles(int n);

// ---------------------------------------------------------------------------
// device-side views passed to kernels by value
// ---------------------------------------------------------------------------

template <typename T>
struct StencilHost;

template <typename T>
struct Band2D {
  int n, wK, wM;
  const T* Kd;
  const T* Md;
  T alpha;
  const StencilHost<T>* st = nullptr;  // stencil form of Kd/Md (host), if any
};

// Stencil form of a level's banded factors, found on the host at setup: the
// rows g >= nbK of K_l are one stencil sK (offsets -wK..wK), the first nbK
// rows differ from it by the correction rows cK[g][0..2wK] (device), and
// likewise for M_l (wM <= 1).  With x zero outside the grid this reproduces
// K_l x exactly.  The fine level is Toeplitz (nb = 0); Galerkin levels
// differ from their stencil only in the first rows (the coarse node J sits
// on fine node 2J, so only the low boundary sees the zero phantom).
constexpr int kStencilMaxW = 32;
template <typename T>
struct StencilHost {
  int valid = 0;
  int wK = 0, wM = 0, nbK = 0, nbM = 0;
  T sK[2 * kStencilMaxW + 1] = {};
  T sM[3] = {};
  const T* cK = nullptr;
  const T* cM = nullptr;
};
// stencil form of a DIA factor (n rows, half-width w): stencil s[2w+1], the
// number nb of leading rows that differ and their corrections corr[nb][2w+1];
// false if another row differs or there is no interior row
bool stencil_form(const std::vector<double>& dia, int n, int w, std::vector<double>& s, int& nb,
                  std::vector<double>& corr);

// weights of one 2D conv layer: w[(ci*9 + tap)*cout + co], bias[co]
template <typename T>
struct ConvW {
  const T* w;
  const T* b;
};

// kernel classes for the optional per-class event timing (nmg_profile_*)
enum KernelKind {
  K_RESIDUAL = 0, K_RESTRICT = 1, K_CNN_FIRST = 2, K_CNN_HIDDEN = 3, K_CNN_LAST = 4,
  K_FILTER = 5, K_COARSE = 6, K_PROLONG = 7, K_REFINE_RESIDUAL = 8, K_OTHER = 9,
  K_CNN_FUSED = 10, K_NKINDS = 11
};

// launch counter and, when profiling is on, CUDA-event records around each
// launch on the launching stream (events come from a reusable pool)
struct ProfRec {
  int kind;
  cudaEvent_t a, b;
  double units;
};
struct LaunchLog {
  long long launches = 0;
  bool prof = false;
  double active_hint = 0;  // right-hand sides currently active (host view)
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  cudaEvent_t get_event() {
    if (pool_used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[pool_used++];
  }
  int begin(int kind, cudaStream_t st) {
    ++launches;
    if (!prof) return -1;
    ProfRec r{kind, get_event(), get_event(), 0.0};
    cudaEventRecord(r.a, st);
    recs.push_back(r);
    return (int)recs.size() - 1;
  }
  void end(int idx, cudaStream_t st, double units) {
    if (idx < 0) return;
    cudaEventRecord(recs[idx].b, st);
    recs[idx].units = units;
  }
};

inline int ceil_div(int a, int b) { return (a + b - 1) / b; }
inline int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

// ---------------------------------------------------------------------------
// kernel launchers (implemented in k_*.cu); every launcher enqueues on `st`
// and adds the number of kernels it launched to `log`.
// `active` is a device int[B]: right-hand sides with active[b] == 0 are
// skipped (their outputs are left untouched).
// ---------------------------------------------------------------------------

// stencil form of the level residual (and residual + restriction): the
// fine-level strip kernel or the persistent pipelined tile kernel; false if
// the level has no stencil form or is not staged that way (the caller then
// launches the generic kernel).  *nparts: partial sums per right-hand side.
template <typename T, bool RESTRICT>
bool launch_stencil_residual(const Band2D<T>& op, int B, const T* x, const T* y, T* out,
                             double* partials, const int* active, int tile, int ntx,
                             cudaStream_t st, int* nparts);
// partial sums per right-hand side of the fine-level strip form (0 if the
// level does not use it)
template <typename T>
int stencil_strip_parts(const Band2D<T>& op);

// wide PSF stencils (k_wide.cu): the fp32 fine-level residual for Toeplitz K
// of half-width 9..32 with M = I and n a multiple of 128 (16-byte aligned
// vectors), as a strip kernel; returns the partial sums written per
// right-hand side.  The full-weighting restriction of a fine residual r
// into yc (n a multiple of 128), with the squared norms per unit.
bool wide_residual_applies(const Band2D<float>& op, const float* x, const float* y);
// kch: chunks per 64-column strip (<= 0: wide_chunks' choice); returns the
// partial sums written per right-hand side
int launch_residual_wide(const Band2D<float>& op, int B, const float* x, const float* y, float* r,
                         double* partials, const int* active, int kch, cudaStream_t st);
bool restrict_fw_applies(int n);
// classical comparators (k_classic.cu): x += omega r / diag(A_l), and one
// conjugate-gradient iteration after q = -A p (scal: (r, r), alpha, beta)
template <typename T>
void launch_jacobi2d(const Band2D<T>& op, int B, T* x, const T* r, double omega, const int* active,
                     cudaStream_t st, LaunchLog& log);
template <typename T>
void launch_jacobi1d(int n, const T* A, int B, T* x, const T* r, double omega, const int* active,
                     cudaStream_t st, LaunchLog& log);
template <typename T>
void launch_cg_iteration(long long len, int B, T* u, T* r, T* p, const T* q, double* scal,
                         double* s, double* partials, const int* active, cudaStream_t st,
                         LaunchLog& log);
void launch_cg_init(int B, const double* s, double* scal, const int* active, cudaStream_t st,
                    LaunchLog& log);
int launch_restrict_fw(int n, int B, const float* r, float* yc, double* partials, const int* active,
                       cudaStream_t st);

// r = y - A x on a 2D level (+ per-tile partial sums of r^2 if partials)
// tile_req: requested tile side (0 = default), see pick_tile
template <typename T>
void launch_residual2d(const Band2D<T>& op, int B, const T* x, const T* y, T* r,
                       double* partials, int* ntiles, const int* active, cudaStream_t st,
                       LaunchLog& log, int tile_req = 0);
// number of partial sums per right-hand side the two residual launchers write
template <typename T>
int residual2d_tiles(const Band2D<T>& op, int tile_req);
int residual1d_tiles(int n);
// yc = R (y - A x) on a 2D level (+ partial sums of yc^2)
template <typename T>
void launch_residual_restrict2d(const Band2D<T>& op, int B, const T* x, const T* y, T* yc,
                                double* partials, int* ntiles, const int* active,
                                cudaStream_t st, LaunchLog& log, int tile_req = 0);
// x += P e (2D)
template <typename T>
void launch_prolong2d(int n, int B, const T* e, T* x, const int* active, cudaStream_t st,
                      LaunchLog& log);

// 1D dense variants
template <typename T>
void launch_residual1d(int n, const T* A, int B, const T* x, const T* y, T* r,
                       double* partials, int* ntiles, const int* active, cudaStream_t st,
                       LaunchLog& log);
template <typename T>
void launch_restrict1d(int n, int B, const T* r, T* yc, double* partials, int* ntiles,
                       const int* active, cudaStream_t st, LaunchLog& log);
template <typename T>
void launch_prolong1d(int n, int B, const T* e, T* x, const int* active, cudaStream_t st,
                      LaunchLog& log);

// s[b] = sqrt(sum_t partials[b*ntiles + t])
void launch_norms(const double* partials, int ntiles, int B, double* s, const int* active,
                  cudaStream_t st, LaunchLog& log);
// partial sums of v^2 for a plain vector batch of `len` elements per item
template <typename T>
void launch_sumsq(const T* v, long long len, int B, double* partials, int* ntiles,
                  const int* active, cudaStream_t st, LaunchLog& log);
// relres = s / fn; deactivate converged (<= rtol) or diverged items;
// cycles[b] += 1 for items still active after the test if count_cycle.
void launch_converge(const double* s, const double* fn, double rtol, int B, int* active,
                     double* relres, int* status, int* nactive, cudaStream_t st,
                     LaunchLog& log);

// CNN smoother (SIMT), 2D: h = s * N(b / s)
// FNO smoother (k_fno.cu): dimensions shared by every smoother level
struct FnoDims {
  int width, layers, ksize, modes;
};
size_t fno_weights_per_level(int c, int layers, int ks, int m);
// Strip kernels of wide stencils (half-width W): a strip of n rows is cut
// into kch chunks of ceil(n / kch) rows, each one warp's unit, at the cost
// of 2W halo rows per chunk.  The launch puts min(units, sms) blocks of nw
// warps on the GPU (one block per SM: the warps' rings fill its shared
// memory) and deals the units to them block-cyclically.  The warps are
// latency-bound (measured: a row step takes about as long with 4 warps on
// the SM as with 9), so one SM's time is (waves of nw units) x (rows per
// unit): wide_chunks picks the chunk count (chunks of at least
// kWideChunkMinH rows) that minimises ceil(ceil(units / sms) / nw) x
// (ceil(n / k) + 2W), the larger count on ties.
constexpr int kWideChunkMinH = 32;
// partial-sum slots of one right-hand side in a hierarchy's workspace
constexpr int kMaxPartsPerItem = 4096;
// the largest chunk count a launch may use: chunks of >= kWideChunkMinH
// rows and at most kMaxPartsPerItem units (partial sums) per right-hand side
inline int wide_chunks_max(int n) {
  int k = n / kWideChunkMinH;
  const int cap = kMaxPartsPerItem / (n / 64 > 0 ? n / 64 : 1);
  if (k > cap) k = cap;
  return k < 1 ? 1 : k;
}
inline int wide_chunks(int n, int W, long long strips, int sms, int nw) {
  int best_k = 1;
  long long best = -1;
  for (int k = 1; k <= wide_chunks_max(n); ++k) {
    const long long units = strips * k;
    const long long u = (units + sms - 1) / sms;
    const long long waves = (u + nw - 1) / nw;
    const long long cost = waves * ((n + k - 1) / k + 2 * W);
    if (best < 0 || cost <= best) {
      best = cost;
      best_k = k;
    }
  }
  return best_k;
}

// CNN smoother: the most layers one level may have, and the doubles of one
// level's weights (PyTorch layout, channels 1 -> width -> ... -> 1)
constexpr int kMaxCnnLayers = 16;
inline size_t cnn_weights_per_level(int layers, int width, int ksize, int dim) {
  const size_t kk = dim == 1 ? (size_t)ksize : (size_t)ksize * ksize;
  size_t n = 0;
  for (int i = 0; i < layers; ++i) {
    const size_t cin = i == 0 ? 1 : width, cout = i == layers - 1 ? 1 : width;
    n += cout * cin * kk + cout;
  }
  return n;
}
// h = N_FNO(b / s) s on an n x n level; wts: the level's weights in the
// nmg_smoother_desc layout (type T); tw: e^{-2 pi i j / n}, j < n, as (re, im)
// pairs; z0, z1: [B][width][n][n]; cA: [B][width][n][modes] complex;
// cB: 2 x [B][width][2 modes][modes] complex
template <typename T>
void launch_fno2d(const FnoDims& dm, int n, int B, const T* wts, const T* tw, const T* b,
                  const double* s, T* z0, T* z1, T* cA, T* cB, T* h, const int* active,
                  cudaStream_t st, LaunchLog& log);

template <typename T>
void launch_cnn2d_simt(int n, int B, int layers, int width, const ConvW<T>* layers_w,
                       const T* b, const double* s, T* act0, T* act1, T* h, const int* active,
                       cudaStream_t st, LaunchLog& log);
// CNN smoother, 1D, all layers fused: weights packed per layer as
// w[(co*cin + ci)*k + t] then bias
template <typename T>
void launch_cnn1d(int n, int B, int layers, int width, int ksize, const T* wpacked,
                  const T* b, const double* s, T* h, const int* active, cudaStream_t st,
                  LaunchLog& log);

// filter: x = xstar + F'(h) (2D FFT passes); xstar may be null; x may alias xstar
// mode: -1 default (single kernel when the complex image fits in shared
// memory), 0 three passes, 1 single kernel (if it fits)
template <typename T>
void launch_filter2d(int n, int B, const T* xstar, const T* h, T* x, void* cbuf,
                     const T* twiddles, const double* mask_tab, const int* active,
                     cudaStream_t st, LaunchLog& log, int mode = -1);
template <typename T>
void launch_filter1d(int n, int B, const T* xstar, const T* h, T* x, const double* circ,
                     const int* active, cudaStream_t st, LaunchLog& log);
// x = xstar + h (filter off)
template <typename T>
void launch_axpy_update(long long len, int B, const T* xstar, const T* h, T* x,
                        const int* active, cudaStream_t st, LaunchLog& log);

// coarse: in-place Cholesky of an nc x nc fp64 matrix (device); flag set to
// 1 if a pivot is not positive
void launch_cholesky(int nc, double* A, int* flag, cudaStream_t st, LaunchLog& log);
// L^{-1} and its transpose from the Cholesky factor (setup)
void launch_chol_inverse(int nc, const double* L, double* Li, double* LiT, cudaStream_t st,
                         LaunchLog& log);
// x = L^{-T} L^{-1} y for B right-hand sides (fp64 arithmetic)
template <typename T>
void launch_coarse_solve(int nc, const double* Li, const double* LiT, int B, const T* y, T* x,
                         const int* active, cudaStream_t st, LaunchLog& log);

// active[b] = 1 where newmask[b] (serving admission)
void launch_admit(int B, const int* newmask, int* active, cudaStream_t st, LaunchLog& log);

// cycles[b] += 1 for active items
void launch_count_cycles(int B, const int* active, int* cycles, cudaStream_t st, LaunchLog& log);

// fp64 helpers for the refinement form
// u += d (u fp64, d float)
void launch_update_f64(long long len, int B, const float* d, double* u, const int* active,
                       cudaStream_t st, LaunchLog& log);

}  // namespace nmg
