// Operator kernels of the cycle:
//  * residual r = y - A_l x for A_l = alpha M(x)M + K(x)K with banded 1D
//    factors (Algorithm 4: B_l = Y_l - Mat(A Vec(X*)) and the residual
//    before restriction), as two separable passes over a shared-memory tile
//    (the generic DIA form; levels in stencil form run the pipelined kernel
//    of k_stencil.cuh);
//  * the same residual followed by full-weighting restriction
//    R = (P(x)P)^T / 4, writing only the coarse vector;
//  * prolongation + correction X_l += Mat(I_{l+1}^l Vec(E_{l+1}));
//  * per-tile partial sums of squares for the residual norms ||B_l||.
// The 1D variants use a dense level matrix (Algorithm 3).
#include <cmath>

#include "nmg_internal.h"

namespace nmg {

namespace {

constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ double block_sum(double v, double* red) {
  // warp shuffle then one value per warp in shared memory
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) s += red[i];  // fixed order: deterministic
  }
  return s;
}

// Fine region handled by one block: rows [r0, r0+RH), cols [c0, c0+RW).
// Shared memory: xs (RH+2W) x (RW+2W), tk (RH+2wK) x RW, tm (RH+2wM) x RW,
// rs RH x RW (restrict only).  W = max(wK, wM).
template <typename T, bool RESTRICT>
__global__ void __launch_bounds__(kThreads)
k_residual2d(Band2D<T> op, const T* __restrict__ x, const T* __restrict__ y,
             T* __restrict__ out, double* __restrict__ partials, const int* __restrict__ active,
             int tile, int tiles_x) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  __shared__ double red[32];
  const int n = op.n, wK = op.wK, wM = op.wM;
  const int W = wK > wM ? wK : wM;
  const int ty = blockIdx.x / tiles_x, tx = blockIdx.x % tiles_x;
  int r0, c0, RH, RW, nc = n / 2, CH = 0, CW = 0;
  if (RESTRICT) {
    int I0 = ty * tile, J0 = tx * tile;
    CH = min(tile, nc - I0);
    CW = min(tile, nc - J0);
    r0 = 2 * I0 - 1;
    c0 = 2 * J0 - 1;
    RH = 2 * CH + 1;
    RW = 2 * CW + 1;
  } else {
    r0 = ty * tile;
    c0 = tx * tile;
    RH = min(tile, n - r0);
    RW = min(tile, n - c0);
  }
  const int XH = RH + 2 * W, XW = RW + 2 * W;
  const int nk = 2 * wK + 1, nm = 2 * wM + 1;
  T* xs = sm;
  T* tk = xs + XH * XW;
  T* tm = tk + (RH + 2 * wK) * RW;
  T* rs = tm + (RH + 2 * wM) * RW;
  // banded coefficients of the tile's columns (row pass) and rows (column pass)
  T* kcol = rs + (RESTRICT ? RH * RW : 0);
  T* mcol = kcol + RW * nk;
  T* krow = mcol + RW * nm;
  T* mrow = krow + RH * nk;
  const size_t plane = (size_t)n * n;
  const T* xb = x + (size_t)b * plane;
  const T* yb = y ? y + (size_t)b * plane : nullptr;

  for (int idx = threadIdx.x; idx < XH * XW; idx += blockDim.x) {
    int a = idx / XW, c = idx % XW;
    int gr = r0 - W + a, gc = c0 - W + c;
    xs[idx] = (gr >= 0 && gr < n && gc >= 0 && gc < n) ? xb[(size_t)gr * n + gc] : T(0);
  }
  for (int idx = threadIdx.x; idx < RW * nk; idx += blockDim.x) {
    int j = idx / nk, g = c0 + j;
    kcol[idx] = (g >= 0 && g < n) ? op.Kd[(size_t)g * nk + idx % nk] : T(0);
  }
  for (int idx = threadIdx.x; idx < RW * nm; idx += blockDim.x) {
    int j = idx / nm, g = c0 + j;
    mcol[idx] = (g >= 0 && g < n) ? op.Md[(size_t)g * nm + idx % nm] : T(0);
  }
  for (int idx = threadIdx.x; idx < RH * nk; idx += blockDim.x) {
    int i = idx / nk, g = r0 + i;
    krow[idx] = (g >= 0 && g < n) ? op.Kd[(size_t)g * nk + idx % nk] : T(0);
  }
  for (int idx = threadIdx.x; idx < RH * nm; idx += blockDim.x) {
    int i = idx / nm, g = r0 + i;
    mrow[idx] = (g >= 0 && g < n) ? op.Md[(size_t)g * nm + idx % nm] : T(0);
  }
  __syncthreads();
  // row pass: tk[a][j] = sum_d K[gj][gj+d-wK] x[row][gj+d-wK]
  // (coefficients of out-of-range columns are staged as zero)
  {
    const int HK = RH + 2 * wK, HM = RH + 2 * wM;
    for (int idx = threadIdx.x; idx < HK * RW; idx += blockDim.x) {
      int a = idx / RW, j = idx % RW;
      const T* kr = kcol + j * nk;
      const T* xr = xs + (a + W - wK) * XW + (j + W - wK);
      T acc = T(0);
      for (int d = 0; d < nk; ++d) acc += kr[d] * xr[d];
      tk[idx] = acc;
    }
    for (int idx = threadIdx.x; idx < HM * RW; idx += blockDim.x) {
      int a = idx / RW, j = idx % RW;
      const T* mr = mcol + j * nm;
      const T* xr = xs + (a + W - wM) * XW + (j + W - wM);
      T acc = T(0);
      for (int d = 0; d < nm; ++d) acc += mr[d] * xr[d];
      tm[idx] = acc;
    }
  }
  __syncthreads();
  // column pass and residual
  T ss = T(0);
  {
    for (int idx = threadIdx.x; idx < RH * RW; idx += blockDim.x) {
      int i = idx / RW, j = idx % RW;
      int gi = r0 + i, gj = c0 + j;
      T r = T(0);
      if (gi >= 0 && gi < n && gj >= 0 && gj < n) {
        const T* kr = krow + i * nk;
        const T* mr = mrow + i * nm;
        T zk = T(0), zm = T(0);
        for (int d = 0; d < nk; ++d) zk += kr[d] * tk[(i + d) * RW + j];
        for (int d = 0; d < nm; ++d) zm += mr[d] * tm[(i + d) * RW + j];
        T yv = yb ? yb[(size_t)gi * n + gj] : T(0);
        r = yv - (op.alpha * zm + zk);
        if (!RESTRICT) {
          out[(size_t)b * plane + (size_t)gi * n + gj] = r;
          ss += r * r;
        }
      }
      if (RESTRICT) rs[idx] = r;
    }
  }
  if (RESTRICT) {
    __syncthreads();
    const size_t cplane = (size_t)nc * nc;
    const int I0 = ty * tile, J0 = tx * tile;
    for (int idx = threadIdx.x; idx < CH * CW; idx += blockDim.x) {
      int ci = idx / CW, cj = idx % CW;
      int li = 2 * ci + 1, lj = 2 * cj + 1;  // local fine center
      const T* c = rs + li * RW + lj;
      T v = T(0.25) * (T(0.25) * c[-RW - 1] + T(0.5) * c[-RW] + T(0.25) * c[-RW + 1]) +
            T(0.5) * (T(0.25) * c[-1] + T(0.5) * c[0] + T(0.25) * c[1]) +
            T(0.25) * (T(0.25) * c[RW - 1] + T(0.5) * c[RW] + T(0.25) * c[RW + 1]);
      out[(size_t)b * cplane + (size_t)(I0 + ci) * nc + (J0 + cj)] = v;
      ss += v * v;
    }
  }
  if (partials) {
    double s = block_sum<T>((double)ss, red);
    if (threadIdx.x == 0) partials[(size_t)b * gridDim.x + blockIdx.x] = s;
  }
}

// X_l += I_{l+1}^l E: one thread per coarse node (I, J) adds its share to
// the 2 x 2 fine block (2I, 2J) .. (2I+1, 2J+1); coarse node J sits on fine
// node 2J, fine odd nodes interpolate linearly, the phantom node nc is zero.
template <typename T>
__global__ void k_prolong2d(int n, int B, const T* __restrict__ e, T* __restrict__ x,
                            const int* __restrict__ active) {
  const int nc = n / 2, cplane = nc * nc;
  const size_t plane = (size_t)n * n;
  for (int b = blockIdx.y; b < B; b += gridDim.y) {
    if (!active[b]) continue;
    const T* eb = e + (size_t)b * cplane;
    T* xb = x + (size_t)b * plane;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cplane; c += gridDim.x * blockDim.x) {
      const int I = c / nc, J = c - I * nc;
      const bool r = J + 1 < nc, d = I + 1 < nc;
      const T a = eb[c];
      const T c1 = r ? eb[c + 1] : T(0);
      const T c2 = d ? eb[c + nc] : T(0);
      const T c3 = (r && d) ? eb[c + nc + 1] : T(0);
      T* x0 = xb + (size_t)(2 * I) * n + 2 * J;
      x0[0] += a;
      x0[1] += T(0.5) * (a + c1);
      x0[n] += T(0.5) * (a + c2);
      x0[n + 1] += T(0.25) * ((a + c1) + (c2 + c3));
    }
  }
}

// ---- 1D dense ---------------------------------------------------------------

// r[b][i] = y[b][i] - sum_j A[i][j] x[b][j]; one warp per output row
template <typename T>
__global__ void k_residual1d(int n, const T* __restrict__ A, const T* __restrict__ x,
                             const T* __restrict__ y, T* __restrict__ r,
                             double* __restrict__ partials, const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int rows_per_block = nw;
  double ss = 0.0;
  int i = blockIdx.x * rows_per_block + wid;
  if (i < n) {
    const T* ar = A + (size_t)i * n;
    const T* xb = x + (size_t)b * n;
    T acc = T(0);
    for (int j = lane; j < n; j += 32) acc += ar[j] * xb[j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      T v = (y ? y[(size_t)b * n + i] : T(0)) - acc;
      r[(size_t)b * n + i] = v;
      ss = (double)v * (double)v;
    }
  }
  if (partials) {
    double s = block_sum<T>(ss, red);
    if (threadIdx.x == 0) partials[(size_t)b * gridDim.x + blockIdx.x] = s;
  }
}

template <typename T>
__global__ void k_restrict1d(int n, const T* __restrict__ r, T* __restrict__ yc,
                             double* __restrict__ partials, const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  __shared__ double red[32];
  const int nc = n / 2;
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  double ss = 0.0;
  if (I < nc) {
    const T* rb = r + (size_t)b * n;
    T lo = (2 * I - 1 >= 0) ? rb[2 * I - 1] : T(0);
    T v = T(0.25) * lo + T(0.5) * rb[2 * I] + T(0.25) * rb[2 * I + 1];
    yc[(size_t)b * nc + I] = v;
    ss = (double)v * (double)v;
  }
  if (partials) {
    double s = block_sum<T>(ss, red);
    if (threadIdx.x == 0) partials[(size_t)b * gridDim.x + blockIdx.x] = s;
  }
}

template <typename T>
__global__ void k_prolong1d(int n, int B, const T* __restrict__ e, T* __restrict__ x,
                            const int* __restrict__ active) {
  const int nc = n / 2;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * B; idx += gridDim.x * blockDim.x) {
    int b = idx / n, i = idx % n;
    if (!active[b]) continue;
    const T* eb = e + (size_t)b * nc;
    int I = i >> 1;
    T v = (i & 1) ? T(0.5) * (eb[I] + ((I + 1 < nc) ? eb[I + 1] : T(0))) : eb[I];
    x[idx] += v;
  }
}

// ---- norms, convergence -------------------------------------------------------

__global__ void k_norms(const double* __restrict__ partials, int ntiles, int B,
                        double* __restrict__ s, const int* __restrict__ active) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !active[b]) return;
  double acc = 0.0;
  for (int t = 0; t < ntiles; ++t) acc += partials[(size_t)b * ntiles + t];
  s[b] = sqrt(acc);
}

template <typename T>
__global__ void k_sumsq(const T* __restrict__ v, long long len, double* __restrict__ partials,
                        const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  __shared__ double red[32];
  double ss = 0.0;
  const T* vb = v + (size_t)b * len;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x) {
    double t = (double)vb[i];
    ss += t * t;
  }
  double s = block_sum<T>(ss, red);
  if (threadIdx.x == 0) partials[(size_t)b * gridDim.x + blockIdx.x] = s;
}

__global__ void k_converge(const double* __restrict__ s, const double* __restrict__ fn,
                           double rtol, int B, int* __restrict__ active,
                           double* __restrict__ relres, int* __restrict__ status,
                           int* __restrict__ nactive) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !active[b]) return;
  double f = fn[b];
  // ||f|| = 0: converged (u = 0 solves it); ||f|| NaN (a NaN in f): rr stays
  // NaN and the right-hand side is reported as diverged
  double rr = f > 0.0 ? s[b] / f : (f == 0.0 ? 0.0 : f);
  relres[b] = rr;
  if (!(rr == rr) || rr > 1e30) {
    status[b] = NMG_DIVERGED;
    active[b] = 0;
  } else if (rr <= rtol) {
    status[b] = NMG_CONVERGED;
    active[b] = 0;
  } else {
    atomicAdd(nactive, 1);
  }
}

template <typename T>
__global__ void k_axpy_update(int len, int B, const T* xs, const T* __restrict__ h, T* x,
                              const int* __restrict__ active) {
  for (int b = blockIdx.y; b < B; b += gridDim.y) {
    if (!active[b]) continue;
    const size_t o = (size_t)b * len;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x)
      x[o + i] = (xs ? xs[o + i] : T(0)) + h[o + i];
  }
}

__global__ void k_update_f64(int len, int B, const float* __restrict__ d, double* __restrict__ u,
                             const int* __restrict__ active) {
  for (int b = blockIdx.y; b < B; b += gridDim.y) {
    if (!active[b]) continue;
    const size_t o = (size_t)b * len;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x)
      u[o + i] += (double)d[o + i];
  }
}

__global__ void k_count_cycles(int B, const int* __restrict__ active, int* __restrict__ cycles) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B && active[b]) cycles[b] += 1;
}

// slots newly admitted into a serving pool join the active set
__global__ void k_admit(int B, const int* __restrict__ newmask, int* __restrict__ active) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B && newmask[b]) active[b] = 1;
}

int grid_for(long long total, int threads) {
  long long g = (total + threads - 1) / threads;
  if (g > 152LL * 16) g = 152LL * 16;
  if (g < 1) g = 1;
  return (int)g;
}

// grid of a per-right-hand-side elementwise kernel: y over the batch, x over
// `len` elements, about 16 blocks per SM in total
dim3 grid_batched(long long len, int B, int threads) {
  long long gx = (len + threads - 1) / threads;
  const long long cap = (152LL * 16 + B - 1) / (B > 0 ? B : 1);
  if (gx > cap) gx = cap;
  if (gx < 1) gx = 1;
  return dim3((unsigned)gx, (unsigned)(B < 1 ? 1 : (B > 65535 ? 65535 : B)));
}

template <typename T>
size_t residual_smem(int RH, int RW, int wK, int wM, bool restrict_) {
  int W = wK > wM ? wK : wM;
  size_t e = (size_t)(RH + 2 * W) * (RW + 2 * W) + (size_t)(RH + 2 * wK) * RW +
             (size_t)(RH + 2 * wM) * RW + (restrict_ ? (size_t)RH * RW : 0) +
             (size_t)(RW + RH) * (2 * wK + 1 + 2 * wM + 1);
  return e * sizeof(T);
}

// tile sizes: fine tile for the residual, coarse tile for residual+restrict;
// shrunk until the shared-memory footprint fits in 200 KB
// tile side: the requested one (0 = default: 64 fine / 32 coarse), clipped to
// the grid, halved until the shared-memory footprint fits in 200 KB, and
// doubled while one right-hand side would need more than 4096 tiles (the
// partial-sum slots per item)
template <typename T>
int pick_tile(int n, int wK, int wM, bool restrict_, int req) {
  int t = req > 0 ? req : (restrict_ ? 32 : 64);
  int lim = restrict_ ? n / 2 : n;
  if (t > lim) t = lim;
  while (t > 4) {
    int R = restrict_ ? 2 * t + 1 : t;
    if (residual_smem<T>(R, R, wK, wM, restrict_) <= 200 * 1024) break;
    t /= 2;
  }
  while (t < lim && (long long)ceil_div(lim, t) * ceil_div(lim, t) > 4096) t *= 2;
  return t;
}

}  // namespace

template <typename T>
void launch_residual2d(const Band2D<T>& op, int B, const T* x, const T* y, T* r,
                       double* partials, int* ntiles, const int* active, cudaStream_t st,
                       LaunchLog& log, int tile_req) {
  // tile_req <= 0 on a wide-stencil level: the strip kernel with -tile_req
  // chunks per strip (0: its own choice); > 0: the tiled pipeline
  int tile = pick_tile<T>(op.n, op.wK, op.wM, false, tile_req > 0 ? tile_req : 0);
  int tx = ceil_div(op.n, tile);
  int pi_ = log.begin(K_RESIDUAL, st);
  int nparts = tx * tx;
  if constexpr (std::is_same<T, float>::value) {
    if (tile_req <= 0 && wide_residual_applies(op, x, y)) {
      nparts = launch_residual_wide(op, B, x, y, r, partials, active, -tile_req, st);
      if (ntiles) *ntiles = nparts;
      log.end(pi_, st, (double)op.n * op.n * log.active_hint);
      return;
    }
  }
  if (!launch_stencil_residual<T, false>(op, B, x, y, r, partials, active, tile, tx, st, &nparts)) {
    nparts = tx * tx;
    size_t sm = residual_smem<T>(tile, tile, op.wK, op.wM, false);
    auto kern = k_residual2d<T, false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kern<<<dim3(tx * tx, B), kThreads, sm, st>>>(op, x, y, r, partials, active, tile, tx);
  }
  if (ntiles) *ntiles = nparts;
  log.end(pi_, st, (double)op.n * op.n * log.active_hint);
}

// Upper bound of the partial sums launch_residual2d writes per right-hand
// side (one per tile or strip unit), for a caller that has to size their
// buffer before the launch (the launch reports the exact count).
template <typename T>
int residual2d_tiles(const Band2D<T>& op, int tile_req) {
  const int tx = ceil_div(op.n, pick_tile<T>(op.n, op.wK, op.wM, false, tile_req));
  int strip = stencil_strip_parts<T>(op);
  if (op.n % 64 == 0) {
    const int wide = (op.n / 64) * wide_chunks_max(op.n);  // the wide strip form's units
    strip = wide > strip ? wide : strip;
  }
  return tx * tx > strip ? tx * tx : strip;
}

template <typename T>
void launch_residual_restrict2d(const Band2D<T>& op, int B, const T* x, const T* y, T* yc,
                                double* partials, int* ntiles, const int* active,
                                cudaStream_t st, LaunchLog& log, int tile_req) {
  int tile = pick_tile<T>(op.n, op.wK, op.wM, true, tile_req);
  int nc = op.n / 2;
  int tx = ceil_div(nc, tile);
  int pi_ = log.begin(K_RESTRICT, st);
  int nparts = tx * tx;
  if (!launch_stencil_residual<T, true>(op, B, x, y, yc, partials, active, tile, tx, st, &nparts)) {
    nparts = tx * tx;
    size_t sm = residual_smem<T>(2 * tile + 1, 2 * tile + 1, op.wK, op.wM, true);
    auto kern = k_residual2d<T, true>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kern<<<dim3(tx * tx, B), kThreads, sm, st>>>(op, x, y, yc, partials, active, tile, tx);
  }
  if (ntiles) *ntiles = nparts;
  log.end(pi_, st, (double)op.n * op.n * log.active_hint);
}

template <typename T>
void launch_prolong2d(int n, int B, const T* e, T* x, const int* active, cudaStream_t st,
                      LaunchLog& log) {
  int pi_ = log.begin(K_PROLONG, st);
  k_prolong2d<T><<<grid_batched((long long)(n / 2) * (n / 2), B, 256), 256, 0, st>>>(n, B, e, x,
                                                                                     active);
  log.end(pi_, st, (double)n * n * log.active_hint);
}

template <typename T>
void launch_residual1d(int n, const T* A, int B, const T* x, const T* y, T* r,
                       double* partials, int* ntiles, const int* active, cudaStream_t st,
                       LaunchLog& log) {
  int rows = 8;  // warps per block
  dim3 grid(ceil_div(n, rows), B);
  int pi_ = log.begin(K_RESIDUAL, st);
  k_residual1d<T><<<grid, rows * 32, 0, st>>>(n, A, x, y, r, partials, active);
  if (ntiles) *ntiles = grid.x;
  log.end(pi_, st, (double)n * log.active_hint);
}

// Partial sums launch_residual1d writes per right-hand side: one per block
// of 8 rows (its grid).
int residual1d_tiles(int n) { return ceil_div(n, 8); }

template <typename T>
void launch_restrict1d(int n, int B, const T* r, T* yc, double* partials, int* ntiles,
                       const int* active, cudaStream_t st, LaunchLog& log) {
  dim3 grid(ceil_div(n / 2, 128), B);
  int pi_ = log.begin(K_RESTRICT, st);
  k_restrict1d<T><<<grid, 128, 0, st>>>(n, r, yc, partials, active);
  if (ntiles) *ntiles = grid.x;
  log.end(pi_, st, (double)n * log.active_hint);
}

template <typename T>
void launch_prolong1d(int n, int B, const T* e, T* x, const int* active, cudaStream_t st,
                      LaunchLog& log) {
  int pi_ = log.begin(K_PROLONG, st);
  k_prolong1d<T><<<grid_for((long long)n * B, 256), 256, 0, st>>>(n, B, e, x, active);
  log.end(pi_, st, (double)n * log.active_hint);
}

void launch_norms(const double* partials, int ntiles, int B, double* s, const int* active,
                  cudaStream_t st, LaunchLog& log) {
  int pi_ = log.begin(K_OTHER, st);
  k_norms<<<ceil_div(B, 128), 128, 0, st>>>(partials, ntiles, B, s, active);
  log.end(pi_, st, 0.0);
}

template <typename T>
void launch_sumsq(const T* v, long long len, int B, double* partials, int* ntiles,
                  const int* active, cudaStream_t st, LaunchLog& log) {
  int g = (int)std::min<long long>(64, (len + 255) / 256);
  if (g < 1) g = 1;
  dim3 grid(g, B);
  int pi_ = log.begin(K_OTHER, st);
  k_sumsq<T><<<grid, 256, 0, st>>>(v, len, partials, active);
  if (ntiles) *ntiles = g;
  log.end(pi_, st, 0.0);
}

void launch_converge(const double* s, const double* fn, double rtol, int B, int* active,
                     double* relres, int* status, int* nactive, cudaStream_t st,
                     LaunchLog& log) {
  int pi_ = log.begin(K_OTHER, st);
  k_converge<<<ceil_div(B, 128), 128, 0, st>>>(s, fn, rtol, B, active, relres, status, nactive);
  log.end(pi_, st, 0.0);
}

template <typename T>
void launch_axpy_update(long long len, int B, const T* xstar, const T* h, T* x,
                        const int* active, cudaStream_t st, LaunchLog& log) {
  int pi_ = log.begin(K_OTHER, st);
  k_axpy_update<T><<<grid_batched(len, B, 256), 256, 0, st>>>((int)len, B, xstar, h, x, active);
  log.end(pi_, st, 0.0);
}

void launch_count_cycles(int B, const int* active, int* cycles, cudaStream_t st, LaunchLog& log) {
  int pi_ = log.begin(K_OTHER, st);
  k_count_cycles<<<ceil_div(B, 128), 128, 0, st>>>(B, active, cycles);
  log.end(pi_, st, 0.0);
}

void launch_admit(int B, const int* newmask, int* active, cudaStream_t st, LaunchLog& log) {
  int pi_ = log.begin(K_OTHER, st);
  k_admit<<<ceil_div(B, 128), 128, 0, st>>>(B, newmask, active);
  log.end(pi_, st, 0.0);
}

void launch_update_f64(long long len, int B, const float* d, double* u, const int* active,
                       cudaStream_t st, LaunchLog& log) {
  int pi_ = log.begin(K_OTHER, st);
  k_update_f64<<<grid_batched(len, B, 256), 256, 0, st>>>((int)len, B, d, u, active);
  log.end(pi_, st, (double)len * log.active_hint);
}

#define NMG_INST(T)                                                                          \
  template void launch_residual2d<T>(const Band2D<T>&, int, const T*, const T*, T*, double*, \
                                     int*, const int*, cudaStream_t, LaunchLog&, int);       \
  template int residual2d_tiles<T>(const Band2D<T>&, int);                                   \
  template void launch_residual_restrict2d<T>(const Band2D<T>&, int, const T*, const T*,     \
                                              T*, double*, int*, const int*, cudaStream_t,   \
                                              LaunchLog&, int);                              \
  template void launch_prolong2d<T>(int, int, const T*, T*, const int*, cudaStream_t,        \
                                    LaunchLog&);                                             \
  template void launch_residual1d<T>(int, const T*, int, const T*, const T*, T*, double*,    \
                                     int*, const int*, cudaStream_t, LaunchLog&);            \
  template void launch_restrict1d<T>(int, int, const T*, T*, double*, int*, const int*,      \
                                     cudaStream_t, LaunchLog&);                              \
  template void launch_prolong1d<T>(int, int, const T*, T*, const int*, cudaStream_t,        \
                                    LaunchLog&);                                             \
  template void launch_sumsq<T>(const T*, long long, int, double*, int*, const int*,         \
                                cudaStream_t, LaunchLog&);                                   \
  template void launch_axpy_update<T>(long long, int, const T*, const T*, T*, const int*,    \
                                      cudaStream_t, LaunchLog&);
NMG_INST(float)
NMG_INST(double)
#undef NMG_INST

}  // namespace nmg
