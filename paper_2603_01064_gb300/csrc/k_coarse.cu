// Coarsest-level exact solve x_L = (A^(L))^{-1} y_L (Algorithms 3 and 4)
// in fp64: a one-block right-looking Cholesky factorisation A = L L^T and
// the inverse factor L^{-1} at setup, then per cycle the two triangular
// products x = L^{-T} (L^{-1} y) for the whole batch.
#include "nmg_internal.h"

namespace nmg {

namespace {

// In-place lower Cholesky of the nc x nc row-major matrix A (upper part is
// left as is and never read).  flag = 1 if a pivot is not positive.
__global__ void k_cholesky(int nc, double* A, int* flag) {
  __shared__ double piv;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < nc; ++k) {
    if (threadIdx.x == 0) {
      double d = A[(size_t)k * nc + k];
      if (!(d > 0.0)) {
        bad = 1;
        d = 1.0;
      }
      piv = sqrt(d);
      A[(size_t)k * nc + k] = piv;
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < nc; i += blockDim.x) A[(size_t)i * nc + k] /= piv;
    __syncthreads();
    const int m = nc - k - 1;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      int i = k + 1 + t / m, j = k + 1 + t % m;
      if (j <= i) A[(size_t)i * nc + j] -= A[(size_t)i * nc + k] * A[(size_t)j * nc + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *flag = bad;
}

// Inverse of the Cholesky factor, once at setup: block j solves L z = e_j
// by forward substitution and writes column j of L^{-1} (and row j of its
// transpose), so that every cycle's coarsest solve is two dense triangular
// products instead of 2 nc sequential substitution steps.
__global__ void k_chol_inverse(int nc, const double* __restrict__ L, double* __restrict__ Li,
                               double* __restrict__ LiT) {
  const int j = blockIdx.x;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* z = reinterpret_cast<double*>(smem_raw);
  for (int i = threadIdx.x; i < nc; i += blockDim.x) z[i] = i == j ? 1.0 : 0.0;
  __syncthreads();
  for (int k = j; k < nc; ++k) {
    const double zk = z[k] / L[(size_t)k * nc + k];
    __syncthreads();
    if (threadIdx.x == 0) z[k] = zk;
    for (int i = k + 1 + threadIdx.x; i < nc; i += blockDim.x) z[i] -= L[(size_t)i * nc + k] * zk;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    Li[(size_t)i * nc + j] = z[i];
    LiT[(size_t)j * nc + i] = z[i];
  }
}

// x = L^{-T} (L^{-1} y) in fp64, one block per right-hand side.  Each warp
// forms 8 rows of a triangular product at a time (lanes along the row, the
// 8 rows' loads in flight together, then interleaved warp reductions), so
// the factors are read coalesced and load latency is paid once per 8 rows.
template <bool UPPER>
__device__ __forceinline__ void tri_rows(int nc, const double* __restrict__ F, const double* in,
                                         double* out, int lane, int warp, int nw) {
  constexpr int R = 8;
  for (int i0 = warp * R; i0 < nc; i0 += nw * R) {
    double acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0;
    // column chunks outer, rows inner: the R rows' loads of a chunk are
    // independent and in flight together (entries outside the triangle are
    // zero in F, so only the row bounds are tested)
    const int c_lo = UPPER ? (i0 & ~31) : 0;
    const int c_hi = UPPER ? nc : (i0 + R < nc ? i0 + R : nc);
    for (int cb = c_lo; cb < c_hi; cb += 32) {
      const int c = cb + lane;
      const double vin = c < nc ? in[c] : 0.0;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = i0 + r;
        if (i < nc && c < nc) acc[r] += F[(size_t)i * nc + c] * vin;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    if (lane == 0) {
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (i0 + r < nc) out[i0 + r] = acc[r];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_coarse_apply(int nc, const double* __restrict__ Li, const double* __restrict__ LiT,
               const T* __restrict__ y, T* __restrict__ x, const int* __restrict__ active) {
  const int b = blockIdx.x;
  if (!active[b]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* v = reinterpret_cast<double*>(smem_raw);
  double* z = v + nc;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < nc; i += blockDim.x) v[i] = (double)y[(size_t)b * nc + i];
  __syncthreads();
  tri_rows<false>(nc, Li, v, z, lane, warp, nw);  // z = L^{-1} v
  __syncthreads();
  tri_rows<true>(nc, LiT, z, v, lane, warp, nw);  // v = L^{-T} z
  __syncthreads();
  for (int i = threadIdx.x; i < nc; i += blockDim.x) x[(size_t)b * nc + i] = (T)v[i];
}

// nc <= 64: one block of two warps per right-hand side, thread i owning
// row i, two accumulation chains per row (fp64 runs at 1/64 of the fp32 rate
// on this GPU: two warps per right-hand side spread the multiply-adds over
// twice the SM sub-partitions of one warp owning two rows per lane);
// both products read the stored transposes row by row, so the 32 lanes load
// consecutive entries: z = L^{-1} v as z_i = sum_j (L^{-T})[j][i] v_j and
// x = L^{-T} z as x_i = sum_j (L^{-1})[j][i] z_j
template <typename T>
__global__ void __launch_bounds__(64)
k_coarse_apply_warp(int nc, const double* __restrict__ Li, const double* __restrict__ LiT, int B,
                    const T* __restrict__ y, T* __restrict__ x, const int* __restrict__ active) {
  __shared__ double v[64];
  const int t = threadIdx.x;
  const int b = blockIdx.x;
  if (!active[b]) return;
  if (t < nc) v[t] = (double)y[(size_t)b * nc + t];
  __syncthreads();
  const bool in = t < nc;
  const int c = in ? t : 0;  // in-bounds column
  double za = 0.0, zb = 0.0;
  int j = 0;
  for (; j + 1 < nc; j += 2) {
    za = fma(LiT[(size_t)j * nc + c], v[j], za);
    zb = fma(LiT[(size_t)(j + 1) * nc + c], v[j + 1], zb);
  }
  if (j < nc) za = fma(LiT[(size_t)j * nc + c], v[j], za);
  __syncthreads();
  if (in) v[t] = za + zb;
  __syncthreads();
  double xa = 0.0, xb = 0.0;
  for (j = 0; j + 1 < nc; j += 2) {
    xa = fma(Li[(size_t)j * nc + c], v[j], xa);
    xb = fma(Li[(size_t)(j + 1) * nc + c], v[j + 1], xb);
  }
  if (j < nc) xa = fma(Li[(size_t)j * nc + c], v[j], xa);
  if (in) x[(size_t)b * nc + t] = (T)(xa + xb);
}

}  // namespace

void launch_cholesky(int nc, double* A, int* flag, cudaStream_t st, LaunchLog& log) {
  int pi_ = log.begin(K_OTHER, st);
  k_cholesky<<<1, 256, 0, st>>>(nc, A, flag);
  log.end(pi_, st, 0.0);
}

void launch_chol_inverse(int nc, const double* L, double* Li, double* LiT, cudaStream_t st,
                         LaunchLog& log) {
  const int threads = nc < 64 ? 32 : (nc < 256 ? 64 : 256);
  int pi_ = log.begin(K_OTHER, st);
  k_chol_inverse<<<nc, threads, nc * sizeof(double), st>>>(nc, L, Li, LiT);
  log.end(pi_, st, 0.0);
}

template <typename T>
void launch_coarse_solve(int nc, const double* Li, const double* LiT, int B, const T* y, T* x,
                         const int* active, cudaStream_t st, LaunchLog& log) {
  int pi_ = log.begin(K_COARSE, st);
  if (nc <= 64) {
    k_coarse_apply_warp<T><<<B, 64, 0, st>>>(nc, Li, LiT, B, y, x, active);
  } else {
    k_coarse_apply<T><<<B, 256, 2 * nc * sizeof(double), st>>>(nc, Li, LiT, y, x, active);
  }
  log.end(pi_, st, (double)nc * log.active_hint);
}

template void launch_coarse_solve<float>(int, const double*, const double*, int, const float*,
                                         float*, const int*, cudaStream_t, LaunchLog&);
template void launch_coarse_solve<double>(int, const double*, const double*, int, const double*,
                                          double*, const int*, cudaStream_t, LaunchLog&);

}  // namespace nmg
