// Coarsest-level exact solve x_L = (A^(L))^{-1} y_L (Algorithms 3 and 4)
// in fp64: a one-block right-looking Cholesky factorisation at setup and
// batched forward/back substitution per cycle.
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

// One block per right-hand side: z = L^{-1} y, x = L^{-T} z in fp64.
template <typename T>
__global__ void k_coarse_solve(int nc, const double* __restrict__ L, const T* __restrict__ y,
                               T* __restrict__ x, const int* __restrict__ active) {
  const int b = blockIdx.x;
  if (!active[b]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* z = reinterpret_cast<double*>(smem_raw);
  for (int i = threadIdx.x; i < nc; i += blockDim.x) z[i] = (double)y[(size_t)b * nc + i];
  __syncthreads();
  for (int j = 0; j < nc; ++j) {
    double zj = z[j] / L[(size_t)j * nc + j];
    __syncthreads();
    if (threadIdx.x == 0) z[j] = zj;
    for (int i = j + 1 + threadIdx.x; i < nc; i += blockDim.x) z[i] -= L[(size_t)i * nc + j] * zj;
    __syncthreads();
  }
  for (int j = nc - 1; j >= 0; --j) {
    double xj = z[j] / L[(size_t)j * nc + j];
    __syncthreads();
    if (threadIdx.x == 0) z[j] = xj;
    for (int i = threadIdx.x; i < j; i += blockDim.x) z[i] -= L[(size_t)j * nc + i] * xj;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < nc; i += blockDim.x) x[(size_t)b * nc + i] = (T)z[i];
}

}  // namespace

void launch_cholesky(int nc, double* A, int* flag, cudaStream_t st, LaunchLog& log) {
  int pi_ = log.begin(K_OTHER, st);
  k_cholesky<<<1, 256, 0, st>>>(nc, A, flag);
  log.end(pi_, st, 0.0);
}

template <typename T>
void launch_coarse_solve(int nc, const double* L, int B, const T* y, T* x, const int* active,
                         cudaStream_t st, LaunchLog& log) {
  int threads = nc < 64 ? 32 : (nc < 256 ? 64 : 256);
  int pi_ = log.begin(K_COARSE, st);
  k_coarse_solve<T><<<B, threads, nc * sizeof(double), st>>>(nc, L, y, x, active);
  log.end(pi_, st, (double)nc * log.active_hint);
}

template void launch_coarse_solve<float>(int, const double*, int, const float*, float*,
                                         const int*, cudaStream_t, LaunchLog&);
template void launch_coarse_solve<double>(int, const double*, int, const double*, double*,
                                          const int*, cudaStream_t, LaunchLog&);

}  // namespace nmg
