// Kernels of the classical comparators the paper measures the neural
// multigrid against: the weighted Jacobi step of Section 2.2 (the smoother of
// the backslash V-cycle of Algorithm 1) and the vector operations of
// conjugate gradients (Section 4.2, Table 4).  The operator applies,
// transfers and the coarsest solve are the hierarchy's own kernels.
#include "nmg_internal.h"

namespace nmg {

namespace {

// x += omega r / diag(A_l); 2D diag = alpha m_i m_j + k_i k_j with k_i, m_i
// the diagonals of the DIA factors K_l, M_l
template <typename T>
__global__ void k_jacobi2d(Band2D<T> op, int B, T* __restrict__ x, const T* __restrict__ r,
                           T omega, const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const int n = op.n;
  const size_t plane = (size_t)n * n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)plane;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx - (long long)i * n);
    const T ki = op.Kd[(size_t)i * (2 * op.wK + 1) + op.wK];
    const T kj = op.Kd[(size_t)j * (2 * op.wK + 1) + op.wK];
    const T mi = op.Md[(size_t)i * (2 * op.wM + 1) + op.wM];
    const T mj = op.Md[(size_t)j * (2 * op.wM + 1) + op.wM];
    const size_t g = (size_t)b * plane + idx;
    x[g] += omega * r[g] / (op.alpha * mi * mj + ki * kj);
  }
}

template <typename T>
__global__ void k_jacobi1d(int n, const T* __restrict__ A, int B, T* __restrict__ x,
                           const T* __restrict__ r, T omega, const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const size_t g = (size_t)b * n + i;
    x[g] += omega * r[g] / A[(size_t)i * n + i];
  }
}

constexpr int kDotThreads = 256;

// per-block partial sums of a . b (fp64) for every active right-hand side:
// partials[b * gridDim.x + block]
template <typename T>
__global__ void __launch_bounds__(kDotThreads)
k_dot_partials(const T* __restrict__ a, const T* __restrict__ c, long long len,
               double* __restrict__ partials, const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  __shared__ double red[kDotThreads / 32];
  double s = 0.0;
  const T* ab = a + (size_t)b * len;
  const T* cb = c + (size_t)b * len;
  for (long long i = blockIdx.x * (long long)kDotThreads + threadIdx.x; i < len;
       i += (long long)gridDim.x * kDotThreads)
    s += (double)ab[i] * (double)cb[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kDotThreads / 32; ++w) t += red[w];
    partials[(size_t)b * gridDim.x + blockIdx.x] = t;
  }
}

// q = -A p (the residual kernel with y = 0): alpha = (r, r) / (p, A p)
__global__ void k_cg_alpha(int B, const double* __restrict__ partials, int nblk,
                           const double* __restrict__ rr, double* __restrict__ alpha,
                           const int* __restrict__ active) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !active[b]) return;
  double pq = 0.0;
  for (int k = 0; k < nblk; ++k) pq += partials[(size_t)b * nblk + k];
  alpha[b] = rr[b] / (-pq);
}

// u += alpha p, r += alpha q (= r - alpha A p), partial sums of the new r . r
template <typename T>
__global__ void __launch_bounds__(kDotThreads)
k_cg_update(long long len, T* __restrict__ u, T* __restrict__ r, const T* __restrict__ p,
            const T* __restrict__ q, const double* __restrict__ alpha,
            double* __restrict__ partials, const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  __shared__ double red[kDotThreads / 32];
  const T a = (T)alpha[b];
  double s = 0.0;
  const size_t off = (size_t)b * len;
  for (long long i = blockIdx.x * (long long)kDotThreads + threadIdx.x; i < len;
       i += (long long)gridDim.x * kDotThreads) {
    u[off + i] += a * p[off + i];
    const T rn = r[off + i] + a * q[off + i];
    r[off + i] = rn;
    s += (double)rn * (double)rn;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kDotThreads / 32; ++w) t += red[w];
    partials[(size_t)b * gridDim.x + blockIdx.x] = t;
  }
}

// rr_new = sum of partials; beta = rr_new / rr; rr = rr_new; s = sqrt(rr_new)
__global__ void k_cg_beta(int B, const double* __restrict__ partials, int nblk,
                          double* __restrict__ rr, double* __restrict__ beta,
                          double* __restrict__ s, const int* __restrict__ active) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !active[b]) return;
  double t = 0.0;
  for (int k = 0; k < nblk; ++k) t += partials[(size_t)b * nblk + k];
  beta[b] = t / rr[b];
  rr[b] = t;
  s[b] = sqrt(t);
}

// rr = s^2 (the first residual's squared norm)
__global__ void k_cg_init(int B, const double* __restrict__ s, double* __restrict__ rr,
                          const int* __restrict__ active) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !active[b]) return;
  rr[b] = s[b] * s[b];
}

template <typename T>
__global__ void k_cg_p(long long len, T* __restrict__ p, const T* __restrict__ r,
                       const double* __restrict__ beta, const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const T be = (T)beta[b];
  const size_t off = (size_t)b * len;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    p[off + i] = r[off + i] + be * p[off + i];
}

int blocks_for(long long len) {
  long long g = (len + kDotThreads - 1) / kDotThreads;
  if (g > 64) g = 64;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

template <typename T>
void launch_jacobi2d(const Band2D<T>& op, int B, T* x, const T* r, double omega, const int* active,
                     cudaStream_t st, LaunchLog& log) {
  const long long plane = (long long)op.n * op.n;
  int pi_ = log.begin(K_OTHER, st);
  k_jacobi2d<T><<<dim3(blocks_for(plane), B), kDotThreads, 0, st>>>(op, B, x, r, (T)omega, active);
  log.end(pi_, st, (double)plane * log.active_hint);
}

template <typename T>
void launch_jacobi1d(int n, const T* A, int B, T* x, const T* r, double omega, const int* active,
                     cudaStream_t st, LaunchLog& log) {
  int pi_ = log.begin(K_OTHER, st);
  k_jacobi1d<T><<<dim3(blocks_for(n), B), kDotThreads, 0, st>>>(n, A, B, x, r, (T)omega, active);
  log.end(pi_, st, (double)n * log.active_hint);
}

// one CG iteration after q = -A p: alpha, the u / r update with the new
// (r, r), beta and p (five launches); scal: rr, alpha, beta (B each)
template <typename T>
void launch_cg_iteration(long long len, int B, T* u, T* r, T* p, const T* q, double* scal,
                         double* s, double* partials, const int* active, cudaStream_t st,
                         LaunchLog& log) {
  double* rr = scal;
  double* alpha = scal + B;
  double* beta = scal + 2 * B;
  const int nblk = blocks_for(len);
  const int sb = (B + 127) / 128;
  int pi_ = log.begin(K_OTHER, st);
  k_dot_partials<T><<<dim3(nblk, B), kDotThreads, 0, st>>>(p, q, len, partials, active);
  log.end(pi_, st, (double)len * log.active_hint);
  pi_ = log.begin(K_OTHER, st);
  k_cg_alpha<<<sb, 128, 0, st>>>(B, partials, nblk, rr, alpha, active);
  log.end(pi_, st, 0.0);
  pi_ = log.begin(K_OTHER, st);
  k_cg_update<T><<<dim3(nblk, B), kDotThreads, 0, st>>>(len, u, r, p, q, alpha, partials, active);
  log.end(pi_, st, (double)len * log.active_hint);
  pi_ = log.begin(K_OTHER, st);
  k_cg_beta<<<sb, 128, 0, st>>>(B, partials, nblk, rr, beta, s, active);
  log.end(pi_, st, 0.0);
  pi_ = log.begin(K_OTHER, st);
  k_cg_p<T><<<dim3(nblk, B), kDotThreads, 0, st>>>(len, p, r, beta, active);
  log.end(pi_, st, (double)len * log.active_hint);
}

void launch_cg_init(int B, const double* s, double* scal, const int* active, cudaStream_t st,
                    LaunchLog& log) {
  int pi_ = log.begin(K_OTHER, st);
  k_cg_init<<<(B + 127) / 128, 128, 0, st>>>(B, s, scal, active);
  log.end(pi_, st, 0.0);
}

template void launch_jacobi2d<float>(const Band2D<float>&, int, float*, const float*, double,
                                     const int*, cudaStream_t, LaunchLog&);
template void launch_jacobi2d<double>(const Band2D<double>&, int, double*, const double*, double,
                                      const int*, cudaStream_t, LaunchLog&);
template void launch_jacobi1d<float>(int, const float*, int, float*, const float*, double,
                                     const int*, cudaStream_t, LaunchLog&);
template void launch_jacobi1d<double>(int, const double*, int, double*, const double*, double,
                                      const int*, cudaStream_t, LaunchLog&);
template void launch_cg_iteration<float>(long long, int, float*, float*, float*, const float*,
                                         double*, double*, double*, const int*, cudaStream_t,
                                         LaunchLog&);
template void launch_cg_iteration<double>(long long, int, double*, double*, double*,
                                          const double*, double*, double*, double*, const int*,
                                          cudaStream_t, LaunchLog&);

}  // namespace nmg
