// Output filter of the cycle, x = x* + F'_l(h) with
// F'_l(h) = Re(IDFT(m'_l . DFT(h))) (Sections 3.2 and 3.3).
//
// 2D: three passes over a complex [B][n][n] buffer, each an in-shared-memory
// radix-2 Cooley-Tukey FFT over whole rows/columns:
//   1. forward FFT of every row of h (real input);
//   2. per block of columns: forward FFT down the column, multiply by the
//      mask m'(k1, k2) = sqrt(max(|w1|, |w2|) / pi), inverse FFT;
//   3. inverse FFT of every row, x = x* + Re(.) / n^2.
// The mask is real and even in each axis, so the result is real up to
// rounding, which Re(.) drops as the paper states.
// 1D: x = x* + C h with C the real symmetric circulant of the filter,
// applied directly from its first column.
#include "nmg_internal.h"

namespace nmg {

namespace {

template <typename T>
struct Cx {
  T x, y;
};

__device__ __forceinline__ int bitrev(int v, int logn) { return __brev(v) >> (32 - logn); }

// In-place iterative radix-2 DIT FFT of `cnt` sequences of length n stored
// back to back in shared memory, input in bit-reversed order, output in
// natural order.  tw[k] = exp(-2 pi i k / n), k < n/2.  sign = +1 forward,
// -1 inverse (conjugated twiddles, no scaling).
template <typename T>
__device__ void fft_stages(Cx<T>* buf, int n, int logn, int cnt, const Cx<T>* tw, int sign) {
  const int halfn = n >> 1;
  for (int s = 1; s <= logn; ++s) {
    const int half = 1 << (s - 1);
    const int tstride = n >> s;
    for (int t = threadIdx.x; t < cnt * halfn; t += blockDim.x) {
      int seq = t / halfn, k = t % halfn;
      int grp = k / half, pos = k % half;
      int i = seq * n + grp * 2 * half + pos;
      int j = i + half;
      Cx<T> w = tw[pos * tstride];
      if (sign < 0) w.y = -w.y;
      Cx<T> a = buf[i], bb = buf[j];
      Cx<T> p{w.x * bb.x - w.y * bb.y, w.x * bb.y + w.y * bb.x};
      buf[i] = Cx<T>{a.x + p.x, a.y + p.y};
      buf[j] = Cx<T>{a.x - p.x, a.y - p.y};
    }
    __syncthreads();
  }
}

// pass 1: rows of real h -> complex spectrum rows
template <typename T>
__global__ void k_fft_rows_fwd(int n, int logn, int rpc, const T* __restrict__ h,
                               Cx<T>* __restrict__ C, const Cx<T>* __restrict__ twg,
                               const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<T>* tw = reinterpret_cast<Cx<T>*>(smem_raw);
  Cx<T>* buf = tw + n / 2;
  for (int k = threadIdx.x; k < n / 2; k += blockDim.x) tw[k] = twg[k];
  const int row0 = blockIdx.x * rpc;
  const size_t plane = (size_t)n * n;
  for (int t = threadIdx.x; t < rpc * n; t += blockDim.x) {
    int r = t / n, j = t % n;
    T v = h[(size_t)b * plane + (size_t)(row0 + r) * n + j];
    buf[r * n + bitrev(j, logn)] = Cx<T>{v, T(0)};
  }
  __syncthreads();
  fft_stages(buf, n, logn, rpc, tw, +1);
  for (int t = threadIdx.x; t < rpc * n; t += blockDim.x) {
    int r = t / n, j = t % n;
    C[(size_t)b * plane + (size_t)(row0 + r) * n + j] = buf[t];
  }
}

// pass 2: column FFT, mask, inverse column FFT (in place on C)
template <typename T>
__global__ void k_fft_cols_mask(int n, int logn, int cpc, Cx<T>* __restrict__ C,
                                const Cx<T>* __restrict__ twg, const double* __restrict__ mtab,
                                const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<T>* tw = reinterpret_cast<Cx<T>*>(smem_raw);
  Cx<T>* buf = tw + n / 2;  // cpc sequences of length n (one per column)
  for (int k = threadIdx.x; k < n / 2; k += blockDim.x) tw[k] = twg[k];
  const int col0 = blockIdx.x * cpc;
  const size_t plane = (size_t)n * n;
  Cx<T>* Cb = C + (size_t)b * plane;
  for (int t = threadIdx.x; t < cpc * n; t += blockDim.x) {
    int r = t / cpc, c = t % cpc;  // consecutive threads: consecutive columns
    buf[c * n + bitrev(r, logn)] = Cb[(size_t)r * n + col0 + c];
  }
  __syncthreads();
  fft_stages(buf, n, logn, cpc, tw, +1);
  // mask, then back to bit-reversed order for the inverse transform
  for (int t = threadIdx.x; t < cpc * n; t += blockDim.x) {
    int c = t / n, k1 = t % n;
    int k2 = col0 + c;
    int f1 = k1 < n - k1 ? k1 : n - k1;
    int f2 = k2 < n - k2 ? k2 : n - k2;
    T m = (T)mtab[f1 > f2 ? f1 : f2];
    Cx<T> v = buf[t];
    v.x *= m;
    v.y *= m;
    buf[t] = v;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < cpc * n; t += blockDim.x) {
    int c = t / n, k = t % n;
    int rk = bitrev(k, logn);
    if (k < rk) {
      Cx<T> a = buf[c * n + k];
      buf[c * n + k] = buf[c * n + rk];
      buf[c * n + rk] = a;
    }
  }
  __syncthreads();
  fft_stages(buf, n, logn, cpc, tw, -1);
  for (int t = threadIdx.x; t < cpc * n; t += blockDim.x) {
    int r = t / cpc, c = t % cpc;
    Cb[(size_t)r * n + col0 + c] = buf[c * n + r];
  }
}

// pass 3: inverse row FFT and the update x = x* + Re(.) / n^2
template <typename T>
__global__ void k_fft_rows_inv(int n, int logn, int rpc, const Cx<T>* __restrict__ C,
                               const T* xstar, T* x,
                               const Cx<T>* __restrict__ twg, const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<T>* tw = reinterpret_cast<Cx<T>*>(smem_raw);
  Cx<T>* buf = tw + n / 2;
  for (int k = threadIdx.x; k < n / 2; k += blockDim.x) tw[k] = twg[k];
  const int row0 = blockIdx.x * rpc;
  const size_t plane = (size_t)n * n;
  for (int t = threadIdx.x; t < rpc * n; t += blockDim.x) {
    int r = t / n, j = t % n;
    buf[r * n + bitrev(j, logn)] = C[(size_t)b * plane + (size_t)(row0 + r) * n + j];
  }
  __syncthreads();
  fft_stages(buf, n, logn, rpc, tw, -1);
  const T scale = T(1.0 / ((double)n * (double)n));
  for (int t = threadIdx.x; t < rpc * n; t += blockDim.x) {
    int r = t / n, j = t % n;
    size_t gi = (size_t)b * plane + (size_t)(row0 + r) * n + j;
    T base = xstar ? xstar[gi] : T(0);
    x[gi] = base + buf[t].x * scale;
  }
}

// Whole filter of one right-hand side in shared memory (levels whose complex
// n x n image fits): row FFTs, column FFTs, mask, inverse column FFTs,
// inverse row FFTs, update.  One launch, h read once and x written once.
template <typename T>
__global__ void __launch_bounds__(512)
k_filter_fused(int n, int logn, const T* xstar, const T* __restrict__ h, T* x,
               const Cx<T>* __restrict__ twg, const double* __restrict__ mtab,
               const int* __restrict__ active) {
  const int b = blockIdx.x;
  if (!active[b]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<T>* tw = reinterpret_cast<Cx<T>*>(smem_raw);
  Cx<T>* buf = tw + n / 2;
  const int nn = n * n, halfn = n / 2;
  for (int k = threadIdx.x; k < halfn; k += blockDim.x) tw[k] = twg[k];
  const size_t base = (size_t)b * nn;
  for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
    const int r = idx / n, c = idx % n;
    buf[r * n + bitrev(c, logn)] = Cx<T>{h[base + idx], T(0)};
  }
  __syncthreads();
  fft_stages(buf, n, logn, n, tw, +1);  // rows
  // rows into bit-reversed order for the column transform
  auto permute_rows = [&]() {
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
      const int r = idx / n, c = idx % n, rr = bitrev(r, logn);
      if (r < rr) {
        Cx<T> t = buf[r * n + c];
        buf[r * n + c] = buf[rr * n + c];
        buf[rr * n + c] = t;
      }
    }
    __syncthreads();
  };
  auto col_stages = [&](int sign) {
    for (int st = 1; st <= logn; ++st) {
      const int half = 1 << (st - 1), tstride = n >> st;
      for (int t = threadIdx.x; t < halfn * n; t += blockDim.x) {
        const int c = t % n, k = t / n;
        const int grp = k / half, pos = k % half;
        const int i = (grp * 2 * half + pos) * n + c, j = i + half * n;
        Cx<T> w = tw[pos * tstride];
        if (sign < 0) w.y = -w.y;
        const Cx<T> a = buf[i], bb = buf[j];
        const Cx<T> p{w.x * bb.x - w.y * bb.y, w.x * bb.y + w.y * bb.x};
        buf[i] = Cx<T>{a.x + p.x, a.y + p.y};
        buf[j] = Cx<T>{a.x - p.x, a.y - p.y};
      }
      __syncthreads();
    }
  };
  permute_rows();
  col_stages(+1);
  for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
    const int k1 = idx / n, k2 = idx % n;
    const int f1 = k1 < n - k1 ? k1 : n - k1, f2 = k2 < n - k2 ? k2 : n - k2;
    const T m = (T)mtab[f1 > f2 ? f1 : f2];
    buf[idx].x *= m;
    buf[idx].y *= m;
  }
  __syncthreads();
  permute_rows();
  col_stages(-1);
  // columns of every row into bit-reversed order for the inverse row transform
  for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
    const int r = idx / n, c = idx % n, rc = bitrev(c, logn);
    if (c < rc) {
      Cx<T> t = buf[r * n + c];
      buf[r * n + c] = buf[r * n + rc];
      buf[r * n + rc] = t;
    }
  }
  __syncthreads();
  fft_stages(buf, n, logn, n, tw, -1);
  const T scale = T(1.0 / ((double)n * (double)n));
  for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
    const T bv = xstar ? xstar[base + idx] : T(0);
    x[base + idx] = bv + buf[idx].x * scale;
  }
}

// 1D: x[b][i] = x*[b][i] + sum_k c[(i - k) mod n] h[b][k]; one warp per output
template <typename T>
__global__ void k_filter1d(int n, const T* xs, const T* __restrict__ h, T* x, const double* __restrict__ circ,
                           const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int i = blockIdx.x * (blockDim.x >> 5) + wid;
  if (i >= n) return;
  const T* hb = h + (size_t)b * n;
  T acc = T(0);
  for (int k = lane; k < n; k += 32) {
    int d = i - k;
    if (d < 0) d += n;
    acc += (T)circ[d] * hb[k];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    size_t gi = (size_t)b * n + i;
    x[gi] = (xs ? xs[gi] : T(0)) + acc;
  }
}

}  // namespace

template <typename T>
void launch_filter2d(int n, int B, const T* xstar, const T* h, T* x, void* cbuf,
                     const T* twiddles, const double* mask_tab, const int* active,
                     cudaStream_t st, LaunchLog& log, int mode) {
  const int logn = ilog2(n);
  // sequences per block: about 64 KB of complex data
  int per = (int)((64 * 1024) / (n * sizeof(Cx<T>)));
  if (per < 1) per = 1;
  if (per > n) per = n;
  if (per > 32) per = 32;
  while (n % per) --per;
  Cx<T>* C = reinterpret_cast<Cx<T>*>(cbuf);
  const Cx<T>* tw = reinterpret_cast<const Cx<T>*>(twiddles);
  const size_t fused_sm = (size_t)(n / 2 + n * n) * sizeof(Cx<T>);
  if (fused_sm <= 160 * 1024 && mode != 0) {
    cudaFuncSetAttribute(k_filter_fused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_sm);
    const int threads = n * n / 2 < 512 ? (n * n / 2 < 32 ? 32 : n * n / 2) : 512;
    int pi_ = log.begin(K_FILTER, st);
    k_filter_fused<T><<<B, threads, fused_sm, st>>>(n, logn, xstar, h, x, tw, mask_tab, active);
    log.end(pi_, st, (double)n * n * log.active_hint);
    return;
  }
  size_t sm = (size_t)(n / 2 + per * n) * sizeof(Cx<T>);
  cudaFuncSetAttribute(k_fft_rows_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_fft_cols_mask<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_fft_rows_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  dim3 grid(n / per, B);
  const double units = (double)n * n * log.active_hint;
  int pi_ = log.begin(K_FILTER, st);
  k_fft_rows_fwd<T><<<grid, 256, sm, st>>>(n, logn, per, h, C, tw, active);
  log.end(pi_, st, units);
  pi_ = log.begin(K_FILTER, st);
  k_fft_cols_mask<T><<<grid, 256, sm, st>>>(n, logn, per, C, tw, mask_tab, active);
  log.end(pi_, st, units);
  pi_ = log.begin(K_FILTER, st);
  k_fft_rows_inv<T><<<grid, 256, sm, st>>>(n, logn, per, C, xstar, x, tw, active);
  log.end(pi_, st, units);
}

template <typename T>
void launch_filter1d(int n, int B, const T* xstar, const T* h, T* x, const double* circ,
                     const int* active, cudaStream_t st, LaunchLog& log) {
  dim3 grid(ceil_div(n, 8), B);
  int pi_ = log.begin(K_FILTER, st);
  k_filter1d<T><<<grid, 256, 0, st>>>(n, xstar, h, x, circ, active);
  log.end(pi_, st, (double)n * log.active_hint);
}

template void launch_filter2d<float>(int, int, const float*, const float*, float*, void*,
                                     const float*, const double*, const int*, cudaStream_t,
                                     LaunchLog&, int);
template void launch_filter2d<double>(int, int, const double*, const double*, double*, void*,
                                      const double*, const double*, const int*, cudaStream_t,
                                      LaunchLog&, int);
template void launch_filter1d<float>(int, int, const float*, const float*, float*,
                                     const double*, const int*, cudaStream_t, LaunchLog&);
template void launch_filter1d<double>(int, int, const double*, const double*, double*,
                                      const double*, const int*, cudaStream_t, LaunchLog&);

}  // namespace nmg
