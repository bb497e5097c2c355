// Neural smoother h = N_theta(b / ||b||) ||b|| (Algorithms 3/4) with a CNN
// N_theta = conv -> ReLU -> ... -> conv, zero 'same' padding (SIMT path for
// the fp64 and fp32 forms).
//
// 2D: one kernel per layer over 16x16 output tiles.  A block stages the
// input tile with a one-pixel halo for all input channels and the layer's
// weights ([cin][tap][cout]) in shared memory; each thread owns a 4-row x
// 1-column strip and 8 output channels (32 fp accumulators).  The first
// layer reads the level vector scaled by 1/||b||, the last layer writes
// ||b|| * output; activations in between are [B][width][n][n].
//
// 1D: all layers fused in one kernel per 256-point segment with a halo of
// layers*(k/2) points per side recomputed.
#include "nmg_internal.h"

namespace nmg {

namespace {

constexpr int CT = 16;      // output tile side
constexpr int IS = CT + 4;  // shared row stride (18 used; 20 avoids bank conflicts)

// MODE 0: first layer (input = level vector / s), 1: hidden layer,
// 2: last layer (COUT == 1, output * s)
template <typename T, int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(256)
k_conv3x3(int n, const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ w,
          const T* __restrict__ bias, const double* __restrict__ snorm,
          const int* __restrict__ active, int tiles_x) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ws = reinterpret_cast<T*>(smem_raw);
  T* xs = ws + CIN * 9 * COUT;
  // ||b||: zero tested on the fp64 bits, the fp32 scale formed once per
  // block (fp64 arithmetic runs at 1/64 of the fp32 rate on this part)
  const long long sbits = __double_as_longlong(snorm[b]);
  const int ty = blockIdx.x / tiles_x, tx = blockIdx.x % tiles_x;
  const int r0 = ty * CT, c0 = tx * CT;
  const size_t plane = (size_t)n * n;
  if ((sbits << 1) == 0) {
    // ||b|| = 0: h = 0 (only the last layer's output is observable)
    if (MODE == 2) {
      for (int p = threadIdx.x; p < CT * CT; p += blockDim.x) {
        int r = r0 + p / CT, c = c0 + p % CT;
        if (r < n && c < n) out[(size_t)b * plane + (size_t)r * n + c] = T(0);
      }
    }
    return;
  }
  for (int i = threadIdx.x; i < CIN * 9 * COUT; i += blockDim.x) ws[i] = w[i];
  __shared__ T scale_s;
  if (MODE != 1 && threadIdx.x == 0) {
    const double s = __longlong_as_double(sbits);
    scale_s = MODE == 0 ? T(1.0 / s) : T(s);
  }
  __syncthreads();
  const T scale = MODE == 0 ? scale_s : T(1);
  const T* inb = in + (size_t)b * plane * CIN;
  for (int i = threadIdx.x; i < CIN * (CT + 2) * (CT + 2); i += blockDim.x) {
    int c = i / ((CT + 2) * (CT + 2));
    int rem = i % ((CT + 2) * (CT + 2));
    int rr = rem / (CT + 2), cc = rem % (CT + 2);
    int gr = r0 - 1 + rr, gc = c0 - 1 + cc;
    T v = T(0);
    if (gr >= 0 && gr < n && gc >= 0 && gc < n) v = inb[(size_t)c * plane + (size_t)gr * n + gc] * scale;
    xs[(c * (CT + 2) + rr) * IS + cc] = v;
  }
  __syncthreads();
  if constexpr (COUT > 1) {
    static_assert(COUT % 8 == 0, "COUT must be a multiple of 8");
    constexpr int NG = COUT / 8;  // channel groups
    // 256 threads = 16 columns x 4 row groups x 4 channel groups when COUT=32
    for (int task = threadIdx.x; task < CT * (CT / 4) * NG; task += blockDim.x) {
      const int col = task & (CT - 1);
      const int rg = (task / CT) % (CT / 4);
      const int cg = task / (CT * (CT / 4));
      T acc[4][8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        T bv = bias[cg * 8 + q];
#pragma unroll
        for (int p = 0; p < 4; ++p) acc[p][q] = bv;
      }
      for (int ci = 0; ci < CIN; ++ci) {
        T xv[6][3];
        const T* xr = xs + (ci * (CT + 2) + rg * 4) * IS + col;
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
          for (int k = 0; k < 3; ++k) xv[r][k] = xr[r * IS + k];
        const T* wr = ws + (ci * 9) * COUT + cg * 8;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
          for (int kx = 0; kx < 3; ++kx) {
            T wv[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) wv[q] = wr[(ky * 3 + kx) * COUT + q];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
              for (int q = 0; q < 8; ++q) acc[p][q] += xv[p + ky][kx] * wv[q];
          }
      }
      T* ob = out + (size_t)b * plane * COUT;
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        int r = r0 + rg * 4 + p, c = c0 + col;
        if (r < n && c < n) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            T v = acc[p][q];
            v = v > T(0) ? v : T(0);  // ReLU after every hidden layer
            ob[(size_t)(cg * 8 + q) * plane + (size_t)r * n + c] = v;
          }
        }
      }
    }
  } else {
    for (int p = threadIdx.x; p < CT * CT; p += blockDim.x) {
      const int rr = p / CT, cc = p % CT;
      T acc = bias[0];
      for (int ci = 0; ci < CIN; ++ci) {
        const T* xr = xs + (ci * (CT + 2) + rr) * IS + cc;
        const T* wr = ws + ci * 9;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
          for (int kx = 0; kx < 3; ++kx) acc += xr[ky * IS + kx] * wr[ky * 3 + kx];
      }
      int r = r0 + rr, c = c0 + cc;
      if (r < n && c < n) out[(size_t)b * plane + (size_t)r * n + c] = acc * scale_s;
    }
  }
}

template <typename T, int CIN, int COUT, int MODE>
void launch_layer(int n, int B, const T* in, T* out, const ConvW<T>& cw, const double* s,
                  const int* active, cudaStream_t st, LaunchLog& log) {
  int tx = ceil_div(n, CT);
  size_t sm = (size_t)(CIN * 9 * COUT + CIN * (CT + 2) * IS) * sizeof(T);
  auto kern = k_conv3x3<T, CIN, COUT, MODE>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  dim3 grid(tx * tx, B);
  int pi_ = log.begin(MODE == 0 ? K_CNN_FIRST : (MODE == 1 ? K_CNN_HIDDEN : K_CNN_LAST), st);
  kern<<<grid, 256, sm, st>>>(n, in, out, cw.w, cw.b, s, active, tx);
  log.end(pi_, st, (double)n * n * log.active_hint);
}

// ---- 1D fused ---------------------------------------------------------------

constexpr int SEG = 256;

template <typename T>
__global__ void __launch_bounds__(256)
k_cnn1d(int n, int layers, int width, int ksize, const T* __restrict__ wp,
        const T* __restrict__ bvec, const double* __restrict__ snorm, T* __restrict__ h,
        const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int half = ksize / 2;
  const int H = layers * half;  // halo per side of the input region
  const int s0 = blockIdx.x * SEG;
  const int len0 = SEG + 2 * H;
  T* bufA = sm;                        // width * len0
  T* bufB = bufA + (size_t)width * len0;  // width * len0
  const double s = snorm[b];
  if (s == 0.0) {
    for (int i = threadIdx.x; i < SEG; i += blockDim.x)
      if (s0 + i < n) h[(size_t)b * n + s0 + i] = T(0);
    return;
  }
  const T inv = T(1.0 / s);
  // input region [s0 - H, s0 + SEG + H), zero outside the grid
  for (int i = threadIdx.x; i < len0; i += blockDim.x) {
    int g = s0 - H + i;
    bufA[i] = (g >= 0 && g < n) ? bvec[(size_t)b * n + g] * inv : T(0);
  }
  __syncthreads();
  T* cur = bufA;
  T* nxt = bufB;
  int cin = 1;
  int lo = s0 - H, len = len0;  // current region
  size_t woff = 0;
  for (int li = 0; li < layers; ++li) {
    const int cout = li == layers - 1 ? 1 : width;
    const int nlo = lo + half, nlen = len - 2 * half;
    const T* W = wp + woff;
    const T* bias = W + (size_t)cout * cin * ksize;
    for (int idx = threadIdx.x; idx < cout * nlen; idx += blockDim.x) {
      int co = idx / nlen, p = idx % nlen;
      int g = nlo + p;
      T acc = bias[co];
      for (int ci = 0; ci < cin; ++ci) {
        const T* wr = W + ((size_t)co * cin + ci) * ksize;
        const T* xr = cur + (size_t)ci * len + p;  // input index p + t for tap t
        for (int t = 0; t < ksize; ++t) acc += wr[t] * xr[t];
      }
      if (li < layers - 1) {
        acc = acc > T(0) ? acc : T(0);
        if (g < 0 || g >= n) acc = T(0);  // zero padding for the next layer
        nxt[(size_t)co * nlen + p] = acc;
      } else if (g >= 0 && g < n) {
        h[(size_t)b * n + g] = acc * T(s);
      }
    }
    __syncthreads();
    woff += (size_t)cout * cin * ksize + cout;
    T* tmp = cur;
    cur = nxt;
    nxt = tmp;
    cin = cout;
    lo = nlo;
    len = nlen;
  }
}

}  // namespace

template <typename T>
void launch_cnn2d_simt(int n, int B, int layers, int width, const ConvW<T>* lw, const T* b,
                       const double* s, T* act0, T* act1, T* h, const int* active,
                       cudaStream_t st, LaunchLog& log) {
  // the build implements the paper-configured 2D smoother: width 32, 3x3
  launch_layer<T, 1, 32, 0>(n, B, b, act0, lw[0], s, active, st, log);
  T* cur = act0;
  T* nxt = act1;
  for (int li = 1; li < layers - 1; ++li) {
    launch_layer<T, 32, 32, 1>(n, B, cur, nxt, lw[li], s, active, st, log);
    T* t = cur;
    cur = nxt;
    nxt = t;
  }
  launch_layer<T, 32, 1, 2>(n, B, cur, h, lw[layers - 1], s, active, st, log);
  (void)width;
}

template <typename T>
void launch_cnn1d(int n, int B, int layers, int width, int ksize, const T* wpacked,
                  const T* b, const double* s, T* h, const int* active, cudaStream_t st,
                  LaunchLog& log) {
  int H = layers * (ksize / 2);
  size_t sm = 2 * (size_t)width * (SEG + 2 * H) * sizeof(T);
  cudaFuncSetAttribute(k_cnn1d<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  dim3 grid(ceil_div(n, SEG), B);
  int pi_ = log.begin(K_CNN_FUSED, st);
  k_cnn1d<T><<<grid, 256, sm, st>>>(n, layers, width, ksize, wpacked, b, s, h, active);
  log.end(pi_, st, (double)n * log.active_hint);
}

template void launch_cnn2d_simt<float>(int, int, int, int, const ConvW<float>*, const float*,
                                       const double*, float*, float*, float*, const int*,
                                       cudaStream_t, LaunchLog&);
template void launch_cnn2d_simt<double>(int, int, int, int, const ConvW<double>*,
                                        const double*, const double*, double*, double*,
                                        double*, const int*, cudaStream_t, LaunchLog&);
template void launch_cnn1d<float>(int, int, int, int, int, const float*, const float*,
                                  const double*, float*, const int*, cudaStream_t, LaunchLog&);
template void launch_cnn1d<double>(int, int, int, int, int, const double*, const double*,
                                   const double*, double*, const int*, cudaStream_t, LaunchLog&);

}  // namespace nmg
