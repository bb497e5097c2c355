// FNO smoother h = N(b / ||b||) ||b|| (Section 3.1; Appendix A), 2D, in the
// level type T (fp32 or fp64 SIMT):
//   lift        z = W_l (b / s) + b_l                      (pointwise, 1 -> c)
//   L layers    z <- ReLU(W * z + B + DFT^{-1}(R . DFT(z)))
//   projection  h = s (W_p . z + b_p)                      (pointwise, c -> 1)
// The spectral part keeps the half spectrum of the real 2D DFT on the modes
// k1 in [0, m) and [n - m, n), k2 in [0, m), and is computed by truncated
// DFT sums (the retained block is small, m <= n / 2):
//   rows    T1[x][k2]  = sum_y z[x][y] e^{-2 pi i k2 y / n}           (k2 < m)
//   columns Zh[k1][k2] = sum_x T1[x][k2] e^{-2 pi i k1 x / n}         (2m rows)
//   modes   Yh[o][k]   = sum_i Zh[i][k] R[blk][i][o][k]               (complex)
//   columns U[x][k2]   = (1/n) sum_k1 Yh[k1][k2] e^{+2 pi i k1 x / n}
//   rows    S[x][y]    = (1/n) (Re U[x][0] + 2 sum_{k2 >= 1} Re(U[x][k2] e^{+2 pi i k2 y / n}))
// which is the real inverse of a half spectrum (the imaginary part of the
// k2 = 0 column is dropped, as a real inverse FFT does).  The last row pass
// is fused into the W-term convolution, whose epilogue adds S, the bias and
// the activation.
//
// Weights per level (device, T, the host layout): lift W [c], b [c]; per
// layer W [c][c][k][k] (PyTorch Conv2d), b [c], R real [2][c][c][m][m],
// R imaginary [2][c][c][m][m] (block 0: k1 = 0..m-1, block 1: k1 =
// n-m..n-1; [block][in][out][k1][k2]); projection W [c], b [1].
#include <algorithm>

#include "nmg_internal.h"

namespace nmg {

namespace {

template <typename T>
struct C2 {
  T x, y;
};

// acc += w * v, both lanes of the register pairs (fma.rn.f32x2)
__device__ __forceinline__ void fma2_acc(float2& acc, float2 w, float2 v) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(d)
      : "l"(*reinterpret_cast<const unsigned long long*>(&w)),
        "l"(*reinterpret_cast<const unsigned long long*>(&v)),
        "l"(*reinterpret_cast<const unsigned long long*>(&acc)));
  acc = *reinterpret_cast<const float2*>(&d);
}

template <typename T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  return C2<T>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// z[img][ch][p] = lw[ch] * b[p] / s + lb[ch]
template <typename T>
__global__ void k_fno_lift(int n, int c, const T* __restrict__ b, const double* __restrict__ snorm,
                           const T* __restrict__ wts, T* __restrict__ z,
                           const int* __restrict__ active) {
  const int img = blockIdx.y;
  if (!active[img]) return;
  const double s = snorm[img];
  if (s == 0.0) return;
  const T inv = T(1.0 / s);
  const size_t plane = (size_t)n * n;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < (int)plane; p += gridDim.x * blockDim.x) {
    const T v = b[(size_t)img * plane + p] * inv;
    for (int ch = 0; ch < c; ++ch) z[((size_t)img * c + ch) * plane + p] = wts[ch] * v + wts[c + ch];
  }
}

// T1[img][ch][x][k2] = sum_y z[img][ch][x][y] tw[(k2 y) mod n]; threadIdx.x =
// k2, threadIdx.y = row within the block's 8 rows
template <typename T>
__global__ void k_fno_dft_rows(int n, int m, int rows, const T* __restrict__ z,
                               const C2<T>* __restrict__ tw, C2<T>* __restrict__ t1,
                               const int* __restrict__ active, int c) {
  const int row = blockIdx.x * blockDim.y + threadIdx.y;  // (img, ch, x) flattened
  const int k2 = threadIdx.x;
  if (row >= rows || k2 >= m) return;
  const int img = row / (c * n);
  if (!active[img]) return;
  const T* zr = z + (size_t)row * n;
  C2<T> acc{T(0), T(0)};
  int idx = 0;  // (k2 * y) mod n
  for (int y = 0; y < n; ++y) {
    const T v = zr[y];
    acc.x += v * tw[idx].x;
    acc.y += v * tw[idx].y;
    idx += k2;
    if (idx >= n) idx -= n;
  }
  t1[(size_t)row * m + k2] = acc;
}

// Zh[img][ch][j][k2] = sum_x T1[img][ch][x][k2] tw[(k1 x) mod n], k1 = j (j < m)
// or n - 2m + j; one block per (img, ch), threads over the 2m x m modes
template <typename T>
__global__ void k_fno_dft_cols(int n, int m, int c, const C2<T>* __restrict__ t1,
                               const C2<T>* __restrict__ tw, C2<T>* __restrict__ zh,
                               const int* __restrict__ active) {
  const int ic = blockIdx.x;
  if (!active[ic / c]) return;
  const C2<T>* src = t1 + (size_t)ic * n * m;
  for (int q = threadIdx.x; q < 2 * m * m; q += blockDim.x) {
    const int j = q / m, k2 = q - j * m;
    const int k1 = j < m ? j : n - 2 * m + j;
    C2<T> acc{T(0), T(0)};
    int idx = 0;
    for (int x = 0; x < n; ++x) {
      const C2<T> p = cmul(src[(size_t)x * m + k2], tw[idx]);
      acc.x += p.x;
      acc.y += p.y;
      idx += k1;
      if (idx >= n) idx -= n;
    }
    zh[(size_t)ic * 2 * m * m + q] = acc;
  }
}

// Yh[img][o][j][k2] = sum_i Zh[img][i][j][k2] R[blk][i][o][j mod m][k2]
template <typename T>
__global__ void k_fno_mix(int m, int c, const C2<T>* __restrict__ zh, const T* __restrict__ rre,
                          const T* __restrict__ rim, C2<T>* __restrict__ yh,
                          const int* __restrict__ active) {
  const int img = blockIdx.y;
  if (!active[img]) return;
  const int modes = 2 * m * m;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < c * modes; t += gridDim.x * blockDim.x) {
    const int o = t / modes, q = t - o * modes;
    const int j = q / m, k2 = q - j * m;
    const int blk = j < m ? 0 : 1, k1 = j < m ? j : j - m;
    C2<T> acc{T(0), T(0)};
    for (int i = 0; i < c; ++i) {
      const size_t r = ((((size_t)blk * c + i) * c + o) * m + k1) * m + k2;
      const C2<T> p = cmul(zh[((size_t)img * c + i) * modes + q], C2<T>{rre[r], rim[r]});
      acc.x += p.x;
      acc.y += p.y;
    }
    yh[((size_t)img * c + o) * modes + q] = acc;
  }
}

// U[img][o][x][k2] = (1/n) sum_j Yh[img][o][j][k2] conj(tw[(k1 x) mod n])
template <typename T>
__global__ void k_fno_idft_cols(int n, int m, int c, const C2<T>* __restrict__ yh,
                                const C2<T>* __restrict__ tw, C2<T>* __restrict__ u,
                                const int* __restrict__ active) {
  const int ic = blockIdx.x;  // (img, channel)
  if (!active[ic / c]) return;
  const C2<T>* src = yh + (size_t)ic * 2 * m * m;
  const T inv_n = T(1) / T(n);
  for (int q = threadIdx.x; q < n * m; q += blockDim.x) {
    const int x = q / m, k2 = q - x * m;
    C2<T> acc{T(0), T(0)};
    for (int j = 0; j < 2 * m; ++j) {
      const int k1 = j < m ? j : n - 2 * m + j;
      const int idx = (int)(((long long)k1 * x) % n);
      const C2<T> w{tw[idx].x, -tw[idx].y};
      const C2<T> p = cmul(src[(size_t)j * m + k2], w);
      acc.x += p.x;
      acc.y += p.y;
    }
    u[(size_t)ic * n * m + q] = C2<T>{acc.x * inv_n, acc.y * inv_n};
  }
}

constexpr int FTW = 16;  // W-term tile: 16 columns
constexpr int FTH = 32;  // x 32 rows (two pixels per thread, rows ty and ty + 16)
constexpr int FOC = 16;  // output channels per block

// input channels staged per pass (the tile with halo, and the block's
// weights for them)
template <typename T> struct FnoCC { static constexpr int value = sizeof(T) == 4 ? 16 : 8; };

template <typename T>
size_t fno_wconv_smem(int ks) {
  constexpr int CC = FnoCC<T>::value;
  return ((size_t)CC * (FTH + ks - 1) * (FTW + ks - 1) + (size_t)CC * ks * ks * FOC) * sizeof(T);
}

// z_out[img][o][p] = ReLU(b[o] + sum_{i,t} W[o][i][t] z_in[img][i][p + t] + S[o][p]),
// S the last (row) pass of the inverse DFT from U.  One block per 16 x 32
// tile, 16 output channels and image; input channels pass through shared
// memory CC at a time together with their weights, laid out [i][tap][16
// outputs] so that a thread reads the 16 weights of a (channel, tap) with
// vector loads and applies them to its two pixels.
template <typename T>
__global__ void __launch_bounds__(256)
k_fno_wconv(int n, int m, int c, int ks, const T* __restrict__ zin, const C2<T>* __restrict__ u,
            const C2<T>* __restrict__ tw, const T* __restrict__ W, const T* __restrict__ bias,
            T* __restrict__ zout, const int* __restrict__ active, int tiles_x) {
  constexpr int CC = FnoCC<T>::value;
  const int img = blockIdx.z;
  if (!active[img]) return;
  extern __shared__ __align__(16) unsigned char fno_smem[];
  const int hw = ks / 2, SW = FTW + ks - 1, SH = FTH + ks - 1, KK = ks * ks;
  T* ws = reinterpret_cast<T*>(fno_smem);  // [CC][KK][FOC]
  T* xs = ws + (size_t)CC * KK * FOC;      // [CC][SH][SW]
  const int y0 = (blockIdx.x / tiles_x) * FTH, x0 = (blockIdx.x % tiles_x) * FTW;
  const int o0 = blockIdx.y * FOC;
  const size_t plane = (size_t)n * n;
  const T* zb = zin + (size_t)img * c * plane;
  const int tx = threadIdx.x % FTW, ty = threadIdx.x / FTW;  // ty < 16
  T acc0[FOC], acc1[FOC];
#pragma unroll
  for (int q = 0; q < FOC; ++q) acc0[q] = acc1[q] = T(0);
  // fp32: output-channel pairs accumulate in packed two-lane FMAs
  // (fma.rn.f32x2), the pixel value duplicated into both lanes
  float2 p0[FOC / 2], p1[FOC / 2];
#pragma unroll
  for (int q = 0; q < FOC / 2; ++q) p0[q] = p1[q] = make_float2(0.f, 0.f);
  const int st_c0 = threadIdx.x / (SH * SW), st_r0 = threadIdx.x - st_c0 * SH * SW;
  const int st_y0 = st_r0 / SW, st_x0 = st_r0 - st_y0 * SW;
  const int st_dy = blockDim.x / SW, st_dx = blockDim.x - st_dy * SW;
  for (int ch0 = 0; ch0 < c; ch0 += CC) {
    __syncthreads();  // the previous pass is done with xs and ws
    {
      // (channel, row, column) of staged element i, stepped along with i
      // (no integer division per element)
      int cc = st_c0, ry = st_y0, rx = st_x0;
      for (int i = threadIdx.x; i < CC * SH * SW; i += blockDim.x) {
        const int yy = y0 - hw + ry, xx = x0 - hw + rx;
        const bool in = ch0 + cc < c && yy >= 0 && yy < n && xx >= 0 && xx < n;
        xs[i] = in ? zb[(size_t)(ch0 + cc) * plane + (size_t)yy * n + xx] : T(0);
        rx += st_dx;
        ry += st_dy;
        if (rx >= SW) {
          rx -= SW;
          ++ry;
        }
        while (ry >= SH) {
          ry -= SH;
          ++cc;
        }
      }
    }
    for (int i = threadIdx.x; i < CC * KK * FOC; i += blockDim.x) {
      const int cc = i / (KK * FOC), r = i - cc * KK * FOC, t = r / FOC, q = r - t * FOC;
      const bool in = ch0 + cc < c && o0 + q < c;
      ws[i] = in ? W[((size_t)(o0 + q) * c + ch0 + cc) * KK + t] : T(0);
    }
    __syncthreads();
    if constexpr (sizeof(T) == 4) {
      for (int cc = 0; cc < CC; ++cc) {
        const float* xc = reinterpret_cast<const float*>(xs) + (size_t)cc * SH * SW + ty * SW + tx;
        const float* wc = reinterpret_cast<const float*>(ws) + (size_t)cc * KK * FOC;
        auto tap = [&](int dy, int dx) {
          const float v0 = xc[dy * SW + dx], v1 = xc[(dy + 16) * SW + dx];
          const float2 d0 = make_float2(v0, v0), d1 = make_float2(v1, v1);
          const float4* wt = reinterpret_cast<const float4*>(wc + (dy * ks + dx) * FOC);
#pragma unroll
          for (int q4 = 0; q4 < FOC / 4; ++q4) {
            const float4 w = wt[q4];
            const float2 wa = make_float2(w.x, w.y), wb = make_float2(w.z, w.w);
            fma2_acc(p0[2 * q4], wa, d0);
            fma2_acc(p0[2 * q4 + 1], wb, d0);
            fma2_acc(p1[2 * q4], wa, d1);
            fma2_acc(p1[2 * q4 + 1], wb, d1);
          }
        };
        if (ks == 3) {
#pragma unroll
          for (int t = 0; t < 9; ++t) tap(t / 3, t % 3);
        } else {
          for (int dy = 0; dy < ks; ++dy)
            for (int dx = 0; dx < ks; ++dx) tap(dy, dx);
        }
      }
    } else {
      for (int cc = 0; cc < CC; ++cc) {
        const T* xc = xs + (size_t)cc * SH * SW + ty * SW + tx;
        const T* wc = ws + (size_t)cc * KK * FOC;
        for (int dy = 0; dy < ks; ++dy)
          for (int dx = 0; dx < ks; ++dx) {
            const T v0 = xc[dy * SW + dx], v1 = xc[(dy + 16) * SW + dx];
            const T* wt = wc + (dy * ks + dx) * FOC;
#pragma unroll
            for (int q = 0; q < FOC; ++q) {
              const T wq = wt[q];
              acc0[q] += wq * v0;
              acc1[q] += wq * v1;
            }
          }
      }
    }
  }
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int q = 0; q < FOC / 2; ++q) {
      acc0[2 * q] = p0[q].x;
      acc0[2 * q + 1] = p0[q].y;
      acc1[2 * q] = p1[q].x;
      acc1[2 * q + 1] = p1[q].y;
    }
  }
  const T inv_n = T(1) / T(n);
  const int x = x0 + tx;
#pragma unroll 1
  for (int half = 0; half < 2; ++half) {
    const int y = y0 + ty + 16 * half;
    if (y >= n || x >= n) continue;
#pragma unroll
    for (int q = 0; q < FOC; ++q) {
      const int o = o0 + q;
      if (o >= c) break;
      // row pass of the inverse DFT at (y, x): row y of U, column x
      const C2<T>* ur = u + (((size_t)img * c + o) * n + y) * m;
      T sp = ur[0].x;
      int idx = x;
      for (int k2 = 1; k2 < m; ++k2) {
        // e^{+2 pi i k2 x / n} = conj(tw[(k2 x) mod n])
        sp += T(2) * (ur[k2].x * tw[idx].x + ur[k2].y * tw[idx].y);
        idx += x;
        if (idx >= n) idx -= n;
      }
      const T v = (half ? acc1[q] : acc0[q]) + bias[o] + sp * inv_n;
      zout[((size_t)img * c + o) * plane + (size_t)y * n + x] = v > T(0) ? v : T(0);
    }
  }
}

// h[img][p] = s (W_p . z[img][:][p] + b_p); h = 0 where ||b|| = 0
template <typename T>
__global__ void k_fno_proj(int n, int c, const T* __restrict__ z, const T* __restrict__ wts,
                           const double* __restrict__ snorm, T* __restrict__ h,
                           const int* __restrict__ active) {
  const int img = blockIdx.y;
  if (!active[img]) return;
  const double s = snorm[img];
  const size_t plane = (size_t)n * n;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < (int)plane; p += gridDim.x * blockDim.x) {
    T acc = wts[c];
    if (s != 0.0) {
      for (int ch = 0; ch < c; ++ch) acc += wts[ch] * z[((size_t)img * c + ch) * plane + p];
      acc *= T(s);
    } else {
      acc = T(0);
    }
    h[(size_t)img * plane + p] = acc;
  }
}

}  // namespace

size_t fno_weights_per_level(int c, int layers, int ks, int m) {
  return 2 * (size_t)c + (size_t)layers * ((size_t)c * c * ks * ks + c + 4 * (size_t)c * c * m * m) +
         (size_t)c + 1;
}

template <typename T>
void launch_fno2d(const FnoDims& dm, int n, int B, const T* wts, const T* tw, const T* b,
                  const double* s, T* z0, T* z1, T* cA, T* cB, T* h, const int* active,
                  cudaStream_t st, LaunchLog& log) {
  const int c = dm.width, m = dm.modes, ks = dm.ksize;
  const size_t plane = (size_t)n * n;
  const C2<T>* twc = reinterpret_cast<const C2<T>*>(tw);
  C2<T>* t1 = reinterpret_cast<C2<T>*>(cA);  // [B][c][n][m], also U
  C2<T>* zh = reinterpret_cast<C2<T>*>(cB);  // [B][c][2m][m] (Zh, then Yh after it)
  C2<T>* yh = zh + (size_t)B * c * 2 * m * m;
  const double units = (double)plane * log.active_hint;
  const dim3 gp((unsigned)std::min<size_t>((plane + 255) / 256, 64), (unsigned)B);
  int pi_ = log.begin(K_CNN_FIRST, st);
  k_fno_lift<T><<<gp, 256, 0, st>>>(n, c, b, s, wts, z0, active);
  log.end(pi_, st, units);
  const size_t per_layer = (size_t)c * c * ks * ks + c + 4 * (size_t)c * c * m * m;
  const int tiles_x = (n + FTW - 1) / FTW, tiles_y = (n + FTH - 1) / FTH;
  const size_t sm = fno_wconv_smem<T>(ks);
  cudaFuncSetAttribute(k_fno_wconv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  T* zi = z0;
  T* zo = z1;
  for (int l = 0; l < dm.layers; ++l) {
    const T* Wl = wts + 2 * c + l * per_layer;
    const T* bl = Wl + (size_t)c * c * ks * ks;
    const T* rre = bl + c;
    const T* rim = rre + 2 * (size_t)c * c * m * m;
    pi_ = log.begin(K_CNN_HIDDEN, st);
    const int rows = B * c * n;
    k_fno_dft_rows<T><<<(rows + 7) / 8, dim3(32, 8), 0, st>>>(n, m, rows, zi, twc, t1, active, c);
    k_fno_dft_cols<T><<<B * c, 128, 0, st>>>(n, m, c, t1, twc, zh, active);
    k_fno_mix<T><<<dim3((unsigned)std::min(64, (c * 2 * m * m + 255) / 256), (unsigned)B), 256, 0,
                   st>>>(m, c, zh, rre, rim, yh, active);
    k_fno_idft_cols<T><<<B * c, 256, 0, st>>>(n, m, c, yh, twc, t1, active);
    k_fno_wconv<T><<<dim3(tiles_x * tiles_y, (c + FOC - 1) / FOC, B), FTW * 16, sm, st>>>(
        n, m, c, ks, zi, t1, twc, Wl, bl, zo, active, tiles_x);
    log.launches += 4;
    log.end(pi_, st, units);
    T* t = zi;
    zi = zo;
    zo = t;
  }
  pi_ = log.begin(K_CNN_LAST, st);
  k_fno_proj<T><<<gp, 256, 0, st>>>(n, c, zi, wts + 2 * c + dm.layers * per_layer, s, h, active);
  log.end(pi_, st, units);
}

template void launch_fno2d<float>(const FnoDims&, int, int, const float*, const float*,
                                  const float*, const double*, float*, float*, float*, float*,
                                  float*, const int*, cudaStream_t, LaunchLog&);
template void launch_fno2d<double>(const FnoDims&, int, int, const double*, const double*,
                                   const double*, const double*, double*, double*, double*,
                                   double*, double*, const int*, cudaStream_t, LaunchLog&);

}  // namespace nmg
