// Outer residual of the refinement form, r = f - A u, with u held in fp64
// and the banded apply done in compensated fp32 ("double-float") arithmetic:
// every operand is split into a pair of floats (hi + lo), products use the
// FMA-based error-free TwoProduct and sums the error-free TwoSum (Knuth),
// following the compensated dot product Dot2 of Ogita, Rump and Oishi,
// "Accurate sum and dot product" (SIAM J. Sci. Comput. 26, 2005).  The
// level-1 coefficients are stored as float pairs of their fp64 values, so
// the result carries about 2^-44 relative error, far below the 1e-6
// tolerance even when ||A|| ||u|| >> ||f||.  The final combination with f,
// the norm ||r|| and the update of u are fp64.
#include "nmg_internal.h"

namespace nmg {

namespace {

struct DF {
  float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// acc += a * x with a, x double-float
__device__ __forceinline__ void df_fma(DF& acc, float ah, float al, float xh, float xl) {
  float p = ah * xh;
  float pe = fmaf(ah, xh, -p);
  pe = fmaf(ah, xl, pe);
  pe = fmaf(al, xh, pe);
  float s, e;
  two_sum(acc.h, p, s, e);
  acc.h = s;
  acc.l += e + pe;
}

__device__ __forceinline__ DF df_norm(DF a) {
  float s = a.h + a.l;
  float e = a.l - (s - a.h);
  return DF{s, e};
}

template <int dummy>
__global__ void __launch_bounds__(256)
k_refine_residual2d(Band2D<float> op, const float* __restrict__ Klo, const float* __restrict__ Mlo,
                    double alpha, const double* __restrict__ u, const float* __restrict__ f,
                    float* __restrict__ r, double* __restrict__ partials,
                    const int* __restrict__ active, int tile, int tiles_x) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  const int n = op.n, wK = op.wK, wM = op.wM;
  const int W = wK > wM ? wK : wM;
  const int ty = blockIdx.x / tiles_x, tx = blockIdx.x % tiles_x;
  const int r0 = ty * tile, c0 = tx * tile;
  const int RH = min(tile, n - r0), RW = min(tile, n - c0);
  const int XH = RH + 2 * W, XW = RW + 2 * W;
  const int nk = 2 * wK + 1, nm = 2 * wM + 1;
  DF* xs = reinterpret_cast<DF*>(smem_raw);
  DF* tk = xs + XH * XW;
  DF* tm = tk + (RH + 2 * wK) * RW;
  // banded coefficients (hi, lo) of the tile's columns and rows
  DF* kcol = tm + (RH + 2 * wM) * RW;
  DF* mcol = kcol + RW * nk;
  DF* krow = mcol + RW * nm;
  DF* mrow = krow + RH * nk;
  const size_t plane = (size_t)n * n;
  const double* ub = u + (size_t)b * plane;
  for (int idx = threadIdx.x; idx < XH * XW; idx += blockDim.x) {
    int a = idx / XW, c = idx % XW;
    int gr = r0 - W + a, gc = c0 - W + c;
    double v = (gr >= 0 && gr < n && gc >= 0 && gc < n) ? ub[(size_t)gr * n + gc] : 0.0;
    float hi = (float)v;
    xs[idx] = DF{hi, (float)(v - (double)hi)};
  }
  for (int idx = threadIdx.x; idx < RW * nk; idx += blockDim.x) {
    const size_t g = (size_t)(c0 + idx / nk) * nk + idx % nk;
    kcol[idx] = DF{op.Kd[g], Klo[g]};
  }
  for (int idx = threadIdx.x; idx < RW * nm; idx += blockDim.x) {
    const size_t g = (size_t)(c0 + idx / nm) * nm + idx % nm;
    mcol[idx] = DF{op.Md[g], Mlo[g]};
  }
  for (int idx = threadIdx.x; idx < RH * nk; idx += blockDim.x) {
    const size_t g = (size_t)(r0 + idx / nk) * nk + idx % nk;
    krow[idx] = DF{op.Kd[g], Klo[g]};
  }
  for (int idx = threadIdx.x; idx < RH * nm; idx += blockDim.x) {
    const size_t g = (size_t)(r0 + idx / nm) * nm + idx % nm;
    mrow[idx] = DF{op.Md[g], Mlo[g]};
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < (RH + 2 * wK) * RW; idx += blockDim.x) {
    int a = idx / RW, j = idx % RW;
    int gj = c0 + j;
    (void)gj;
    DF acc{0.f, 0.f};
    const DF* kc = kcol + j * nk;
    const DF* xr = xs + (a + W - wK) * XW + (j + W - wK);
    for (int d = 0; d < nk; ++d) df_fma(acc, kc[d].h, kc[d].l, xr[d].h, xr[d].l);
    tk[idx] = df_norm(acc);
  }
  for (int idx = threadIdx.x; idx < (RH + 2 * wM) * RW; idx += blockDim.x) {
    int a = idx / RW, j = idx % RW;
    int gj = c0 + j;
    (void)gj;
    DF acc{0.f, 0.f};
    const DF* mc = mcol + j * nm;
    const DF* xr = xs + (a + W - wM) * XW + (j + W - wM);
    for (int d = 0; d < nm; ++d) df_fma(acc, mc[d].h, mc[d].l, xr[d].h, xr[d].l);
    tm[idx] = df_norm(acc);
  }
  __syncthreads();
  double ss = 0.0;
  for (int idx = threadIdx.x; idx < RH * RW; idx += blockDim.x) {
    int i = idx / RW, j = idx % RW;
    int gi = r0 + i, gj = c0 + j;
    DF zk{0.f, 0.f}, zm{0.f, 0.f};
    const DF* kr = krow + i * nk;
    const DF* mr = mrow + i * nm;
    for (int d = 0; d < nk; ++d) {
      DF t = tk[(i + d) * RW + j];
      df_fma(zk, kr[d].h, kr[d].l, t.h, t.l);
    }
    for (int d = 0; d < nm; ++d) {
      DF t = tm[(i + d) * RW + j];
      df_fma(zm, mr[d].h, mr[d].l, t.h, t.l);
    }
    size_t gidx = (size_t)b * plane + (size_t)gi * n + gj;
    double az = alpha * ((double)zm.h + (double)zm.l) + ((double)zk.h + (double)zk.l);
    double rv = (double)f[gidx] - az;
    r[gidx] = (float)rv;
    ss += rv * rv;
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    partials[(size_t)b * gridDim.x + blockIdx.x] = s;
  }
}

}  // namespace

void refine_residual2d(const Band2D<float>& hi, const float* Kd_lo, const float* Md_lo,
                       double alpha, int B, const double* u, const float* f, float* r,
                       double* partials, int* ntiles, const int* active, cudaStream_t st,
                       LaunchLog& log, int tile_req) {
  const int W = hi.wK > hi.wM ? hi.wK : hi.wM;
  int tile = tile_req > 0 ? tile_req : 32;
  if (tile > hi.n) tile = hi.n;
  auto smem = [&](int t) {
    return ((size_t)(t + 2 * W) * (t + 2 * W) + (size_t)(t + 2 * hi.wK) * t +
            (size_t)(t + 2 * hi.wM) * t + (size_t)2 * t * (2 * hi.wK + 1 + 2 * hi.wM + 1)) *
           sizeof(DF);
  };
  while (tile > 4 && smem(tile) > 200 * 1024) tile /= 2;
  while (tile < hi.n && (long long)ceil_div(hi.n, tile) * ceil_div(hi.n, tile) > 4096) tile *= 2;
  int tx = ceil_div(hi.n, tile);
  size_t sm = smem(tile);
  cudaFuncSetAttribute(k_refine_residual2d<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  dim3 grid(tx * tx, B);
  int pi_ = log.begin(K_REFINE_RESIDUAL, st);
  k_refine_residual2d<0><<<grid, 256, sm, st>>>(hi, Kd_lo, Md_lo, alpha, u, f, r, partials, active,
                                                tile, tx);
  if (ntiles) *ntiles = tx * tx;
  log.end(pi_, st, (double)hi.n * hi.n * log.active_hint);
}

}  // namespace nmg
