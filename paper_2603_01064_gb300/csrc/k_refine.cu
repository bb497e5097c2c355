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

// ---------------------------------------------------------------------------
// Stencil form for a Toeplitz fine level with M = I (every fine level built
// from taps): r = f - (alpha u + K U K^T) with the stencil's double-float
// pairs in kernel parameters.  Persistent blocks prefetch the next tile's u
// (fp64, with halo) and f with cp.async into a double buffer; u is split
// into float pairs once per staged value with integer operations (fp64
// arithmetic runs at 1/64 of the fp32 rate on this GPU); each pass keeps a
// register window of S + 2 WK pairs for S outputs.
// ---------------------------------------------------------------------------
template <int WK>
struct RefineArgs {
  int n;
  float ah, al;  // alpha as a float pair
  float sKh[2 * WK + 1], sKl[2 * WK + 1];
  // the same as two-lane pairs (c, c) for the packed strip kernel; nKh = -sKh
  float2 kh2[2 * WK + 1], nkh2[2 * WK + 1], kl2[2 * WK + 1];
};

template <int WK> struct RSeg { static constexpr int value = WK <= 8 ? 8 : 4; };

struct RefineGeom {
  int XH, XW, XPD, XPF, YP, TKH, TP, words;  // words of 4 bytes
  __host__ __device__ RefineGeom(int tile, int WK, int S) {
    XH = tile + 2 * WK;
    XW = tile + 2 * WK;
    XPD = (1 + XW + 1) / 2 * 2;                       // doubles per staged row (offset <= 1)
    const int reach = (tile + S - 1) / S * S + 2 * WK;  // window reach of the row pass
    XPF = (reach + 3) / 4 * 4;
    if (((XPF / 4) & 1) == 0) XPF += 4;               // odd number of 16-byte chunks
    YP = (3 + tile + 3) / 4 * 4;
    TKH = (tile + S - 1) / S * S + 2 * WK;
    TP = ((tile + S - 1) / S * S) | 1;
    words = 2 * 2 * XH * XPD + 2 * tile * YP + 2 * XH * XPF + 2 * TKH * TP;
  }
};

__device__ __forceinline__ void cp_async_16r(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src),
               "r"(valid ? 16u : 0u)
               : "memory");
}

// v = hi + lo with hi = v truncated to 24 significant bits (exact in fp32)
// and lo the rest rounded to fp32 (~2^-47 relative), by integer operations;
// values below 2^-74 in magnitude split to (0, 0), values beyond the fp32
// range to (+-inf, 0).
__device__ __forceinline__ void split_double(double v, float& hi, float& lo) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((u >> 52) & 0x7FF);
  const unsigned sign = (unsigned)(u >> 63) << 31;
  if (e < 949) {  // also zero
    hi = 0.f;
    lo = 0.f;
    return;
  }
  if (e > 1150) {  // beyond fp32 range: an infinite residual (reported as diverged)
    hi = __uint_as_float(sign | 0x7F800000u);
    lo = 0.f;
    return;
  }
  const unsigned m_hi = (unsigned)((u >> 29) & 0x7FFFFFu);
  const unsigned m_lo = (unsigned)(u & 0x1FFFFFFFu);
  hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | m_hi);
  const float scale = __uint_as_float((unsigned)(e - 948) << 23);  // 2^(e - 1075)
  lo = __uint_as_float(sign | __float_as_uint(__uint2float_rn(m_lo) * scale));
}

template <int WK>
__global__ void __launch_bounds__(256)
k_refine_pipe(RefineArgs<WK> op, int B, const double* __restrict__ u, const float* __restrict__ f,
              float* __restrict__ r, double* __restrict__ partials,
              const int* __restrict__ active, int tile, int tiles_x) {
  constexpr int S = RSeg<WK>::value, NW = S + 2 * WK;
  const RefineGeom g(tile, WK, S);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float red[32];
  double* ubuf = reinterpret_cast<double*>(smem_raw);  // [2][XH][XPD]
  float* fbuf = reinterpret_cast<float*>(ubuf + 2 * g.XH * g.XPD);  // [2][tile][YP]
  float* xh = fbuf + 2 * tile * g.YP;                  // [XH][XPF]
  float* xl = xh + g.XH * g.XPF;
  float* tkh = xl + g.XH * g.XPF;                      // [TKH][TP]
  float* tkl = tkh + g.TKH * g.TP;
  const int n = op.n;
  const int per_img = tiles_x * tiles_x;
  const int total = B * per_img;
  const size_t plane = (size_t)n * n;
  auto next_valid = [&](int t) {
    while (t < total && !active[t / per_img]) t += gridDim.x;
    return t;
  };
  auto origin = [&](int t, int& b, int& ty, int& tx, int& r0, int& c0, int& RH, int& RW) {
    b = t / per_img;
    const int tt = t - b * per_img;
    ty = tt / tiles_x;
    tx = tt - ty * tiles_x;
    r0 = ty * tile;
    c0 = tx * tile;
    RH = min(tile, n - r0);
    RW = min(tile, n - c0);
  };
  auto prefetch = [&](int t, int buf) {
    if (t < total) {
      int b, ty, tx, r0, c0, RH, RW;
      origin(t, b, ty, tx, r0, c0, RH, RW);
      const double* ub = u + (size_t)b * plane;
      const int cs = (c0 - WK) & ~1;
      const int uch = g.XPD / 2;
      double* ud = ubuf + buf * g.XH * g.XPD;
      for (int i = threadIdx.x; i < g.XH * uch; i += blockDim.x) {
        const int a = i / uch, ch = i - a * uch;
        const int gr = r0 - WK + a, gc = cs + 2 * ch;
        const bool in = gr >= 0 && gr < n && gc >= 0 && gc < n;
        cp_async_16r(ud + a * g.XPD + 2 * ch, in ? ub + (size_t)gr * n + gc : ub, in);
      }
      const float* fb = f + (size_t)b * plane;
      const int cy = c0 & ~3;
      const int fch = g.YP / 4;
      float* fd = fbuf + buf * tile * g.YP;
      for (int i = threadIdx.x; i < RH * fch; i += blockDim.x) {
        const int a = i / fch, ch = i - a * fch;
        const int gr = r0 + a, gc = cy + 4 * ch;
        const bool in = gr < n && gc < n;
        cp_async_16r(fd + a * g.YP + 4 * ch, in ? fb + (size_t)gr * n + gc : fb, in);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  int cur = next_valid(blockIdx.x);
  int nxt = cur < total ? next_valid(cur + gridDim.x) : total;
  prefetch(cur, 0);
  prefetch(nxt, 1);
  for (int k = 0; cur < total; ++k) {
    const int buf = k & 1;
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncthreads();
    int b, ty, tx, r0, c0, RH, RW;
    origin(cur, b, ty, tx, r0, c0, RH, RW);
    const int XH = RH + 2 * WK, XW = RW + 2 * WK;
    const int ofs = (c0 - WK) - ((c0 - WK) & ~1);
    const int oy = c0 - (c0 & ~3);
    const double* us = ubuf + buf * g.XH * g.XPD;
    const float* fs = fbuf + buf * tile * g.YP;
    // split the staged u into float pairs (logical column c at physical c)
    for (int i = threadIdx.x; i < XH * XW; i += blockDim.x) {
      const int a = i / XW, c = i - a * XW;
      float h, l;
      split_double(us[a * g.XPD + c + ofs], h, l);
      xh[a * g.XPF + c] = h;
      xl[a * g.XPF + c] = l;
    }
    __syncthreads();
    // row pass: t[a][j] = sum_d K[d] u[a][j + d] (double-float)
    const int nseg_r = (RW + S - 1) / S;
    for (int item = threadIdx.x; item < XH * nseg_r; item += blockDim.x) {
      const int a = item % XH, P = (item / XH) * S;
      float wh[NW], wl[NW];
      const float* rh = xh + a * g.XPF + P;
      const float* rl = xl + a * g.XPF + P;
#pragma unroll
      for (int q = 0; q < NW / 4; ++q) {
        const float4 vh = *reinterpret_cast<const float4*>(rh + 4 * q);
        const float4 vl = *reinterpret_cast<const float4*>(rl + 4 * q);
        wh[4 * q] = vh.x; wh[4 * q + 1] = vh.y; wh[4 * q + 2] = vh.z; wh[4 * q + 3] = vh.w;
        wl[4 * q] = vl.x; wl[4 * q + 1] = vl.y; wl[4 * q + 2] = vl.z; wl[4 * q + 3] = vl.w;
      }
      DF acc[S];
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) acc[s2] = DF{0.f, 0.f};
#pragma unroll
      for (int d = 0; d < 2 * WK + 1; ++d)
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) df_fma(acc[s2], op.sKh[d], op.sKl[d], wh[s2 + d], wl[s2 + d]);
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) {
        const DF t = df_norm(acc[s2]);
        tkh[a * g.TP + P + s2] = t.h;
        tkl[a * g.TP + P + s2] = t.l;
      }
    }
    __syncthreads();
    // column pass, alpha u, residual
    const int nseg_c = (RH + S - 1) / S;
    float ss = 0.f;
    for (int item = threadIdx.x; item < RW * nseg_c; item += blockDim.x) {
      const int j = item % RW, i0 = (item / RW) * S;
      float th[NW], tl[NW];
#pragma unroll
      for (int q = 0; q < NW; ++q) {
        th[q] = tkh[(i0 + q) * g.TP + j];
        tl[q] = tkl[(i0 + q) * g.TP + j];
      }
      DF z[S];
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) z[s2] = DF{0.f, 0.f};
#pragma unroll
      for (int d = 0; d < 2 * WK + 1; ++d)
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) df_fma(z[s2], op.sKh[d], op.sKl[d], th[s2 + d], tl[s2 + d]);
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) {
        const int i = i0 + s2;
        if (i >= RH) break;
        // A u = alpha u + K U K^T, then r = f - A u (double-float, rounded once)
        const int xc = (i + WK) * g.XPF + j + WK;
        df_fma(z[s2], op.ah, op.al, xh[xc], xl[xc]);
        const DF az = df_norm(z[s2]);
        float s, e;
        two_sum(fs[i * g.YP + j + oy], -az.h, s, e);
        const float rv = s + (e - az.l);
        r[(size_t)b * plane + (size_t)(r0 + i) * n + (c0 + j)] = rv;
        ss = fmaf(rv, rv, ss);
      }
    }
    if (partials) {
      // fp32 tree over the tile (fp64 adds run at 1/64 of the fp32 rate and
      // stalled the whole block on this reduction); fp64 across tiles
      float v = ss;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
      __syncthreads();
      if (threadIdx.x == 0) {
        float sum = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
        partials[(size_t)b * per_img + ty * tiles_x + tx] = (double)sum;
      }
    }
    __syncthreads();  // the buffer, the split tile and red[] are free
    const int after = nxt < total ? next_valid(nxt + gridDim.x) : total;
    prefetch(after, buf);
    cur = nxt;
    nxt = after;
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

int num_sms_refine() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms;
}

template <int WK>
RefineArgs<WK> refine_args(const StencilHost<double>& sd, double alpha, int n) {
  RefineArgs<WK> a{};
  a.n = n;
  a.ah = (float)alpha;
  a.al = (float)(alpha - (double)a.ah);
  for (int d = 0; d <= 2 * sd.wK; ++d) {
    const double v = sd.sK[d];
    a.sKh[WK - sd.wK + d] = (float)v;
    a.sKl[WK - sd.wK + d] = (float)(v - (double)(float)v);
  }
  for (int d = 0; d <= 2 * WK; ++d) {
    a.kh2[d] = make_float2(a.sKh[d], a.sKh[d]);
    a.nkh2[d] = make_float2(-a.sKh[d], -a.sKh[d]);
    a.kl2[d] = make_float2(a.sKl[d], a.sKl[d]);
  }
  return a;
}

// two-lane fp32 arithmetic (add/sub/mul/fma.rn.f32x2): each lane of the
// strip kernel owns two adjacent columns, whose double-float operations are
// independent and run as one packed instruction each
__device__ __forceinline__ unsigned long long f2u(float2 v) {
  return *reinterpret_cast<unsigned long long*>(&v);
}
__device__ __forceinline__ float2 u2f(unsigned long long v) {
  return *reinterpret_cast<float2*>(&v);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)));
  return u2f(d);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)));
  return u2f(d);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)));
  return u2f(d);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)), "l"(f2u(c)));
  return u2f(d);
}
// (h, l) += (ah + al)(xh + xl) on two lanes: the operations of df_fma with
// p kept negated (pn = -ah xh, exact in sign), so that TwoProduct's error
// term is fma(ah, xh, pn) and TwoSum subtracts pn; bitwise the same results
__device__ __forceinline__ void df_fma2(float2& h, float2& l, float2 ah, float2 nah, float2 al,
                                        float2 xh, float2 xl) {
  const float2 pn = mul2(nah, xh);
  float2 pe = fma2(ah, xh, pn);
  pe = fma2(ah, xl, pe);
  pe = fma2(al, xh, pe);
  const float2 s = sub2(h, pn);
  const float2 bb = sub2(s, h);
  const float2 e = sub2(sub2(h, sub2(s, bb)), add2(pn, bb));
  h = s;
  l = add2(l, add2(e, pe));
}
__device__ __forceinline__ void df_norm2(float2& h, float2& l) {
  const float2 s = add2(h, l);
  l = sub2(l, sub2(s, h));
  h = s;
}

// ---------------------------------------------------------------------------
// Strip form of the same residual for stencils of half-width <= 8 and n a
// multiple of 64: one warp computes kRsH consecutive rows of a 64-column
// strip of one right-hand side, lane j owning columns 2j and 2j + 1.  Input
// rows stream through a warp-private ring (cp.async, kRsPF rows ahead); each
// staged row of u is split into float pairs once, into a one-row buffer the
// lanes' windows read; the double-float row-pass outputs of the last 2 WK + 1
// rows stay in registers, shifted down by one row per input row (one loop
// body: the double-float column pass is too long to specialise per ring
// phase), so no warp waits on another.
// ---------------------------------------------------------------------------
constexpr int kRsH = 32;      // output rows per warp unit
constexpr int kRsWarps = 4;   // warps per block
constexpr int kRsPF = 6;      // rows staged ahead
constexpr int kRsRing = 16;   // staged rows per warp: > kRsPF + max WK
constexpr int kRsHalo = 8;    // staged halo columns per side (>= WK)
constexpr int kRsSW = 64;     // columns per strip
constexpr int kRsXW = kRsSW + 2 * kRsHalo;  // staged u row (doubles)
// per-warp shared memory in 4-byte words: u ring, split row (hi, lo), f ring
constexpr int kRsWords = kRsRing * kRsXW * 2 + 2 * kRsXW + kRsRing * kRsSW;

template <int WK>
__global__ void __launch_bounds__(32 * kRsWarps, 2)
k_refine_strip(RefineArgs<WK> op, int B, const double* __restrict__ u,
               const float* __restrict__ f, float* __restrict__ r,
               double* __restrict__ partials, const int* __restrict__ active) {
  static_assert(WK <= kRsHalo && kRsRing > kRsPF + WK, "ring too short");
  constexpr int P = 2 * WK + 1;
  extern __shared__ __align__(16) float rs_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* uring = reinterpret_cast<double*>(rs_smem + wib * kRsWords);  // [ring][XW]
  float* xh = reinterpret_cast<float*>(uring + kRsRing * kRsXW);         // [XW]
  float* xl = xh + kRsXW;                                                // [XW]
  float* fring = xl + kRsXW;                                             // [ring][SW]
  const int n = op.n;
  const int ns = n / kRsSW, upi = ns * (n / kRsH);
  const int total = B * upi;
  const size_t plane = (size_t)n * n;

  for (int unit = blockIdx.x * kRsWarps + wib; unit < total; unit += gridDim.x * kRsWarps) {
    const int b = unit / upi;
    if (!active[b]) continue;  // warp-uniform
    const int rem = unit - b * upi;
    const int c0 = (rem % ns) * kRsSW, i0 = (rem / ns) * kRsH;
    const int alo = i0 - WK, ahi = i0 + kRsH + WK;  // input rows
    const double* ub = u + (size_t)b * plane;
    const float* fb = f + (size_t)b * plane;
    auto stage = [&](int a) {
      if (a < ahi) {
        const int slot = (a - alo) % kRsRing;
        const bool rin = a >= 0 && a < n;
        double* ud = uring + slot * kRsXW;
        for (int ch = lane; ch < kRsXW / 2; ch += 32) {
          const int gc = c0 - kRsHalo + 2 * ch;
          const bool in = rin && gc >= 0 && gc < n;
          cp_async_16r(ud + 2 * ch, in ? ub + (size_t)a * n + gc : ub, in);
        }
        if (a >= i0 && a < i0 + kRsH) {
          float* fd = fring + slot * kRsSW;
          for (int ch = lane; ch < kRsSW / 4; ch += 32)
            cp_async_16r(fd + 4 * ch, fb + (size_t)a * n + c0 + 4 * ch, true);
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
#pragma unroll
    for (int k = 0; k < kRsPF; ++k) stage(alo + k);

    // row-pass outputs of input rows a - 2 WK .. a, double-float, the lane's
    // two columns as pairs
    float2 twh[P], twl[P];
#pragma unroll
    for (int k = 0; k < P; ++k) twh[k] = twl[k] = make_float2(0.f, 0.f);
    float ss = 0.f;
#pragma unroll 1
    for (int a = alo; a < ahi; ++a) {
      asm volatile("cp.async.wait_group %0;" ::"n"(kRsPF - 1) : "memory");
      __syncwarp();
      stage(a + kRsPF);
      // split the staged row once (the previous row's window reads are
      // ordered before this by the barrier above)
      const double* us = uring + ((a - alo) % kRsRing) * kRsXW;
      for (int k = lane; k < kRsXW; k += 32) {
        float h, l;
        split_double(us[k], h, l);
        xh[k] = h;
        xl[k] = l;
      }
      __syncwarp();
      // row pass: t[c] = sum_d K[d] u[a][c0 + 2 lane + c + d - WK]
      float wh[2 + 2 * kRsHalo], wl[2 + 2 * kRsHalo];
#pragma unroll
      for (int k2 = 0; k2 < 1 + kRsHalo; ++k2) {
        const float2 vh = *reinterpret_cast<const float2*>(xh + 2 * lane + 2 * k2);
        const float2 vl = *reinterpret_cast<const float2*>(xl + 2 * lane + 2 * k2);
        wh[2 * k2] = vh.x; wh[2 * k2 + 1] = vh.y;
        wl[2 * k2] = vl.x; wl[2 * k2 + 1] = vl.y;
      }
      float2 ah2 = make_float2(0.f, 0.f), al2 = make_float2(0.f, 0.f);
#pragma unroll
      for (int d = 0; d < P; ++d) {
        const int j = kRsHalo - WK + d;
        df_fma2(ah2, al2, op.kh2[d], op.nkh2[d], op.kl2[d], make_float2(wh[j], wh[j + 1]),
                make_float2(wl[j], wl[j + 1]));
      }
      df_norm2(ah2, al2);
#pragma unroll
      for (int k = 0; k + 1 < P; ++k) {
        twh[k] = twh[k + 1];
        twl[k] = twl[k + 1];
      }
      twh[P - 1] = ah2;
      twl[P - 1] = al2;
      if (a >= i0 + WK) {
        // column pass for output row i = a - WK, alpha u, r = f - A u
        const int i = a - WK;
        float2 zh2 = make_float2(0.f, 0.f), zl2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int d = 0; d < P; ++d)
          df_fma2(zh2, zl2, op.kh2[d], op.nkh2[d], op.kl2[d], twh[d], twl[d]);
        DF z[2] = {DF{zh2.x, zl2.x}, DF{zh2.y, zl2.y}};
        const int slot = (i - alo) % kRsRing;
        const double2 uc = *reinterpret_cast<const double2*>(uring + slot * kRsXW + kRsHalo + 2 * lane);
        const float2 fv = *reinterpret_cast<const float2*>(fring + slot * kRsSW + 2 * lane);
        float rv[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          float h, l;
          split_double(c ? uc.y : uc.x, h, l);
          df_fma(z[c], op.ah, op.al, h, l);
          const DF az = df_norm(z[c]);
          float s2, e;
          two_sum(c ? fv.y : fv.x, -az.h, s2, e);
          rv[c] = s2 + (e - az.l);
          ss = fmaf(rv[c], rv[c], ss);
        }
        *reinterpret_cast<float2*>(r + (size_t)b * plane + (size_t)i * n + c0 + 2 * lane) =
            make_float2(rv[0], rv[1]);
      }
    }
    __syncwarp();  // every lane is done with the ring before the next unit restages it
    if (partials) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      if (lane == 0) partials[(size_t)b * upi + rem] = (double)ss;
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Strip form for wide stencils (half-width 9..32, n a multiple of 64): one
// warp computes a chunk of consecutive output rows of a 64-column strip (the
// launch cuts every strip into kch chunks so that the units spread evenly
// over the SMs), lane j owning columns 2j and 2j + 1 (two-lane packed
// double-float operations).  Input rows stream through a warp-private
// cp.async ring; each staged row is split into float pairs once; the row
// pass reads the lane's window from that split row.  The double-float
// row-pass outputs of the last 2 W + 1 rows live in a warp-private
// shared-memory ring (each lane reads back only its own columns, so the
// ring needs no barrier), and the column pass of output row i = a - W
// gathers them from there.  f is staged with u for the output rows, and
// g = f - alpha u of row a (double-float) is kept in a second ring of W + 1
// rows until row a's column pass, so no global load waits inside the row
// loop and no staged row has to outlive the prefetch window.
// ---------------------------------------------------------------------------
// staged rows ahead.  The warps are latency-bound, so warps per SM matter
// more than prefetch depth: two rows ahead, the split row written over its
// own staged doubles and f read straight from global memory leave room for
// 8 warps at half-width 16 (measured per 64-RHS 512x512 launch: 0.69 ms;
// 7 warps: 0.73 ms; 6 warps with 4 rows ahead: 0.93 ms)
constexpr int kRwPF = 2;
constexpr int kRwRing = kRwPF + 2;
template <int W> struct RwWarps { static constexpr int value = W <= 16 ? 8 : 4; };
template <int W> struct RwGeom {
  static constexpr int XW = kRsSW + 2 * W;                   // staged u row (doubles)
  static constexpr int P = 2 * W + 1;                        // row-pass ring rows
  static constexpr int Q = W + 1;                            // g ring rows
  // per-warp shared memory in 4-byte words: t ring and g ring (float4 per
  // lane and row), u ring (a slot's XW doubles are replaced by its split
  // row, XW hi floats then XW lo floats, once the row is current)
  static constexpr int words = (P + Q) * 128 + kRwRing * XW * 2;
};

template <int W>
__global__ void __launch_bounds__(32 * RwWarps<W>::value, 1)
k_refine_wide(RefineArgs<W> op, int B, const double* __restrict__ u,
              const float* __restrict__ f, float* __restrict__ r,
              double* __restrict__ partials, const int* __restrict__ active, int kch) {
  using G = RwGeom<W>;
  constexpr int XW = G::XW, P = G::P, Q = G::Q;
  extern __shared__ __align__(16) float rw_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* wbase = rw_smem + (size_t)wib * G::words;
  float4* tring = reinterpret_cast<float4*>(wbase);                 // [P][32 lanes]
  float4* gring = tring + P * 32;                                   // [Q][32 lanes]
  double* uring = reinterpret_cast<double*>(gring + Q * 32);        // [ring][XW]
  const int n = op.n;
  const int ns = n / kRsSW, upi = ns * kch, hu = (n + kch - 1) / kch;
  const int total = B * upi;
  const size_t plane = (size_t)n * n;

  // units dealt block-cyclically: every SM gets the same number to within one
  for (int j = wib;; j += RwWarps<W>::value) {
    const int unit = j * gridDim.x + blockIdx.x;
    if (unit >= total) break;
    const int b = unit / upi;
    if (!active[b]) continue;  // warp-uniform
    const int rem = unit - b * upi;
    const int c0 = (rem % ns) * kRsSW, i0 = (rem / ns) * hu;
    const int H = min(hu, n - i0);                  // output rows of this unit
    const int alo = i0 - W, ahi = i0 + H + W;  // input rows
    const double* ub = u + (size_t)b * plane;
    const float* fb = f + (size_t)b * plane;
    auto stage = [&](int a) {
      if (a < ahi) {
        const int slot = (a - alo) % kRwRing;
        const bool rin = a >= 0 && a < n;
        double* ud = uring + slot * XW;
        for (int ch = lane; ch < XW / 2; ch += 32) {
          const int gc = c0 - W + 2 * ch;
          const bool in = rin && gc >= 0 && gc < n;
          cp_async_16r(ud + 2 * ch, in ? ub + (size_t)a * n + gc : ub, in);
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
#pragma unroll
    for (int k = 0; k < kRwPF; ++k) stage(alo + k);
    float ss = 0.f;
#pragma unroll 1
    for (int a = alo; a < ahi; ++a) {
      asm volatile("cp.async.wait_group %0;" ::"n"(kRwPF - 1) : "memory");
      __syncwarp();
      stage(a + kRwPF);
      // f of this row's two columns, read now and used after the row pass
      const bool grow = a >= i0 && a < i0 + H;  // warp-uniform
      float2 fv = make_float2(0.f, 0.f);
      if (grow) fv = __ldg(reinterpret_cast<const float2*>(fb + (size_t)a * n + c0 + 2 * lane));
      // split the staged row once, over its own slot: every lane reads its
      // doubles first, then the slot holds XW hi floats and XW lo floats
      // (the slot is restaged only kRwPF rows on, after this row is done)
      double* us = uring + ((a - alo) % kRwRing) * XW;
      constexpr int PER = (XW + 31) / 32;
      double uv[PER];
#pragma unroll
      for (int j = 0; j < PER; ++j) uv[j] = lane + 32 * j < XW ? us[lane + 32 * j] : 0.0;
      __syncwarp();
      float* xh = reinterpret_cast<float*>(us);
      float* xl = xh + XW;
#pragma unroll
      for (int j = 0; j < PER; ++j)
        if (lane + 32 * j < XW) {
          float h, l;
          split_double(uv[j], h, l);
          xh[lane + 32 * j] = h;
          xl[lane + 32 * j] = l;
        }
      __syncwarp();
      // row pass: t[c] = sum_d K[d] u[a][c0 + 2 lane + c + d - W], the
      // lane's window read as aligned pairs (odd taps take the halves of
      // two neighbouring pairs)
      float2 th = make_float2(0.f, 0.f), tl = make_float2(0.f, 0.f);
      {
        const float2* h2 = reinterpret_cast<const float2*>(xh) + lane;
        const float2* l2 = reinterpret_cast<const float2*>(xl) + lane;
        float2 ph = h2[0], pl = l2[0];
        // W = 32: partial unrolling keeps the window loads from being all
        // hoisted into registers (the kernel then spills)
#pragma unroll(W > 16 ? 8 : W)
        for (int k = 0; k < W; ++k) {
          const float2 qh = h2[k + 1], ql = l2[k + 1];
          df_fma2(th, tl, op.kh2[2 * k], op.nkh2[2 * k], op.kl2[2 * k], ph, pl);
          df_fma2(th, tl, op.kh2[2 * k + 1], op.nkh2[2 * k + 1], op.kl2[2 * k + 1],
                  make_float2(ph.y, qh.x), make_float2(pl.y, ql.x));
          ph = qh;
          pl = ql;
        }
        df_fma2(th, tl, op.kh2[2 * W], op.nkh2[2 * W], op.kl2[2 * W], ph, pl);
      }
      df_norm2(th, tl);
      const int sa = (a - alo) % P;
      tring[sa * 32 + lane] = make_float4(th.x, th.y, tl.x, tl.y);
      if (grow) {
        // g = f - alpha u of this row (double-float), kept until its column
        // pass W rows on; u's pairs are the split row's (index W + 2 lane)
        const float2 uh = *reinterpret_cast<const float2*>(xh + W + 2 * lane);
        const float2 ulp = *reinterpret_cast<const float2*>(xl + W + 2 * lane);
        float gh[2], gl[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          DF au{0.f, 0.f};
          df_fma(au, op.ah, op.al, c ? uh.y : uh.x, c ? ulp.y : ulp.x);
          au = df_norm(au);
          float s2, e;
          two_sum(c ? fv.y : fv.x, -au.h, s2, e);
          const DF g = df_norm(DF{s2, e - au.l});
          gh[c] = g.h;
          gl[c] = g.l;
        }
        gring[((a - i0) % Q) * 32 + lane] = make_float4(gh[0], gh[1], gl[0], gl[1]);
      }
      if (a >= i0 + W) {
        // column pass for output row i = a - W over the rows a - 2W .. a
        const int i = a - W;
        int s0 = sa - 2 * W;
        if (s0 < 0) s0 += P;
        float2 zh2 = make_float2(0.f, 0.f), zl2 = make_float2(0.f, 0.f);
#pragma unroll(W > 16 ? 5 : P)
        for (int d = 0; d < P; ++d) {
          int sl = s0 + d;
          sl = sl >= P ? sl - P : sl;
          const float4 t = tring[sl * 32 + lane];
          df_fma2(zh2, zl2, op.kh2[d], op.nkh2[d], op.kl2[d], make_float2(t.x, t.y),
                  make_float2(t.z, t.w));
        }
        df_norm2(zh2, zl2);
        // r = g - z (double-float, rounded once)
        const float4 g4 = gring[((i - i0) % Q) * 32 + lane];
        const size_t g = (size_t)i * n + c0 + 2 * lane;
        float rv[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          float s2, e;
          two_sum(c ? g4.y : g4.x, -(c ? zh2.y : zh2.x), s2, e);
          rv[c] = s2 + (e + ((c ? g4.w : g4.z) - (c ? zl2.y : zl2.x)));
          ss = fmaf(rv[c], rv[c], ss);
        }
        *reinterpret_cast<float2*>(r + (size_t)b * plane + g) = make_float2(rv[0], rv[1]);
      }
    }
    __syncwarp();  // every lane is done with the rings before the next unit restages them
    if (partials) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      if (lane == 0) partials[(size_t)b * upi + rem] = (double)ss;
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

template <int W>
int launch_refine_wide(const StencilHost<double>& sd, double alpha, int n, int B, const double* u,
                       const float* f, float* r, double* partials, const int* active, int kch,
                       cudaStream_t st) {
  constexpr int NW = RwWarps<W>::value;
  const size_t sm = (size_t)NW * RwGeom<W>::words * 4;
  auto kern = k_refine_wide<W>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (kch > wide_chunks_max(n)) kch = wide_chunks_max(n);
  if (kch <= 0) kch = wide_chunks(n, W, (long long)B * (n / kRsSW), num_sms_refine(), NW);
  const long long units = (long long)B * (n / kRsSW) * kch;
  long long grid = units;  // one block per SM while there are units for every SM
  const long long cap = (long long)num_sms_refine();
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  kern<<<(int)grid, 32 * NW, sm, st>>>(refine_args<W>(sd, alpha, n), B, u, f, r, partials, active,
                                       kch);
  return (n / kRsSW) * kch;
}

template <int WK>
void launch_refine_strip(const StencilHost<double>& sd, double alpha, int n, int B,
                         const double* u, const float* f, float* r, double* partials,
                         const int* active, cudaStream_t st) {
  const size_t sm = (size_t)kRsWarps * kRsWords * 4;
  auto kern = k_refine_strip<WK>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kRsWarps, sm);
  if (per_sm < 1) per_sm = 1;
  const long long units = (long long)B * (n / kRsSW) * (n / kRsH);
  long long grid = (units + kRsWarps - 1) / kRsWarps;
  const long long cap = (long long)num_sms_refine() * per_sm;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  kern<<<(int)grid, 32 * kRsWarps, sm, st>>>(refine_args<WK>(sd, alpha, n), B, u, f, r, partials,
                                             active);
}

template <int WK>
bool launch_refine_pipe(const StencilHost<double>& sd, double alpha, int n, int B, const double* u,
                        const float* f, float* r, double* partials, const int* active, int tile,
                        int tx, cudaStream_t st) {
  const RefineGeom g(tile, WK, RSeg<WK>::value);
  const size_t sm = (size_t)g.words * 4;
  if (sm > 200 * 1024) return false;
  const RefineArgs<WK> a = refine_args<WK>(sd, alpha, n);
  auto kern = k_refine_pipe<WK>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, sm);
  long long grid = (long long)num_sms_refine() * (per_sm > 0 ? per_sm : 1);
  const long long total = (long long)B * tx * tx;
  if (grid > total) grid = total;
  if (grid < 1) grid = 1;
  kern<<<(int)grid, 256, sm, st>>>(a, B, u, f, r, partials, active, tile, tx);
  return true;
}

// the stencil kernels when the level qualifies (Toeplitz K, M = I, aligned
// buffers, n a multiple of 4): the strip form for half-widths <= 8 and n a
// multiple of 64, the wide strip form for half-widths <= 32 and n a
// multiple of 64 (if wide_req <= 0: -wide_req chunks per strip, 0 its own
// choice), else the tiled pipeline; false otherwise.  *nparts:
// partial sums written per right-hand side.
bool try_refine_pipe(const StencilHost<double>* sd, double alpha, int n, int B, const double* u,
                     const float* f, float* r, double* partials, const int* active, int tile,
                     int tx, int wide_req, cudaStream_t st, int* nparts) {
  if (!sd || !sd->valid || sd->nbK != 0 || sd->wM != 0 || sd->sM[0] != 1.0 || n % 4 != 0 ||
      (reinterpret_cast<uintptr_t>(u) & 15) || (reinterpret_cast<uintptr_t>(f) & 15))
    return false;
  const int w = sd->wK;
  if (w <= kRsHalo && n % kRsSW == 0) {
    if (w <= 2) launch_refine_strip<2>(*sd, alpha, n, B, u, f, r, partials, active, st);
    else if (w <= 4) launch_refine_strip<4>(*sd, alpha, n, B, u, f, r, partials, active, st);
    else launch_refine_strip<8>(*sd, alpha, n, B, u, f, r, partials, active, st);
    *nparts = (n / kRsSW) * (n / kRsH);
    return true;
  }
  if (wide_req <= 0 && w <= 32 && n % kRsSW == 0 && n >= 2 * kRsSW) {
    *nparts = w <= 16 ? launch_refine_wide<16>(*sd, alpha, n, B, u, f, r, partials, active,
                                               -wide_req, st)
                      : launch_refine_wide<32>(*sd, alpha, n, B, u, f, r, partials, active,
                                               -wide_req, st);
    return true;
  }
  *nparts = tx * tx;
  if (w <= 2) return launch_refine_pipe<2>(*sd, alpha, n, B, u, f, r, partials, active, tile, tx, st);
  if (w <= 4) return launch_refine_pipe<4>(*sd, alpha, n, B, u, f, r, partials, active, tile, tx, st);
  if (w <= 8) return launch_refine_pipe<8>(*sd, alpha, n, B, u, f, r, partials, active, tile, tx, st);
  if (w <= 16) return launch_refine_pipe<16>(*sd, alpha, n, B, u, f, r, partials, active, tile, tx, st);
  if (w <= 32) return launch_refine_pipe<32>(*sd, alpha, n, B, u, f, r, partials, active, tile, tx, st);
  return false;
}

}  // namespace

void refine_residual2d(const Band2D<float>& hi, const float* Kd_lo, const float* Md_lo,
                       const StencilHost<double>* stencil, double alpha, int B, const double* u,
                       const float* f, float* r, double* partials, int* ntiles,
                       const int* active, cudaStream_t st, LaunchLog& log, int tile_req) {
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
  int pi_ = log.begin(K_REFINE_RESIDUAL, st);
  int nparts = tx * tx;
  // tile_req <= 0 (the default): the wide strip kernel where it applies,
  // with -tile_req chunks per strip (0: its own choice)
  if (!try_refine_pipe(stencil, alpha, hi.n, B, u, f, r, partials, active, tile, tx, tile_req,
                       st, &nparts)) {
    nparts = tx * tx;
    size_t sm = smem(tile);
    cudaFuncSetAttribute(k_refine_residual2d<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_refine_residual2d<0><<<dim3(tx * tx, B), 256, sm, st>>>(hi, Kd_lo, Md_lo, alpha, u, f, r,
                                                              partials, active, tile, tx);
  }
  if (ntiles) *ntiles = nparts;
  log.end(pi_, st, (double)hi.n * hi.n * log.active_hint);
}

}  // namespace nmg
