// Stencil form of the level residual r = y - A_l x (and of the residual
// followed by full-weighting restriction, Algorithm 4: B_l = Y_l -
// Mat(A Vec(X*)) and R = (P(x)P)^T / 4) for levels whose banded factors are
// one stencil except for a few leading correction rows (see StencilHost).
// Included by one translation unit per element type.
//
// Persistent blocks walk the tiles of all right-hand sides; the x tile (with
// its halo) and the y tile of the next tile are copied into the other half of
// a double buffer with cp.async while the current one is computed, so global
// latency is hidden.  The stencil lives in kernel parameters (constant bank):
// each FMA reads one staged operand, and every pass keeps a window of
// S + 2 WK staged values in registers for S consecutive outputs:
//   row pass    t_K[a][j] = sum_d sK[d] x[a][j + d - WK],  t_M likewise
//               (thread: one staged row a, S consecutive columns, 16-byte
//               shared loads)
//   column pass z[i][j] = sum_d sK[d] t_K[i + d - WK][j] + alpha (M pass)
//               (thread: one column j, S consecutive rows)
// Rows/columns g < nb add their correction rows (read from shared memory:
// the register windows are only indexed at compile-time offsets).  WK >= wK
// is the padded half-width (compile time: 2, 4, 6, 8, 16, or the maximum;
// even, so that the S + 2 WK window is whole 16-byte chunks of fp32 and
// fp64); the M factor is padded to
// half-width 1.  Staged tiles start on 16-byte-aligned global columns
// (n % (16 / sizeof(T)) == 0): a 16-byte chunk is either inside the image or
// outside it and then zero-filled.
//
// fp32: the K taps run as packed two-lane FMAs (fma.rn.f32x2) on register
// pairs (w[2k], w[2k+1]) of the window: even taps d accumulate the output
// pairs (2p, 2p+1), odd taps the pairs (2p-1, 2p), so both read natural
// pairs; the two partial sums of each output are added at the end.
// MID: the level's M factor is the identity (the fine level, M_1 = I): the
// M passes reduce to alpha x at the centre and are skipped.
#pragma once

#include <type_traits>

#include "nmg_internal.h"

namespace nmg {
namespace stencil {

constexpr int kThreads = 256;

// fused multiply-add in the argument type (fp32 stays fp32)
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(*reinterpret_cast<unsigned long long*>(&d))
      : "l"(*reinterpret_cast<unsigned long long*>(&a)),
        "l"(*reinterpret_cast<unsigned long long*>(&b)),
        "l"(*reinterpret_cast<unsigned long long*>(&c)));
  return d;
}

// block-wide sum in the level type T (warp shuffles, then one value per
// warp in shared memory, added in a fixed order: deterministic); the result
// is valid in thread 0.  fp32 levels stay in fp32: fp64 adds run at 1/64 of
// the fp32 rate, and a tree of them held every warp of the block at the next
// barrier.
template <typename T>
__device__ __forceinline__ double block_sum(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T s = T(0);
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) s += red[i];
  }
  return (double)s;
}

template <typename T, int WK>
struct StencilArgs {
  int n, wK, wM, nbK, nbM;
  T alpha;
  T sK[2 * WK + 1];  // stencil padded to WK: entry WK + o is offset o
  T sM[3];
  const T* cK;  // nbK x (2 wK + 1)
  const T* cM;  // nbM x (2 wM + 1)
};

template <int WK> struct SegLen { static constexpr int value = WK <= 8 ? 8 : 4; };

// staged geometry of one tile shape (host and device)
template <typename T, bool RESTRICT, int WK, bool MID>
struct PipeGeom {
  static constexpr int E = 16 / (int)sizeof(T);  // elements per 16-byte chunk
  static constexpr int S = SegLen<WK>::value;
  // t_K / t_M columns start TOFF words in, so that every output of a
  // row-pass segment (logical columns -E+1 .. RW+S-1) has a slot and the
  // stores need no bounds test; the rows run to whole column-pass segments
  // (rows past the tile only feed discarded outputs)
  static constexpr int TOFF = E;
  int RH, RW, XH, XP, YP, TP, TKH, TMH, words;
  __host__ __device__ PipeGeom(int tile) {
    RH = RESTRICT ? 2 * tile + 1 : tile;
    RW = RH;
    XH = RH + 2 * WK;
    // columns staged: offset (< E) + the segments' reach + the halo
    const int reach = ((E - 1 + RW + S - 1) / S) * S + 2 * WK;
    XP = (reach + E - 1) / E * E;
    if (((XP / E) & 1) == 0) XP += E;  // odd number of chunks: conflict-free 16-byte lanes
    YP = (E - 1 + RW + E - 1) / E * E;
    TP = (TOFF + RW + 2 * S) | 1;
    const int rh_seg = (RH + S - 1) / S * S;
    TKH = rh_seg + 2 * WK;
    TMH = MID ? 0 : rh_seg + 2;
    words = 2 * XH * XP + 2 * RH * YP + TKH * TP + TMH * TP + (RESTRICT ? RH * TP : 0);
  }
};

__device__ __forceinline__ void cp_async_16(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src),
               "r"(valid ? 16u : 0u)
               : "memory");
}

// z[o] = sum_{d=0}^{2WK} c[d] w[o + d], o = 0 .. S-1, from the window held as
// register pairs W2[k] = (w[2k], w[2k+1]), k < S/2 + WK (packed fp32 FMAs)
template <int WK, int S>
__device__ __forceinline__ void taps_packed(const float2 (&W2)[S / 2 + WK], const float (&c)[2 * WK + 1],
                                            float (&z)[S]) {
  float2 ev[S / 2], od[S / 2 + 1];  // od[q] holds outputs (2q - 1, 2q)
#pragma unroll
  for (int p = 0; p < S / 2; ++p) ev[p] = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q <= S / 2; ++q) od[q] = make_float2(0.f, 0.f);
#pragma unroll
  for (int e = 0; e <= WK; ++e) {
    const float2 c2 = make_float2(c[2 * e], c[2 * e]);
#pragma unroll
    for (int p = 0; p < S / 2; ++p) ev[p] = ffma2(c2, W2[p + e], ev[p]);
  }
#pragma unroll
  for (int e = 0; e < WK; ++e) {
    const float2 c2 = make_float2(c[2 * e + 1], c[2 * e + 1]);
#pragma unroll
    for (int q = 0; q <= S / 2; ++q) od[q] = ffma2(c2, W2[q + e], od[q]);
  }
#pragma unroll
  for (int p = 0; p < S / 2; ++p) {
    z[2 * p] = ev[p].x + od[p].y;
    z[2 * p + 1] = ev[p].y + od[p + 1].x;
  }
}

template <typename T, bool RESTRICT, int WK, bool MID>
__global__ void __launch_bounds__(kThreads)
k_res2d_pipe(StencilArgs<T, WK> op, int B, const T* __restrict__ x, const T* __restrict__ y,
             T* __restrict__ out, double* __restrict__ partials, const int* __restrict__ active,
             int tile, int tiles_x) {
  using G = PipeGeom<T, RESTRICT, WK, MID>;
  constexpr int E = G::E, S = G::S, NW = S + 2 * WK;
  static_assert(NW % E == 0, "the row pass loads its window as whole 16-byte chunks");
  constexpr bool PACK = std::is_same<T, float>::value;
  const G g(tile);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T red[32];
  T* xbuf = reinterpret_cast<T*>(smem_raw);  // [2][XH][XP]
  T* ybuf = xbuf + 2 * g.XH * g.XP;          // [2][RH][YP]
  T* tk = ybuf + 2 * g.RH * g.YP + G::TOFF;  // [TKH][TP], column j at j + TOFF
  T* tm = tk + g.TKH * g.TP;                 // [TMH][TP]
  T* rs = tm + g.TMH * g.TP;                 // [RH][TP]
  const int n = op.n, nc = n / 2;
  const int per_img = tiles_x * tiles_x;
  const int total = B * per_img;  // B <= 65535, per_img <= 4096
  const size_t plane = (size_t)n * n;
  // the K stencil as a register array (compile-time indexed)
  float cf[2 * WK + 1];
  if (PACK) {
#pragma unroll
    for (int d = 0; d <= 2 * WK; ++d) cf[d] = (float)op.sK[d];
  }

  auto next_valid = [&](int t) {
    while (t < total && !active[t / per_img]) t += gridDim.x;
    return t;
  };
  // tile origin: fine rows/cols of the tile's region and its extent
  auto origin = [&](int t, int& b, int& ty, int& tx, int& r0, int& c0, int& RH, int& RW) {
    b = t / per_img;
    const int tt = t - b * per_img;
    ty = tt / tiles_x;
    tx = tt % tiles_x;
    if (RESTRICT) {
      const int CH = min(tile, nc - ty * tile), CW = min(tile, nc - tx * tile);
      r0 = 2 * ty * tile - 1;
      c0 = 2 * tx * tile - 1;
      RH = 2 * CH + 1;
      RW = 2 * CW + 1;
    } else {
      r0 = ty * tile;
      c0 = tx * tile;
      RH = min(tile, n - r0);
      RW = min(tile, n - c0);
    }
  };
  auto prefetch = [&](int t, int buf) {
    if (t < total) {
      int b, ty, tx, r0, c0, RH, RW;
      origin(t, b, ty, tx, r0, c0, RH, RW);
      const T* xb = x + (size_t)b * plane;
      const int cs = (c0 - WK) & ~(E - 1);  // floor to a chunk boundary
      const int xch = g.XP / E;
      T* xd = xbuf + buf * g.XH * g.XP;
      for (int i = threadIdx.x; i < g.XH * xch; i += blockDim.x) {
        const int a = i / xch, ch = i % xch;
        const int gr = r0 - WK + a, gc = cs + ch * E;
        const bool in = gr >= 0 && gr < n && gc >= 0 && gc < n;
        cp_async_16(xd + a * g.XP + ch * E, in ? xb + (size_t)gr * n + gc : xb, in);
      }
      if (y) {
        const T* yb = y + (size_t)b * plane;
        const int cy = c0 & ~(E - 1);
        const int ych = g.YP / E;
        T* yd = ybuf + buf * g.RH * g.YP;
        for (int i = threadIdx.x; i < RH * ych; i += blockDim.x) {
          const int a = i / ych, ch = i % ych;
          const int gr = r0 + a, gc = cy + ch * E;
          const bool in = gr >= 0 && gr < n && gc >= 0 && gc < n;
          cp_async_16(yd + a * g.YP + ch * E, in ? yb + (size_t)gr * n + gc : yb, in);
        }
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
    const int XH = RH + 2 * WK;
    const int ofs = (c0 - WK) - ((c0 - WK) & ~(E - 1));
    const int oy = c0 - (c0 & ~(E - 1));
    const T* xs = xbuf + buf * g.XH * g.XP;
    const T* ys = ybuf + buf * g.RH * g.YP;
    // row pass: item -> (staged row a, segment of S physical columns)
    const int nseg_r = (ofs + RW + S - 1) / S;
    const int offK = WK - op.wK, offM = 1 - op.wM;
    for (int item = threadIdx.x; item < XH * nseg_r; item += blockDim.x) {
      const int a = item % XH, P = (item / XH) * S;
      const T* xr = xs + a * g.XP + P;
      T w[NW];
#pragma unroll
      for (int k4 = 0; k4 < NW / E; ++k4) {
        const uint4 v = *reinterpret_cast<const uint4*>(xr + k4 * E);
        const T* vv = reinterpret_cast<const T*>(&v);
#pragma unroll
        for (int e = 0; e < E; ++e) w[k4 * E + e] = vv[e];
      }
      // d outer, outputs inner: S independent accumulation chains
      T acc[S], am[S];
      if constexpr (PACK) {
        float2 W2[NW / 2];
#pragma unroll
        for (int k2 = 0; k2 < NW / 2; ++k2) W2[k2] = make_float2(w[2 * k2], w[2 * k2 + 1]);
        taps_packed<WK, S>(W2, cf, acc);
      } else {
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) acc[s2] = T(0);
#pragma unroll
        for (int d = 0; d < 2 * WK + 1; ++d)
#pragma unroll
          for (int s2 = 0; s2 < S; ++s2) acc[s2] = fma_t(op.sK[d], w[s2 + d], acc[s2]);
      }
      if (!MID) {
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) am[s2] = T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int s2 = 0; s2 < S; ++s2) am[s2] = fma_t(op.sM[d], w[s2 + WK - 1 + d], am[s2]);
      }
      const int jb = P - ofs;  // logical column of output s2 = 0
      if (c0 + jb < op.nbK || (!MID && c0 + jb < op.nbM)) {  // leading columns: correction rows
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) {
          const int gcol = c0 + jb + s2;
          if (gcol < 0) continue;
          if (gcol < op.nbK) {
            const T* cr = op.cK + (size_t)gcol * (2 * op.wK + 1);
            for (int d = 0; d <= 2 * op.wK; ++d) acc[s2] = fma_t(cr[d], xr[s2 + offK + d], acc[s2]);
          }
          if (!MID && gcol < op.nbM) {
            const T* cr = op.cM + (size_t)gcol * (2 * op.wM + 1);
            for (int d = 0; d <= 2 * op.wM; ++d)
              am[s2] = fma_t(cr[d], xr[s2 + WK - 1 + offM + d], am[s2]);
          }
        }
      }
      T* tkr = tk + a * g.TP + jb;
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) tkr[s2] = acc[s2];
      if (!MID && a >= WK - 1 && a <= WK + RH) {  // t_M rows r0-1 .. r0+RH
        T* tmr = tm + (a - (WK - 1)) * g.TP + jb;
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) tmr[s2] = am[s2];
      }
    }
    __syncthreads();
    // column pass and residual: item -> (column j, segment of S rows)
    const int nseg_c = (RH + S - 1) / S;
    T ss = T(0);  // this thread's sum of squares (T: no fp64 arithmetic per point in fp32)
    for (int item = threadIdx.x; item < RW * nseg_c; item += blockDim.x) {
      const int j = item % RW, i0 = (item / RW) * S;
      T wk[NW];
      const T* tkc = tk + i0 * g.TP + j;
#pragma unroll
      for (int q = 0; q < NW; ++q) wk[q] = tkc[q * g.TP];
      T zk[S], zm[S];
      if constexpr (PACK) {
        float2 W2[NW / 2];
#pragma unroll
        for (int k2 = 0; k2 < NW / 2; ++k2) W2[k2] = make_float2(wk[2 * k2], wk[2 * k2 + 1]);
        taps_packed<WK, S>(W2, cf, zk);
      } else {
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) zk[s2] = T(0);
#pragma unroll
        for (int d = 0; d < 2 * WK + 1; ++d)
#pragma unroll
          for (int s2 = 0; s2 < S; ++s2) zk[s2] = fma_t(op.sK[d], wk[s2 + d], zk[s2]);
      }
      const T* tmc = tm + i0 * g.TP + j;
      if (!MID) {
        T wm[S + 2];
#pragma unroll
        for (int q = 0; q < S + 2; ++q) wm[q] = tmc[q * g.TP];
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) zm[s2] = T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int s2 = 0; s2 < S; ++s2) zm[s2] = fma_t(op.sM[d], wm[s2 + d], zm[s2]);
      }
      if (r0 + i0 < op.nbK || (!MID && r0 + i0 < op.nbM)) {  // leading rows: correction rows
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) {
          const int gi = r0 + i0 + s2;
          if (gi < 0) continue;
          if (gi < op.nbK) {
            const T* cr = op.cK + (size_t)gi * (2 * op.wK + 1);
            for (int d = 0; d <= 2 * op.wK; ++d)
              zk[s2] = fma_t(cr[d], tkc[(s2 + offK + d) * g.TP], zk[s2]);
          }
          if (!MID && gi < op.nbM) {
            const T* cr = op.cM + (size_t)gi * (2 * op.wM + 1);
            for (int d = 0; d <= 2 * op.wM; ++d)
              zm[s2] = fma_t(cr[d], tmc[(s2 + offM + d) * g.TP], zm[s2]);
          }
        }
      }
      const int gj = c0 + j;
      const bool colin = gj >= 0 && gj < n;
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) {
        const int i = i0 + s2, gi = r0 + i;
        if (i >= RH) break;
        T r = T(0);
        if (colin && gi >= 0 && gi < n) {
          const T yv = y ? ys[i * g.YP + j + oy] : T(0);
          // M = I: the M (x) M term is x itself (staged row i + WK, physical
          // column j + ofs + WK)
          const T mv = MID ? xs[(i + WK) * g.XP + j + ofs + WK] : zm[s2];
          r = yv - (op.alpha * mv + zk[s2]);
          if (!RESTRICT) {
            out[(size_t)b * plane + (size_t)gi * n + gj] = r;
            ss = fma_t(r, r, ss);
          }
        }
        if (RESTRICT) rs[i * g.TP + j] = r;
      }
    }
    if (RESTRICT) {
      __syncthreads();
      const size_t cplane = (size_t)nc * nc;
      const int CH = (RH - 1) / 2, CW = (RW - 1) / 2, I0 = ty * tile, J0 = tx * tile;
      for (int idx = threadIdx.x; idx < CH * CW; idx += blockDim.x) {
        const int ci = idx / CW, cj = idx % CW;
        const T* c = rs + (2 * ci + 1) * g.TP + (2 * cj + 1);  // local fine center
        const T v = T(0.25) * (T(0.25) * c[-g.TP - 1] + T(0.5) * c[-g.TP] + T(0.25) * c[-g.TP + 1]) +
                    T(0.5) * (T(0.25) * c[-1] + T(0.5) * c[0] + T(0.25) * c[1]) +
                    T(0.25) * (T(0.25) * c[g.TP - 1] + T(0.5) * c[g.TP] + T(0.25) * c[g.TP + 1]);
        out[(size_t)b * cplane + (size_t)(I0 + ci) * nc + (J0 + cj)] = v;
        ss = fma_t(v, v, ss);
      }
    }
    if (partials) {
      const double s = block_sum<T>(ss, red);
      if (threadIdx.x == 0) partials[(size_t)b * per_img + (ty * tiles_x + tx)] = s;
    }
    __syncthreads();  // everyone is done with this buffer and with red[]
    const int after = nxt < total ? next_valid(nxt + gridDim.x) : total;
    prefetch(after, buf);
    cur = nxt;
    nxt = after;
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

inline int num_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms;
}

template <typename T, int WK>
StencilArgs<T, WK> stencil_args(const Band2D<T>& op) {
  const StencilHost<T>& h = *op.st;
  StencilArgs<T, WK> a{};
  a.n = op.n;
  a.wK = h.wK;
  a.wM = h.wM;
  a.nbK = h.nbK;
  a.nbM = h.nbM;
  a.alpha = op.alpha;
  for (int d = 0; d <= 2 * h.wK; ++d) a.sK[WK - h.wK + d] = h.sK[d];
  for (int d = 0; d <= 2 * h.wM; ++d) a.sM[1 - h.wM + d] = h.sM[d];
  a.cK = h.cK;
  a.cM = h.cM;
  return a;
}

template <typename T, bool RESTRICT, int WK, bool MID>
bool launch_st(const Band2D<T>& op, int B, const T* x, const T* y, T* out, double* partials,
               const int* active, int tile, int ntx, cudaStream_t st) {
  const PipeGeom<T, RESTRICT, WK, MID> g(tile);
  const size_t sm = (size_t)g.words * sizeof(T);
  if (sm > 200 * 1024) return false;  // this tile side is the generic kernel's
  auto kern = k_res2d_pipe<T, RESTRICT, WK, MID>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, sm);
  if (per_sm < 1) per_sm = 1;
  const long long total = (long long)B * ntx * ntx;
  long long grid = (long long)num_sms() * per_sm;
  if (grid > total) grid = total;
  if (grid < 1) grid = 1;
  kern<<<(int)grid, kThreads, sm, st>>>(stencil_args<T, WK>(op), B, x, y, out, partials, active,
                                        tile, ntx);
  return true;
}

template <typename T, bool RESTRICT, int WK>
bool launch_st_m(const Band2D<T>& op, int B, const T* x, const T* y, T* out, double* partials,
                 const int* active, int tile, int ntx, cudaStream_t st) {
  const StencilHost<T>& h = *op.st;
  const bool mid = h.wM == 0 && h.nbM == 0 && h.sM[0] == T(1);
  return mid ? launch_st<T, RESTRICT, WK, true>(op, B, x, y, out, partials, active, tile, ntx, st)
             : launch_st<T, RESTRICT, WK, false>(op, B, x, y, out, partials, active, tile, ntx, st);
}

// ---------------------------------------------------------------------------
// Fine-level strip form: M = I (alpha X + K X K^T), K one Toeplitz stencil
// of half-width <= 8 with no correction rows, n = 32 C with C in {2, 4}.
// One warp computes the residual (RESTRICT: and its full-weighting
// restriction) of kStripH consecutive rows of one right-hand side over the
// whole row width, lane j owning columns C j .. C j + C - 1.  Input rows
// stream through a warp-private shared-memory ring (cp.async, kStripPF rows
// ahead); the row-pass outputs t of the last 2 WK + 1 rows stay in registers
// (a ring of register rows indexed at compile time: the row loop is unrolled
// by 2 WK + 1), so the column pass reads no shared memory and no warp waits
// on another.  Column pairs of a lane form the packed fp32 FMA operands.
// ---------------------------------------------------------------------------
constexpr int kStripH = 16;     // fine output rows per warp unit
constexpr int kStripWarps = 4;  // warps per block
constexpr int kStripPF = 6;     // rows staged ahead
constexpr int kStripRing = 16;  // staged rows per warp: > kStripPF + max WK
constexpr int kStripHalo = 8;   // staged halo columns per side (>= WK)

template <int WK>
struct StripArgs {
  int n;
  float alpha;
  float sK[2 * WK + 1];  // stencil padded to WK: entry WK + o is offset o
};

template <int C>
__host__ __device__ constexpr int strip_words() {
  return kStripRing * ((32 * C + 2 * kStripHalo) + 32 * C);
}

template <bool RESTRICT, int WK, int C>
__global__ void __launch_bounds__(32 * kStripWarps, 3)
k_res_strip(StripArgs<WK> op, int B, const float* __restrict__ x, const float* __restrict__ y,
            float* __restrict__ out, double* __restrict__ partials,
            const int* __restrict__ active) {
  static_assert(C == 2 || C == 4, "two or four columns per lane");
  static_assert(WK <= kStripHalo && kStripRing > kStripPF + WK, "ring too short");
  constexpr int SW = 32 * C;               // columns per unit: the whole row
  constexpr int XW = SW + 2 * kStripHalo;  // staged x row (staged index k = column k - halo)
  constexpr int P = 2 * WK + 1;
  constexpr int CC = C / 2;                // column pairs (and coarse columns) per lane
  extern __shared__ __align__(16) float strip_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* xring = strip_smem + wib * strip_words<C>();  // [ring][XW]
  float* yring = xring + kStripRing * XW;              // [ring][SW]
  const int n = op.n;                                  // == SW
  const int upi = n / kStripH;                         // units per right-hand side
  const int total = B * upi;
  const size_t plane = (size_t)n * n;
  float cf[P];
#pragma unroll
  for (int d = 0; d < P; ++d) cf[d] = op.sK[d];
  const float alpha = op.alpha;

  for (int u = blockIdx.x * kStripWarps + wib; u < total; u += gridDim.x * kStripWarps) {
    const int b = u / upi;
    if (!active[b]) continue;  // warp-uniform
    const int i0 = (u - b * upi) * kStripH;
    const int olo = RESTRICT ? i0 - 1 : i0, ohi = i0 + kStripH;  // fine output rows
    const int alo = olo - WK, ahi = ohi + WK;                     // input rows
    const float* xb = x + (size_t)b * plane;
    const float* yb = y ? y + (size_t)b * plane : nullptr;
    // stage input row a (x with halo; y for output rows) into ring slot
    // (a - alo) mod ring; one commit group per row (empty past the end)
    auto stage = [&](int a) {
      if (a < ahi) {
        const int slot = (a - alo) % kStripRing;
        const bool rin = a >= 0 && a < n;
        float* xd = xring + slot * XW;
        for (int ch = lane; ch < XW / 4; ch += 32) {
          const int gc = ch * 4 - kStripHalo;
          const bool in = rin && gc >= 0 && gc < n;
          cp_async_16(xd + ch * 4, in ? xb + (size_t)a * n + gc : xb, in);
        }
        if (yb && a >= olo && a < ohi) {
          float* yd = yring + slot * SW;
          for (int ch = lane; ch < SW / 4; ch += 32)
            cp_async_16(yd + ch * 4, rin ? yb + (size_t)a * n + ch * 4 : yb, rin);
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
#pragma unroll
    for (int k = 0; k < kStripPF; ++k) stage(alo + k);

    float2 tw[P][CC];  // row-pass outputs of the last P input rows (column pairs)
    float hm1[CC], hm2[CC];  // horizontally restricted residual rows i-1, i-2
#pragma unroll
    for (int q = 0; q < CC; ++q) hm1[q] = hm2[q] = 0.f;
    float ss = 0.f;
    for (int a0 = alo; a0 < ahi; a0 += P) {
#pragma unroll
      for (int ph = 0; ph < P; ++ph) {
        const int a = a0 + ph;  // input row; its t goes to register row ph
        if (a < ahi) {
          asm volatile("cp.async.wait_group %0;" ::"n"(kStripPF - 1) : "memory");
          __syncwarp();
          stage(a + kStripPF);
          // row pass: t[c] = sum_d sK[d] x[a][C lane + c + d - WK]
          const float* xs = xring + ((a - alo) % kStripRing) * XW + C * lane;
          float w[C + 2 * kStripHalo];
          if (C == 4) {
#pragma unroll
            for (int k4 = 0; k4 < (C + 2 * kStripHalo) / 4; ++k4) {
              const float4 v = *reinterpret_cast<const float4*>(xs + 4 * k4);
              w[4 * k4] = v.x; w[4 * k4 + 1] = v.y; w[4 * k4 + 2] = v.z; w[4 * k4 + 3] = v.w;
            }
          } else {
#pragma unroll
            for (int k2 = 0; k2 < (C + 2 * kStripHalo) / 2; ++k2) {
              const float2 v = *reinterpret_cast<const float2*>(xs + 2 * k2);
              w[2 * k2] = v.x; w[2 * k2 + 1] = v.y;
            }
          }
          float t[C];
#pragma unroll
          for (int c = 0; c < C; ++c) t[c] = 0.f;
#pragma unroll
          for (int d = 0; d < P; ++d)
#pragma unroll
            for (int c = 0; c < C; ++c) t[c] = fmaf(cf[d], w[c + kStripHalo - WK + d], t[c]);
#pragma unroll
          for (int q = 0; q < CC; ++q) tw[ph][q] = make_float2(t[2 * q], t[2 * q + 1]);
          if (a >= olo + WK) {
            // column pass for output row i = a - WK: rows i - WK + d sit in
            // register rows (ph + 1 + d) mod P
            const int i = a - WK;
            float2 z[CC];
#pragma unroll
            for (int q = 0; q < CC; ++q) z[q] = make_float2(0.f, 0.f);
#pragma unroll
            for (int d = 0; d < P; ++d) {
              const float2 c2 = make_float2(cf[d], cf[d]);
#pragma unroll
              for (int q = 0; q < CC; ++q) z[q] = ffma2(c2, tw[(ph + 1 + d) % P][q], z[q]);
            }
            const int slot = (i - alo) % kStripRing;
            const float* xc = xring + slot * XW + kStripHalo + C * lane;
            const float* yc = yring + slot * SW + C * lane;
            const bool rin = i >= 0 && i < n;
            float r[C];
#pragma unroll
            for (int q = 0; q < CC; ++q) {
              const float2 xv = *reinterpret_cast<const float2*>(xc + 2 * q);
              const float2 yv = yb ? *reinterpret_cast<const float2*>(yc + 2 * q) : make_float2(0.f, 0.f);
              r[2 * q] = rin ? yv.x - fmaf(alpha, xv.x, z[q].x) : 0.f;
              r[2 * q + 1] = rin ? yv.y - fmaf(alpha, xv.y, z[q].y) : 0.f;
            }
            if (!RESTRICT) {
              if (rin) {
                float* o = out + (size_t)b * plane + (size_t)i * n + C * lane;
                if (C == 4)
                  *reinterpret_cast<float4*>(o) = make_float4(r[0], r[1], r[2], r[3]);
                else
                  *reinterpret_cast<float2*>(o) = make_float2(r[0], r[1]);
#pragma unroll
                for (int c = 0; c < C; ++c) ss = fmaf(r[c], r[c], ss);
              }
            } else {
              // [1 2 1] / 4 along the row: coarse column CC lane + q is
              // centred on fine column C lane + 2q; fine column C lane - 1
              // comes from the left lane (zero left of the grid)
              float left = __shfl_up_sync(0xffffffffu, r[C - 1], 1);
              if (lane == 0) left = 0.f;
              float h[CC];
#pragma unroll
              for (int q = 0; q < CC; ++q)
                h[q] = 0.25f * (q == 0 ? left : r[2 * q - 1]) + 0.5f * r[2 * q] + 0.25f * r[2 * q + 1];
              // [1 2 1] / 4 down the column: coarse row I = (i - 1) / 2 once
              // its bottom fine row i = 2I + 1 is done
              if ((i & 1) && i >= olo + 2) {
                const int I = (i - 1) >> 1;
                float v[CC];
#pragma unroll
                for (int q = 0; q < CC; ++q) {
                  v[q] = 0.25f * hm2[q] + 0.5f * hm1[q] + 0.25f * h[q];
                  ss = fmaf(v[q], v[q], ss);
                }
                float* o = out + (size_t)b * (plane / 4) + (size_t)I * (n / 2) + CC * lane;
                if (CC == 2)
                  *reinterpret_cast<float2*>(o) = make_float2(v[0], v[CC - 1]);
                else
                  o[0] = v[0];
              }
#pragma unroll
              for (int q = 0; q < CC; ++q) {
                hm2[q] = hm1[q];
                hm1[q] = h[q];
              }
            }
          }
        }
      }
    }
    __syncwarp();  // every lane is done with the ring before the next unit restages it
    if (partials) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      if (lane == 0) partials[(size_t)b * upi + (u - b * upi)] = (double)ss;
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// the strip form applies: fp32 fine level (M = I, Toeplitz K, WK <= 8),
// n = 64 or 128, 16-byte aligned vectors
template <typename T>
bool strip_applies(const Band2D<T>& op, const T* x, const T* y) {
  if (!std::is_same<T, float>::value || !op.st || !op.st->valid) return false;
  const StencilHost<T>& h = *op.st;
  if (h.wM != 0 || h.nbM != 0 || h.nbK != 0 || h.sM[0] != T(1) || h.wK > kStripHalo) return false;
  if (op.n != 64 && op.n != 128) return false;
  return !((reinterpret_cast<uintptr_t>(x) & 15) || (y && (reinterpret_cast<uintptr_t>(y) & 15)));
}

template <bool RESTRICT, int WK, int C>
void launch_strip(const Band2D<float>& op, int B, const float* x, const float* y, float* out,
                  double* partials, const int* active, cudaStream_t st) {
  StripArgs<WK> a{};
  a.n = op.n;
  a.alpha = op.alpha;
  const StencilHost<float>& h = *op.st;
  for (int d = 0; d <= 2 * h.wK; ++d) a.sK[WK - h.wK + d] = h.sK[d];
  const size_t sm = (size_t)kStripWarps * strip_words<C>() * sizeof(float);
  auto kern = k_res_strip<RESTRICT, WK, C>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kStripWarps, sm);
  if (per_sm < 1) per_sm = 1;
  const long long units = (long long)B * (op.n / kStripH);
  long long grid = (units + kStripWarps - 1) / kStripWarps;
  const long long cap = (long long)num_sms() * per_sm;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  kern<<<(int)grid, 32 * kStripWarps, sm, st>>>(a, B, x, y, out, partials, active);
}

template <typename T, bool RESTRICT>
bool launch_strip_any(const Band2D<T>& op, int B, const T* x, const T* y, T* out,
                      double* partials, const int* active, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    const int w = op.st->wK;
    if (op.n == 128) {
      if (w <= 2) launch_strip<RESTRICT, 2, 4>(op, B, x, y, out, partials, active, st);
      else if (w <= 4) launch_strip<RESTRICT, 4, 4>(op, B, x, y, out, partials, active, st);
      else launch_strip<RESTRICT, 8, 4>(op, B, x, y, out, partials, active, st);
    } else {
      if (w <= 2) launch_strip<RESTRICT, 2, 2>(op, B, x, y, out, partials, active, st);
      else if (w <= 4) launch_strip<RESTRICT, 4, 2>(op, B, x, y, out, partials, active, st);
      else launch_strip<RESTRICT, 8, 2>(op, B, x, y, out, partials, active, st);
    }
    return true;
  }
  return false;
}

}  // namespace stencil

// partial sums per right-hand side the strip form writes (0: not used)
template <typename T>
int stencil_strip_parts(const Band2D<T>& op) {
  if (!std::is_same<T, float>::value || !op.st || !op.st->valid) return 0;
  const StencilHost<T>& h = *op.st;
  if (h.wM != 0 || h.nbM != 0 || h.nbK != 0 || h.sM[0] != T(1) || h.wK > stencil::kStripHalo)
    return 0;
  return (op.n == 64 || op.n == 128) ? op.n / stencil::kStripH : 0;
}

// the stencil kernel for this level (the strip form on an fp32 fine level,
// else the tiled pipeline), or false (generic kernel) if the level has no
// stencil form or a half-width above kStencilMaxW; *nparts: partial sums
// written per right-hand side
template <typename T, bool RESTRICT>
bool launch_stencil_residual(const Band2D<T>& op, int B, const T* x, const T* y, T* out,
                             double* partials, const int* active, int tile, int ntx,
                             cudaStream_t st, int* nparts) {
  using namespace stencil;
  if (!op.st || !op.st->valid || op.st->wM > 1) return false;
  if (strip_applies<T>(op, x, y) && launch_strip_any<T, RESTRICT>(op, B, x, y, out, partials, active, st)) {
    *nparts = op.n / kStripH;
    return true;
  }
  *nparts = ntx * ntx;
  // 16-byte chunks of x and y must not straddle the image edge
  constexpr int E = 16 / (int)sizeof(T);
  if (op.n % E != 0 || (reinterpret_cast<uintptr_t>(x) & 15) ||
      (y && (reinterpret_cast<uintptr_t>(y) & 15)))
    return false;
  const int w = op.st->wK;
  if (w <= 2) return launch_st_m<T, RESTRICT, 2>(op, B, x, y, out, partials, active, tile, ntx, st);
  if (w <= 4) return launch_st_m<T, RESTRICT, 4>(op, B, x, y, out, partials, active, tile, ntx, st);
  if (w <= 6) return launch_st_m<T, RESTRICT, 6>(op, B, x, y, out, partials, active, tile, ntx, st);
  if (w <= 8) return launch_st_m<T, RESTRICT, 8>(op, B, x, y, out, partials, active, tile, ntx, st);
  if (w <= 16) return launch_st_m<T, RESTRICT, 16>(op, B, x, y, out, partials, active, tile, ntx, st);
  if (w <= kStencilMaxW)
    return launch_st_m<T, RESTRICT, kStencilMaxW>(op, B, x, y, out, partials, active, tile, ntx, st);
  return false;
}

}  // namespace nmg
