// Fine-level residual r = y - A x for wide PSF stencils (Algorithm 4's
// b = Y - Mat(A Vec(X)) with A = alpha I (x) I + K (x) K, Section 4.2; K
// Toeplitz with half-width 9..32, e.g. sigma 4 px -> 16, sigma 8 px -> 32),
// and the full-weighting restriction y_{l+1} = R r (R = (P (x) P)^T / 4, the
// [1 2 1] / 4 stencil per axis) of such a residual.
//
// Strip form: one warp computes a chunk of consecutive output rows of a
// 64-column strip of one right-hand side (the launch cuts every strip into
// kch chunks, so that the units spread evenly over the SMs), lane j owning columns 2j and
// 2j + 1 (the two columns' multiply-adds are one packed fma.rn.f32x2).
// Input rows of x stream through a warp-private cp.async ring; the row pass
// of input row a reads the lane's window from the staged row; its outputs t
// (the last 2W + 1 rows) live in a warp-private shared-memory ring that each
// lane reads back only at its own columns (no barrier), and the column pass
// of output row i = a - W gathers them.  y is staged with x for the output
// rows, and g = y - alpha x of row a is kept in a second ring (W + 1 rows)
// until row a's column pass, so no global load waits inside the row loop.
// No block barriers anywhere.
//
// A fused residual + restriction would need each strip's left neighbour
// column; with wide stencils the two are separate launches instead: the
// residual writes r (12 bytes per grid point: x, y in, r out), the
// restriction reads r back (mostly from L2) and writes the quarter-size
// coarse vector with its per-unit squared norms.
#include "nmg_internal.h"

namespace nmg {

namespace {

constexpr int kWideSW = 64;   // columns per strip
constexpr int kWidePF = 4;    // rows staged ahead
constexpr int kWideRing = kWidePF + 2;

// warps per block: the per-warp rings fill most of an SM's shared memory
template <int W> struct WideWarps { static constexpr int value = W <= 16 ? 9 : 4; };

template <int W>
struct WideArgs {
  int n;
  float alpha;
  float2 k2[2 * W + 1];  // stencil taps as (c, c) pairs, padded to W
};

template <int W>
struct WideGeom {
  static constexpr int XW = kWideSW + 2 * W;  // staged x row (floats)
  static constexpr int P = 2 * W + 1;         // row-pass rows a column pass reads
  static constexpr int Q = W + 1;             // ring rows of g = y - alpha x
  // per-warp shared memory in 4-byte words: t ring written twice (slots s
  // and s + P, so a column pass reads 2W + 1 consecutive slots without
  // wrapping), g ring, x ring (XW per row), its copy shifted by one column
  // (odd taps read aligned pairs from it), y ring (64 per row)
  static constexpr int words = (2 * P + Q) * kWideSW + kWideRing * (XW + kWideSW) + XW;
};

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(d)
      : "l"(*reinterpret_cast<unsigned long long*>(&a)),
        "l"(*reinterpret_cast<unsigned long long*>(&b)),
        "l"(*reinterpret_cast<unsigned long long*>(&c)));
  return *reinterpret_cast<float2*>(&d);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src),
               "r"(valid ? 16u : 0u)
               : "memory");
}

int g_sms = 0;
int sms() {
  if (g_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 148;
  }
  return g_sms;
}

template <int W>
__global__ void __launch_bounds__(32 * WideWarps<W>::value, 1)
k_res_wide(WideArgs<W> op, int B, const float* __restrict__ x, const float* __restrict__ y,
           float* __restrict__ r, double* __restrict__ partials,
           const int* __restrict__ active, int kch) {
  using G = WideGeom<W>;
  constexpr int XW = G::XW, P = G::P, Q = G::Q;
  extern __shared__ __align__(16) float wide_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* wbase = wide_smem + (size_t)wib * G::words;
  float2* tring = reinterpret_cast<float2*>(wbase);         // [2P][32 lanes]
  float2* gring = tring + 2 * P * 32;                       // [Q][32 lanes]
  float* xring = reinterpret_cast<float*>(gring + Q * 32);  // [ring][XW]
  float* yring = xring + kWideRing * XW;                    // [ring][64]
  float* xodd = yring + kWideRing * kWideSW;                // [XW]: staged row from column + 1
  const int n = op.n;
  const int ns = n / kWideSW, upi = ns * kch, hu = (n + kch - 1) / kch;
  const int total = B * upi;
  const size_t plane = (size_t)n * n;
  const float alpha = op.alpha;
  // the taps as register pairs for the packed FMAs (loaded once: a pair
  // formed from the parameter bank at every use costs two moves); W = 32
  // reads them from the parameter bank (its loops are only partly unrolled)
  constexpr int KR = W <= 16 ? 2 * W + 1 : 1;
  float2 kr[KR];
#pragma unroll
  for (int d = 0; d < KR; ++d) kr[d] = op.k2[d];
  auto K = [&](int d) -> float2 { return W <= 16 ? kr[d < KR ? d : 0] : op.k2[d]; };

  // units dealt block-cyclically (block blockIdx.x takes units blockIdx.x,
  // + gridDim.x, ...; its warps take those in turn), so every SM gets the
  // same number of units to within one
  for (int j = wib;; j += WideWarps<W>::value) {
    const int unit = j * gridDim.x + blockIdx.x;
    if (unit >= total) break;
    const int b = unit / upi;
    if (!active[b]) continue;  // warp-uniform
    const int rem = unit - b * upi;
    const int c0 = (rem % ns) * kWideSW, i0 = (rem / ns) * hu;
    const int H = min(hu, n - i0);                  // output rows of this unit
    const int alo = i0 - W, ahi = i0 + H + W;  // input rows
    const float* xb = x + (size_t)b * plane;
    const float* yb = y ? y + (size_t)b * plane : nullptr;
    float* rb = r + (size_t)b * plane;
    // stage input row a: x with its halo, and y's 64 columns for output rows
    auto stage = [&](int a) {
      if (a < ahi) {
        const int slot = (a - alo) % kWideRing;
        float* xd = xring + slot * XW;
        const bool rin = a >= 0 && a < n;
        for (int ch = lane; ch < XW / 4; ch += 32) {
          const int gc = c0 - W + 4 * ch;
          const bool in = rin && gc >= 0 && gc < n;
          cp_async16(xd + 4 * ch, in ? xb + (size_t)a * n + gc : xb, in);
        }
        if (yb && a >= i0 && a < i0 + H && lane < kWideSW / 4)
          cp_async16(yring + slot * kWideSW + 4 * lane, yb + (size_t)a * n + c0 + 4 * lane, true);
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
#pragma unroll
    for (int k = 0; k < kWidePF; ++k) stage(alo + k);
    float ss = 0.f;
    int sa = 0;  // (a - alo) mod P
#pragma unroll 1
    for (int a = alo; a < ahi; ++a) {
      asm volatile("cp.async.wait_group %0;" ::"n"(kWidePF - 1) : "memory");
      __syncwarp();
      stage(a + kWidePF);
      const int slot = (a - alo) % kWideRing;
      const float* xs = xring + slot * XW;
      // the staged row shifted by one column, so that odd taps read aligned
      // pairs (the previous row's reads of xodd are ordered before this by
      // the barrier above)
      for (int k = lane; k < XW - 1; k += 32) xodd[k] = xs[k + 1];
      __syncwarp();
      const bool out = a >= i0 + W;  // warp-uniform
      // column pass for output row i = a - W: rows a - 2W .. a - 1 from the
      // ring (consecutive slots sa + 1 .. sa + 2W), in four chains that
      // interleave with the row pass below
      float2 z0 = make_float2(0.f, 0.f), z1 = z0, z2 = z0, z3 = z0;
      if (out) {
        const float2* tr = tring + (sa + 1) * 32 + lane;
#pragma unroll(W > 16 ? 4 : W / 2)
        for (int d = 0; d < 2 * W; d += 4) {
          z0 = fma2(K(d), tr[d * 32], z0);
          z1 = fma2(K(d + 1), tr[(d + 1) * 32], z1);
          z2 = fma2(K(d + 2), tr[(d + 2) * 32], z2);
          z3 = fma2(K(d + 3), tr[(d + 3) * 32], z3);
        }
      }
      // row pass: t[c] = sum_d K[d] x[a][c0 + 2 lane + c + d - W]; even taps
      // from the staged row, odd taps from its shifted copy, four chains
      const float2* xe = reinterpret_cast<const float2*>(xs) + lane;
      const float2* xo = reinterpret_cast<const float2*>(xodd) + lane;
      float2 t0 = make_float2(0.f, 0.f), t1 = t0, t2 = t0, t3 = t0;
#pragma unroll(W > 16 ? 4 : W / 2)
      for (int k = 0; k < W; k += 2) {
        t0 = fma2(K(2 * k), xe[k], t0);
        t1 = fma2(K(2 * k + 1), xo[k], t1);
        t2 = fma2(K(2 * k + 2), xe[k + 1], t2);
        t3 = fma2(K(2 * k + 3), xo[k + 1], t3);
      }
      t0 = fma2(K(2 * W), xe[W], t0);
      const float2 t = add2(add2(t0, t1), add2(t2, t3));
      tring[sa * 32 + lane] = t;
      tring[(sa + P) * 32 + lane] = t;
      if (a >= i0 && a < i0 + H) {
        // g = y - alpha x of this row, kept until its column pass W rows on
        const float2 xv = xe[W / 2];  // columns c0 + 2 lane, + 1 (staged index W + 2 lane)
        const float2 yv = yb ? *reinterpret_cast<const float2*>(yring + slot * kWideSW + 2 * lane)
                             : make_float2(0.f, 0.f);
        gring[((a - i0) % Q) * 32 + lane] =
            make_float2(yv.x - alpha * xv.x, yv.y - alpha * xv.y);
      }
      if (out) {
        const int i = a - W;
        const float2 z = fma2(K(2 * W), t, add2(add2(z0, z1), add2(z2, z3)));
        const float2 g = gring[((i - i0) % Q) * 32 + lane];
        const float2 rv = make_float2(g.x - z.x, g.y - z.y);
        *reinterpret_cast<float2*>(rb + (size_t)i * n + c0 + 2 * lane) = rv;
        ss = fmaf(rv.x, rv.x, ss);
        ss = fmaf(rv.y, rv.y, ss);
      }
      sa = sa + 1 == P ? 0 : sa + 1;
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

// Full weighting of a fine residual r ([B][n][n]) into yc ([B][n/2][n/2]):
// yc[I][J] = sum over (a, c) in {-1, 0, 1}^2 of w_a w_c r[2I + a][2J + c]
// with w = (1/4, 1/2, 1/4) and r = 0 outside the grid.  One warp per unit of
// 128 fine columns x kRsBand coarse rows: lane j reads four fine columns per
// row as one 16-byte load (the column left of them from the left lane, or
// from memory for lane 0), the horizontal sums of a fine row are reused by
// the two coarse rows it serves, and each fine row is read once.
constexpr int kRsBand = 8;   // coarse rows per unit (many short units: the loads of
                             // enough warps in flight to cover the memory latency)
constexpr int kRsWarps = 8;

__global__ void __launch_bounds__(32 * kRsWarps)
k_restrict_fw(int n, int B, const float* __restrict__ r, float* __restrict__ yc,
              double* __restrict__ partials, const int* __restrict__ active) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nc = n / 2;
  const int ncs = n / 128, nbands = nc / kRsBand, upi = ncs * nbands;
  const int total = B * upi;
  const size_t plane = (size_t)n * n;
  for (int unit = blockIdx.x * kRsWarps + wib; unit < total; unit += gridDim.x * kRsWarps) {
    const int b = unit / upi;
    if (!active[b]) continue;  // warp-uniform
    const int rem = unit - b * upi;
    const int c0 = (rem % ncs) * 128, I0 = (rem / ncs) * kRsBand;
    const float* rb = r + (size_t)b * plane;
    // horizontal full weighting of fine row fr at coarse columns c0/2 + 2 lane + {0, 1}
    auto hrow = [&](int fr) {
      float2 hz = make_float2(0.f, 0.f);
      if (fr < 0 || fr >= n) return hz;  // uniform across the warp
      const float* row = rb + (size_t)fr * n + c0;
      const float4 v = *reinterpret_cast<const float4*>(row + 4 * lane);
      float left = __shfl_up_sync(0xffffffffu, v.w, 1);
      if (lane == 0) left = c0 > 0 ? row[-1] : 0.f;
      hz.x = 0.25f * left + 0.5f * v.x + 0.25f * v.y;
      hz.y = 0.25f * v.y + 0.5f * v.z + 0.25f * v.w;
      return hz;
    };
    float2 hprev = hrow(2 * I0 - 1);
    float ss = 0.f;
    for (int I = I0; I < I0 + kRsBand; ++I) {
      const float2 hc = hrow(2 * I), hn = hrow(2 * I + 1);
      const float2 v = make_float2(0.25f * hprev.x + 0.5f * hc.x + 0.25f * hn.x,
                                   0.25f * hprev.y + 0.5f * hc.y + 0.25f * hn.y);
      *reinterpret_cast<float2*>(yc + (size_t)b * (plane / 4) + (size_t)I * nc + c0 / 2 +
                                 2 * lane) = v;
      ss = fmaf(v.x, v.x, ss);
      ss = fmaf(v.y, v.y, ss);
      hprev = hn;
    }
    if (partials) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      if (lane == 0) partials[(size_t)b * upi + rem] = (double)ss;
    }
  }
}

template <int W>
int launch_wide(const Band2D<float>& op, int B, const float* x, const float* y, float* r,
                double* partials, const int* active, int kch, cudaStream_t st) {
  WideArgs<W> a{};
  a.n = op.n;
  a.alpha = op.alpha;
  const StencilHost<float>& h = *op.st;
  for (int d = 0; d <= 2 * h.wK; ++d) {
    const float c = h.sK[d];
    a.k2[W - h.wK + d] = make_float2(c, c);
  }
  constexpr int NW = WideWarps<W>::value;
  const size_t sm = (size_t)NW * WideGeom<W>::words * sizeof(float);
  auto kern = k_res_wide<W>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (kch <= 0) kch = wide_chunks(op.n, W, (long long)B * (op.n / kWideSW), sms(), NW);
  const long long units = (long long)B * (op.n / kWideSW) * kch;
  long long grid = units;  // one block per SM while there are units for every SM
  if (grid > sms()) grid = sms();
  if (grid < 1) grid = 1;
  kern<<<(int)grid, 32 * NW, sm, st>>>(a, B, x, y, r, partials, active, kch);
  return (op.n / kWideSW) * kch;
}

}  // namespace

bool wide_residual_applies(const Band2D<float>& op, const float* x, const float* y) {
  if (!op.st || !op.st->valid) return false;
  const StencilHost<float>& h = *op.st;
  if (h.wM != 0 || h.nbM != 0 || h.nbK != 0 || h.sM[0] != 1.f) return false;
  if (h.wK <= 8 || h.wK > 32 || op.n % kWideSW != 0 || op.n < 2 * kWideSW) return false;
  return !((reinterpret_cast<uintptr_t>(x) & 15) || (y && (reinterpret_cast<uintptr_t>(y) & 15)));
}

int launch_residual_wide(const Band2D<float>& op, int B, const float* x, const float* y, float* r,
                         double* partials, const int* active, int kch, cudaStream_t st) {
  if (kch > wide_chunks_max(op.n)) kch = wide_chunks_max(op.n);
  return op.st->wK <= 16 ? launch_wide<16>(op, B, x, y, r, partials, active, kch, st)
                         : launch_wide<32>(op, B, x, y, r, partials, active, kch, st);
}

bool restrict_fw_applies(int n) {
  return n % 128 == 0 && (n / 2) % kRsBand == 0 &&
         (long long)(n / 128) * ((n / 2) / kRsBand) <= kMaxPartsPerItem;
}

int launch_restrict_fw(int n, int B, const float* r, float* yc, double* partials, const int* active,
                       cudaStream_t st) {
  const long long units = (long long)B * (n / 128) * ((n / 2) / kRsBand);
  long long grid = (units + kRsWarps - 1) / kRsWarps;
  const long long cap = 16LL * sms();
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  k_restrict_fw<<<(int)grid, 32 * kRsWarps, 0, st>>>(n, B, r, yc, partials, active);
  return (n / 128) * ((n / 2) / kRsBand);
}

}  // namespace nmg
