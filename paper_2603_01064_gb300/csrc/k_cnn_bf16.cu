// CNN smoother h = N(b / ||b||) ||b|| (Algorithms 3/4) of the bf16
// refinement forms: hidden 32 -> 32 layers on the tensor cores with
// tcgen05.mma (fp32 accumulators in tensor memory), first (1 -> 32) and
// last (32 -> 1) layers in fp32 SIMT (2% of the flops; they are bound by
// their activation traffic).
//
// Hidden layer = implicit GEMM  D[pixel][cout] = sum over the 9 taps and 32
// input channels of A[pixel + shift(tap)][cin] * W[tap][cin][cout].  One MMA
// tile is M = 128 output pixels arranged as 16 image rows x 8 columns, so the
// eight-row groups of the K-major no-swizzle operand layout are image rows:
// with the input tile staged in shared memory as [channel chunk of 8][tile
// row][tile column][8 channels], the operand of tap (dy, dx) is the same
// layout started dy rows and dx pixels further on, and the group stride
// (SBO) is one staged row.  A block tile is 16 x 16 output pixels (two M
// tiles side by side): 9 taps x 2 K halves = 18 MMAs of 128 x 32 x 16 per M
// tile and operand pair.
//
// Levels with n >= 32 use a warp-specialised persistent kernel: one warp
// issues TMA tensor copies of the input tiles (the halo outside the image is
// zero-filled by the copy engine) into a ring of shared-memory stages, one
// warp (fast form) or one warp per M tile (split forms) issues the MMAs of a
// tile into one of two tensor-memory accumulators as soon as its stage is
// full, and four (fast form) or eight (split forms)
// warps drain the other accumulator (tensor memory -> registers -> bias,
// ReLU -> 16-bit values -> global).  Stages and
// accumulators are handed over with mbarriers (full/empty, acc_full/
// acc_empty).  Smaller levels use a single-role version that stages with
// cp.async and overlaps one tile ahead.  Every mbarrier wait is bounded; on
// timeout the block records an error code, stops and releases its tensor
// memory.
//
// Split form (SPLIT = 1, the default bf16 form): the trained smoothers
// amplify rounding of their hidden activations (large, cancelling weights),
// so a single bf16 rounding (2^-9 relative) moves a cycle's iterate by
// percents.  Activations are stored as hi + lo bf16 pairs (v = hi + lo,
// |lo| <= 2^-9 |v|; hi channels in chunks 0-3, lo in chunks 4-7) and each
// product is formed from bf16 MMAs a_hi*w_hi + a_hi*w_lo + a_lo*w_hi,
// accumulated in fp32.  The SIMT layers compute in fp32.
//
// Three-term bf16 form (SPLIT = 3): every operand is a sum of three bf16
// values, v = v1 + v2 + v3 (each the bf16 rounding of what the previous
// terms leave, 2^-25 relative together: fp32-level), activations in chunks
// 0-3 / 4-7 / 8-11, weights in three 32-column blocks of B.  Each product
// is formed from the six MMAs whose terms are of order 2^-16 or larger,
// a1*(w1 + w2 + w3) + a2*(w1 + w2) + a3*w1, accumulated in fp32; the dropped
// products are below 2^-24 relative.  Trained smoothers with large,
// cancelling weights amplify the pair forms' 2^-16 .. 2^-18 errors (of the
// activations and of the weights alike) past a 1e-3 per-cycle error; this
// form keeps a cycle within about 1e-5 of fp64.
//
// fp16 split form (SPLIT = 2): the same [hi | lo] pairs and MMAs with fp16
// operands (11-bit significands: hi + lo carries 2^-22 instead of 2^-16).
// fp16's range is narrow, so the network runs on sigma-scaled values: the
// input b / ||b|| (RMS 1/n on an n x n level) is multiplied by sigma =
// max(1, n/4), every bias by sigma, and the output by 1/sigma.  ReLU is
// positively homogeneous and sigma is a power of two, so the scaling is
// exact; hidden activations then have RMS between about 0.25 and 10, and
// values above fp16's largest finite value are clamped to it rather than
// becoming infinite.
#include <cuda.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "nmg_internal.h"

namespace nmg {

namespace {

constexpr int TILE = 16;                // output tile side (pixels)
constexpr int NT = 2;                   // M tiles per block tile (columns 0-7, 8-15)
constexpr int RW = TILE + 2;            // staged input row pitch in pixels
constexpr int RH = TILE + 2;            // staged input rows
constexpr int CH_BYTES = RH * RW * 16;  // one 8-channel chunk of the staged tile
constexpr int WIDTH = 32;
constexpr int THREADS = 128;
// 16-bit terms per operand: 1 (fast form), 2 (pair forms), 3 (SPLIT = 3)
template <int SPLIT> struct TERMS { static constexpr int value = SPLIT == 3 ? 3 : (SPLIT ? 2 : 1); };
// MMA N of the hi A operand: one 32-column block per weight term.  Pair
// forms: 64 = [w_hi | w_lo], so the hi A operand's MMA forms a_hi*w_hi and
// a_hi*w_lo (summed in the epilogue) and the lo A operand's MMA uses N = 32
// (w_hi only).  SPLIT = 3: 96 = [w_1 | w_2 | w_3]; the middle A term takes
// N = 64 ([w_1 | w_2]) and the last N = 32 (w_1).
template <int SPLIT> struct NB { static constexpr int value = 32 * TERMS<SPLIT>::value; };
// TMEM columns allocated: two accumulators of NT x NB columns, rounded up to
// a power of two
template <int SPLIT> struct TMC { static constexpr int value = SPLIT == 3 ? 512 : (SPLIT ? 256 : 128); };
// 8-channel chunk planes of one pixel's activations (4 per term)
template <int SPLIT> struct ACHS { static constexpr int value = 4 * TERMS<SPLIT>::value; };
// Every mbarrier wait is bounded by the context's wait limit (ctl[0], in
// nanoseconds, set on the host; 2 s by default).  A block that gives up
// records the error, stops its roles and then drains what it still has in
// flight (its tensor-copy writes into shared memory, its MMAs into tensor
// memory) before it releases tensor memory and exits; those drain waits are
// bounded by kDrainNs, not by the settable limit.  ctl[1] != 0 is a test
// hook: the MMA issuers of the warp-specialised kernel first wait on a
// barrier nothing arrives at, so the launch gives up after the wait limit.
constexpr unsigned long long kDrainNs = 1000000000ull;
constexpr int B_HALF = 9 * 4 * WIDTH * 16;  // bf16 weights of a hidden layer for N = 32

// per layer: hidden layers use bf16 weights in the MMA B layout
// [tap 9][kchunk 4][n NB][8 cin] with n = cout (fast) or n = cout for w_hi and
// 32 + cout for w_lo (split); first/last layers use fp32 weights [c][tap]
// and fp32 biases.
struct LayerPack {
  const __nv_bfloat16* w;
  const float* wf;
  const float* bias;
  int has_lo;
  float bias0;          // host copy of the output layer's bias
  int bias_host_valid;
};
// first layer's weights [cout][tap] and biases, passed by value as kernel
// parameters: every multiply-add of the layer reads its weight straight from
// the constant bank
struct FirstW {
  float w[WIDTH * 9];
  float b[WIDTH];
  float2 w2[9][WIDTH / 2];  // w2[t][p] = (w[2p][t], w[2p + 1][t]): channel pairs
};
// the 32 -> 1 output layer's weights as channel pairs per tap, passed by
// value to the last hidden layer (its epilogue's packed FMAs read them from
// the constant bank): w[t][p] = (w4[2p][t], w4[2p + 1][t])
struct OutW {
  float2 w[9][WIDTH / 2];
};
struct Bf16Pack {
  int layers;
  int split;
  LayerPack l[kMaxCnnLayers];
  FirstW first;  // host copy of layer 0
  OutW last;     // host copy of the output layer
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// SM100 shared-memory matrix descriptor, no swizzle (K-major canonical
// layout ((8, m), 2) : ((16 B, SBO), LBO)).
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;
}

// instruction descriptor, kind::f16: bf16 (f16 = false) or fp16 A and B
// (format fields 0 = f16, 1 = bf16), fp32 D, both K-major
__host__ __device__ constexpr uint32_t make_idesc(int M, int N, bool f16 = false) {
  return (1u << 4) | (f16 ? 0u : (1u << 7) | (1u << 10)) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// scale of the fp16 split form's network values on an n x n level (see the
// header comment); 1 for the bf16 forms
template <int SPLIT>
__host__ __device__ __forceinline__ float net_scale(int n) {
  return SPLIT == 2 ? (float)(n >= 4 ? n / 4 : 1) : 1.f;
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait for a phase of an mbarrier, giving up after limit_ns
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity,
                                                  unsigned long long limit_ns) {
  if (mbar_try_wait(mbar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (unsigned it = 1;; ++it) {
    if (mbar_try_wait(mbar, parity)) return true;
    if ((it & 63u) == 0 && global_ns() - t0 > limit_ns) return false;
  }
}

// commit every MMA this thread issued to `mbar` and wait (bounded by
// kDrainNs) until they have completed: their tensor-memory writes are done
__device__ __forceinline__ void drain_mmas(uint32_t mbar, int* err) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
  if (!mbar_wait_bounded(mbar, 0u, kDrainNs)) atomicExch(err, 2);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}

// 32 lanes x 32 columns of fp32 from tensor memory (this warp's lane quarter)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Activations live in a chunk-planar layout: [image][chunk][y][x][8]
// (16-bit values; chunk c holds channels 8c .. 8c+7, chunks 0-3 the hi parts
// and 4-7 the lo parts in the split forms), so that one 16-byte chunk of a
// pixel row is contiguous in its plane: a TMA tile copy of one chunk moves
// whole 18-pixel rows, and a warp storing chunk c of its 32 pixels writes
// contiguous runs.  px0: the pixel's chunk-0 address (nullptr: not stored),
// cstride: elements between chunk planes.
template <int SPLIT>
__device__ __forceinline__ void store_pixel_planar(const float* a, __nv_bfloat16* px0,
                                                   size_t cstride) {
  if (!px0) return;
  if (SPLIT == 3) {
    // three bf16 terms: t1 = bf16(a), t2 = bf16(a - t1), t3 = bf16(a - t1 - t2)
    // (both differences are exact in fp32)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t t1[4], t2[4], t3[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float a0 = a[8 * q + 2 * c], a1 = a[8 * q + 2 * c + 1];
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(a0, a1);
        const float r0 = a0 - __low2float(h2), r1 = a1 - __high2float(h2);
        const __nv_bfloat162 m2 = __floats2bfloat162_rn(r0, r1);
        const __nv_bfloat162 l2 =
            __floats2bfloat162_rn(r0 - __low2float(m2), r1 - __high2float(m2));
        t1[c] = *reinterpret_cast<const uint32_t*>(&h2);
        t2[c] = *reinterpret_cast<const uint32_t*>(&m2);
        t3[c] = *reinterpret_cast<const uint32_t*>(&l2);
      }
      *reinterpret_cast<uint4*>(px0 + q * cstride) = make_uint4(t1[0], t1[1], t1[2], t1[3]);
      *reinterpret_cast<uint4*>(px0 + (4 + q) * cstride) = make_uint4(t2[0], t2[1], t2[2], t2[3]);
      *reinterpret_cast<uint4*>(px0 + (8 + q) * cstride) = make_uint4(t3[0], t3[1], t3[2], t3[3]);
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float a0 = a[8 * q + 2 * c], a1 = a[8 * q + 2 * c + 1];
      if (SPLIT == 2) {
        const float c0 = fminf(a0, 65504.f), c1 = fminf(a1, 65504.f);
        __half2 h2 = __floats2half2_rn(c0, c1);
        __half2 l2 = __floats2half2_rn(c0 - __low2float(h2), c1 - __high2float(h2));
        hi[c] = *reinterpret_cast<uint32_t*>(&h2);
        lo[c] = *reinterpret_cast<uint32_t*>(&l2);
      } else {
        __nv_bfloat162 h2 = __floats2bfloat162_rn(a0, a1);
        hi[c] = *reinterpret_cast<uint32_t*>(&h2);
        if (SPLIT) {
          __nv_bfloat162 l2 = __floats2bfloat162_rn(a0 - __low2float(h2), a1 - __high2float(h2));
          lo[c] = *reinterpret_cast<uint32_t*>(&l2);
        }
      }
    }
    *reinterpret_cast<uint4*>(px0 + q * cstride) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    if (SPLIT)
      *reinterpret_cast<uint4*>(px0 + (4 + q) * cstride) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
  }
}

// ---------------------------------------------------------------------------
// first layer 1 -> 32 (fp32 SIMT): a = ReLU(b1 + W1 * (b / s)), stored as
// 16-bit values (fp16 split form: a = ReLU(sigma b1 + W1 * (sigma b / s)))
// ---------------------------------------------------------------------------
template <int SPLIT>
__global__ void __launch_bounds__(256)
k_first_simt(int n, const float* __restrict__ bsrc, __nv_bfloat16* __restrict__ aout,
             const __grid_constant__ FirstW fw, const double* __restrict__ snorm,
             const int* __restrict__ active, int tiles_x) {
  constexpr int ACHN = ACHS<SPLIT>::value;  // chunk planes per image
  const int b = blockIdx.y;
  if (!active[b]) return;
  // ||b|| = 0 (tested on the bits): h = 0 is written by the last layer.
  // sigma / ||b|| is formed in fp32 from ||b|| rounded to fp32, once per
  // block (fp64 arithmetic runs at 1/64 of the fp32 rate); the first hidden
  // layer's fused form computes the same value
  const long long sbits = __double_as_longlong(snorm[b]);
  if ((sbits << 1) == 0) return;
  __shared__ float xs[RH][RW + 1];
  __shared__ float inv_s;
  const int tid = threadIdx.x;
  const float sig = net_scale<SPLIT>(n);
  if (tid == 0) inv_s = __fdiv_rn(sig, (float)__longlong_as_double(sbits));
  const int y0 = (blockIdx.x / tiles_x) * TILE, x0 = (blockIdx.x % tiles_x) * TILE;
  const size_t plane = (size_t)n * n;
  __syncthreads();
  const float inv = inv_s;
  const float* bb = bsrc + (size_t)b * plane;
  for (int i = tid; i < RH * RW; i += 256) {
    int ry = i / RW, rx = i % RW;
    int y = y0 + ry - 1, x = x0 + rx - 1;
    xs[ry][rx] = (y >= 0 && y < n && x >= 0 && x < n) ? bb[(size_t)y * n + x] * inv : 0.f;
  }
  __syncthreads();
  const int ry = tid / TILE, rx = tid % TILE;
  const int y = y0 + ry, x = x0 + rx;
  const bool in = y < n && x < n;
  float v[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) v[t] = xs[ry + t / 3][rx + t % 3];
  // channel pairs as packed two-lane FMAs (fma.rn.f32x2)
  float2 v2[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) v2[t] = make_float2(v[t], v[t]);
  float a[WIDTH];
#pragma unroll
  for (int p = 0; p < WIDTH / 2; ++p) {
    float2 acc = make_float2(sig * fw.b[2 * p], sig * fw.b[2 * p + 1]);
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      unsigned long long d;
      const float2 w = fw.w2[t][p];
      asm("fma.rn.f32x2 %0, %1, %2, %3;"
          : "=l"(d)
          : "l"(*reinterpret_cast<const unsigned long long*>(&w)),
            "l"(*reinterpret_cast<const unsigned long long*>(&v2[t])),
            "l"(*reinterpret_cast<const unsigned long long*>(&acc)));
      acc = *reinterpret_cast<float2*>(&d);
    }
    a[2 * p] = fmaxf(acc.x, 0.f);
    a[2 * p + 1] = fmaxf(acc.y, 0.f);
  }
  store_pixel_planar<SPLIT>(
      a, in ? aout + ((size_t)b * ACHN * plane + (size_t)y * n + x) * 8 : nullptr, plane * 8);
}

// All MMAs of one block tile: for each M tile (8-column half), 9 taps x 2 K
// halves, one MMA per A operand (hi, and lo in the split form).  Descriptors
// are built once; per MMA only a compile-time offset is added to their
// start-address field.
template <int SPLIT, int PITCH, int MT0 = 0, int MTN = NT>
__device__ __forceinline__ void issue_tile_mmas(uint32_t a_base, uint32_t b_base, uint32_t d0) {
  constexpr int N = NB<SPLIT>::value;
  constexpr uint32_t idesc = make_idesc(128, N, SPLIT == 2);
  // lo A operand: N = 32 (w_hi only, the first 32 rows of B) accumulating
  // into the hi columns; a_lo * w_lo (~2^-32 relative) is not formed.
  // SPLIT = 3: the middle A term with N = 64 ([w_1 | w_2], the first 64
  // rows of B) and the last with N = 32 (w_1)
  constexpr uint32_t idesc_lo = make_idesc(128, 32, SPLIT == 2);
  constexpr uint32_t idesc_mid = make_idesc(128, 64, false);
  const uint64_t ad0 = make_desc(a_base, PITCH, RW * 16);
  const uint64_t bd0 = make_desc(b_base, N * 16, 128);
  // the M tiles' accumulation chains are interleaved (consecutive MMAs write
  // different accumulators)
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
#pragma unroll
    for (int kh = 0; kh < 2; ++kh) {
      const uint32_t boff = ((tap * 4 + 2 * kh) * N * 16) >> 4;
#pragma unroll
      for (int mt = MT0; mt < MT0 + MTN; ++mt) {
        const uint32_t d = d0 + mt * N;
        const uint32_t aoff = (2 * kh * PITCH + ((tap / 3) * RW + 8 * mt + (tap % 3)) * 16) >> 4;
        mma_bf16(d, ad0 + aoff, bd0 + boff, idesc, (tap | kh) ? 1u : 0u);
      }
      if (SPLIT == 3) {
#pragma unroll
        for (int mt = MT0; mt < MT0 + MTN; ++mt) {
          const uint32_t d = d0 + mt * N;
          const uint32_t aoff = (2 * kh * PITCH + ((tap / 3) * RW + 8 * mt + (tap % 3)) * 16) >> 4;
          mma_bf16(d, ad0 + aoff + ((4 * PITCH) >> 4), bd0 + boff, idesc_mid, 1u);
          mma_bf16(d, ad0 + aoff + ((8 * PITCH) >> 4), bd0 + boff, idesc_lo, 1u);
        }
      } else if (SPLIT) {
#pragma unroll
        for (int mt = MT0; mt < MT0 + MTN; ++mt) {
          const uint32_t d = d0 + mt * N;
          const uint32_t aoff = (2 * kh * PITCH + ((tap / 3) * RW + 8 * mt + (tap % 3)) * 16) >> 4;
          mma_bf16(d, ad0 + aoff + ((4 * PITCH) >> 4), bd0 + boff, idesc_lo, 1u);
        }
      }
    }
  }
}

// Epilogue of one pixel from 32 (fast) or 64 (split: hi + lo weight halves)
// accumulator columns: bias, ReLU, then either the bf16 activation store
// (FUSE = 0) or, for the last hidden layer (FUSE = 1), the contraction with
// the 32 -> 1 output layer's weights w4[c][tap] into 9 per-tap partial sums
// written as fp32 planes g[tap][pixel] (plane stride gstride).
template <int SPLIT, int FUSE>
__device__ __forceinline__ void finish_pixel(uint32_t taddr, const float* __restrict__ bsc,
                                             const float* __restrict__ bias_g,
                                             __nv_bfloat16* dst, size_t cstride,
                                             float* gdst, size_t gstride,
                                             const float* __restrict__ w4, const OutW& ow,
                                             bool store) {
  float v[32];
  tmem_ld32(taddr, v);
  if (SPLIT == 3) {
    // the w_2 and w_3 column blocks added in turn (one 32-column block of
    // registers at a time)
#pragma unroll
    for (int blk = 1; blk < 3; ++blk) {
      float w[32];
      tmem_ld32(taddr + 32 * blk, w);
#pragma unroll
      for (int c = 0; c < 32; c += 2) {
        unsigned long long* vp = reinterpret_cast<unsigned long long*>(&v[c]);
        asm("add.rn.f32x2 %0, %0, %1;" : "+l"(*vp) : "l"(*reinterpret_cast<const unsigned long long*>(&w[c])));
      }
    }
  } else if (SPLIT) {
    float w[32];
    tmem_ld32(taddr + 32, w);
#pragma unroll
    for (int c = 0; c < 32; c += 2) {  // packed fp32x2 adds
      unsigned long long* vp = reinterpret_cast<unsigned long long*>(&v[c]);
      asm("add.rn.f32x2 %0, %0, %1;" : "+l"(*vp) : "l"(*reinterpret_cast<const unsigned long long*>(&w[c])));
    }
  }
  if (SPLIT) {
#pragma unroll
    for (int c = 0; c < 32; c += 2) {
      unsigned long long* vp = reinterpret_cast<unsigned long long*>(&v[c]);
      asm("add.rn.f32x2 %0, %0, %1;" : "+l"(*vp) : "l"(*reinterpret_cast<const unsigned long long*>(&bsc[c])));
      v[c] = fmaxf(v[c], 0.f);
      v[c + 1] = fmaxf(v[c + 1], 0.f);
    }
  } else {
    // single-bf16 form (network scale 1): the bias from global memory (its
    // epilogue warps hold two M tiles; loads hoisted from shared memory
    // would cost the registers of a second CTA per SM)
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = fmaxf(v[c] + bias_g[c], 0.f);
  }
  if (!FUSE) {
    store_pixel_planar<SPLIT>(v, store ? dst : nullptr, cstride);
    return;
  }
  if (!store) return;
  {
    // w4 is staged in shared memory as [tap][32 channels]; in the split
    // forms even and odd channels accumulate in the two lanes of packed
    // fp32x2 FMAs (the single-bf16 form keeps scalar FMAs: its epilogue
    // warps hold two M tiles and run out of registers otherwise)
    if (!SPLIT) {
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        const float4* wt = reinterpret_cast<const float4*>(w4 + t * 32);
        float g = 0.f;
#pragma unroll
        for (int c4 = 0; c4 < 8; ++c4) {
          const float4 w = wt[c4];
          g = fmaf(w.x, v[4 * c4], g);
          g = fmaf(w.y, v[4 * c4 + 1], g);
          g = fmaf(w.z, v[4 * c4 + 2], g);
          g = fmaf(w.w, v[4 * c4 + 3], g);
        }
        gdst[t * gstride] = g;
      }
      return;
    }
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      unsigned long long g2 = 0ull;  // (0.f, 0.f)
#pragma unroll
      for (int c4 = 0; c4 < 8; ++c4) {
        const float2 wa = ow.w[t][2 * c4], wb = ow.w[t][2 * c4 + 1];
        const float2 va = make_float2(v[4 * c4], v[4 * c4 + 1]);
        const float2 vb = make_float2(v[4 * c4 + 2], v[4 * c4 + 3]);
        asm("fma.rn.f32x2 %0, %1, %2, %0;"
            : "+l"(g2)
            : "l"(*reinterpret_cast<const unsigned long long*>(&wa)),
              "l"(*reinterpret_cast<const unsigned long long*>(&va)));
        asm("fma.rn.f32x2 %0, %1, %2, %0;"
            : "+l"(g2)
            : "l"(*reinterpret_cast<const unsigned long long*>(&wb)),
              "l"(*reinterpret_cast<const unsigned long long*>(&vb)));
      }
      const float2 g = *reinterpret_cast<const float2*>(&g2);
      gdst[t * gstride] = g.x + g.y;
    }
  }
}

// ---------------------------------------------------------------------------
// hidden layer 32 -> 32 on the tensor cores (pipelined, persistent)
// ---------------------------------------------------------------------------
template <int SPLIT, int FUSE>
__global__ void __launch_bounds__(THREADS)
k_hidden_tc(int n, int nimg, const __nv_bfloat16* __restrict__ ain,
            __nv_bfloat16* __restrict__ aout, float* __restrict__ gout, LayerPack lp,
            const float* __restrict__ w4, const __grid_constant__ OutW ow,
            const double* __restrict__ snorm, const int* __restrict__ active,
            int* __restrict__ err, int nbuf, const long long* __restrict__ ctl) {
  constexpr int ACH = ACHS<SPLIT>::value;  // 8-channel chunks per staged pixel
  constexpr int ABUF = ACH * CH_BYTES;
  constexpr int B_BYTES = TERMS<SPLIT>::value * B_HALF;
  constexpr int TMEM_COLS = TMC<SPLIT>::value;
  constexpr int NACC = NT * NB<SPLIT>::value;  // columns of one accumulator
  extern __shared__ __align__(16) unsigned char smem[];
  // nbuf operand buffers (1 when the grid covers every tile: no tile is
  // staged ahead, and two CTAs fit on an SM), then the weights
  unsigned char* Bs = smem + nbuf * ABUF;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ __align__(8) uint64_t drain_bar;  // completion of all MMAs issued (abort path)
  const unsigned long long wait_ns = (unsigned long long)ctl[0];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  __shared__ __align__(16) float w4s[FUSE ? 9 * 32 : 4];
  __shared__ __align__(16) float bsc[32];  // the layer's bias times the network scale
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  {
    const uint4* src = reinterpret_cast<const uint4*>(lp.w);
    uint4* dst = reinterpret_cast<uint4*>(Bs);
    for (int i = tid; i < B_BYTES / 16; i += THREADS) dst[i] = src[i];
    if (FUSE)
      for (int i = tid; i < 9 * 32; i += THREADS) w4s[i] = w4[(i % 32) * 9 + i / 32];
    if (tid < 32) bsc[tid] = net_scale<SPLIT>(n) * lp.bias[tid];
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[1])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&drain_bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t a_base0 = smem_u32(smem), b_base = smem_u32(Bs);
  const int tiles_x = (n + TILE - 1) / TILE;
  const int per_img = tiles_x * tiles_x;
  const int total = nimg * per_img;  // the launcher checks it fits
  const size_t plane = (size_t)n * n;

  auto valid = [&](int t) {
    const int b = t / per_img;
    return active[b] != 0 && snorm[b] != 0.0;
  };
  auto advance = [&](int t) {
    t += gridDim.x;
    while (t < total && !valid(t)) t += gridDim.x;
    return t;
  };
  auto stage = [&](int t, int buf) {
    const int b = t / per_img, tt = t - b * per_img;
    const int y0 = (tt / tiles_x) * TILE, x0 = (tt % tiles_x) * TILE;
    const __nv_bfloat16* ab = ain + (size_t)b * ACH * plane * 8;
    const uint32_t base = a_base0 + buf * ABUF;
    for (int i = tid; i < RH * RW * ACH; i += THREADS) {
      const int c = i % ACH, p = i / ACH;
      const int ry = p / RW, rx = p % RW;
      const int y = y0 + ry - 1, x = x0 + rx - 1;
      const bool in = y >= 0 && y < n && x >= 0 && x < n;
      const __nv_bfloat16* src = in ? ab + ((size_t)c * plane + (size_t)y * n + x) * 8 : ain;
      cp_async16(base + c * CH_BYTES + (ry * RW + rx) * 16, src, in ? 16u : 0u);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  auto wait_mma = [&](int buf, uint32_t parity) {
    if (!mbar_wait_bounded(smem_u32(&mbar[buf]), parity, wait_ns)) {
      atomicExch(err, 1);
      abort_flag = 1;
    }
  };
  auto epilogue = [&](int t, int acc) {
    const int b = t / per_img, tt = t - b * per_img;
    const int y0 = (tt / tiles_x) * TILE, x0 = (tt % tiles_x) * TILE;
    for (int mt = 0; mt < NT; ++mt) {
      const int m = warp * 32 + lane;
      const int y = y0 + (m >> 3), x = x0 + mt * 8 + (m & 7);
      const bool in = y < n && x < n;
      const size_t pix = (size_t)b * plane + (size_t)y * n + x;
      finish_pixel<SPLIT, FUSE>(
          tmem + ((uint32_t)(warp * 32) << 16) + acc * NACC + mt * NB<SPLIT>::value, bsc, lp.bias,
          aout + ((size_t)b * ACH * plane + (size_t)y * n + x) * 8, plane * 8,
          in ? gout + pix : gout, (size_t)nimg * plane, w4s, ow, in);
    }
  };

  int cur = blockIdx.x;
  while (cur < total && !valid(cur)) cur += gridDim.x;
  int prev = -1;
  uint32_t parity[2] = {0u, 0u};
  int k = 0;
  if (cur < total) stage(cur, 0);
  while (cur < total) {
    const int sb = k & 1;
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      issue_tile_mmas<SPLIT, CH_BYTES>(a_base0 + sb * ABUF, b_base, tmem + sb * NACC);
      mma_commit(smem_u32(&mbar[sb]));
    }
    const int nxt = advance(cur);
    if (prev >= 0) {
      // MMAs of the previous tile are done: its operand buffer is free and its
      // accumulator can be read
      wait_mma(sb ^ 1, parity[sb ^ 1]);
      parity[sb ^ 1] ^= 1u;
    }
    __syncthreads();
    if (abort_flag) break;
    if (nxt < total) stage(nxt, sb ^ 1);
    if (prev >= 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      epilogue(prev, sb ^ 1);
    }
    prev = cur;
    cur = nxt;
    ++k;
  }
  if (!abort_flag && prev >= 0) {
    const int lb = (k - 1) & 1;
    wait_mma(lb, parity[lb]);
    __syncthreads();
    if (!abort_flag) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      epilogue(prev, lb);
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  // after a timed-out wait, MMAs issued by thread 0 may still be writing
  // tensor memory: wait for all of them before releasing it
  if (abort_flag && tid == 0 && k > 0) drain_mmas(smem_u32(&drain_bar), err);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// ---------------------------------------------------------------------------
// hidden layer, warp-specialised: TMA producer / MMA issuer(s) / epilogue warps
// ---------------------------------------------------------------------------
constexpr int CH_PITCH = 5248;       // chunk stride in shared memory (128-byte multiple)
// warp 0 TMA, then the MMA issuer(s), then the epilogue warps in groups of
// four (one per tensor-memory lane quarter): the fast form has one group for
// both M tiles (it runs 2 CTAs per SM), the split forms one group per M tile
// (the epilogue converts twice the accumulator columns and is latency-bound
// with one warp per sub-partition)
template <int SPLIT, int FUSE> struct EPI { static constexpr int value = SPLIT ? 8 : 4; };
// MMA issuers: one per M tile in the split forms (a single issuing thread
// does not keep the tensor pipe fed with the split form's 72 MMAs per tile)
template <int SPLIT> struct ISS { static constexpr int value = SPLIT ? NT : 1; };
// warps that compute the first layer into the operand stages (FIRST = 1)
constexpr int kFirstWarps = 4;
template <int SPLIT, int FUSE, int FIRST = 0> struct WST {
  static constexpr int value =
      32 * (1 + ISS<SPLIT>::value + EPI<SPLIT, FUSE>::value + (FIRST ? kFirstWarps : 0));
};
__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
constexpr int kMaskImgs = 32768;  // images whose validity bits a block keeps in shared memory

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, int c4, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
      "r"(mbar)
      : "memory");
}

// FIRST = 1 (first hidden layer of the split forms): the operand stages are
// not copied from a first-layer output in global memory but computed in
// place by kFirstWarps extra warps from the level's input b: the 20 x 20
// input window of a tile (zero outside the image), then the 1 -> 32 layer
// a = ReLU(sigma b1 + W1 * (sigma b / s)) on the 18 x 18 pixels of the
// staged tile (zero outside the image, as the copy engine's fill), split
// into hi + lo 16-bit values in the stage's chunk-planar layout.  The 128
// bytes per pixel of the first layer's output never reach global memory.
template <int SPLIT, int STAGES, int FUSE, int FIRST = 0>
__global__ void __launch_bounds__(WST<SPLIT, FUSE, FIRST>::value, SPLIT ? 1 : 2)
k_hidden_ws(const __grid_constant__ CUtensorMap amap, int n, int nimg,
            __nv_bfloat16* __restrict__ aout, float* __restrict__ gout, LayerPack lp,
            const float* __restrict__ w4, const __grid_constant__ OutW ow,
            const double* __restrict__ snorm, const int* __restrict__ active,
            int* __restrict__ err, const float* __restrict__ bsrc,
            const __grid_constant__ FirstW fw, const long long* __restrict__ ctl) {
  constexpr int NTHR = WST<SPLIT, FUSE, FIRST>::value;
  static_assert(!FIRST || (SPLIT && !FUSE), "the fused first layer serves the split forms' first hidden layer");
  constexpr int ACH = ACHS<SPLIT>::value;
  constexpr int SBYTES = ACH * CH_PITCH;           // one stage
  constexpr uint32_t TX = ACH * RH * RW * 16;      // bytes the copies of one stage write
  constexpr int B_BYTES = TERMS<SPLIT>::value * B_HALF;
  constexpr int TMEM_COLS = TMC<SPLIT>::value;
  constexpr int NACC = NT * NB<SPLIT>::value;
  extern __shared__ __align__(16) unsigned char smem_raw_ws[];
  // stage buffers start on a 1024-byte boundary (TMA destinations need 128)
  unsigned char* smem = smem_raw_ws + ((1024u - (smem_u32(smem_raw_ws) & 1023u)) & 1023u);
  unsigned char* Bs = smem + STAGES * SBYTES;
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], acc_full[2], acc_empty[2];
  // drain[i]: completion of MMA issuer i's MMAs (abort path); stall_bar:
  // the barrier nothing arrives at (test hook ctl[1])
  __shared__ __align__(8) uint64_t drain[NT], stall_bar;
  const unsigned long long wait_ns = (unsigned long long)ctl[0];
  const bool stall = ctl[1] != 0;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  __shared__ __align__(16) float w4s[FUSE ? 9 * 32 : 4];
  __shared__ __align__(16) float bsc[32];  // the layer's bias times the network scale
  // one bit per image: active and with a nonzero norm.  Every role walks the
  // tile sequence; reading these from global memory per tile would put an L2
  // round trip between consecutive tiles of the MMA issuer.
  __shared__ uint32_t vmask[kMaskImgs / 32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  {
    const uint4* src = reinterpret_cast<const uint4*>(lp.w);
    uint4* dst = reinterpret_cast<uint4*>(Bs);
    for (int i = tid; i < B_BYTES / 16; i += NTHR) dst[i] = src[i];
    if (FUSE)
      for (int i = tid; i < 9 * 32; i += NTHR) w4s[i] = w4[(i % 32) * 9 + i / 32];
    if (tid < 32) bsc[tid] = net_scale<SPLIT>(n) * lp.bias[tid];
    if (nimg <= kMaskImgs)
      for (int b0 = warp * 32; b0 < nimg; b0 += NTHR) {  // warp-uniform loop
        const int b = b0 + lane;
        const unsigned m = __ballot_sync(0xffffffffu, b < nimg && active[b] != 0 && snorm[b] != 0.0);
        if (lane == 0) vmask[b0 >> 5] = m;
      }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 32) {
    for (int i = 0; i < STAGES; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[i])),
                   "r"(FIRST ? 32 * kFirstWarps : 1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[i])),
                   "r"(ISS<SPLIT>::value));
    }
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&acc_full[i])),
                   "r"(ISS<SPLIT>::value));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&acc_empty[i])),
                   "r"(EPI<SPLIT, FUSE>::value));
    }
    for (int i = 0; i < NT; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&drain[i])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&stall_bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const int tiles_x = (n + TILE - 1) / TILE;
  const int per_img = tiles_x * tiles_x;
  const int total = nimg * per_img;  // the launcher checks it fits
  const size_t plane = (size_t)n * n;
  auto valid = [&](int t) {
    const int b = t / per_img;
    if (nimg <= kMaskImgs) return ((vmask[b >> 5] >> (b & 31)) & 1u) != 0;
    return active[b] != 0 && snorm[b] != 0.0;
  };
  auto first = [&]() {
    int t = blockIdx.x;
    while (t < total && !valid(t)) t += gridDim.x;
    return t;
  };
  auto advance = [&](int t) {
    t += gridDim.x;
    while (t < total && !valid(t)) t += gridDim.x;
    return t;
  };
  // bounded wait; returns false (and flags the error) on timeout
  auto wait = [&](uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(smem_u32(bar), parity)) return true;
    const uint64_t t0 = global_ns();
    for (unsigned it = 1;; ++it) {
      if (mbar_try_wait(smem_u32(bar), parity)) return true;
      if ((it & 63u) == 0 && (*(volatile int*)&abort_flag || global_ns() - t0 > wait_ns)) {
        atomicExch(err, 1);
        abort_flag = 1;
        return false;
      }
    }
  };

  constexpr int FW0 = 1 + ISS<SPLIT>::value + EPI<SPLIT, FUSE>::value;  // first producer warp
  if (FIRST && warp >= FW0) {
    // ---- first-layer producers (FIRST = 1)
    constexpr int PT = 32 * kFirstWarps;
    constexpr int XW = TILE + 4;  // input window side
    constexpr int XPT = (XW * XW + PT - 1) / PT;  // window values per thread
    __shared__ float xs[2][XW * XW];
    __shared__ int stop_sh[2];
    const int pt = tid - 32 * FW0;
    const float sig = net_scale<SPLIT>(n);
    // the next tile's input window and ||b|| are loaded into registers one
    // tile ahead, so their latency hides behind the current tile's layer
    float pre[XPT];
    float pre_s = 1.f;
    auto fetch = [&](int t) {
      const int b = t / per_img, tt = t - b * per_img;
      const int y0 = (tt / tiles_x) * TILE, x0 = (tt % tiles_x) * TILE;
      const float* bb = bsrc + (size_t)b * plane;
#pragma unroll
      for (int j = 0; j < XPT; ++j) {
        const int k = pt + j * PT;
        const int y = y0 + k / XW - 2, x = x0 + k % XW - 2;
        pre[j] = (k < XW * XW && y >= 0 && y < n && x >= 0 && x < n) ? bb[(size_t)y * n + x] : 0.f;
      }
      pre_s = (float)snorm[b];
    };
    int i = 0;
    int t = first();
    if (t < total) fetch(t);
    for (; t < total; ++i) {
      const int s = i % STAGES, xb = i & 1;
      const int b = t / per_img, tt = t - b * per_img;
      const int y0 = (tt / tiles_x) * TILE, x0 = (tt % tiles_x) * TILE;
#pragma unroll
      for (int j = 0; j < XPT; ++j)
        if (pt + j * PT < XW * XW) xs[xb][pt + j * PT] = pre[j];
      // sigma / ||b|| in fp32 (fp64 arithmetic runs at 1/64 of the fp32
      // rate); the same value k_first_simt forms
      const float inv = __fdiv_rn(sig, pre_s);
      const int tn = advance(t);
      if (tn < total) fetch(tn);
      // one thread waits for the stage to be free; the decision to stop
      // reaches the other producers through the barrier
      if (pt == 0)
        stop_sh[xb] = (i >= STAGES && !wait(&empty[s], (uint32_t)((i / STAGES - 1) & 1))) ? 1 : 0;
      named_bar_sync(1, PT);
      if (stop_sh[xb]) break;
      unsigned char* stage = smem + s * SBYTES;
      for (int p = pt; p < RH * RW; p += PT) {
        const int ry = p / RW, rx = p % RW;
        const int y = y0 + ry - 1, x = x0 + rx - 1;
        float a[WIDTH];
        if (y >= 0 && y < n && x >= 0 && x < n) {
          float2 v2[9];
#pragma unroll
          for (int tp = 0; tp < 9; ++tp) {
            const float v = xs[xb][(ry + tp / 3) * XW + rx + tp % 3] * inv;
            v2[tp] = make_float2(v, v);
          }
#pragma unroll
          for (int q2 = 0; q2 < WIDTH / 2; ++q2) {
            float2 acc = make_float2(sig * fw.b[2 * q2], sig * fw.b[2 * q2 + 1]);
#pragma unroll
            for (int tp = 0; tp < 9; ++tp) {
              unsigned long long d;
              const float2 w = fw.w2[tp][q2];
              asm("fma.rn.f32x2 %0, %1, %2, %3;"
                  : "=l"(d)
                  : "l"(*reinterpret_cast<const unsigned long long*>(&w)),
                    "l"(*reinterpret_cast<const unsigned long long*>(&v2[tp])),
                    "l"(*reinterpret_cast<const unsigned long long*>(&acc)));
              acc = *reinterpret_cast<float2*>(&d);
            }
            a[2 * q2] = fmaxf(acc.x, 0.f);
            a[2 * q2 + 1] = fmaxf(acc.y, 0.f);
          }
        } else {
#pragma unroll
          for (int c = 0; c < WIDTH; ++c) a[c] = 0.f;
        }
        store_pixel_planar<SPLIT>(a, reinterpret_cast<__nv_bfloat16*>(stage + p * 16),
                                  CH_PITCH / 2);
      }
      // generic-proxy writes made visible to the tensor core's reads
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(&full[s]));
      t = tn;
    }
  } else if (warp == 0) {
    // ---- TMA producer
    if (lane == 0 && !FIRST) {
      int i = 0;
      for (int t = first(); t < total; t = advance(t), ++i) {
        const int s = i % STAGES;
        if (i >= STAGES && !wait(&empty[s], (uint32_t)((i / STAGES - 1) & 1))) break;
        const int b = t / per_img, tt = t - b * per_img;
        const int y0 = (tt / tiles_x) * TILE, x0 = (tt % tiles_x) * TILE;
        const uint32_t fb = smem_u32(&full[s]);
        mbar_expect_tx(fb, TX);
        const uint32_t dst = smem_u32(smem + s * SBYTES);
        for (int c = 0; c < ACH; ++c) tma_load_5d(dst + c * CH_PITCH, &amap, 0, x0 - 1, y0 - 1, c, b, fb);
      }
      if (*(volatile int*)&abort_flag) {
        // copies issued for a stage land whether or not its tile was
        // consumed: wait for the last one of every stage (the phase of tile
        // j is (j / STAGES) & 1; a phase already completed returns at once)
        for (int s = 0; s < STAGES && s < i; ++s) {
          const int last = s + ((i - 1 - s) / STAGES) * STAGES;
          if (!mbar_wait_bounded(smem_u32(&full[s]), (uint32_t)((last / STAGES) & 1), kDrainNs))
            atomicExch(err, 2);
        }
      }
    }
  } else if (warp <= ISS<SPLIT>::value) {
    // ---- MMA issuer(s): all M tiles, or M tile warp - 1
    if (lane == 0) {
      const uint32_t b_base = smem_u32(Bs);
      int i = 0;
      // test hook: a wait that runs out before any MMA is issued
      const bool go = !stall || wait(&stall_bar, 0u);
      for (int t = go ? first() : total; t < total; t = advance(t), ++i) {
        const int s = i % STAGES, a = i & 1;
        if (!wait(&full[s], (uint32_t)((i / STAGES) & 1))) break;
        if (i >= 2 && !wait(&acc_empty[a], (uint32_t)((i / 2 - 1) & 1))) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sa = smem_u32(smem + s * SBYTES), d0 = tmem + a * NACC;
        if (ISS<SPLIT>::value == 1)
          issue_tile_mmas<SPLIT, CH_PITCH>(sa, b_base, d0);
        else if (warp == 1)
          issue_tile_mmas<SPLIT, CH_PITCH, 0, 1>(sa, b_base, d0);
        else
          issue_tile_mmas<SPLIT, CH_PITCH, 1, 1>(sa, b_base, d0);
        mma_commit(smem_u32(&empty[s]));
        mma_commit(smem_u32(&acc_full[a]));
      }
      // after an abort this issuer's MMAs may still be writing tensor memory
      if (*(volatile int*)&abort_flag && i > 0) drain_mmas(smem_u32(&drain[warp - 1]), err);
    }
  } else {
    // ---- epilogue warps: lane quarter q = warp % 4 of tensor memory; group
    // g of four consecutive warps takes M tile g (both with one group)
    constexpr int GROUPS = EPI<SPLIT, FUSE>::value / 4;
    constexpr int MTW = GROUPS >= NT ? 1 : NT;  // M tiles per epilogue warp
    const int q = warp & 3;
    const int mt0 = GROUPS >= NT ? (warp - 1 - ISS<SPLIT>::value) >> 2 : 0;
    int i = 0;
    for (int t = first(); t < total; t = advance(t), ++i) {
      const int a = i & 1;
      if (!wait(&acc_full[a], (uint32_t)((i / 2) & 1))) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int b = t / per_img, tt = t - b * per_img;
      const int y0 = (tt / tiles_x) * TILE, x0 = (tt % tiles_x) * TILE;
      const int m = q * 32 + lane;
      const int y = y0 + (m >> 3);
      for (int mt = mt0; mt < mt0 + MTW; ++mt) {
        const int x = x0 + mt * 8 + (m & 7);
        const bool in = y < n && x < n;
        const size_t pix = (size_t)b * plane + (size_t)y * n + x;
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + a * NACC + mt * NB<SPLIT>::value;
        __nv_bfloat16* dst = aout + ((size_t)b * ACH * plane + (size_t)y * n + x) * 8;
        float* gd = in ? gout + pix : gout;
        finish_pixel<SPLIT, FUSE>(ta, bsc, lp.bias, dst, plane * 8, gd, (size_t)nimg * plane, w4s,
                                  ow, in);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&acc_empty[a]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// tensor maps over the chunk-planar activation buffers, created on first use
struct MapEntry {
  const void* ptr;
  int n, nimg, cw;
  CUtensorMap map;
};
std::vector<MapEntry>& map_cache() {
  static std::vector<MapEntry> v;
  return v;
}
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}
const CUtensorMap* act_map(const void* ptr, int n, int nimg, int cw) {
  for (auto& e : map_cache())
    if (e.ptr == ptr && e.n == n && e.nimg == nimg && e.cw == cw) return &e.map;
  EncodeTiledFn fn = encode_fn();
  if (!fn) return nullptr;
  MapEntry e{ptr, n, nimg, cw, {}};
  // chunk-planar activations [image][chunk][y][x][8]: one 16-byte chunk per
  // pixel and plane; the box is one chunk of an 18 x 18 pixel tile
  const cuuint64_t ch = (cuuint64_t)cw / 8;
  cuuint64_t dims[5] = {8, (cuuint64_t)n, (cuuint64_t)n, ch, (cuuint64_t)nimg};
  cuuint64_t strides[4] = {16, (cuuint64_t)n * 16, (cuuint64_t)n * n * 16, ch * n * n * 16};
  cuuint32_t box[5] = {8, (cuuint32_t)RW, (cuuint32_t)RH, 1, 1};
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  CUresult r = fn(&e.map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(ptr), dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return nullptr;
  map_cache().push_back(e);
  return &map_cache().back().map;
}

// last layer from the fused partial sums: h[p] = s (b4 + sum_tap g[tap][p + off(tap)])
// with zero padding outside the image; fp16 split form (g carries the
// network scale sigma): h = (s / sigma) (sigma b4 + sum_tap g), bscale = sigma.
// Four pixels of a row per thread (n % 4 == 0): each tap reads one aligned
// 16-byte run of its plane's row and takes the column shifted by -1 / +1 from
// the neighbouring lanes' runs (zero past the row ends).
__global__ void __launch_bounds__(256)
k_last_gather(int n, int nimg, const float* __restrict__ g, float* __restrict__ hout,
              float bias0, float bscale, const double* __restrict__ snorm,
              const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  // ||b|| as fp32, formed once per block (fp64 conversions run at 1/64 of
  // the fp32 rate); zero tested on the fp64 bits
  __shared__ float s_sh;
  const long long sbits = __double_as_longlong(snorm[b]);
  if (threadIdx.x == 0) s_sh = (float)__longlong_as_double(sbits);
  __syncthreads();
  const float sf = s_sh;
  const bool nz = (sbits << 1) != 0;
  const size_t plane = (size_t)n * n, gstride = (size_t)nimg * plane;
  const int quads = (int)(plane / 4);
  // every lane of a warp takes part in the shuffles: the loop runs to a
  // multiple of the warp size
  const int span = (quads + 31) / 32 * 32;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q - (int)(threadIdx.x & 31) < span;
       q += gridDim.x * blockDim.x) {
    const bool live = q < quads;
    const int lane = threadIdx.x & 31;
    const int p = 4 * (live ? q : 0);
    const int y = p / n, x = p % n;
    float acc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = bscale * bias0;
#pragma unroll
    for (int ty = 0; ty < 3; ++ty) {
      const int yy = y + ty - 1;
      const bool rin = live && yy >= 0 && yy < n;
#pragma unroll
      for (int tx = 0; tx < 3; ++tx) {
        const float* grow = g + (ty * 3 + tx) * gstride + (size_t)b * plane + (size_t)yy * n;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (rin) v = *reinterpret_cast<const float4*>(grow + x);
        if (tx == 1) {
          acc[0] += v.x;
          acc[1] += v.y;
          acc[2] += v.z;
          acc[3] += v.w;
        } else if (tx == 0) {
          // columns x - 1 .. x + 2: x - 1 is the left lane's last value (read
          // directly by lane 0, whose left quad belongs to another warp)
          float l = __shfl_up_sync(0xffffffffu, v.w, 1);
          if (lane == 0) l = (rin && x > 0) ? grow[x - 1] : 0.f;
          else if (x == 0) l = 0.f;
          acc[0] += l;
          acc[1] += v.x;
          acc[2] += v.y;
          acc[3] += v.z;
        } else {
          // columns x + 1 .. x + 4: x + 4 is the right lane's first value
          float r = __shfl_down_sync(0xffffffffu, v.x, 1);
          if (lane == 31) r = (rin && x + 4 < n) ? grow[x + 4] : 0.f;
          else if (x + 4 >= n) r = 0.f;
          acc[0] += v.y;
          acc[1] += v.z;
          acc[2] += v.w;
          acc[3] += r;
        }
      }
    }
    if (live) {
      float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
      if (nz) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          acc[k] *= sf;
          acc[k] *= 1.f / bscale;  // a power of two: exact
        }
        o = make_float4(acc[0], acc[1], acc[2], acc[3]);
      }
      *reinterpret_cast<float4*>(hout + (size_t)b * plane + p) = o;
    }
  }
}

// host bf16 round-to-nearest-even of a finite float
uint16_t bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

// host fp16 round-to-nearest (CUDA's conversion) and its value
uint16_t f16_bits(float f) {
  const __half h = __float2half_rn(f);
  uint16_t b;
  std::memcpy(&b, &h, 2);
  return b;
}
float f16_value(uint16_t b) {
  __half h;
  std::memcpy(&h, &b, 2);
  return __half2float(h);
}

int g_num_sms = 0;
int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 148;
  }
  return g_num_sms;
}

// FIRST = 1: the first layer is computed inside the kernel from bsrc / fw
// (persistent path only; ain then only names the tensor map's buffer)
template <int SPLIT, int FUSE, int FIRST = 0>
void launch_hidden(int n, int nimg, int map_imgs, const __nv_bfloat16* ain, __nv_bfloat16* aout,
                   float* gout, const LayerPack& lp, const float* w4, const OutW& ow,
                   const double* s, const int* active, int* err, const long long* ctl,
                   cudaStream_t st, LaunchLog& log, const float* bsrc = nullptr,
                   const FirstW* fw = nullptr) {
  constexpr int CWs = TERMS<SPLIT>::value * WIDTH;
  const CUtensorMap* map = n >= 32 ? act_map(ain, n, map_imgs, CWs) : nullptr;
  if (map) {
    // three operand stages (two for the three-term form, whose stages are
    // 1.5x larger)
    constexpr int STAGES = SPLIT == 3 ? 2 : 3;
    constexpr int ACHs = ACHS<SPLIT>::value;
    constexpr int B_BYTESs = TERMS<SPLIT>::value * B_HALF;
    const size_t sm = (size_t)STAGES * ACHs * CH_PITCH + B_BYTESs + 1024;
    const int tiles_x = (n + TILE - 1) / TILE;
    long long total = (long long)nimg * tiles_x * tiles_x;
    long long grid = (long long)num_sms() * (SPLIT ? 1 : 2);
    if (grid > total) grid = total;
    if (grid < 1) grid = 1;
    cudaFuncSetAttribute(k_hidden_ws<SPLIT, STAGES, FUSE, FIRST>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int pi_ = log.begin(K_CNN_HIDDEN, st);
    k_hidden_ws<SPLIT, STAGES, FUSE, FIRST><<<(int)grid, WST<SPLIT, FUSE, FIRST>::value, sm, st>>>(
        *map, n, map_imgs, aout, gout, lp, w4, ow, s, active, err, bsrc, fw ? *fw : FirstW{}, ctl);
    log.end(pi_, st, (double)n * n * log.active_hint);
    return;
  }
  if (FIRST) return;  // not reached: run_layers takes FIRST only where a map exists
  constexpr int ACH = ACHS<SPLIT>::value;
  constexpr int B_BYTES = TERMS<SPLIT>::value * B_HALF;
  const int tiles_x = (n + TILE - 1) / TILE;
  long long total = (long long)nimg * tiles_x * tiles_x;
  long long grid = (long long)num_sms() * (SPLIT ? 1 : 3);
  // few tiles (the 16 x 16 level): one tile per CTA with a single operand
  // buffer, two CTAs per SM
  const int nbuf = total <= 2LL * num_sms() ? 1 : 2;
  if (nbuf == 1) grid = total;
  const size_t sm = (size_t)nbuf * ACH * CH_BYTES + B_BYTES;
  if (grid > total) grid = total;
  if (grid < 1) grid = 1;
  cudaFuncSetAttribute(k_hidden_tc<SPLIT, FUSE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int pi_ = log.begin(K_CNN_HIDDEN, st);
  k_hidden_tc<SPLIT, FUSE><<<(int)grid, THREADS, sm, st>>>(n, nimg, ain, aout, gout, lp, w4, ow, s, active,
                                                           err, nbuf, ctl);
  log.end(pi_, st, (double)n * n * log.active_hint);
}

template <int SPLIT>
void run_layers(int n, int B, int map_imgs, int layers, const Bf16Pack& P, const float* b, const double* s,
                __nv_bfloat16* a0, __nv_bfloat16* a1, float* h, const int* active, int* err,
                const long long* ctl, cudaStream_t st, LaunchLog& log) {
  const int tiles_x = (n + TILE - 1) / TILE;
  dim3 grid(tiles_x * tiles_x, B);
  const double units = (double)n * n * log.active_hint;
  constexpr int CWs = TERMS<SPLIT>::value * WIDTH;
  // split forms with a first hidden layer that is not the last one, on the
  // persistent path: the first layer runs inside that layer's kernel
  const bool fused_first = SPLIT && layers >= 4 && n >= 32 && act_map(a0, n, map_imgs, CWs);
  __nv_bfloat16* cur = a0;
  __nv_bfloat16* nxt = a1;
  int li0 = 1;
  if (fused_first) {
    launch_hidden<SPLIT, 0, SPLIT ? 1 : 0>(n, B, map_imgs, cur, nxt, nullptr, P.l[1], nullptr, P.last,
                                          s, active, err, ctl, st, log, b, &P.first);
    cur = a1;
    nxt = a0;
    li0 = 2;
  } else {
    int pi_ = log.begin(K_CNN_FIRST, st);
    k_first_simt<SPLIT><<<grid, 256, 0, st>>>(n, b, a0, P.first, s, active, tiles_x);
    log.end(pi_, st, units);
  }
  // hidden layers; the last one also applies the 32 -> 1 output layer's
  // weights in its epilogue and writes 9 per-tap partial-sum planes
  const LayerPack& L4 = P.l[layers - 1];
  for (int li = li0; li < layers - 1; ++li) {
    if (li < layers - 2) {
      launch_hidden<SPLIT, 0>(n, B, map_imgs, cur, nxt, nullptr, P.l[li], nullptr, P.last, s, active, err,
                              ctl, st, log);
      __nv_bfloat16* t = cur;
      cur = nxt;
      nxt = t;
    } else {
      launch_hidden<SPLIT, 1>(n, B, map_imgs, cur, nxt, reinterpret_cast<float*>(nxt), P.l[li],
                              L4.wf, P.last, s, active, err, ctl, st, log);
    }
  }
  float bias0 = 0.f;
  if (L4.bias_host_valid) bias0 = L4.bias0;
  int pi_ = log.begin(K_CNN_LAST, st);
  k_last_gather<<<dim3(ceil_div(n * n / 4, 256) < 64 ? ceil_div(n * n / 4, 256) : 64, B), 256, 0, st>>>(
      n, map_imgs, reinterpret_cast<const float*>(nxt), h, bias0, net_scale<SPLIT>(n), s, active);
  log.end(pi_, st, units);
}

std::vector<std::pair<const void*, Bf16Pack>> g_headers;

}  // namespace

// Build the device weight pack of one smoother level from PyTorch-layout
// fp64 weights (width 32, 3x3, at least 3 layers).  split = 1: the bf16
// pair form; 2: the fp16 pair form; 3: the three-term bf16 form; 0: plain
// bf16.  Returns one device allocation holding packed
// weights and biases; the per-layer device pointers are kept in a host
// table keyed by it.
void* bf16_cnn_pack(int layers, const std::vector<const double*>& W,
                    const std::vector<const double*>& bias, int split) {
  if (layers < 3 || layers > kMaxCnnLayers) return nullptr;
  std::vector<std::vector<unsigned char>> wl(layers), bl(layers);
  std::vector<int> has_lo(layers, 0);
  FirstW first{};
  OutW last{};
  for (int li = 0; li < layers; ++li) {
    const int cin = li == 0 ? 1 : WIDTH, cout = li == layers - 1 ? 1 : WIDTH;
    const double* w = W[li];
    std::vector<float> bb(WIDTH, 0.f);
    for (int co = 0; co < cout; ++co) bb[co] = (float)bias[li][co];
    bl[li].resize(WIDTH * sizeof(float));
    std::memcpy(bl[li].data(), bb.data(), WIDTH * sizeof(float));
    if (li == 0 || li == layers - 1) {
      // fp32 [c][tap]: first layer c = cout, last layer c = cin
      std::vector<float> f(WIDTH * 9, 0.f);
      for (int c = 0; c < WIDTH; ++c)
        for (int t = 0; t < 9; ++t) f[c * 9 + t] = (float)w[c * 9 + t];
      if (li == layers - 1)
        for (int t = 0; t < 9; ++t)
          for (int p2 = 0; p2 < WIDTH / 2; ++p2)
            last.w[t][p2] = make_float2(f[(2 * p2) * 9 + t], f[(2 * p2 + 1) * 9 + t]);
      if (li == 0) {
        std::memcpy(first.w, f.data(), sizeof(first.w));
        std::memcpy(first.b, bb.data(), sizeof(first.b));
        for (int t = 0; t < 9; ++t)
          for (int p2 = 0; p2 < WIDTH / 2; ++p2)
            first.w2[t][p2] = make_float2(f[(2 * p2) * 9 + t], f[(2 * p2 + 1) * 9 + t]);
      }
      wl[li].assign(reinterpret_cast<const unsigned char*>(f.data()),
                    reinterpret_cast<const unsigned char*>(f.data() + f.size()));
      continue;
    }
    const int N = (split == 3 ? 3 : (split ? 2 : 1)) * WIDTH;
    std::vector<uint16_t> p((size_t)9 * 4 * N * 8, 0);
    for (int co = 0; co < cout; ++co)
      for (int ci = 0; ci < cin; ++ci)
        for (int tap = 0; tap < 9; ++tap) {
          const double v = w[((size_t)co * cin + ci) * 9 + tap];
          uint16_t hb;
          float hf;
          if (split == 2) {
            hb = f16_bits((float)v);
            hf = f16_value(hb);
          } else {
            hb = bf16_bits((float)v);
            uint32_t u = (uint32_t)hb << 16;
            std::memcpy(&hf, &u, 4);
          }
          const size_t row = ((size_t)tap * 4 + ci / 8) * N;
          p[(row + co) * 8 + ci % 8] = hb;
          if (split == 3) {
            // w = w1 + w2 + w3, each the bf16 rounding of the remainder
            // (the remainders formed in fp64)
            const double r1 = v - (double)hf;
            const uint16_t b2 = bf16_bits((float)r1);
            float f2;
            {
              const uint32_t u2 = (uint32_t)b2 << 16;
              std::memcpy(&f2, &u2, 4);
            }
            const uint16_t b3 = bf16_bits((float)(r1 - (double)f2));
            p[(row + WIDTH + co) * 8 + ci % 8] = b2;
            p[(row + 2 * WIDTH + co) * 8 + ci % 8] = b3;
            if ((b2 != 0 && b2 != 0x8000) || (b3 != 0 && b3 != 0x8000)) has_lo[li] = 1;
          } else if (split) {
            const float rest = (float)(v - (double)hf);
            const uint16_t lb = split == 2 ? f16_bits(rest) : bf16_bits(rest);
            p[(row + WIDTH + co) * 8 + ci % 8] = lb;
            if (lb != 0 && lb != 0x8000) has_lo[li] = 1;
          }
        }
    wl[li].resize(p.size() * 2);
    std::memcpy(wl[li].data(), p.data(), wl[li].size());
  }
  size_t bytes = 0;
  std::vector<size_t> woff(layers), boff(layers);
  for (int li = 0; li < layers; ++li) {
    woff[li] = bytes;
    bytes += (wl[li].size() + 255) / 256 * 256;
    boff[li] = bytes;
    bytes += 256;
  }
  unsigned char* dptr = nullptr;
  if (cudaMalloc(&dptr, bytes) != cudaSuccess) return nullptr;
  std::vector<unsigned char> host(bytes, 0);
  Bf16Pack hdr{};
  hdr.layers = layers;
  hdr.split = split;
  hdr.first = first;
  hdr.last = last;
  for (int li = 0; li < layers; ++li) {
    std::memcpy(host.data() + woff[li], wl[li].data(), wl[li].size());
    std::memcpy(host.data() + boff[li], bl[li].data(), bl[li].size());
    const bool simt = li == 0 || li == layers - 1;
    hdr.l[li].w = simt ? nullptr : reinterpret_cast<const __nv_bfloat16*>(dptr + woff[li]);
    hdr.l[li].wf = simt ? reinterpret_cast<const float*>(dptr + woff[li]) : nullptr;
    hdr.l[li].bias = reinterpret_cast<const float*>(dptr + boff[li]);
    hdr.l[li].has_lo = split ? has_lo[li] : 0;
    hdr.l[li].bias0 = (float)bias[li][0];
    hdr.l[li].bias_host_valid = 1;
  }
  if (cudaMemcpy(dptr, host.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(dptr);
    return nullptr;
  }
  g_headers.emplace_back(dptr, hdr);
  return dptr;
}

void bf16_cnn_forget(const void* pack) {
  for (size_t i = 0; i < g_headers.size(); ++i)
    if (g_headers[i].first == pack) {
      g_headers.erase(g_headers.begin() + i);
      return;
    }
}

// h = s N(b / s) for `B` images of side n; act0/act1 hold chunk-planar
// 16-bit activations (B * n * n * 32 elements, x2 in the split forms),
// described to the copy engine as map_imgs >= B images so one tensor map
// serves every chunk; err: device error word of the bounded waits.
void bf16_cnn_launch(int n, int B, int map_imgs, int layers, const void* pack, const float* b,
                     const double* s, float* act0, float* act1, float* h, const int* active,
                     int* err, const long long* ctl, cudaStream_t st, LaunchLog& log) {
  const Bf16Pack* P = nullptr;
  for (auto& e : g_headers)
    if (e.first == pack) P = &e.second;
  if (!P) return;
  __nv_bfloat16* a0 = reinterpret_cast<__nv_bfloat16*>(act0);
  __nv_bfloat16* a1 = reinterpret_cast<__nv_bfloat16*>(act1);
  if (P->split == 3)
    run_layers<3>(n, B, map_imgs, layers, *P, b, s, a0, a1, h, active, err, ctl, st, log);
  else if (P->split == 2)
    run_layers<2>(n, B, map_imgs, layers, *P, b, s, a0, a1, h, active, err, ctl, st, log);
  else if (P->split)
    run_layers<1>(n, B, map_imgs, layers, *P, b, s, a0, a1, h, active, err, ctl, st, log);
  else
    run_layers<0>(n, B, map_imgs, layers, *P, b, s, a0, a1, h, active, err, ctl, st, log);
}

}  // namespace nmg
