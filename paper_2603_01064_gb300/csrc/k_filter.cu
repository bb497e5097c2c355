// Output filter of the cycle, x = x* + F'_l(h) with
// F'_l(h) = Re(IDFT(m'_l . DFT(h))) (Sections 3.2 and 3.3).
//
// 2D: in-shared-memory radix-2 Cooley-Tukey FFTs over whole rows/columns on
// the half spectrum of each real image (row pairs packed as one complex
// row, see the layout note below); the mask
// m'(k1, k2) = sqrt(max(|w1|, |w2|) / pi) is real and even in each axis, so
// the filtered image is real and is produced as such (the Re(.) of the
// definition is implied).  Levels whose n/2 x n complex layout fits in
// shared memory run one fused launch per image; larger levels run three
// passes over a [B][n/2][n] complex buffer (row pairs, column pairs, row
// pairs).
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

// ---------------------------------------------------------------------------
// Half-spectrum 2D transform of one real image.
//
// h is real and the mask is real and even in both axes, so only the n/2 + 1
// column frequencies 0..n/2 of the row spectra are needed.  Rows 2k and
// 2k+1 travel together as one complex row z_k = h[2k] + i h[2k+1]
// ("row-pair layout", n/2 rows of n complex values):
//   after the row FFT and the split below, row k holds
//     position t, 0 < t < n/2 : X_{2k}[t]      (spectrum of row 2k)
//     position n - t          : X_{2k+1}[t]    (spectrum of row 2k+1)
//     position 0              : X_{2k}[0]   + i X_{2k}[n/2]
//     position n/2            : X_{2k+1}[0] + i X_{2k+1}[n/2]
//   (the four values at 0 and n/2 are real for real rows).
// Column j (0 < j < n/2) of the full row-spectrum array is then split by
// row parity between layout columns j (even rows) and n - j (odd rows):
// the first decimation-in-time step of the length-n column FFT.  Columns 0
// and n/2 of the spectrum, both real sequences, travel together as the
// complex sequence q[r] = X_r[0] + i X_r[n/2], even rows in layout column 0
// and odd rows in layout column n/2; their different masks are applied
// after separating the two real sequences' spectra by Hermitian symmetry.
// Everything a right-hand side's result depends on is that right-hand
// side's own image: results do not depend on the batch composition.
// ---------------------------------------------------------------------------

__device__ __forceinline__ int bitrev_bits(int v, int bits) { return bits ? bitrev(v, bits) : 0; }

// Separate the FFTs of the row pairs of `nrows` layout rows (natural order)
// into the row-pair layout above.  Each (row, t) touches only positions t
// and n - t of its row: no synchronisation inside.
template <typename T>
__device__ void rows_split(Cx<T>* buf, int nrows, int n) {
  const int halfn = n >> 1;
  for (int idx = threadIdx.x; idx < nrows * halfn; idx += blockDim.x) {
    const int k = idx / halfn, t = idx % halfn;
    Cx<T>* row = buf + (size_t)k * n;
    if (t == 0) {
      const Cx<T> a = row[0], b = row[halfn];
      row[0] = Cx<T>{a.x, b.x};
      row[halfn] = Cx<T>{a.y, b.y};
    } else {
      const Cx<T> za = row[t], zb = row[n - t];
      // X_a = (Z[t] + conj Z[n-t]) / 2,  X_b = (Z[t] - conj Z[n-t]) / 2i
      row[t] = Cx<T>{T(0.5) * (za.x + zb.x), T(0.5) * (za.y - zb.y)};
      row[n - t] = Cx<T>{T(0.5) * (za.y + zb.y), T(0.5) * (zb.x - za.x)};
    }
  }
}

// Inverse of rows_split: rebuild the full spectrum of z_k = row 2k + i row
// 2k+1 from the row-pair layout, Z[t] = X_a[t] + i X_b[t] for all t, using
// X[n - t] = conj X[t].  Natural order in and out.
template <typename T>
__device__ void rows_join(Cx<T>* buf, int nrows, int n) {
  const int halfn = n >> 1;
  for (int idx = threadIdx.x; idx < nrows * halfn; idx += blockDim.x) {
    const int k = idx / halfn, t = idx % halfn;
    Cx<T>* row = buf + (size_t)k * n;
    if (t == 0) {
      const Cx<T> a = row[0], b = row[halfn];
      row[0] = Cx<T>{a.x, b.x};
      row[halfn] = Cx<T>{a.y, b.y};
    } else {
      const Cx<T> xa = row[t], xb = row[n - t];
      row[t] = Cx<T>{xa.x - xb.y, xa.y + xb.x};
      row[n - t] = Cx<T>{xa.x + xb.y, xb.x - xa.y};
    }
  }
}

// Bit-reverse the element order within each of `nrows` rows of length n.
template <typename T>
__device__ void rows_bitrev(Cx<T>* buf, int nrows, int n, int logn) {
  for (int idx = threadIdx.x; idx < nrows * n; idx += blockDim.x) {
    const int r = idx / n, c = idx % n, rc = bitrev(c, logn);
    if (c < rc) {
      Cx<T> t = buf[r * n + c];
      buf[r * n + c] = buf[r * n + rc];
      buf[r * n + rc] = t;
    }
  }
}

// Bit-reverse the row order of a [len][pitch] array (every column at once).
template <typename T>
__device__ void cols_bitrev(Cx<T>* buf, int pitch, int ncols, int len, int loglen) {
  for (int idx = threadIdx.x; idx < len * ncols; idx += blockDim.x) {
    const int k = idx / ncols, c = idx % ncols, rk = bitrev_bits(k, loglen);
    if (k < rk) {
      Cx<T> t = buf[k * pitch + c];
      buf[k * pitch + c] = buf[rk * pitch + c];
      buf[rk * pitch + c] = t;
    }
  }
}

// Radix-2 DIT FFT of length len = 2^loglen down each of ncols columns of a
// [len][pitch] array (rows in bit-reversed order in, natural order out).
// tw is the length-n table exp(-2 pi i k / n), k < n/2, with len <= n.
template <typename T>
__device__ void cols_fft(Cx<T>* buf, int pitch, int ncols, int loglen, int n, const Cx<T>* tw,
                         int sign) {
  const int len = 1 << loglen;
  for (int s = 1; s <= loglen; ++s) {
    const int half = 1 << (s - 1), tstride = n >> s;
    for (int t = threadIdx.x; t < (len >> 1) * ncols; t += blockDim.x) {
      const int c = t % ncols, k = t / ncols;
      const int grp = k / half, pos = k % half;
      const int i = (grp * 2 * half + pos) * pitch + c, j = i + half * pitch;
      Cx<T> w = tw[pos * tstride];
      if (sign < 0) w.y = -w.y;
      const Cx<T> a = buf[i], bb = buf[j];
      const Cx<T> p{w.x * bb.x - w.y * bb.y, w.x * bb.y + w.y * bb.x};
      buf[i] = Cx<T>{a.x + p.x, a.y + p.y};
      buf[j] = Cx<T>{a.x - p.x, a.y - p.y};
    }
    __syncthreads();
  }
}

// Column pairs of the row-pair layout in shared memory: pair p has its
// even-row column at slot ev(p), its odd-row column at slot od(p) and
// column frequency fr(p) (0 means the packed pair of frequencies 0 and n/2).
struct FusedPairs {  // whole image: slots are layout columns
  int n;
  __device__ int ev(int p) const { return p; }
  __device__ int od(int p) const { return p == 0 ? n / 2 : n - p; }
  __device__ int fr(int p) const { return p; }
  __device__ int special() const { return 0; }
};
struct BlockPairs {  // a block of cpc frequencies j0..j0+cpc-1
  int cpc, j0;
  __device__ int ev(int p) const { return p; }
  __device__ int od(int p) const { return cpc + p; }
  __device__ int fr(int p) const { return j0 + p; }
  __device__ int special() const { return j0 == 0 ? 0 : -1; }
};

// Given the length-n/2 column FFTs of both halves of every pair (natural
// order), finish the length-n column transform, multiply by the mask and
// undo the last step again, leaving for every pair the length-n/2 spectra
// of the even and odd rows of the masked column's inverse:
//   Y[k1] = E[k1] + w^k1 O[k1],  Y[k1 + n/2] = E[k1] - w^k1 O[k1]
//   Y *= m';  E' = Y[k1] + Y[k1 + n/2],  O' = (Y[k1] - Y[k1 + n/2]) conj(w^k1)
// Column frequency j > 0: Y is the column spectrum itself, mask
// m'(k1, j) = mtab[max(fold(k1), j)].  The packed pair (frequency 0 and n/2)
// holds Q = A + iB with A, B the spectra of two real sequences; with
// masks m_a(K) = mtab[fold(K)], m_b(K) = mtab[n/2]:
//   Q'[K] = (m_a + m_b)/2 Q[K] + (m_a - m_b)/2 conj Q[n - K].
template <typename T, typename Map>
__device__ void spectral_pairs(Cx<T>* buf, int pitch, int npairs, Map map, int n,
                               const Cx<T>* tw, const double* __restrict__ mtab) {
  const int halfn = n >> 1;
  for (int idx = threadIdx.x; idx < npairs * halfn; idx += blockDim.x) {
    const int p = idx % npairs, k1 = idx / npairs;
    const int j = map.fr(p);
    Cx<T>* pe = buf + k1 * pitch + map.ev(p);
    Cx<T>* po = buf + k1 * pitch + map.od(p);
    const Cx<T> w = tw[k1];
    const Cx<T> e = *pe, o = *po;
    const Cx<T> wo{w.x * o.x - w.y * o.y, w.x * o.y + w.y * o.x};
    Cx<T> y0{e.x + wo.x, e.y + wo.y}, y1{e.x - wo.x, e.y - wo.y};
    if (j == 0) {  // packed pair: separation needs K and n - K, done below
      *pe = y0;
      *po = y1;
      continue;
    }
    const T m0 = (T)mtab[k1 > j ? k1 : j];
    const T m1 = (T)mtab[halfn - k1 > j ? halfn - k1 : j];
    y0.x *= m0; y0.y *= m0;
    y1.x *= m1; y1.y *= m1;
    const Cx<T> d{y0.x - y1.x, y0.y - y1.y};
    *pe = Cx<T>{y0.x + y1.x, y0.y + y1.y};
    *po = Cx<T>{w.x * d.x + w.y * d.y, w.x * d.y - w.y * d.x};
  }
  const int sp = map.special();
  if (sp < 0) return;  // uniform across the block: no barrier skipped unevenly
  __syncthreads();
  Cx<T>* ce = buf + map.ev(sp);
  Cx<T>* co = buf + map.od(sp);
  // Q[K] sits at row K of ce for K < n/2, at row K - n/2 of co otherwise
  auto at = [&](int K) -> Cx<T>* { return K < halfn ? ce + K * pitch : co + (K - halfn) * pitch; };
  const T mb = (T)mtab[halfn];
  for (int K = threadIdx.x; K <= halfn; K += blockDim.x) {
    const int Kp = K == 0 ? 0 : n - K;
    const T ma = (T)mtab[K];
    const T c1 = T(0.5) * (ma + mb), c2 = T(0.5) * (ma - mb);
    Cx<T>* a = at(K);
    Cx<T>* b = at(Kp);
    const Cx<T> qa = *a, qb = *b;
    *a = Cx<T>{c1 * qa.x + c2 * qb.x, c1 * qa.y - c2 * qb.y};
    if (Kp != K) *b = Cx<T>{c1 * qb.x + c2 * qa.x, c1 * qb.y - c2 * qa.y};
  }
  __syncthreads();
  for (int k1 = threadIdx.x; k1 < halfn; k1 += blockDim.x) {
    const Cx<T> w = tw[k1];
    const Cx<T> y0 = ce[k1 * pitch], y1 = co[k1 * pitch];
    const Cx<T> d{y0.x - y1.x, y0.y - y1.y};
    ce[k1 * pitch] = Cx<T>{y0.x + y1.x, y0.y + y1.y};
    co[k1 * pitch] = Cx<T>{w.x * d.x + w.y * d.y, w.x * d.y - w.y * d.x};
  }
}

// pass 1: row pairs of real h -> row-pair layout spectra in C ([B][n/2][n])
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
  const int k0 = blockIdx.x * rpc;  // first layout row (row pair)
  const size_t plane = (size_t)n * n;
  const T* hb = h + (size_t)b * plane;
  for (int t = threadIdx.x; t < rpc * n; t += blockDim.x) {
    const int r = t / n, j = t % n;
    const size_t g = (size_t)(2 * (k0 + r)) * n + j;
    buf[r * n + bitrev(j, logn)] = Cx<T>{hb[g], hb[g + n]};
  }
  __syncthreads();
  fft_stages(buf, n, logn, rpc, tw, +1);
  rows_split(buf, rpc, n);
  __syncthreads();
  Cx<T>* Cb = C + (size_t)b * (plane / 2);
  for (int t = threadIdx.x; t < rpc * n; t += blockDim.x) Cb[(size_t)k0 * n + t] = buf[t];
}

// pass 2: column transforms, mask, inverse column transforms for cpc column
// frequencies j0..j0+cpc-1 (in place on C)
template <typename T>
__global__ void k_fft_cols_mask(int n, int logn, int cpc, Cx<T>* __restrict__ C,
                                const Cx<T>* __restrict__ twg, const double* __restrict__ mtab,
                                const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<T>* tw = reinterpret_cast<Cx<T>*>(smem_raw);
  Cx<T>* buf = tw + n / 2;  // [n/2][2 cpc]: even-row columns, then odd-row columns
  const int halfn = n / 2, pitch = 2 * cpc;
  for (int k = threadIdx.x; k < halfn; k += blockDim.x) tw[k] = twg[k];
  const BlockPairs map{cpc, (int)blockIdx.x * cpc};
  Cx<T>* Cb = C + (size_t)b * ((size_t)n * n / 2);
  // layout column of slot s: even slots j0 + s, odd slots their partners
  auto gcol = [&](int s) {
    const int j = map.j0 + (s < cpc ? s : s - cpc);
    return s < cpc ? j : (j == 0 ? halfn : n - j);
  };
  for (int t = threadIdx.x; t < halfn * pitch; t += blockDim.x) {
    const int k = t / pitch, s = t % pitch;
    buf[bitrev_bits(k, logn - 1) * pitch + s] = Cb[(size_t)k * n + gcol(s)];
  }
  __syncthreads();
  cols_fft(buf, pitch, pitch, logn - 1, n, tw, +1);
  spectral_pairs(buf, pitch, cpc, map, n, tw, mtab);
  __syncthreads();
  cols_bitrev(buf, pitch, pitch, halfn, logn - 1);
  __syncthreads();
  cols_fft(buf, pitch, pitch, logn - 1, n, tw, -1);
  for (int t = threadIdx.x; t < halfn * pitch; t += blockDim.x) {
    const int k = t / pitch, s = t % pitch;
    Cb[(size_t)k * n + gcol(s)] = buf[t];
  }
}

// pass 3: rebuild the row-pair spectra, inverse row FFT, x = x* + z / n^2
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
  const int k0 = blockIdx.x * rpc;
  const size_t plane = (size_t)n * n;
  const Cx<T>* Cb = C + (size_t)b * (plane / 2);
  for (int t = threadIdx.x; t < rpc * n; t += blockDim.x) buf[t] = Cb[(size_t)k0 * n + t];
  __syncthreads();
  rows_join(buf, rpc, n);
  __syncthreads();
  rows_bitrev(buf, rpc, n, logn);
  __syncthreads();
  fft_stages(buf, n, logn, rpc, tw, -1);
  const T scale = T(1.0 / ((double)n * (double)n));
  for (int t = threadIdx.x; t < rpc * n; t += blockDim.x) {
    const int r = t / n, j = t % n;
    const size_t g = (size_t)b * plane + (size_t)(2 * (k0 + r)) * n + j;
    const T b0 = xstar ? xstar[g] : T(0), b1 = xstar ? xstar[g + n] : T(0);
    x[g] = b0 + buf[t].x * scale;
    x[g + n] = b1 + buf[t].y * scale;
  }
}

// Whole filter of one right-hand side in shared memory (levels whose
// row-pair layout, n/2 x n complex values, fits): row transforms, column
// transforms, mask, inverse column and row transforms and the update in one
// launch; h read once and x written once.
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
  const int halfn = n / 2, nh = n * halfn;
  for (int k = threadIdx.x; k < halfn; k += blockDim.x) tw[k] = twg[k];
  const size_t base = (size_t)b * n * n;
  for (int idx = threadIdx.x; idx < nh; idx += blockDim.x) {
    const int k = idx / n, c = idx % n;
    const size_t g = base + (size_t)(2 * k) * n + c;
    buf[k * n + bitrev(c, logn)] = Cx<T>{h[g], h[g + n]};
  }
  __syncthreads();
  fft_stages(buf, n, logn, halfn, tw, +1);
  rows_split(buf, halfn, n);
  __syncthreads();
  cols_bitrev(buf, n, n, halfn, logn - 1);
  __syncthreads();
  cols_fft(buf, n, n, logn - 1, n, tw, +1);
  spectral_pairs(buf, n, halfn, FusedPairs{n}, n, tw, mtab);
  __syncthreads();
  cols_bitrev(buf, n, n, halfn, logn - 1);
  __syncthreads();
  cols_fft(buf, n, n, logn - 1, n, tw, -1);
  rows_join(buf, halfn, n);
  __syncthreads();
  rows_bitrev(buf, halfn, n, logn);
  __syncthreads();
  fft_stages(buf, n, logn, halfn, tw, -1);
  const T scale = T(1.0 / ((double)n * (double)n));
  for (int idx = threadIdx.x; idx < nh; idx += blockDim.x) {
    const int k = idx / n, c = idx % n;
    const size_t g = base + (size_t)(2 * k) * n + c;
    const T b0 = xstar ? xstar[g] : T(0), b1 = xstar ? xstar[g + n] : T(0);
    x[g] = b0 + buf[idx].x * scale;
    x[g + n] = b1 + buf[idx].y * scale;
  }
}

// ---------------------------------------------------------------------------
// Warp-level form of the fused filter for n = 64 and 128: the same
// half-spectrum layout, but every row and column transform is done by one
// warp in registers (M = length / 32 values per lane, radix-2 stages within
// a lane's registers for spans >= 32 and across lanes with shuffles below),
// so the block synchronises only between the row, column and row phases.
// Forward transforms are decimation in frequency (natural order in, bit-
// reversed out) and inverse ones decimation in time (bit-reversed in,
// natural out), so the column spectra are masked in bit-reversed order and
// no permutation pass is needed.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
  return Cx<T>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ Cx<T> cmulc(Cx<T> a, Cx<T> b) {  // a * conj(b)
  return Cx<T>{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename T>
__device__ __forceinline__ Cx<T> shfl_cx(Cx<T> v, int mask) {
  return Cx<T>{__shfl_xor_sync(0xffffffffu, v.x, mask), __shfl_xor_sync(0xffffffffu, v.y, mask)};
}

// length-L DIF FFT (L = 32 M), natural order in, slot s = lane + 32 m holds
// the spectrum at bitrev_L(s) on return; tw: exp(-2 pi i k / N), k < N / 2
template <typename T, int L, int N>
__device__ __forceinline__ void warp_dif(Cx<T> (&v)[L / 32], const Cx<T>* tw, int lane) {
  constexpr int M = L / 32;
#pragma unroll
  for (int span = L / 2; span >= 32; span >>= 1) {
    const int ms = span / 32;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      if (m & ms) continue;
      const int j = lane + 32 * (m & (2 * ms - 1));  // position in the sub-transform
      const Cx<T> a = v[m], b = v[m + ms];
      v[m] = Cx<T>{a.x + b.x, a.y + b.y};
      v[m + ms] = cmul(Cx<T>{a.x - b.x, a.y - b.y}, tw[j * (N / (2 * span))]);
    }
  }
#pragma unroll
  for (int span = (L / 2 < 16 ? L / 2 : 16); span >= 1; span >>= 1) {
    const bool upper = lane & span;
    const Cx<T> w = tw[((lane & (2 * span - 1)) - (upper ? span : 0)) * (N / (2 * span))];
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const Cx<T> o = shfl_cx(v[m], span);
      v[m] = upper ? cmul(Cx<T>{o.x - v[m].x, o.y - v[m].y}, w) : Cx<T>{v[m].x + o.x, v[m].y + o.y};
    }
  }
}

// length-L inverse DIT FFT (unnormalised), slot s holds the input at
// bitrev_L(s), natural order out
template <typename T, int L, int N>
__device__ __forceinline__ void warp_dit_inv(Cx<T> (&v)[L / 32], const Cx<T>* tw, int lane) {
  constexpr int M = L / 32;
#pragma unroll
  for (int span = 1; span <= (L / 2 < 16 ? L / 2 : 16); span <<= 1) {
    const bool upper = lane & span;
    const Cx<T> w = tw[((lane & (2 * span - 1)) - (upper ? span : 0)) * (N / (2 * span))];
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const Cx<T> o = shfl_cx(v[m], span);
      // lower: a + b w with a = mine, b = partner; upper: a - b w, a = partner
      v[m] = upper ? Cx<T>{o.x - cmulc(v[m], w).x, o.y - cmulc(v[m], w).y}
                   : Cx<T>{v[m].x + cmulc(o, w).x, v[m].y + cmulc(o, w).y};
    }
  }
#pragma unroll
  for (int span = 32; span <= L / 2; span <<= 1) {
    const int ms = span / 32;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      if (m & ms) continue;
      const int j = lane + 32 * (m & (2 * ms - 1));
      const Cx<T> a = v[m], t = cmulc(v[m + ms], tw[j * (N / (2 * span))]);
      v[m] = Cx<T>{a.x + t.x, a.y + t.y};
      v[m + ms] = Cx<T>{a.x - t.x, a.y - t.y};
    }
  }
}

template <int L>
__device__ __forceinline__ int brev_len(int s) {
  constexpr int bits = L == 32 ? 5 : L == 64 ? 6 : L == 128 ? 7 : L == 256 ? 8 : 9;
  static_assert(L == (1 << bits), "transform length: a power of two from 32 to 512");
  return __brev(s) >> (32 - bits);
}

// threads of the warp-level filter: one warp per row / column pair at a
// time; 16 warps for 128 x 128 (a block holds one image, so more warps
// shorten the per-image chain of row and column passes)
template <int N> struct FWThreads { static constexpr int value = N == 128 ? 512 : 256; };

template <typename T, int N>
__global__ void __launch_bounds__(FWThreads<N>::value)
k_filter_warp(const T* xstar, const T* __restrict__ h, T* x, const Cx<T>* __restrict__ twg,
              const double* __restrict__ mtab, const int* __restrict__ active) {
  constexpr int HN = N / 2, MR = N / 32, MC = HN / 32, P = N + 1;  // odd pitch
  const int b = blockIdx.x;
  if (!active[b]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<T>* tw = reinterpret_cast<Cx<T>*>(smem_raw);
  Cx<T>* q = tw + HN;     // scratch of the packed column pair (N values)
  T* mt = reinterpret_cast<T*>(q + N);  // mask table, HN + 1 values
  Cx<T>* buf = reinterpret_cast<Cx<T>*>(mt + ((HN + 1 + 1) & ~1));  // [HN][P]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = threadIdx.x; k < HN; k += blockDim.x) tw[k] = twg[k];
  for (int k = threadIdx.x; k <= HN; k += blockDim.x) mt[k] = (T)mtab[k];
  __syncthreads();
  const size_t base = (size_t)b * N * N;
  // ---- rows: z_k = h[2k] + i h[2k+1], FFT, split into the row-pair layout
  for (int k = warp; k < HN; k += nw) {
    Cx<T> v[MR];
    const T* h0 = h + base + (size_t)(2 * k) * N;
#pragma unroll
    for (int m = 0; m < MR; ++m) v[m] = Cx<T>{h0[lane + 32 * m], h0[N + lane + 32 * m]};
    warp_dif<T, N, N>(v, tw, lane);
    Cx<T>* row = buf + k * P;
#pragma unroll
    for (int m = 0; m < MR; ++m) row[brev_len<N>(lane + 32 * m)] = v[m];
    __syncwarp();
    for (int t = lane; t < HN; t += 32) {
      if (t == 0) {
        const Cx<T> a = row[0], c = row[HN];
        row[0] = Cx<T>{a.x, c.x};
        row[HN] = Cx<T>{a.y, c.y};
      } else {
        const Cx<T> za = row[t], zb = row[N - t];
        row[t] = Cx<T>{T(0.5) * (za.x + zb.x), T(0.5) * (za.y - zb.y)};
        row[N - t] = Cx<T>{T(0.5) * (za.y + zb.y), T(0.5) * (zb.x - za.x)};
      }
    }
    __syncwarp();
  }
  __syncthreads();
  // ---- column pairs: even rows in column p, odd rows in its partner
  for (int p = warp; p < HN; p += nw) {
    const int ce = p, co = p == 0 ? HN : N - p;
    Cx<T> e[MC], o[MC];
#pragma unroll
    for (int m = 0; m < MC; ++m) {
      e[m] = buf[(lane + 32 * m) * P + ce];
      o[m] = buf[(lane + 32 * m) * P + co];
    }
    warp_dif<T, HN, N>(e, tw, lane);
    warp_dif<T, HN, N>(o, tw, lane);
#pragma unroll
    for (int m = 0; m < MC; ++m) {
      const int k1 = brev_len<HN>(lane + 32 * m);
      const Cx<T> w = tw[k1], wo = cmul(o[m], w);
      Cx<T> y0{e[m].x + wo.x, e[m].y + wo.y}, y1{e[m].x - wo.x, e[m].y - wo.y};
      if (p == 0) {  // packed pair: separated below
        q[k1] = y0;
        q[k1 + HN] = y1;
        continue;
      }
      const T m0 = mt[k1 > p ? k1 : p], m1 = mt[HN - k1 > p ? HN - k1 : p];
      y0.x *= m0; y0.y *= m0;
      y1.x *= m1; y1.y *= m1;
      e[m] = Cx<T>{y0.x + y1.x, y0.y + y1.y};
      o[m] = cmulc(Cx<T>{y0.x - y1.x, y0.y - y1.y}, w);
    }
    if (p == 0) {
      __syncwarp();
      const T mb = mt[HN];
      for (int K = lane; K <= HN; K += 32) {
        const int Kp = K == 0 ? 0 : N - K;
        const T ma = mt[K], c1 = T(0.5) * (ma + mb), c2 = T(0.5) * (ma - mb);
        const Cx<T> qa = q[K], qb = q[Kp];
        q[K] = Cx<T>{c1 * qa.x + c2 * qb.x, c1 * qa.y - c2 * qb.y};
        if (Kp != K) q[Kp] = Cx<T>{c1 * qb.x + c2 * qa.x, c1 * qb.y - c2 * qa.y};
      }
      __syncwarp();
#pragma unroll
      for (int m = 0; m < MC; ++m) {
        const int k1 = brev_len<HN>(lane + 32 * m);
        const Cx<T> y0 = q[k1], y1 = q[k1 + HN];
        e[m] = Cx<T>{y0.x + y1.x, y0.y + y1.y};
        o[m] = cmulc(Cx<T>{y0.x - y1.x, y0.y - y1.y}, tw[k1]);
      }
    }
    warp_dit_inv<T, HN, N>(e, tw, lane);
    warp_dit_inv<T, HN, N>(o, tw, lane);
#pragma unroll
    for (int m = 0; m < MC; ++m) {
      buf[(lane + 32 * m) * P + ce] = e[m];
      buf[(lane + 32 * m) * P + co] = o[m];
    }
  }
  __syncthreads();
  // ---- rows: rebuild z_k's spectrum, inverse FFT, x = x* + z / N^2
  const T scale = T(1.0 / ((double)N * (double)N));
  for (int k = warp; k < HN; k += nw) {
    Cx<T>* row = buf + k * P;
    for (int t = lane; t < HN; t += 32) {
      if (t == 0) {
        const Cx<T> a = row[0], c = row[HN];
        row[0] = Cx<T>{a.x, c.x};
        row[HN] = Cx<T>{a.y, c.y};
      } else {
        const Cx<T> xa = row[t], xb = row[N - t];
        row[t] = Cx<T>{xa.x - xb.y, xa.y + xb.x};
        row[N - t] = Cx<T>{xa.x + xb.y, xb.x - xa.y};
      }
    }
    __syncwarp();
    Cx<T> v[MR];
#pragma unroll
    for (int m = 0; m < MR; ++m) v[m] = row[brev_len<N>(lane + 32 * m)];
    warp_dit_inv<T, N, N>(v, tw, lane);
    const size_t g0 = base + (size_t)(2 * k) * N;
#pragma unroll
    for (int m = 0; m < MR; ++m) {
      const size_t g = g0 + lane + 32 * m;
      x[g] = (xstar ? xstar[g] : T(0)) + v[m].x * scale;
      x[g + N] = (xstar ? xstar[g + N] : T(0)) + v[m].y * scale;
    }
    __syncwarp();
  }
}

template <typename T, int N>
size_t filter_warp_smem() {
  return (size_t)(N / 2 + N) * sizeof(Cx<T>) + (size_t)((N / 2 + 2) & ~1) * sizeof(T) +
         (size_t)(N / 2) * (N + 1) * sizeof(Cx<T>);
}

// ---------------------------------------------------------------------------
// Warp-level form for levels too large for one block (n = 256, 512): the
// same half-spectrum transforms as k_filter_warp, in three launches over the
// row-pair layout buffer C ([B][n/2][n] complex, global memory, mostly
// L2-resident between the passes):
//   rows: one warp per row pair, h in, forward row FFT in registers, split,
//         coalesced row write;
//   cols: one block per kFcCols column pairs (even-row columns p and their
//         odd-row partners), staged through shared memory so that every
//         global access is a contiguous run; one warp per column pair does
//         the forward column FFTs, the mask and the inverse FFTs;
//   rows: one warp per row pair, join, inverse row FFT, x = x* + z / n^2.
// ---------------------------------------------------------------------------
constexpr int kFrWarps = 8;  // row pairs per block (row passes)
constexpr int kFcCols = 8;   // column pairs per block (column pass), one warp each

template <typename T, int N>
__global__ void __launch_bounds__(32 * kFrWarps)
k_fwarp_rows_fwd(const T* __restrict__ h, Cx<T>* __restrict__ C, const Cx<T>* __restrict__ twg,
                 const int* __restrict__ active) {
  constexpr int HN = N / 2, MR = N / 32;
  const int b = blockIdx.y;
  if (!active[b]) return;
  extern __shared__ __align__(16) unsigned char fr_smem[];
  Cx<T>* tw = reinterpret_cast<Cx<T>*>(fr_smem);  // [HN], then one row per warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < HN; k += blockDim.x) tw[k] = twg[k];
  __syncthreads();
  const int k = blockIdx.x * kFrWarps + warp;  // row pair (HN is a multiple of kFrWarps)
  const size_t plane = (size_t)N * N;
  const T* h0 = h + (size_t)b * plane + (size_t)(2 * k) * N;
  Cx<T> v[MR];
#pragma unroll
  for (int m = 0; m < MR; ++m) v[m] = Cx<T>{h0[lane + 32 * m], h0[N + lane + 32 * m]};
  warp_dif<T, N, N>(v, tw, lane);
  Cx<T>* row = tw + HN + warp * N;
#pragma unroll
  for (int m = 0; m < MR; ++m) row[brev_len<N>(lane + 32 * m)] = v[m];
  __syncwarp();
  Cx<T>* Cr = C + (size_t)b * (plane / 2) + (size_t)k * N;
  for (int t = lane; t < HN; t += 32) {
    if (t == 0) {
      const Cx<T> a = row[0], c = row[HN];
      Cr[0] = Cx<T>{a.x, c.x};
      Cr[HN] = Cx<T>{a.y, c.y};
    } else {
      const Cx<T> za = row[t], zb = row[N - t];
      Cr[t] = Cx<T>{T(0.5) * (za.x + zb.x), T(0.5) * (za.y - zb.y)};
      Cr[N - t] = Cx<T>{T(0.5) * (za.y + zb.y), T(0.5) * (zb.x - za.x)};
    }
  }
}

template <typename T, int N>
__global__ void __launch_bounds__(32 * kFcCols)
k_fwarp_cols(Cx<T>* __restrict__ C, const Cx<T>* __restrict__ twg,
             const double* __restrict__ mtab, const int* __restrict__ active) {
  constexpr int HN = N / 2, MC = HN / 32, PT = kFcCols + 1;  // odd tile pitch
  const int b = blockIdx.y;
  if (!active[b]) return;
  extern __shared__ __align__(16) unsigned char fc_smem[];
  Cx<T>* tw = reinterpret_cast<Cx<T>*>(fc_smem);
  Cx<T>* q = tw + HN;                                  // packed pair scratch (N)
  Cx<T>* E = q + N;                                    // [HN][PT]: even-row columns
  Cx<T>* O = E + HN * PT;                              // [HN][PT]: odd-row partners
  T* mt = reinterpret_cast<T*>(O + HN * PT);           // mask table, HN + 1
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < HN; k += blockDim.x) tw[k] = twg[k];
  for (int k = threadIdx.x; k <= HN; k += blockDim.x) mt[k] = (T)mtab[k];
  const int p0 = blockIdx.x * kFcCols;
  Cx<T>* Cb = C + (size_t)b * ((size_t)N * N / 2);
  // stage: column p0 + s (even rows) and its partner (odd rows) of every row
  for (int t = threadIdx.x; t < HN * kFcCols; t += blockDim.x) {
    const int k = t / kFcCols, s2 = t % kFcCols;
    const int p = p0 + s2;
    const int co = p == 0 ? HN : N - p;
    E[k * PT + s2] = Cb[(size_t)k * N + p];
    O[k * PT + s2] = Cb[(size_t)k * N + co];
  }
  __syncthreads();
  const int p = p0 + warp;
  Cx<T> e[MC], o[MC];
#pragma unroll
  for (int m = 0; m < MC; ++m) {
    e[m] = E[(lane + 32 * m) * PT + warp];
    o[m] = O[(lane + 32 * m) * PT + warp];
  }
  warp_dif<T, HN, N>(e, tw, lane);
  warp_dif<T, HN, N>(o, tw, lane);
#pragma unroll
  for (int m = 0; m < MC; ++m) {
    const int k1 = brev_len<HN>(lane + 32 * m);
    const Cx<T> w = tw[k1], wo = cmul(o[m], w);
    Cx<T> y0{e[m].x + wo.x, e[m].y + wo.y}, y1{e[m].x - wo.x, e[m].y - wo.y};
    if (p == 0) {  // packed pair: separated below
      q[k1] = y0;
      q[k1 + HN] = y1;
      continue;
    }
    const T m0 = mt[k1 > p ? k1 : p], m1 = mt[HN - k1 > p ? HN - k1 : p];
    y0.x *= m0; y0.y *= m0;
    y1.x *= m1; y1.y *= m1;
    e[m] = Cx<T>{y0.x + y1.x, y0.y + y1.y};
    o[m] = cmulc(Cx<T>{y0.x - y1.x, y0.y - y1.y}, w);
  }
  if (p == 0) {  // warp-uniform
    __syncwarp();
    const T mb = mt[HN];
    for (int K = lane; K <= HN; K += 32) {
      const int Kp = K == 0 ? 0 : N - K;
      const T ma = mt[K], c1 = T(0.5) * (ma + mb), c2 = T(0.5) * (ma - mb);
      const Cx<T> qa = q[K], qb = q[Kp];
      q[K] = Cx<T>{c1 * qa.x + c2 * qb.x, c1 * qa.y - c2 * qb.y};
      if (Kp != K) q[Kp] = Cx<T>{c1 * qb.x + c2 * qa.x, c1 * qb.y - c2 * qa.y};
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < MC; ++m) {
      const int k1 = brev_len<HN>(lane + 32 * m);
      const Cx<T> y0 = q[k1], y1 = q[k1 + HN];
      e[m] = Cx<T>{y0.x + y1.x, y0.y + y1.y};
      o[m] = cmulc(Cx<T>{y0.x - y1.x, y0.y - y1.y}, tw[k1]);
    }
  }
  warp_dit_inv<T, HN, N>(e, tw, lane);
  warp_dit_inv<T, HN, N>(o, tw, lane);
#pragma unroll
  for (int m = 0; m < MC; ++m) {
    E[(lane + 32 * m) * PT + warp] = e[m];
    O[(lane + 32 * m) * PT + warp] = o[m];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < HN * kFcCols; t += blockDim.x) {
    const int k = t / kFcCols, s2 = t % kFcCols;
    const int pp = p0 + s2;
    const int co = pp == 0 ? HN : N - pp;
    Cb[(size_t)k * N + pp] = E[k * PT + s2];
    Cb[(size_t)k * N + co] = O[k * PT + s2];
  }
}

template <typename T, int N>
size_t fwarp_cols_smem() {
  return (size_t)(N / 2 + N + 2 * (N / 2) * (kFcCols + 1)) * sizeof(Cx<T>) +
         (size_t)(N / 2 + 2) * sizeof(T);
}

template <typename T, int N>
__global__ void __launch_bounds__(32 * kFrWarps)
k_fwarp_rows_inv(const Cx<T>* __restrict__ C, const T* xstar, T* x, const Cx<T>* __restrict__ twg,
                 const int* __restrict__ active) {
  constexpr int HN = N / 2, MR = N / 32;
  const int b = blockIdx.y;
  if (!active[b]) return;
  extern __shared__ __align__(16) unsigned char fr_smem[];
  Cx<T>* tw = reinterpret_cast<Cx<T>*>(fr_smem);  // [HN], then one row per warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < HN; k += blockDim.x) tw[k] = twg[k];
  __syncthreads();
  const int k = blockIdx.x * kFrWarps + warp;
  const size_t plane = (size_t)N * N;
  const Cx<T>* Cr = C + (size_t)b * (plane / 2) + (size_t)k * N;
  Cx<T>* row = tw + HN + warp * N;
  for (int t = lane; t < HN; t += 32) {
    if (t == 0) {
      const Cx<T> a = Cr[0], c = Cr[HN];
      row[0] = Cx<T>{a.x, c.x};
      row[HN] = Cx<T>{a.y, c.y};
    } else {
      const Cx<T> xa = Cr[t], xb = Cr[N - t];
      row[t] = Cx<T>{xa.x - xb.y, xa.y + xb.x};
      row[N - t] = Cx<T>{xa.x + xb.y, xb.x - xa.y};
    }
  }
  __syncwarp();
  Cx<T> v[MR];
#pragma unroll
  for (int m = 0; m < MR; ++m) v[m] = row[brev_len<N>(lane + 32 * m)];
  warp_dit_inv<T, N, N>(v, tw, lane);
  const T scale = T(1.0 / ((double)N * (double)N));
  const size_t g0 = (size_t)b * plane + (size_t)(2 * k) * N;
#pragma unroll
  for (int m = 0; m < MR; ++m) {
    const size_t g = g0 + lane + 32 * m;
    x[g] = (xstar ? xstar[g] : T(0)) + v[m].x * scale;
    x[g + N] = (xstar ? xstar[g + N] : T(0)) + v[m].y * scale;
  }
}

template <typename T, int N>
void launch_fwarp3(int B, const T* xstar, const T* h, T* x, Cx<T>* C, const Cx<T>* tw,
                   const double* mask_tab, const int* active, cudaStream_t st, LaunchLog& log,
                   double units) {
  const size_t smc = fwarp_cols_smem<T, N>();
  const size_t smr = (size_t)(N / 2 + kFrWarps * N) * sizeof(Cx<T>);
  cudaFuncSetAttribute(k_fwarp_cols<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc);
  cudaFuncSetAttribute(k_fwarp_rows_fwd<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr);
  cudaFuncSetAttribute(k_fwarp_rows_inv<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr);
  int pi_ = log.begin(K_FILTER, st);
  k_fwarp_rows_fwd<T, N><<<dim3(N / 2 / kFrWarps, B), 32 * kFrWarps, smr, st>>>(h, C, tw, active);
  log.end(pi_, st, units);
  pi_ = log.begin(K_FILTER, st);
  k_fwarp_cols<T, N><<<dim3(N / 2 / kFcCols, B), 32 * kFcCols, smc, st>>>(C, tw, mask_tab, active);
  log.end(pi_, st, units);
  pi_ = log.begin(K_FILTER, st);
  k_fwarp_rows_inv<T, N><<<dim3(N / 2 / kFrWarps, B), 32 * kFrWarps, smr, st>>>(C, xstar, x, tw, active);
  log.end(pi_, st, units);
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
  const int logn = ilog2(n), halfn = n / 2;
  Cx<T>* C = reinterpret_cast<Cx<T>*>(cbuf);
  const Cx<T>* tw = reinterpret_cast<const Cx<T>*>(twiddles);
  const double units = (double)n * n * log.active_hint;
  // warp-level form (default where it applies; autotuner mode 2)
  if ((n == 64 || n == 128) && (mode == 2 || mode < 0)) {
    const size_t sm = n == 64 ? filter_warp_smem<T, 64>() : filter_warp_smem<T, 128>();
    if (sm <= 200 * 1024) {
      auto kern = n == 64 ? k_filter_warp<T, 64> : k_filter_warp<T, 128>;
      const int threads = n == 64 ? FWThreads<64>::value : FWThreads<128>::value;
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      int pi_ = log.begin(K_FILTER, st);
      kern<<<B, threads, sm, st>>>(xstar, h, x, tw, mask_tab, active);
      log.end(pi_, st, units);
      return;
    }
  }
  // warp-level three-pass form (default for 256 and 512; autotuner mode 3)
  if ((n == 256 || n == 512) && (mode == 3 || mode < 0)) {
    if (n == 256)
      launch_fwarp3<T, 256>(B, xstar, h, x, C, tw, mask_tab, active, st, log, units);
    else
      launch_fwarp3<T, 512>(B, xstar, h, x, C, tw, mask_tab, active, st, log, units);
    return;
  }
  const size_t fused_sm = (size_t)(halfn + (size_t)n * halfn) * sizeof(Cx<T>);
  if (fused_sm <= 160 * 1024 && mode != 0 && mode != 3) {
    cudaFuncSetAttribute(k_filter_fused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_sm);
    const int work = n * n / 4;
    const int threads = work < 32 ? 32 : (work > 512 ? 512 : work);
    int pi_ = log.begin(K_FILTER, st);
    k_filter_fused<T><<<B, threads, fused_sm, st>>>(n, logn, xstar, h, x, tw, mask_tab, active);
    log.end(pi_, st, units);
    return;
  }
  // row pairs per block (rows passes) and column frequencies per block
  // (column pass): about 64 KB of complex data per block
  int per = (int)((64 * 1024) / (n * sizeof(Cx<T>)));
  per = per < 1 ? 1 : (per > 32 ? 32 : per);
  if (per > halfn) per = halfn;
  while (halfn % per) --per;
  int cpc = (int)((64 * 1024) / (n * sizeof(Cx<T>)));
  cpc = cpc < 1 ? 1 : (cpc > 16 ? 16 : cpc);
  if (cpc > halfn) cpc = halfn;
  while (halfn % cpc) --cpc;
  const size_t sm_rows = (size_t)(halfn + per * n) * sizeof(Cx<T>);
  const size_t sm_cols = (size_t)(halfn + 2 * cpc * halfn) * sizeof(Cx<T>);
  cudaFuncSetAttribute(k_fft_rows_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_rows);
  cudaFuncSetAttribute(k_fft_cols_mask<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_cols);
  cudaFuncSetAttribute(k_fft_rows_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_rows);
  const dim3 grows(halfn / per, B), gcols(halfn / cpc, B);
  int pi_ = log.begin(K_FILTER, st);
  k_fft_rows_fwd<T><<<grows, 256, sm_rows, st>>>(n, logn, per, h, C, tw, active);
  log.end(pi_, st, units);
  pi_ = log.begin(K_FILTER, st);
  k_fft_cols_mask<T><<<gcols, 256, sm_cols, st>>>(n, logn, cpc, C, tw, mask_tab, active);
  log.end(pi_, st, units);
  pi_ = log.begin(K_FILTER, st);
  k_fft_rows_inv<T><<<grows, 256, sm_rows, st>>>(n, logn, per, C, xstar, x, tw, active);
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
