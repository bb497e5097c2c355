// Host-side setup of the level hierarchy in fp64.
//
// Galerkin coarse operators (Algorithm 1's A^(l+1) = I_l^{l+1} A^(l) I_{l+1}^l,
// used by Algorithms 3 and 4) with linear interpolation P and full weighting
// R = P^T / 2 per axis.  In 2D the operator keeps the Kronecker form
// alpha M(x)M + K(x)K, so only the 1D factors are coarsened:
// M_{l+1} = R M_l P, K_{l+1} = R K_l P.  P and R have three nonzeros per
// column/row, so each coarse entry is a 3x3 weighted sum of fine entries and
// the band half-width grows as w -> floor(w/2) + 1.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "nmg_internal.h"

namespace nmg {

namespace {

// P[f][J] for fine index f and coarse index J (nc coarse points)
inline double pw(int f, int J, int nc) {
  if (J < 0 || J >= nc) return 0.0;
  int d = f - 2 * J;
  if (d == 0) return 1.0;
  if (d == 1 || d == -1) return (f >= 0 && f < 2 * nc) ? 0.5 : 0.0;
  return 0.0;
}

// generic banded accessor for a DIA matrix
struct Dia {
  int n, w;
  const double* d;
  double at(int i, int j) const {
    if (i < 0 || i >= n || j < 0 || j >= n) return 0.0;
    int k = j - i + w;
    if (k < 0 || k > 2 * w) return 0.0;
    return d[(size_t)i * (2 * w + 1) + k];
  }
};

// coarse = R F P for a DIA fine matrix; returns DIA with half-width w/2+1
std::vector<double> galerkin_dia(const Dia& F, int& wc) {
  int nf = F.n, nc = nf / 2;
  wc = F.w / 2 + 1;
  std::vector<double> out((size_t)nc * (2 * wc + 1), 0.0);
  for (int I = 0; I < nc; ++I) {
    for (int k = 0; k <= 2 * wc; ++k) {
      int J = I + k - wc;
      if (J < 0 || J >= nc) continue;
      double acc = 0.0;
      for (int da = -1; da <= 1; ++da) {
        int a = 2 * I + da;
        double r = 0.5 * pw(a, I, nc);  // R[I][a] = P[a][I] / 2
        if (r == 0.0) continue;
        for (int db = -1; db <= 1; ++db) {
          int b = 2 * J + db;
          double p = pw(b, J, nc);
          if (p == 0.0) continue;
          acc += r * F.at(a, b) * p;
        }
      }
      out[(size_t)I * (2 * wc + 1) + k] = acc;
    }
  }
  return out;
}

std::vector<double> galerkin_dense(const std::vector<double>& A, int nf) {
  int nc = nf / 2;
  std::vector<double> out((size_t)nc * nc, 0.0);
  for (int I = 0; I < nc; ++I)
    for (int J = 0; J < nc; ++J) {
      double acc = 0.0;
      for (int da = -1; da <= 1; ++da) {
        int a = 2 * I + da;
        if (a < 0 || a >= nf) continue;
        double r = 0.5 * pw(a, I, nc);
        for (int db = -1; db <= 1; ++db) {
          int b = 2 * J + db;
          if (b < 0 || b >= nf) continue;
          acc += r * A[(size_t)a * nf + b] * pw(b, J, nc);
        }
      }
      out[(size_t)I * nc + J] = acc;
    }
  return out;
}

}  // namespace

bool build_host_hierarchy(const nmg_operator_desc& op, HostHierarchy& H, std::string& err) {
  if (op.dim != 1 && op.dim != 2) { err = "dim must be 1 or 2"; return false; }
  if (op.levels < 1 || op.levels > 16) { err = "levels must be in [1, 16]"; return false; }
  if (op.n < 2 || (op.n & (op.n - 1)) != 0) { err = "n must be a power of two >= 2"; return false; }
  if (op.n % (1 << (op.levels - 1)) != 0 || (op.n >> (op.levels - 1)) < 1) {
    err = "n must be divisible by 2^(levels-1)";
    return false;
  }
  if (!op.taps) { err = "taps is NULL"; return false; }
  if (!(std::isfinite(op.alpha))) { err = "alpha is not finite"; return false; }
  H.dim = op.dim;
  H.n = op.n;
  H.levels = op.levels;
  H.alpha = op.alpha;
  H.lv.assign(op.levels, HostLevel());
  int ncoarse = op.n >> (op.levels - 1);
  H.nc = op.dim == 1 ? ncoarse : ncoarse * ncoarse;
  if (H.nc > 1024) { err = "coarsest level has more than 1024 unknowns"; return false; }
  if (op.reg && op.dim != 1) { err = "reg (tridiagonal D) is 1D only"; return false; }
  if (op.reg && op.nreg != 2 * op.n - 1) { err = "reg must hold 2n-1 values (diagonal, off-diagonal)"; return false; }
  if (op.dim == 1) {
    if (op.ntaps != op.n) { err = "1D: ntaps must equal n (first Toeplitz column)"; return false; }
    int n = op.n;
    std::vector<double> A((size_t)n * n);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = op.taps[std::abs(i - j)] + (i == j && !op.reg ? op.alpha : 0.0);
    if (op.reg) {
      // A = Toeplitz(t) + alpha D, D symmetric tridiagonal (Section 4.1)
      for (int i = 0; i < n; ++i) {
        A[(size_t)i * n + i] += op.alpha * op.reg[i];
        if (i + 1 < n) {
          A[(size_t)i * n + i + 1] += op.alpha * op.reg[n + i];
          A[(size_t)(i + 1) * n + i] += op.alpha * op.reg[n + i];
        }
      }
    }
    H.lv[0].n = n;
    H.lv[0].A = A;
    for (int l = 1; l < op.levels; ++l) {
      int nf = H.lv[l - 1].n;
      H.lv[l].n = nf / 2;
      H.lv[l].A = galerkin_dense(H.lv[l - 1].A, nf);
    }
    H.coarse = H.lv[op.levels - 1].A;
    return true;
  }
  int w = op.ntaps - 1;
  if (w < 0 || w >= op.n) { err = "2D: need 1 <= ntaps <= n"; return false; }
  HostLevel& L0 = H.lv[0];
  L0.n = op.n;
  L0.wK = w;
  L0.wM = 0;
  L0.Kd.assign((size_t)op.n * (2 * w + 1), 0.0);
  L0.Md.assign((size_t)op.n, 1.0);
  for (int i = 0; i < op.n; ++i)
    for (int k = 0; k <= 2 * w; ++k) {
      int j = i + k - w;
      if (j >= 0 && j < op.n) L0.Kd[(size_t)i * (2 * w + 1) + k] = op.taps[std::abs(k - w)];
    }
  for (int l = 1; l < op.levels; ++l) {
    const HostLevel& F = H.lv[l - 1];
    HostLevel& C = H.lv[l];
    C.n = F.n / 2;
    C.Kd = galerkin_dia(Dia{F.n, F.wK, F.Kd.data()}, C.wK);
    C.Md = galerkin_dia(Dia{F.n, F.wM, F.Md.data()}, C.wM);
    // the Galerkin band of M stays tridiagonal (w: 0 -> 1 -> 1 ...)
  }
  // dense coarsest operator alpha M(x)M + K(x)K, row-major index i*nl + j
  const HostLevel& C = H.lv[op.levels - 1];
  int nl = C.n;
  Dia K{nl, C.wK, C.Kd.data()}, M{nl, C.wM, C.Md.data()};
  H.coarse.assign((size_t)H.nc * H.nc, 0.0);
  for (int i = 0; i < nl; ++i)
    for (int j = 0; j < nl; ++j)
      for (int a = 0; a < nl; ++a)
        for (int b = 0; b < nl; ++b)
          H.coarse[(size_t)(i * nl + j) * H.nc + (a * nl + b)] =
              op.alpha * M.at(i, a) * M.at(j, b) + K.at(i, a) * K.at(j, b);
  return true;
}

// m'(k) = sqrt(|omega_k| / pi) with |omega_k| = 2 pi k / n for the folded
// bin k = min(j, n - j) (Section 3.2; the same local symbol on every level).
std::vector<double> filter_mask_table(int n) {
  std::vector<double> t(n / 2 + 1);
  for (int k = 0; k <= n / 2; ++k) t[k] = std::sqrt(2.0 * k / n);
  return t;
}

// First column of the real symmetric circulant Re(IDFT(m' . DFT(.))):
// c[d] = (1/n) sum_j m'_j cos(2 pi j d / n).
std::vector<double> filter_circulant_1d(int n) {
  std::vector<double> c(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int d = 0; d < n; ++d) {
    double acc = 0.0;
    for (int j = 0; j < n; ++j) {
      int k = j < n - j ? j : n - j;
      double m = std::sqrt(2.0 * k / n);
      // reduce the angle exactly in integers before the cosine
      long long q = ((long long)j * d) % n;
      acc += m * std::cos(2.0 * pi * (double)q / n);
    }
    c[d] = acc / n;
  }
  return c;
}

bool stencil_form(const std::vector<double>& dia, int n, int w, std::vector<double>& s, int& nb,
                  std::vector<double>& corr) {
  const int nk = 2 * w + 1;
  const int ref = n / 2;  // an interior row: all of its band lies in the grid
  if (ref - w < 0 || ref + w >= n) return false;
  s.assign(dia.begin() + (size_t)ref * nk, dia.begin() + (size_t)(ref + 1) * nk);
  double smax = 0.0;
  for (double v : s) smax = std::max(smax, std::fabs(v));
  const double tol = 1e-14 * smax;
  auto differs = [&](int g) {
    for (int k = 0; k < nk; ++k) {
      const int j = g + k - w;
      if (j >= 0 && j < n && std::fabs(dia[(size_t)g * nk + k] - s[k]) > tol) return true;
    }
    return false;
  };
  nb = 0;
  for (int g = 0; g < n; ++g)
    if (differs(g)) nb = g + 1;
  if (nb > w) return false;  // only the first w rows may differ
  corr.assign((size_t)nb * nk, 0.0);
  for (int g = 0; g < nb; ++g)
    for (int k = 0; k < nk; ++k) {
      const int j = g + k - w;
      if (j >= 0 && j < n) corr[(size_t)g * nk + k] = dia[(size_t)g * nk + k] - s[k];
    }
  return true;
}

std::vector<double> fft_twiddles(int n) {
  const double pi = 3.14159265358979323846;
  std::vector<double> t(n);  // n/2 complex
  for (int k = 0; k < n / 2; ++k) {
    t[2 * k] = std::cos(2.0 * pi * k / n);
    t[2 * k + 1] = -std::sin(2.0 * pi * k / n);
  }
  return t;
}

}  // namespace nmg
