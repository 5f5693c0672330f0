// Dense Hermitian eigendecomposition on the host (the p x p Rayleigh-Ritz
// problems of the setup eigensolver, p up to a few thousand).
//
// Method (Householder 1958; Golub & Van Loan, Matrix Computations, 4th ed.,
// Sections 8.3.1 and 8.3.5):
//   1. reduce H to Hermitian tridiagonal form T = P^H H P by n - 2 Householder
//      reflections I - 2 v v^H, each applied to the trailing block as the
//      rank-2 update H <- H - v w^H - w v^H with p = H v, w = 2 p - 2 (v^H p) v;
//   2. make T real symmetric with a diagonal unitary D (phases of the
//      sub-diagonal): T = D T_r D^H;
//   3. diagonalise T_r by the implicit symmetric QL iteration with Wilkinson
//      shifts, accumulating the Givens rotations in a real matrix W;
//   4. eigenvectors of H: P D W (the reflections applied in reverse order).
// All arithmetic is FP64.  Eigenvalues ascending; vectors as columns of a
// row-major n x n complex matrix.
#pragma once

#include <algorithm>
#include <cmath>
#include <complex>
#include <thread>
#include <vector>

namespace dtr {

typedef std::complex<double> zc;

// Run f(lo, hi) over [0, n) split across the host's cores (serially when the
// range is small): the O(n^3) loops of the host linear algebra.
template <typename F> inline void host_parallel_for(int64_t n, int64_t serial_below, F f) {
  unsigned nt = std::thread::hardware_concurrency();
  if (nt > 32) nt = 32;
  if (nt <= 1 || n < serial_below) {
    f((int64_t)0, n);
    return;
  }
  if ((int64_t)nt > n) nt = (unsigned)n;
  std::vector<std::thread> th;
  th.reserve(nt);
  for (unsigned t = 0; t < nt; ++t) {
    const int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
    th.emplace_back([=] { f(lo, hi); });
  }
  for (auto &x : th) x.join();
}

// H: row-major n x n Hermitian (only used, not kept).  Returns 0 on success,
// 1 if the QL iteration did not converge (more than 60 sweeps per eigenvalue).
inline int herm_eig(int n, const std::vector<zc> &Hin, std::vector<double> &lam, std::vector<zc> &X) {
  lam.assign(n, 0.0);
  X.assign((size_t)n * n, zc(0.0, 0.0));
  if (n == 0) return 0;
  std::vector<zc> H(Hin);
  auto h = [&](int i, int j) -> zc & { return H[(size_t)i * n + j]; };
  std::vector<std::vector<zc>> refl;  // reflector k acts on rows/cols k+1 .. n-1
  std::vector<zc> p(n), v(n);
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;  // length of the column below the diagonal
    double xn = 0.0;
    for (int i = 0; i < m; ++i) xn += std::norm(h(k + 1 + i, k));
    xn = std::sqrt(xn);
    std::vector<zc> vk(m, zc(0.0, 0.0));
    if (xn == 0.0) {
      refl.push_back(vk);
      continue;
    }
    const zc x0 = h(k + 1, k);
    const zc ph = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : zc(1.0, 0.0);
    const zc alpha = -ph * xn;  // the column maps to alpha e1
    for (int i = 0; i < m; ++i) vk[i] = h(k + 1 + i, k);
    vk[0] -= alpha;
    double vn = 0.0;
    for (int i = 0; i < m; ++i) vn += std::norm(vk[i]);
    vn = std::sqrt(vn);
    for (int i = 0; i < m; ++i) vk[i] /= vn;
    // trailing block B = H[k+1:, k+1:]: p = B v, c = v^H p, w = 2 p - 2 c v
    host_parallel_for(m, 384, [&](int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i) {
        zc s(0.0, 0.0);
        const zc *row = &h(k + 1 + (int)i, k + 1);
        for (int j = 0; j < m; ++j) s += row[j] * vk[j];
        p[i] = s;
      }
    });
    zc c(0.0, 0.0);
    for (int i = 0; i < m; ++i) c += std::conj(vk[i]) * p[i];
    for (int i = 0; i < m; ++i) p[i] = 2.0 * p[i] - 2.0 * c.real() * vk[i];
    host_parallel_for(m, 384, [&](int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i) {
        zc *row = &h(k + 1 + (int)i, k + 1);
        const zc vi = vk[i], wi = p[i];
        for (int j = 0; j < m; ++j) row[j] -= vi * std::conj(p[j]) + wi * std::conj(vk[j]);
      }
    });
    // the column (and row) k becomes alpha e1
    h(k + 1, k) = alpha;
    h(k, k + 1) = std::conj(alpha);
    for (int i = 1; i < m; ++i) h(k + 1 + i, k) = h(k, k + 1 + i) = zc(0.0, 0.0);
    refl.push_back(vk);
  }
  // real symmetric tridiagonal: d_i = Re T_ii, e_i = |T_(i+1),i|, D_(i+1) = D_i * phase(T_(i+1),i)
  std::vector<double> d(n), e(n, 0.0);
  std::vector<zc> D(n);
  D[0] = zc(1.0, 0.0);
  for (int i = 0; i < n; ++i) d[i] = h(i, i).real();
  for (int i = 0; i + 1 < n; ++i) {
    const zc t = h(i + 1, i);
    const double a = std::abs(t);
    e[i] = a;
    D[i + 1] = a > 0.0 ? D[i] * (t / a) : D[i];
  }
  // implicit QL with Wilkinson shifts on (d, e), rotations accumulated in W, kept
  // transposed (Wt row i = column i of W) so a rotation of two columns streams two rows
  std::vector<double> Wt((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Wt[(size_t)i * n + i] = 1.0;
  for (int l = 0; l < n; ++l) {
    int iter = 0;
    for (;;) {
      int m = l;
      for (; m + 1 < n; ++m) {
        const double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
        if (std::fabs(e[m]) <= 1e-16 * dd) break;
      }
      if (m == l) break;
      if (++iter > 60) return 1;
      // shift from the leading 2 x 2 block of the unreduced part
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = std::hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + (g >= 0.0 ? r : -r));
      double s = 1.0, c = 1.0, pp = 0.0;
      int i = m - 1;
      bool early = false;
      for (; i >= l; --i) {
        double f = s * e[i];
        const double b = c * e[i];
        r = std::hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {  // the rotation underflowed: deflate and restart
          d[i + 1] -= pp;
          e[m] = 0.0;
          early = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - pp;
        r = (d[i] - g) * s + 2.0 * c * b;
        pp = s * r;
        d[i + 1] = g + pp;
        g = c * r - b;
        // accumulate the rotation in columns i, i+1 of W (rows i, i+1 of Wt)
        double *w0 = &Wt[(size_t)i * n], *w1 = &Wt[(size_t)(i + 1) * n];
        for (int q = 0; q < n; ++q) {
          const double a0 = w0[q], a1 = w1[q];
          w1[q] = s * a0 + c * a1;
          w0[q] = c * a0 - s * a1;
        }
      }
      if (early) continue;
      d[l] -= pp;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  // sort ascending
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  for (int i = 1; i < n; ++i) {  // insertion sort (n is modest, and d is nearly sorted)
    const int t = ord[i];
    int j = i - 1;
    while (j >= 0 && d[ord[j]] > d[t]) {
      ord[j + 1] = ord[j];
      --j;
    }
    ord[j + 1] = t;
  }
  // X = P D W: start from D W (column order by ord), then apply the reflectors in reverse
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) X[(size_t)i * n + j] = D[i] * Wt[(size_t)ord[j] * n + i];
  for (int j = 0; j < n; ++j) lam[j] = d[ord[j]];
  std::vector<zc> t(n);
  for (int k = (int)refl.size() - 1; k >= 0; --k) {
    const std::vector<zc> &vk = refl[k];
    const int m = (int)vk.size();
    bool zero = true;
    for (int i = 0; i < m && zero; ++i) zero = vk[i] == zc(0.0, 0.0);
    if (zero) continue;
    // rows k+1 .. n-1 of X: X <- (I - 2 v v^H) X, columns split across threads
    host_parallel_for(n, 256, [&](int64_t lo, int64_t hi) {
      for (int64_t j = lo; j < hi; ++j) t[j] = zc(0.0, 0.0);
      for (int i = 0; i < m; ++i) {
        const zc cv = std::conj(vk[i]);
        const zc *row = &X[(size_t)(k + 1 + i) * n];
        for (int64_t j = lo; j < hi; ++j) t[j] += cv * row[j];
      }
      for (int i = 0; i < m; ++i) {
        const zc vi = 2.0 * vk[i];
        zc *row = &X[(size_t)(k + 1 + i) * n];
        for (int64_t j = lo; j < hi; ++j) row[j] -= vi * t[j];
      }
    });
  }
  return 0;
}

}  // namespace dtr
