// sld_hritz.cu -- harmonic Ritz pairs of an Arnoldi cycle (host code), for
// GMRES with harmonic-Ritz deflation (Section 3.2.1, eq. (defleig), form (a)):
//
//   F = H_m + h_{m+1,m}^2 H_m^{-T} e_m e_m^T,   F y = theta y,   z = V_m y.
//
// F is H_m with its last column changed, so it stays upper Hessenberg.  Its
// eigenvalues come from the Francis double-shift QR iteration on a
// Hessenberg matrix (Francis 1961; Golub and Van Loan, "Matrix
// Computations", the implicit double-shift step with 3x3 Householder
// reflectors and deflation at negligible subdiagonals); its eigenvectors from
// inverse iteration on F - theta I (complex arithmetic for complex theta).
// The d pairs of smallest |theta| are returned as a real basis: a
// complex-conjugate pair contributes its real and imaginary parts (the
// paper's transformation to real Schur vectors).
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "sld_internal.h"

namespace sld {
namespace {

using cd = std::complex<double>;

// Eigenvalues of the upper Hessenberg n x n matrix a (row-major, destroyed).
bool hessenberg_eigenvalues(std::vector<double>& a, int n, std::vector<cd>* ev) {
  auto A = [&](int i, int j) -> double& { return a[(size_t)i * n + j]; };
  double norm = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = std::max(0, i - 1); j < n; ++j) norm += std::fabs(A(i, j));
  const double eps = 2.220446049250313e-16;
  int hi = n - 1, iter = 0, total = 0;
  while (hi >= 0) {
    int l = hi;
    while (l > 0) {  // a negligible subdiagonal splits the active block
      double s = std::fabs(A(l - 1, l - 1)) + std::fabs(A(l, l));
      if (s == 0.0) s = norm;
      if (std::fabs(A(l, l - 1)) <= eps * s) {
        A(l, l - 1) = 0.0;
        break;
      }
      --l;
    }
    if (l == hi) {  // 1 x 1 block
      ev->push_back(cd(A(hi, hi), 0.0));
      --hi;
      iter = 0;
      continue;
    }
    if (l == hi - 1) {  // 2 x 2 block: roots of its characteristic polynomial
      const double p = A(hi - 1, hi - 1), q = A(hi - 1, hi), r = A(hi, hi - 1), t = A(hi, hi);
      const double half = 0.5 * (p - t), disc = half * half + q * r, mid = 0.5 * (p + t);
      if (disc >= 0.0) {
        const double sq = std::sqrt(disc);
        // the root of larger magnitude first, the other from the product (no cancellation)
        const double r1 = mid + (mid >= 0.0 ? sq : -sq);
        const double det = p * t - q * r;
        const double r2 = r1 != 0.0 ? det / r1 : mid - (mid >= 0.0 ? sq : -sq);
        ev->push_back(cd(r1, 0.0));
        ev->push_back(cd(r2, 0.0));
      } else {
        const double im = std::sqrt(-disc);
        ev->push_back(cd(mid, im));
        ev->push_back(cd(mid, -im));
      }
      hi -= 2;
      iter = 0;
      continue;
    }
    if (++iter > 80 || ++total > 40 * n) return false;
    // shifts: the eigenvalues of the trailing 2 x 2 block (sum s, product t),
    // replaced by an ad hoc pair every tenth step of a stuck block
    double s = A(hi - 1, hi - 1) + A(hi, hi);
    double t = A(hi - 1, hi - 1) * A(hi, hi) - A(hi - 1, hi) * A(hi, hi - 1);
    if (iter % 10 == 0) {
      const double w = std::fabs(A(hi, hi - 1)) + std::fabs(A(hi - 1, hi - 2));
      s = 1.5 * w;
      t = w * w;
    }
    // first column of (H - s1 I)(H - s2 I) = H^2 - s H + t I on the block
    double x = A(l, l) * A(l, l) + A(l, l + 1) * A(l + 1, l) - s * A(l, l) + t;
    double y = A(l + 1, l) * (A(l, l) + A(l + 1, l + 1) - s);
    double z = A(l + 1, l) * A(l + 2, l + 1);
    for (int k = l; k <= hi - 2; ++k) {
      // Householder reflector P = I - 2 v v^T / v^T v with P (x, y, z)^T = (alpha, 0, 0)^T
      // A zero (x, y, z) needs no reflector; the bulge chase still moves on
      // to the next column, so the reload below runs on every k.
      const double nrm = std::sqrt(x * x + y * y + z * z);
      const double alpha = x > 0.0 ? -nrm : nrm;
      const double v0 = x - alpha, v1 = y, v2 = z;
      const double vv = v0 * v0 + v1 * v1 + v2 * v2;
      if (nrm != 0.0 && vv != 0.0) {
        const double f = 2.0 / vv;
        const int c0 = std::max(l, k - 1);
        for (int j = c0; j < n; ++j) {  // rows k .. k+2 from the left
          const double dot = v0 * A(k, j) + v1 * A(k + 1, j) + v2 * A(k + 2, j);
          A(k, j) -= f * v0 * dot;
          A(k + 1, j) -= f * v1 * dot;
          A(k + 2, j) -= f * v2 * dot;
        }
        const int r1 = std::min(hi, k + 3);
        for (int i = 0; i <= r1; ++i) {  // columns k .. k+2 from the right
          const double dot = v0 * A(i, k) + v1 * A(i, k + 1) + v2 * A(i, k + 2);
          A(i, k) -= f * v0 * dot;
          A(i, k + 1) -= f * v1 * dot;
          A(i, k + 2) -= f * v2 * dot;
        }
      }
      x = A(k + 1, k);
      y = A(k + 2, k);
      z = k < hi - 2 ? A(k + 3, k) : 0.0;
    }
    {  // last step: a 2 x 2 reflector on rows/columns hi-1, hi
      const int k = hi - 1;
      const double nrm = std::hypot(x, y);
      if (nrm != 0.0) {
        const double alpha = x > 0.0 ? -nrm : nrm;
        const double v0 = x - alpha, v1 = y;
        const double vv = v0 * v0 + v1 * v1;
        if (vv != 0.0) {
          const double f = 2.0 / vv;
          for (int j = std::max(l, k - 1); j < n; ++j) {
            const double dot = v0 * A(k, j) + v1 * A(k + 1, j);
            A(k, j) -= f * v0 * dot;
            A(k + 1, j) -= f * v1 * dot;
          }
          for (int i = 0; i <= hi; ++i) {
            const double dot = v0 * A(i, k) + v1 * A(i, k + 1);
            A(i, k) -= f * v0 * dot;
            A(i, k + 1) -= f * v1 * dot;
          }
        }
      }
    }
  }
  return true;
}

// y with (F - theta I) y = 0 by inverse iteration (Gaussian elimination with
// partial pivoting, complex).  F: n x n row-major.
bool inverse_iteration(const std::vector<double>& F, int n, cd theta, std::vector<cd>* y) {
  const double scale = [&] {
    double s = 0.0;
    for (double v : F) s = std::max(s, std::fabs(v));
    return s > 0.0 ? s : 1.0;
  }();
  const cd shift = theta + cd(1e-10 * scale, 0.0);
  std::vector<cd> M((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) M[(size_t)i * n + j] = cd(F[(size_t)i * n + j], 0.0) - (i == j ? shift : cd(0.0));
  std::vector<int> piv(n);
  for (int c = 0; c < n; ++c) {  // LU with partial pivoting, in place
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::abs(M[(size_t)r * n + c]) > std::abs(M[(size_t)p * n + c])) p = r;
    piv[c] = p;
    if (p != c)
      for (int j = 0; j < n; ++j) std::swap(M[(size_t)c * n + j], M[(size_t)p * n + j]);
    cd d = M[(size_t)c * n + c];
    if (std::abs(d) == 0.0) d = M[(size_t)c * n + c] = cd(1e-300, 0.0);
    for (int r = c + 1; r < n; ++r) {
      const cd f = M[(size_t)r * n + c] / d;
      M[(size_t)r * n + c] = f;
      for (int j = c + 1; j < n; ++j) M[(size_t)r * n + j] -= f * M[(size_t)c * n + j];
    }
  }
  y->assign(n, cd(1.0, 0.0));
  for (int it = 0; it < 3; ++it) {
    std::vector<cd>& b = *y;
    // whole rows were swapped during the factorisation (P F' = L U): all the
    // interchanges first, then the unit lower triangle
    for (int c = 0; c < n; ++c)
      if (piv[c] != c) std::swap(b[c], b[piv[c]]);
    for (int c = 0; c < n; ++c)
      for (int r = c + 1; r < n; ++r) b[r] -= M[(size_t)r * n + c] * b[c];
    for (int r = n - 1; r >= 0; --r) {
      cd t = b[r];
      for (int j = r + 1; j < n; ++j) t -= M[(size_t)r * n + j] * b[j];
      b[r] = t / M[(size_t)r * n + r];
    }
    double nb = 0.0;
    for (const cd& v : b) nb += std::norm(v);
    nb = std::sqrt(nb);
    if (!(nb > 0.0) || !std::isfinite(nb)) return false;
    for (cd& v : b) v /= nb;
  }
  return true;
}

}  // namespace

int harmonic_ritz(const double* Hbar, int m, int d, double* Y, double* theta_re, double* theta_im) {
  // Work on Hbar / 2^e with 2^e near its largest entry (an exact scaling):
  // F scales with Hbar, its eigenvectors do not, and products of entries
  // (h^2, the QR shifts, the 3-vectors of the bulge chase) then neither
  // underflow nor overflow for Hbar of any magnitude.
  double amax = 0.0;
  for (int i = 0; i < (m + 1) * m; ++i) {
    if (!std::isfinite(Hbar[i])) return SLD_ERR_BREAKDOWN;
    amax = std::max(amax, std::fabs(Hbar[i]));
  }
  if (amax == 0.0) return SLD_ERR_BREAKDOWN;
  int ex = 0;
  std::frexp(amax, &ex);
  const double unscale = std::ldexp(1.0, ex);
  // F = H_m + h_{m+1,m}^2 f e_m^T with H_m^T f = e_m
  std::vector<double> F((size_t)m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) F[(size_t)i * m + j] = std::ldexp(Hbar[(size_t)i * m + j], -ex);
  const double h = std::ldexp(Hbar[(size_t)m * m + (m - 1)], -ex);
  if (h != 0.0) {
    std::vector<double> HT((size_t)m * m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) HT[(size_t)i * m + j] = F[(size_t)j * m + i];
    // solve H_m^T f = e_m: inverse iteration machinery with shift 0 would
    // perturb it, so a plain elimination here
    std::vector<double> M = HT, rhs(m, 0.0);
    rhs[m - 1] = 1.0;
    for (int c = 0; c < m; ++c) {
      int p = c;
      for (int r = c + 1; r < m; ++r)
        if (std::fabs(M[(size_t)r * m + c]) > std::fabs(M[(size_t)p * m + c])) p = r;
      if (M[(size_t)p * m + c] == 0.0) return SLD_ERR_BREAKDOWN;
      if (p != c) {
        for (int j = 0; j < m; ++j) std::swap(M[(size_t)c * m + j], M[(size_t)p * m + j]);
        std::swap(rhs[c], rhs[p]);
      }
      for (int r = c + 1; r < m; ++r) {
        const double g = M[(size_t)r * m + c] / M[(size_t)c * m + c];
        for (int j = c; j < m; ++j) M[(size_t)r * m + j] -= g * M[(size_t)c * m + j];
        rhs[r] -= g * rhs[c];
      }
    }
    std::vector<double> fv(m);
    for (int r = m - 1; r >= 0; --r) {
      double t = rhs[r];
      for (int j = r + 1; j < m; ++j) t -= M[(size_t)r * m + j] * fv[j];
      fv[r] = t / M[(size_t)r * m + r];
    }
    for (int i = 0; i < m; ++i) F[(size_t)i * m + (m - 1)] += h * h * fv[i];
  }
  std::vector<double> work = F;
  std::vector<cd> ev;
  if (!hessenberg_eigenvalues(work, m, &ev) || (int)ev.size() != m) return SLD_ERR_BREAKDOWN;
  std::vector<int> order(m);
  for (int i = 0; i < m; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return std::abs(ev[a]) < std::abs(ev[b]); });
  int got = 0;
  std::vector<bool> used(m, false);
  for (int oi = 0; oi < m && got < d; ++oi) {
    const int k = order[oi];
    if (used[k]) continue;
    used[k] = true;
    std::vector<cd> y;
    if (!inverse_iteration(F, m, ev[k], &y)) return SLD_ERR_BREAKDOWN;
    const bool cplx = ev[k].imag() != 0.0;
    if (cplx) {  // skip the conjugate; its space is the same
      for (int oj = oi + 1; oj < m; ++oj) {
        const int k2 = order[oj];
        if (!used[k2] && std::abs(ev[k2] - std::conj(ev[k])) <= 1e-12 * std::abs(ev[k]) + 1e-300) {
          used[k2] = true;
          break;
        }
      }
    }
    // fix the phase so that the largest entry is real (a deterministic basis)
    int big = 0;
    for (int i = 1; i < m; ++i)
      if (std::abs(y[i]) > std::abs(y[big])) big = i;
    const cd ph = std::abs(y[big]) > 0.0 ? std::conj(y[big]) / std::abs(y[big]) : cd(1.0);
    for (cd& v : y) v *= ph;
    for (int i = 0; i < m; ++i) Y[(size_t)i * d + got] = y[i].real();
    theta_re[got] = ev[k].real() * unscale;
    theta_im[got] = ev[k].imag() * unscale;
    ++got;
    if (cplx && got < d) {
      for (int i = 0; i < m; ++i) Y[(size_t)i * d + got] = y[i].imag();
      theta_re[got] = ev[k].real() * unscale;
      theta_im[got] = -ev[k].imag() * unscale;
      ++got;
    }
  }
  return got == d ? SLD_OK : SLD_ERR_BREAKDOWN;
}

}  // namespace sld

extern "C" sld_status sld_harmonic_ritz(const double* Hbar, int m, int d, double* Y, double* theta_re,
                                        double* theta_im) {
  if (!Hbar || !Y || !theta_re || !theta_im || m < 2 || m > 64 || d < 1 || d > m) {
    sld::set_last_error("sld_harmonic_ritz: need Hbar, Y, theta arrays, 2 <= m <= 64, 1 <= d <= m");
    return SLD_ERR_INVALID_ARG;
  }
  const int code = sld::harmonic_ritz(Hbar, m, d, Y, theta_re, theta_im);
  if (code != SLD_OK) sld::set_last_error("sld_harmonic_ritz: the QR iteration or inverse iteration failed");
  return (sld_status)code;
}
