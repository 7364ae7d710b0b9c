// Real eigen-decomposition A = S diag(lam) S^-1 of a small dense non-symmetric matrix with a
// real spectrum, on the host: the fast-diagonalisation factors of the paper's mapped
// second-derivative matrices (the Sec. 4.2 preconditioner on the Sec. 3.1 grid).
//
// Steps (Golub & Van Loan, Matrix Computations, 4th ed., ch. 7): Householder reduction to
// upper Hessenberg form; shifted QR steps on the active window (Wilkinson shift from the
// trailing 2 x 2 block, Givens rotations, deflation at negligible subdiagonals) to an
// upper-triangular Schur form T = Q^T A Q; eigenvectors of T by back substitution; S = Q X
// with unit columns; S^-1 by Gauss-Jordan elimination with partial pivoting.  A complex
// pair (a trailing 2 x 2 block with complex eigenvalues) is an error.
#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <vector>

#include "tps_internal.h"

namespace tps {

namespace {

constexpr double kEps = 2.220446049250313e-16;

// Givens pair (c, s) with [c s; -s c] (a, b)^T = (r, 0)^T
inline void givens(double a, double b, double &c, double &s) {
  const double r = std::hypot(a, b);
  if (r == 0.0) {
    c = 1.0;
    s = 0.0;
  } else {
    c = a / r;
    s = b / r;
  }
}

}  // namespace

int real_eig(int n, const double *A, double *lam, double *S, double *Sinv) {
  if (n < 1) return 1;
  const size_t nn = (size_t)n * n;
  std::vector<double> H(A, A + nn), Q(nn, 0.0), v(n);
  auto h = [&](int i, int j) -> double & { return H[(size_t)i * n + j]; };
  auto q = [&](int i, int j) -> double & { return Q[(size_t)i * n + j]; };
  for (int i = 0; i < n; ++i) q(i, i) = 1.0;
  double anorm = 0.0;
  for (size_t e = 0; e < nn; ++e) anorm = std::max(anorm, std::fabs(H[e]));
  if (anorm == 0.0) anorm = 1.0;

  // ---- Householder reduction to Hessenberg form, H <- P H P, Q <- Q P
  for (int k = 0; k + 2 < n; ++k) {
    double xnorm = 0.0;
    for (int i = k + 1; i < n; ++i) xnorm += h(i, k) * h(i, k);
    xnorm = std::sqrt(xnorm);
    if (xnorm == 0.0) continue;
    const double alpha = h(k + 1, k) > 0.0 ? -xnorm : xnorm;  // P x = alpha e_1
    std::fill(v.begin(), v.end(), 0.0);
    for (int i = k + 1; i < n; ++i) v[i] = h(i, k);
    v[k + 1] -= alpha;
    double vv = 0.0;
    for (int i = k + 1; i < n; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    const double beta = 2.0 / vv;
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int i = k + 1; i < n; ++i) s += v[i] * h(i, j);
      s *= beta;
      for (int i = k + 1; i < n; ++i) h(i, j) -= s * v[i];
    }
    for (int i = 0; i < n; ++i) {
      double s = 0.0, t = 0.0;
      for (int j = k + 1; j < n; ++j) {
        s += h(i, j) * v[j];
        t += q(i, j) * v[j];
      }
      s *= beta;
      t *= beta;
      for (int j = k + 1; j < n; ++j) {
        h(i, j) -= s * v[j];
        q(i, j) -= t * v[j];
      }
    }
    h(k + 1, k) = alpha;
    for (int i = k + 2; i < n; ++i) h(i, k) = 0.0;
  }

  // ---- shifted QR steps on the window [l, hi] until every subdiagonal is negligible
  std::vector<double> cs(n), sn(n);
  int hi = n - 1, iter = 0;
  while (hi > 0) {
    int l = hi;
    while (l > 0) {
      double s = std::fabs(h(l - 1, l - 1)) + std::fabs(h(l, l));
      if (s == 0.0) s = anorm;
      if (std::fabs(h(l, l - 1)) <= kEps * s) {
        h(l, l - 1) = 0.0;
        break;
      }
      --l;
    }
    if (l == hi) {  // a 1 x 1 block has converged
      --hi;
      iter = 0;
      continue;
    }
    if (++iter > 200) return 1;
    const double a = h(hi - 1, hi - 1), b = h(hi - 1, hi), c = h(hi, hi - 1), d = h(hi, hi);
    const double disc = 0.25 * (a - d) * (a - d) + b * c;
    double mu;
    if (disc >= 0.0) {
      const double r = std::sqrt(disc), m1 = 0.5 * (a + d) + r, m2 = 0.5 * (a + d) - r;
      mu = std::fabs(m1 - d) < std::fabs(m2 - d) ? m1 : m2;
    } else {
      if (l == hi - 1) return 1;  // an isolated complex pair
      mu = d;
    }
    if (iter % 20 == 19) mu = d + std::fabs(c);  // exceptional shift against cycling
    for (int k = l; k <= hi; ++k) h(k, k) -= mu;
    for (int k = l; k < hi; ++k) {  // H - mu = R: left rotations on rows k, k+1
      givens(h(k, k), h(k + 1, k), cs[k], sn[k]);
      for (int j = k; j < n; ++j) {
        const double x = h(k, j), y = h(k + 1, j);
        h(k, j) = cs[k] * x + sn[k] * y;
        h(k + 1, j) = -sn[k] * x + cs[k] * y;
      }
      h(k + 1, k) = 0.0;
    }
    for (int k = l; k < hi; ++k) {  // R G^T: right rotations on columns k, k+1; Q likewise
      const int top = std::min(k + 1, hi);
      for (int i = 0; i <= top; ++i) {
        const double x = h(i, k), y = h(i, k + 1);
        h(i, k) = cs[k] * x + sn[k] * y;
        h(i, k + 1) = -sn[k] * x + cs[k] * y;
      }
      for (int i = 0; i < n; ++i) {
        const double x = q(i, k), y = q(i, k + 1);
        q(i, k) = cs[k] * x + sn[k] * y;
        q(i, k + 1) = -sn[k] * x + cs[k] * y;
      }
    }
    for (int k = l; k <= hi; ++k) h(k, k) += mu;
  }

  // ---- eigenvectors of the triangular T by back substitution, then S = Q X, unit columns
  std::vector<double> X(nn, 0.0), ev(n);
  for (int k = 0; k < n; ++k) ev[k] = h(k, k);
  const double tiny = kEps * anorm;
  for (int k = 0; k < n; ++k) {
    X[(size_t)k * n + k] = 1.0;
    for (int j = k - 1; j >= 0; --j) {
      double s = 0.0;
      for (int m = j + 1; m <= k; ++m) s += h(j, m) * X[(size_t)m * n + k];
      double den = h(j, j) - ev[k];
      if (std::fabs(den) < tiny) den = den < 0.0 ? -tiny : tiny;
      X[(size_t)j * n + k] = -s / den;
      if (std::fabs(X[(size_t)j * n + k]) > 1e100) {  // rescale a growing vector
        for (int m = j; m <= k; ++m) X[(size_t)m * n + k] *= 1e-100;
      }
    }
  }
  std::vector<double> Sm(nn, 0.0);
  for (int i = 0; i < n; ++i)
    for (int m = 0; m < n; ++m) {
      const double qim = q(i, m);
      if (qim == 0.0) continue;
      for (int k = m; k < n; ++k) Sm[(size_t)i * n + k] += qim * X[(size_t)m * n + k];
    }
  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += Sm[(size_t)i * n + k] * Sm[(size_t)i * n + k];
    s = 1.0 / std::sqrt(s);
    for (int i = 0; i < n; ++i) Sm[(size_t)i * n + k] *= s;
  }

  // ---- ascending eigenvalues, columns permuted alike
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return ev[x] < ev[y]; });
  for (int k = 0; k < n; ++k) {
    lam[k] = ev[order[k]];
    for (int i = 0; i < n; ++i) S[(size_t)i * n + k] = Sm[(size_t)i * n + order[k]];
  }

  // ---- S^-1 by Gauss-Jordan elimination with partial pivoting
  if (Sinv) {
    std::vector<double> M(S, S + nn);
    for (size_t e = 0; e < nn; ++e) Sinv[e] = 0.0;
    for (int i = 0; i < n; ++i) Sinv[(size_t)i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
      int p = c;
      for (int r = c + 1; r < n; ++r)
        if (std::fabs(M[(size_t)r * n + c]) > std::fabs(M[(size_t)p * n + c])) p = r;
      if (M[(size_t)p * n + c] == 0.0) return 2;
      if (p != c)
        for (int j = 0; j < n; ++j) {
          std::swap(M[(size_t)p * n + j], M[(size_t)c * n + j]);
          std::swap(Sinv[(size_t)p * n + j], Sinv[(size_t)c * n + j]);
        }
      const double inv = 1.0 / M[(size_t)c * n + c];
      for (int j = 0; j < n; ++j) {
        M[(size_t)c * n + j] *= inv;
        Sinv[(size_t)c * n + j] *= inv;
      }
      for (int r = 0; r < n; ++r) {
        if (r == c) continue;
        const double f = M[(size_t)r * n + c];
        if (f == 0.0) continue;
        for (int j = 0; j < n; ++j) {
          M[(size_t)r * n + j] -= f * M[(size_t)c * n + j];
          Sinv[(size_t)r * n + j] -= f * Sinv[(size_t)c * n + j];
        }
      }
    }
  }
  return 0;
}

}  // namespace tps

// ---------------------------------------------------------------------------------------
// The k eigenvalues of smallest real part of a small real non-symmetric matrix and their
// eigenvectors, for the Rayleigh-Ritz step of the non-symmetric eigensolver (the projected
// matrix of the Sec. 3.1 discretisation, whose Ritz values may form complex pairs among
// the unwanted ones).  Complex arithmetic throughout (Golub & Van Loan, ch. 7): Hessenberg
// reduction by Householder reflections, single-shift QR steps with Wilkinson shifts and
// deflation to the complex Schur form T = Q^H A Q, eigenvectors of T by back substitution,
// S = Q X.  Each returned vector is the real part of the eigenvector after the phase that
// makes its largest entry real, with unit 2-norm; imag_max receives the largest |Im lambda|
// among the returned eigenvalues (zero for a real spectrum, up to rounding).
namespace tps {

int complex_eig_lowest(int n, const double *A, int k, double *lam, double *Y, int ldy,
                       double *imag_max) {
  using cd = std::complex<double>;
  if (n < 1 || k < 1 || k > n) return 1;
  const size_t nn = (size_t)n * n;
  std::vector<cd> H(nn), Q(nn, cd(0.0, 0.0)), v(n);
  for (size_t e = 0; e < nn; ++e) H[e] = cd(A[e], 0.0);
  auto h = [&](int i, int j) -> cd & { return H[(size_t)i * n + j]; };
  auto q = [&](int i, int j) -> cd & { return Q[(size_t)i * n + j]; };
  for (int i = 0; i < n; ++i) q(i, i) = cd(1.0, 0.0);
  double anorm = 0.0;
  for (size_t e = 0; e < nn; ++e) anorm = std::max(anorm, std::abs(H[e]));
  if (anorm == 0.0) anorm = 1.0;
  // Householder reduction to Hessenberg form (real input: the reflections are real)
  for (int c = 0; c + 2 < n; ++c) {
    double xnorm = 0.0;
    for (int i = c + 1; i < n; ++i) xnorm += std::norm(h(i, c));
    xnorm = std::sqrt(xnorm);
    if (xnorm == 0.0) continue;
    const cd x0 = h(c + 1, c);
    const cd alpha = (std::abs(x0) > 0.0 ? -x0 / std::abs(x0) : cd(-1.0, 0.0)) * xnorm;
    std::fill(v.begin(), v.end(), cd(0.0, 0.0));
    for (int i = c + 1; i < n; ++i) v[i] = h(i, c);
    v[c + 1] -= alpha;
    double vv = 0.0;
    for (int i = c + 1; i < n; ++i) vv += std::norm(v[i]);
    if (vv == 0.0) continue;
    const double beta = 2.0 / vv;
    for (int j = 0; j < n; ++j) {  // H <- (I - beta v v^H) H
      cd s(0.0, 0.0);
      for (int i = c + 1; i < n; ++i) s += std::conj(v[i]) * h(i, j);
      s *= beta;
      for (int i = c + 1; i < n; ++i) h(i, j) -= s * v[i];
    }
    for (int i = 0; i < n; ++i) {  // H <- H (I - beta v v^H), Q likewise
      cd s(0.0, 0.0), t(0.0, 0.0);
      for (int j = c + 1; j < n; ++j) {
        s += h(i, j) * v[j];
        t += q(i, j) * v[j];
      }
      s *= beta;
      t *= beta;
      for (int j = c + 1; j < n; ++j) {
        h(i, j) -= s * std::conj(v[j]);
        q(i, j) -= t * std::conj(v[j]);
      }
    }
    for (int i = c + 2; i < n; ++i) h(i, c) = cd(0.0, 0.0);
  }
  // single-shift QR on the active window until every subdiagonal is negligible
  constexpr double eps = 2.220446049250313e-16;
  int hi = n - 1, iter = 0;
  std::vector<cd> cs(n), sn(n);
  while (hi > 0) {
    int l = hi;
    while (l > 0) {
      double s = std::abs(h(l - 1, l - 1)) + std::abs(h(l, l));
      if (s == 0.0) s = anorm;
      if (std::abs(h(l, l - 1)) <= eps * s) {
        h(l, l - 1) = cd(0.0, 0.0);
        break;
      }
      --l;
    }
    if (l == hi) {
      --hi;
      iter = 0;
      continue;
    }
    if (++iter > 300) return 1;
    const cd a = h(hi - 1, hi - 1), b = h(hi - 1, hi), c = h(hi, hi - 1), d = h(hi, hi);
    const cd tr = 0.5 * (a + d), disc = std::sqrt(0.25 * (a - d) * (a - d) + b * c);
    const cd m1 = tr + disc, m2 = tr - disc;
    cd mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
    if (iter % 20 == 19) mu = d + std::abs(c);  // exceptional shift
    for (int i = l; i <= hi; ++i) h(i, i) -= mu;
    for (int i = l; i < hi; ++i) {  // complex Givens G_i zeroes h(i+1, i)
      const cd x = h(i, i), y = h(i + 1, i);
      const double r = std::sqrt(std::norm(x) + std::norm(y));
      cd cc(1.0, 0.0), ss(0.0, 0.0);
      if (r > 0.0) {
        cc = x / r;
        ss = y / r;
      }
      cs[i] = cc;
      sn[i] = ss;
      for (int j = i; j < n; ++j) {  // rows i, i+1 <- [c^* s^*; -s c] rows
        const cd u = h(i, j), w = h(i + 1, j);
        h(i, j) = std::conj(cc) * u + std::conj(ss) * w;
        h(i + 1, j) = -ss * u + cc * w;
      }
    }
    for (int i = l; i < hi; ++i) {  // columns i, i+1 <- cols [c s^*... ] (the adjoint)
      const cd cc = cs[i], ss = sn[i];
      const int top = std::min(i + 1, hi);
      for (int r = 0; r <= top; ++r) {
        const cd u = h(r, i), w = h(r, i + 1);
        h(r, i) = u * cc + w * ss;
        h(r, i + 1) = -u * std::conj(ss) + w * std::conj(cc);
      }
      for (int r = 0; r < n; ++r) {
        const cd u = q(r, i), w = q(r, i + 1);
        q(r, i) = u * cc + w * ss;
        q(r, i + 1) = -u * std::conj(ss) + w * std::conj(cc);
      }
    }
    for (int i = l; i <= hi; ++i) h(i, i) += mu;
  }
  // the k eigenvalues of smallest real part
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return h(x, x).real() < h(y, y).real(); });
  double im = 0.0;
  const double tiny = eps * anorm;
  std::vector<cd> x(n), s(n);
  for (int c = 0; c < k; ++c) {
    const int kk = order[c];
    const cd ev = h(kk, kk);
    lam[c] = ev.real();
    im = std::max(im, std::abs(ev.imag()));
    // back substitution: (T - ev) x = 0 with x_kk = 1, x_j = 0 for j > kk
    std::fill(x.begin(), x.end(), cd(0.0, 0.0));
    x[kk] = cd(1.0, 0.0);
    for (int j = kk - 1; j >= 0; --j) {
      cd acc(0.0, 0.0);
      for (int m = j + 1; m <= kk; ++m) acc += h(j, m) * x[m];
      cd den = h(j, j) - ev;
      if (std::abs(den) < tiny) den = cd(tiny, 0.0);
      x[j] = -acc / den;
    }
    for (int i = 0; i < n; ++i) {
      cd t(0.0, 0.0);
      for (int m = 0; m <= kk; ++m) t += q(i, m) * x[m];
      s[i] = t;
    }
    int imax = 0;
    for (int i = 1; i < n; ++i)
      if (std::abs(s[i]) > std::abs(s[imax])) imax = i;
    const cd ph = std::abs(s[imax]) > 0.0 ? std::conj(s[imax]) / std::abs(s[imax]) : cd(1.0, 0.0);
    double nrm = 0.0;
    for (int i = 0; i < n; ++i) {
      const double re = (s[i] * ph).real();
      Y[(size_t)c * ldy + i] = re;
      nrm += re * re;
    }
    nrm = nrm > 0.0 ? 1.0 / std::sqrt(nrm) : 0.0;
    for (int i = 0; i < n; ++i) Y[(size_t)c * ldy + i] *= nrm;
  }
  if (imag_max) *imag_max = im;
  return 0;
}

}  // namespace tps
