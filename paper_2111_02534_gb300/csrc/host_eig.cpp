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
