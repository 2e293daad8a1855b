// Host dense complex linear algebra used by the Krylov drivers (see dense.h).
#include "dense.h"

#include <algorithm>
#include <cmath>
#include <limits>

namespace dense {

static const double EPS = std::numeric_limits<double>::epsilon();

Mat matmul(const Mat &A, const Mat &B) {
  Mat C(A.r, B.c);
  for (int j = 0; j < B.c; ++j)
    for (int k = 0; k < A.c; ++k) {
      const cd b = B(k, j);
      if (b == cd(0.0, 0.0)) continue;
      for (int i = 0; i < A.r; ++i) C(i, j) += A(i, k) * b;
    }
  return C;
}

Mat adjoint(const Mat &A) {
  Mat B(A.c, A.r);
  for (int i = 0; i < A.r; ++i)
    for (int j = 0; j < A.c; ++j) B(j, i) = std::conj(A(i, j));
  return B;
}

// Householder vector for column x: returns v (v[0] real-normalised form) and beta such that
// (I - beta v v^H) x = alpha e_1.
static void householder(std::vector<cd> &x, cd &alpha, double &beta) {
  double nrm = 0.0;
  for (const cd &v : x) nrm += std::norm(v);
  nrm = std::sqrt(nrm);
  if (nrm == 0.0) {
    alpha = 0.0;
    beta = 0.0;
    return;
  }
  const double ax0 = std::abs(x[0]);
  const cd ph = ax0 > 0.0 ? x[0] / ax0 : cd(1.0, 0.0);
  alpha = -ph * nrm;
  x[0] -= alpha;
  double vn = 0.0;
  for (const cd &v : x) vn += std::norm(v);
  beta = vn > 0.0 ? 2.0 / vn : 0.0;
}

QRFact qr_factor(const Mat &A0) {
  QRFact f;
  f.a = A0;
  Mat &A = f.a;
  const int m = A.r, n = A.c;
  f.v.resize(n);
  f.beta.assign(n, 0.0);
  for (int k = 0; k < n; ++k) {
    std::vector<cd> &v = f.v[k];
    v.resize(m - k);
    for (int i = k; i < m; ++i) v[i - k] = A(i, k);
    cd alpha;
    double beta;
    householder(v, alpha, beta);
    f.beta[k] = beta;
    if (beta == 0.0) continue;
    for (int j = k; j < n; ++j) {
      cd s = 0.0;
      for (int i = k; i < m; ++i) s += std::conj(v[i - k]) * A(i, j);
      s *= beta;
      for (int i = k; i < m; ++i) A(i, j) -= s * v[i - k];
    }
  }
  return f;
}

std::vector<cd> qr_solve(const QRFact &f, const std::vector<cd> &c0) {
  const Mat &A = f.a;
  const int m = A.r, n = A.c;
  std::vector<cd> c = c0;
  for (int k = 0; k < n; ++k) {
    const double beta = f.beta[k];
    if (beta == 0.0) continue;
    const std::vector<cd> &v = f.v[k];
    cd s = 0.0;
    for (int i = k; i < m; ++i) s += std::conj(v[i - k]) * c[i];
    s *= beta;
    for (int i = k; i < m; ++i) c[i] -= s * v[i - k];
  }
  std::vector<cd> d(n);
  for (int i = n - 1; i >= 0; --i) {
    cd s = c[i];
    for (int j = i + 1; j < n; ++j) s -= A(i, j) * d[j];
    d[i] = (A(i, i) != cd(0.0, 0.0)) ? s / A(i, i) : cd(0.0, 0.0);
  }
  return d;
}

std::vector<cd> lstsq(const Mat &A0, const std::vector<cd> &c0) { return qr_solve(qr_factor(A0), c0); }

bool solve(const Mat &A0, const std::vector<cd> &b, std::vector<cd> &x) {
  Mat A = A0;
  const int n = A.r;
  x = b;
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::abs(A(k, k));
    for (int i = k + 1; i < n; ++i)
      if (std::abs(A(i, k)) > best) { best = std::abs(A(i, k)); p = i; }
    if (best == 0.0) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A(k, j), A(p, j));
      std::swap(x[k], x[p]);
    }
    for (int i = k + 1; i < n; ++i) {
      const cd f = A(i, k) / A(k, k);
      A(i, k) = f;
      for (int j = k + 1; j < n; ++j) A(i, j) -= f * A(k, j);
      x[i] -= f * x[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    cd s = x[i];
    for (int j = i + 1; j < n; ++j) s -= A(i, j) * x[j];
    x[i] = s / A(i, i);
  }
  return true;
}

// unitary G = [[c, s], [-conj(s), c]] with G [x; y] = [r; 0]
static void givens(cd x, cd y, double &c, cd &s) {
  const double ax = std::abs(x), ay = std::abs(y);
  if (ay == 0.0) { c = 1.0; s = 0.0; return; }
  if (ax == 0.0) { c = 0.0; s = 1.0; return; }
  const double rho = std::hypot(ax, ay);
  c = ax / rho;
  s = (x / ax) * std::conj(y) / rho;
}

bool schur(const Mat &A, Mat &T, Mat &Z) {
  const int n = A.r;
  T = A;
  Z = Mat(n, n);
  for (int i = 0; i < n; ++i) Z(i, i) = 1.0;
  // Hessenberg reduction by Householder similarity transforms
  for (int k = 0; k + 2 < n; ++k) {
    std::vector<cd> v(n - k - 1);
    for (int i = k + 1; i < n; ++i) v[i - k - 1] = T(i, k);
    cd alpha;
    double beta;
    householder(v, alpha, beta);
    if (beta == 0.0) continue;
    for (int j = 0; j < n; ++j) {  // rows k+1.. : T = H T
      cd s = 0.0;
      for (int i = k + 1; i < n; ++i) s += std::conj(v[i - k - 1]) * T(i, j);
      s *= beta;
      for (int i = k + 1; i < n; ++i) T(i, j) -= s * v[i - k - 1];
    }
    for (int i = 0; i < n; ++i) {  // columns k+1.. : T = T H, Z = Z H
      cd s = 0.0, sz = 0.0;
      for (int j = k + 1; j < n; ++j) {
        s += T(i, j) * v[j - k - 1];
        sz += Z(i, j) * v[j - k - 1];
      }
      s *= beta;
      sz *= beta;
      for (int j = k + 1; j < n; ++j) {
        T(i, j) -= s * std::conj(v[j - k - 1]);
        Z(i, j) -= sz * std::conj(v[j - k - 1]);
      }
    }
    for (int i = k + 2; i < n; ++i) T(i, k) = 0.0;
  }
  double anorm = 0.0;
  for (const cd &v : T.a) anorm = std::max(anorm, std::abs(v));
  if (anorm == 0.0) return true;
  int hi = n - 1;
  int iter = 0, total = 0;
  while (hi > 0) {
    int l = hi;
    while (l > 0) {
      const double sd = std::abs(T(l, l - 1));
      const double dd = std::abs(T(l - 1, l - 1)) + std::abs(T(l, l));
      if (sd <= EPS * (dd > 0.0 ? dd : anorm)) { T(l, l - 1) = 0.0; break; }
      --l;
    }
    if (l == hi) { --hi; iter = 0; continue; }
    if (++iter > 60 || ++total > 100 * n) return false;
    // Wilkinson shift from the trailing 2x2 block (exceptional shifts every tenth step)
    cd mu;
    if (iter % 10 == 0) {
      mu = T(hi, hi) + std::abs(T(hi, hi - 1)) * 0.75;
    } else {
      const cd a = T(hi - 1, hi - 1), b = T(hi - 1, hi), c = T(hi, hi - 1), d = T(hi, hi);
      const cd half = 0.5 * (a - d);
      const cd disc = std::sqrt(half * half + b * c);
      const cd m1 = 0.5 * (a + d) + disc, m2 = 0.5 * (a + d) - disc;
      mu = (std::abs(m1 - d) < std::abs(m2 - d)) ? m1 : m2;
    }
    // implicit single-shift QR sweep on rows/columns l..hi (full Schur form kept)
    for (int k = l; k < hi; ++k) {
      cd x, y;
      if (k == l) { x = T(l, l) - mu; y = T(l + 1, l); }
      else { x = T(k, k - 1); y = T(k + 1, k - 1); }
      double c;
      cd s;
      givens(x, y, c, s);
      const int j0 = (k == l) ? l : k - 1;
      for (int j = j0; j < n; ++j) {
        const cd t1 = T(k, j), t2 = T(k + 1, j);
        T(k, j) = c * t1 + s * t2;
        T(k + 1, j) = -std::conj(s) * t1 + c * t2;
      }
      if (k > l) T(k + 1, k - 1) = 0.0;
      const int i1 = std::min(k + 2, hi);
      for (int i = 0; i <= i1; ++i) {
        const cd t1 = T(i, k), t2 = T(i, k + 1);
        T(i, k) = c * t1 + std::conj(s) * t2;
        T(i, k + 1) = -s * t1 + c * t2;
      }
      for (int i = 0; i < n; ++i) {
        const cd z1 = Z(i, k), z2 = Z(i, k + 1);
        Z(i, k) = c * z1 + std::conj(s) * z2;
        Z(i, k + 1) = -s * z1 + c * z2;
      }
    }
  }
  for (int j = 0; j < n; ++j)
    for (int i = j + 1; i < n; ++i) T(i, j) = 0.0;
  return true;
}

bool eig(const Mat &A, std::vector<cd> &w, Mat &X) {
  const int n = A.r;
  Mat T, Z;
  if (!schur(A, T, Z)) return false;
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = T(i, i);
  double tnorm = 0.0;
  for (const cd &v : T.a) tnorm = std::max(tnorm, std::abs(v));
  const double small = EPS * std::max(tnorm, 1e-300);
  Mat Y(n, n);
  for (int k = 0; k < n; ++k) {
    Y(k, k) = 1.0;
    for (int i = k - 1; i >= 0; --i) {
      cd s = 0.0;
      for (int j = i + 1; j <= k; ++j) s += T(i, j) * Y(j, k);
      cd den = T(i, i) - T(k, k);
      if (std::abs(den) < small) den = small;
      Y(i, k) = -s / den;
    }
  }
  X = matmul(Z, Y);
  for (int k = 0; k < n; ++k) {
    double nrm = 0.0;
    for (int i = 0; i < n; ++i) nrm += std::norm(X(i, k));
    nrm = std::sqrt(nrm);
    if (nrm > 0.0)
      for (int i = 0; i < n; ++i) X(i, k) /= nrm;
  }
  return true;
}

bool eigh(const Mat &A0, std::vector<double> &w, Mat &X) {
  const int n = A0.r;
  Mat A(n, n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) A(i, j) = 0.5 * (A0(i, j) + std::conj(A0(j, i)));
  Mat T, Z;
  if (!schur(A, T, Z)) return false;
  // a Hermitian matrix has a diagonal Schur form: Z holds orthonormal eigenvectors
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return T(a, a).real() < T(b, b).real(); });
  w.resize(n);
  X = Mat(n, n);
  for (int k = 0; k < n; ++k) {
    w[k] = T(order[k], order[k]).real();
    for (int i = 0; i < n; ++i) X(i, k) = Z(i, order[k]);
  }
  return true;
}

bool eigh_gen(const Mat &A, const Mat &B, std::vector<double> &mu, Mat &G) {
  const int n = A.r;
  // Cholesky B = L L^H
  Mat L(n, n);
  for (int j = 0; j < n; ++j) {
    double d = B(j, j).real();
    for (int k = 0; k < j; ++k) d -= std::norm(L(j, k));
    if (d <= 0.0) return false;
    L(j, j) = std::sqrt(d);
    for (int i = j + 1; i < n; ++i) {
      cd s = B(i, j);
      for (int k = 0; k < j; ++k) s -= L(i, k) * std::conj(L(j, k));
      L(i, j) = s / L(j, j);
    }
  }
  // C = L^{-1} A L^{-H}: first W = L^{-1} A, then C = L^{-1} W^H (A Hermitian)
  Mat W(n, n);
  for (int col = 0; col < n; ++col)
    for (int i = 0; i < n; ++i) {
      cd s = A(i, col);
      for (int k = 0; k < i; ++k) s -= L(i, k) * W(k, col);
      W(i, col) = s / L(i, i);
    }
  Mat Wh = adjoint(W);
  Mat C(n, n);
  for (int col = 0; col < n; ++col)
    for (int i = 0; i < n; ++i) {
      cd s = Wh(i, col);
      for (int k = 0; k < i; ++k) s -= L(i, k) * C(k, col);
      C(i, col) = s / L(i, i);
    }
  Mat Y;
  if (!eigh(C, mu, Y)) return false;
  // G = L^{-H} Y
  G = Mat(n, n);
  for (int col = 0; col < n; ++col)
    for (int i = n - 1; i >= 0; --i) {
      cd s = Y(i, col);
      for (int k = i + 1; k < n; ++k) s -= std::conj(L(k, i)) * G(k, col);
      G(i, col) = s / L(i, i);
    }
  return true;
}

Mat orthonormalize(const Mat &A) {
  Mat Q = A;
  for (int j = 0; j < Q.c; ++j) {
    for (int pass = 0; pass < 2; ++pass) {
      std::vector<cd> h(j, 0.0);
      for (int p = 0; p < j; ++p)
        for (int i = 0; i < Q.r; ++i) h[p] += std::conj(Q(i, p)) * Q(i, j);
      for (int p = 0; p < j; ++p)
        for (int i = 0; i < Q.r; ++i) Q(i, j) -= h[p] * Q(i, p);
    }
    double nrm = 0.0;
    for (int i = 0; i < Q.r; ++i) nrm += std::norm(Q(i, j));
    nrm = std::sqrt(nrm);
    for (int i = 0; i < Q.r; ++i) Q(i, j) = nrm > 0.0 ? Q(i, j) / nrm : cd(0.0, 0.0);
  }
  return Q;
}

}  // namespace dense
