// Test harness (compiled by tests/test_dense_host.py with the host C++ compiler): plain C entry
// points over the library's host dense routines, so the CPU tests can compare them with numpy and
// scipy.  Matrices are column-major interleaved complex doubles.
#include <complex>
#include <cstring>
#include <vector>

#include "dense.h"

using dense::Mat;
using dense::cd;

static Mat load(const double *a, int r, int c) {
  Mat m(r, c);
  std::memcpy(m.a.data(), a, sizeof(cd) * (size_t)r * c);
  return m;
}
static void store(const Mat &m, double *out) { std::memcpy(out, m.a.data(), sizeof(cd) * m.a.size()); }

extern "C" {

int shim_lstsq(const double *A, int r, int c, const double *b, double *x) {
  std::vector<cd> cv(r);
  std::memcpy(cv.data(), b, sizeof(cd) * r);
  std::vector<cd> d = dense::lstsq(load(A, r, c), cv);
  std::memcpy(x, d.data(), sizeof(cd) * c);
  return 0;
}

int shim_solve(const double *A, int n, const double *b, double *x) {
  std::vector<cd> bv(n), xv;
  std::memcpy(bv.data(), b, sizeof(cd) * n);
  if (!dense::solve(load(A, n, n), bv, xv)) return 1;
  std::memcpy(x, xv.data(), sizeof(cd) * n);
  return 0;
}

int shim_schur(const double *A, int n, double *T, double *Z) {
  Mat t, z;
  if (!dense::schur(load(A, n, n), t, z)) return 1;
  store(t, T);
  store(z, Z);
  return 0;
}

int shim_eig(const double *A, int n, double *w, double *X) {
  std::vector<cd> wv;
  Mat x;
  if (!dense::eig(load(A, n, n), wv, x)) return 1;
  std::memcpy(w, wv.data(), sizeof(cd) * n);
  store(x, X);
  return 0;
}

int shim_eigh(const double *A, int n, double *w, double *X) {
  std::vector<double> wv;
  Mat x;
  if (!dense::eigh(load(A, n, n), wv, x)) return 1;
  std::memcpy(w, wv.data(), sizeof(double) * n);
  store(x, X);
  return 0;
}

int shim_eigh_gen(const double *A, const double *B, int n, double *mu, double *G) {
  std::vector<double> m;
  Mat g;
  if (!dense::eigh_gen(load(A, n, n), load(B, n, n), m, g)) return 1;
  std::memcpy(mu, m.data(), sizeof(double) * n);
  store(g, G);
  return 0;
}

int shim_orthonormalize(const double *A, int r, int c, double *Q) {
  store(dense::orthonormalize(load(A, r, c)), Q);
  return 0;
}

}  // extern "C"
