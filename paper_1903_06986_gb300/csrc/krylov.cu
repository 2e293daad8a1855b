// GMRES-DR(m, k), its Hermitian form (MINRES-DR) and GMRES-Proj on the GPU (Sec. 5.3, 7, 8).
//
// Every right-hand side of a block has its own Krylov basis; all of them advance together, so
// each Arnoldi step is one multi-RHS Wilson launch plus batched classical Gram-Schmidt (applied
// twice) and a batched norm, all without a host round trip.  At the end of a cycle the Hessenberg
// coefficients come back to the host, where the small FP64 problems are solved per right-hand
// side (least squares, harmonic Ritz values, the restart basis P_{k+1}); the restart
// V_{k+1} <- V_{m+1} P_{k+1} and the solution update x += V_m d run on the GPU.
//
// GMRES-DR cycle (Morgan's algorithm, as used in Sec. 7):
//   Arnoldi from column j0 to m;  d = argmin ||c - Hbar d||;  x += V_m d;  s = c - Hbar d;
//   harmonic Ritz (H_m + |h_{m+1,m}|^2 H_m^{-H} e_m e_m^T) g = theta g, k smallest |theta|;
//   P_{k+1} = orthonormal [g_1..g_k (zero-padded), s];  V <- V P;  Hbar <- P^H Hbar P_k;
//   c <- P^H s;  j0 = k.
// Hermitian form (MINRES-DR, Sec. 8): minimum residual over the same spaces of the Hermitian
// M' = M gamma_5; the harmonic Ritz values are real (rounding-level imaginary parts dropped) and the
// final Rayleigh-Ritz problem is Hermitian, giving orthonormal eigenvectors and real eigenvalues.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <memory>
#include <type_traits>

#include "common.cuh"
#include "dense.h"

using dense::cd;
using dense::Mat;

namespace {

constexpr int OP_MASKED = 4;

// Polynomial right preconditioner of a solve (the Min-Res polynomial of Sec. 5.2 used inside the
// solver): the Krylov methods work on B = A p(A), p(A) = sum_j a_j A^j, and x = p(A) y.  degree 0:
// none.  t1, t2: two scratch blocks of the solve's right-hand sides (reserved before use, so that
// graph capture never allocates).
constexpr int MAX_POLY = 32;
struct Poly {
  int degree = 0;
  double2 a[MAX_POLY + 1] = {};
  void *t1 = nullptr, *t2 = nullptr;
  void append_key(std::string &k) const {
    key_add(k, degree);
    for (int j = 0; j <= degree && degree > 0; ++j) key_add(k, a[j]);
    key_add(k, t1);
    key_add(k, t2);
  }
};

// out = [A] p(A) in by Horner's rule with the operator's plain application (times_A: B = A p(A),
// d + 1 applications; else p(A) alone, d applications).  in and out must not overlap t1 / t2.
template <typename S, typename OP>
lqcd_status poly_apply_op(lqcd_ctx *ctx, const OP &op, const Poly &pp, const S *in, S *out, int nrhs, bool times_A) {
  const long long n = (long long)nrhs * ctx->N;
  const int d = pp.degree;
  S *t = (S *)pp.t1, *u = (S *)pp.t2;
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  LQCD_TRY(blas_zero(ctx, t, n));
  LQCD_TRY(blas_axpby(ctx, pp.a[d], in, zero, t, n));
  for (int j = d - 1; j >= 0; --j) {
    LQCD_TRY(op.apply_base(ctx, t, u, nrhs));
    LQCD_TRY(blas_axpby(ctx, pp.a[j], in, one, u, n));
    std::swap(t, u);
  }
  if (times_A) return op.apply_base(ctx, t, out, nrhs);
  return blas_copy(ctx, (const S *)t, out, n);
}

// The operator of a solve: M or M gamma_5 (flags LQCD_APPLY_M / LQCD_APPLY_G5R) on FP64 storage
// (arithmetic prec) or on FP32 storage with FP32 arithmetic (the inner solver of mixed precision),
// times p(A) when a polynomial preconditioner is set.
template <typename S, typename Derived> struct PolyApply {
  lqcd_status apply(lqcd_ctx *ctx, const S *in, S *out, int nrhs) const {
    const Derived &d = static_cast<const Derived &>(*this);
    if (d.pp.degree == 0) return d.apply_base(ctx, in, out, nrhs);
    return poly_apply_op<S>(ctx, d, d.pp, in, out, nrhs, true);
  }
  // out = p(A) in (the solution x = p(A) y of a preconditioned solve); a plain copy without p
  lqcd_status apply_poly(lqcd_ctx *ctx, const S *in, S *out, int nrhs) const {
    const Derived &d = static_cast<const Derived &>(*this);
    if (d.pp.degree == 0) return blas_copy(ctx, in, out, (long long)nrhs * ctx->N);
    return poly_apply_op<S>(ctx, d, d.pp, in, out, nrhs, false);
  }
  // reserve the scratch blocks of the polynomial for nrhs right-hand sides
  lqcd_status reserve(lqcd_ctx *ctx, int nrhs) {
    Derived &d = static_cast<Derived &>(*this);
    LQCD_TRY(eo_reserve(ctx, nrhs));
    if (d.pp.degree == 0) return LQCD_OK;
    const size_t bytes = sizeof(S) * (size_t)nrhs * ctx->N;
    LQCD_TRY(ws_get(ctx, WS_POLY1, bytes, &d.pp.t1));
    return ws_get(ctx, WS_POLY2, bytes, &d.pp.t2);
  }
};
template <typename S> struct OpT;
template <> struct OpT<double2> : PolyApply<double2, OpT<double2>> {
  const double2 *U;
  double kappa;
  int flags;                    // LQCD_APPLY_M, LQCD_APPLY_G5R, or OP_MASKED
  int prec;
  unsigned long long g5mask;    // OP_MASKED: right-hand side r uses M gamma_5 when bit r is set
  Poly pp;
  OpT() = default;
  OpT(const double2 *U_, double kappa_, int flags_, int prec_, unsigned long long g5mask_)
      : U(U_), kappa(kappa_), flags(flags_), prec(prec_), g5mask(g5mask_) {}
  lqcd_status apply_base(lqcd_ctx *ctx, const double2 *in, double2 *out, int nrhs) const {
    if (flags == OP_MASKED) return wilson_launch_masked(ctx, U, kappa, in, out, nrhs, g5mask);
    return wilson_launch(ctx, U, kappa, in, out, nrhs, prec, flags);
  }
  void append_key(std::string &k) const {
    key_add(k, U);
    key_add(k, kappa);
    key_add(k, flags);
    key_add(k, prec);
    key_add(k, g5mask);
    pp.append_key(k);
  }
};
// FP32 fields of the inner solver are in the packed layout (see wilson.cu); the level-1/2 kernels
// treat them as plain float2 arrays of the same length, which is all they need.
template <> struct OpT<float2> : PolyApply<float2, OpT<float2>> {
  const float4 *U;  // packed links
  int recon;
  double kappa;
  int flags;
  Poly pp;
  lqcd_status apply_base(lqcd_ctx *ctx, const float2 *in, float2 *out, int nrhs) const {
    return wilson_launch_packed(ctx, U, recon, kappa, (const float4 *)in, (float4 *)out, nrhs, flags, ctx->packed_nr);
  }
  void append_key(std::string &k) const {
    key_add(k, U);
    key_add(k, recon);
    key_add(k, kappa);
    key_add(k, flags);
    pp.append_key(k);
  }
};
// FP16 / BF16 fields of the inner solver: the same packed operator on reduced-precision storage
template <typename S> struct OpLP : PolyApply<S, OpLP<S>> {
  const float4 *U;
  int recon;
  double kappa;
  int flags;
  Poly pp;
  lqcd_status apply_base(lqcd_ctx *ctx, const S *in, S *out, int nrhs) const {
    return wilson_launch_packed_lp<S>(ctx, U, recon, kappa, in, out, nrhs, flags);
  }
  void append_key(std::string &k) const {
    key_add(k, U);
    key_add(k, recon);
    key_add(k, kappa);
    key_add(k, flags);
    pp.append_key(k);
  }
};
template <> struct OpT<__half2> : OpLP<__half2> {};
template <> struct OpT<__nv_bfloat162> : OpLP<__nv_bfloat162> {};
using Op = OpT<double2>;

lqcd_status apply_op(lqcd_ctx *ctx, const Op &op, const double2 *in, double2 *out, int nrhs) {
  return op.apply(ctx, in, out, nrhs);
}

// Host -> device copy of small coefficient arrays.  From pageable memory cudaMemcpyAsync stages the
// source before it returns and does not wait for earlier work in the stream, so the host vector
// may be released immediately and the GPU keeps running.
lqcd_status upload(lqcd_ctx *ctx, const std::vector<cd> &h, void *dev) {
  if (h.empty()) return LQCD_OK;
  LQCD_CUDA(ctx, cudaMemcpyAsync(dev, h.data(), sizeof(cd) * h.size(), cudaMemcpyHostToDevice, ctx->stream));
  return LQCD_OK;
}

// Device -> host copy through the pinned staging buffer; waits for the stream.
template <typename T>
lqcd_status download(lqcd_ctx *ctx, const void *dev, std::vector<T> &h, size_t count) {
  h.resize(count);
  if (count == 0) return LQCD_OK;
  double *st = nullptr;
  LQCD_TRY(host_stage(ctx, sizeof(T) * count, &st));
  LQCD_CUDA(ctx, cudaMemcpyAsync(st, dev, sizeof(T) * count, cudaMemcpyDeviceToHost, ctx->stream));
  LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  memcpy(h.data(), st, sizeof(T) * count);
  return LQCD_OK;
}

bool finite(cd v) { return std::isfinite(v.real()) && std::isfinite(v.imag()); }

// Per right-hand side host state of a cycle
struct Rhs {
  Mat H;                 // (m+1) x m
  std::vector<cd> c;     // m+1
  bool active = true;
  double bnorm = 0.0;
  double rel = 0.0;
  double eres = 0.0;     // largest Rayleigh-Ritz residual of the restart space (when tracked)
};

// Enqueue Arnoldi steps j0..m-1 for every right-hand side (basis Vb with vector stride vs =
// nrhs * N) and fill columns j0..m-1 of each Rhs::H.  Inactive right-hand sides are processed
// too (their results are ignored).
template <typename S> struct ArnoldiT {
  lqcd_ctx *ctx;
  OpT<S> op;
  int nrhs, m;
  long long N;
  S *Vb;
  double2 *hd1, *hd2;  // [j][i][r] device, (m) x (m+1) x nrhs
  double *nrm;         // [j][r]
  int passes = 2;      // Gram-Schmidt passes per step: 2 (CGS2), or 1 (CGS) for reduced-precision bases
  int window = 0;      // > 0 (Hermitian operators only): orthogonalise against the last `window` vectors
};

// First basis vector step j is orthogonalised against: all of them, or the last a.window (for a
// Hermitian operator the Arnoldi recurrence is the three-term Lanczos one, h_ij = 0 for i < j - 1,
// so a window of 2 drops only terms that vanish in exact arithmetic)
template <typename S> inline int gs_first(const ArnoldiT<S> &a, int j) {
  return a.window > 0 ? std::max(0, j + 1 - a.window) : 0;
}
using Arnoldi = ArnoldiT<double2>;

// The launches of Arnoldi steps j0..m-1 (CGS2: two passes of inner products and updates, or one
// pass when a.passes == 1, then the norm and the normalisation), nothing else: no synchronisation,
// so the sequence can be captured.
template <typename S> struct ArnoldiLaunch {
  ArnoldiT<S> *a;
  int j0;
};
template <typename S>
lqcd_status arnoldi_enqueue(void *arg) {
  ArnoldiT<S> &a = *((ArnoldiLaunch<S> *)arg)->a;
  const int j0 = ((ArnoldiLaunch<S> *)arg)->j0;
  lqcd_ctx *ctx = a.ctx;
  const long long N = a.N, vs = (long long)a.nrhs * N;
  for (int j = j0; j < a.m; ++j) {
    S *vj = a.Vb + j * vs, *w = a.Vb + (j + 1) * vs;
    LQCD_TRY(a.op.apply(ctx, vj, w, a.nrhs));
    double2 *h1 = a.hd1 + (long long)j * (a.m + 1) * a.nrhs;
    double2 *h2 = a.hd2 + (long long)j * (a.m + 1) * a.nrhs;
    const int lo = gs_first(a, j);
    const S *vlo = a.Vb + lo * vs;
    LQCD_TRY(blas_multidot(ctx, vlo, vs, N, j + 1 - lo, w, N, a.nrhs, h1 + (long long)lo * a.nrhs));
    LQCD_TRY(blas_multiaxpy(ctx, vlo, vs, N, j + 1 - lo, h1 + (long long)lo * a.nrhs, -1.0, w, N, a.nrhs));
    if (a.passes > 1) {
      LQCD_TRY(blas_multidot(ctx, vlo, vs, N, j + 1 - lo, w, N, a.nrhs, h2 + (long long)lo * a.nrhs));
      LQCD_TRY(blas_multiaxpy(ctx, vlo, vs, N, j + 1 - lo, h2 + (long long)lo * a.nrhs, -1.0, w, N, a.nrhs));
    }
    LQCD_TRY(blas_norms(ctx, w, N, a.nrhs, a.nrm + (long long)j * a.nrhs));
    LQCD_TRY(blas_invscale(ctx, w, a.nrm + (long long)j * a.nrhs, N, a.nrhs));
  }
  return LQCD_OK;
}

// Enqueue the steps, through a cached CUDA graph of the whole sequence when graphs are enabled:
// the key holds every pointer and parameter the launches bake in.
template <typename S>
lqcd_status arnoldi_launch(ArnoldiT<S> &a, int j0) {
  if (j0 >= a.m) return LQCD_OK;
  LQCD_TRY(blas_reserve(a.ctx, a.N, a.nrhs, a.m));
  LQCD_TRY(a.op.reserve(a.ctx, a.nrhs));
  std::string key("arnoldi");
  key_add(key, StoreTag<S>::value);
  a.op.append_key(key);
  key_add(key, a.nrhs);
  key_add(key, a.m);
  key_add(key, a.N);
  key_add(key, a.Vb);
  key_add(key, a.hd1);
  key_add(key, a.hd2);
  key_add(key, a.nrm);
  key_add(key, j0);
  key_add(key, a.passes);
  key_add(key, a.window);
  key_add(key, a.ctx->packed_nr);
  ArnoldiLaunch<S> arg{&a, j0};
  return graph_cached(a.ctx, key, &arnoldi_enqueue<S>, &arg);
}

template <typename S>
lqcd_status arnoldi_run(ArnoldiT<S> &a, int j0, std::vector<Rhs> &R, long long &matvecs) {
  lqcd_ctx *ctx = a.ctx;
  LQCD_TRY(arnoldi_launch(a, j0));
  for (int r = 0; r < a.nrhs; ++r)
    if (R[r].active) matvecs += a.m - j0;
  if (j0 >= a.m) return LQCD_OK;
  const size_t hcount = (size_t)a.m * (a.m + 1) * a.nrhs;
  std::vector<double2> h1, h2;
  std::vector<double> nr;
  LQCD_TRY(download(ctx, a.hd1, h1, hcount));
  if (a.passes > 1) {
    LQCD_TRY(download(ctx, a.hd2, h2, hcount));
  } else {
    h2.assign(hcount, make_double2(0.0, 0.0));
  }
  LQCD_TRY(download(ctx, a.nrm, nr, (size_t)a.m * a.nrhs));
  for (int r = 0; r < a.nrhs; ++r) {
    if (!R[r].active) continue;
    for (int j = j0; j < a.m; ++j) {
      const int lo = gs_first(a, j);
      for (int i = 0; i < lo; ++i) R[r].H(i, j) = cd(0.0, 0.0);
      for (int i = lo; i <= j; ++i) {
        const double2 x1 = h1[((size_t)j * (a.m + 1) + i) * a.nrhs + r];
        const double2 x2 = h2[((size_t)j * (a.m + 1) + i) * a.nrhs + r];
        R[r].H(i, j) = cd(x1.x + x2.x, x1.y + x2.y);
      }
      R[r].H(j + 1, j) = cd(nr[(size_t)j * a.nrhs + r], 0.0);
      for (int i = 0; i <= j + 1; ++i)
        if (!finite(R[r].H(i, j)))
          return set_err(ctx, LQCD_ERR_NONFINITE, "non-finite Hessenberg entry (rhs %d, column %d)", r, j);
    }
  }
  return LQCD_OK;
}

// Harmonic Ritz pairs of Hbar ((m+1) x m), k with smallest |theta| first
bool harmonic_ritz(const Mat &H, int k, bool hermitian, std::vector<cd> &theta, Mat &G) {
  const int m = H.c;
  Mat Hm(m, m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) Hm(i, j) = H(i, j);
  std::vector<int> order(m);
  std::vector<cd> th(m);
  Mat X;
  // the general form for both: the equivalent Hermitian-definite form with H_m symmetrised keeps the
  // restart relation only to the rounding asymmetry of H_m, and that error grows from cycle to cycle
  // on long runs; for Hermitian A the theta are real and their rounding-level imaginary parts dropped
  std::vector<cd> em(m, cd(0.0, 0.0)), f;
  em[m - 1] = 1.0;
  if (!dense::solve(dense::adjoint(Hm), em, f)) return false;
  const double h2 = std::norm(H(m, m - 1));
  Mat F = Hm;
  for (int i = 0; i < m; ++i) F(i, m - 1) += h2 * f[i];
  if (!dense::eig(F, th, X)) return false;
  if (hermitian)
    for (int i = 0; i < m; ++i) th[i] = cd(th[i].real(), 0.0);
  for (int i = 0; i < m; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return std::abs(th[a]) < std::abs(th[b]); });
  theta.resize(k);
  G = Mat(m, k);
  for (int q = 0; q < k; ++q) {
    theta[q] = th[order[q]];
    for (int i = 0; i < m; ++i) G(i, q) = X(i, order[q]);
  }
  return true;
}

// Unit vector spanning the orthogonal complement of range(Hbar) ((m+1) x m, H_m nonsingular):
// Hbar^H w = 0 gives w = [-conj(h_{m+1,m}) H_m^{-H} e_m; 1].  The least-squares residual s and every
// harmonic Ritz residual Hbar g - theta [g; 0] are parallel to it in exact arithmetic; once the
// system has converged s is rounding noise, so the restart uses w (keeping A V_k = V_{k+1} Hbar_k
// exact to rounding).  Falls back to s when H_m is singular.
std::vector<cd> lsq_complement(const Mat &H, const std::vector<cd> &s) {
  const int m = H.c;
  Mat Hm(m, m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) Hm(i, j) = H(i, j);
  std::vector<cd> em(m, cd(0.0, 0.0)), f;
  em[m - 1] = 1.0;
  if (!dense::solve(dense::adjoint(Hm), em, f)) return s;
  std::vector<cd> w(m + 1);
  const cd h = std::conj(H(m, m - 1));
  double nrm = 1.0;
  for (int i = 0; i < m; ++i) {
    w[i] = -h * f[i];
    nrm += std::norm(w[i]);
  }
  w[m] = 1.0;
  nrm = std::sqrt(nrm);
  if (!std::isfinite(nrm)) return s;
  for (cd &v : w) v /= nrm;
  return w;
}

// Largest Rayleigh-Ritz residual ||Hbar_k y - lambda [y; 0]|| of a deflation space's (k+1) x k
// Hbar_k (the eigen residual ||A e - lambda e|| of its unit Ritz vectors); infinity on failure
double ritz_resid_max(const Mat &Hk, bool hermitian) {
  const int k = Hk.c;
  Mat T(k, k);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) T(i, j) = Hk(i, j);
  std::vector<cd> lam(k);
  Mat Y;
  if (hermitian) {
    std::vector<double> w;
    if (!dense::eigh(T, w, Y)) return INFINITY;
    for (int i = 0; i < k; ++i) lam[i] = cd(w[i], 0.0);
  } else if (!dense::eig(T, lam, Y)) {
    return INFINITY;
  }
  double worst = 0.0;
  for (int q = 0; q < k; ++q) {
    double r2 = 0.0;
    for (int i = 0; i <= k; ++i) {
      cd v = 0.0;
      for (int j = 0; j < k; ++j) v += Hk(i, j) * Y(j, q);
      if (i < k) v -= lam[q] * Y(i, q);
      r2 += std::norm(v);
    }
    worst = std::max(worst, std::sqrt(r2));
  }
  return worst;
}

// P_{k+1}: orthonormal [g (zero-padded to m+1 rows) | w]
Mat restart_basis(const Mat &G, const std::vector<cd> &s) {
  const int m1 = (int)s.size(), k = G.c;
  Mat A(m1, k + 1);
  for (int q = 0; q < k; ++q)
    for (int i = 0; i + 1 < m1; ++i) A(i, q) = G(i, q);
  for (int i = 0; i < m1; ++i) A(i, k) = s[i];
  return dense::orthonormalize(A);
}

template <typename S> struct WorkspaceT {
  S *Vb = nullptr, *Vt = nullptr, *tmp = nullptr;
  double2 *hd1 = nullptr, *hd2 = nullptr, *coef = nullptr;
  double *nrm = nullptr;
};
using Workspace = WorkspaceT<double2>;

template <typename S>
lqcd_status get_workspace(lqcd_ctx *ctx, int m, int k, int nrhs, WorkspaceT<S> &w) {
  const long long vs = (long long)nrhs * ctx->N;
  void *p;
  LQCD_TRY(ws_get(ctx, WS_BASIS, sizeof(S) * (size_t)(m + 1) * vs, &p));
  w.Vb = (S *)p;
  LQCD_TRY(ws_get(ctx, WS_BASIS2, sizeof(S) * (size_t)(std::max(k, 1) + 1) * vs, &p));
  w.Vt = (S *)p;
  const size_t hc = (size_t)std::max(m, 1) * (m + 1) * nrhs;
  LQCD_TRY(ws_get(ctx, WS_HESS, sizeof(double2) * 2 * hc + sizeof(double) * (size_t)std::max(m, 1) * nrhs + 64, &p));
  w.hd1 = (double2 *)p;
  w.hd2 = w.hd1 + hc;
  w.nrm = (double *)(w.hd2 + hc);
  LQCD_TRY(ws_get(ctx, WS_COEF, sizeof(double2) * (size_t)(m + 2) * (m + 2) * nrhs, &p));
  w.coef = (double2 *)p;
  LQCD_TRY(ws_get(ctx, WS_TMP0, sizeof(S) * (size_t)vs, &p));
  w.tmp = (S *)p;
  return LQCD_OK;
}

// relative true residuals ||b - A x|| / ||b|| for every right-hand side
lqcd_status true_residuals(lqcd_ctx *ctx, const Op &op, const double2 *b, const double2 *x, double2 *tmp, int nrhs,
                           const std::vector<Rhs> &R, std::vector<double> &rel) {
  const long long N = ctx->N;
  LQCD_TRY(apply_op(ctx, op, x, tmp, nrhs));
  // tmp = b - tmp  via tmp = -tmp + b
  LQCD_TRY(blas_bminus(ctx, tmp, b, (long long)nrhs * N));
  double *nd;
  LQCD_TRY(ws_get(ctx, WS_TMP5, sizeof(double) * nrhs, (void **)&nd));
  LQCD_TRY(blas_norms(ctx, tmp, N, nrhs, nd));
  std::vector<double> h;
  LQCD_TRY(download(ctx, nd, h, nrhs));
  rel.resize(nrhs);
  for (int r = 0; r < nrhs; ++r) rel[r] = R[r].bnorm > 0.0 ? h[r] / R[r].bnorm : h[r];
  return LQCD_OK;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

lqcd_status check_opts(lqcd_ctx *ctx, const lqcd_krylov_opts *o, int nrhs) {
  if (!o) return set_err(ctx, LQCD_ERR_INVALID_ARG, "NULL solver options");
  if (o->m < 1 || o->m > 1000 || o->k < 0 || o->k >= o->m)
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "need 0 <= k < m <= 1000 (m=%d k=%d)", o->m, o->k);
  if (!(o->tol > 0.0) || o->max_cycles < 1) return set_err(ctx, LQCD_ERR_INVALID_ARG, "need tol > 0 and max_cycles >= 1");
  if (!(o->eig_tol >= 0.0)) return set_err(ctx, LQCD_ERR_INVALID_ARG, "need eig_tol >= 0");
  if (nrhs < 1 || nrhs > 4096) return set_err(ctx, LQCD_ERR_INVALID_ARG, "nrhs %d out of range", nrhs);
  if (o->prec < LQCD_PREC_F64 || o->prec > LQCD_PREC_BF16) return set_err(ctx, LQCD_ERR_INVALID_ARG, "bad precision");
  return LQCD_OK;
}

// Rayleigh-Ritz eigenpairs on span(V_k): T = Hbar_k[:k,:k]
// Y = V C for one right-hand side's basis V (nv fields of N at stride vstride; C: device nv x ncol):
// the dense FP64 product that rotates a Krylov basis.  With the tensor-core engine selected and a
// contiguous basis it runs as the split-precision FP64 emulation of the deflation contractions (an
// FP64 GEMM of 8 N nv ncol flop otherwise, FP64-pipe bound: 1.7 s for the 241 x 201 restart of
// MINRES-DR(240,200) on 24^3 x 32), else on the FP64 combine kernel.
lqcd_status basis_combine(lqcd_ctx *ctx, const double2 *V, long long vstride, int nv, const double2 *C, int ncol,
                          double2 *Y) {
  const long long N = ctx->N;
  if (ctx->defl_engine == LQCD_DEFL_TENSOR && vstride == N) return tc_vc_oneshot(ctx, V, nv, C, ncol, Y);
  return blas_combine(ctx, V, vstride, 0, nv, C, ncol, Y, N, N, 1);
}

lqcd_status ritz_pairs(lqcd_ctx *ctx, lqcd_defl *d) {
  const int k = d->k;
  Mat T(k, k);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      const double2 v = d->Hbar[(size_t)i * k + j];
      T(i, j) = cd(v.x, v.y);
    }
  std::vector<cd> lam(k);
  Mat Y;
  if (d->hermitian) {
    std::vector<double> w;
    if (!dense::eigh(T, w, Y)) return set_err(ctx, LQCD_ERR_NOT_CONVERGED, "Rayleigh-Ritz eigensolver failed");
    for (int i = 0; i < k; ++i) lam[i] = cd(w[i], 0.0);
  } else {
    if (!dense::eig(T, lam, Y)) return set_err(ctx, LQCD_ERR_NOT_CONVERGED, "Rayleigh-Ritz eigensolver failed");
  }
  std::vector<int> order(k);
  for (int i = 0; i < k; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return std::abs(lam[a]) < std::abs(lam[b]); });
  d->lam.resize(k);
  d->eres.resize(k);
  std::vector<cd> C((size_t)k * k);
  for (int q = 0; q < k; ++q) {
    const int o = order[q];
    d->lam[q] = make_double2(lam[o].real(), lam[o].imag());
    for (int i = 0; i < k; ++i) C[(size_t)i * k + q] = Y(i, o);
    // ||Hbar_k y - lam [y; 0]||
    double r2 = 0.0;
    for (int i = 0; i <= k; ++i) {
      cd s = 0.0;
      for (int j = 0; j < k; ++j) {
        const double2 hv = d->Hbar[(size_t)i * k + j];
        s += cd(hv.x, hv.y) * Y(j, o);
      }
      if (i < k) s -= lam[o] * Y(i, o);
      r2 += std::norm(s);
    }
    d->eres[q] = std::sqrt(r2);
  }
  void *p;
  LQCD_TRY(ws_get(ctx, WS_COEF, sizeof(cd) * C.size(), &p));
  LQCD_TRY(upload(ctx, C, p));
  return basis_combine(ctx, d->V, d->N, k, (const double2 *)p, k, d->E);
}

// hermitian[r]: right-hand side r uses the Hermitian (MINRES-DR) form of the harmonic Ritz problem.
// defl_out (may be NULL): receives one deflation space per right-hand side.
lqcd_status gmresdr_core(lqcd_ctx *ctx, const Op &op, const double2 *b, double2 *x, int nrhs,
                         const lqcd_krylov_opts *o, const std::vector<char> &hermitian, lqcd_solve_info *info,
                         std::vector<lqcd_defl *> *defl_out) {
  const double t0 = now_s();
  LQCD_TRY(check_opts(ctx, o, nrhs));
  const int m = o->m, k = o->k;
  const long long N = ctx->N, vs = (long long)nrhs * N;
  Workspace W;
  LQCD_TRY(get_workspace(ctx, m, k, nrhs, W));
  std::vector<Rhs> R(nrhs);
  for (auto &r : R) {
    r.H = Mat(m + 1, m);
    r.c.assign(m + 1, cd(0.0, 0.0));
  }
  // x = 0, v_0 = b / ||b||, c = ||b|| e_1
  LQCD_TRY(blas_zero(ctx, x, vs));
  LQCD_TRY(blas_copy(ctx, b, W.Vb, vs));
  LQCD_TRY(blas_norms(ctx, b, N, nrhs, W.nrm));
  std::vector<double> bn;
  LQCD_TRY(download(ctx, W.nrm, bn, nrhs));
  for (int r = 0; r < nrhs; ++r) {
    R[r].bnorm = bn[r];
    R[r].c[0] = bn[r];
    if (!(bn[r] > 0.0)) R[r].active = false;
  }
  LQCD_TRY(blas_invscale(ctx, W.Vb, W.nrm, N, nrhs));
  Arnoldi A{ctx, op, nrhs, m, N, W.Vb, W.hd1, W.hd2, W.nrm};
  long long matvecs = 0;
  int j0 = 0, cycles = 0;
  bool all_conv = false;
  std::vector<std::vector<cd>> theta_keep(nrhs);
  std::vector<Mat> P_keep(nrhs), Hn_keep(nrhs);
  // a right-hand side is done when its residual is below tol and, with eig_tol > 0, the Ritz
  // residuals of its restart space are below eig_tol (super-convergence, Sec. 5.4, 7)
  auto rhs_done = [&](const Rhs &q) { return q.rel <= o->tol && (o->eig_tol <= 0.0 || q.eres <= o->eig_tol); };
  std::vector<char> rotated(nrhs, 0);
  for (int cyc = 0; cyc < o->max_cycles; ++cyc) {
    cycles = cyc + 1;
    NvtxRange nv("GMRES-DR cycle");
    LQCD_TRY(arnoldi_run(A, j0, R, matvecs));
    // least squares per right-hand side, x += V_m d
    std::vector<cd> dcoef((size_t)m * nrhs, cd(0.0, 0.0));
    std::vector<std::vector<cd>> s(nrhs);
    for (int r = 0; r < nrhs; ++r) {
      if (!R[r].active) continue;
      std::vector<cd> d = dense::lstsq(R[r].H, R[r].c);
      s[r] = R[r].c;
      for (int i = 0; i <= m; ++i)
        for (int j = 0; j < m; ++j) s[r][i] -= R[r].H(i, j) * d[j];
      double sn = 0.0;
      for (const cd &v : s[r]) sn += std::norm(v);
      R[r].rel = std::sqrt(sn) / R[r].bnorm;
      for (int j = 0; j < m; ++j) dcoef[(size_t)j * nrhs + r] = d[j];
    }
    LQCD_TRY(upload(ctx, dcoef, W.coef));
    LQCD_TRY(blas_multiaxpy(ctx, W.Vb, vs, N, m, W.coef, 1.0, x, N, nrhs));
    // harmonic Ritz restart (also computed on the final cycle: it defines the deflation space)
    all_conv = true;
    std::vector<cd> pcoef((size_t)(m + 1) * (k + 1) * nrhs, cd(0.0, 0.0));
    for (int r = 0; r < nrhs; ++r) {
      if (!R[r].active) {
        for (int i = 0; i <= k; ++i) pcoef[((size_t)i * (k + 1) + i) * nrhs + r] = 1.0;
        continue;
      }
      std::vector<cd> th;
      Mat G;
      if (k > 0) {
        if (!harmonic_ritz(R[r].H, k, hermitian[r] != 0, th, G))
          return set_err(ctx, LQCD_ERR_NOT_CONVERGED, "harmonic Ritz eigenproblem failed (rhs %d, cycle %d)", r, cyc);
      } else {
        G = Mat(m, 0);
      }
      Mat P = restart_basis(G, lsq_complement(R[r].H, s[r]));
      for (int i = 0; i <= m; ++i)
        for (int c = 0; c <= k; ++c) pcoef[((size_t)i * (k + 1) + c) * nrhs + r] = P(i, c);
      theta_keep[r] = th;
      P_keep[r] = P;
      // Hbar_k of the restart space (the next cycle's start, and the deflation space if last)
      Mat Pk(m, k);
      for (int i = 0; i < m; ++i)
        for (int c = 0; c < k; ++c) Pk(i, c) = P(i, c);
      Hn_keep[r] = dense::matmul(dense::adjoint(P), dense::matmul(R[r].H, Pk));
      R[r].eres = (o->eig_tol > 0.0 && k > 0) ? ritz_resid_max(Hn_keep[r], hermitian[r] != 0) : 0.0;
      if (!rhs_done(R[r])) all_conv = false;
    }
    const bool last = all_conv || cyc + 1 == o->max_cycles;
    if (last) break;
    LQCD_TRY(upload(ctx, pcoef, W.coef));
    if (nrhs == 1) {
      LQCD_TRY(basis_combine(ctx, W.Vb, vs, m + 1, W.coef, k + 1, W.Vt));
    } else {
      LQCD_TRY(blas_combine(ctx, W.Vb, vs, N, m + 1, W.coef, k + 1, W.Vt, vs, N, nrhs));
    }
    LQCD_TRY(blas_copy(ctx, W.Vt, W.Vb, (long long)(k + 1) * vs));
    for (int r = 0; r < nrhs; ++r) {
      if (!R[r].active) continue;
      const Mat &P = P_keep[r];
      // Hbar_new = P^H Hbar P_k  ((k+1) x k), c_new = P^H s
      const Mat &Hn = Hn_keep[r];
      Mat Hfull(m + 1, m);
      for (int i = 0; i <= k; ++i)
        for (int j = 0; j < k; ++j) Hfull(i, j) = Hn(i, j);
      R[r].H = Hfull;
      std::vector<cd> cn(m + 1, cd(0.0, 0.0));
      for (int i = 0; i <= k; ++i) {
        cd v = 0.0;
        for (int q = 0; q <= m; ++q) v += std::conj(P(q, i)) * s[r][q];
        cn[i] = v;
      }
      R[r].c = cn;
      if (rhs_done(R[r])) {
        R[r].active = false;
        rotated[r] = 1;  // V[0..k] and H already hold this right-hand side's deflation space
      }
    }
    j0 = k;
  }
  std::vector<double> rel;
  LQCD_TRY(true_residuals(ctx, op, b, x, W.tmp, nrhs, R, rel));
  double worst = 0.0;
  for (int r = 0; r < nrhs; ++r) worst = std::max(worst, rel[r]);
  matvecs += nrhs;
  if (op.pp.degree > 0) {
    // solved B y = b with B = A p(A): the solution of A x = b is x = p(A) y (same residual)
    LQCD_TRY(op.apply_poly(ctx, x, W.tmp, nrhs));
    LQCD_TRY(blas_copy(ctx, (const double2 *)W.tmp, x, vs));
  }
  if (defl_out && k > 0) {
    for (int r = 0; r < nrhs; ++r) {
      lqcd_defl *d = new lqcd_defl();
      d->ctx = ctx;
      d->k = k;
      d->hermitian = hermitian[r] ? 1 : 0;
      d->N = N;
      d->V = d->E = nullptr;
      d->Hbar_dev = nullptr;
      cudaError_t e1 = cudaMalloc(&d->V, sizeof(double2) * (size_t)(k + 1) * N);
      cudaError_t e2 = cudaMalloc(&d->E, sizeof(double2) * (size_t)k * N);
      cudaError_t e3 = cudaMalloc(&d->Hbar_dev, sizeof(double2) * (size_t)(k + 1) * k);
      if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        cudaGetLastError();
        if (d->V) cudaFree(d->V);
        if (d->E) cudaFree(d->E);
        if (d->Hbar_dev) cudaFree(d->Hbar_dev);
        delete d;
        return set_err(ctx, LQCD_ERR_OOM, "deflation space allocation failed");
      }
      defl_out->push_back(d);
      // a right-hand side that converged before the last cycle was already restarted: its space is
      // V[0..k] with Hbar = H[0..k][0..k-1]; otherwise rotate by the final cycle's P
      Mat P = P_keep[r];
      Mat Hsrc = R[r].H;
      if (rotated[r]) {
        P = Mat(m + 1, k + 1);
        for (int i = 0; i <= k; ++i) P(i, i) = 1.0;
      }
      std::vector<cd> pc((size_t)(m + 1) * (k + 1));
      for (int i = 0; i <= m; ++i)
        for (int c = 0; c <= k; ++c) pc[(size_t)i * (k + 1) + c] = P(i, c);
      LQCD_TRY(upload(ctx, pc, W.coef));
      LQCD_TRY(basis_combine(ctx, W.Vb + (long long)r * N, vs, m + 1, W.coef, k + 1, d->V));
      Mat Pk(m, k);
      for (int i = 0; i < m; ++i)
        for (int c = 0; c < k; ++c) Pk(i, c) = P(i, c);
      Mat Hn = dense::matmul(dense::adjoint(P), dense::matmul(Hsrc, Pk));
      d->Hbar.resize((size_t)(k + 1) * k);
      std::vector<cd> hrow((size_t)(k + 1) * k);
      for (int i = 0; i <= k; ++i)
        for (int j = 0; j < k; ++j) {
          d->Hbar[(size_t)i * k + j] = make_double2(Hn(i, j).real(), Hn(i, j).imag());
          hrow[(size_t)i * k + j] = Hn(i, j);
        }
      LQCD_TRY(upload(ctx, hrow, d->Hbar_dev));
      LQCD_TRY(ritz_pairs(ctx, d));
      LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
  }
  if (info) {
    info->cycles = cycles;
    info->matvecs = (long)matvecs;
    info->converged = (worst <= o->tol) ? 1 : 0;
    info->true_resid = worst;
    info->seconds = now_s() - t0;
  }
  bool conv = all_conv;
  return conv ? LQCD_OK : set_err(ctx, LQCD_ERR_NOT_CONVERGED, "GMRES-DR: no convergence in %d cycles (rel %.3e)", cycles, worst);
}

}  // namespace

// ---- GMRES-Proj ----------------------------------------------------------------------------
// One GMRES-Proj run on storage S: cycles of (i) minimum-residual projection over the deflation
// space (V_{k+1} = Vd on the device, Hbar_k = Hk on the host), (ii) one GMRES(m) cycle, until the
// recursive residual of every right-hand side is below tol; with check_true (FP64 only) the
// result is then confirmed with the true residual, continuing from it where the recursion drifted.
struct ProjResult {
  int cycles = 0;
  long long matvecs = 0;
  double worst = 0.0;     // largest relative residual (true if checked, else recursive)
  bool converged = false;
};

// S: storage of the Krylov basis; SX: storage of b, x and the residual (S itself, or FP32 under an
// FP16 / BF16 basis); SD: storage of the deflation space Vd (FP32 under an FP16 / BF16 basis: its
// projection multiplies by 1 / lambda and would amplify a coarser rounding of it).
template <typename S, typename SX = S, typename SD = S>
lqcd_status proj_run(lqcd_ctx *ctx, const OpT<S> &op, const SD *Vd, const Mat &Hk, const dense::QRFact &Hq, const SX *b,
                     SX *x, int nrhs, int m, double tol, int max_cycles, bool check_true, ProjResult &res,
                     int window = 0) {
  const int k = Hk.c;
  const long long N = ctx->N, vs = (long long)nrhs * N;
  WorkspaceT<S> W;
  LQCD_TRY(get_workspace(ctx, m, 0, nrhs, W));
  if ((size_t)(k + 2) * nrhs > (size_t)(m + 2) * (m + 2) * nrhs) {
    // the projection's coefficients ((k + 1) x nrhs) need more than the cycle's; the basis does not
    LQCD_TRY(ws_get(ctx, WS_COEF, sizeof(double2) * (size_t)(k + 2) * nrhs, (void **)&W.coef));
  }
  SX *r_dev;
  LQCD_TRY(ws_get(ctx, WS_TMP1, sizeof(SX) * (size_t)vs, (void **)&r_dev));
  std::vector<Rhs> R(nrhs);
  LQCD_TRY(blas_zero(ctx, x, vs));
  LQCD_TRY(blas_copy(ctx, b, r_dev, vs));
  LQCD_TRY(blas_norms(ctx, b, N, nrhs, W.nrm));
  std::vector<double> bn;
  LQCD_TRY(download(ctx, W.nrm, bn, nrhs));
  for (int r = 0; r < nrhs; ++r) {
    R[r].bnorm = bn[r];
    R[r].H = Mat(m + 1, m);
    if (!(bn[r] > 0.0)) R[r].active = false;
  }
  ArnoldiT<S> A{ctx, op, nrhs, m, N, W.Vb, W.hd1, W.hd2, W.nrm};
  // reduced-precision inner cycles: one pass for FP16 / BF16 bases (4-byte complex), two for FP32,
  // unless the context sets it
  if (!std::is_same<S, double2>::value) A.passes = ctx->inner_gs_passes ? ctx->inner_gs_passes : (sizeof(S) == 4 ? 1 : 2);
  A.window = window;
  long long matvecs = 0;
  int cycles = 0;
  bool all_conv = false;
  double worst = 0.0;
  for (int cyc = 0; cyc < max_cycles; ++cyc) {
    cycles = cyc + 1;
    NvtxRange nv("GMRES-Proj cycle");
    // (i) projection over the deflation space: d = argmin ||V_{k+1}^H r - Hbar_k d||
    LQCD_TRY(blas_multidot(ctx, Vd, N, 0, k + 1, r_dev, N, nrhs, W.coef));
    std::vector<double2> cp;
    LQCD_TRY(download(ctx, W.coef, cp, (size_t)(k + 1) * nrhs));
    std::vector<cd> dk((size_t)k * nrhs, cd(0.0, 0.0)), zk((size_t)(k + 1) * nrhs, cd(0.0, 0.0));
    for (int r = 0; r < nrhs; ++r) {
      if (!R[r].active) continue;
      std::vector<cd> c(k + 1);
      for (int i = 0; i <= k; ++i) c[i] = cd(cp[(size_t)i * nrhs + r].x, cp[(size_t)i * nrhs + r].y);
      std::vector<cd> d = dense::qr_solve(Hq, c);
      for (int j = 0; j < k; ++j) dk[(size_t)j * nrhs + r] = d[j];
      for (int i = 0; i <= k; ++i) {
        cd v = 0.0;
        for (int j = 0; j < k; ++j) v += Hk(i, j) * d[j];
        zk[(size_t)i * nrhs + r] = v;
      }
    }
    LQCD_TRY(upload(ctx, dk, W.coef));
    LQCD_TRY(blas_multiaxpy(ctx, Vd, N, 0, k, W.coef, 1.0, x, N, nrhs));
    LQCD_TRY(upload(ctx, zk, W.coef));
    LQCD_TRY(blas_multiaxpy(ctx, Vd, N, 0, k + 1, W.coef, -1.0, r_dev, N, nrhs));
    // (ii) one GMRES(m) cycle from r
    LQCD_TRY(blas_norms(ctx, r_dev, N, nrhs, W.nrm));
    std::vector<double> beta;
    LQCD_TRY(download(ctx, W.nrm, beta, nrhs));
    LQCD_TRY(blas_copy(ctx, r_dev, W.Vb, vs));
    LQCD_TRY(blas_invscale(ctx, W.Vb, W.nrm, N, nrhs));
    for (int r = 0; r < nrhs; ++r) {
      R[r].c.assign(m + 1, cd(0.0, 0.0));
      R[r].c[0] = beta[r];
      if (R[r].active && !(beta[r] > 0.0)) R[r].active = false;
    }
    LQCD_TRY(arnoldi_run(A, 0, R, matvecs));
    std::vector<cd> dcoef((size_t)m * nrhs, cd(0.0, 0.0)), scoef((size_t)(m + 1) * nrhs, cd(0.0, 0.0));
    all_conv = true;
    worst = 0.0;
    for (int r = 0; r < nrhs; ++r) {
      if (!R[r].active) {
        scoef[r] = beta[r];  // keep r unchanged: r = V_0 * beta
        continue;
      }
      std::vector<cd> d = dense::lstsq(R[r].H, R[r].c);
      std::vector<cd> sv = R[r].c;
      for (int i = 0; i <= m; ++i)
        for (int j = 0; j < m; ++j) sv[i] -= R[r].H(i, j) * d[j];
      double sn = 0.0;
      for (const cd &v : sv) sn += std::norm(v);
      R[r].rel = std::sqrt(sn) / R[r].bnorm;
      worst = std::max(worst, R[r].rel);
      for (int j = 0; j < m; ++j) dcoef[(size_t)j * nrhs + r] = d[j];
      for (int i = 0; i <= m; ++i) scoef[(size_t)i * nrhs + r] = sv[i];
      if (R[r].rel > tol) all_conv = false;
    }
    LQCD_TRY(upload(ctx, dcoef, W.coef));
    LQCD_TRY(blas_multiaxpy(ctx, W.Vb, vs, N, m, W.coef, 1.0, x, N, nrhs));
    LQCD_TRY(upload(ctx, scoef, W.coef));
    LQCD_TRY(blas_combine(ctx, W.Vb, vs, N, m + 1, W.coef, 1, r_dev, vs, N, nrhs));
    if (all_conv) {
      if (!check_true) break;
      // confirm with the true residual; continue from it where the recursion drifted
      std::vector<double> rel;
      if constexpr (std::is_same<S, double2>::value && std::is_same<SX, double2>::value) {
        LQCD_TRY(true_residuals(ctx, op, b, x, W.tmp, nrhs, R, rel));
      } else {
        break;
      }
      matvecs += nrhs;
      worst = 0.0;
      bool ok = true;
      for (int r = 0; r < nrhs; ++r) {
        worst = std::max(worst, rel[r]);
        if (rel[r] > tol) ok = false;
      }
      if (ok) break;
      all_conv = false;
      LQCD_TRY(blas_copy(ctx, W.tmp, r_dev, vs));
      for (int r = 0; r < nrhs; ++r) R[r].active = rel[r] > tol;
    }
    for (int r = 0; r < nrhs; ++r)
      if (R[r].active && R[r].rel <= tol) R[r].active = false;
  }
  if constexpr (std::is_same<S, double2>::value && std::is_same<SX, double2>::value) {
    if (!all_conv && check_true) {
      std::vector<double> rel;
      LQCD_TRY(true_residuals(ctx, op, b, x, W.tmp, nrhs, R, rel));
      matvecs += nrhs;
      worst = 0.0;
      for (int r = 0; r < nrhs; ++r) worst = std::max(worst, rel[r]);
    }
  }
  res.cycles = cycles;
  res.matvecs = matvecs;
  res.worst = worst;
  res.converged = worst <= tol;
  return LQCD_OK;
}

Mat defl_hbar(const lqcd_defl *defl) {
  const int k = defl->k;
  Mat Hk(k + 1, k);
  for (int i = 0; i <= k; ++i)
    for (int j = 0; j < k; ++j) {
      const double2 v = defl->Hbar[(size_t)i * k + j];
      Hk(i, j) = cd(v.x, v.y);
    }
  return Hk;
}

// the space's Hbar factorised once (the projection of every GMRES-Proj cycle solves with it)
const dense::QRFact &defl_qr(const lqcd_defl *defl) {
  lqcd_defl *d = const_cast<lqcd_defl *>(defl);
  if (!d->hqr) d->hqr = std::make_shared<dense::QRFact>(dense::qr_factor(defl_hbar(defl)));
  return *d->hqr;
}

// Plain FP64 GMRES-Proj
lqcd_status proj_core(lqcd_ctx *ctx, const Op &op, const lqcd_defl *defl, const double2 *b, double2 *x, int nrhs,
                      const lqcd_krylov_opts *o, lqcd_solve_info *info) {
  const double t0 = now_s();
  LQCD_TRY(check_opts(ctx, o, nrhs));
  if (!defl || !defl->V || !defl->Hbar_dev) return set_err(ctx, LQCD_ERR_INVALID_ARG, "GMRES-Proj needs a solver-made deflation space");
  ProjResult res;
  LQCD_TRY(proj_run<double2>(ctx, op, defl->V, defl_hbar(defl), defl_qr(defl), b, x, nrhs, o->m, o->tol,
                             o->max_cycles, true, res));
  if (op.pp.degree > 0) {
    // solved B y = b: the solution of A x = b is x = p(A) y (same residual)
    double2 *t;
    LQCD_TRY(ws_get(ctx, WS_POLY3, sizeof(double2) * (size_t)nrhs * ctx->N, (void **)&t));
    LQCD_TRY(op.apply_poly(ctx, x, t, nrhs));
    LQCD_TRY(blas_copy(ctx, (const double2 *)t, x, (long long)nrhs * ctx->N));
  }
  if (info) {
    info->cycles = res.cycles;
    info->matvecs = (long)res.matvecs;
    info->converged = res.converged ? 1 : 0;
    info->true_resid = res.worst;
    info->seconds = now_s() - t0;
  }
  return res.converged ? LQCD_OK
                       : set_err(ctx, LQCD_ERR_NOT_CONVERGED, "GMRES-Proj: no convergence in %d cycles (rel %.3e)", res.cycles, res.worst);
}

// Mixed precision: FP64 defect correction around a reduced-precision GMRES-Proj.  Each outer step
// solves M e = r / ||r|| approximately (inner relative residual inner_tol) with FP32 arithmetic, the
// Krylov basis stored as S (FP32, FP16 or BF16), the deflation space, e and r in FP32; it adds
// ||r|| e to the FP64 solution and recomputes the true residual r = b - M x with the FP64
// operator, and stops when every right-hand side has ||r|| <= tol ||b|| in FP64.
constexpr int MAX_OUTER = 100;

double default_inner_tol(int prec) {
  // a few tens of the storage unit roundoff for FP16 (2^-11) and BF16 (2^-8): the Arnoldi relation
  // of a basis stored in them holds only to about that level, so tighter inner solves mostly
  // spend cycles the outer correction discards (measured on 8^3 x 16 at kappa 0.157); FP32 inner
  // solves pay off down to 5e-6
  return prec == LQCD_PREC_F16 ? 2e-2 : prec == LQCD_PREC_BF16 ? 5e-2 : 5e-6;
}

template <typename S>
lqcd_status mixed_core(lqcd_ctx *ctx, const Op &op, const lqcd_defl *defl, const double2 *b, double2 *x, int nrhs,
                       const lqcd_krylov_opts *o, lqcd_solve_info *info) {
  const double t0 = now_s();
  LQCD_TRY(check_opts(ctx, o, nrhs));
  if (!defl || !defl->V || !defl->Hbar_dev) return set_err(ctx, LQCD_ERR_INVALID_ARG, "GMRES-Proj needs a solver-made deflation space");
  if (!(o->inner_tol >= 0.0 && o->inner_tol < 1.0)) return set_err(ctx, LQCD_ERR_INVALID_ARG, "inner_tol must be in [0, 1)");
  const double inner_tol = o->inner_tol > 0.0 ? o->inner_tol : default_inner_tol(o->prec);
  const long long N = ctx->N, vs = (long long)nrhs * N;
  const int k = defl->k;
  float2 *Vlp;
  float2 *r32, *e32;
  float4 *U32;
  double2 *r;
  double *sc;
  const int recon = ctx->recon;
  LQCD_TRY(ws_get(ctx, WS_MIX_U, sizeof(float) * (size_t)ctx->V * 4 * (recon == 12 ? 12 : 20), (void **)&U32));
  LQCD_TRY(ws_get(ctx, WS_MIX_R32, sizeof(float2) * (size_t)vs, (void **)&r32));
  LQCD_TRY(ws_get(ctx, WS_MIX_E32, sizeof(float2) * (size_t)vs, (void **)&e32));
  LQCD_TRY(ws_get(ctx, WS_MIX_R, sizeof(double2) * (size_t)vs, (void **)&r));
  LQCD_TRY(ws_get(ctx, WS_MIX_S, sizeof(double) * (size_t)nrhs, (void **)&sc));
  LQCD_TRY(pack_links_f32(ctx, op.U, U32, recon));
  // the FP32 copy of the deflation space is made once per space and kept with it
  lqcd_defl *dmut = const_cast<lqcd_defl *>(defl);
  if (!dmut->Vf32) {
    if (cudaMalloc(&dmut->Vf32, sizeof(float2) * (size_t)(k + 1) * N) != cudaSuccess) {
      cudaGetLastError();
      dmut->Vf32 = nullptr;
      return set_err(ctx, LQCD_ERR_OOM, "mixed solve: FP32 copy of the deflation space does not fit");
    }
    LQCD_TRY(pack_f32(ctx, defl->V, nullptr, (float4 *)dmut->Vf32, k + 1));
  }
  Vlp = (float2 *)dmut->Vf32;
  // inner operator B = A p(A) in storage S; p applied to the inner solutions in FP32; the outer
  // residual is that of A itself
  OpT<float2> opf;
  opf.U = U32;
  opf.recon = recon;
  opf.kappa = op.kappa;
  opf.flags = op.flags;
  opf.pp = op.pp;
  LQCD_TRY(opf.reserve(ctx, nrhs));
  OpT<S> opl;
  opl.U = U32;
  opl.recon = recon;
  opl.kappa = op.kappa;
  opl.flags = op.flags;
  opl.pp = opf.pp;        // the same scratch (sized for FP32 >= S), used one after the other
  Op opA = op;
  opA.pp.degree = 0;
  float2 *e32p = e32;
  if (op.pp.degree > 0) LQCD_TRY(ws_get(ctx, WS_POLY3, sizeof(float2) * (size_t)vs, (void **)&e32p));
  const Mat Hk = defl_hbar(defl);
  const dense::QRFact &Hq = defl_qr(defl);
  // Lanczos window of the inner cycles: only for the Hermitian operator M' = M gamma_5 (times a
  // polynomial with real coefficients)
  const int window = op.flags == LQCD_APPLY_G5R ? ctx->inner_window : 0;
  LQCD_TRY(blas_zero(ctx, x, vs));
  LQCD_TRY(blas_copy(ctx, b, r, vs));
  LQCD_TRY(blas_norms(ctx, b, N, nrhs, sc));
  std::vector<double> bn, rn;
  LQCD_TRY(download(ctx, sc, bn, nrhs));
  long long matvecs = 0;
  int outer = 0, inner_cycles = 0;
  double worst = 0.0;
  bool conv = false;
  NvtxRange nv("mixed-precision defect correction");
  for (outer = 0; outer <= MAX_OUTER; ++outer) {
    LQCD_TRY(blas_norms(ctx, r, N, nrhs, sc));
    LQCD_TRY(download(ctx, sc, rn, nrhs));
    worst = 0.0;
    std::vector<double> scale(nrhs);
    for (int i = 0; i < nrhs; ++i) {
      const double rel = bn[i] > 0.0 ? rn[i] / bn[i] : 0.0;
      if (!std::isfinite(rel)) return set_err(ctx, LQCD_ERR_NONFINITE, "mixed solve: non-finite residual (rhs %d)", i);
      worst = std::max(worst, rel);
      scale[i] = rel > o->tol ? rn[i] : 0.0;  // converged right-hand sides get a zero inner problem
    }
    if (worst <= o->tol) {
      conv = true;
      break;
    }
    if (outer == MAX_OUTER || inner_cycles >= o->max_cycles) break;
    LQCD_CUDA(ctx, cudaMemcpyAsync(sc, scale.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, ctx->stream));
    LQCD_TRY(pack_f32(ctx, r, sc, (float4 *)r32, nrhs));
    ProjResult pr;
    LQCD_TRY((proj_run<S, float2, float2>(ctx, opl, Vlp, Hk, Hq, r32, e32, nrhs, o->m, inner_tol,
                                  std::max(1, o->max_cycles - inner_cycles), false, pr, window)));
    inner_cycles += pr.cycles;
    matvecs += pr.matvecs;
    if (op.pp.degree > 0) LQCD_TRY(opf.apply_poly(ctx, e32, e32p, nrhs));   // e = p(A) e'
    LQCD_TRY(unpack_f32(ctx, (const float4 *)e32p, sc, x, nrhs));
    // FP64 true residual r = b - A x
    LQCD_TRY(opA.apply(ctx, x, r, nrhs));
    LQCD_TRY(blas_bminus(ctx, r, b, vs));
    matvecs += nrhs;
  }
  if (info) {
    info->cycles = inner_cycles;
    info->matvecs = (long)matvecs;
    info->converged = conv ? 1 : 0;
    info->true_resid = worst;
    info->seconds = now_s() - t0;
  }
  return conv ? LQCD_OK
              : set_err(ctx, LQCD_ERR_NOT_CONVERGED, "mixed GMRES-Proj: no convergence after %d outer steps (rel %.3e)", outer, worst);
}

lqcd_status mixed_dispatch(lqcd_ctx *ctx, const Op &op, const lqcd_defl *defl, const double2 *b, double2 *x, int nrhs,
                           const lqcd_krylov_opts *o, lqcd_solve_info *info) {
  if (o->prec == LQCD_PREC_F16) return mixed_core<__half2>(ctx, op, defl, b, x, nrhs, o, info);
  if (o->prec == LQCD_PREC_BF16) return mixed_core<__nv_bfloat162>(ctx, op, defl, b, x, nrhs, o, info);
  return mixed_core<float2>(ctx, op, defl, b, x, nrhs, o, info);
}

// the polynomial preconditioner of a solve from its options (none when poly_degree is 0)
lqcd_status set_poly(lqcd_ctx *ctx, Op &op, const lqcd_krylov_opts *o, int nrhs) {
  if (o->poly_degree == 0) return LQCD_OK;
  if (o->poly_degree < 0 || o->poly_degree > MAX_POLY || !o->poly_coeffs)
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "polynomial preconditioner: degree 0..%d with coefficients", MAX_POLY);
  if (op.flags == OP_MASKED) return set_err(ctx, LQCD_ERR_INVALID_ARG, "polynomial preconditioner: not with a masked operator");
  op.pp.degree = o->poly_degree;
  for (int j = 0; j <= o->poly_degree; ++j) {
    op.pp.a[j] = make_double2(o->poly_coeffs[2 * j], o->poly_coeffs[2 * j + 1]);
    if (!std::isfinite(op.pp.a[j].x) || !std::isfinite(op.pp.a[j].y))
      return set_err(ctx, LQCD_ERR_NONFINITE, "polynomial preconditioner: non-finite coefficient");
  }
  return op.reserve(ctx, nrhs);
}

lqcd_status proj_core_entry(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_defl *defl, const double2 *b,
                            double2 *x, int nrhs, const lqcd_krylov_opts *o, lqcd_solve_info *info) {
  const int sys = defl->hermitian ? LQCD_SYS_MG5 : o->system;
  Op op{(const double2 *)links, kappa, sys == LQCD_SYS_MG5 ? LQCD_APPLY_G5R : LQCD_APPLY_M, LQCD_PREC_F64, 0ull};
  LQCD_TRY(set_poly(ctx, op, o, nrhs));
  if (o->prec != LQCD_PREC_F64) {
    LQCD_TRY(require_full(ctx, "mixed-precision proj_solve"));
    return mixed_dispatch(ctx, op, defl, b, x, nrhs, o, info);
  }
  return proj_core(ctx, op, defl, b, x, nrhs, o, info);
}

// The two special solves of the loop estimate in one batched run: right-hand side 0 is GMRES-DR
// on M (its space serves GMRES-Proj), right-hand side 1 is the Hermitian form on M gamma_5 (its
// Rayleigh-Ritz pairs serve deflation).  b2 holds the same source twice; x2 receives both solutions.
lqcd_status special_solves(lqcd_ctx *ctx, const double *links, double kappa, const double2 *b2, double2 *x2,
                           const lqcd_krylov_opts *o, lqcd_solve_info *info, lqcd_defl **defl_m, lqcd_defl **defl_h) {
  Op op{(const double2 *)links, kappa, OP_MASKED, LQCD_PREC_F64, 2ull};
  std::vector<lqcd_defl *> defls;
  const lqcd_status st = gmresdr_core(ctx, op, b2, x2, 2, o, std::vector<char>{0, 1}, info, &defls);
  *defl_m = defls.size() > 0 ? defls[0] : nullptr;
  *defl_h = defls.size() > 1 ? defls[1] : nullptr;
  return st;
}

lqcd_status gmresdr_entry(lqcd_ctx *ctx, const double *links, double kappa, const double *b, double *x, int nrhs,
                          const lqcd_krylov_opts *opts, lqcd_solve_info *info, lqcd_defl **defl_out, bool hermitian) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  if (!links || !b || !x || !opts) return set_err(ctx, LQCD_ERR_INVALID_ARG, "NULL argument");
  if (defl_out) *defl_out = nullptr;
  const int sys = hermitian ? LQCD_SYS_MG5 : opts->system;
  if (sys != LQCD_SYS_M && sys != LQCD_SYS_MG5) return set_err(ctx, LQCD_ERR_INVALID_ARG, "bad system %d", sys);
  if (opts->prec != LQCD_PREC_F64 && opts->prec != LQCD_PREC_F32)
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "GMRES-DR / MINRES-DR: prec must be LQCD_PREC_F64 or LQCD_PREC_F32");
  Op op{(const double2 *)links, kappa, sys == LQCD_SYS_MG5 ? LQCD_APPLY_G5R : LQCD_APPLY_M, opts->prec, 0ull};
  LQCD_TRY(set_poly(ctx, op, opts, nrhs));
  std::vector<lqcd_defl *> defls;
  const lqcd_status st = gmresdr_core(ctx, op, (const double2 *)b, (double2 *)x, nrhs, opts,
                                      std::vector<char>(nrhs, hermitian ? 1 : 0), info,
                                      (defl_out && nrhs == 1) ? &defls : nullptr);
  if (defl_out && !defls.empty()) *defl_out = defls[0];
  return st;
}

// Eigenvalues of A on the Ritz vectors E of a deflation space made with a polynomial preconditioner
// (a space of B = A p(A): its Ritz vectors approximate eigenvectors of A, B being a function of A):
// lam_q = e_q^dag A e_q (real for the Hermitian A = M gamma_5), eres_q = ||A e_q - lam_q e_q||.
lqcd_status defl_rayleigh(lqcd_ctx *ctx, lqcd_defl *d, const double *links, double kappa, int flags) {
  const int k = d->k;
  const long long N = ctx->N;
  const int chunk = 16;
  double2 *Y, *h;
  double *nr;
  LQCD_TRY(ws_get(ctx, WS_TMP4, sizeof(double2) * (size_t)std::min(k, chunk) * N, (void **)&Y));
  LQCD_TRY(ws_get(ctx, WS_EST1, sizeof(double2) * (size_t)chunk * 2 + sizeof(double) * chunk, (void **)&h));
  nr = (double *)(h + 2 * chunk);
  Op op{(const double2 *)links, kappa, flags, LQCD_PREC_F64, 0ull};
  for (int q0 = 0; q0 < k; q0 += chunk) {
    const int nb = std::min(chunk, k - q0);
    const double2 *E = d->E + (size_t)q0 * N;
    LQCD_TRY(op.apply(ctx, E, Y, nb));
    // <e_q, A e_q>: the basis of right-hand side q is e_q itself
    LQCD_TRY(blas_multidot(ctx, E, 0, N, 1, Y, N, nb, h));
    std::vector<double2> lh;
    LQCD_TRY(download(ctx, h, lh, (size_t)nb));
    std::vector<cd> neg(nb);
    for (int r = 0; r < nb; ++r) {
      const cd l = d->hermitian ? cd(lh[r].x, 0.0) : cd(lh[r].x, lh[r].y);
      d->lam[q0 + r] = make_double2(l.real(), l.imag());
      neg[r] = -l;
    }
    LQCD_TRY(upload(ctx, neg, h + chunk));
    LQCD_TRY(blas_multiaxpy(ctx, E, 0, N, 1, h + chunk, 1.0, Y, N, nb));   // Y = A e - lam e
    LQCD_TRY(blas_norms(ctx, Y, N, nb, nr));
    std::vector<double> rh;
    LQCD_TRY(download(ctx, nr, rh, (size_t)nb));
    for (int r = 0; r < nb; ++r) d->eres[q0 + r] = rh[r];
  }
  return LQCD_OK;
}

extern "C" {

lqcd_status lqcd_gmresdr_solve(lqcd_ctx *ctx, const double *links, double kappa, const double *b, double *x, int nrhs,
                               const lqcd_krylov_opts *opts, lqcd_solve_info *info, lqcd_defl **defl_out) {
  return gmresdr_entry(ctx, links, kappa, b, x, nrhs, opts, info, defl_out, false);
}

lqcd_status lqcd_minresdr_solve(lqcd_ctx *ctx, const double *links, double kappa, const double *b, double *x, int nrhs,
                                const lqcd_krylov_opts *opts, lqcd_solve_info *info, lqcd_defl **defl_out) {
  return gmresdr_entry(ctx, links, kappa, b, x, nrhs, opts, info, defl_out, true);
}

lqcd_status lqcd_proj_solve(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_defl *defl, const double *b,
                            double *x, int nrhs, const lqcd_krylov_opts *opts, lqcd_solve_info *info) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  if (!links || !b || !x || !opts || !defl) return set_err(ctx, LQCD_ERR_INVALID_ARG, "NULL argument");
  return proj_core_entry(ctx, links, kappa, defl, (const double2 *)b, (double2 *)x, nrhs, opts, info);
}

lqcd_status lqcd_defl_destroy(lqcd_defl *d) {
  if (!d) return LQCD_ERR_INVALID_ARG;
  if (d->ctx) cudaStreamSynchronize(d->ctx->stream);
  if (d->V) cudaFree(d->V);
  if (d->E) cudaFree(d->E);
  if (d->Hbar_dev) cudaFree(d->Hbar_dev);
  if (d->Vf32) cudaFree(d->Vf32);
  if (d->tc) tc_slices_free(d->tc);
  delete d;
  return LQCD_OK;
}

lqcd_status lqcd_defl_info(const lqcd_defl *d, int *k, int *hermitian) {
  if (!d) return LQCD_ERR_INVALID_ARG;
  if (k) *k = d->k;
  if (hermitian) *hermitian = d->hermitian;
  return LQCD_OK;
}

lqcd_status lqcd_defl_export(const lqcd_defl *d, double *V, double *Hbar, double *lam, double *E, double *eig_resid) {
  if (!d) return LQCD_ERR_INVALID_ARG;
  lqcd_ctx *ctx = d->ctx;
  if (V) {
    if (!d->V) return set_err(ctx, LQCD_ERR_INVALID_ARG, "deflation object has no Krylov basis");
    LQCD_CUDA(ctx, cudaMemcpyAsync(V, d->V, sizeof(double2) * (size_t)(d->k + 1) * d->N, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  if (E) LQCD_CUDA(ctx, cudaMemcpyAsync(E, d->E, sizeof(double2) * (size_t)d->k * d->N, cudaMemcpyDeviceToDevice, ctx->stream));
  if (Hbar) {
    if (d->Hbar.empty()) return set_err(ctx, LQCD_ERR_INVALID_ARG, "deflation object has no Hessenberg matrix");
    memcpy(Hbar, d->Hbar.data(), sizeof(double2) * d->Hbar.size());
  }
  if (lam) memcpy(lam, d->lam.data(), sizeof(double2) * d->lam.size());
  if (eig_resid) memcpy(eig_resid, d->eres.data(), sizeof(double) * d->eres.size());
  LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return LQCD_OK;
}

lqcd_status lqcd_defl_import(lqcd_ctx *ctx, int k, const double *E, const double *lam, lqcd_defl **out) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  if (!E || !lam || !out || k < 1) return set_err(ctx, LQCD_ERR_INVALID_ARG, "defl_import: bad arguments");
  lqcd_defl *d = new lqcd_defl();
  d->ctx = ctx;
  d->k = k;
  d->hermitian = 1;
  d->N = ctx->N;
  d->V = nullptr;
  d->Hbar_dev = nullptr;
  d->E = nullptr;
  if (cudaMalloc(&d->E, sizeof(double2) * (size_t)k * ctx->N) != cudaSuccess) {
    cudaGetLastError();
    delete d;
    return set_err(ctx, LQCD_ERR_OOM, "defl_import: allocation failed");
  }
  cudaError_t e = cudaMemcpyAsync(d->E, E, sizeof(double2) * (size_t)k * ctx->N, cudaMemcpyDeviceToDevice, ctx->stream);
  if (e != cudaSuccess) {
    cudaFree(d->E);
    delete d;
    return set_err(ctx, LQCD_ERR_CUDA, "defl_import: copy failed: %s", cudaGetErrorString(e));
  }
  d->lam.resize(k);
  memcpy(d->lam.data(), lam, sizeof(double2) * k);
  d->eres.assign(k, 0.0);
  cudaStreamSynchronize(ctx->stream);
  *out = d;
  return LQCD_OK;
}

lqcd_status lqcd_defl_import_space(lqcd_ctx *ctx, int k, const double *V, const double *Hbar, int hermitian,
                                   lqcd_defl **out) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  if (!V || !Hbar || !out || k < 1 || k > 4096) return set_err(ctx, LQCD_ERR_INVALID_ARG, "defl_import_space: bad arguments");
  *out = nullptr;
  for (size_t i = 0; i < (size_t)(k + 1) * k * 2; ++i)
    if (!std::isfinite(Hbar[i])) return set_err(ctx, LQCD_ERR_NONFINITE, "defl_import_space: non-finite Hbar entry");
  lqcd_defl *d = new lqcd_defl();
  d->ctx = ctx;
  d->k = k;
  d->hermitian = hermitian ? 1 : 0;
  d->N = ctx->N;
  d->V = d->E = nullptr;
  d->Hbar_dev = nullptr;
  d->tc = nullptr;
  std::unique_ptr<lqcd_defl, lqcd_status (*)(lqcd_defl *)> guard(d, lqcd_defl_destroy);
  cudaError_t e1 = cudaMalloc(&d->V, sizeof(double2) * (size_t)(k + 1) * d->N);
  cudaError_t e2 = cudaMalloc(&d->E, sizeof(double2) * (size_t)k * d->N);
  cudaError_t e3 = cudaMalloc(&d->Hbar_dev, sizeof(double2) * (size_t)(k + 1) * k);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, LQCD_ERR_OOM, "defl_import_space: allocation failed");
  }
  LQCD_CUDA(ctx, cudaMemcpyAsync(d->V, V, sizeof(double2) * (size_t)(k + 1) * d->N, cudaMemcpyDeviceToDevice, ctx->stream));
  d->Hbar.resize((size_t)(k + 1) * k);
  memcpy(d->Hbar.data(), Hbar, sizeof(double2) * d->Hbar.size());
  std::vector<cd> hrow((size_t)(k + 1) * k);
  for (size_t i = 0; i < hrow.size(); ++i) hrow[i] = cd(d->Hbar[i].x, d->Hbar[i].y);
  LQCD_TRY(upload(ctx, hrow, d->Hbar_dev));
  LQCD_TRY(ritz_pairs(ctx, d));
  LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *out = guard.release();
  return LQCD_OK;
}

}  // extern "C"
