// Even/odd preconditioning of the Wilson matrix (Sec. 7) on the GPU.
//
// With every extent even and a site's parity (x + y + z + t) mod 2, the hopping matrix P of
// Eq. xyz556 couples only sites of opposite parity, so in (even, odd) order
//   M = [[1, -kappa P_eo], [-kappa P_oe, 1]],
// and the odd unknowns are eliminated exactly:
//   hat M = 1 - kappa^2 P_eo P_oe,   hat M x_e = b_e + kappa P_eo b_o,   x_o = b_o + kappa P_oe x_e.
// hat M is gamma_5-hermitian (gamma_5 P_eo gamma_5 = P_oe^dag), so hat M' = hat M gamma_5 is
// Hermitian on the even sites, and the Krylov solvers run on either unchanged.
//
// Reduced (compact) field layout: the sites of one parity in lexicographic order of the full site
// index s = x + Lx (y + Ly (z + Lz t)); since Lx is even, compact index i = s >> 1 for both parities
// ([rhs][i][spin 4][colour 3] complex128).  A reduced context (lqcd_ctx_create_evenodd) has the
// dims (Lx/2, Ly, Lz, Lt), so its field length 12 V/2 is what every level-1/2 kernel and Krylov
// solver of the library already works with; its Wilson operator is hat M (two hopping launches
// through a workspace odd field), taking the full links [mu][V][3][3].
#include <complex>

#include "common.cuh"
#include "spin.cuh"

using cd = std::complex<double>;

namespace {

using namespace spin;

// bits of FL: gamma_5 on the hopping input; add a same-parity field; gamma_5 on that field;
// gamma_5 on the result; hopping input / added field / output in the full (not compact) layout
constexpr int EO_HOP_G5 = 1, EO_SELF = 2, EO_SELF_G5 = 4, EO_LEFT_G5 = 8, EO_IN_FULL = 16, EO_SELF_FULL = 32,
              EO_OUT_FULL = 64;

template <typename R>
__device__ __forceinline__ void g5p(Cx<R> p[4][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Cx<R> a0 = p[0][c], a1 = p[1][c];
    p[0][c] = neg(p[2][c]);
    p[1][c] = neg(p[3][c]);
    p[2][c] = neg(a0);
    p[3][c] = neg(a1);
  }
}

// out(i) = [self(i)] + coef * sum_mu [(1 - g_mu) U_mu(x) in(x + mu) + (1 + g_mu) U_mu(x - mu)^dag in(x - mu)]
// for the sites x of parity par (one thread per (site, right-hand side)); the neighbours have the
// other parity.  Vh = V / 2 sites per parity; links [mu][V] with V = 2 Vh.
template <typename R, int FL>
__global__ void __launch_bounds__(128) eo_hop_kernel(const double2 *__restrict__ U, const double2 *__restrict__ in,
                                                     const double2 *__restrict__ self, double2 *__restrict__ out,
                                                     double coef, int Lx, int Ly, int Lz, int Lt, int Vh, int par) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Vh) return;
  const long long V = 2LL * Vh;
  const int Lxh = Lx >> 1;
  int r = i / Lxh;
  const int xh = i - r * Lxh;
  const int y = r % Ly;
  r /= Ly;
  const int z = r % Lz;
  const int t = r / Lz;
  const int x = 2 * xh + ((y + z + t + par) & 1);
  const int s = x + Lx * (y + Ly * (z + Lz * t));
  const int sy = Lx, sz = Lx * Ly, st = Lx * Ly * Lz;
  int nb[8];
  nb[0] = (x + 1 == Lx) ? s - (Lx - 1) : s + 1;
  nb[1] = (x == 0) ? s + (Lx - 1) : s - 1;
  nb[2] = (y + 1 == Ly) ? s - (Ly - 1) * sy : s + sy;
  nb[3] = (y == 0) ? s + (Ly - 1) * sy : s - sy;
  nb[4] = (z + 1 == Lz) ? s - (Lz - 1) * sz : s + sz;
  nb[5] = (z == 0) ? s + (Lz - 1) * sz : s - sz;
  nb[6] = (t + 1 == Lt) ? s - (Lt - 1) * st : s + st;
  nb[7] = (t == 0) ? s + (Lt - 1) * st : s - st;
  const long long rb = blockIdx.y;
  const double2 *src = in + rb * ((FL & EO_IN_FULL) ? V : Vh) * 12;
  Cx<R> acc[4][3], p[4][3], u[9];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[a][c] = mk<R>(0, 0);
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    const int mu = d >> 1;
    const long long n = (FL & EO_IN_FULL) ? nb[d] : (nb[d] >> 1);
    load_spinor<R, (FL & EO_HOP_G5) != 0>(src + 12 * n, p);
    load_link<R>(U, mu * V + ((d & 1) ? nb[d] : s), u);
    if (d == 0) term_fwd<R, 0>(p, u, acc);
    if (d == 1) term_bwd<R, 0>(p, u, acc);
    if (d == 2) term_fwd<R, 1>(p, u, acc);
    if (d == 3) term_bwd<R, 1>(p, u, acc);
    if (d == 4) term_fwd<R, 2>(p, u, acc);
    if (d == 5) term_bwd<R, 2>(p, u, acc);
    if (d == 6) term_fwd<R, 3>(p, u, acc);
    if (d == 7) term_bwd<R, 3>(p, u, acc);
  }
  const R k = (R)coef;
  Cx<R> o[4][3];
  if (FL & EO_SELF) {
    const long long si = (FL & EO_SELF_FULL) ? rb * V * 12 + 12LL * s : rb * Vh * 12 + 12LL * i;
    load_spinor<R, (FL & EO_SELF_G5) != 0>(self + si, p);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) o[a][c] = mk<R>(fma(k, acc[a][c].x, p[a][c].x), fma(k, acc[a][c].y, p[a][c].y));
  } else {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) o[a][c] = mk<R>(k * acc[a][c].x, k * acc[a][c].y);
  }
  if (FL & EO_LEFT_G5) g5p(o);
  double2 *dst = out + ((FL & EO_OUT_FULL) ? rb * V * 12 + 12LL * s : rb * Vh * 12 + 12LL * i);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) store_c(dst + 3 * a + c, o[a][c]);
}

// full field <-> (even, odd) compact fields; either compact pointer may be NULL (not copied)
template <bool SPLIT>
__global__ void eo_copy_kernel(double2 *__restrict__ full, double2 *__restrict__ ev, double2 *__restrict__ od, int Lx,
                               int Ly, int Lz, int Vh) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (site, component) of one rhs
  const long long V = 2LL * Vh;
  if (j >= V * 12) return;
  const int s = (int)(j / 12), comp = (int)(j % 12);
  int r = s / Lx;
  const int x = s - r * Lx;
  const int y = r % Ly;
  r /= Ly;
  const int z = r % Lz;
  const int t = r / Lz;
  double2 *half = ((x + y + z + t) & 1) ? od : ev;
  if (!half) return;
  const long long rb = blockIdx.y;
  const long long fi = rb * V * 12 + j, hi = rb * (long long)Vh * 12 + 12LL * (s >> 1) + comp;
  if (SPLIT)
    half[hi] = full[fi];
  else
    full[fi] = half[hi];
}

// out(r) = join(ve(q), c_r * po(q)) with q = r / 2 (the two full eigenvectors of one reduced pair)
__global__ void eo_pair_kernel(const double2 *__restrict__ ve, const double2 *__restrict__ po,
                               const double2 *__restrict__ c, double2 *__restrict__ out, int Lx, int Ly, int Lz,
                               int Vh) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long V = 2LL * Vh;
  if (j >= V * 12) return;
  const int s = (int)(j / 12), comp = (int)(j % 12);
  int r = s / Lx;
  const int x = s - r * Lx;
  const int y = r % Ly;
  r /= Ly;
  const int z = r % Lz;
  const int t = r / Lz;
  const long long ro = blockIdx.y, q = ro >> 1;
  const long long hi = q * (long long)Vh * 12 + 12LL * (s >> 1) + comp;
  out[ro * V * 12 + j] = ((x + y + z + t) & 1) ? cmul(c[ro], po[hi]) : ve[hi];
}

template <typename R, int FL>
lqcd_status hop_launch(lqcd_ctx *ctx, const double2 *U, const double2 *in, const double2 *self, double2 *out,
                       double coef, int nrhs, int par) {
  int bs = 128;
  while (bs > 32 && (long long)ceil_div(ctx->V, bs) * nrhs < 2LL * ctx->sms) bs /= 2;
  const int *d = ctx->eo_dims;
  kbegin(ctx);
  eo_hop_kernel<R, FL><<<dim3(ceil_div(ctx->V, bs), nrhs), bs, 0, ctx->stream>>>(U, in, self, out, coef, d[0], d[1],
                                                                               d[2], d[3], ctx->V, par);
  // compulsory bytes: the input half read, the output half written (plus the added half), links once
  const double bytes = (2.0 + ((FL & EO_SELF) ? 1.0 : 0.0)) * nrhs * ctx->V * 12 * 16.0 + 36.0 * 2 * ctx->V * 16.0;
  return launch_check_bytes(ctx, "eo_hop_kernel", K_WILSON, (double)ctx->V * nrhs, bytes);
}

template <bool SPLIT>
lqcd_status copy_launch(lqcd_ctx *ctx, double2 *full, double2 *ev, double2 *od, int nrhs) {
  const long long n = 24LL * ctx->V;
  kbegin(ctx);
  eo_copy_kernel<SPLIT><<<dim3(ceil_div(n, 256), nrhs), 256, 0, ctx->stream>>>(full, ev, od, ctx->eo_dims[0],
                                                                               ctx->eo_dims[1], ctx->eo_dims[2], ctx->V);
  return launch_check_bytes(ctx, "eo_copy_kernel", K_BLAS1, (double)n * nrhs, 2.0 * n * nrhs * 16.0);
}

lqcd_status check_nrhs(lqcd_ctx *ctx, int nrhs, const char *what) {
  if (nrhs < 1 || nrhs > 65535) return set_err(ctx, LQCD_ERR_INVALID_ARG, "%s: nrhs %d out of range", what, nrhs);
  return LQCD_OK;
}

}  // namespace

// hat M (flags LQCD_APPLY_M), hat M gamma_5 (LQCD_APPLY_G5R), hat M^dag = gamma_5 hat M gamma_5
// (LQCD_APPLY_DAG) or P_eo P_oe (LQCD_APPLY_HOP) on the even sites: the Wilson operator of a reduced
// context.  R = double (FP64) or float (FP32 arithmetic on FP64 storage).
template <typename R>
lqcd_status eo_schur_launch_t(lqcd_ctx *ctx, const double2 *U, double kappa, const double2 *in, double2 *out,
                              int nrhs, int flags) {
  double2 *tmp;
  LQCD_TRY(ws_get(ctx, WS_EO, sizeof(double2) * (size_t)nrhs * ctx->N, (void **)&tmp));
  const double k2 = -kappa * kappa;
  switch (flags) {
    case LQCD_APPLY_M:
      LQCD_TRY((hop_launch<R, 0>(ctx, U, in, nullptr, tmp, 1.0, nrhs, 1)));
      return hop_launch<R, EO_SELF>(ctx, U, tmp, in, out, k2, nrhs, 0);
    case LQCD_APPLY_G5R:
      LQCD_TRY((hop_launch<R, EO_HOP_G5>(ctx, U, in, nullptr, tmp, 1.0, nrhs, 1)));
      return hop_launch<R, EO_SELF | EO_SELF_G5>(ctx, U, tmp, in, out, k2, nrhs, 0);
    case LQCD_APPLY_DAG:
      LQCD_TRY((hop_launch<R, EO_HOP_G5>(ctx, U, in, nullptr, tmp, 1.0, nrhs, 1)));
      return hop_launch<R, EO_SELF | EO_SELF_G5 | EO_LEFT_G5>(ctx, U, tmp, in, out, k2, nrhs, 0);
    case LQCD_APPLY_HOP:
      LQCD_TRY((hop_launch<R, 0>(ctx, U, in, nullptr, tmp, 1.0, nrhs, 1)));
      return hop_launch<R, 0>(ctx, U, tmp, nullptr, out, 1.0, nrhs, 0);
    default:
      return set_err(ctx, LQCD_ERR_INVALID_ARG, "wilson_apply (even/odd): unknown flags %d", flags);
  }
}

lqcd_status eo_schur_launch(lqcd_ctx *ctx, const double2 *U, double kappa, const double2 *in, double2 *out, int nrhs,
                            int prec, int flags) {
  if (prec == LQCD_PREC_F64) return eo_schur_launch_t<double>(ctx, U, kappa, in, out, nrhs, flags);
  if (prec == LQCD_PREC_F32) return eo_schur_launch_t<float>(ctx, U, kappa, in, out, nrhs, flags);
  return set_err(ctx, LQCD_ERR_INVALID_ARG, "wilson_apply (even/odd): precision %d not available", prec);
}

lqcd_status eo_reserve(lqcd_ctx *ctx, int nrhs) {
  if (!ctx->eo) return LQCD_OK;
  void *p;
  return ws_get(ctx, WS_EO, sizeof(double2) * (size_t)nrhs * ctx->N, &p);
}

lqcd_status require_full(lqcd_ctx *ctx, const char *what) {
  if (ctx->eo) return set_err(ctx, LQCD_ERR_INVALID_ARG, "%s: not available on an even/odd reduced context", what);
  return LQCD_OK;
}

lqcd_status eo_rhs_launch(lqcd_ctx *ctx, const double2 *U, double kappa, const double2 *b, double2 *be, int nrhs) {
  return hop_launch<double, EO_IN_FULL | EO_SELF | EO_SELF_FULL>(ctx, U, b, b, be, kappa, nrhs, 0);
}

lqcd_status eo_reconstruct_launch(lqcd_ctx *ctx, const double2 *U, double kappa, const double2 *xe, const double2 *b,
                                  double2 *x, int nrhs) {
  LQCD_TRY(copy_launch<false>(ctx, x, const_cast<double2 *>(xe), nullptr, nrhs));
  return hop_launch<double, EO_SELF | EO_SELF_FULL | EO_OUT_FULL>(ctx, U, xe, b, x, kappa, nrhs, 1);
}

namespace {
lqcd_status require_eo(lqcd_ctx *ctx, const char *what) {
  if (!ctx->eo) return set_err(ctx, LQCD_ERR_INVALID_ARG, "%s: needs an even/odd reduced context", what);
  return LQCD_OK;
}
}  // namespace

extern "C" lqcd_status lqcd_ctx_create_evenodd(lqcd_ctx **out, const int dims[4], int link_recon, void *stream) {
  if (!out || !dims) return LQCD_ERR_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < 4; ++i)
    if (dims[i] < 2 || dims[i] > 1024 || (dims[i] & 1)) return LQCD_ERR_INVALID_ARG;
  // the reduced context: half the sites, so every field and solver has length 12 V / 2; its dims
  // (Lx/2, Ly, Lz, Lt) describe that length, the full lattice is kept in eo_dims
  int hd[4] = {dims[0] / 2, dims[1], dims[2], dims[3]};
  int cd[4] = {2, 2, 2, 2};  // placeholder extents accepted by the plain constructor
  lqcd_ctx *c = nullptr;
  const lqcd_status st = lqcd_ctx_create(&c, cd, link_recon, stream);
  if (st != LQCD_OK) return st;
  const long long V = (long long)hd[0] * hd[1] * hd[2] * hd[3];
  if (2 * V > (1LL << 28)) {
    lqcd_ctx_destroy(c);
    return LQCD_ERR_INVALID_ARG;
  }
  for (int i = 0; i < 4; ++i) {
    c->dims[i] = hd[i];
    c->eo_dims[i] = dims[i];
  }
  c->V = (int)V;
  c->N = 12 * V;
  c->eo = 1;
  *out = c;
  return LQCD_OK;
}

extern "C" lqcd_status lqcd_eo_split(lqcd_ctx *ctx, const double *full, double *even, double *odd, int nrhs) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_eo(ctx, "eo_split"));
  LQCD_TRY(check_nrhs(ctx, nrhs, "eo_split"));
  if (!full || (!even && !odd)) return set_err(ctx, LQCD_ERR_INVALID_ARG, "eo_split: NULL pointer");
  return copy_launch<true>(ctx, (double2 *)full, (double2 *)even, (double2 *)odd, nrhs);
}

extern "C" lqcd_status lqcd_eo_join(lqcd_ctx *ctx, const double *even, const double *odd, double *full, int nrhs) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_eo(ctx, "eo_join"));
  LQCD_TRY(check_nrhs(ctx, nrhs, "eo_join"));
  if (!full || !even || !odd) return set_err(ctx, LQCD_ERR_INVALID_ARG, "eo_join: NULL pointer");
  return copy_launch<false>(ctx, (double2 *)full, (double2 *)even, (double2 *)odd, nrhs);
}

extern "C" lqcd_status lqcd_eo_hop(lqcd_ctx *ctx, const double *links, const double *in, double *out, int nrhs,
                                   int parity_out) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_eo(ctx, "eo_hop"));
  LQCD_TRY(check_nrhs(ctx, nrhs, "eo_hop"));
  if (!links || !in || !out || in == out) return set_err(ctx, LQCD_ERR_INVALID_ARG, "eo_hop: bad pointers");
  if (parity_out != 0 && parity_out != 1) return set_err(ctx, LQCD_ERR_INVALID_ARG, "eo_hop: parity must be 0 or 1");
  return hop_launch<double, 0>(ctx, (const double2 *)links, (const double2 *)in, nullptr, (double2 *)out, 1.0, nrhs,
                               parity_out);
}

extern "C" lqcd_status lqcd_eo_rhs(lqcd_ctx *ctx, const double *links, double kappa, const double *b, double *be,
                                   int nrhs) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_eo(ctx, "eo_rhs"));
  LQCD_TRY(check_nrhs(ctx, nrhs, "eo_rhs"));
  if (!links || !b || !be || b == be) return set_err(ctx, LQCD_ERR_INVALID_ARG, "eo_rhs: bad pointers");
  return eo_rhs_launch(ctx, (const double2 *)links, kappa, (const double2 *)b, (double2 *)be, nrhs);
}

extern "C" lqcd_status lqcd_eo_reconstruct(lqcd_ctx *ctx, const double *links, double kappa, const double *xe,
                                           const double *b, double *x, int nrhs) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_eo(ctx, "eo_reconstruct"));
  LQCD_TRY(check_nrhs(ctx, nrhs, "eo_reconstruct"));
  if (!links || !xe || !b || !x || x == b || x == xe)
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "eo_reconstruct: bad pointers");
  return eo_reconstruct_launch(ctx, (const double2 *)links, kappa, (const double2 *)xe, (const double2 *)b,
                               (double2 *)x, nrhs);
}

extern "C" lqcd_status lqcd_eo_full_eigenpairs(lqcd_ctx *ctx, const double *links, double kappa, const double *mu,
                                               const double *Ve, int Q, double tol, double *lam, double *E) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_eo(ctx, "eo_full_eigenpairs"));
  LQCD_TRY(check_nrhs(ctx, Q, "eo_full_eigenpairs"));
  if (Q > 32767) return set_err(ctx, LQCD_ERR_INVALID_ARG, "eo_full_eigenpairs: Q %d out of range", Q);
  if (!links || !mu || !Ve || !lam || !E || !(tol >= 0.0))
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "eo_full_eigenpairs: bad arguments");
  // host: 1 - lambda = +-sqrt(1 - mu) (principal root), coefficients 1 / (1 - lambda) of the odd part
  std::vector<cd> c(2 * (size_t)Q);
  for (int q = 0; q < Q; ++q) {
    const cd m(mu[2 * q], mu[2 * q + 1]);
    if (!std::isfinite(m.real()) || !std::isfinite(m.imag()))
      return set_err(ctx, LQCD_ERR_NONFINITE, "eo_full_eigenpairs: non-finite mu[%d]", q);
    const cd r = std::sqrt(cd(1.0, 0.0) - m);
    if (std::abs(r) <= tol)
      return set_err(ctx, LQCD_ERR_INVALID_ARG, "eo_full_eigenpairs: mu[%d] is 1 within tol (lambda = 1)", q);
    for (int sg = 0; sg < 2; ++sg) {
      const cd oml = sg ? -r : r;
      c[2 * q + sg] = 1.0 / oml;
      lam[2 * (2 * q + sg)] = 1.0 - oml.real();
      lam[2 * (2 * q + sg) + 1] = -oml.imag();
    }
  }
  double2 *po, *cd_dev;
  LQCD_TRY(ws_get(ctx, WS_EO, sizeof(double2) * (size_t)Q * ctx->N, (void **)&po));
  LQCD_TRY(ws_get(ctx, WS_TMP0, sizeof(double2) * 2 * (size_t)Q, (void **)&cd_dev));
  LQCD_CUDA(ctx, cudaMemcpyAsync(cd_dev, c.data(), sizeof(cd) * c.size(), cudaMemcpyHostToDevice, ctx->stream));
  // P_oe v_e (kappa folded into the coefficients below)
  LQCD_TRY((hop_launch<double, 0>(ctx, (const double2 *)links, (const double2 *)Ve, nullptr, po, kappa, Q, 1)));
  const long long n = 24LL * ctx->V;
  kbegin(ctx);
  eo_pair_kernel<<<dim3(ceil_div(n, 256), 2 * Q), 256, 0, ctx->stream>>>((const double2 *)Ve, po, cd_dev, (double2 *)E,
                                                                       ctx->eo_dims[0], ctx->eo_dims[1],
                                                                       ctx->eo_dims[2], ctx->V);
  LQCD_TRY(launch_check_bytes(ctx, "eo_pair_kernel", K_BLAS1, (double)n * 2 * Q, 2.0 * n * 2 * Q * 16.0));
  // unit length
  double *nrm;
  LQCD_TRY(ws_get(ctx, WS_TMP1, sizeof(double) * 2 * (size_t)Q, (void **)&nrm));
  LQCD_TRY(blas_norms(ctx, (const double2 *)E, n, 2 * Q, nrm));
  LQCD_TRY(blas_invscale(ctx, (double2 *)E, nrm, n, 2 * Q));
  // the staged coefficients must outlive the copy
  LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return LQCD_OK;
}
