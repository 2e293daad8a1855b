// Derivatives of the loop estimates with respect to kappa and to the gauge links (an addition:
// the paper has no derivatives).
//
// With M = 1 - kappa P (Eq. xyz556): d M^{-1}/dkappa = M^{-1} P M^{-1}, so per noise, with
// x = M^{-1} eta and y = M^{-1} P x,
//     d(eta^dag Theta x)/dkappa = eta^dag Theta y + eta^dag (dTheta/dkappa) x,
// where dTheta/dkappa = Theta/kappa for the point-split operators (their kappa prefactor, Table
// Table903) and 0 for the local ones.  PS subtraction is differentiated term by term.
// For the scalar estimate T = eta^dag M^{-1} eta and z = M^{-dag} eta = g5 M^{-1} g5 eta:
//     dT = kappa z^dag dP x;
// under U_mu(s) -> exp(i w lambda_a / 2) U_mu(s) (Gell-Mann lambda_a)
//     dT/dw_a = (i kappa / 2) tr(lambda_a B),
//     B = sum_spin [(1 - g_mu) U x(s+mu)] z(s)^dag - sum_spin [(1 + g_mu) x(s)] (U z(s+mu))^dag,
// and the complex-matrix derivatives are
//     dT/dU_ab  = kappa sum_spin z(s)*_a [(1 - g_mu) x(s+mu)]_b,
//     dT/dU*_ab = kappa sum_spin z(s+mu)*_b [(1 + g_mu) x(s)]_a.
// The gradient of Re T in torch's convention for complex leaves is dT/dU* + conj(dT/dU).
// Krylov bases are not stored: the derivative call re-solves the systems it needs.
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>

#include "common.cuh"
#include "spin.cuh"

using cd = std::complex<double>;

namespace {

using namespace spin;

// Gell-Mann matrices, row-major, as (re, im) pairs
__constant__ double c_lambda[8][9][2] = {
    {{0, 0}, {1, 0}, {0, 0}, {1, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}},
    {{0, 0}, {0, -1}, {0, 0}, {0, 1}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}},
    {{1, 0}, {0, 0}, {0, 0}, {0, 0}, {-1, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}},
    {{0, 0}, {0, 0}, {1, 0}, {0, 0}, {0, 0}, {0, 0}, {1, 0}, {0, 0}, {0, 0}},
    {{0, 0}, {0, 0}, {0, -1}, {0, 0}, {0, 0}, {0, 0}, {0, 1}, {0, 0}, {0, 0}},
    {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {1, 0}, {0, 0}, {1, 0}, {0, 0}},
    {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, -1}, {0, 0}, {0, 1}, {0, 0}},
    {{0.57735026918962576, 0}, {0, 0}, {0, 0}, {0, 0}, {0.57735026918962576, 0}, {0, 0}, {0, 0}, {0, 0},
     {-1.1547005383792515, 0}}};

__device__ __forceinline__ void zero4(Cx<double> a[4][3]) {
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) a[s][c] = mk<double>(0.0, 0.0);
}

// (1 + g_mu) p as a full spinor, through the backward term with the unit colour matrix
template <int MU>
__device__ __forceinline__ void proj_plus(const Cx<double> p[4][3], Cx<double> o[4][3]) {
  Cx<double> one[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) one[i] = mk<double>((i % 4 == 0) ? 1.0 : 0.0, 0.0);
  zero4(o);
  term_bwd<double, MU>(p, one, o);
}

template <int MU>
__device__ __forceinline__ void proj_minus(const Cx<double> p[4][3], Cx<double> o[4][3]) {
  Cx<double> one[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) one[i] = mk<double>((i % 4 == 0) ? 1.0 : 0.0, 0.0);
  zero4(o);
  term_fwd<double, MU>(p, one, o);
}

template <int MU>
__device__ void link_terms(const Cx<double> u[9], const Cx<double> zs[4][3], const Cx<double> zf[4][3],
                           const Cx<double> xs[4][3], const Cx<double> xf[4][3], Cx<double> B[9], Cx<double> dU[9],
                           Cx<double> dUc[9]) {
  Cx<double> w1[4][3], pm[4][3], v2[4][3];
  // w1 = (1 - g) U x(s+mu); pm = (1 - g) x(s+mu); v2 = (1 + g) x(s)
  zero4(w1);
  term_fwd<double, MU>(xf, u, w1);
  proj_minus<MU>(xf, pm);
  proj_plus<MU>(xs, v2);
#pragma unroll
  for (int sp = 0; sp < 4; ++sp) {
    // q = U z(s+mu) for this spin
    Cx<double> q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        re = fma(u[3 * a + b].x, zf[sp][b].x, re);
        re = fma(-u[3 * a + b].y, zf[sp][b].y, re);
        im = fma(u[3 * a + b].x, zf[sp][b].y, im);
        im = fma(u[3 * a + b].y, zf[sp][b].x, im);
      }
      q[a] = mk<double>(re, im);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        // B[c][d] += w1_c conj(z_d) - v2_c conj(q_d)
        const Cx<double> a1 = w1[sp][c], z = zs[sp][d], v = v2[sp][c], qq = q[d];
        B[3 * c + d].x += a1.x * z.x + a1.y * z.y - (v.x * qq.x + v.y * qq.y);
        B[3 * c + d].y += a1.y * z.x - a1.x * z.y - (v.y * qq.x - v.x * qq.y);
        // dU[c][d] += conj(z_c) pm_d ;  dUc[c][d] += conj(z(s+mu)_d) v2_c
        const Cx<double> zc = zs[sp][c], pmd = pm[sp][d], zfd = zf[sp][d], vc = v2[sp][c];
        dU[3 * c + d].x += zc.x * pmd.x + zc.y * pmd.y;
        dU[3 * c + d].y += zc.x * pmd.y - zc.y * pmd.x;
        dUc[3 * c + d].x += zfd.x * vc.x + zfd.y * vc.y;
        dUc[3 * c + d].y += zfd.x * vc.y - zfd.y * vc.x;
      }
  }
}

// One thread per (site, direction): accumulates scale * sum over right-hand sides into grad
// (dT/dw_a, 8 per link) and, when given, into gU = dT/dU* + conj(dT/dU) (torch convention for Re T).
__global__ void link_grad_kernel(const double2 *__restrict__ U, double kappa, const double2 *__restrict__ z,
                                 const double2 *__restrict__ x, int nrhs, double scale, int Lx, int Ly, int Lz, int Lt,
                                 double2 *__restrict__ grad, double2 *__restrict__ gU) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int mu = blockIdx.y;
  const int V = Lx * Ly * Lz * Lt;
  if (s >= V) return;
  const int xx = s % Lx, y = (s / Lx) % Ly, zz = (s / (Lx * Ly)) % Lz, t = s / (Lx * Ly * Lz);
  int sf;
  if (mu == 0) sf = (xx + 1 == Lx) ? s - (Lx - 1) : s + 1;
  else if (mu == 1) sf = (y + 1 == Ly) ? s - (Ly - 1) * Lx : s + Lx;
  else if (mu == 2) sf = (zz + 1 == Lz) ? s - (Lz - 1) * Lx * Ly : s + Lx * Ly;
  else sf = (t + 1 == Lt) ? s - (Lt - 1) * Lx * Ly * Lz : s + Lx * Ly * Lz;
  Cx<double> u[9];
  load_link<double>(U, (long long)mu * V + s, u);
  Cx<double> B[9], dU[9], dUc[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) B[i] = dU[i] = dUc[i] = mk<double>(0.0, 0.0);
  for (int r = 0; r < nrhs; ++r) {
    const long long off = (long long)r * V * 12;
    Cx<double> zs[4][3], zf[4][3], xs[4][3], xf[4][3];
    load_spinor<double, false>(z + off + 12LL * s, zs);
    load_spinor<double, false>(z + off + 12LL * sf, zf);
    load_spinor<double, false>(x + off + 12LL * s, xs);
    load_spinor<double, false>(x + off + 12LL * sf, xf);
    if (mu == 0) link_terms<0>(u, zs, zf, xs, xf, B, dU, dUc);
    if (mu == 1) link_terms<1>(u, zs, zf, xs, xf, B, dU, dUc);
    if (mu == 2) link_terms<2>(u, zs, zf, xs, xf, B, dU, dUc);
    if (mu == 3) link_terms<3>(u, zs, zf, xs, xf, B, dU, dUc);
  }
  // dT/dw_a = (i kappa / 2) tr(lambda_a B)
  double2 *g = grad + ((long long)mu * V + s) * 8;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    double re = 0.0, im = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double lr = c_lambda[a][3 * c + d][0], li = c_lambda[a][3 * c + d][1];
        const Cx<double> b = B[3 * d + c];
        re += lr * b.x - li * b.y;
        im += lr * b.y + li * b.x;
      }
    // times i kappa / 2 and the caller's scale
    const double f = 0.5 * kappa * scale;
    double2 v = g[a];
    v.x += -f * im;
    v.y += f * re;
    g[a] = v;
  }
  if (gU) {
    double2 *o = gU + ((long long)mu * V + s) * 9;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      // dT/dU* + conj(dT/dU), both carrying kappa
      double2 v = o[i];
      v.x += scale * kappa * (dUc[i].x + dU[i].x);
      v.y += scale * kappa * (dUc[i].y - dU[i].y);
      o[i] = v;
    }
  }
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

lqcd_status link_grad_launch(lqcd_ctx *ctx, const double2 *U, double kappa, const double2 *z, const double2 *x,
                             int nrhs, double scale, double2 *grad, double2 *gU) {
  const int *d = ctx->dims;
  kbegin(ctx);
  link_grad_kernel<<<dim3(ceil_div(ctx->V, 128), 4), 128, 0, ctx->stream>>>(U, kappa, z, x, nrhs, scale, d[0], d[1],
                                                                          d[2], d[3], grad, gU);
  return launch_check(ctx, "link_grad_kernel", K_CONTRACT, (double)ctx->V * 4 * nrhs);
}

extern "C" lqcd_status lqcd_link_grad(lqcd_ctx *ctx, const double *links, double kappa, const double *z, const double *x,
                                      int nrhs, double scale, double *grad, double *grad_links) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_full(ctx, "link_grad"));
  if (!links || !z || !x || !grad || nrhs < 1) return set_err(ctx, LQCD_ERR_INVALID_ARG, "link_grad: bad arguments");
  return link_grad_launch(ctx, (const double2 *)links, kappa, (const double2 *)z, (const double2 *)x, nrhs, scale,
                          (double2 *)grad, (double2 *)grad_links);
}

// ---- derivatives of the loop estimates -------------------------------------------------------------
lqcd_status proj_core_entry(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_defl *defl, const double2 *b,
                            double2 *x, int nrhs, const lqcd_krylov_opts *o, lqcd_solve_info *info);
lqcd_status hop_series_launch(lqcd_ctx *ctx, const double2 *U, double kappa, const double2 *eta, double2 *out, int nrhs,
                              int K, const cd *c);
lqcd_status hop_traces_launch(lqcd_ctx *ctx, const double2 *U, double kappa, int K, std::vector<cd> &tr);

extern "C" lqcd_status lqcd_loop_derivs(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_est_opts *o,
                                        lqcd_derivs *out) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_full(ctx, "loop_derivs"));
  if (!links || !o || !out) return set_err(ctx, LQCD_ERR_INVALID_ARG, "loop_derivs: NULL argument");
  if (o->nnoise < 1 || o->block < 1 || o->m < 2 || o->k < 1 || o->k >= o->m || o->K < 1 || o->K > 64 ||
      !(o->tol > 0) || !(o->tol_special > 0) || o->max_cycles < 1 || !(kappa != 0.0))
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "loop_derivs: bad options");
  if (o->prec < LQCD_PREC_F64 || o->prec > LQCD_PREC_BF16)
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "loop_derivs: prec must be one of LQCD_PREC_*");
  if (o->system != LQCD_SYS_M && o->system != LQCD_SYS_MG5)
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "loop_derivs: system must be LQCD_SYS_M or LQCD_SYS_MG5");
  if (o->evenodd) return set_err(ctx, LQCD_ERR_INVALID_ARG, "loop_derivs: even/odd solves are not available here");
  const double t0 = now_s();
  const double2 *U = (const double2 *)links;
  const int Lt = ctx->dims[3];
  const long long N = ctx->N;
  const int nn = o->nnoise;
  // deflation space for GMRES-Proj from the special right-hand side (GMRES-DR on M)
  double2 *bs = nullptr, *xs = nullptr;
  LQCD_CUDA(ctx, cudaMalloc(&bs, sizeof(double2) * (size_t)N * 2));
  xs = bs + N;
  lqcd_defl *dm = nullptr;
  struct Guard {
    void *p;
    lqcd_defl **d;
    ~Guard() {
      if (p) cudaFree(p);
      if (*d) lqcd_defl_destroy(*d);
    }
  } guard{bs, &dm};
  LQCD_TRY(noise_launch(ctx, o->seed, 0xFFFFFFFEu, 1, bs));
  lqcd_krylov_opts ko{o->m, o->k, o->tol_special, o->max_cycles, LQCD_SYS_M, LQCD_PREC_F64, 0.0, o->eig_tol};
  lqcd_solve_info si{};
  // system M: GMRES-DR on M; the Hermitian path: MINRES-DR on M' = M gamma_5, and every solve of
  // M x = b below is M' y = b, x = gamma_5 y
  const bool herm = o->system == LQCD_SYS_MG5;
  lqcd_status st = herm ? lqcd_minresdr_solve(ctx, links, kappa, (const double *)bs, (double *)xs, 1, &ko, &si, &dm)
                        : lqcd_gmresdr_solve(ctx, links, kappa, (const double *)bs, (double *)xs, 1, &ko, &si, &dm);
  if (st != LQCD_OK && st != LQCD_ERR_NOT_CONVERGED) return st;
  if (!dm) return set_err(ctx, LQCD_ERR_NOT_CONVERGED, "loop_derivs: no deflation space");
  long matvecs = si.matvecs;
  // PS add-back derivative per timeslice: sum_k k kappa^{k-1} t_k (+ point-split: sum_k kappa^k t_k / kappa)
  std::vector<cd> tr;
  LQCD_TRY(hop_traces_launch(ctx, U, kappa, o->K, tr));
  std::vector<cd> dadd((size_t)9 * Lt, cd(0.0, 0.0));
  for (int op = 0; op < 9; ++op)
    for (int t = 0; t < Lt; ++t) {
      cd v = 0.0, w = 0.0;
      for (int k = 0; k < o->K; ++k) {
        const cd tk = tr[((size_t)k * 9 + op) * Lt + t];
        if (k >= 1) v += (double)k * std::pow(kappa, k - 1) * tk;
        w += std::pow(kappa, k) * tk;
      }
      if (op >= 5) v += w / kappa;
      dadd[(size_t)op * Lt + t] = v;
    }
  // noise blocks
  const int bw = std::min(o->block, nn);
  const long long bn = (long long)bw * N;
  double2 *eta;
  LQCD_CUDA(ctx, cudaMalloc(&eta, sizeof(double2) * (size_t)bn * 9));
  struct Guard2 { void *p; ~Guard2() { if (p) cudaFree(p); } } g2{eta};
  double2 *x = eta + bn, *px = x + bn, *y = px + bn, *g5e = y + bn, *w = g5e + bn, *xp = w + bn, *dxp = xp + bn;
  double2 *hy = dxp + bn;  // the Hermitian path's M' solution before gamma_5
  double2 *cdv;
  LQCD_TRY(ws_get(ctx, WS_EST0, sizeof(double2) * (size_t)bw * 9 * Lt * 4, (void **)&cdv));
  if (out->link_grad) LQCD_CUDA(ctx, cudaMemsetAsync(out->link_grad, 0, sizeof(double2) * (size_t)ctx->V * 32, ctx->stream));
  if (out->grad_links) LQCD_CUDA(ctx, cudaMemsetAsync(out->grad_links, 0, sizeof(double2) * (size_t)ctx->V * 36, ctx->stream));
  lqcd_krylov_opts po{o->m_inner > 0 ? o->m_inner : o->m - o->k, 0, o->tol, o->max_cycles, LQCD_SYS_M, o->prec, o->inner_tol};
  std::vector<cd> per((size_t)2 * nn * 9, cd(0.0, 0.0));
  std::vector<cd> ck(o->K);
  for (int k = 0; k < o->K; ++k) ck[k] = cd((double)k / kappa, 0.0);  // sum (k/kappa)(kappa P)^k = d/dkappa sum (kappa P)^k
  double worst = 0.0;
  int conv = 1;
  std::vector<double2> h;
  for (int first = 0; first < nn; first += bw) {
    const int nb = std::min(bw, nn - first);
    const long long len = (long long)nb * N;
    LQCD_TRY(noise_launch(ctx, o->seed, (uint32_t)first, nb, eta));
    lqcd_solve_info a{}, b{}, c{};
    // x = M^{-1} rhs (directly, or gamma_5 M'^{-1} rhs on the Hermitian path)
    auto solve = [&](const double2 *rhs, double2 *xo, lqcd_solve_info *inf) -> lqcd_status {
      const lqcd_status s2 = proj_core_entry(ctx, links, kappa, dm, rhs, herm ? hy : xo, nb, &po, inf);
      if (s2 != LQCD_OK && s2 != LQCD_ERR_NOT_CONVERGED) return s2;
      return herm ? blas_g5(ctx, hy, xo, nb) : LQCD_OK;
    };
    LQCD_TRY(solve(eta, x, &a));
    LQCD_TRY(wilson_launch(ctx, U, kappa, x, px, nb, LQCD_PREC_F64, LQCD_APPLY_HOP));
    LQCD_TRY(solve(px, y, &b));
    LQCD_TRY(blas_g5(ctx, eta, g5e, nb));
    LQCD_TRY(solve(g5e, w, &c));
    LQCD_TRY(blas_g5(ctx, w, g5e, nb));  // z = g5 M^{-1} g5 eta (reuses the g5e buffer)
    for (const lqcd_solve_info *i : {&a, &b, &c}) {
      matvecs += i->matvecs;
      worst = std::max(worst, i->true_resid);
      if (!i->converged) conv = 0;
    }
    LQCD_TRY(hop_series_launch(ctx, U, kappa, eta, xp, nb, o->K, nullptr));
    LQCD_TRY(hop_series_launch(ctx, U, kappa, eta, dxp, nb, o->K, ck.data()));
    const size_t sl = (size_t)nb * 9 * Lt;
    LQCD_TRY(contract_launch(ctx, U, kappa, eta, y, nb, cdv));
    LQCD_TRY(contract_launch(ctx, U, kappa, eta, x, nb, cdv + sl));
    LQCD_TRY(contract_launch(ctx, U, kappa, eta, dxp, nb, cdv + 2 * sl));
    LQCD_TRY(contract_launch(ctx, U, kappa, eta, xp, nb, cdv + 3 * sl));
    if (out->link_grad)
      LQCD_TRY(link_grad_launch(ctx, U, kappa, g5e, x, nb, out->grad_scale / nn, (double2 *)out->link_grad,
                                (double2 *)out->grad_links));
    h.resize(4 * sl);
    LQCD_CUDA(ctx, cudaMemcpyAsync(h.data(), cdv, sizeof(double2) * 4 * sl, cudaMemcpyDeviceToHost, ctx->stream));
    LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int r = 0; r < nb; ++r)
      for (int op = 0; op < 9; ++op) {
        cd sy = 0.0, sx = 0.0, sdp = 0.0, sp = 0.0;
        for (int t = 0; t < Lt; ++t) {
          const size_t i = ((size_t)r * 9 + op) * Lt + t;
          sy += cd(h[i].x, h[i].y);
          sx += cd(h[sl + i].x, h[sl + i].y);
          sdp += cd(h[2 * sl + i].x, h[2 * sl + i].y);
          sp += cd(h[3 * sl + i].x, h[3 * sl + i].y);
        }
        cd none = sy, pert = sy - sdp;
        if (op >= 5) {
          none += sx / kappa;
          pert += (sx - sp) / kappa;
        }
        per[((size_t)0 * nn + first + r) * 9 + op] = none;
        per[((size_t)1 * nn + first + r) * 9 + op] = pert;
      }
    (void)len;
  }
  // summary: mean and error bar of the signal part (Re scalar, Im vector) per mode and operator
  for (int mode = 0; mode < 2; ++mode)
    for (int op = 0; op < 9; ++op) {
      cd addtot = 0.0;
      if (mode == 1)
        for (int t = 0; t < Lt; ++t) addtot += dadd[(size_t)op * Lt + t];
      cd mean = 0.0;
      double pm = 0.0;
      for (int n = 0; n < nn; ++n) {
        const cd v = per[((size_t)mode * nn + n) * 9 + op] + addtot;
        if (out->per_noise) {
          out->per_noise[(((size_t)mode * nn + n) * 9 + op) * 2] = v.real();
          out->per_noise[(((size_t)mode * nn + n) * 9 + op) * 2 + 1] = v.imag();
        }
        mean += v;
        pm += (op == 0) ? v.real() : v.imag();
      }
      mean /= (double)nn;
      pm /= nn;
      double ss = 0.0;
      for (int n = 0; n < nn; ++n) {
        const cd v = per[((size_t)mode * nn + n) * 9 + op] + addtot;
        const double d = ((op == 0) ? v.real() : v.imag()) - pm;
        ss += d * d;
      }
      if (out->dkappa) {
        out->dkappa[((size_t)mode * 9 + op) * 2] = mean.real();
        out->dkappa[((size_t)mode * 9 + op) * 2 + 1] = mean.imag();
      }
      if (out->dkappa_err) out->dkappa_err[(size_t)mode * 9 + op] = nn > 1 ? std::sqrt(ss / (nn - 1) / nn) : NAN;
    }
  LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  out->matvecs = matvecs;
  out->seconds = now_s() - t0;
  out->max_true_resid = worst;
  out->converged = conv;
  return conv ? LQCD_OK : set_err(ctx, LQCD_ERR_NOT_CONVERGED, "loop_derivs: a solve did not converge (rel %.3e)", worst);
}
