// Wilson-Dirac operator M = 1 - kappa P (Eq. xyz556) on blocks of right-hand sides.
//
// One thread owns one (site, right-hand side) pair and produces its 12 output components.  Each
// of the eight hopping terms is computed in the two-component ("half spinor") form: the spin
// projector (1 -+ gamma_mu) has rank two in the Dirac basis, so the neighbour spinor is projected
// to 2 spin x 3 colour components, multiplied by the colour matrix U_mu(x) or U_mu(x-mu)^dag, and
// the lower two spin components are rebuilt from the upper ones by a fixed phase permutation.
// That is 2 x 9 complex multiply-adds per term instead of 4 x 9.
//
// Dirac-basis projections used below (h = upper pair after projection, rows 2,3 = rebuilt lower):
//   mu = x:  1 - g: h = (p0 + i p3, p1 + i p2), lower = (-i h1, -i h0)
//            1 + g: h = (p0 - i p3, p1 - i p2), lower = ( i h1,  i h0)
//   mu = y:  1 - g: h = (p0 + p3,   p1 - p2),   lower = (-h1,  h0)
//            1 + g: h = (p0 - p3,   p1 + p2),   lower = ( h1, -h0)
//   mu = z:  1 - g: h = (p0 + i p2, p1 - i p3), lower = (-i h0,  i h1)
//            1 + g: h = (p0 - i p2, p1 + i p3), lower = ( i h0, -i h1)
//   mu = t:  1 - g = diag(0,0,2,2): only the lower pair, (2 p2, 2 p3)
//            1 + g = diag(2,2,0,0): only the upper pair, (2 p0, 2 p1)
// gamma_5 = -[[0, 1], [1, 0]] in this basis: (g5 p) = (-p2, -p3, -p0, -p1).
#include "common.cuh"
#include "spin.cuh"

namespace {

using namespace spin;

template <typename R>
__device__ __forceinline__ void g5_inplace(Cx<R> p[4][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Cx<R> a0 = p[0][c], a1 = p[1][c];
    p[0][c] = neg(p[2][c]);
    p[1][c] = neg(p[3][c]);
    p[2][c] = neg(a0);
    p[3][c] = neg(a1);
  }
}

// MODE: 0 = M, 1 = M g5, 2 = M^dag = g5 M g5, 3 = P, 4 = per right-hand side M or M g5 (bit r of
// g5mask set: M g5).  R: arithmetic; S: storage of spinors and links (double2 with R = double or
// float; float2 with R = float).
template <typename R, int MODE, typename S>
__global__ void __launch_bounds__(128) wilson_kernel(const S *__restrict__ U, const S *__restrict__ in,
                                                     S *__restrict__ out, double kappa, int Lx, int Ly,
                                                     int Lz, int Lt, int V, unsigned long long g5mask) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  constexpr bool G5IN = (MODE == 1 || MODE == 2);
  const bool g5rt = (MODE == 4) && ((g5mask >> blockIdx.y) & 1ull);
  const long long base = (long long)blockIdx.y * V * 12;
  const S *src = in + base;
  int x = s % Lx;
  int r = s / Lx;
  int y = r % Ly;
  r /= Ly;
  int z = r % Lz;
  int t = r / Lz;
  const int sx = 1, sy = Lx, sz = Lx * Ly, st = Lx * Ly * Lz;
  const int xp = (x + 1 == Lx) ? s - (Lx - 1) * sx : s + sx;
  const int xm = (x == 0) ? s + (Lx - 1) * sx : s - sx;
  const int yp = (y + 1 == Ly) ? s - (Ly - 1) * sy : s + sy;
  const int ym = (y == 0) ? s + (Ly - 1) * sy : s - sy;
  const int zp = (z + 1 == Lz) ? s - (Lz - 1) * sz : s + sz;
  const int zm = (z == 0) ? s + (Lz - 1) * sz : s - sz;
  const int tp = (t + 1 == Lt) ? s - (Lt - 1) * st : s + st;
  const int tm = (t == 0) ? s + (Lt - 1) * st : s - st;

  Cx<R> acc[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[a][c] = mk<R>(0, 0);
  Cx<R> p[4][3], u[9];
  const long long V4 = V;
  load_spinor<R, G5IN>(src + 12LL * xp, p); if (g5rt) g5_inplace(p); load_link<R>(U, 0 * V4 + s, u); term_fwd<R, 0>(p, u, acc);
  load_spinor<R, G5IN>(src + 12LL * xm, p); if (g5rt) g5_inplace(p); load_link<R>(U, 0 * V4 + xm, u); term_bwd<R, 0>(p, u, acc);
  load_spinor<R, G5IN>(src + 12LL * yp, p); if (g5rt) g5_inplace(p); load_link<R>(U, 1 * V4 + s, u); term_fwd<R, 1>(p, u, acc);
  load_spinor<R, G5IN>(src + 12LL * ym, p); if (g5rt) g5_inplace(p); load_link<R>(U, 1 * V4 + ym, u); term_bwd<R, 1>(p, u, acc);
  load_spinor<R, G5IN>(src + 12LL * zp, p); if (g5rt) g5_inplace(p); load_link<R>(U, 2 * V4 + s, u); term_fwd<R, 2>(p, u, acc);
  load_spinor<R, G5IN>(src + 12LL * zm, p); if (g5rt) g5_inplace(p); load_link<R>(U, 2 * V4 + zm, u); term_bwd<R, 2>(p, u, acc);
  load_spinor<R, G5IN>(src + 12LL * tp, p); if (g5rt) g5_inplace(p); load_link<R>(U, 3 * V4 + s, u); term_fwd<R, 3>(p, u, acc);
  load_spinor<R, G5IN>(src + 12LL * tm, p); if (g5rt) g5_inplace(p); load_link<R>(U, 3 * V4 + tm, u); term_bwd<R, 3>(p, u, acc);

  S *dst = out + base + 12LL * s;
  if (MODE == 3) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) store_c(dst + 3 * a + c, acc[a][c]);
    return;
  }
  load_spinor<R, G5IN>(src + 12LL * s, p);
  if (g5rt) g5_inplace(p);
  const R k = (R)kappa;
  Cx<R> o[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) o[a][c] = mk<R>(fma(-k, acc[a][c].x, p[a][c].x), fma(-k, acc[a][c].y, p[a][c].y));
  if (MODE == 2) {  // left gamma_5
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Cx<R> a0 = o[0][c], a1 = o[1][c];
      o[0][c] = neg(o[2][c]);
      o[1][c] = neg(o[3][c]);
      o[2][c] = neg(a0);
      o[3][c] = neg(a1);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) store_c(dst + 3 * a + c, o[a][c]);
}

template <typename R, typename S>
lqcd_status launch_mode(lqcd_ctx *ctx, const S *U, double kappa, const S *in, S *out, int nrhs, int flags,
                        unsigned long long g5mask = 0) {
  // 128 threads per block unless that leaves fewer than two blocks per SM (few right-hand sides on
  // a small lattice): then smaller blocks spread the sites over more SMs
  int bs = 128;
  while (bs > 32 && (long long)ceil_div(ctx->V, bs) * nrhs < 2LL * ctx->sms) bs /= 2;
  dim3 block(bs);
  dim3 grid(ceil_div(ctx->V, bs), nrhs);
  const int *d = ctx->dims;
  kbegin(ctx);
  switch (flags) {
    case LQCD_APPLY_M: wilson_kernel<R, 0, S><<<grid, block, 0, ctx->stream>>>(U, in, out, kappa, d[0], d[1], d[2], d[3], ctx->V, 0ull); break;
    case LQCD_APPLY_G5R: wilson_kernel<R, 1, S><<<grid, block, 0, ctx->stream>>>(U, in, out, kappa, d[0], d[1], d[2], d[3], ctx->V, 0ull); break;
    case LQCD_APPLY_DAG: wilson_kernel<R, 2, S><<<grid, block, 0, ctx->stream>>>(U, in, out, kappa, d[0], d[1], d[2], d[3], ctx->V, 0ull); break;
    case LQCD_APPLY_HOP: wilson_kernel<R, 3, S><<<grid, block, 0, ctx->stream>>>(U, in, out, kappa, d[0], d[1], d[2], d[3], ctx->V, 0ull); break;
    case 4: wilson_kernel<R, 4, S><<<grid, block, 0, ctx->stream>>>(U, in, out, kappa, d[0], d[1], d[2], d[3], ctx->V, g5mask); break;
    default: return set_err(ctx, LQCD_ERR_INVALID_ARG, "wilson_apply: unknown flags %d", flags);
  }
  return launch_check(ctx, "wilson_kernel", K_WILSON, (double)ctx->V * nrhs);
}

}  // namespace

lqcd_status wilson_launch(lqcd_ctx *ctx, const double2 *U, double kappa, const double2 *in, double2 *out, int nrhs,
                          int prec, int flags) {
  if (nrhs <= 0 || nrhs > 65535) return set_err(ctx, LQCD_ERR_INVALID_ARG, "wilson_apply: nrhs %d out of range", nrhs);
  if (prec == LQCD_PREC_F64) return launch_mode<double, double2>(ctx, U, kappa, in, out, nrhs, flags);
  if (prec == LQCD_PREC_F32) return launch_mode<float, double2>(ctx, U, kappa, in, out, nrhs, flags);
  return set_err(ctx, LQCD_ERR_INVALID_ARG, "wilson_apply: unknown precision %d", prec);
}

lqcd_status wilson_launch_masked(lqcd_ctx *ctx, const double2 *U, double kappa, const double2 *in, double2 *out,
                                 int nrhs, unsigned long long g5mask) {
  if (nrhs <= 0 || nrhs > 64) return set_err(ctx, LQCD_ERR_INVALID_ARG, "wilson (masked): nrhs %d out of range", nrhs);
  return launch_mode<double, double2>(ctx, U, kappa, in, out, nrhs, 4, g5mask);
}

lqcd_status wilson_launch_f32(lqcd_ctx *ctx, const float2 *U, double kappa, const float2 *in, float2 *out, int nrhs,
                              int flags) {
  if (nrhs <= 0 || nrhs > 65535) return set_err(ctx, LQCD_ERR_INVALID_ARG, "wilson (f32): nrhs %d out of range", nrhs);
  return launch_mode<float, float2>(ctx, U, kappa, in, out, nrhs, flags);
}

extern "C" lqcd_status lqcd_wilson_apply(lqcd_ctx *ctx, const double *links, double kappa, const double *in,
                                         double *out, int nrhs, int prec, int flags) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  if (!links || !in || !out) return set_err(ctx, LQCD_ERR_INVALID_ARG, "wilson_apply: NULL pointer");
  if (in == out) return set_err(ctx, LQCD_ERR_INVALID_ARG, "wilson_apply: in and out must not overlap");
  return wilson_launch(ctx, (const double2 *)links, kappa, (const double2 *)in, (double2 *)out, nrhs, prec, flags);
}

extern "C" lqcd_status lqcd_wilson_apply_f32(lqcd_ctx *ctx, const float *links32, double kappa, const float *in,
                                             float *out, int nrhs, int flags) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  if (!links32 || !in || !out) return set_err(ctx, LQCD_ERR_INVALID_ARG, "wilson_apply_f32: NULL pointer");
  if (in == out) return set_err(ctx, LQCD_ERR_INVALID_ARG, "wilson_apply_f32: in and out must not overlap");
  if (flags < 0 || flags > 3) return set_err(ctx, LQCD_ERR_INVALID_ARG, "wilson_apply_f32: unknown flags %d", flags);
  return wilson_launch_f32(ctx, (const float2 *)links32, kappa, (const float2 *)in, (float2 *)out, nrhs, flags);
}

extern "C" lqcd_status lqcd_to_f32(lqcd_ctx *ctx, const double *in, float *out, long long n) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  if (!in || !out || n < 0) return set_err(ctx, LQCD_ERR_INVALID_ARG, "to_f32: bad arguments");
  return blas_to_f32(ctx, (const double2 *)in, (float2 *)out, n);
}
