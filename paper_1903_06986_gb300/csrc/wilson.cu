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
  // compulsory bytes: each field read and written once, the links once
  const double bytes = 2.0 * nrhs * ctx->V * 12 * sizeof(S) + 36.0 * ctx->V * sizeof(S);
  return launch_check_bytes(ctx, "wilson_kernel", K_WILSON, (double)ctx->V * nrhs, bytes);
}

}  // namespace

lqcd_status wilson_launch(lqcd_ctx *ctx, const double2 *U, double kappa, const double2 *in, double2 *out, int nrhs,
                          int prec, int flags) {
  if (nrhs <= 0 || nrhs > 65535) return set_err(ctx, LQCD_ERR_INVALID_ARG, "wilson_apply: nrhs %d out of range", nrhs);
  if (ctx->eo) return eo_schur_launch(ctx, U, kappa, in, out, nrhs, prec, flags);
  if (prec == LQCD_PREC_F64) return launch_mode<double, double2>(ctx, U, kappa, in, out, nrhs, flags);
  if (prec == LQCD_PREC_F32) return launch_mode<float, double2>(ctx, U, kappa, in, out, nrhs, flags);
  return set_err(ctx, LQCD_ERR_INVALID_ARG, "wilson_apply: unknown precision %d", prec);
}

lqcd_status wilson_launch_masked(lqcd_ctx *ctx, const double2 *U, double kappa, const double2 *in, double2 *out,
                                 int nrhs, unsigned long long g5mask) {
  if (nrhs <= 0 || nrhs > 64) return set_err(ctx, LQCD_ERR_INVALID_ARG, "wilson (masked): nrhs %d out of range", nrhs);
  LQCD_TRY(require_full(ctx, "wilson (masked)"));
  return launch_mode<double, double2>(ctx, U, kappa, in, out, nrhs, 4, g5mask);
}

lqcd_status wilson_launch_f32(lqcd_ctx *ctx, const float2 *U, double kappa, const float2 *in, float2 *out, int nrhs,
                              int flags) {
  if (nrhs <= 0 || nrhs > 65535) return set_err(ctx, LQCD_ERR_INVALID_ARG, "wilson (f32): nrhs %d out of range", nrhs);
  LQCD_TRY(require_full(ctx, "wilson_apply_f32"));
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

// ---- packed FP32 operator (the inner operator of mixed precision) ---------------------------------
// Packed layout of FP32 fields: the 24 reals of a site (canonical order spin, colour, re/im) are six
// float4 chunks, chunk q holding complex components 2q and 2q+1, stored chunk-major per right-hand
// side: element (r, q, s) at [(r * 6 + q) * V + s].  A warp of consecutive sites then reads 512
// contiguous bytes per chunk.  Links are packed per direction the same way: with RECON = 12 only
// rows 0 and 1 are stored (three float4: (u00,u01), (u02,u10), (u11,u12)) and row 2 is rebuilt as
// conj(row0 x row1), exact for SU(3); with RECON = 18 all nine entries are stored in five float4
// (the last half padded).  One thread owns one site for NR right-hand sides, so every link is
// loaded once per NR right-hand sides.
namespace {

using namespace spin;

template <int RECON>
__device__ __forceinline__ void load_link_packed(const float4 *__restrict__ U, int mu, int V, int s, Cx<float> u[9]) {
  constexpr int NC = RECON == 12 ? 3 : 5;
  const float4 *p = U + (long long)mu * NC * V + s;
  const float4 a = __ldg(p), b = __ldg(p + V), c = __ldg(p + 2LL * V);
  u[0] = mk<float>(a.x, a.y); u[1] = mk<float>(a.z, a.w);
  u[2] = mk<float>(b.x, b.y); u[3] = mk<float>(b.z, b.w);
  u[4] = mk<float>(c.x, c.y); u[5] = mk<float>(c.z, c.w);
  if (RECON == 12) {
    // row 2 = conj(row0 x row1)
    auto cm = [](Cx<float> x, Cx<float> y) { return mk<float>(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x); };
    Cx<float> t;
    t = cm(u[1], u[5]) - cm(u[2], u[4]); u[6] = mk<float>(t.x, -t.y);
    t = cm(u[2], u[3]) - cm(u[0], u[5]); u[7] = mk<float>(t.x, -t.y);
    t = cm(u[0], u[4]) - cm(u[1], u[3]); u[8] = mk<float>(t.x, -t.y);
  } else {
    const float4 d = __ldg(p + 3LL * V), e = __ldg(p + 4LL * V);
    u[6] = mk<float>(d.x, d.y); u[7] = mk<float>(d.z, d.w);
    u[8] = mk<float>(e.x, e.y);
  }
}

// A chunk of the packed layout: two complex components of one site, as one float4 (FP32) or as an
// 8-byte pair of FP16 / BF16 complex numbers; Chunk<S>::get / put convert to and from FP32.
struct alignas(8) h2x2 { __half2 a, b; };
struct alignas(8) b2x2 { __nv_bfloat162 a, b; };
template <typename S> struct Chunk;
template <> struct Chunk<float2> {
  using T = float4;
  static __device__ __forceinline__ void get(const T *p, Cx<float> &a, Cx<float> &b) {
    const float4 v = __ldg(p);
    a = mk<float>(v.x, v.y);
    b = mk<float>(v.z, v.w);
  }
  static __device__ __forceinline__ void put(T *p, Cx<float> a, Cx<float> b) { *p = make_float4(a.x, a.y, b.x, b.y); }
};
template <> struct Chunk<__half2> {
  using T = h2x2;
  static __device__ __forceinline__ void get(const T *__restrict__ p, Cx<float> &a, Cx<float> &b) {
    const T v = *p;
    const float2 fa = __half22float2(v.a), fb = __half22float2(v.b);
    a = mk<float>(fa.x, fa.y);
    b = mk<float>(fb.x, fb.y);
  }
  static __device__ __forceinline__ void put(T *p, Cx<float> a, Cx<float> b) {
    T v;
    v.a = __floats2half2_rn(a.x, a.y);
    v.b = __floats2half2_rn(b.x, b.y);
    *p = v;
  }
};
template <> struct Chunk<__nv_bfloat162> {
  using T = b2x2;
  static __device__ __forceinline__ void get(const T *__restrict__ p, Cx<float> &a, Cx<float> &b) {
    const T v = *p;
    const float2 fa = __bfloat1622float2(v.a), fb = __bfloat1622float2(v.b);
    a = mk<float>(fa.x, fa.y);
    b = mk<float>(fb.x, fb.y);
  }
  static __device__ __forceinline__ void put(T *p, Cx<float> a, Cx<float> b) {
    T v;
    v.a = __floats2bfloat162_rn(a.x, a.y);
    v.b = __floats2bfloat162_rn(b.x, b.y);
    *p = v;
  }
};

template <typename S>
__device__ __forceinline__ void load_spinor_packed(const typename Chunk<S>::T *__restrict__ p, int V, Cx<float> s[4][3]) {
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const int c0 = 2 * q, c1 = 2 * q + 1;
    Chunk<S>::get(p + (long long)q * V, s[c0 / 3][c0 % 3], s[c1 / 3][c1 % 3]);
  }
}

template <typename S>
__device__ __forceinline__ void store_spinor_packed(typename Chunk<S>::T *__restrict__ p, int V, const Cx<float> s[4][3]) {
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const int c0 = 2 * q, c1 = 2 * q + 1;
    Chunk<S>::put(p + (long long)q * V, s[c0 / 3][c0 % 3], s[c1 / 3][c1 % 3]);
  }
}

template <typename S, int NR, int RECON, int MODE>
__global__ void __launch_bounds__(128) wilson_packed_kernel(const float4 *__restrict__ U,
                                                            const typename Chunk<S>::T *__restrict__ in,
                                                            typename Chunk<S>::T *__restrict__ out, float kappa,
                                                            int Lx, int Ly, int Lz, int Lt, int V, int nrhs,
                                                            int groups) {
  // the right-hand-side group varies fastest along the grid, so the blocks of all groups of one
  // site block run together and read its links (and neighbour spinor lines) from L2, not DRAM
  const int s = (blockIdx.x / groups) * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const int r0 = (blockIdx.x % groups) * NR;
  const int nr = min(NR, nrhs - r0);
  constexpr bool G5IN = (MODE == 1 || MODE == 2);
  int x = s % Lx, rr = s / Lx;
  int y = rr % Ly;
  rr /= Ly;
  int z = rr % Lz;
  int t = rr / Lz;
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
  Cx<float> acc[NR][4][3];
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[r][a][c] = mk<float>(0.f, 0.f);
  Cx<float> u[9], p[4][3];
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    const int mu = d >> 1;
    const bool fwd = (d & 1) == 0;
    load_link_packed<RECON>(U, mu, V, fwd ? s : nb[d], u);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (r < nr) {
        load_spinor_packed<S>(in + (long long)(r0 + r) * 6 * V + nb[d], V, p);
        if (G5IN) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            Cx<float> a0 = p[0][c], a1 = p[1][c];
            p[0][c] = neg(p[2][c]); p[1][c] = neg(p[3][c]); p[2][c] = neg(a0); p[3][c] = neg(a1);
          }
        }
        if (fwd) {
          if (mu == 0) term_fwd<float, 0>(p, u, acc[r]);
          if (mu == 1) term_fwd<float, 1>(p, u, acc[r]);
          if (mu == 2) term_fwd<float, 2>(p, u, acc[r]);
          if (mu == 3) term_fwd<float, 3>(p, u, acc[r]);
        } else {
          if (mu == 0) term_bwd<float, 0>(p, u, acc[r]);
          if (mu == 1) term_bwd<float, 1>(p, u, acc[r]);
          if (mu == 2) term_bwd<float, 2>(p, u, acc[r]);
          if (mu == 3) term_bwd<float, 3>(p, u, acc[r]);
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    if (r >= nr) break;
    typename Chunk<S>::T *dst = out + (long long)(r0 + r) * 6 * V + s;
    if (MODE == 3) {
      store_spinor_packed<S>(dst, V, acc[r]);
      continue;
    }
    load_spinor_packed<S>(in + (long long)(r0 + r) * 6 * V + s, V, p);
    if (G5IN) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Cx<float> a0 = p[0][c], a1 = p[1][c];
        p[0][c] = neg(p[2][c]); p[1][c] = neg(p[3][c]); p[2][c] = neg(a0); p[3][c] = neg(a1);
      }
    }
    Cx<float> o[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        o[a][c] = mk<float>(fmaf(-kappa, acc[r][a][c].x, p[a][c].x), fmaf(-kappa, acc[r][a][c].y, p[a][c].y));
    if (MODE == 2) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Cx<float> a0 = o[0][c], a1 = o[1][c];
        o[0][c] = neg(o[2][c]); o[1][c] = neg(o[3][c]); o[2][c] = neg(a0); o[3][c] = neg(a1);
      }
    }
    store_spinor_packed<S>(dst, V, o);
  }
}

// ---- paired-lane variant: two right-hand sides per thread in the two lanes of packed FP32
// arithmetic (__fadd2_rn / __fmul2_rn / __ffma2_rn, one instruction for both lanes).  The stencil
// code is the scalar one instantiated on the lane pair P2; the links are shared by both lanes
// (loaded and rebuilt once), the spinors of the two right-hand sides are paired component by
// component when loaded and split when stored.
struct P2 {
  float2 v;
};
__device__ __forceinline__ P2 p2(float a, float b) { return P2{make_float2(a, b)}; }
__device__ __forceinline__ P2 operator+(P2 a, P2 b) { return P2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ P2 operator-(P2 a) { return P2{make_float2(-a.v.x, -a.v.y)}; }
__device__ __forceinline__ P2 operator-(P2 a, P2 b) { return P2{__fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y))}; }
__device__ __forceinline__ P2 operator*(P2 a, P2 b) { return P2{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ P2 fma(P2 a, P2 b, P2 c) { return P2{__ffma2_rn(a.v, b.v, c.v)}; }
using ::fma;  // keep the math overloads visible next to the lane-pair one

// spinors of right-hand sides r and r + 1 (pointers a, b, chunk-major) -> lane pairs
template <typename S> struct PairIO;
template <> struct PairIO<float2> {
  using T = float4;
  static __device__ __forceinline__ void load(const T *__restrict__ a, const T *__restrict__ b, int V, Cx<P2> s[4][3]) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const float4 u = __ldg(a + (long long)q * V), w = __ldg(b + (long long)q * V);
      const int c0 = 2 * q, c1 = 2 * q + 1;
      s[c0 / 3][c0 % 3] = mk<P2>(p2(u.x, w.x), p2(u.y, w.y));
      s[c1 / 3][c1 % 3] = mk<P2>(p2(u.z, w.z), p2(u.w, w.w));
    }
  }
  static __device__ __forceinline__ void store(T *a, T *b, int V, const Cx<P2> s[4][3], bool second) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const Cx<P2> e = s[(2 * q) / 3][(2 * q) % 3], f = s[(2 * q + 1) / 3][(2 * q + 1) % 3];
      a[(long long)q * V] = make_float4(e.x.v.x, e.y.v.x, f.x.v.x, f.y.v.x);
      if (second) b[(long long)q * V] = make_float4(e.x.v.y, e.y.v.y, f.x.v.y, f.y.v.y);
    }
  }
};
template <typename H, typename T2, H (*LO)(H, H), H (*HI)(H, H), float2 (*TOF)(H), H (*FROMF)(float2)>
struct PairIOHalf {
  using T = T2;
  static __device__ __forceinline__ void load(const T *__restrict__ a, const T *__restrict__ b, int V, Cx<P2> s[4][3]) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const T u = a[(long long)q * V], w = b[(long long)q * V];
      const int c0 = 2 * q, c1 = 2 * q + 1;
      // (re_r, im_r) and (re_r+1, im_r+1) -> (re_r, re_r+1) and (im_r, im_r+1), then to FP32
      s[c0 / 3][c0 % 3] = mk<P2>(P2{TOF(LO(u.a, w.a))}, P2{TOF(HI(u.a, w.a))});
      s[c1 / 3][c1 % 3] = mk<P2>(P2{TOF(LO(u.b, w.b))}, P2{TOF(HI(u.b, w.b))});
    }
  }
  static __device__ __forceinline__ void store(T *a, T *b, int V, const Cx<P2> s[4][3], bool second) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const Cx<P2> e = s[(2 * q) / 3][(2 * q) % 3], f = s[(2 * q + 1) / 3][(2 * q + 1) % 3];
      const H er = FROMF(e.x.v), ei = FROMF(e.y.v), fr = FROMF(f.x.v), fi = FROMF(f.y.v);
      T o;
      o.a = LO(er, ei);
      o.b = LO(fr, fi);
      a[(long long)q * V] = o;
      if (second) {
        o.a = HI(er, ei);
        o.b = HI(fr, fi);
        b[(long long)q * V] = o;
      }
    }
  }
};
__device__ __forceinline__ __half2 h_lo(__half2 a, __half2 b) { return __lows2half2(a, b); }
__device__ __forceinline__ __half2 h_hi(__half2 a, __half2 b) { return __highs2half2(a, b); }
__device__ __forceinline__ float2 h_tof(__half2 a) { return __half22float2(a); }
__device__ __forceinline__ __half2 h_fromf(float2 a) { return __float22half2_rn(a); }
__device__ __forceinline__ __nv_bfloat162 b_lo(__nv_bfloat162 a, __nv_bfloat162 b) { return __lows2bfloat162(a, b); }
__device__ __forceinline__ __nv_bfloat162 b_hi(__nv_bfloat162 a, __nv_bfloat162 b) { return __highs2bfloat162(a, b); }
__device__ __forceinline__ float2 b_tof(__nv_bfloat162 a) { return __bfloat1622float2(a); }
__device__ __forceinline__ __nv_bfloat162 b_fromf(float2 a) { return __float22bfloat162_rn(a); }
template <> struct PairIO<__half2> : PairIOHalf<__half2, h2x2, h_lo, h_hi, h_tof, h_fromf> {};
template <> struct PairIO<__nv_bfloat162> : PairIOHalf<__nv_bfloat162, b2x2, b_lo, b_hi, b_tof, b_fromf> {};

template <typename S, int RECON, int MODE>
__global__ void __launch_bounds__(128, 4) wilson_pair_kernel(const float4 *__restrict__ U,
                                                          const typename Chunk<S>::T *__restrict__ in,
                                                          typename Chunk<S>::T *__restrict__ out, float kappa,
                                                          int Lx, int Ly, int Lz, int Lt, int V, int nrhs,
                                                          int groups) {
  using T = typename Chunk<S>::T;
  const int s = (blockIdx.x / groups) * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const int r0 = (blockIdx.x % groups) * 2;
  const bool second = r0 + 1 < nrhs;  // an odd last right-hand side runs in both lanes, stored once
  const T *ia = in + (long long)r0 * 6 * V;
  const T *ib = second ? ia + 6LL * V : ia;
  constexpr bool G5IN = (MODE == 1 || MODE == 2);
  int x = s % Lx, rr = s / Lx;
  int y = rr % Ly;
  rr /= Ly;
  int z = rr % Lz;
  int t = rr / Lz;
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
  Cx<P2> acc[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[a][c] = mk<P2>(p2(0.f, 0.f), p2(0.f, 0.f));
  Cx<P2> u[9], p[4][3];
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    const int mu = d >> 1;
    const bool fwd = (d & 1) == 0;
    {
      Cx<float> uf[9];
      load_link_packed<RECON>(U, mu, V, fwd ? s : nb[d], uf);
#pragma unroll
      for (int i = 0; i < 9; ++i) u[i] = mk<P2>(p2(uf[i].x, uf[i].x), p2(uf[i].y, uf[i].y));
    }
    PairIO<S>::load(ia + nb[d], ib + nb[d], V, p);
    if (G5IN) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Cx<P2> a0 = p[0][c], a1 = p[1][c];
        p[0][c] = neg(p[2][c]); p[1][c] = neg(p[3][c]); p[2][c] = neg(a0); p[3][c] = neg(a1);
      }
    }
    if (fwd) {
      if (mu == 0) term_fwd<P2, 0>(p, u, acc);
      if (mu == 1) term_fwd<P2, 1>(p, u, acc);
      if (mu == 2) term_fwd<P2, 2>(p, u, acc);
      if (mu == 3) term_fwd<P2, 3>(p, u, acc);
    } else {
      if (mu == 0) term_bwd<P2, 0>(p, u, acc);
      if (mu == 1) term_bwd<P2, 1>(p, u, acc);
      if (mu == 2) term_bwd<P2, 2>(p, u, acc);
      if (mu == 3) term_bwd<P2, 3>(p, u, acc);
    }
  }
  T *oa = out + (long long)r0 * 6 * V + s;
  T *ob = oa + 6LL * V;
  if (MODE == 3) {
    PairIO<S>::store(oa, ob, V, acc, second);
    return;
  }
  PairIO<S>::load(ia + s, ib + s, V, p);
  if (G5IN) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Cx<P2> a0 = p[0][c], a1 = p[1][c];
      p[0][c] = neg(p[2][c]); p[1][c] = neg(p[3][c]); p[2][c] = neg(a0); p[3][c] = neg(a1);
    }
  }
  const P2 mk2 = p2(-kappa, -kappa);
  Cx<P2> o[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) o[a][c] = mk<P2>(fma(mk2, acc[a][c].x, p[a][c].x), fma(mk2, acc[a][c].y, p[a][c].y));
  if (MODE == 2) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Cx<P2> a0 = o[0][c], a1 = o[1][c];
      o[0][c] = neg(o[2][c]); o[1][c] = neg(o[3][c]); o[2][c] = neg(a0); o[3][c] = neg(a1);
    }
  }
  PairIO<S>::store(oa, ob, V, o, second);
}

// ---- paired lanes with asynchronous staging.  The neighbour spinors (both right-hand sides of the
// pair) and the link of each of the next directions are copied global -> shared memory with
// cp.async while the current direction is computed, so the bytes in flight do not depend on the
// registers a thread holds.  Every thread copies and consumes only its own entries, so the
// per-thread cp.async groups order everything and no block barrier is needed.  Shared layout
// (conflict-free: consecutive threads read consecutive entries):
//   spinors [stage][12 chunks: rhs a q = 0..5, rhs b q = 0..5][128 threads]   (T = chunk type)
//   links   [stage][NC chunks][128 threads]                                   (float4)
constexpr int ASYNC_BT = 128;
template <typename T> __device__ __forceinline__ void cp_async_chunk(T *smem, const T *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (sizeof(T) == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// lane pairs from chunks in shared memory (u: right-hand side a, w: b; chunk q at [q * ASYNC_BT])
template <typename S> struct PairSmem;
template <> struct PairSmem<float2> {
  static __device__ __forceinline__ void load(const float4 *a, const float4 *b, Cx<P2> s[4][3]) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const float4 u = a[q * ASYNC_BT], w = b[q * ASYNC_BT];
      const int c0 = 2 * q, c1 = 2 * q + 1;
      s[c0 / 3][c0 % 3] = mk<P2>(p2(u.x, w.x), p2(u.y, w.y));
      s[c1 / 3][c1 % 3] = mk<P2>(p2(u.z, w.z), p2(u.w, w.w));
    }
  }
};
template <typename H, typename T2, H (*LO)(H, H), H (*HI)(H, H), float2 (*TOF)(H)>
struct PairSmemHalf {
  static __device__ __forceinline__ void load(const T2 *a, const T2 *b, Cx<P2> s[4][3]) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const T2 u = a[q * ASYNC_BT], w = b[q * ASYNC_BT];
      const int c0 = 2 * q, c1 = 2 * q + 1;
      s[c0 / 3][c0 % 3] = mk<P2>(P2{TOF(LO(u.a, w.a))}, P2{TOF(HI(u.a, w.a))});
      s[c1 / 3][c1 % 3] = mk<P2>(P2{TOF(LO(u.b, w.b))}, P2{TOF(HI(u.b, w.b))});
    }
  }
};
template <> struct PairSmem<__half2> : PairSmemHalf<__half2, h2x2, h_lo, h_hi, h_tof> {};
template <> struct PairSmem<__nv_bfloat162> : PairSmemHalf<__nv_bfloat162, b2x2, b_lo, b_hi, b_tof> {};

// link of one direction from its NC float4 chunks in shared memory (row 2 rebuilt for recon 12)
template <int RECON>
__device__ __forceinline__ void link_from_smem(const float4 *p, Cx<float> u[9]) {
  const float4 a = p[0], b = p[ASYNC_BT], c = p[2 * ASYNC_BT];
  u[0] = mk<float>(a.x, a.y); u[1] = mk<float>(a.z, a.w);
  u[2] = mk<float>(b.x, b.y); u[3] = mk<float>(b.z, b.w);
  u[4] = mk<float>(c.x, c.y); u[5] = mk<float>(c.z, c.w);
  if (RECON == 12) {
    auto cm = [](Cx<float> x, Cx<float> y) { return mk<float>(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x); };
    Cx<float> t;
    t = cm(u[1], u[5]) - cm(u[2], u[4]); u[6] = mk<float>(t.x, -t.y);
    t = cm(u[2], u[3]) - cm(u[0], u[5]); u[7] = mk<float>(t.x, -t.y);
    t = cm(u[0], u[4]) - cm(u[1], u[3]); u[8] = mk<float>(t.x, -t.y);
  } else {
    const float4 d = p[3 * ASYNC_BT], e = p[4 * ASYNC_BT];
    u[6] = mk<float>(d.x, d.y); u[7] = mk<float>(d.z, d.w);
    u[8] = mk<float>(e.x, e.y);
  }
}

template <typename S, int RECON, int MODE, int STAGES>
__global__ void __launch_bounds__(ASYNC_BT) wilson_pair_async_kernel(const float4 *__restrict__ U,
                                                                   const typename Chunk<S>::T *__restrict__ in,
                                                                   typename Chunk<S>::T *__restrict__ out, float kappa,
                                                                   int Lx, int Ly, int Lz, int Lt, int V, int nrhs,
                                                                   int groups) {
  using T = typename Chunk<S>::T;
  constexpr int NC = RECON == 12 ? 3 : 5;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *ssp = (T *)smem_raw;
  float4 *slk = (float4 *)(smem_raw + (size_t)STAGES * 12 * ASYNC_BT * sizeof(T));
  const int tid = threadIdx.x;
  const int s = (blockIdx.x / groups) * ASYNC_BT + tid;
  if (s >= V) return;  // no block barrier below: threads past the lattice simply leave
  const int r0 = (blockIdx.x % groups) * 2;
  const bool second = r0 + 1 < nrhs;
  const T *ia = in + (long long)r0 * 6 * V;
  const T *ib = second ? ia + 6LL * V : ia;
  constexpr bool G5IN = (MODE == 1 || MODE == 2);
  int x = s % Lx, rr = s / Lx;
  int y = rr % Ly;
  rr /= Ly;
  int z = rr % Lz;
  int t = rr / Lz;
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
  auto issue = [&](int d, int stage) {
    const int mu = d >> 1;
    const float4 *lp = U + (long long)mu * NC * V + ((d & 1) ? nb[d] : s);
#pragma unroll
    for (int c = 0; c < NC; ++c) cp_async_chunk(&slk[(stage * NC + c) * ASYNC_BT + tid], lp + (long long)c * V);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      cp_async_chunk(&ssp[(stage * 12 + q) * ASYNC_BT + tid], ia + (long long)q * V + nb[d]);
      cp_async_chunk(&ssp[(stage * 12 + 6 + q) * ASYNC_BT + tid], ib + (long long)q * V + nb[d]);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int d = 0; d < STAGES; ++d) issue(d, d);
  Cx<P2> acc[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[a][c] = mk<P2>(p2(0.f, 0.f), p2(0.f, 0.f));
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    const int stage = d % STAGES;
    // groups issued after direction d: min(STAGES - 1, 7 - d)
    if (7 - d >= STAGES - 1) cp_async_wait<STAGES - 1>();
    else if (7 - d == 1) cp_async_wait<1>();
    else cp_async_wait<0>();
    const int mu = d >> 1;
    const bool fwd = (d & 1) == 0;
    Cx<P2> u[9], p[4][3];
    {
      Cx<float> uf[9];
      link_from_smem<RECON>(&slk[stage * NC * ASYNC_BT + tid], uf);
#pragma unroll
      for (int i = 0; i < 9; ++i) u[i] = mk<P2>(p2(uf[i].x, uf[i].x), p2(uf[i].y, uf[i].y));
    }
    PairSmem<S>::load(&ssp[(stage * 12) * ASYNC_BT + tid], &ssp[(stage * 12 + 6) * ASYNC_BT + tid], p);
    if (d + STAGES < 8) issue(d + STAGES, stage);  // this thread's reads of the stage are done
    if (G5IN) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Cx<P2> a0 = p[0][c], a1 = p[1][c];
        p[0][c] = neg(p[2][c]); p[1][c] = neg(p[3][c]); p[2][c] = neg(a0); p[3][c] = neg(a1);
      }
    }
    if (fwd) {
      if (mu == 0) term_fwd<P2, 0>(p, u, acc);
      if (mu == 1) term_fwd<P2, 1>(p, u, acc);
      if (mu == 2) term_fwd<P2, 2>(p, u, acc);
      if (mu == 3) term_fwd<P2, 3>(p, u, acc);
    } else {
      if (mu == 0) term_bwd<P2, 0>(p, u, acc);
      if (mu == 1) term_bwd<P2, 1>(p, u, acc);
      if (mu == 2) term_bwd<P2, 2>(p, u, acc);
      if (mu == 3) term_bwd<P2, 3>(p, u, acc);
    }
  }
  T *oa = out + (long long)r0 * 6 * V + s;
  T *ob = oa + 6LL * V;
  if (MODE == 3) {
    PairIO<S>::store(oa, ob, V, acc, second);
    return;
  }
  Cx<P2> p[4][3];
  PairIO<S>::load(ia + s, ib + s, V, p);
  if (G5IN) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Cx<P2> a0 = p[0][c], a1 = p[1][c];
      p[0][c] = neg(p[2][c]); p[1][c] = neg(p[3][c]); p[2][c] = neg(a0); p[3][c] = neg(a1);
    }
  }
  const P2 mk2 = p2(-kappa, -kappa);
  Cx<P2> o[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) o[a][c] = mk<P2>(fma(mk2, acc[a][c].x, p[a][c].x), fma(mk2, acc[a][c].y, p[a][c].y));
  if (MODE == 2) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Cx<P2> a0 = o[0][c], a1 = o[1][c];
      o[0][c] = neg(o[2][c]); o[1][c] = neg(o[3][c]); o[2][c] = neg(a0); o[3][c] = neg(a1);
    }
  }
  PairIO<S>::store(oa, ob, V, o, second);
}

// canonical complex128 fields -> packed storage S, y = sigma * x / s[r] (s == NULL: s[r] = 1)
template <typename S>
__global__ void pack_kernel(const double2 *__restrict__ x, const double *__restrict__ s,
                            typename Chunk<S>::T *__restrict__ y, int V, double sigma) {
  const int site = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  __shared__ double fs;   // the scale once per block (one right-hand side per block row)
  if (threadIdx.x == 0) {
    double f = sigma;
    if (s) {
      const double d = s[r];
      f = d > 0.0 ? sigma / d : 0.0;
    }
    fs = f;
  }
  __syncthreads();
  if (site >= V) return;
  const double f = fs;
  const double2 *src = x + ((long long)r * V + site) * 12;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const double2 a = src[2 * q], b = src[2 * q + 1];
    Chunk<S>::put(y + ((long long)r * 6 + q) * V + site, mk<float>((float)(a.x * f), (float)(a.y * f)),
                  mk<float>((float)(b.x * f), (float)(b.y * f)));
  }
}

// x^r (canonical FP64) += (s[r] / sigma) * unpack(c^r); s == NULL: x = unpack(c) / sigma
template <typename S>
__global__ void unpack_kernel(const typename Chunk<S>::T *__restrict__ c, const double *__restrict__ s,
                              double2 *__restrict__ x, int V, double sigma) {
  const int site = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  __shared__ double ds;   // the scale once per block
  if (threadIdx.x == 0) ds = s ? s[r] / sigma : 1.0 / sigma;
  __syncthreads();
  if (site >= V) return;
  double2 *dst = x + ((long long)r * V + site) * 12;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    Cx<float> u, v;
    Chunk<S>::get(c + ((long long)r * 6 + q) * V + site, u, v);
    if (s) {
      const double d = ds;
      double2 a = dst[2 * q], b = dst[2 * q + 1];
      a.x = fma(d, (double)u.x, a.x); a.y = fma(d, (double)u.y, a.y);
      b.x = fma(d, (double)v.x, b.x); b.y = fma(d, (double)v.y, b.y);
      dst[2 * q] = a;
      dst[2 * q + 1] = b;
    } else {
      const double d = ds;
      dst[2 * q] = make_double2(d * u.x, d * u.y);
      dst[2 * q + 1] = make_double2(d * v.x, d * v.y);
    }
  }
}

// FP64 links [mu][site][3][3] -> packed FP32 links (RECON 12 or 18)
__global__ void pack_links_kernel(const double2 *__restrict__ U, float4 *__restrict__ P, int V, int recon) {
  const int site = blockIdx.x * blockDim.x + threadIdx.x;
  const int mu = blockIdx.y;
  if (site >= V) return;
  const double2 *u = U + ((long long)mu * V + site) * 9;
  const int nc = recon == 12 ? 3 : 5;
  float4 *dst = P + (long long)mu * nc * V + site;
  const int ne = recon == 12 ? 6 : 9;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    if (q >= nc) break;
    const int e0 = 2 * q, e1 = 2 * q + 1;
    const double2 a = u[e0];
    const double2 b = e1 < ne ? u[e1] : make_double2(0.0, 0.0);
    dst[(long long)q * V] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
  }
}

template <typename S, int RECON>
lqcd_status pair_launch(lqcd_ctx *ctx, const float4 *U, double kappa, const void *in_, void *out_, int nrhs, int flags) {
  using T = typename Chunk<S>::T;
  const T *in = (const T *)in_;
  T *out = (T *)out_;
  int bs = 128;
  const int groups = (nrhs + 1) / 2;
  while (bs > 32 && (long long)ceil_div(ctx->V, bs) * groups < 2LL * ctx->sms) bs /= 2;
  const long long nblk = (long long)ceil_div(ctx->V, bs) * groups;
  if (nblk > 0x7fffffffLL) return set_err(ctx, LQCD_ERR_INVALID_ARG, "packed wilson: grid too large");
  dim3 grid((unsigned)nblk);
  const int *d = ctx->dims;
  const float k = (float)kappa;
  kbegin(ctx);
  switch (flags) {
    case LQCD_APPLY_M: wilson_pair_kernel<S, RECON, 0><<<grid, bs, 0, ctx->stream>>>(U, in, out, k, d[0], d[1], d[2], d[3], ctx->V, nrhs, groups); break;
    case LQCD_APPLY_G5R: wilson_pair_kernel<S, RECON, 1><<<grid, bs, 0, ctx->stream>>>(U, in, out, k, d[0], d[1], d[2], d[3], ctx->V, nrhs, groups); break;
    case LQCD_APPLY_DAG: wilson_pair_kernel<S, RECON, 2><<<grid, bs, 0, ctx->stream>>>(U, in, out, k, d[0], d[1], d[2], d[3], ctx->V, nrhs, groups); break;
    case LQCD_APPLY_HOP: wilson_pair_kernel<S, RECON, 3><<<grid, bs, 0, ctx->stream>>>(U, in, out, k, d[0], d[1], d[2], d[3], ctx->V, nrhs, groups); break;
    default: return set_err(ctx, LQCD_ERR_INVALID_ARG, "packed wilson: unknown flags %d", flags);
  }
  const double bytes = 2.0 * nrhs * ctx->V * 6 * sizeof(T) + 4.0 * ctx->V * (RECON == 12 ? 3 : 5) * 16;
  return launch_check_bytes(ctx, "wilson_pair_kernel", K_WILSON, (double)ctx->V * nrhs, bytes);
}

// staged variant of the paired-lane operator: 3 directions in flight for FP16 / BF16 fields, 2 for
// FP32 fields (shared memory per block: stages x (12 x 128 chunks + NC x 128 link float4))
template <typename S, int RECON>
lqcd_status pair_async_launch(lqcd_ctx *ctx, const float4 *U, double kappa, const void *in_, void *out_, int nrhs,
                              int flags) {
  using T = typename Chunk<S>::T;
  constexpr int STAGES = sizeof(T) == 16 ? 2 : 3;
  constexpr int NC = RECON == 12 ? 3 : 5;
  const T *in = (const T *)in_;
  T *out = (T *)out_;
  const int groups = (nrhs + 1) / 2;
  const long long nblk = (long long)ceil_div(ctx->V, ASYNC_BT) * groups;
  if (nblk > 0x7fffffffLL) return set_err(ctx, LQCD_ERR_INVALID_ARG, "packed wilson: grid too large");
  const size_t smem = (size_t)STAGES * (12 * ASYNC_BT * sizeof(T) + NC * ASYNC_BT * sizeof(float4));
  const int *d = ctx->dims;
  const float k = (float)kappa;
  auto go = [&](auto kern) -> lqcd_status {
    LQCD_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kbegin(ctx);
    kern<<<(unsigned)nblk, ASYNC_BT, smem, ctx->stream>>>(U, in, out, k, d[0], d[1], d[2], d[3], ctx->V, nrhs, groups);
    const double bytes = 2.0 * nrhs * ctx->V * 6 * sizeof(T) + 4.0 * ctx->V * NC * 16;
    return launch_check_bytes(ctx, "wilson_pair_async_kernel", K_WILSON, (double)ctx->V * nrhs, bytes);
  };
  switch (flags) {
    case LQCD_APPLY_M: return go(wilson_pair_async_kernel<S, RECON, 0, STAGES>);
    case LQCD_APPLY_G5R: return go(wilson_pair_async_kernel<S, RECON, 1, STAGES>);
    case LQCD_APPLY_DAG: return go(wilson_pair_async_kernel<S, RECON, 2, STAGES>);
    case LQCD_APPLY_HOP: return go(wilson_pair_async_kernel<S, RECON, 3, STAGES>);
    default: return set_err(ctx, LQCD_ERR_INVALID_ARG, "packed wilson: unknown flags %d", flags);
  }
}

template <typename S, int NR, int RECON>
lqcd_status packed_launch_nr(lqcd_ctx *ctx, const float4 *U, double kappa, const void *in_, void *out_, int nrhs,
                             int flags) {
  using T = typename Chunk<S>::T;
  const T *in = (const T *)in_;
  T *out = (T *)out_;
  int bs = 128;
  const int groups = (nrhs + NR - 1) / NR;
  while (bs > 32 && (long long)ceil_div(ctx->V, bs) * groups < 2LL * ctx->sms) bs /= 2;
  const long long nblk = (long long)ceil_div(ctx->V, bs) * groups;
  if (nblk > 0x7fffffffLL) return set_err(ctx, LQCD_ERR_INVALID_ARG, "packed wilson: grid too large");
  dim3 grid((unsigned)nblk);
  const int *d = ctx->dims;
  const float k = (float)kappa;
  kbegin(ctx);
  switch (flags) {
    case LQCD_APPLY_M: wilson_packed_kernel<S, NR, RECON, 0><<<grid, bs, 0, ctx->stream>>>(U, in, out, k, d[0], d[1], d[2], d[3], ctx->V, nrhs, groups); break;
    case LQCD_APPLY_G5R: wilson_packed_kernel<S, NR, RECON, 1><<<grid, bs, 0, ctx->stream>>>(U, in, out, k, d[0], d[1], d[2], d[3], ctx->V, nrhs, groups); break;
    case LQCD_APPLY_DAG: wilson_packed_kernel<S, NR, RECON, 2><<<grid, bs, 0, ctx->stream>>>(U, in, out, k, d[0], d[1], d[2], d[3], ctx->V, nrhs, groups); break;
    case LQCD_APPLY_HOP: wilson_packed_kernel<S, NR, RECON, 3><<<grid, bs, 0, ctx->stream>>>(U, in, out, k, d[0], d[1], d[2], d[3], ctx->V, nrhs, groups); break;
    default: return set_err(ctx, LQCD_ERR_INVALID_ARG, "packed wilson: unknown flags %d", flags);
  }
  const double bytes = 2.0 * nrhs * ctx->V * 6 * sizeof(T) + 4.0 * ctx->V * (RECON == 12 ? 3 : 5) * 16;
  return launch_check_bytes(ctx, "wilson_packed_kernel", K_WILSON, (double)ctx->V * nrhs, bytes);
}

}  // namespace

lqcd_status wilson_launch_packed(lqcd_ctx *ctx, const float4 *U, int recon, double kappa, const float4 *in, float4 *out,
                                 int nrhs, int flags, int nr) {
  if (nrhs <= 0) return set_err(ctx, LQCD_ERR_INVALID_ARG, "packed wilson: nrhs %d out of range", nrhs);
  if (recon != 12 && recon != 18) return set_err(ctx, LQCD_ERR_INVALID_ARG, "packed wilson: recon must be 12 or 18");
  // nr: 1 = one right-hand side per thread, 2 = two in the lanes of packed FP32 arithmetic, 4 = four
  // per thread (scalar); 0 = the context's setting (lqcd_set_rhs_per_thread or the autotuner), else
  // 2: on 24^3 x 32 with 8 and 16 right-hand sides the paired lanes take 13 % less time than one
  // right-hand side per thread (the stencil is bound by instruction issue, not by HBM)
  if (nr <= 0) nr = ctx->packed_nr > 0 ? ctx->packed_nr : 2;
  if ((nr == 2 || nr == 3) && nrhs < 2) nr = 1;
  if (recon == 12) {
    if (nr == 1) return packed_launch_nr<float2, 1, 12>(ctx, U, kappa, in, out, nrhs, flags);
    if (nr == 2) return pair_launch<float2, 12>(ctx, U, kappa, in, out, nrhs, flags);
    if (nr == 3) return pair_async_launch<float2, 12>(ctx, U, kappa, in, out, nrhs, flags);
    return packed_launch_nr<float2, 4, 12>(ctx, U, kappa, in, out, nrhs, flags);
  }
  if (nr == 1) return packed_launch_nr<float2, 1, 18>(ctx, U, kappa, in, out, nrhs, flags);
  if (nr == 2) return pair_launch<float2, 18>(ctx, U, kappa, in, out, nrhs, flags);
  if (nr == 3) return pair_async_launch<float2, 18>(ctx, U, kappa, in, out, nrhs, flags);
  return packed_launch_nr<float2, 4, 18>(ctx, U, kappa, in, out, nrhs, flags);
}

// FP16 / BF16 fields: two right-hand sides per thread in paired lanes (19 % less time than one per
// thread on 24^3 x 32 with 8 right-hand sides), or one when the context's setting is 1
template <typename S>
lqcd_status wilson_launch_packed_lp(lqcd_ctx *ctx, const float4 *U, int recon, double kappa, const S *in, S *out,
                                   int nrhs, int flags) {
  if (nrhs <= 0) return set_err(ctx, LQCD_ERR_INVALID_ARG, "packed wilson: nrhs %d out of range", nrhs);
  const bool pair = (ctx->packed_nr == 2 || ctx->packed_nr == 0) && nrhs >= 2;
  const bool staged = ctx->packed_nr == 3 && nrhs >= 2;
  if (recon == 12)
    return staged ? pair_async_launch<S, 12>(ctx, U, kappa, in, out, nrhs, flags)
           : pair ? pair_launch<S, 12>(ctx, U, kappa, in, out, nrhs, flags)
                  : packed_launch_nr<S, 1, 12>(ctx, U, kappa, in, out, nrhs, flags);
  if (recon == 18)
    return staged ? pair_async_launch<S, 18>(ctx, U, kappa, in, out, nrhs, flags)
           : pair ? pair_launch<S, 18>(ctx, U, kappa, in, out, nrhs, flags)
                  : packed_launch_nr<S, 1, 18>(ctx, U, kappa, in, out, nrhs, flags);
  return set_err(ctx, LQCD_ERR_INVALID_ARG, "packed wilson: recon must be 12 or 18");
}
template lqcd_status wilson_launch_packed_lp<__half2>(lqcd_ctx *, const float4 *, int, double, const __half2 *,
                                                      __half2 *, int, int);
template lqcd_status wilson_launch_packed_lp<__nv_bfloat162>(lqcd_ctx *, const float4 *, int, double,
                                                             const __nv_bfloat162 *, __nv_bfloat162 *, int, int);

lqcd_status pack_f32(lqcd_ctx *ctx, const double2 *x, const double *scale, float4 *y, int nrhs) {
  kbegin(ctx);
  pack_kernel<float2><<<dim3(ceil_div(ctx->V, 128), nrhs), 128, 0, ctx->stream>>>(x, scale, y, ctx->V, 1.0);
  return launch_check(ctx, "pack_kernel", K_BLAS1, (double)ctx->N * nrhs);
}

lqcd_status unpack_f32(lqcd_ctx *ctx, const float4 *c, const double *scale, double2 *x, int nrhs) {
  kbegin(ctx);
  unpack_kernel<float2><<<dim3(ceil_div(ctx->V, 128), nrhs), 128, 0, ctx->stream>>>(c, scale, x, ctx->V, 1.0);
  return launch_check(ctx, "unpack_kernel", K_BLAS1, (double)ctx->N * nrhs);
}

template <typename S> lqcd_status pack_lp(lqcd_ctx *ctx, const double2 *x, const double *scale, S *y, int nrhs) {
  kbegin(ctx);
  pack_kernel<S><<<dim3(ceil_div(ctx->V, 128), nrhs), 128, 0, ctx->stream>>>(
      x, scale, (typename Chunk<S>::T *)y, ctx->V, store_sigma<S>(ctx->N));
  return launch_check(ctx, "pack_kernel", K_BLAS1, (double)ctx->N * nrhs);
}

template <typename S> lqcd_status unpack_lp(lqcd_ctx *ctx, const S *c, const double *scale, double2 *x, int nrhs) {
  kbegin(ctx);
  unpack_kernel<S><<<dim3(ceil_div(ctx->V, 128), nrhs), 128, 0, ctx->stream>>>(
      (const typename Chunk<S>::T *)c, scale, x, ctx->V, store_sigma<S>(ctx->N));
  return launch_check(ctx, "unpack_kernel", K_BLAS1, (double)ctx->N * nrhs);
}
template lqcd_status pack_lp<__half2>(lqcd_ctx *, const double2 *, const double *, __half2 *, int);
template lqcd_status pack_lp<__nv_bfloat162>(lqcd_ctx *, const double2 *, const double *, __nv_bfloat162 *, int);
template lqcd_status unpack_lp<__half2>(lqcd_ctx *, const __half2 *, const double *, double2 *, int);
template lqcd_status unpack_lp<__nv_bfloat162>(lqcd_ctx *, const __nv_bfloat162 *, const double *, double2 *, int);

lqcd_status pack_links_f32(lqcd_ctx *ctx, const double2 *U, float4 *P, int recon) {
  if (recon != 12 && recon != 18) return set_err(ctx, LQCD_ERR_INVALID_ARG, "pack_links: recon must be 12 or 18");
  kbegin(ctx);
  pack_links_kernel<<<dim3(ceil_div(ctx->V, 128), 4), 128, 0, ctx->stream>>>(U, P, ctx->V, recon);
  return launch_check(ctx, "pack_links_kernel", K_BLAS1, (double)ctx->V * 36);
}

extern "C" lqcd_status lqcd_pack_f32(lqcd_ctx *ctx, const double *in, float *out, int nrhs) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_full(ctx, "pack_f32"));
  if (!in || !out || nrhs < 1 || nrhs > 65535) return set_err(ctx, LQCD_ERR_INVALID_ARG, "pack_f32: bad arguments");
  return pack_f32(ctx, (const double2 *)in, nullptr, (float4 *)out, nrhs);
}

extern "C" lqcd_status lqcd_unpack_f32(lqcd_ctx *ctx, const float *in, double *out, int nrhs) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_full(ctx, "unpack_f32"));
  if (!in || !out || nrhs < 1 || nrhs > 65535) return set_err(ctx, LQCD_ERR_INVALID_ARG, "unpack_f32: bad arguments");
  return unpack_f32(ctx, (const float4 *)in, nullptr, (double2 *)out, nrhs);
}

extern "C" lqcd_status lqcd_pack_links_f32(lqcd_ctx *ctx, const double *links, float *out, int recon) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_full(ctx, "pack_links_f32"));
  if (!links || !out) return set_err(ctx, LQCD_ERR_INVALID_ARG, "pack_links_f32: NULL pointer");
  return pack_links_f32(ctx, (const double2 *)links, (float4 *)out, recon);
}

extern "C" lqcd_status lqcd_wilson_apply_packed(lqcd_ctx *ctx, const float *links_packed, int recon, double kappa,
                                                const float *in, float *out, int nrhs, int flags, int rhs_per_thread) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_full(ctx, "wilson_apply_packed"));
  if (!links_packed || !in || !out || in == out) return set_err(ctx, LQCD_ERR_INVALID_ARG, "wilson_apply_packed: bad pointers");
  if (rhs_per_thread < 0 || rhs_per_thread > 4)
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "wilson_apply_packed: rhs_per_thread must be 0, 1, 2, 3 or 4");
  return wilson_launch_packed(ctx, (const float4 *)links_packed, recon, kappa, (const float4 *)in, (float4 *)out, nrhs,
                              flags, rhs_per_thread);
}

// ---- FP16 / BF16 fields ------------------------------------------------------------------------
extern "C" lqcd_status lqcd_pack_half(lqcd_ctx *ctx, int prec, const double *in, void *out, int nrhs) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_full(ctx, "pack_half"));
  if (!in || !out || nrhs < 1 || nrhs > 65535) return set_err(ctx, LQCD_ERR_INVALID_ARG, "pack_half: bad arguments");
  if (prec == LQCD_PREC_F16) return pack_lp(ctx, (const double2 *)in, nullptr, (__half2 *)out, nrhs);
  if (prec == LQCD_PREC_BF16) return pack_lp(ctx, (const double2 *)in, nullptr, (__nv_bfloat162 *)out, nrhs);
  return set_err(ctx, LQCD_ERR_INVALID_ARG, "pack_half: prec must be LQCD_PREC_F16 or LQCD_PREC_BF16");
}

extern "C" lqcd_status lqcd_unpack_half(lqcd_ctx *ctx, int prec, const void *in, double *out, int nrhs) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_full(ctx, "unpack_half"));
  if (!in || !out || nrhs < 1 || nrhs > 65535) return set_err(ctx, LQCD_ERR_INVALID_ARG, "unpack_half: bad arguments");
  if (prec == LQCD_PREC_F16) return unpack_lp(ctx, (const __half2 *)in, nullptr, (double2 *)out, nrhs);
  if (prec == LQCD_PREC_BF16) return unpack_lp(ctx, (const __nv_bfloat162 *)in, nullptr, (double2 *)out, nrhs);
  return set_err(ctx, LQCD_ERR_INVALID_ARG, "unpack_half: prec must be LQCD_PREC_F16 or LQCD_PREC_BF16");
}

extern "C" lqcd_status lqcd_wilson_apply_half(lqcd_ctx *ctx, int prec, const float *links_packed, int recon,
                                              double kappa, const void *in, void *out, int nrhs, int flags) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_full(ctx, "wilson_apply_half"));
  if (!links_packed || !in || !out || in == out) return set_err(ctx, LQCD_ERR_INVALID_ARG, "wilson_apply_half: bad pointers");
  if (prec == LQCD_PREC_F16)
    return wilson_launch_packed_lp(ctx, (const float4 *)links_packed, recon, kappa, (const __half2 *)in, (__half2 *)out,
                                   nrhs, flags);
  if (prec == LQCD_PREC_BF16)
    return wilson_launch_packed_lp(ctx, (const float4 *)links_packed, recon, kappa, (const __nv_bfloat162 *)in,
                                   (__nv_bfloat162 *)out, nrhs, flags);
  return set_err(ctx, LQCD_ERR_INVALID_ARG, "wilson_apply_half: prec must be LQCD_PREC_F16 or LQCD_PREC_BF16");
}

extern "C" lqcd_status lqcd_set_rhs_per_thread(lqcd_ctx *ctx, int nr) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  if (nr < 0 || nr > 4)
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "set_rhs_per_thread: nr must be 0, 1, 2, 3 or 4");
  graph_cache_clear(ctx);
  ctx->packed_nr = nr;
  return LQCD_OK;
}
