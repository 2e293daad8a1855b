// Loop-estimate stage: operator contractions (Sec. 6), perturbative / polynomial series (Sec. 5.1,
// 5.2), deflation projection (Sec. 5.4), 1/xi' (Sec. 5.5), hopping traces by probing (Sec. 5.1)
// and the whole estimate on one gauge configuration.
//
// Contraction densities of eta^dag Theta w at base site x (Table Table903):
//   scalar       eta(x)^dag w(x)
//   local        eta(x)^dag gamma_mu w(x)
//   point-split  kappa [ eta(x+mu)^dag (1 + g_mu) U_mu(x)^dag w(x) - eta(x)^dag (1 - g_mu) U_mu(x) w(x+mu) ]
// summed per timeslice with Neumaier-compensated FP64 accumulation.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <memory>
#include <mutex>

#include <cuda.h>  // driver types of the context-id query (entry points come from the runtime)

#include "common.cuh"
#include "dense.h"
#include "spin.cuh"

using dense::cd;

namespace {

using namespace spin;

constexpr int CBT = 128;  // threads per contraction block

__device__ __forceinline__ Cx<double> dotc(const Cx<double> a[4][3], const Cx<double> b[4][3]) {
  double re = 0.0, im = 0.0;
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      re = fma(a[s][c].x, b[s][c].x, re);
      re = fma(a[s][c].y, b[s][c].y, re);
      im = fma(a[s][c].x, b[s][c].y, im);
      im = fma(-a[s][c].y, b[s][c].x, im);
    }
  return mk<double>(re, im);
}

// gamma_mu w in the Dirac basis
template <int MU>
__device__ __forceinline__ void gamma_apply(const Cx<double> w[4][3], Cx<double> o[4][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (MU == 0) { o[0][c] = tmi(w[3][c]); o[1][c] = tmi(w[2][c]); o[2][c] = ti(w[1][c]); o[3][c] = ti(w[0][c]); }
    if (MU == 1) { o[0][c] = neg(w[3][c]); o[1][c] = w[2][c]; o[2][c] = w[1][c]; o[3][c] = neg(w[0][c]); }
    if (MU == 2) { o[0][c] = tmi(w[2][c]); o[1][c] = ti(w[3][c]); o[2][c] = ti(w[0][c]); o[3][c] = tmi(w[1][c]); }
    if (MU == 3) { o[0][c] = w[0][c]; o[1][c] = w[1][c]; o[2][c] = neg(w[2][c]); o[3][c] = neg(w[3][c]); }
  }
}

template <int MU>
__device__ __forceinline__ void zero_sp(Cx<double> a[4][3]) {
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) a[s][c] = mk<double>(0.0, 0.0);
}

// point-split density of direction MU at site s
template <int MU>
__device__ __forceinline__ Cx<double> psplit(const double2 *U, const double2 *eta, const double2 *w, int s, int sp,
                                             long long V, const Cx<double> eta_s[4][3], const Cx<double> w_s[4][3]) {
  Cx<double> u[9], a[4][3], nb[4][3];
  load_link<double>(U, (long long)MU * V + s, u);
  // (1 + g_mu) U_mu(s)^dag w(s), then contracted with eta(s + mu)
  zero_sp<MU>(a);
  term_bwd<double, MU>(w_s, u, a);
  load_spinor<double, false>(eta + 12LL * sp, nb);
  Cx<double> t1 = dotc(nb, a);
  // (1 - g_mu) U_mu(s) w(s + mu), contracted with eta(s)
  zero_sp<MU>(a);
  load_spinor<double, false>(w + 12LL * sp, nb);
  term_fwd<double, MU>(nb, u, a);
  Cx<double> t2 = dotc(eta_s, a);
  return t1 - t2;
}

// partial[((r * Lt + t) * nchunk + chunk) * 9 + op]; grid (nchunk * Lt, nrhs)
__global__ void __launch_bounds__(CBT) contract_kernel(const double2 *__restrict__ U, double kappa,
                                                       const double2 *__restrict__ eta, const double2 *__restrict__ w,
                                                       int Lx, int Ly, int Lz, int Lt, int nchunk,
                                                       double2 *__restrict__ partial) {
  const int r = blockIdx.y;
  const int t = blockIdx.x / nchunk;
  const int chunk = blockIdx.x % nchunk;
  const int Vs = Lx * Ly * Lz;
  const long long V = (long long)Vs * Lt;
  const double2 *er = eta + (long long)r * V * 12, *wr = w + (long long)r * V * 12;
  const int per = (Vs + nchunk - 1) / nchunk;
  const int i0 = chunk * per, i1 = min(Vs, i0 + per);
  KSum acc[18];
#pragma unroll
  for (int q = 0; q < 18; ++q) acc[q].init();
  for (int i = i0 + threadIdx.x; i < i1; i += CBT) {
    const int s = t * Vs + i;
    const int x = i % Lx, y = (i / Lx) % Ly, z = i / (Lx * Ly);
    Cx<double> es[4][3], ws[4][3], g[4][3];
    load_spinor<double, false>(er + 12LL * s, es);
    load_spinor<double, false>(wr + 12LL * s, ws);
    Cx<double> d = dotc(es, ws);
    acc[0].add(d.x); acc[1].add(d.y);
    gamma_apply<0>(ws, g); d = dotc(es, g); acc[2].add(d.x); acc[3].add(d.y);
    gamma_apply<1>(ws, g); d = dotc(es, g); acc[4].add(d.x); acc[5].add(d.y);
    gamma_apply<2>(ws, g); d = dotc(es, g); acc[6].add(d.x); acc[7].add(d.y);
    gamma_apply<3>(ws, g); d = dotc(es, g); acc[8].add(d.x); acc[9].add(d.y);
    const int xp = (x + 1 == Lx) ? s - (Lx - 1) : s + 1;
    const int yp = (y + 1 == Ly) ? s - (Ly - 1) * Lx : s + Lx;
    const int zp = (z + 1 == Lz) ? s - (Lz - 1) * Lx * Ly : s + Lx * Ly;
    const int tp = (t + 1 == Lt) ? s - (Lt - 1) * Vs : s + Vs;
    d = psplit<0>(U, er, wr, s, xp, V, es, ws); acc[10].add(kappa * d.x); acc[11].add(kappa * d.y);
    d = psplit<1>(U, er, wr, s, yp, V, es, ws); acc[12].add(kappa * d.x); acc[13].add(kappa * d.y);
    d = psplit<2>(U, er, wr, s, zp, V, es, ws); acc[14].add(kappa * d.x); acc[15].add(kappa * d.y);
    d = psplit<3>(U, er, wr, s, tp, V, es, ws); acc[16].add(kappa * d.x); acc[17].add(kappa * d.y);
  }
  __shared__ double red[CBT / 32][18];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 18; ++q) {
    double v = acc[q].value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    double re = 0.0, im = 0.0;
    for (int q = 0; q < CBT / 32; ++q) {
      re += red[q][2 * threadIdx.x];
      im += red[q][2 * threadIdx.x + 1];
    }
    partial[(((long long)r * Lt + t) * nchunk + chunk) * 9 + threadIdx.x] = make_double2(re, im);
  }
}

// out[(r * 9 + op) * Lt + t] = sum over chunks (fixed order)
__global__ void contract_final(const double2 *__restrict__ partial, int nchunk, int Lt, int nrhs,
                               double2 *__restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nrhs * 9 * Lt) return;
  const int t = idx % Lt, op = (idx / Lt) % 9, r = idx / (9 * Lt);
  double re = 0.0, ce = 0.0, im = 0.0, ci = 0.0;
  for (int c = 0; c < nchunk; ++c) {
    const double2 v = partial[(((long long)r * Lt + t) * nchunk + c) * 9 + op];
    double tt = re + v.x;
    ce += (fabs(re) >= fabs(v.x)) ? (re - tt) + v.x : (v.x - tt) + re;
    re = tt;
    tt = im + v.y;
    ci += (fabs(im) >= fabs(v.y)) ? (im - tt) + v.y : (v.y - tt) + im;
    im = tt;
  }
  out[idx] = make_double2(re + ce, im + ci);
}

// y = a * x + y over nrhs fields with a per-rhs scale a[r] (device); one thread per element
__global__ void scaled_acc_kernel(const double2 *__restrict__ x, double2 *__restrict__ y, double2 a, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double2 v = y[e];
    cfma(v, a, x[e]);
    y[e] = v;
  }
}

// Probing colourings for the hopping traces.  Two sites of one colour class must be more than K
// hops apart on the torus (K - 1 hops of P^k plus the one hop of a point-split operator), so that
// every off-diagonal term of z_c^dag Theta P^k z_c vanishes.
//   * sublattice colouring: with s = ceil((K + 1) / 2) and an integer q >= 2, classes are the
//     cosets of  {s w : w in Z^4, sum(w) = 0 mod q}, whose shortest non-zero vector has 2 s >= K + 1
//     hops (s (e_mu - e_nu), or q s e_mu); class = (x mod s per direction, sum_mu floor(x_mu / s)
//     mod q); q s^4 classes.  The torus periods L_mu e_mu lie in the sublattice when s divides
//     every extent and q divides every L_mu / s; q = 2 is the scaled D4 lattice (extents divisible
//     by 2 s, e.g. 8^3 x 16 at K = 7), q = 3 serves 12^4 and 12^3 x 24.
//   * Cartesian fallback: class = (x mod p_mu) with p_mu the smallest divisor of L_mu that is
//     >= K + 1, else L_mu.
// The colouring with fewer classes is used.
struct Colouring {
  int s[4];
  int q;     // 1: Cartesian
  int ncls;
};

__host__ __device__ __forceinline__ int class_of(const Colouring &c, int x, int y, int z, int t) {
  const int base = (x % c.s[0]) + c.s[0] * ((y % c.s[1]) + c.s[1] * ((z % c.s[2]) + c.s[2] * (t % c.s[3])));
  if (c.q == 1) return base;
  const int res = (x / c.s[0] + y / c.s[1] + z / c.s[2] + t / c.s[3]) % c.q;
  return c.q * base + res;
}

// Probe vectors: probe p of the batch (global probe first + p) has colour class g / 12 and
// spin-colour component g % 12: a unit entry at that component on every site of the class.
__global__ void probe_kernel(int first, int nprobe, int Lx, int Ly, int Lz, int Lt, Colouring col,
                             double2 *__restrict__ out) {
  const long long V = (long long)Lx * Ly * Lz * Lt;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (s >= V || p >= nprobe) return;
  const int x = s % Lx, y = (s / Lx) % Ly, z = (s / (Lx * Ly)) % Lz, t = s / (Lx * Ly * Lz);
  const int cls = class_of(col, x, y, z, t);
  const int g = first + p;
  const int pc = g / 12, comp = g % 12;
  double2 *o = out + ((long long)p * V + s) * 12;
#pragma unroll
  for (int e = 0; e < 12; ++e) o[e] = make_double2((cls == pc && e == comp) ? 1.0 : 0.0, 0.0);
}

__device__ __forceinline__ Cx<double> pick(const Cx<double> a[4][3], int comp) {
  Cx<double> r = mk<double>(0.0, 0.0);
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (3 * sp + c == comp) r = a[sp][c];
  return r;
}

template <int MU>
__device__ __forceinline__ Cx<double> ps_term1(const double2 *U, const double2 *w, int b, long long V, int comp) {
  // ((1 + g_mu) U_mu(b)^dag w(b))_comp
  Cx<double> u[9], ws[4][3], a[4][3];
  load_link<double>(U, (long long)MU * V + b, u);
  load_spinor<double, false>(w + 12LL * b, ws);
  zero_sp<MU>(a);
  term_bwd<double, MU>(ws, u, a);
  return pick(a, comp);
}

template <int MU>
__device__ __forceinline__ Cx<double> ps_term2(const double2 *U, const double2 *w, int m, int mp, long long V, int comp) {
  // ((1 - g_mu) U_mu(m) w(m + mu))_comp
  Cx<double> u[9], ws[4][3], a[4][3];
  load_link<double>(U, (long long)MU * V + m, u);
  load_spinor<double, false>(w + 12LL * mp, ws);
  zero_sp<MU>(a);
  term_fwd<double, MU>(ws, u, a);
  return pick(a, comp);
}

// Sparse contraction of probes with P^k probes: out[p][op][t] = sum over the base sites x in
// timeslice t of the density of z_p^dag Theta_op w_p.  z_p is a unit entry (component comp) on
// the members of its class, so only terms at class members (and at x = member - mu for the first
// point-split term) survive.  One block per probe, one thread per (op, t); each thread sums its
// few members in a fixed order.
__global__ void probe_contract_kernel(const double2 *__restrict__ U, double kappa, const double2 *__restrict__ W,
                                      int first, int nprobe, int Lx, int Ly, int Lz, int Lt, Colouring col,
                                      double2 *__restrict__ out) {
  const int p = blockIdx.x;
  if (p >= nprobe) return;
  const long long V = (long long)Lx * Ly * Lz * Lt;
  const double2 *w = W + (long long)p * V * 12;
  const int g = first + p;
  const int cls = g / 12, comp = g % 12;
  // decode the class into its residues (and the sum residue mod q of the sublattice colouring)
  const int par = cls % col.q;
  int base = cls / col.q;
  const int rx = base % col.s[0];
  base /= col.s[0];
  const int ry = base % col.s[1];
  base /= col.s[1];
  const int rz = base % col.s[2];
  const int rt = base / col.s[2];
  for (int idx = threadIdx.x; idx < 9 * Lt; idx += blockDim.x) {
    const int op = idx / Lt, t = idx % Lt;
    // members m of the class whose relevant base site lies in slice t: slice t itself, except for
    // the first point-split term in the t direction (base m - t_hat), whose members are in t + 1
    double re = 0.0, im = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
      const int tm = (pass == 0) ? t : (t + 1) % Lt;
      if (pass == 1 && op != 8) break;
      if (tm % col.s[3] != rt) continue;
      const int nt = tm / col.s[3];
      for (int nz = 0; nz < Lz / col.s[2]; ++nz)
        for (int ny = 0; ny < Ly / col.s[1]; ++ny)
          for (int nx = 0; nx < Lx / col.s[0]; ++nx) {
            if (col.q > 1 && (nx + ny + nz + nt) % col.q != par) continue;
            const int x = rx + col.s[0] * nx, y = ry + col.s[1] * ny, z = rz + col.s[2] * nz;
            const int m = x + Lx * (y + Ly * (z + Lz * tm));
            Cx<double> v = mk<double>(0.0, 0.0);
            if (op == 0 && pass == 0) {
              v = load_c<double>(w + 12LL * m + comp);
            } else if (op <= 4 && pass == 0) {
              Cx<double> ws[4][3], gw[4][3];
              load_spinor<double, false>(w + 12LL * m, ws);
              if (op == 1) gamma_apply<0>(ws, gw);
              if (op == 2) gamma_apply<1>(ws, gw);
              if (op == 3) gamma_apply<2>(ws, gw);
              if (op == 4) gamma_apply<3>(ws, gw);
              v = pick(gw, comp);
            } else if (op >= 5) {
              const int mu = op - 5;
              if (pass == 0) {
                // second term at base m: - (1 - g) U(m) w(m + mu); first term for mu != t at base m - mu
                const int xp = (x + 1) % Lx, yp = (y + 1) % Ly, zp = (z + 1) % Lz, tp = (tm + 1) % Lt;
                const int xm = (x + Lx - 1) % Lx, ym = (y + Ly - 1) % Ly, zm = (z + Lz - 1) % Lz;
                Cx<double> t1 = mk<double>(0.0, 0.0), t2;
                if (mu == 0) {
                  t2 = ps_term2<0>(U, w, m, xp + Lx * (y + Ly * (z + Lz * tm)), V, comp);
                  t1 = ps_term1<0>(U, w, xm + Lx * (y + Ly * (z + Lz * tm)), V, comp);
                } else if (mu == 1) {
                  t2 = ps_term2<1>(U, w, m, x + Lx * (yp + Ly * (z + Lz * tm)), V, comp);
                  t1 = ps_term1<1>(U, w, x + Lx * (ym + Ly * (z + Lz * tm)), V, comp);
                } else if (mu == 2) {
                  t2 = ps_term2<2>(U, w, m, x + Lx * (y + Ly * (zp + Lz * tm)), V, comp);
                  t1 = ps_term1<2>(U, w, x + Lx * (y + Ly * (zm + Lz * tm)), V, comp);
                } else {
                  t2 = ps_term2<3>(U, w, m, x + Lx * (y + Ly * (z + Lz * tp)), V, comp);
                }
                v = mk<double>(kappa * (t1.x - t2.x), kappa * (t1.y - t2.y));
              } else {
                // first term in the t direction: member m in slice t + 1, base m - t_hat in slice t
                const int b = x + Lx * (y + Ly * (z + Lz * t));
                Cx<double> t1 = ps_term1<3>(U, w, b, V, comp);
                v = mk<double>(kappa * t1.x, kappa * t1.y);
              }
            }
            re += v.x;
            im += v.y;
          }
    }
    out[((long long)p * 9 + op) * Lt + t] = make_double2(re, im);
  }
}

// Local completion of a probe field (meet-in-the-middle hopping traces).  The contraction of order
// k reads P^k z only at the members of the probe's class and at their eight neighbours, and
// (P^k z)(y) needs P^(k-1) z only at the neighbours of y.  So once P^h z is known everywhere, the
// orders k > h are needed only in the taxicab balls of radius K - k around the members: this
// kernel evaluates (P z)(y) for every y = member + offset (offsets: the ball, as char4 (dx, dy, dz,
// dt)), reading `in` at the neighbours of y and writing `out` at y alone.  Sites outside the balls
// keep whatever `out` held; the next order and the contraction never read them.  One site can be
// named twice (two offsets of one ball on a small torus, or the touching balls of two members):
// both threads then compute it from the same inputs and store the same value.
// One thread per (member, offset) pair and probe (blockIdx.y).
__global__ void __launch_bounds__(128) hop_listed_kernel(const double2 *__restrict__ U, const double2 *__restrict__ in,
                                                         double2 *__restrict__ out, const char4 *__restrict__ offs,
                                                         int noff, int first, int nprobe, int Lx, int Ly, int Lz,
                                                         int Lt, Colouring col) {
  const int p = blockIdx.y;
  if (p >= nprobe) return;
  const int Nx = Lx / col.s[0], Ny = Ly / col.s[1], Nz = Lz / col.s[2], Nt = Lt / col.s[3];
  const long long nmem = (long long)Nx * Ny * Nz * (Nt / col.q);
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nmem * noff) return;
  const int o = (int)(i % noff);
  long long mi = i / noff;
  const int cls = (first + p) / 12;
  const int par = cls % col.q;
  int b = cls / col.q;
  const int rx = b % col.s[0];
  b /= col.s[0];
  const int ry = b % col.s[1];
  b /= col.s[1];
  const int rz = b % col.s[2];
  const int rt = b / col.s[2];
  const int nx = (int)(mi % Nx);
  mi /= Nx;
  const int ny = (int)(mi % Ny);
  mi /= Ny;
  const int nz = (int)(mi % Nz);
  const int m = (int)(mi / Nz);
  // the member's sublattice coordinates satisfy nx + ny + nz + nt = par (mod q)
  const int nt = col.q * m + (((par - nx - ny - nz) % col.q) + col.q) % col.q;
  const char4 d = offs[o];
  const int x = ((rx + col.s[0] * nx + d.x) % Lx + Lx) % Lx;
  const int y = ((ry + col.s[1] * ny + d.y) % Ly + Ly) % Ly;
  const int z = ((rz + col.s[2] * nz + d.z) % Lz + Lz) % Lz;
  const int t = ((rt + col.s[3] * nt + d.w) % Lt + Lt) % Lt;
  const long long V = (long long)Lx * Ly * Lz * Lt;
  const int s = x + Lx * (y + Ly * (z + Lz * t));
  const int xp = (x + 1) % Lx + Lx * (y + Ly * (z + Lz * t)), xm = (x + Lx - 1) % Lx + Lx * (y + Ly * (z + Lz * t));
  const int yp = x + Lx * ((y + 1) % Ly + Ly * (z + Lz * t)), ym = x + Lx * ((y + Ly - 1) % Ly + Ly * (z + Lz * t));
  const int zp = x + Lx * (y + Ly * ((z + 1) % Lz + Lz * t)), zm = x + Lx * (y + Ly * ((z + Lz - 1) % Lz + Lz * t));
  const int tp = x + Lx * (y + Ly * (z + Lz * ((t + 1) % Lt))), tm = x + Lx * (y + Ly * (z + Lz * ((t + Lt - 1) % Lt)));
  const double2 *src = in + (long long)p * V * 12;
  Cx<double> acc[4][3], q[4][3], u[9];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[a][c] = mk<double>(0.0, 0.0);
  load_spinor<double, false>(src + 12LL * xp, q); load_link<double>(U, 0 * V + s, u);  term_fwd<double, 0>(q, u, acc);
  load_spinor<double, false>(src + 12LL * xm, q); load_link<double>(U, 0 * V + xm, u); term_bwd<double, 0>(q, u, acc);
  load_spinor<double, false>(src + 12LL * yp, q); load_link<double>(U, 1 * V + s, u);  term_fwd<double, 1>(q, u, acc);
  load_spinor<double, false>(src + 12LL * ym, q); load_link<double>(U, 1 * V + ym, u); term_bwd<double, 1>(q, u, acc);
  load_spinor<double, false>(src + 12LL * zp, q); load_link<double>(U, 2 * V + s, u);  term_fwd<double, 2>(q, u, acc);
  load_spinor<double, false>(src + 12LL * zm, q); load_link<double>(U, 2 * V + zm, u); term_bwd<double, 2>(q, u, acc);
  load_spinor<double, false>(src + 12LL * tp, q); load_link<double>(U, 3 * V + s, u);  term_fwd<double, 3>(q, u, acc);
  load_spinor<double, false>(src + 12LL * tm, q); load_link<double>(U, 3 * V + tm, u); term_bwd<double, 3>(q, u, acc);
  double2 *dst = out + (long long)p * V * 12 + 12LL * s;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) store_c(dst + 3 * a + c, acc[a][c]);
}

// Taxicab ball of radius r in Z^4 (all offsets with |dx| + |dy| + |dz| + |dt| <= r).
static std::vector<char4> taxicab_ball(int r) {
  std::vector<char4> o;
  for (int dt = -r; dt <= r; ++dt)
    for (int dz = -r; dz <= r; ++dz)
      for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx)
          if (std::abs(dx) + std::abs(dy) + std::abs(dz) + std::abs(dt) <= r)
            o.push_back(make_char4((signed char)dx, (signed char)dy, (signed char)dz, (signed char)dt));
  return o;
}

// Radius of the neighbourhood in which order k of a K-term trace is still read: the contraction
// reads offsets 0 and +-mu (radius 1), and each further order widens it by one hop.
static inline int completion_radius(int K, int k) { return std::max(1, K - k); }
static constexpr int PROBE_MAX_RADIUS = 8;

// Full-lattice applications of P per probe for the hopping traces: every order k <= depth is a
// full application, every order above it a local completion (hop_listed_kernel).  Chosen to
// minimise the site updates per probe, depth + sum_{k > depth} min(1, members x |ball| / V), unless
// the context fixes it (lqcd_set_probe_depth).
static int probe_depth_for(int fixed, const Colouring &col, int K) {
  if (K <= 2) return K - 1;
  // a fixed depth still keeps every completion ball within PROBE_MAX_RADIUS
  if (fixed > 0) return std::min(std::max(fixed, K - 1 - PROBE_MAX_RADIUS), K - 1);
  const double per_member = (double)col.ncls;  // sites per class member
  int best = K - 1;
  double best_cost = (double)(K - 1);
  for (int h = 1; h < K - 1; ++h) {
    if (completion_radius(K, h + 1) > PROBE_MAX_RADIUS) continue;
    double cost = h;
    for (int k = h + 1; k < K; ++k) cost += std::min(1.0, (double)taxicab_ball(completion_radius(K, k)).size() / per_member);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = h;
    }
  }
  // orders whose ball holds at least a member's share of the lattice run in full anyway: count them
  // in the depth, so that it is the number of full applications
  while (best < K - 1 && (double)taxicab_ball(completion_radius(K, best + 1)).size() >= per_member) ++best;
  return best;
}

static int probe_depth(const lqcd_ctx *ctx, const Colouring &col, int K) {
  return probe_depth_for(ctx->probe_depth, col, K);
}

template <typename T>
lqcd_status download_v(lqcd_ctx *ctx, const void *dev, std::vector<T> &h, size_t count) {
  h.resize(count);
  if (!count) return LQCD_OK;
  LQCD_CUDA(ctx, cudaMemcpyAsync(h.data(), dev, sizeof(T) * count, cudaMemcpyDeviceToHost, ctx->stream));
  LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return LQCD_OK;
}

lqcd_status upload_v(lqcd_ctx *ctx, const void *host, void *dev, size_t bytes) {
  if (!bytes) return LQCD_OK;
  LQCD_CUDA(ctx, cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, ctx->stream));
  LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return LQCD_OK;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

Colouring choose_colouring(const int *d, int K) {
  Colouring c;
  c.q = 1;
  c.ncls = 1;
  for (int i = 0; i < 4; ++i) {
    int p = d[i];
    for (int q = K + 1; q < d[i]; ++q)
      if (d[i] % q == 0) { p = q; break; }
    c.s[i] = p;
    c.ncls *= p;
  }
  const int sd = (K + 2) / 2;  // ceil((K + 1) / 2)
  int g = 0;
  for (int i = 0; i < 4; ++i) {
    if (d[i] % sd != 0) return c;
    int a = d[i] / sd, b = g;
    while (b) { const int t = a % b; a = b; b = t; }
    g = a;  // gcd of the L_mu / s
  }
  for (int q = 2; q <= g; ++q)
    if (g % q == 0) {
      const long long n = (long long)q * sd * sd * sd * sd;
      if (n < c.ncls) {
        for (int i = 0; i < 4; ++i) c.s[i] = sd;
        c.q = q;
        c.ncls = (int)n;
      }
      break;
    }
  return c;
}

}  // namespace

lqcd_status contract_launch(lqcd_ctx *ctx, const double2 *U, double kappa, const double2 *eta, const double2 *w,
                            int nrhs, double2 *out_dev) {
  const int *d = ctx->dims;
  const int Lt = d[3], Vs = d[0] * d[1] * d[2];
  int nchunk = std::max(1, std::min((Vs + CBT - 1) / CBT, std::max(1, (4 * ctx->sms) / std::max(1, nrhs * Lt))));
  void *p;
  LQCD_TRY(ws_get(ctx, WS_EST2, sizeof(double2) * (size_t)nrhs * Lt * nchunk * 9, &p));
  kbegin(ctx);
  contract_kernel<<<dim3(nchunk * Lt, nrhs), CBT, 0, ctx->stream>>>(U, kappa, eta, w, d[0], d[1], d[2], d[3], nchunk,
                                                                   (double2 *)p);
  // compulsory bytes: eta and w once, the links once (point-split operators)
  LQCD_TRY(launch_check_bytes(ctx, "contract_kernel", K_CONTRACT, (double)ctx->V * nrhs,
                              2.0 * nrhs * ctx->N * sizeof(double2) + 36.0 * ctx->V * sizeof(double2)));
  const int tot = nrhs * 9 * Lt;
  kbegin(ctx);
  contract_final<<<ceil_div(tot, 128), 128, 0, ctx->stream>>>((const double2 *)p, nchunk, Lt, nrhs, out_dev);
  return launch_check(ctx, "contract_final", K_CONTRACT, 0.0);
}

static lqcd_status scaled_acc(lqcd_ctx *ctx, const double2 *x, double2 *y, cd a, long long n) {
  kbegin(ctx);
  scaled_acc_kernel<<<std::min(ceil_div(n, 256), 8 * ctx->sms), 256, 0, ctx->stream>>>(x, y, make_double2(a.real(), a.imag()), n);
  return launch_check(ctx, "scaled_acc_kernel", K_BLAS1, (double)n);
}

// out = sum_k c_k (kappa P)^k eta   (c == NULL: all ones)
static lqcd_status hop_series_dev(lqcd_ctx *ctx, const double2 *U, double kappa, const double2 *eta, double2 *out,
                                  int nrhs, int K, const cd *c) {
  const long long n = (long long)nrhs * ctx->N;
  double2 *t0, *t1;
  LQCD_TRY(ws_get(ctx, WS_TMP2, sizeof(double2) * (size_t)n, (void **)&t0));
  LQCD_TRY(ws_get(ctx, WS_TMP3, sizeof(double2) * (size_t)n, (void **)&t1));
  LQCD_TRY(blas_zero(ctx, out, n));
  LQCD_TRY(scaled_acc(ctx, eta, out, c ? c[0] : cd(1.0, 0.0), n));
  const double2 *cur = eta;
  for (int k = 1; k < K; ++k) {
    double2 *nxt = (k & 1) ? t0 : t1;
    LQCD_TRY(wilson_launch(ctx, U, kappa, cur, nxt, nrhs, LQCD_PREC_F64, LQCD_APPLY_HOP));
    // term_k = kappa P term_{k-1}: fold kappa^k into the coefficient
    LQCD_TRY(scaled_acc(ctx, nxt, out, (c ? c[k] : cd(1.0, 0.0)) * std::pow(kappa, k), n));
    cur = nxt;
  }
  return LQCD_OK;
}

// out = sum_j a_j M^j eta
static lqcd_status poly_apply_dev(lqcd_ctx *ctx, const double2 *U, double kappa, const double2 *eta, double2 *out,
                                  int nrhs, int n, const cd *a) {
  const long long len = (long long)nrhs * ctx->N;
  double2 *t0, *t1;
  LQCD_TRY(ws_get(ctx, WS_TMP2, sizeof(double2) * (size_t)len, (void **)&t0));
  LQCD_TRY(ws_get(ctx, WS_TMP3, sizeof(double2) * (size_t)len, (void **)&t1));
  LQCD_TRY(blas_zero(ctx, out, len));
  LQCD_TRY(scaled_acc(ctx, eta, out, a[0], len));
  const double2 *cur = eta;
  for (int j = 1; j <= n; ++j) {
    double2 *nxt = (j & 1) ? t0 : t1;
    LQCD_TRY(wilson_launch(ctx, U, kappa, cur, nxt, nrhs, LQCD_PREC_F64, LQCD_APPLY_M));
    LQCD_TRY(scaled_acc(ctx, nxt, out, a[j], len));
    cur = nxt;
  }
  return LQCD_OK;
}

// out = gamma_5 E diag(d) E^dag eta
static lqcd_status deflate_dev(lqcd_ctx *ctx, const lqcd_defl *defl, const double2 *eta, double2 *out, int nrhs,
                               const cd *d) {
  const int k = defl->k;
  const long long N = ctx->N;
  double2 *coef, *tmp;
  LQCD_TRY(ws_get(ctx, WS_EST1, sizeof(double2) * (size_t)k * nrhs, (void **)&coef));
  LQCD_TRY(ws_get(ctx, WS_TMP4, sizeof(double2) * (size_t)nrhs * N, (void **)&tmp));
  if (ctx->defl_engine == LQCD_DEFL_TENSOR) {
    // split-precision tensor-core products; the slices of E are cached in the deflation object
    lqcd_defl *dm = const_cast<lqcd_defl *>(defl);
    if (!dm->tc) LQCD_TRY(tc_slices_make(ctx, defl->E, k, &dm->tc));
    double2 *dd;
    LQCD_TRY(ws_get(ctx, WS_TC_D, sizeof(double2) * (size_t)k, (void **)&dd));
    std::vector<double2> dh(k);
    for (int q = 0; q < k; ++q) dh[q] = make_double2(d[q].real(), d[q].imag());
    LQCD_TRY(upload_v(ctx, dh.data(), dd, sizeof(double2) * (size_t)k));
    LQCD_TRY(tc_vhx(ctx, dm->tc, eta, nrhs, coef));
    LQCD_TRY(tc_vc(ctx, dm->tc, coef, dd, nrhs, tmp));
    return blas_g5(ctx, tmp, out, nrhs);
  }
  LQCD_TRY(blas_multidot(ctx, defl->E, N, 0, k, eta, N, nrhs, coef));
  std::vector<double2> c;
  LQCD_TRY(download_v(ctx, coef, c, (size_t)k * nrhs));
  for (int q = 0; q < k; ++q)
    for (int r = 0; r < nrhs; ++r) {
      const double2 v = c[(size_t)q * nrhs + r];
      const cd w = cd(v.x, v.y) * d[q];
      c[(size_t)q * nrhs + r] = make_double2(w.real(), w.imag());
    }
  LQCD_TRY(upload_v(ctx, c.data(), coef, sizeof(double2) * c.size()));
  LQCD_TRY(blas_combine(ctx, defl->E, N, 0, k, coef, 1, tmp, N, N, nrhs));
  return blas_g5(ctx, tmp, out, nrhs);
}

// Min-Res coefficients: QR (classical Gram-Schmidt twice) of v = (M b, .., M^{n+1} b)
static lqcd_status poly_coeffs_dev(lqcd_ctx *ctx, const double2 *U, double kappa, uint64_t seed, int n,
                                   std::vector<cd> &a, int flags = LQCD_APPLY_M) {
  const long long N = ctx->N;
  double2 *Q, *b, *h;
  double *nrm;
  LQCD_TRY(ws_get(ctx, WS_PROBE, sizeof(double2) * (size_t)(n + 2) * N, (void **)&Q));
  LQCD_TRY(ws_get(ctx, WS_TMP4, sizeof(double2) * (size_t)N, (void **)&b));
  LQCD_TRY(ws_get(ctx, WS_EST1, sizeof(double2) * (size_t)(2 * (n + 2) + 4), (void **)&h));
  nrm = (double *)(h + 2 * (n + 2));
  LQCD_TRY(noise_launch(ctx, seed, 0xFFFFFFFFu, 1, b));
  // column j of v is M^{j+1} b; build the powers in place, then orthogonalise
  const double2 *prev = b;
  for (int j = 0; j <= n; ++j) {
    LQCD_TRY(wilson_launch(ctx, U, kappa, prev, Q + (long long)j * N, 1, LQCD_PREC_F64, flags));
    prev = Q + (long long)j * N;
  }
  dense::Mat R(n + 1, n + 1);
  for (int j = 0; j <= n; ++j) {
    double2 *w = Q + (long long)j * N;
    std::vector<double2> h1, h2;
    if (j > 0) {
      LQCD_TRY(blas_multidot(ctx, Q, N, 0, j, w, N, 1, h));
      LQCD_TRY(blas_multiaxpy(ctx, Q, N, 0, j, h, -1.0, w, N, 1));
      LQCD_TRY(download_v(ctx, h, h1, j));
      LQCD_TRY(blas_multidot(ctx, Q, N, 0, j, w, N, 1, h));
      LQCD_TRY(blas_multiaxpy(ctx, Q, N, 0, j, h, -1.0, w, N, 1));
      LQCD_TRY(download_v(ctx, h, h2, j));
    }
    LQCD_TRY(blas_norms(ctx, w, N, 1, nrm));
    std::vector<double> nr;
    LQCD_TRY(download_v(ctx, nrm, nr, 1));
    for (int i = 0; i < j; ++i) R(i, j) = cd(h1[i].x + h2[i].x, h1[i].y + h2[i].y);
    R(j, j) = nr[0];
    if (!(nr[0] > 0.0)) return set_err(ctx, LQCD_ERR_INVALID_ARG, "poly_coeffs: Krylov powers are linearly dependent");
    LQCD_TRY(blas_invscale(ctx, w, nrm, N, 1));
  }
  LQCD_TRY(blas_multidot(ctx, Q, N, 0, n + 1, b, N, 1, h));
  std::vector<double2> y;
  LQCD_TRY(download_v(ctx, h, y, n + 1));
  a.assign(n + 1, cd(0.0, 0.0));
  for (int i = n; i >= 0; --i) {
    cd s = cd(y[i].x, y[i].y);
    for (int j = i + 1; j <= n; ++j) s -= R(i, j) * a[j];
    a[i] = s / R(i, i);
  }
  return LQCD_OK;
}

// t[(k * 9 + op) * Lt + t] for k < K
static lqcd_status hop_traces_dev(lqcd_ctx *ctx, const double2 *U, double kappa, int K, std::vector<cd> &tr) {
  const int *d = ctx->dims;
  const int Lt = d[3];
  const long long N = ctx->N;
  const Colouring col = choose_colouring(d, K);
  const long long nprobes = 12LL * col.ncls;
  // probes per batch: bounded by memory (three probe-sized buffers of at most 2 GiB together)
  const int B = (int)std::min<long long>(nprobes, std::max<long long>(1, std::min<long long>(192, (1LL << 31) / (N * 16 * 3))));
  double2 *Z, *W0, *W1, *cd_dev;
  LQCD_TRY(ws_get(ctx, WS_PROBE, sizeof(double2) * (size_t)B * N, (void **)&Z));
  LQCD_TRY(ws_get(ctx, WS_TMP2, sizeof(double2) * (size_t)B * N, (void **)&W0));
  LQCD_TRY(ws_get(ctx, WS_TMP3, sizeof(double2) * (size_t)B * N, (void **)&W1));
  LQCD_TRY(ws_get(ctx, WS_EST0, sizeof(double2) * (size_t)K * B * 9 * Lt, (void **)&cd_dev));
  tr.assign((size_t)K * 9 * Lt, cd(0.0, 0.0));
  // meet in the middle: full applications up to `depth`, local completion above it; the offsets of
  // every completion ball, concatenated (ball_at[r] = first offset of radius r)
  const int depth = probe_depth(ctx, col, K);
  const long long nmem = ctx->V / col.ncls;
  std::vector<char4> all_offs;
  std::vector<int> ball_at(PROBE_MAX_RADIUS + 1, 0), ball_n(PROBE_MAX_RADIUS + 1, 0);
  for (int r = 1; r <= std::min(PROBE_MAX_RADIUS, K); ++r) {
    const std::vector<char4> b = taxicab_ball(r);
    ball_at[r] = (int)all_offs.size();
    ball_n[r] = (int)b.size();
    all_offs.insert(all_offs.end(), b.begin(), b.end());
  }
  char4 *offs = nullptr;
  if (depth < K - 1) {
    LQCD_TRY(ws_get(ctx, WS_PROBE_OFF, sizeof(char4) * all_offs.size(), (void **)&offs));
    LQCD_CUDA(ctx, cudaMemcpyAsync(offs, all_offs.data(), sizeof(char4) * all_offs.size(), cudaMemcpyHostToDevice,
                                   ctx->stream));
    LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  std::vector<double2> h;
  // one thread per (operator, timeslice), at most what the kernel's register use allows per block
  // (the kernel strides over the rest)
  cudaFuncAttributes fa;
  LQCD_CUDA(ctx, cudaFuncGetAttributes(&fa, probe_contract_kernel));
  const int cthreads = std::max(32, std::min(std::min(1024, fa.maxThreadsPerBlock) / 32 * 32, ((9 * Lt + 31) / 32) * 32));
  for (long long p0 = 0; p0 < nprobes; p0 += B) {
    const int nb = (int)std::min<long long>(B, nprobes - p0);
    kbegin(ctx);
    probe_kernel<<<dim3(ceil_div(ctx->V, 128), nb), 128, 0, ctx->stream>>>((int)p0, nb, d[0], d[1], d[2], d[3], col, Z);
    LQCD_TRY(launch_check(ctx, "probe_kernel", K_PROBE, (double)ctx->V * nb));
    const double2 *cur = Z;
    for (int k = 0; k < K; ++k) {
      double2 *nxt = (k & 1) ? W0 : W1;
      if (k > 0 && k <= depth) {
        LQCD_TRY(wilson_launch(ctx, U, kappa, cur, nxt, nb, LQCD_PREC_F64, LQCD_APPLY_HOP));
      } else if (k > depth) {
        const int r = completion_radius(K, k);
        const long long work = nmem * (long long)ball_n[r];
        if (work >= ctx->V) {
          LQCD_TRY(wilson_launch(ctx, U, kappa, cur, nxt, nb, LQCD_PREC_F64, LQCD_APPLY_HOP));
        } else {
          kbegin(ctx);
          hop_listed_kernel<<<dim3((unsigned)ceil_div(work, 128), nb), 128, 0, ctx->stream>>>(
              U, cur, nxt, offs + ball_at[r], ball_n[r], (int)p0, nb, d[0], d[1], d[2], d[3], col);
          LQCD_TRY(launch_check(ctx, "hop_listed_kernel", K_PROBE, (double)work * nb));
        }
      } else {
        nxt = Z;
      }
      kbegin(ctx);
      probe_contract_kernel<<<nb, cthreads, 0, ctx->stream>>>(U, kappa, nxt, (int)p0, nb, d[0], d[1], d[2], d[3], col,
                                                               cd_dev + (size_t)k * nb * 9 * Lt);
      LQCD_TRY(launch_check(ctx, "probe_contract_kernel", K_PROBE, (double)nb * ctx->V / col.ncls));
      cur = nxt;
    }
    LQCD_TRY(download_v(ctx, cd_dev, h, (size_t)K * nb * 9 * Lt));
    for (int k = 0; k < K; ++k)
      for (int p = 0; p < nb; ++p)
        for (int q = 0; q < 9 * Lt; ++q) {
          const double2 v = h[((size_t)k * nb + p) * 9 * Lt + q];
          tr[(size_t)k * 9 * Lt + q] += cd(v.x, v.y);
        }
  }
  return LQCD_OK;
}

// xi[q] = e_q^dag gamma_5 tilde M^{-1} e_q
static lqcd_status xi_dev(lqcd_ctx *ctx, const double2 *U, double kappa, const lqcd_defl *defl, int sub, int K,
                          const cd *coeffs, std::vector<cd> &xi) {
  const int k = defl->k;
  const long long N = ctx->N;
  double2 *T, *G, *h;
  LQCD_TRY(ws_get(ctx, WS_TMP5, sizeof(double2) * (size_t)k * N, (void **)&T));
  LQCD_TRY(ws_get(ctx, WS_TMP1, sizeof(double2) * (size_t)k * N, (void **)&G));
  LQCD_TRY(ws_get(ctx, WS_EST1, sizeof(double2) * (size_t)k, (void **)&h));
  if (sub == LQCD_SUB_PERT) {
    LQCD_TRY(hop_series_dev(ctx, U, kappa, defl->E, T, k, K, nullptr));
  } else if (sub == LQCD_SUB_POLY) {
    LQCD_TRY(poly_apply_dev(ctx, U, kappa, defl->E, T, k, K - 1, coeffs));
  } else {
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "xi_inverse: sub must be LQCD_SUB_PERT or LQCD_SUB_POLY");
  }
  LQCD_TRY(blas_g5(ctx, T, G, k));
  // per-vector dot <e_q, g5 T_q>: basis of right-hand side q is e_q itself (vrs = N)
  LQCD_TRY(blas_multidot(ctx, defl->E, 0, N, 1, G, N, k, h));
  std::vector<double2> hv;
  LQCD_TRY(download_v(ctx, h, hv, k));
  xi.resize(k);
  for (int q = 0; q < k; ++q) xi[q] = cd(hv[q].x, hv[q].y);
  return LQCD_OK;
}

lqcd_status hop_series_launch(lqcd_ctx *ctx, const double2 *U, double kappa, const double2 *eta, double2 *out, int nrhs,
                              int K, const cd *c) {
  return hop_series_dev(ctx, U, kappa, eta, out, nrhs, K, c);
}

lqcd_status hop_traces_launch(lqcd_ctx *ctx, const double2 *U, double kappa, int K, std::vector<cd> &tr) {
  return hop_traces_dev(ctx, U, kappa, K, tr);
}

// ---- C ABI -----------------------------------------------------------------------------------
extern "C" {

lqcd_status lqcd_contract(lqcd_ctx *ctx, const double *links, double kappa, const double *eta, const double *w,
                          int nrhs, double *out) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_full(ctx, "contract"));
  if (!links || !eta || !w || !out || nrhs < 1 || nrhs > 65535) return set_err(ctx, LQCD_ERR_INVALID_ARG, "contract: bad arguments");
  double2 *dev;
  const size_t cnt = (size_t)nrhs * 9 * ctx->dims[3];
  LQCD_TRY(ws_get(ctx, WS_EST0, sizeof(double2) * cnt, (void **)&dev));
  LQCD_TRY(contract_launch(ctx, (const double2 *)links, kappa, (const double2 *)eta, (const double2 *)w, nrhs, dev));
  LQCD_CUDA(ctx, cudaMemcpyAsync(out, dev, sizeof(double2) * cnt, cudaMemcpyDeviceToHost, ctx->stream));
  LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return LQCD_OK;
}

lqcd_status lqcd_hop_series(lqcd_ctx *ctx, const double *links, double kappa, const double *eta, double *out, int nrhs,
                            int K, const double *c) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_full(ctx, "hop_series"));
  if (!links || !eta || !out || nrhs < 1 || K < 1 || K > 64 || eta == out)
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "hop_series: bad arguments");
  std::vector<cd> cc;
  if (c) cc.assign((const cd *)c, (const cd *)c + K);
  return hop_series_dev(ctx, (const double2 *)links, kappa, (const double2 *)eta, (double2 *)out, nrhs, K,
                        c ? cc.data() : nullptr);
}

lqcd_status lqcd_poly_apply(lqcd_ctx *ctx, const double *links, double kappa, const double *eta, double *out, int nrhs,
                            int n, const double *a) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  if (!links || !eta || !out || !a || nrhs < 1 || n < 0 || n > 64 || eta == out)
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "poly_apply: bad arguments");
  std::vector<cd> aa((const cd *)a, (const cd *)a + n + 1);
  return poly_apply_dev(ctx, (const double2 *)links, kappa, (const double2 *)eta, (double2 *)out, nrhs, n, aa.data());
}

lqcd_status lqcd_poly_coeffs(lqcd_ctx *ctx, const double *links, double kappa, uint64_t seed, int n, double *a) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_full(ctx, "poly_coeffs"));
  if (!links || !a || n < 0 || n > 64) return set_err(ctx, LQCD_ERR_INVALID_ARG, "poly_coeffs: bad arguments");
  std::vector<cd> av;
  LQCD_TRY(poly_coeffs_dev(ctx, (const double2 *)links, kappa, seed, n, av));
  memcpy(a, av.data(), sizeof(cd) * av.size());
  return LQCD_OK;
}

lqcd_status lqcd_deflate_project(lqcd_ctx *ctx, const lqcd_defl *defl, const double *eta, double *out, int nrhs,
                                 const double *d) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  if (!defl || !eta || !out || !d || nrhs < 1 || eta == out) return set_err(ctx, LQCD_ERR_INVALID_ARG, "deflate_project: bad arguments");
  std::vector<cd> dd((const cd *)d, (const cd *)d + defl->k);
  return deflate_dev(ctx, defl, (const double2 *)eta, (double2 *)out, nrhs, dd.data());
}

lqcd_status lqcd_probe_classes(const int dims[4], int K, int *nclasses, int *classes) {
  if (!dims || !nclasses || K < 1 || K > 64) return LQCD_ERR_INVALID_ARG;
  for (int i = 0; i < 4; ++i)
    if (dims[i] < 2 || dims[i] > 1024) return LQCD_ERR_INVALID_ARG;
  const Colouring c = choose_colouring(dims, K);
  *nclasses = c.ncls;
  if (classes) {
    long long s = 0;
    for (int t = 0; t < dims[3]; ++t)
      for (int z = 0; z < dims[2]; ++z)
        for (int y = 0; y < dims[1]; ++y)
          for (int x = 0; x < dims[0]; ++x) classes[s++] = class_of(c, x, y, z, t);
  }
  return LQCD_OK;
}

lqcd_status lqcd_probe_depth(const int dims[4], int K, int fixed, int *depth) {
  if (!dims || !depth || K < 1 || K > 64 || fixed < 0 || fixed > 64) return LQCD_ERR_INVALID_ARG;
  for (int i = 0; i < 4; ++i)
    if (dims[i] < 2 || dims[i] > 1024) return LQCD_ERR_INVALID_ARG;
  *depth = probe_depth_for(fixed, choose_colouring(dims, K), K);
  return LQCD_OK;
}

lqcd_status lqcd_hop_traces(lqcd_ctx *ctx, const double *links, double kappa, int K, double *t) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_full(ctx, "hop_traces"));
  if (!links || !t || K < 1 || K > 64) return set_err(ctx, LQCD_ERR_INVALID_ARG, "hop_traces: bad arguments");
  std::vector<cd> tr;
  LQCD_TRY(hop_traces_dev(ctx, (const double2 *)links, kappa, K, tr));
  memcpy(t, tr.data(), sizeof(cd) * tr.size());
  return LQCD_OK;
}

lqcd_status lqcd_xi_inverse(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_defl *defl, int sub, int K,
                            const double *coeffs, double *xi) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_full(ctx, "xi_inverse"));
  if (!links || !defl || !xi || K < 1 || K > 65 || (sub == LQCD_SUB_POLY && !coeffs))
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "xi_inverse: bad arguments");
  std::vector<cd> cc;
  if (coeffs) cc.assign((const cd *)coeffs, (const cd *)coeffs + K);
  std::vector<cd> out;
  LQCD_TRY(xi_dev(ctx, (const double2 *)links, kappa, defl, sub, K, coeffs ? cc.data() : nullptr, out));
  memcpy(xi, out.data(), sizeof(cd) * out.size());
  return LQCD_OK;
}

}  // extern "C"

// ---- whole loop estimate: per-configuration setup, then noise batches ------------------------------
lqcd_status special_solves(lqcd_ctx *ctx, const double *links, double kappa, const double2 *b2, double2 *x2,
                           const lqcd_krylov_opts *o, lqcd_solve_info *info, lqcd_defl **defl_m, lqcd_defl **defl_h);
lqcd_status defl_rayleigh(lqcd_ctx *ctx, lqcd_defl *d, const double *links, double kappa, int flags);
lqcd_status proj_core_entry(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_defl *defl, const double2 *b,
                            double2 *x, int nrhs, const lqcd_krylov_opts *o, lqcd_solve_info *info);

// Setup state of one gauge configuration (steps 1-3): the two deflation spaces, the polynomial, the
// 1/xi' of both combined modes and every add-back; the noise phase (step 4) reads it.
struct lqcd_loop {
  lqcd_ctx *ctx = nullptr;
  double kappa = 0.0;
  lqcd_est_opts o{};
  int modes = 0, Kt = 0, Q = 0, block = 0;
  lqcd_defl *dm = nullptr, *dh = nullptr;  // GMRES-Proj space of M; eigenpairs of M'
  bool own_m = false, own_h = false;
  std::vector<cd> a, bcoef, xi_p, xi_q, lam, dl, dlp, dlq;
  std::vector<cd> add;  // [LQCD_NMODES][9][Lt]
  // ES (Sec. 5.3): Ritz pairs (lambda_q, e_R^q) of M on dm; left vectors e_L^q = gamma_5 e_R^{p(q)} /
  // conj(n_q) with lambda_p(q) = conj(lambda_q), n_q = (gamma_5 e_R^p)^dag e_R^q; es_coef[q] =
  // 1 / (lambda_q n_q) (0 for a mode without a partner); g5E = gamma_5 e_R (k fields, device)
  int es_k = 0, es_found = 0;
  std::vector<int> es_perm;
  std::vector<cd> es_coef;
  double2 *g5E = nullptr;
  std::vector<double> prec_a;  // polynomial preconditioner of the noise solves (interleaved complex)
  // even/odd noise solves (opts.evenodd): the reduced context, its GMRES-Proj space, and the full
  // eigenpairs of M mapped from the reduced ones for ES; des = the ES space (dm without even/odd)
  lqcd_ctx *ce = nullptr;
  lqcd_defl *dme = nullptr, *des_own = nullptr;
  const lqcd_defl *des = nullptr;
  long matvecs = 0;
  double seconds = 0.0, eres = 0.0;
  ~lqcd_loop() {
    if (g5E) cudaFree(g5E);
    if (own_m && dm) lqcd_defl_destroy(dm);
    if (own_h && dh) lqcd_defl_destroy(dh);
    if (des_own) lqcd_defl_destroy(des_own);
    if (dme) lqcd_defl_destroy(dme);
    if (ce) lqcd_ctx_destroy(ce);
  }
};

namespace {

lqcd_status check_est_opts(lqcd_ctx *ctx, const lqcd_est_opts *o) {
  if (o->nnoise < 1 || o->block < 0 || o->m < 2 || o->k < 1 || o->k >= o->m || o->K < 1 || o->npoly < 0 ||
      o->npoly > 63 || o->K > 64 || !(o->tol > 0) || !(o->tol_special > 0) || o->max_cycles < 1 || !(o->eig_tol >= 0))
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "loop estimate: bad options");
  if (o->prec < LQCD_PREC_F64 || o->prec > LQCD_PREC_BF16)
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "loop estimate: prec must be one of LQCD_PREC_*");
  if (o->system != LQCD_SYS_M && o->system != LQCD_SYS_MG5)
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "loop estimate: system must be LQCD_SYS_M or LQCD_SYS_MG5");
  if (o->prec_degree < 0 || o->prec_degree > 32)
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "loop estimate: prec_degree must be in 0..32");
  if (o->evenodd != 0 && o->evenodd != 1) return set_err(ctx, LQCD_ERR_INVALID_ARG, "loop estimate: evenodd must be 0 or 1");
  if (o->evenodd) {
    for (int i = 0; i < 4; ++i)
      if (ctx->dims[i] & 1) return set_err(ctx, LQCD_ERR_INVALID_ARG, "loop estimate: even/odd needs even extents");
    if (o->prec != LQCD_PREC_F64 || o->prec_degree != 0)
      return set_err(ctx, LQCD_ERR_INVALID_ARG, "loop estimate: even/odd solves are plain FP64 without preconditioner");
  }
  return LQCD_OK;
}

lqcd_krylov_opts noise_solver_opts(const lqcd_loop *L) {
  const lqcd_est_opts *o = &L->o;
  lqcd_krylov_opts k{o->m_inner > 0 ? o->m_inner : o->m - o->k, 0, o->tol, o->max_cycles, LQCD_SYS_M, o->prec,
                     o->inner_tol, 0.0};
  if (!L->prec_a.empty()) {
    k.poly_degree = (int)L->prec_a.size() / 2 - 1;
    k.poly_coeffs = L->prec_a.data();
  }
  return k;
}

// ES data (Sec. 5.3, left vectors by gamma_5-hermiticity) from the Ritz pairs of M on L->dm, and the
// ES add-back sum_q (1 / lambda_q) e_L^q^dag Theta e_R^q per timeslice into addES(op, t)
template <typename F>
lqcd_status es_setup(lqcd_loop *L, const double2 *U, F addES) {
  lqcd_ctx *ctx = L->ctx;
  const lqcd_defl *dm = L->des;
  const int k = dm->k, Lt = ctx->dims[3];
  const long long N = ctx->N;
  L->es_k = k;
  L->es_perm.assign(k, 0);
  L->es_coef.assign(k, cd(0.0, 0.0));
  L->es_found = 0;
  std::vector<char> found(k, 0);
  for (int q = 0; q < k; ++q) {
    const cd lq(dm->lam[q].x, dm->lam[q].y);
    int best = 0;
    double dist = INFINITY;
    for (int p = 0; p < k; ++p) {
      const double d = std::abs(cd(dm->lam[p].x, dm->lam[p].y) - std::conj(lq));
      if (d < dist) { dist = d; best = p; }
    }
    L->es_perm[q] = best;
    found[q] = dist <= 1e-8 * std::max(std::abs(lq), 1e-300);
  }
  if (cudaMalloc(&L->g5E, sizeof(double2) * (size_t)k * N) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, LQCD_ERR_OOM, "ES: allocation of the left-vector basis failed");
  }
  LQCD_TRY(blas_g5(ctx, dm->E, L->g5E, k));
  double2 *P5, *h, *cdv;
  LQCD_TRY(ws_get(ctx, WS_PROBE, sizeof(double2) * (size_t)k * N, (void **)&P5));
  LQCD_TRY(ws_get(ctx, WS_EST1, sizeof(double2) * (size_t)k, (void **)&h));
  LQCD_TRY(ws_get(ctx, WS_EST0, sizeof(double2) * (size_t)k * 9 * Lt, (void **)&cdv));
  for (int q = 0; q < k; ++q) LQCD_TRY(blas_copy(ctx, L->g5E + (size_t)L->es_perm[q] * N, P5 + (size_t)q * N, N));
  // n_q = <gamma_5 e_R^p(q), e_R^q>: the basis of right-hand side q is P5_q itself
  LQCD_TRY(blas_multidot(ctx, P5, 0, N, 1, dm->E, N, k, h));
  std::vector<double2> nh, dens;
  LQCD_TRY(download_v(ctx, h, nh, (size_t)k));
  LQCD_TRY(contract_launch(ctx, U, L->kappa, P5, dm->E, k, cdv));
  LQCD_TRY(download_v(ctx, cdv, dens, (size_t)k * 9 * Lt));
  for (int q = 0; q < k; ++q) {
    const cd nq(nh[q].x, nh[q].y), lq(dm->lam[q].x, dm->lam[q].y);
    if (!found[q] || std::abs(nq) == 0.0) continue;
    L->es_coef[q] = 1.0 / (lq * nq);
    ++L->es_found;
    for (int op = 0; op < 9; ++op)
      for (int t = 0; t < Lt; ++t) {
        const double2 v = dens[((size_t)q * 9 + op) * Lt + t];
        addES(op, t) += L->es_coef[q] * cd(v.x, v.y);
      }
  }
  return LQCD_OK;
}

// y = sum_q e_R^q (1 / lambda_q) (e_L^q^dag eta) for nb fields (the ES subtraction vector)
lqcd_status es_vector(lqcd_loop *L, const double2 *eta, double2 *y, int nb) {
  lqcd_ctx *ctx = L->ctx;
  const int k = L->es_k;
  const long long N = ctx->N;
  double2 *g;
  LQCD_TRY(ws_get(ctx, WS_EST1, sizeof(double2) * (size_t)k * nb, (void **)&g));
  LQCD_TRY(blas_multidot(ctx, L->g5E, N, 0, k, eta, N, nb, g));
  std::vector<double2> gh, c((size_t)k * nb);
  LQCD_TRY(download_v(ctx, g, gh, (size_t)k * nb));
  for (int q = 0; q < k; ++q)
    for (int r = 0; r < nb; ++r) {
      const double2 v = gh[(size_t)L->es_perm[q] * nb + r];
      const cd w = cd(v.x, v.y) * L->es_coef[q];
      c[(size_t)q * nb + r] = make_double2(w.real(), w.imag());
    }
  LQCD_TRY(upload_v(ctx, c.data(), g, sizeof(double2) * c.size()));
  return blas_combine(ctx, L->des->E, N, 0, k, g, 1, y, N, N, nb);
}

// ES space of an even/odd loop: the full eigenpairs of M from the Ritz pairs (mu_q, v_e^q) of hat M
// on L->dme (both full pairs of each; a pair with mu = 1 within 1e-12 is left out)
lqcd_status eo_es_space(lqcd_loop *L, const double *links) {
  lqcd_ctx *ctx = L->ctx, *ce = L->ce;
  const lqcd_defl *d = L->dme;
  std::vector<double> mu;
  std::vector<int> keep;
  for (int q = 0; q < d->k; ++q) {
    const cd m(d->lam[q].x, d->lam[q].y);
    if (std::abs(std::sqrt(cd(1.0, 0.0) - m)) > 1e-12) {
      keep.push_back(q);
      mu.push_back(m.real());
      mu.push_back(m.imag());
    }
  }
  const int Q = (int)keep.size();
  if (Q == 0) return LQCD_OK;
  double2 *Ve = nullptr, *E = nullptr;
  if (cudaMalloc(&Ve, sizeof(double2) * (size_t)Q * ce->N) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, LQCD_ERR_OOM, "ES (even/odd): allocation failed");
  }
  struct G { void *p; ~G() { if (p) cudaFree(p); } } g{Ve};
  for (int i = 0; i < Q; ++i) LQCD_TRY(blas_copy(ce, d->E + (size_t)keep[i] * ce->N, Ve + (size_t)i * ce->N, ce->N));
  if (cudaMalloc(&E, sizeof(double2) * 2 * (size_t)Q * ctx->N) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, LQCD_ERR_OOM, "ES (even/odd): allocation failed");
  }
  struct G2 { void *p; ~G2() { if (p) cudaFree(p); } } g2{E};
  std::vector<double> lam(4 * (size_t)Q);
  const lqcd_status st = lqcd_eo_full_eigenpairs(ce, links, L->kappa, mu.data(), (const double *)Ve, Q, 1e-12,
                                                 lam.data(), (double *)E);
  if (st != LQCD_OK) return set_err(ctx, st, "ES (even/odd): %s", ce->err.c_str());
  LQCD_TRY(lqcd_defl_import(ctx, 2 * Q, (const double *)E, lam.data(), &L->des_own));
  L->des_own->hermitian = 0;
  return LQCD_OK;
}

// x = M^{-1} eta for nb noises through the reduced system: be = eta_e + kappa P_eo eta_o, hat M x_e =
// be (or hat M' y_e = be, x_e = gamma_5 y_e) by GMRES-Proj to tol * min(1, ||eta|| / ||be||) (so that
// the full relative residual, equal to ||be - hat M x_e|| / ||eta||, is at most tol), then
// x_o = eta_o + kappa P_oe x_e; info->true_resid is the full FP64 true residual of x (r in scratch)
lqcd_status eo_noise_solve(lqcd_loop *L, const double2 *U, const double2 *eta, double2 *x, double2 *r, int nb,
                           lqcd_solve_info *info) {
  lqcd_ctx *ctx = L->ctx, *ce = L->ce;
  ce->stream = ctx->stream;
  const long long Ne = ce->N, N = ctx->N;
  double2 *be, *xe, *ye;
  LQCD_TRY(ws_get(ce, WS_NBLK, sizeof(double2) * (size_t)nb * Ne * 3, (void **)&be));
  xe = be + (size_t)nb * Ne;
  ye = xe + (size_t)nb * Ne;
  LQCD_TRY(eo_rhs_launch(ce, U, L->kappa, eta, be, nb));
  double *nrm;
  LQCD_TRY(ws_get(ctx, WS_EST2, sizeof(double) * 2 * (size_t)nb, (void **)&nrm));
  LQCD_TRY(blas_norms(ctx, eta, N, nb, nrm));
  LQCD_TRY(blas_norms(ce, be, Ne, nb, nrm + nb));
  std::vector<double> nh;
  LQCD_TRY(download_v(ctx, nrm, nh, 2 * (size_t)nb));
  lqcd_krylov_opts po = noise_solver_opts(L);
  double ratio = 1.0;
  for (int i = 0; i < nb; ++i)
    if (nh[nb + i] > 0.0) ratio = std::min(ratio, nh[i] / nh[nb + i]);
  po.tol = L->o.tol * ratio;
  const bool herm = L->dme->hermitian;
  lqcd_solve_info pi{};
  const lqcd_status st = proj_core_entry(ce, (const double *)U, L->kappa, L->dme, be, herm ? ye : xe, nb, &po, &pi);
  if (st != LQCD_OK && st != LQCD_ERR_NOT_CONVERGED) return set_err(ctx, st, "even/odd noise solve: %s", ce->err.c_str());
  if (herm) LQCD_TRY(blas_g5(ce, ye, xe, nb));
  LQCD_TRY(eo_reconstruct_launch(ce, U, L->kappa, xe, eta, x, nb));
  // full true residual r = eta - M x
  LQCD_TRY(wilson_launch(ctx, U, L->kappa, x, r, nb, LQCD_PREC_F64, LQCD_APPLY_M));
  LQCD_TRY(scaled_acc(ctx, eta, r, cd(-1.0, 0.0), (long long)nb * N));
  LQCD_TRY(blas_norms(ctx, r, N, nb, nrm + nb));
  LQCD_TRY(download_v(ctx, nrm, nh, 2 * (size_t)nb));
  double worst = 0.0;
  for (int i = 0; i < nb; ++i) worst = std::max(worst, nh[i] > 0.0 ? nh[nb + i] / nh[i] : 0.0);
  *info = pi;
  info->true_resid = worst;
  info->converged = pi.converged && worst <= L->o.tol;
  return LQCD_OK;
}

// Steps 2-3 given the two spaces (L->dm, L->dh set): Min-Res coefficients (unless given), b_k,
// hopping traces, 1/xi', the eigen add-back densities and the add-backs of all six modes; then the
// block width (autotuned when opts->block == 0).
lqcd_status loop_finish_setup(lqcd_loop *L, const double2 *U, const double *links, const double *a_given) {
  lqcd_ctx *ctx = L->ctx;
  const lqcd_est_opts *o = &L->o;
  const double kappa = L->kappa;
  const int Lt = ctx->dims[3];
  const long long N = ctx->N;
  const lqcd_defl *dh = L->dh;
  L->Q = dh->k;
  const int Q = L->Q;
  NvtxRange nv("loop setup: polynomial, traces, 1/xi', add-backs");
  if (a_given) {
    L->a.assign((const cd *)a_given, (const cd *)a_given + o->npoly + 1);
  } else {
    LQCD_TRY(poly_coeffs_dev(ctx, U, kappa, o->seed, o->npoly, L->a));
    L->matvecs += o->npoly + 1;
  }
  L->bcoef.assign(o->npoly + 1, cd(0.0, 0.0));  // b_k = (-1)^k sum_{j>=k} C(j,k) a_j
  for (int k = 0; k <= o->npoly; ++k) {
    double binom = 1.0;  // C(j, k) for j = k
    for (int j = k; j <= o->npoly; ++j) {
      L->bcoef[k] += ((k & 1) ? -1.0 : 1.0) * binom * L->a[j];
      binom = binom * (j + 1) / (j + 1 - k);
    }
  }
  std::vector<cd> tr;
  LQCD_TRY(hop_traces_dev(ctx, U, kappa, L->Kt, tr));
  LQCD_TRY(xi_dev(ctx, U, kappa, dh, LQCD_SUB_PERT, o->K, nullptr, L->xi_p));
  LQCD_TRY(xi_dev(ctx, U, kappa, dh, LQCD_SUB_POLY, o->npoly + 1, L->a.data(), L->xi_q));
  L->matvecs += (long)Q * (o->K - 1 + o->npoly);
  // eigen add-back densities: contract(e_q, g5 e_q) per q
  std::vector<cd> eig_t((size_t)Q * 9 * Lt);
  {
    double2 *G, *cdv;
    LQCD_TRY(ws_get(ctx, WS_TMP1, sizeof(double2) * (size_t)Q * N, (void **)&G));
    LQCD_TRY(ws_get(ctx, WS_EST0, sizeof(double2) * (size_t)Q * 9 * Lt, (void **)&cdv));
    LQCD_TRY(blas_g5(ctx, dh->E, G, Q));
    LQCD_TRY(contract_launch(ctx, U, kappa, dh->E, G, Q, cdv));
    std::vector<double2> h;
    LQCD_TRY(download_v(ctx, cdv, h, (size_t)Q * 9 * Lt));
    for (size_t i = 0; i < h.size(); ++i) eig_t[i] = cd(h[i].x, h[i].y);
  }
  L->lam.resize(Q);
  L->dl.resize(Q);
  L->dlp.resize(Q);
  L->dlq.resize(Q);
  L->eres = 0.0;
  for (int q = 0; q < Q; ++q) {
    L->lam[q] = cd(dh->lam[q].x, dh->lam[q].y);
    L->dl[q] = 1.0 / L->lam[q];
    L->dlp[q] = 1.0 / L->lam[q] - L->xi_p[q];
    L->dlq[q] = 1.0 / L->lam[q] - L->xi_q[q];
    if (q < (int)dh->eres.size()) L->eres = std::max(L->eres, dh->eres[q]);
  }
  L->add.assign((size_t)LQCD_NMODES * 9 * Lt, cd(0.0, 0.0));
  auto A = [&](int mode, int op, int t) -> cd & { return L->add[((size_t)mode * 9 + op) * Lt + t]; };
  if ((L->modes & LQCD_SUB_ES) && L->prec_a.empty()) {
    if (L->ce && !L->dme->hermitian) {
      // ES from the full eigenpairs of M built from the reduced pairs (mu, v_e) of hat M (Sec. 7)
      LQCD_TRY(eo_es_space(L, links));
      L->des = L->des_own;
    } else if (!L->ce && !L->dm->hermitian) {
      L->des = L->dm;
    }
    if (L->des) LQCD_TRY(es_setup(L, U, [&](int op, int t) -> cd & { return A(6, op, t); }));
  }
  for (int op = 0; op < 9; ++op)
    for (int t = 0; t < Lt; ++t) {
      cd pert = 0.0, poly = 0.0, e1 = 0.0, ep = 0.0, eq = 0.0;
      double kk = 1.0;
      for (int k = 0; k < L->Kt; ++k) {
        const cd tk = tr[((size_t)k * 9 + op) * Lt + t];
        if (k < o->K) pert += kk * tk;
        if (k <= o->npoly) poly += L->bcoef[k] * kk * tk;
        kk *= kappa;
      }
      for (int q = 0; q < Q; ++q) {
        const cd et = eig_t[((size_t)q * 9 + op) * Lt + t];
        e1 += L->dl[q] * et;
        ep += L->dlp[q] * et;
        eq += L->dlq[q] * et;
      }
      A(1, op, t) = pert;
      A(2, op, t) = poly;
      A(3, op, t) = e1;
      A(4, op, t) = pert + ep;
      A(5, op, t) = poly + eq;
    }
  L->block = o->block;
  if (L->block == 0) {
    // autotuned block width among 8, 16, 32, 64 (those not above the noise count)
    const lqcd_krylov_opts po = noise_solver_opts(L);
    std::vector<int> cand;
    for (int c : {8, 16, 32, 64})
      if (c <= o->nnoise) cand.push_back(c);
    if (cand.empty()) cand.push_back(o->nnoise);
    if (L->ce) {
      L->ce->stream = ctx->stream;
      LQCD_TRY(autotune_block(L->ce, links, kappa, L->dme, &po, cand.data(), (int)cand.size(), &L->block, nullptr));
    } else {
      LQCD_TRY(autotune_block(ctx, links, kappa, L->dm, &po, cand.data(), (int)cand.size(), &L->block, nullptr));
    }
  }
  return LQCD_OK;
}

// Step 4 for noises first .. first+count-1: per_noise_t[((mode * count + n) * 9 + op) * Lt + t]
lqcd_status loop_noises(lqcd_loop *L, const double *links, uint32_t first0, int count, std::vector<cd> &per_noise_t,
                        lqcd_noise_info *info) {
  lqcd_ctx *ctx = L->ctx;
  const lqcd_est_opts *o = &L->o;
  const double kappa = L->kappa;
  const double2 *U = (const double2 *)links;
  const int Lt = ctx->dims[3];
  const long long N = ctx->N;
  const int modes = L->modes;
  const double t0 = now_s();
  NvtxRange nv("noise phase");
  const lqcd_krylov_opts po = noise_solver_opts(L);
  const int bw = std::max(1, std::min(L->block, count));
  const long long bn = (long long)bw * N;
  double2 *eta, *x, *xp, *xq, *y, *w, *cdv;
  LQCD_TRY(ws_get(ctx, WS_NBLK, sizeof(double2) * (size_t)bn * 6, (void **)&eta));
  x = eta + bn;
  xp = x + bn;
  xq = xp + bn;
  y = xq + bn;
  w = y + bn;
  LQCD_TRY(ws_get(ctx, WS_EST0, sizeof(double2) * (size_t)bw * 9 * Lt, (void **)&cdv));
  per_noise_t.assign((size_t)LQCD_NMODES * count * 9 * Lt, cd(0.0, 0.0));
  long matvecs = 0;
  double worst = 0.0;
  int conv = 1;
  std::vector<double2> h;
  const bool need_p = modes & (LQCD_SUB_PERT | LQCD_SUB_DEFL_PERT);
  const bool need_q = modes & (LQCD_SUB_POLY | LQCD_SUB_DEFL_POLY);
  for (int off = 0; off < count; off += bw) {
    const int nb = std::min(bw, count - off);
    const long long len = (long long)nb * N;
    LQCD_TRY(noise_launch(ctx, o->seed, first0 + (uint32_t)off, nb, eta));
    lqcd_solve_info pi{};
    NvtxRange nvb("noise block: solve, subtractions, contractions");
    if (L->ce) {
      LQCD_TRY(eo_noise_solve(L, U, eta, x, y, nb, &pi));
    } else if (L->dm->hermitian) {
      // M' y = eta over the Hermitian space, x = gamma_5 y (y is free until the deflation vectors)
      const lqcd_status st = proj_core_entry(ctx, links, kappa, L->dm, eta, y, nb, &po, &pi);
      if (st != LQCD_OK && st != LQCD_ERR_NOT_CONVERGED) return st;
      LQCD_TRY(blas_g5(ctx, y, x, nb));
    } else {
      const lqcd_status st = proj_core_entry(ctx, links, kappa, L->dm, eta, x, nb, &po, &pi);
      if (st != LQCD_OK && st != LQCD_ERR_NOT_CONVERGED) return st;
    }
    if (!pi.converged) conv = 0;
    worst = std::max(worst, pi.true_resid);
    matvecs += pi.matvecs;
    if (need_p) LQCD_TRY(hop_series_dev(ctx, U, kappa, eta, xp, nb, o->K, nullptr));
    if (need_q) LQCD_TRY(poly_apply_dev(ctx, U, kappa, eta, xq, nb, o->npoly, L->a.data()));
    if (need_p) matvecs += (long)nb * (o->K - 1);
    if (need_q) matvecs += (long)nb * o->npoly;
    for (int mode = 0; mode < LQCD_NMODES; ++mode) {
      if (!(modes & (1 << mode))) continue;
      // w = x - tilde x
      LQCD_TRY(blas_copy(ctx, x, w, len));
      if (mode == 1 || mode == 4) LQCD_TRY(scaled_acc(ctx, xp, w, cd(-1.0, 0.0), len));
      if (mode == 2 || mode == 5) LQCD_TRY(scaled_acc(ctx, xq, w, cd(-1.0, 0.0), len));
      if (mode >= 3 && mode <= 5) {
        const cd *dv = (mode == 3) ? L->dl.data() : (mode == 4 ? L->dlp.data() : L->dlq.data());
        LQCD_TRY(deflate_dev(ctx, L->dh, eta, y, nb, dv));
        LQCD_TRY(scaled_acc(ctx, y, w, cd(-1.0, 0.0), len));
      }
      if (mode == 6 && L->es_found > 0) {
        LQCD_TRY(es_vector(L, eta, y, nb));
        LQCD_TRY(scaled_acc(ctx, y, w, cd(-1.0, 0.0), len));
      }
      LQCD_TRY(contract_launch(ctx, U, kappa, eta, w, nb, cdv));
      LQCD_TRY(download_v(ctx, cdv, h, (size_t)nb * 9 * Lt));
      for (int r = 0; r < nb; ++r)
        for (int q = 0; q < 9 * Lt; ++q)
          per_noise_t[(((size_t)mode * count + off + r) * 9 * Lt) + q] =
              cd(h[(size_t)r * 9 * Lt + q].x, h[(size_t)r * 9 * Lt + q].y);
    }
  }
  if (info) {
    info->matvecs = matvecs;
    info->seconds = now_s() - t0;
    info->max_true_resid = worst;
    info->converged = conv;
    info->block = bw;
  }
  return LQCD_OK;
}

lqcd_status loop_new(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_est_opts *o, lqcd_loop **out) {
  LQCD_TRY(check_est_opts(ctx, o));
  if (!std::isfinite(kappa)) return set_err(ctx, LQCD_ERR_NONFINITE, "loop setup: kappa is not finite");
  LQCD_TRY(check_finite(ctx, links, 72LL * ctx->V, "loop setup: gauge links"));
  lqcd_loop *L = new lqcd_loop();
  L->ctx = ctx;
  L->kappa = kappa;
  L->o = *o;
  L->modes = o->modes ? o->modes : LQCD_SUB_ALL;
  L->Kt = std::max(o->K, o->npoly + 1);
  *out = L;
  return LQCD_OK;
}

// Steps 1-3 from scratch: special solves (GMRES-DR on M, MINRES-DR on M' batched), then the rest
lqcd_status loop_setup(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_est_opts *o, lqcd_loop **out) {
  *out = nullptr;
  const double t0 = now_s();
  lqcd_loop *L = nullptr;
  LQCD_TRY(loop_new(ctx, links, kappa, o, &L));
  std::unique_ptr<lqcd_loop> guard(L);
  const long long N = ctx->N;
  double2 *x0, *bs;
  LQCD_TRY(ws_get(ctx, WS_SPEC, sizeof(double2) * (size_t)N * 4, (void **)&x0));
  bs = x0 + 2 * N;
  LQCD_TRY(noise_launch(ctx, o->seed, 0xFFFFFFFEu, 1, bs));
  LQCD_TRY(noise_launch(ctx, o->seed, 0xFFFFFFFEu, 1, bs + N));
  lqcd_krylov_opts ko{o->m, o->k, o->tol_special, o->max_cycles, LQCD_SYS_M, LQCD_PREC_F64, 0.0, o->eig_tol};
  lqcd_solve_info si{};
  lqcd_status st;
  NvtxRange nv("loop setup: special right-hand side solves");
  const int sflags = o->system == LQCD_SYS_MG5 ? LQCD_APPLY_G5R : LQCD_APPLY_M;
  if (o->prec_degree > 0) {
    // polynomial preconditioner of the noise solves: the Min-Res polynomial of the solver's operator
    // (M, or M' on the Hermitian path, with real coefficients there) on the polynomial noise
    std::vector<cd> ap;
    LQCD_TRY(poly_coeffs_dev(ctx, (const double2 *)links, kappa, o->seed, o->prec_degree, ap, sflags));
    L->matvecs += o->prec_degree + 1;
    L->prec_a.resize(2 * ap.size());
    for (size_t j = 0; j < ap.size(); ++j) {
      L->prec_a[2 * j] = ap[j].real();
      L->prec_a[2 * j + 1] = o->system == LQCD_SYS_MG5 ? 0.0 : ap[j].imag();
    }
  }
  lqcd_krylov_opts kp = ko;
  if (!L->prec_a.empty()) {
    kp.poly_degree = o->prec_degree;
    kp.poly_coeffs = L->prec_a.data();
  }
  if (o->evenodd) {
    // even/odd: the noise solves' space from the reduced system (GMRES-DR on hat M, or MINRES-DR on
    // hat M gamma_5 on the Hermitian path) for the reduced special right-hand side; the HFES
    // eigenpairs from MINRES-DR on the full M'
    if (lqcd_ctx_create_evenodd(&L->ce, ctx->dims, ctx->recon, ctx->stream) != LQCD_OK)
      return set_err(ctx, LQCD_ERR_CUDA, "loop setup: reduced context creation failed");
    L->ce->graphs = ctx->graphs;
    L->ce->defl_engine = ctx->defl_engine;
    const long long Ne = L->ce->N;
    double2 *be;
    LQCD_TRY(ws_get(L->ce, WS_SPEC, sizeof(double2) * (size_t)Ne * 2, (void **)&be));
    LQCD_TRY(eo_rhs_launch(L->ce, (const double2 *)links, kappa, bs, be, 1));
    lqcd_solve_info se{};
    const lqcd_status ste = o->system == LQCD_SYS_MG5
                                ? lqcd_minresdr_solve(L->ce, links, kappa, (const double *)be, (double *)(be + Ne), 1, &ko, &se, &L->dme)
                                : lqcd_gmresdr_solve(L->ce, links, kappa, (const double *)be, (double *)(be + Ne), 1, &ko, &se, &L->dme);
    if (ste != LQCD_OK && ste != LQCD_ERR_NOT_CONVERGED) return set_err(ctx, ste, "loop setup (even/odd): %s", L->ce->err.c_str());
    if (!L->dme) return set_err(ctx, LQCD_ERR_NOT_CONVERGED, "loop setup: no reduced deflation space");
    L->matvecs += se.matvecs;
    st = lqcd_minresdr_solve(ctx, links, kappa, (const double *)bs, (double *)x0, 1, &ko, &si, &L->dh);
    L->dm = L->dh;
    L->own_h = true;
  } else if (o->system == LQCD_SYS_MG5) {
    // Hermitian path: MINRES-DR on M' (or on M' p(M')) alone gives both the eigenpairs and the
    // noise solves' space; with the preconditioner the eigenvalues of M' are the Rayleigh quotients
    st = lqcd_minresdr_solve(ctx, links, kappa, (const double *)bs, (double *)x0, 1, &kp, &si, &L->dh);
    L->dm = L->dh;
    L->own_h = true;
    if (L->dh && !L->prec_a.empty()) LQCD_TRY(defl_rayleigh(ctx, L->dh, links, kappa, LQCD_APPLY_G5R));
  } else if (!L->prec_a.empty()) {
    lqcd_solve_info s2{};
    st = lqcd_gmresdr_solve(ctx, links, kappa, (const double *)bs, (double *)x0, 1, &kp, &si, &L->dm);
    L->own_m = true;
    if (st == LQCD_OK || st == LQCD_ERR_NOT_CONVERGED) {
      const lqcd_status st2 = lqcd_minresdr_solve(ctx, links, kappa, (const double *)bs, (double *)(x0 + N), 1, &ko, &s2,
                                                  &L->dh);
      L->own_h = true;
      si.matvecs += s2.matvecs;
      if (st2 != LQCD_OK && st2 != LQCD_ERR_NOT_CONVERGED) return st2;
    }
  } else {
    st = special_solves(ctx, links, kappa, bs, x0, &ko, &si, &L->dm, &L->dh);
    L->own_m = L->own_h = true;
  }
  (void)sflags;
  if (st != LQCD_OK && st != LQCD_ERR_NOT_CONVERGED) return st;
  if (!L->dm || !L->dh) return set_err(ctx, LQCD_ERR_NOT_CONVERGED, "loop setup: no deflation space");
  L->matvecs += si.matvecs;
  LQCD_TRY(loop_finish_setup(L, (const double2 *)links, links, nullptr));
  L->seconds = now_s() - t0;
  *out = guard.release();
  return LQCD_OK;
}

}  // namespace

extern "C" {

lqcd_status lqcd_loop_setup(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_est_opts *opts,
                            lqcd_loop **out) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_full(ctx, "loop_setup"));
  if (!links || !opts || !out) return set_err(ctx, LQCD_ERR_INVALID_ARG, "loop_setup: NULL argument");
  return loop_setup(ctx, links, kappa, opts, out);
}

lqcd_status lqcd_loop_setup_from(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_est_opts *opts,
                                 const lqcd_defl *proj, const lqcd_defl *eig, const double *a, lqcd_loop **out) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_full(ctx, "loop_setup_from"));
  if (!links || !opts || !proj || !eig || !out) return set_err(ctx, LQCD_ERR_INVALID_ARG, "loop_setup_from: NULL argument");
  *out = nullptr;
  if (!proj->V || !proj->Hbar_dev || proj->N != ctx->N)
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "loop_setup_from: proj must be a Krylov space of this lattice (solver-made or lqcd_defl_import_space)");
  if (!eig->E || eig->N != ctx->N) return set_err(ctx, LQCD_ERR_INVALID_ARG, "loop_setup_from: eig has no eigenvectors of this lattice");
  const double t0 = now_s();
  lqcd_loop *L = nullptr;
  LQCD_TRY(loop_new(ctx, links, kappa, opts, &L));
  std::unique_ptr<lqcd_loop> guard(L);
  L->dm = const_cast<lqcd_defl *>(proj);
  L->dh = const_cast<lqcd_defl *>(eig);
  LQCD_TRY(loop_finish_setup(L, (const double2 *)links, links, a));
  L->seconds = now_s() - t0;
  *out = guard.release();
  return LQCD_OK;
}

lqcd_status lqcd_loop_noises(lqcd_loop *L, const double *links, uint32_t first, int count, double *per_noise_t,
                             lqcd_noise_info *info) {
  if (!L || !L->ctx) return LQCD_ERR_INVALID_ARG;
  if (!links || !per_noise_t || count < 1) return set_err(L->ctx, LQCD_ERR_INVALID_ARG, "loop_noises: bad arguments");
  if ((uint64_t)first + (uint64_t)count > 0xFFFFFFFEull)
    return set_err(L->ctx, LQCD_ERR_INVALID_ARG, "loop_noises: noise indices reach the reserved 2^32-2 / 2^32-1");
  std::vector<cd> pn;
  lqcd_noise_info ni{};
  LQCD_TRY(loop_noises(L, links, first, count, pn, &ni));
  memcpy(per_noise_t, pn.data(), sizeof(cd) * pn.size());
  if (info) *info = ni;
  return ni.converged ? LQCD_OK
                      : set_err(L->ctx, LQCD_ERR_NOT_CONVERGED, "loop_noises: a noise solve did not converge (rel %.3e)",
                                ni.max_true_resid);
}

lqcd_status lqcd_loop_noises_host(lqcd_loop *L, const double *links_host, uint32_t first, int count,
                                  double *per_noise_t, lqcd_noise_info *info) {
  if (!L || !L->ctx) return LQCD_ERR_INVALID_ARG;
  if (!links_host) return set_err(L->ctx, LQCD_ERR_INVALID_ARG, "loop_noises_host: bad arguments");
  lqcd_ctx *ctx = L->ctx;
  const size_t bytes = sizeof(double2) * (size_t)4 * ctx->V * 9;
  double2 *Ud;
  LQCD_TRY(ws_get(ctx, WS_HOST_LINKS, bytes, (void **)&Ud));
  LQCD_CUDA(ctx, cudaMemcpyAsync(Ud, links_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
  return lqcd_loop_noises(L, (const double *)Ud, first, count, per_noise_t, info);
}

lqcd_status lqcd_loop_set_noise_opts(lqcd_loop *L, int prec, double inner_tol, int block) {
  if (!L || !L->ctx) return LQCD_ERR_INVALID_ARG;
  if (prec < LQCD_PREC_F64 || prec > LQCD_PREC_BF16 || !(inner_tol >= 0.0 && inner_tol < 1.0) || block < 0)
    return set_err(L->ctx, LQCD_ERR_INVALID_ARG, "loop_set_noise_opts: bad arguments");
  if (L->ce && prec != LQCD_PREC_F64)
    return set_err(L->ctx, LQCD_ERR_INVALID_ARG, "loop_set_noise_opts: even/odd noise solves are plain FP64");
  L->o.prec = prec;
  L->o.inner_tol = inner_tol;
  if (block > 0) L->block = block;
  return LQCD_OK;
}

lqcd_status lqcd_loop_set_inner_restart(lqcd_loop *L, int m_inner) {
  if (!L || !L->ctx) return LQCD_ERR_INVALID_ARG;
  if (m_inner < 0 || m_inner > 1024) return set_err(L->ctx, LQCD_ERR_INVALID_ARG, "loop_set_inner_restart: m_inner must be in 0..1024");
  L->o.m_inner = m_inner;
  return LQCD_OK;
}

lqcd_status lqcd_loop_get(const lqcd_loop *L, lqcd_loop_info *out) {
  if (!L || !out) return LQCD_ERR_INVALID_ARG;
  const size_t Lt = L->ctx->dims[3];
  if (out->addback) memcpy(out->addback, L->add.data(), sizeof(cd) * L->add.size());
  if (out->lam) memcpy(out->lam, L->lam.data(), sizeof(cd) * L->lam.size());
  if (out->poly_a) memcpy(out->poly_a, L->a.data(), sizeof(cd) * L->a.size());
  if (out->xi_pert) memcpy(out->xi_pert, L->xi_p.data(), sizeof(cd) * L->xi_p.size());
  if (out->xi_poly) memcpy(out->xi_poly, L->xi_q.data(), sizeof(cd) * L->xi_q.size());
  (void)Lt;
  out->Q = L->Q;
  out->block = L->block;
  out->matvecs_setup = L->matvecs;
  out->seconds_setup = L->seconds;
  out->eig_resid_max = L->eres;
  return LQCD_OK;
}

lqcd_status lqcd_loop_destroy(lqcd_loop *L) {
  if (!L) return LQCD_ERR_INVALID_ARG;
  if (L->ctx) cudaStreamSynchronize(L->ctx->stream);
  delete L;
  return LQCD_OK;
}

lqcd_status lqcd_loop_estimate(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_est_opts *o,
                               lqcd_estimate *out) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_full(ctx, "loop_estimate"));
  if (!links || !o || !out) return set_err(ctx, LQCD_ERR_INVALID_ARG, "loop_estimate: NULL argument");
  lqcd_loop *Lp = nullptr;
  LQCD_TRY(loop_setup(ctx, links, kappa, o, &Lp));
  std::unique_ptr<lqcd_loop> guard(Lp);
  const int Lt = ctx->dims[3];
  const int nn = o->nnoise;
  std::vector<cd> per_noise_t;
  lqcd_noise_info ni{};
  LQCD_TRY(loop_noises(Lp, links, 0u, nn, per_noise_t, &ni));
  // 5. summary
  const std::vector<cd> &add = Lp->add;
  auto A = [&](int mode, int op, int t) -> const cd & { return add[((size_t)mode * 9 + op) * Lt + t]; };
  for (int mode = 0; mode < LQCD_NMODES; ++mode) {
    for (int op = 0; op < 9; ++op) {
      cd addtot = 0.0;
      for (int t = 0; t < Lt; ++t) addtot += A(mode, op, t);
      std::vector<cd> tot(nn);
      for (int n = 0; n < nn; ++n) {
        cd s = 0.0;
        for (int t = 0; t < Lt; ++t) s += per_noise_t[(((size_t)mode * nn + n) * 9 + op) * Lt + t];
        tot[n] = s + addtot;
        if (out->per_noise) {
          out->per_noise[((((size_t)mode * nn + n) * 9 + op) * 2)] = tot[n].real();
          out->per_noise[((((size_t)mode * nn + n) * 9 + op) * 2) + 1] = tot[n].imag();
        }
      }
      cd mean = 0.0;
      for (int n = 0; n < nn; ++n) mean += tot[n];
      mean /= (double)nn;
      double ps = 0.0, pm = 0.0;
      for (int n = 0; n < nn; ++n) pm += (op == 0) ? tot[n].real() : tot[n].imag();
      pm /= nn;
      for (int n = 0; n < nn; ++n) {
        const double v = ((op == 0) ? tot[n].real() : tot[n].imag()) - pm;
        ps += v * v;
      }
      const double err = nn > 1 ? std::sqrt(ps / (nn - 1)) / std::sqrt((double)nn) : NAN;
      if (out->mean) {
        out->mean[((size_t)mode * 9 + op) * 2] = mean.real();
        out->mean[((size_t)mode * 9 + op) * 2 + 1] = mean.imag();
      }
      if (out->stderr_) out->stderr_[(size_t)mode * 9 + op] = err;
      for (int t = 0; t < Lt; ++t) {
        cd pt = 0.0;
        for (int n = 0; n < nn; ++n) pt += per_noise_t[(((size_t)mode * nn + n) * 9 + op) * Lt + t];
        pt /= (double)nn;
        if (out->per_t) {
          out->per_t[(((size_t)mode * 9 + op) * Lt + t) * 2] = pt.real();
          out->per_t[(((size_t)mode * 9 + op) * Lt + t) * 2 + 1] = pt.imag();
        }
        if (out->addback) {
          out->addback[(((size_t)mode * 9 + op) * Lt + t) * 2] = A(mode, op, t).real();
          out->addback[(((size_t)mode * 9 + op) * Lt + t) * 2 + 1] = A(mode, op, t).imag();
        }
      }
    }
  }
  if (out->lam) memcpy(out->lam, Lp->lam.data(), sizeof(cd) * Lp->Q);
  if (out->poly_a) memcpy(out->poly_a, Lp->a.data(), sizeof(cd) * Lp->a.size());
  out->matvecs_setup = Lp->matvecs;
  out->matvecs_noise = ni.matvecs;
  out->seconds_setup = Lp->seconds;
  out->seconds_noise = ni.seconds;
  out->max_true_resid = ni.max_true_resid;
  out->converged = ni.converged;
  out->block = ni.block;
  return ni.converged ? LQCD_OK
                      : set_err(ctx, LQCD_ERR_NOT_CONVERGED, "loop_estimate: a noise solve did not converge (rel %.3e)",
                                ni.max_true_resid);
}

}  // extern "C"

// ---- allocation-free contraction -------------------------------------------------------------
// Some callers cannot allocate device memory at all: plug-ins whose host application owns every
// device byte through its own allocator, code under a strict memory budget, or latency-critical
// paths where a cudaMalloc (which may synchronise the device) is not acceptable.
// lqcd_contract_noalloc serves them: the same
// contraction as lqcd_contract, but its per-chunk partial sums live in a fixed device array that
// is part of the library image (loaded with the module, held by every device that loads the
// library until the process exits), the output goes to a caller-provided device buffer, and no
// context, workspace or staging buffer is involved.
namespace {

constexpr int NOALLOC_SCRATCH_ENTRIES = 1 << 16;  // double2 entries: 1 MiB
static __device__ __align__(256) double2 g_noalloc_scratch[NOALLOC_SCRATCH_ENTRIES];

constexpr int NOALLOC_MAX_DEVICES = 64;
struct NoallocSlot {
  double2 *ptr;            // device address of g_noalloc_scratch in the context below
  unsigned long long ctx;  // id of the CUDA context it was looked up in (0: none yet)
  int sms;
};
NoallocSlot g_noalloc[NOALLOC_MAX_DEVICES] = {};
std::mutex g_noalloc_mutex;

// Id of the calling thread's current CUDA context (0 when none is current yet), through the driver
// entry points the runtime hands out (no link against the driver library).  Context ids are never
// reused within a process, so a replaced context (cudaDeviceReset, which also reloads this
// library's device module and moves the scratch array) never matches a stale cache entry.
typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);
lqcd_status current_ctx_id(unsigned long long *id) {
  static PfnCtxGetCurrent get_cur = nullptr;
  static PfnCtxGetId get_id = nullptr;
  if (!get_cur || !get_id) {
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void **)&get_cur, 12000, cudaEnableDefault, &q1) !=
            cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", (void **)&get_id, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !get_cur || !get_id) {
      cudaGetLastError();
      get_cur = nullptr;
      get_id = nullptr;
      return LQCD_ERR_CUDA;
    }
  }
  CUcontext c = nullptr;
  if (get_cur(&c) != CUDA_SUCCESS) return LQCD_ERR_CUDA;
  *id = 0;
  if (c && get_id(c, id) != CUDA_SUCCESS) return LQCD_ERR_CUDA;
  return LQCD_OK;
}

// Device address of the scratch array in the current context of device dev, looked up once per
// device and context.  A host reference to g_noalloc_scratch names a host-side stand-in, not
// device memory, so the address must come from cudaGetSymbolAddress with the device current.
lqcd_status noalloc_setup(int dev, double2 **ptr, int *sms) {
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return LQCD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  unsigned long long id = 0;
  LQCD_TRY(current_ctx_id(&id));
  NoallocSlot &slot = g_noalloc[dev];
  if (!slot.ptr || id == 0 || slot.ctx != id) {
    void *p = nullptr;  // the lookup also makes the device's primary context current if none is
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return LQCD_ERR_CUDA;
    }
    LQCD_TRY(current_ctx_id(&id));
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return LQCD_ERR_CUDA;
    }
    slot.ptr = (double2 *)p;
    slot.ctx = id;
    slot.sms = n;
  }
  *ptr = slot.ptr;
  *sms = slot.sms;
  return LQCD_OK;
}

}  // namespace

extern "C" lqcd_status lqcd_contract_noalloc(const int dims[4], const double *links, double kappa, const double *eta,
                                             const double *w, int nrhs, double *out, void *stream) {
  if (!dims || !links || !eta || !w || !out || nrhs < 1 || nrhs > 65535) return LQCD_ERR_INVALID_ARG;
  long long V = 1;
  for (int i = 0; i < 4; ++i) {
    if (dims[i] < 2 || dims[i] > 1024) return LQCD_ERR_INVALID_ARG;
    V *= dims[i];
  }
  // the context limit: site indices (and 12 V-strided offsets per right-hand side) stay in range
  if (V > (1LL << 28)) return LQCD_ERR_INVALID_ARG;
  const int Lt = dims[3], Vs = dims[0] * dims[1] * dims[2];
  // every (rhs, timeslice, chunk) writes its nine partial sums: at least one chunk must fit
  const long long per_chunk = (long long)nrhs * Lt * 9;
  if (per_chunk > NOALLOC_SCRATCH_ENTRIES) return LQCD_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return LQCD_ERR_CUDA;
  }
  double2 *scratch = nullptr;
  int sms = 0;
  LQCD_TRY(noalloc_setup(dev, &scratch, &sms));
  const long long fit = NOALLOC_SCRATCH_ENTRIES / per_chunk;
  const int want = std::max(1, std::min((Vs + CBT - 1) / CBT, std::max(1, (4 * sms) / std::max(1, nrhs * Lt))));
  const int nchunk = (int)std::max<long long>(1, std::min<long long>(want, fit));
  cudaStream_t st = (cudaStream_t)stream;
  // the kernel writes every partial entry it later reads, so the array needs no clearing
  contract_kernel<<<dim3(nchunk * Lt, nrhs), CBT, 0, st>>>((const double2 *)links, kappa, (const double2 *)eta,
                                                           (const double2 *)w, dims[0], dims[1], dims[2], dims[3],
                                                           nchunk, scratch);
  if (cudaGetLastError() != cudaSuccess) return LQCD_ERR_CUDA;
  const int tot = nrhs * 9 * Lt;
  contract_final<<<ceil_div(tot, 128), 128, 0, st>>>(scratch, nchunk, Lt, nrhs, (double2 *)out);
  if (cudaGetLastError() != cudaSuccess) return LQCD_ERR_CUDA;
  return LQCD_OK;
}
