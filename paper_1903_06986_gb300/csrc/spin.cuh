// Device-side spin and colour algebra of the Wilson hopping term, shared by the operator and the
// point-split contraction kernels.  Dirac-basis projections (h = upper pair after projection,
// rows 2, 3 rebuilt from it):
//   mu = x:  1 - g: h = (p0 + i p3, p1 + i p2), lower = (-i h1, -i h0)
//            1 + g: h = (p0 - i p3, p1 - i p2), lower = ( i h1,  i h0)
//   mu = y:  1 - g: h = (p0 + p3,   p1 - p2),   lower = (-h1,  h0)
//            1 + g: h = (p0 - p3,   p1 + p2),   lower = ( h1, -h0)
//   mu = z:  1 - g: h = (p0 + i p2, p1 - i p3), lower = (-i h0,  i h1)
//            1 + g: h = (p0 - i p2, p1 + i p3), lower = ( i h0, -i h1)
//   mu = t:  1 - g = diag(0,0,2,2);  1 + g = diag(2,2,0,0)
#pragma once

#include "common.cuh"

namespace spin {

template <typename R> struct Cx {
  R x, y;
};
template <typename R> __device__ __forceinline__ Cx<R> mk(R a, R b) { Cx<R> c; c.x = a; c.y = b; return c; }
template <typename R> __device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) { return mk<R>(a.x + b.x, a.y + b.y); }
template <typename R> __device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) { return mk<R>(a.x - b.x, a.y - b.y); }
template <typename R> __device__ __forceinline__ Cx<R> ti(Cx<R> a) { return mk<R>(-a.y, a.x); }    // i a
template <typename R> __device__ __forceinline__ Cx<R> tmi(Cx<R> a) { return mk<R>(a.y, -a.x); }   // -i a
template <typename R> __device__ __forceinline__ Cx<R> neg(Cx<R> a) { return mk<R>(-a.x, -a.y); }

template <typename R> __device__ __forceinline__ Cx<R> load_c(const double2 *p) {
  double2 v = __ldg(p);
  return mk<R>((R)v.x, (R)v.y);
}
template <typename R> __device__ __forceinline__ Cx<R> load_c(const float2 *p) {
  float2 v = __ldg(p);
  return mk<R>((R)v.x, (R)v.y);
}
__device__ __forceinline__ void store_c(double2 *p, Cx<double> v) { *p = make_double2(v.x, v.y); }
__device__ __forceinline__ void store_c(double2 *p, Cx<float> v) { *p = make_double2((double)v.x, (double)v.y); }
__device__ __forceinline__ void store_c(float2 *p, Cx<float> v) { *p = make_float2(v.x, v.y); }

// u * h for a 3x3 colour matrix u (row-major) and colour vector h
template <typename R> __device__ __forceinline__ void mul_u(const Cx<R> u[9], const Cx<R> h[3], Cx<R> o[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R re = u[3 * a].x * h[0].x - u[3 * a].y * h[0].y;
    R im = u[3 * a].x * h[0].y + u[3 * a].y * h[0].x;
#pragma unroll
    for (int b = 1; b < 3; ++b) {
      re = fma(u[3 * a + b].x, h[b].x, re);
      re = fma(-u[3 * a + b].y, h[b].y, re);
      im = fma(u[3 * a + b].x, h[b].y, im);
      im = fma(u[3 * a + b].y, h[b].x, im);
    }
    o[a] = mk<R>(re, im);
  }
}

// u^dagger * h
template <typename R> __device__ __forceinline__ void mul_udag(const Cx<R> u[9], const Cx<R> h[3], Cx<R> o[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R re = u[a].x * h[0].x + u[a].y * h[0].y;
    R im = u[a].x * h[0].y - u[a].y * h[0].x;
#pragma unroll
    for (int b = 1; b < 3; ++b) {
      re = fma(u[3 * b + a].x, h[b].x, re);
      re = fma(u[3 * b + a].y, h[b].y, re);
      im = fma(u[3 * b + a].x, h[b].y, im);
      im = fma(-u[3 * b + a].y, h[b].x, im);
    }
    o[a] = mk<R>(re, im);
  }
}

template <typename R, bool G5IN, typename S>
__device__ __forceinline__ void load_spinor(const S *p, Cx<R> s[4][3]) {
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c) s[sp][c] = load_c<R>(p + 3 * sp + c);
  if (G5IN) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Cx<R> a0 = s[0][c], a1 = s[1][c];
      s[0][c] = neg(s[2][c]);
      s[1][c] = neg(s[3][c]);
      s[2][c] = neg(a0);
      s[3][c] = neg(a1);
    }
  }
}

// Forward term of direction MU: acc += (1 - g_MU) U_MU(x) psi(x + MU)
template <typename R, int MU>
__device__ __forceinline__ void term_fwd(const Cx<R> p[4][3], const Cx<R> u[9], Cx<R> acc[4][3]) {
  Cx<R> h0[3], h1[3], o0[3], o1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (MU == 0) { h0[c] = p[0][c] + ti(p[3][c]); h1[c] = p[1][c] + ti(p[2][c]); }
    if (MU == 1) { h0[c] = p[0][c] + p[3][c];     h1[c] = p[1][c] - p[2][c]; }
    if (MU == 2) { h0[c] = p[0][c] + ti(p[2][c]); h1[c] = p[1][c] - ti(p[3][c]); }
    if (MU == 3) { h0[c] = p[2][c] + p[2][c];     h1[c] = p[3][c] + p[3][c]; }
  }
  mul_u<R>(u, h0, o0);
  mul_u<R>(u, h1, o1);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (MU == 3) {
      acc[2][c] = acc[2][c] + o0[c];
      acc[3][c] = acc[3][c] + o1[c];
    } else {
      acc[0][c] = acc[0][c] + o0[c];
      acc[1][c] = acc[1][c] + o1[c];
      if (MU == 0) { acc[2][c] = acc[2][c] + tmi(o1[c]); acc[3][c] = acc[3][c] + tmi(o0[c]); }
      if (MU == 1) { acc[2][c] = acc[2][c] - o1[c];      acc[3][c] = acc[3][c] + o0[c]; }
      if (MU == 2) { acc[2][c] = acc[2][c] + tmi(o0[c]); acc[3][c] = acc[3][c] + ti(o1[c]); }
    }
  }
}

// Backward term of direction MU: acc += (1 + g_MU) U_MU(x - MU)^dag psi(x - MU)
template <typename R, int MU>
__device__ __forceinline__ void term_bwd(const Cx<R> p[4][3], const Cx<R> u[9], Cx<R> acc[4][3]) {
  Cx<R> h0[3], h1[3], o0[3], o1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (MU == 0) { h0[c] = p[0][c] - ti(p[3][c]); h1[c] = p[1][c] - ti(p[2][c]); }
    if (MU == 1) { h0[c] = p[0][c] - p[3][c];     h1[c] = p[1][c] + p[2][c]; }
    if (MU == 2) { h0[c] = p[0][c] - ti(p[2][c]); h1[c] = p[1][c] + ti(p[3][c]); }
    if (MU == 3) { h0[c] = p[0][c] + p[0][c];     h1[c] = p[1][c] + p[1][c]; }
  }
  mul_udag<R>(u, h0, o0);
  mul_udag<R>(u, h1, o1);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[0][c] = acc[0][c] + o0[c];
    acc[1][c] = acc[1][c] + o1[c];
    if (MU == 0) { acc[2][c] = acc[2][c] + ti(o1[c]); acc[3][c] = acc[3][c] + ti(o0[c]); }
    if (MU == 1) { acc[2][c] = acc[2][c] + o1[c];     acc[3][c] = acc[3][c] - o0[c]; }
    if (MU == 2) { acc[2][c] = acc[2][c] + ti(o0[c]); acc[3][c] = acc[3][c] + tmi(o1[c]); }
  }
}

template <typename R, typename S>
__device__ __forceinline__ void load_link(const S *U, long long idx, Cx<R> u[9]) {
#pragma unroll
  for (int i = 0; i < 9; ++i) u[i] = load_c<R>(U + idx * 9 + i);
}

}  // namespace spin
