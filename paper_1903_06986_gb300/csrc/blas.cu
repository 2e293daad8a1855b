// Batched complex level-1/level-2 kernels for the Krylov solvers, and the Z(4) noise kernel.
//
// A "block" of nrhs vectors of length n is stored vector after vector; a multi-vector (a Krylov
// basis) stores basis vector i of right-hand side r at V + i * vstride + r * vrs.  The kernels are
// templates on the storage type: double2 (the FP64 path) or float2 / __half2 / __nv_bfloat162 (the
// inner solver of the mixed-precision path, FP32 arithmetic; two-type forms combine a reduced-
// precision basis with FP32 vectors).  Each thread accumulates its terms in the arithmetic type and
// the cross-thread reduction is FP64.  Every reduction is two-stage with a fixed order (per-block
// partial sums, then one block per result), so results are reproducible run to run.  FP16 / BF16
// vectors hold store_sigma * value; the host passes the factors that undo it.
#include <algorithm>
#include <type_traits>

#include <cstring>

#include "common.cuh"

namespace {

constexpr int BT = 256;      // threads per block
constexpr int GROUP = 8;     // basis vectors reduced together in multidot (at most BT / 32)
static_assert(GROUP <= BT / 32, "multidot: one warp per vector of a group in the final sums");

// arithmetic type of a storage type
template <typename S> struct ArithT { using T = float2; };
template <> struct ArithT<double2> { using T = double2; };
template <typename S> using Ar = typename ArithT<S>::T;

__device__ __forceinline__ double2 ldc(double2 v) { return v; }
__device__ __forceinline__ float2 ldc(float2 v) { return v; }
__device__ __forceinline__ float2 ldc(__half2 v) { return __half22float2(v); }
__device__ __forceinline__ float2 ldc(__nv_bfloat162 v) { return __bfloat1622float2(v); }
template <typename S> __device__ __forceinline__ S stc(Ar<S> v);
template <> __device__ __forceinline__ double2 stc<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 stc<float2>(float2 v) { return v; }
template <> __device__ __forceinline__ __half2 stc<__half2>(float2 v) { return __float22half2_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat162 stc<__nv_bfloat162>(float2 v) { return __float22bfloat162_rn(v); }

template <typename C> __device__ __forceinline__ C cz();
template <> __device__ __forceinline__ double2 cz<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 cz<float2>() { return make_float2(0.f, 0.f); }
template <typename C> __device__ __forceinline__ C from_d2(double2 v);
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
// acc += a * b and acc += conj(a) * b for double2 / float2
template <typename C> __device__ __forceinline__ void gfma(C &acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
template <typename C> __device__ __forceinline__ void gfma_conj(C &acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

__device__ __forceinline__ double2 warp_sum2(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// conj(V_j[e]) w[e] summed into acc[j] over the elements e0 + t, e0 + t + BT, ... < e1 of this thread
// (t = threadIdx.x), for the first g of the G vectors (all of them when FULL)
template <bool FULL, int G, typename SV, typename SW, typename C>
__device__ __forceinline__ void dot_range(const SV *const *vp, const SW *__restrict__ wr, long long e0, long long e1,
                                          int g, C *acc) {
  for (long long e = e0 + threadIdx.x; e < e1; e += BT) {
    const C wv = ldc(wr[e]);
#pragma unroll
    for (int j = 0; j < G; ++j)
      if (FULL || j < g) gfma_conj(acc[j], ldc(vp[j][e]), wv);
  }
}
// the same with one 16-byte load per vector and thread (KV = 16 / sizeof(SV) elements); e0 and the
// vectors' offsets are multiples of KV elements, the remainder of the range goes element-wise
template <bool FULL, int G, typename SV, typename SW, typename C>
__device__ __forceinline__ void dot_range_vec(const SV *const *vp, const SW *__restrict__ wr, long long e0,
                                              long long e1, int g, C *acc) {
  constexpr int KV = 16 / sizeof(SV);
  const long long ev = e0 + (e1 - e0) / KV * KV;
  for (long long e = e0 + (long long)threadIdx.x * KV; e < ev; e += (long long)BT * KV) {
    // all G + 1 loads of this step issued before any use, so that they are in flight together
    uint4 vraw[G];
    const uint4 wraw = __ldg(reinterpret_cast<const uint4 *>(wr + e));
#pragma unroll
    for (int j = 0; j < G; ++j)
      if (FULL || j < g) vraw[j] = __ldg(reinterpret_cast<const uint4 *>(vp[j] + e));
    SW wv[KV];
    memcpy(wv, &wraw, 16);
#pragma unroll
    for (int j = 0; j < G; ++j) {
      if (FULL || j < g) {
        SV vv[KV];
        memcpy(vv, &vraw[j], 16);
#pragma unroll
        for (int q = 0; q < KV; ++q) gfma_conj(acc[j], ldc(vv[q]), ldc(wv[q]));
      }
    }
  }
  dot_range<FULL, G>(vp, wr, ev, e1, g, acc);
}

// Single-launch batched inner products.  Block b (a 1-D grid) sums conj(V_i^r) w^r over element
// chunk c for the G basis vectors of group g (G = GROUP, or 2 for the two-vector Lanczos steps) and
// writes partial[(i * nrhs + r) * nchunk + c]: with a basis shared by all right-hand sides b = g + ngroup (r + nrhs c), so that the groups and
// right-hand sides of one chunk are neighbours in launch order and the chunk of every basis vector
// and of every w^r is read from DRAM once and then from L2; with a basis per right-hand side
// b = c + nchunk (g + ngroup r), consecutive blocks streaming consecutive chunks.  The last of the
// nchunk blocks of (r, g) to finish (a counter per (r, g), reset by that block) adds the nchunk
// partials of every vector of the group in a fixed order (one warp per vector) and writes
// h[i * nrhs + r]: the result does not depend on block scheduling, and the final sums of the groups
// run in parallel.
template <typename SV, typename SW, bool VEC, int G>
__global__ void __launch_bounds__(BT) multidot_kernel(const SV *__restrict__ V, long long vstride, long long vrs,
                                                      int nvec, const SW *__restrict__ w, long long n, int nrhs,
                                                      int nchunk, double fac, double2 *__restrict__ partial,
                                                      unsigned *__restrict__ counters, double2 *__restrict__ h) {
  using C = Ar<SW>;
  static_assert(std::is_same<C, Ar<SV>>::value, "multidot: storage types of different arithmetic");
  const int ngroup = (nvec + G - 1) / G;
  int g0, r, c;
  if (vrs == 0) {
    // shared basis: the groups and right-hand sides of one chunk are neighbours in launch order
    g0 = blockIdx.x % ngroup;
    r = (blockIdx.x / ngroup) % nrhs;
    c = blockIdx.x / (ngroup * nrhs);
  } else {
    // a basis per right-hand side: consecutive blocks stream consecutive chunks of one vector group
    c = blockIdx.x % nchunk;
    g0 = (blockIdx.x / nchunk) % ngroup;
    r = blockIdx.x / (nchunk * ngroup);
  }
  const int i0 = g0 * G;
  constexpr long long KV = VEC ? 16 / sizeof(SV) : 1;
  const long long chunk = ((n + nchunk - 1) / nchunk + KV - 1) / KV * KV;
  const long long e0 = min(n, c * chunk);
  const long long e1 = min(n, e0 + chunk);
  const SW *wr = w + r * n;
  const SV *vr = V + r * vrs;
  __shared__ double2 red[BT / 32][G];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = min(G, nvec - i0);
  const SV *vp[G];
#pragma unroll
  for (int j = 0; j < G; ++j) vp[j] = vr + (long long)(i0 + min(j, g - 1)) * vstride;
  C acc[G];
#pragma unroll
  for (int j = 0; j < G; ++j) acc[j] = cz<C>();
  if (VEC) {
    if (g == G)
      dot_range_vec<true, G>(vp, wr, e0, e1, g, acc);
    else
      dot_range_vec<false, G>(vp, wr, e0, e1, g, acc);
  } else {
    if (g == G)
      dot_range<true, G>(vp, wr, e0, e1, g, acc);
    else
      dot_range<false, G>(vp, wr, e0, e1, g, acc);
  }
#pragma unroll
  for (int j = 0; j < G; ++j) {
    double2 v = warp_sum2(to_d2(acc[j]));
    if (lane == 0) red[warp][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < g) {
    double2 sum = make_double2(0.0, 0.0);
    for (int q = 0; q < BT / 32; ++q) sum = cadd(sum, red[q][threadIdx.x]);
    partial[((long long)(i0 + threadIdx.x) * nrhs + r) * nchunk + c] = sum;
  }
  __threadfence();
  __syncthreads();
  unsigned *cnt = counters + (long long)r * ngroup + g0;
  if (threadIdx.x == 0) last = (atomicAdd(cnt, 1u) == (unsigned)(nchunk - 1));
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last chunk block of (r, group) finishes the group's vectors, one warp per vector: lanes
  // stride over the chunks, then a fixed shuffle tree (the order of the additions depends only on
  // nchunk)
  if (warp < g) {
    const int i = i0 + warp;
    const double2 *pp = partial + ((long long)i * nrhs + r) * nchunk;
    double2 sum = make_double2(0.0, 0.0);
    for (int q = lane; q < nchunk; q += 32) sum = cadd(sum, __ldcg(pp + q));
    sum = warp_sum2(sum);
    if (lane == 0) h[(long long)i * nrhs + r] = cscale(sum, fac);
  }
  if (threadIdx.x == 0) *cnt = 0u;
}

// Single-launch batched norms ||x^r||, same last-block scheme as multidot_kernel.
template <typename S>
__global__ void __launch_bounds__(BT) norm_kernel(const S *__restrict__ x, long long n, double fac,
                                                  double *__restrict__ partial, unsigned *__restrict__ counters,
                                                  double *__restrict__ out) {
  const int r = blockIdx.y;
  const int nb = gridDim.x;
  const long long chunk = (n + nb - 1) / nb;
  const long long e0 = blockIdx.x * chunk;
  const long long e1 = min(n, e0 + chunk);
  const S *xr = x + r * n;
  decltype(Ar<S>().x) a = 0;
  for (long long e = e0 + threadIdx.x; e < e1; e += BT) {
    const Ar<S> v = ldc(xr[e]);
    a = fma(v.x, v.x, a);
    a = fma(v.y, v.y, a);
  }
  double acc = (double)a;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[BT / 32];
  __shared__ bool last;
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int q = 0; q < BT / 32; ++q) sum += red[q];
    partial[(long long)r * nb + blockIdx.x] = sum;
    __threadfence();
    last = (atomicAdd(&counters[r], 1u) == (unsigned)(nb - 1));
  }
  __syncthreads();
  if (!last || threadIdx.x >= 32) return;
  __threadfence();
  // the first warp adds the nb partials: lanes stride over them, then a fixed shuffle tree
  double sum = 0.0;
  for (int q = threadIdx.x; q < nb; q += 32) sum += __ldcg(partial + (long long)r * nb + q);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (threadIdx.x == 0) {
    out[r] = sqrt(sum) * fac;
    counters[r] = 0u;
  }
}

// Inner products with a basis shared by all right-hand sides: block b = t + ntile (g + ngroup c)
// takes element chunk c of the GROUP vectors of group g against the RT right-hand sides of tile t,
// so every basis element a thread loads is used for RT right-hand sides (the tiles of one chunk and
// group are neighbours in launch order and share it through L2).  Partials and the per-(tile, group)
// last-block final sums as in multidot_kernel.
template <typename SV, typename SW, int RT>
__global__ void __launch_bounds__(BT) multidot_shared_kernel(const SV *__restrict__ V, long long vstride, int nvec,
                                                             const SW *__restrict__ w, long long n, int nrhs,
                                                             int nchunk, double fac, double2 *__restrict__ partial,
                                                             unsigned *__restrict__ counters,
                                                             double2 *__restrict__ h) {
  using C = Ar<SW>;
  const int ngroup = (nvec + GROUP - 1) / GROUP;
  const int ntile = (nrhs + RT - 1) / RT;
  const int t = blockIdx.x % ntile;
  const int g0 = (blockIdx.x / ntile) % ngroup;
  const int c = blockIdx.x / (ntile * ngroup);
  const int i0 = g0 * GROUP, r0 = t * RT;
  const int g = min(GROUP, nvec - i0), nr = min(RT, nrhs - r0);
  const long long chunk = (n + nchunk - 1) / nchunk;
  const long long e0 = min(n, c * chunk);
  const long long e1 = min(n, e0 + chunk);
  const SV *vp[GROUP];
#pragma unroll
  for (int j = 0; j < GROUP; ++j) vp[j] = V + (long long)(i0 + min(j, g - 1)) * vstride;
  const SW *wp[RT];
#pragma unroll
  for (int q = 0; q < RT; ++q) wp[q] = w + (long long)(r0 + min(q, nr - 1)) * n;
  C acc[GROUP][RT];
#pragma unroll
  for (int j = 0; j < GROUP; ++j)
#pragma unroll
    for (int q = 0; q < RT; ++q) acc[j][q] = cz<C>();
  for (long long e = e0 + threadIdx.x; e < e1; e += BT) {
    C vv[GROUP], wv[RT];
#pragma unroll
    for (int j = 0; j < GROUP; ++j) vv[j] = ldc(vp[j][e]);
#pragma unroll
    for (int q = 0; q < RT; ++q) wv[q] = ldc(wp[q][e]);
#pragma unroll
    for (int j = 0; j < GROUP; ++j)
#pragma unroll
      for (int q = 0; q < RT; ++q) gfma_conj(acc[j][q], vv[j], wv[q]);
  }
  __shared__ double2 red[BT / 32][GROUP * RT];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < GROUP; ++j)
#pragma unroll
    for (int q = 0; q < RT; ++q) {
      const double2 v = warp_sum2(to_d2(acc[j][q]));
      if (lane == 0) red[warp][j * RT + q] = v;
    }
  __syncthreads();
  for (int p = threadIdx.x; p < GROUP * RT; p += BT) {
    const int j = p / RT, q = p % RT;
    if (j < g && q < nr) {
      double2 sum = make_double2(0.0, 0.0);
      for (int k = 0; k < BT / 32; ++k) sum = cadd(sum, red[k][p]);
      partial[((long long)(i0 + j) * nrhs + r0 + q) * nchunk + c] = sum;
    }
  }
  __threadfence();
  __syncthreads();
  unsigned *cnt = counters + (long long)t * ngroup + g0;
  if (threadIdx.x == 0) last = (atomicAdd(cnt, 1u) == (unsigned)(nchunk - 1));
  __syncthreads();
  if (!last) return;
  __threadfence();
  // final sums of the tile's (vector, right-hand side) pairs, one warp per pair, in a fixed order
  for (int p = warp; p < GROUP * RT; p += BT / 32) {
    const int j = p / RT, q = p % RT;
    if (j >= g || q >= nr) continue;
    const double2 *pp = partial + ((long long)(i0 + j) * nrhs + r0 + q) * nchunk;
    double2 sum = make_double2(0.0, 0.0);
    for (int k = lane; k < nchunk; k += 32) sum = cadd(sum, __ldcg(pp + k));
    sum = warp_sum2(sum);
    if (lane == 0) h[(long long)(i0 + j) * nrhs + r0 + q] = cscale(sum, fac);
  }
  if (threadIdx.x == 0) *cnt = 0u;
}

// w^r += sign * fac * sum_i V_i^r h[i * nrhs + r]; the coefficients of this right-hand side are
// staged in shared memory (scaled and converted to the arithmetic type).  Block b = r + nrhs e
// (1-D grid): the right-hand sides of one element tile are neighbours in launch order, so a basis
// shared by all right-hand sides is read from DRAM once per tile.
constexpr int AXPY_MAXV = 512;
template <typename SV, typename SW>
__global__ void __launch_bounds__(BT) multiaxpy_kernel(const SV *__restrict__ V, long long vstride,
                                                       long long vrs, int nvec, const double2 *__restrict__ h,
                                                       double sign, SW *__restrict__ w, long long n, int nrhs) {
  using C = Ar<SW>;
  __shared__ C coef[AXPY_MAXV];
  const int r = blockIdx.x % nrhs;
  for (int i = threadIdx.x; i < nvec; i += BT) coef[i] = from_d2<C>(cscale(h[(long long)i * nrhs + r], sign));
  __syncthreads();
  const long long e = (long long)(blockIdx.x / nrhs) * BT + threadIdx.x;
  if (e >= n) return;
  const SV *vp = V + r * vrs + e;
  C acc = ldc(w[r * n + e]);
  for (int i = 0; i < nvec; ++i, vp += vstride) gfma(acc, ldc(*vp), coef[i]);
  w[r * n + e] = stc<SW>(acc);
}

// The same with KV = 16 / sizeof(SV) consecutive elements per thread and one 16-byte load per vector
// (4- and 8-byte storage; every vector starts on a 16-byte boundary, n a multiple of KV).
template <typename SV, typename SW>
__global__ void __launch_bounds__(BT) multiaxpy_vec_kernel(const SV *__restrict__ V, long long vstride,
                                                           long long vrs, int nvec, const double2 *__restrict__ h,
                                                           double sign, SW *__restrict__ w, long long n, int nrhs) {
  using C = Ar<SW>;
  constexpr int KV = 16 / sizeof(SV);
  __shared__ C coef[AXPY_MAXV];
  const int r = blockIdx.x % nrhs;
  for (int i = threadIdx.x; i < nvec; i += BT) coef[i] = from_d2<C>(cscale(h[(long long)i * nrhs + r], sign));
  __syncthreads();
  const long long e = ((long long)(blockIdx.x / nrhs) * BT + threadIdx.x) * KV;
  if (e >= n) return;
  const SV *vp = V + r * vrs + e;
  SW *wp = w + r * n + e;
  SW wv[KV];
  uint4 raw = *reinterpret_cast<const uint4 *>(wp);
  memcpy(wv, &raw, 16);
  C acc[KV];
#pragma unroll
  for (int q = 0; q < KV; ++q) acc[q] = ldc(wv[q]);
  for (int i = 0; i < nvec; ++i, vp += vstride) {
    SV vv[KV];
    const uint4 vr = __ldg(reinterpret_cast<const uint4 *>(vp));
    memcpy(vv, &vr, 16);
    const C cf = coef[i];
#pragma unroll
    for (int q = 0; q < KV; ++q) gfma(acc[q], ldc(vv[q]), cf);
  }
#pragma unroll
  for (int q = 0; q < KV; ++q) wv[q] = stc<SW>(acc[q]);
  memcpy(&raw, wv, 16);
  *reinterpret_cast<uint4 *>(wp) = raw;
}

constexpr int CT = 8;           // output columns per pass in combine
constexpr int COMB_MAXV = 256;  // basis vectors of one combine (coefficient tile in shared memory)
// out_c^r = fac * sum_i V_i^r C[(i * ncol + c) * nrhs + r]; a tile of CT columns of coefficients for
// this right-hand side is staged in shared memory per pass.
template <typename SV, typename SO>
__global__ void __launch_bounds__(BT) combine_kernel(const SV *__restrict__ V, long long vstride,
                                                     long long vrs, int nvec, const double2 *__restrict__ Cf,
                                                     int ncol, double fac, SO *__restrict__ out, long long ostride,
                                                     long long n, int nrhs) {
  using C = Ar<SO>;
  __shared__ C coef[COMB_MAXV * CT];
  // block b = r + nrhs e (1-D grid): a basis shared by the right-hand sides is read once per tile
  const long long e = (long long)(blockIdx.x / nrhs) * BT + threadIdx.x;
  const int r = blockIdx.x % nrhs;
  for (int c0 = 0; c0 < ncol; c0 += CT) {
    const int g = min(CT, ncol - c0);
    __syncthreads();
    for (int q = threadIdx.x; q < nvec * CT; q += BT) {
      const int i = q / CT, j = q % CT;
      coef[q] = (j < g) ? from_d2<C>(cscale(Cf[((long long)i * ncol + c0 + j) * nrhs + r], fac)) : cz<C>();
    }
    __syncthreads();
    if (e >= n) continue;
    C acc[CT];
#pragma unroll
    for (int j = 0; j < CT; ++j) acc[j] = cz<C>();
    const SV *vp = V + r * vrs + e;
    for (int i = 0; i < nvec; ++i, vp += vstride) {
      const C v = ldc(*vp);
#pragma unroll
      for (int j = 0; j < CT; ++j) gfma(acc[j], v, coef[i * CT + j]);
    }
#pragma unroll
    for (int j = 0; j < CT; ++j)
      if (j < g) out[(long long)(c0 + j) * ostride + r * n + e] = stc<SO>(acc[j]);
  }
}

// The same with KV = 16 / sizeof(SV) consecutive elements per thread and one 16-byte load per basis
// vector (4- and 8-byte basis storage on 16-byte boundaries, n a multiple of KV); one output column
// per pass keeps the KV accumulators in registers.
template <typename SV, typename SO>
__global__ void __launch_bounds__(BT) combine_vec_kernel(const SV *__restrict__ V, long long vstride,
                                                         long long vrs, int nvec, const double2 *__restrict__ Cf,
                                                         int ncol, double fac, SO *__restrict__ out,
                                                         long long ostride, long long n, int nrhs) {
  using C = Ar<SO>;
  constexpr int KV = 16 / sizeof(SV);
  __shared__ C coef[COMB_MAXV];
  const long long e = ((long long)(blockIdx.x / nrhs) * BT + threadIdx.x) * KV;
  const int r = blockIdx.x % nrhs;
  for (int c = 0; c < ncol; ++c) {
    __syncthreads();
    for (int i = threadIdx.x; i < nvec; i += BT)
      coef[i] = from_d2<C>(cscale(Cf[((long long)i * ncol + c) * nrhs + r], fac));
    __syncthreads();
    if (e >= n) continue;
    C acc[KV];
#pragma unroll
    for (int q = 0; q < KV; ++q) acc[q] = cz<C>();
    const SV *vp = V + r * vrs + e;
    for (int i = 0; i < nvec; ++i, vp += vstride) {
      SV vv[KV];
      const uint4 raw = __ldg(reinterpret_cast<const uint4 *>(vp));
      memcpy(vv, &raw, 16);
      const C cf = coef[i];
#pragma unroll
      for (int q = 0; q < KV; ++q) gfma(acc[q], ldc(vv[q]), cf);
    }
    SO *op = out + (long long)c * ostride + r * n + e;
#pragma unroll
    for (int q = 0; q < KV; ++q) op[q] = stc<SO>(acc[q]);
  }
}

template <typename S>
__global__ void invscale_kernel(S *__restrict__ x, const double *__restrict__ s, long long n) {
  // the reciprocal once per block, then one multiply per component in the arithmetic type
  using R = decltype(Ar<S>().x);
  __shared__ R f;
  const int r = blockIdx.y;
  if (threadIdx.x == 0) {
    const double d = s[r];
    f = (R)(d > 0.0 ? 1.0 / d : 0.0);
  }
  __syncthreads();
  const long long e = (long long)blockIdx.x * BT + threadIdx.x;
  if (e >= n) return;
  Ar<S> v = ldc(x[r * n + e]);
  v.x *= f;
  v.y *= f;
  x[r * n + e] = stc<S>(v);
}

// The same with KV = 16 / sizeof(S) consecutive elements per thread and one 16-byte access each way
// (4- and 8-byte storage, x on a 16-byte boundary, n a multiple of KV)
template <typename S>
__global__ void invscale_vec_kernel(S *__restrict__ x, const double *__restrict__ s, long long n) {
  using R = decltype(Ar<S>().x);
  constexpr int KV = 16 / sizeof(S);
  __shared__ R f;
  const int r = blockIdx.y;
  if (threadIdx.x == 0) {
    const double d = s[r];
    f = (R)(d > 0.0 ? 1.0 / d : 0.0);
  }
  __syncthreads();
  const long long e = ((long long)blockIdx.x * BT + threadIdx.x) * KV;
  if (e >= n) return;
  uint4 *p = reinterpret_cast<uint4 *>(x + r * n + e);
  uint4 raw = *p;
  S v[KV];
  memcpy(v, &raw, 16);
#pragma unroll
  for (int q = 0; q < KV; ++q) {
    Ar<S> a = ldc(v[q]);
    a.x *= f;
    a.y *= f;
    v[q] = stc<S>(a);
  }
  memcpy(&raw, v, 16);
  *p = raw;
}

// y = fac * x with conversion between storage types (fac = 1 for a plain copy)
template <typename SX, typename SY>
__global__ void copy_kernel(const SX *__restrict__ x, SY *__restrict__ y, long long n, double fac) {
  for (long long e = (long long)blockIdx.x * BT + threadIdx.x; e < n; e += (long long)gridDim.x * BT) {
    if constexpr (std::is_same<SX, SY>::value) {
      y[e] = x[e];
    } else {
      using R = decltype(Ar<SY>().x);
      Ar<SY> v = ldc(x[e]);
      v.x *= (R)fac;
      v.y *= (R)fac;
      y[e] = stc<SY>(v);
    }
  }
}

// y = a x + b y (complex scalars; storage S, arithmetic of S; FP16 / BF16 vectors carry the same
// store_sigma factor on both sides, which the linear combination keeps)
template <typename S>
__global__ void axpby_kernel(double2 a, const S *__restrict__ x, double2 b, S *__restrict__ y, long long n) {
  using C = Ar<S>;
  const C ca = from_d2<C>(a), cb = from_d2<C>(b);
  for (long long e = (long long)blockIdx.x * BT + threadIdx.x; e < n; e += (long long)gridDim.x * BT) {
    const C xv = ldc(x[e]), yv = ldc(y[e]);
    C o = cz<C>();
    gfma(o, ca, xv);
    gfma(o, cb, yv);
    y[e] = stc<S>(o);
  }
}

template <typename S>
__global__ void zero_kernel(S *__restrict__ y, long long n) {
  for (long long e = (long long)blockIdx.x * BT + threadIdx.x; e < n; e += (long long)gridDim.x * BT)
    y[e] = stc<S>(cz<Ar<S>>());
}

// y^r = float(x^r / s[r]): FP64 residual block -> normalised FP32 right-hand side
__global__ void demote_kernel(const double2 *__restrict__ x, const double *__restrict__ s, float2 *__restrict__ y,
                              long long n) {
  const long long e = (long long)blockIdx.x * BT + threadIdx.x;
  const int r = blockIdx.y;
  if (e >= n) return;
  const double d = s[r];
  const double f = d > 0.0 ? 1.0 / d : 0.0;
  const double2 v = x[r * n + e];
  y[r * n + e] = make_float2((float)(v.x * f), (float)(v.y * f));
}

// x^r += s[r] * double(e^r): FP32 correction folded into the FP64 solution
__global__ void promote_acc_kernel(const float2 *__restrict__ c, const double *__restrict__ s, double2 *__restrict__ x,
                                   long long n) {
  const long long e = (long long)blockIdx.x * BT + threadIdx.x;
  const int r = blockIdx.y;
  if (e >= n) return;
  const double d = s[r];
  const float2 v = c[r * n + e];
  double2 o = x[r * n + e];
  o.x = fma(d, (double)v.x, o.x);
  o.y = fma(d, (double)v.y, o.y);
  x[r * n + e] = o;
}

// elementwise conversion double2 -> float2 (gauge links of the FP32 operator)
__global__ void to_f32_kernel(const double2 *__restrict__ x, float2 *__restrict__ y, long long n) {
  for (long long e = (long long)blockIdx.x * BT + threadIdx.x; e < n; e += (long long)gridDim.x * BT)
    y[e] = make_float2((float)x[e].x, (float)x[e].y);
}

__global__ void axpy_kernel(double2 a, const double2 *__restrict__ x, double2 *__restrict__ y, long long n) {
  for (long long e = (long long)blockIdx.x * BT + threadIdx.x; e < n; e += (long long)gridDim.x * BT) {
    double2 v = y[e];
    cfma(v, a, x[e]);
    y[e] = v;
  }
}

__global__ void bminus_kernel(double2 *__restrict__ t, const double2 *__restrict__ b, long long n) {
  for (long long e = (long long)blockIdx.x * BT + threadIdx.x; e < n; e += (long long)gridDim.x * BT)
    t[e] = csub(b[e], t[e]);
}

// gamma_5 = -[[0,1],[1,0]] on spin: one thread per (site, rhs) pair
__global__ void g5_kernel(const double2 *__restrict__ x, double2 *__restrict__ y, long long sites) {
  const long long s = (long long)blockIdx.x * BT + threadIdx.x;
  if (s >= sites) return;
  const double2 *a = x + 12 * s;
  double2 *b = y + 12 * s;
  double2 t[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) t[i] = a[i];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    b[0 + c] = make_double2(-t[6 + c].x, -t[6 + c].y);
    b[3 + c] = make_double2(-t[9 + c].x, -t[9 + c].y);
    b[6 + c] = make_double2(-t[0 + c].x, -t[0 + c].y);
    b[9 + c] = make_double2(-t[3 + c].x, -t[3 + c].y);
  }
}

// ---- Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Z(4) noise -------------------------
struct U4 { uint32_t v[4]; };

__device__ __forceinline__ U4 philox10(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = M0 * c.v[0], hi0 = __umulhi(M0, c.v[0]);
    const uint32_t lo1 = M1 * c.v[2], hi1 = __umulhi(M1, c.v[2]);
    U4 d;
    d.v[0] = hi1 ^ c.v[1] ^ k0;
    d.v[1] = lo1;
    d.v[2] = hi0 ^ c.v[3] ^ k1;
    d.v[3] = lo0;
    c = d;
    k0 += W0;
    k1 += W1;
  }
  return c;
}

__global__ void noise_kernel(uint32_t key0, uint32_t key1, uint32_t first, int V, double2 *__restrict__ out) {
  const int s = blockIdx.x * BT + threadIdx.x;
  const int n = blockIdx.y;
  if (s >= V) return;
  U4 c;
  c.v[0] = first + (uint32_t)n;
  c.v[1] = (uint32_t)s;
  c.v[2] = 0u;
  c.v[3] = 0u;
  const uint32_t w = philox10(c, key0, key1).v[0];
  double2 *o = out + ((long long)n * V + s) * 12;
#pragma unroll
  for (int e = 0; e < 12; ++e) {
    const uint32_t code = (w >> (2 * e)) & 3u;
    // 0 -> 1, 1 -> i, 2 -> -1, 3 -> -i
    const double re = (code == 0u) ? 1.0 : ((code == 2u) ? -1.0 : 0.0);
    const double im = (code == 1u) ? 1.0 : ((code == 3u) ? -1.0 : 0.0);
    o[e] = make_double2(re, im);
  }
}

int blocks_for(long long n) { return (int)std::min<long long>((n + BT - 1) / BT, 1 << 20); }

int partial_blocks(lqcd_ctx *ctx, long long n, int nrhs) {
  long long want = std::max<long long>(1, (4LL * ctx->sms) / std::max(1, nrhs));
  long long maxb = std::max<long long>(1, (n + BT - 1) / BT);
  return (int)std::max<long long>(1, std::min<long long>(std::min(want, maxb), 1024));
}

}  // namespace

template <typename SX, typename SY>
lqcd_status blas_copy(lqcd_ctx *ctx, const SX *x, SY *y, long long n) {
  static_assert(std::is_same<SX, SY>::value || std::is_same<Ar<SX>, Ar<SY>>::value, "copy: incompatible types");
  const double fac = store_sigma<SY>(ctx->N) / store_sigma<SX>(ctx->N);
  kbegin(ctx);
  copy_kernel<SX, SY><<<std::min(blocks_for(n), 8 * ctx->sms), BT, 0, ctx->stream>>>(x, y, n, fac);
  return launch_check(ctx, "copy_kernel", K_BLAS1, (double)n);
}

template <typename S>
lqcd_status blas_zero(lqcd_ctx *ctx, S *y, long long n) {
  kbegin(ctx);
  zero_kernel<S><<<std::min(blocks_for(n), 8 * ctx->sms), BT, 0, ctx->stream>>>(y, n);
  return launch_check(ctx, "zero_kernel", K_BLAS1, (double)n);
}

template <typename S>
lqcd_status blas_axpby(lqcd_ctx *ctx, double2 a, const S *x, double2 b, S *y, long long n) {
  kbegin(ctx);
  axpby_kernel<S><<<std::min(blocks_for(n), 8 * ctx->sms), BT, 0, ctx->stream>>>(a, x, b, y, n);
  return launch_check_bytes(ctx, "axpby_kernel", K_BLAS1, (double)n, 3.0 * sizeof(S) * n);
}

lqcd_status blas_axpy(lqcd_ctx *ctx, double2 a, const double2 *x, double2 *y, long long n) {
  kbegin(ctx);
  axpy_kernel<<<std::min(blocks_for(n), 8 * ctx->sms), BT, 0, ctx->stream>>>(a, x, y, n);
  return launch_check(ctx, "axpy_kernel", K_BLAS1, (double)n);
}

lqcd_status blas_bminus(lqcd_ctx *ctx, double2 *t, const double2 *b, long long n) {
  kbegin(ctx);
  bminus_kernel<<<std::min(blocks_for(n), 8 * ctx->sms), BT, 0, ctx->stream>>>(t, b, n);
  return launch_check(ctx, "bminus_kernel", K_BLAS1, (double)n);
}

lqcd_status blas_g5(lqcd_ctx *ctx, const double2 *x, double2 *y, int nrhs) {
  long long sites = (long long)ctx->V * nrhs;
  kbegin(ctx);
  g5_kernel<<<(int)((sites + BT - 1) / BT), BT, 0, ctx->stream>>>(x, y, sites);
  return launch_check(ctx, "g5_kernel", K_BLAS1, (double)sites * 12);
}

// per-right-hand-side arrival counters of the single-launch reductions (zeroed once, left at zero)
static lqcd_status reduction_counters(lqcd_ctx *ctx, int nrhs, unsigned **c) {
  const size_t need = sizeof(unsigned) * (size_t)std::max(nrhs, 1);
  const bool fresh = ctx->ws_size[WS_COUNT] < need;
  LQCD_TRY(ws_get(ctx, WS_COUNT, need, (void **)c));
  if (fresh) LQCD_CUDA(ctx, cudaMemsetAsync(*c, 0, ctx->ws_size[WS_COUNT], ctx->stream));
  return LQCD_OK;
}

template <typename S>
lqcd_status blas_norms(lqcd_ctx *ctx, const S *x, long long n, int nrhs, double *norms) {
  const int nb = partial_blocks(ctx, n, nrhs);
  void *p = nullptr;
  unsigned *cnt = nullptr;
  LQCD_TRY(ws_get(ctx, WS_SCAL, sizeof(double) * (size_t)nb * nrhs, &p));
  LQCD_TRY(reduction_counters(ctx, nrhs, &cnt));
  kbegin(ctx);
  norm_kernel<S><<<dim3(nb, nrhs), BT, 0, ctx->stream>>>(x, n, 1.0 / store_sigma<S>(ctx->N), (double *)p, cnt, norms);
  return launch_check_bytes(ctx, "norm_kernel", K_NORM, (double)n * nrhs, (double)sizeof(S) * n * nrhs);
}

static int multidot_chunks(lqcd_ctx *ctx, long long n, int nrhs, int nvec, bool shared) {
  // element chunks of at least 8 elements per thread; enough blocks (chunks x vector groups x
  // right-hand sides) for about 16 per SM, several waves of the 4-6 resident ones, so that no SM
  // idles at the end.  With a basis shared by several right-hand
  // sides, also chunks short enough that the blocks in flight (about 8 per SM) touch at most ~32 MB
  // of L2, so that the basis chunk is read from DRAM once for all of them.
  const int ngroup = (nvec + GROUP - 1) / GROUP;
  const long long max_chunks = std::max<long long>(1, n / (8LL * BT));
  long long want = std::max<long long>(1, (16LL * ctx->sms) / std::max<long long>(1, (long long)nrhs * ngroup));
  if (shared && nrhs > 1) {
    const long long per_chunk_blocks = (long long)nrhs * ngroup;
    const long long chunks_in_flight = std::max<long long>(1, 8LL * ctx->sms / per_chunk_blocks);
    const long long bytes_per_elem = 16LL * (nvec + nrhs);        // upper bound (FP64 storage)
    const long long l2_chunk = std::max<long long>(8LL * BT, (32LL << 20) / (chunks_in_flight * bytes_per_elem));
    want = std::max(want, (n + l2_chunk - 1) / l2_chunk);
  }
  return (int)std::min<long long>(std::min(max_chunks, want), 4096);
}

lqcd_status blas_reserve(lqcd_ctx *ctx, long long n, int nrhs, int max_nvec) {
  size_t need = 0;
  for (int v = 1; v <= max_nvec; ++v)
    need = std::max(need, sizeof(double2) * (size_t)std::max(multidot_chunks(ctx, n, nrhs, v, false),
                                                             multidot_chunks(ctx, n, nrhs, v, true)) * nrhs * v);
  void *p = nullptr;
  unsigned *cnt = nullptr;
  LQCD_TRY(ws_get(ctx, WS_PARTIAL, need, &p));
  LQCD_TRY(ws_get(ctx, WS_SCAL, sizeof(double) * (size_t)partial_blocks(ctx, n, nrhs) * nrhs, &p));
  return reduction_counters(ctx, nrhs * ((std::max(max_nvec, 1) + GROUP - 1) / GROUP), &cnt);
}

template <typename SV, typename SW>
lqcd_status blas_multidot(lqcd_ctx *ctx, const SV *V, long long vstride, long long vrs, int nvec, const SW *w,
                          long long n, int nrhs, double2 *h) {
  if (nvec <= 0) return LQCD_OK;
  const int ngroup = (nvec + GROUP - 1) / GROUP;
  if (vrs == 0 && nrhs > 1) {
    // shared basis: RT = 2 right-hand sides per block (register budget: 16 complex accumulators)
    constexpr int RT = 2;
    const int ntile = (nrhs + RT - 1) / RT;
    const int nchunk = multidot_chunks(ctx, n, ntile, nvec, false);
    if ((long long)nchunk * ngroup * ntile > 0x7fffffffLL) return set_err(ctx, LQCD_ERR_INVALID_ARG, "multidot: grid too large");
    void *p = nullptr;
    unsigned *cnt = nullptr;
    LQCD_TRY(ws_get(ctx, WS_PARTIAL, sizeof(double2) * (size_t)nchunk * nrhs * nvec, &p));
    LQCD_TRY(reduction_counters(ctx, ntile * ngroup, &cnt));
    const double fac = 1.0 / (store_sigma<SV>(ctx->N) * store_sigma<SW>(ctx->N));
    kbegin(ctx);
    multidot_shared_kernel<SV, SW, RT><<<(unsigned)((long long)nchunk * ngroup * ntile), BT, 0, ctx->stream>>>(
        V, vstride, nvec, w, n, nrhs, nchunk, fac, (double2 *)p, cnt, h);
    const double bytes = (double)sizeof(SV) * n * nvec + (double)sizeof(SW) * n * nrhs;
    return launch_check_bytes(ctx, "multidot_shared_kernel", K_DOT, (double)n * nrhs * nvec, bytes);
  }
  const int nchunk = multidot_chunks(ctx, n, nrhs, nvec, vrs == 0);
  if ((long long)nchunk * ngroup * nrhs > 0x7fffffffLL) return set_err(ctx, LQCD_ERR_INVALID_ARG, "multidot: grid too large");
  void *p = nullptr;
  unsigned *cnt = nullptr;
  LQCD_TRY(ws_get(ctx, WS_PARTIAL, sizeof(double2) * (size_t)nchunk * nrhs * nvec, &p));
  LQCD_TRY(reduction_counters(ctx, nrhs * ngroup, &cnt));
  const double fac = 1.0 / (store_sigma<SV>(ctx->N) * store_sigma<SW>(ctx->N));
  // 16-byte loads for the 4- and 8-byte storage types when every vector starts on a 16-byte boundary
  const bool vec = sizeof(SV) < 16 && sizeof(SV) == sizeof(SW) && ((uintptr_t)V % 16 == 0) &&
                   ((uintptr_t)w % 16 == 0) && ((vstride * (long long)sizeof(SV)) % 16 == 0) &&
                   ((vrs * (long long)sizeof(SV)) % 16 == 0) && ((n * (long long)sizeof(SW)) % 16 == 0);
  const unsigned grid = (unsigned)((long long)nchunk * ngroup * nrhs);
  kbegin(ctx);
  // at most two vectors (the Lanczos window): the two-vector form, with a quarter of the registers
  // for loads and accumulators, so that more blocks are resident to hide the DRAM latency
  if (vec && nvec <= 2)
    multidot_kernel<SV, SW, true, 2><<<grid, BT, 0, ctx->stream>>>(V, vstride, vrs, nvec, w, n, nrhs, nchunk, fac,
                                                                  (double2 *)p, cnt, h);
  else if (vec)
    multidot_kernel<SV, SW, true, GROUP><<<grid, BT, 0, ctx->stream>>>(V, vstride, vrs, nvec, w, n, nrhs, nchunk,
                                                                      fac, (double2 *)p, cnt, h);
  else
    multidot_kernel<SV, SW, false, GROUP><<<grid, BT, 0, ctx->stream>>>(V, vstride, vrs, nvec, w, n, nrhs, nchunk,
                                                                       fac, (double2 *)p, cnt, h);
  // compulsory bytes: every basis vector once (once per right-hand side when the bases differ),
  // every w once
  const double bytes = (double)sizeof(SV) * n * nvec * (vrs != 0 ? nrhs : 1) + (double)sizeof(SW) * n * nrhs;
  return launch_check_bytes(ctx, "multidot_kernel", K_DOT, (double)n * nrhs * nvec, bytes);
}

template <typename SV, typename SW>
lqcd_status blas_multiaxpy(lqcd_ctx *ctx, const SV *V, long long vstride, long long vrs, int nvec, const double2 *h,
                           double sign, SW *w, long long n, int nrhs) {
  if (nvec <= 0) return LQCD_OK;
  if (nvec > AXPY_MAXV) return set_err(ctx, LQCD_ERR_INVALID_ARG, "multiaxpy: at most %d vectors", AXPY_MAXV);
  const double fac = sign * store_sigma<SW>(ctx->N) / store_sigma<SV>(ctx->N);
  const bool vec = sizeof(SV) < 16 && sizeof(SV) == sizeof(SW) && ((uintptr_t)V % 16 == 0) &&
                   ((uintptr_t)w % 16 == 0) && ((vstride * (long long)sizeof(SV)) % 16 == 0) &&
                   ((vrs * (long long)sizeof(SV)) % 16 == 0) && ((n * (long long)sizeof(SW)) % 16 == 0);
  kbegin(ctx);
  if (vec) {
    const long long kv = 16 / (long long)sizeof(SV);
    multiaxpy_vec_kernel<SV, SW><<<(unsigned)((long long)ceil_div(n / kv, BT) * nrhs), BT, 0, ctx->stream>>>(
        V, vstride, vrs, nvec, h, fac, w, n, nrhs);
  } else {
    multiaxpy_kernel<SV, SW><<<(unsigned)((long long)ceil_div(n, BT) * nrhs), BT, 0, ctx->stream>>>(V, vstride, vrs,
                                                                                                  nvec, h, fac, w, n,
                                                                                                  nrhs);
  }
  // compulsory bytes: every basis vector once (per right-hand side when the bases differ), w read
  // and written once
  const double bytes = (double)sizeof(SV) * n * nvec * (vrs != 0 ? nrhs : 1) + 2.0 * sizeof(SW) * n * nrhs;
  return launch_check_bytes(ctx, "multiaxpy_kernel", K_AXPY, (double)n * nrhs * nvec, bytes);
}

template <typename SV, typename SO>
lqcd_status blas_combine(lqcd_ctx *ctx, const SV *V, long long vstride, long long vrs, int nvec, const double2 *C,
                         int ncol, SO *out, long long ostride, long long n, int nrhs) {
  if (ncol <= 0) return LQCD_OK;
  if (nvec > COMB_MAXV) return set_err(ctx, LQCD_ERR_INVALID_ARG, "combine: at most %d vectors", COMB_MAXV);
  const double fac = store_sigma<SO>(ctx->N) / store_sigma<SV>(ctx->N);
  const bool vec = sizeof(SV) < 16 && ncol <= 2 && ((uintptr_t)V % 16 == 0) &&
                   ((vstride * (long long)sizeof(SV)) % 16 == 0) && ((vrs * (long long)sizeof(SV)) % 16 == 0) &&
                   ((n * (long long)sizeof(SV)) % 16 == 0);
  kbegin(ctx);
  if (vec) {
    const long long kv = 16 / (long long)sizeof(SV);
    combine_vec_kernel<SV, SO><<<(unsigned)((long long)ceil_div(n / kv, BT) * nrhs), BT, 0, ctx->stream>>>(
        V, vstride, vrs, nvec, C, ncol, fac, out, ostride, n, nrhs);
  } else {
    combine_kernel<SV, SO><<<(unsigned)((long long)ceil_div(n, BT) * nrhs), BT, 0, ctx->stream>>>(
        V, vstride, vrs, nvec, C, ncol, fac, out, ostride, n, nrhs);
  }
  const double bytes = (double)sizeof(SV) * n * nvec * (vrs != 0 ? nrhs : 1) + (double)sizeof(SO) * n * ncol * nrhs;
  return launch_check_bytes(ctx, "combine_kernel", K_COMBINE, (double)n * nrhs * nvec * ncol, bytes);
}

template <typename S>
lqcd_status blas_invscale(lqcd_ctx *ctx, S *x, const double *s, long long n, int nrhs) {
  kbegin(ctx);
  if (sizeof(S) < 16 && (uintptr_t)x % 16 == 0 && (n * (long long)sizeof(S)) % 16 == 0) {
    const long long kv = 16 / (long long)sizeof(S);
    invscale_vec_kernel<S><<<dim3(ceil_div(n / kv, BT), nrhs), BT, 0, ctx->stream>>>(x, s, n);
  } else {
    invscale_kernel<S><<<dim3(ceil_div(n, BT), nrhs), BT, 0, ctx->stream>>>(x, s, n);
  }
  return launch_check_bytes(ctx, "invscale_kernel", K_BLAS1, (double)n * nrhs, 2.0 * sizeof(S) * n * nrhs);
}

lqcd_status blas_demote(lqcd_ctx *ctx, const double2 *x, const double *s, float2 *y, long long n, int nrhs) {
  kbegin(ctx);
  demote_kernel<<<dim3(ceil_div(n, BT), nrhs), BT, 0, ctx->stream>>>(x, s, y, n);
  return launch_check(ctx, "demote_kernel", K_BLAS1, (double)n * nrhs);
}

lqcd_status blas_promote_acc(lqcd_ctx *ctx, const float2 *c, const double *s, double2 *x, long long n, int nrhs) {
  kbegin(ctx);
  promote_acc_kernel<<<dim3(ceil_div(n, BT), nrhs), BT, 0, ctx->stream>>>(c, s, x, n);
  return launch_check(ctx, "promote_acc_kernel", K_BLAS1, (double)n * nrhs);
}

lqcd_status blas_to_f32(lqcd_ctx *ctx, const double2 *x, float2 *y, long long n) {
  kbegin(ctx);
  to_f32_kernel<<<std::min(blocks_for(n), 8 * ctx->sms), BT, 0, ctx->stream>>>(x, y, n);
  return launch_check(ctx, "to_f32_kernel", K_BLAS1, (double)n);
}

#define LQCD_BLAS_INSTANTIATE(S)                                                                               \
  template lqcd_status blas_copy<S, S>(lqcd_ctx *, const S *, S *, long long);                                  \
  template lqcd_status blas_axpby<S>(lqcd_ctx *, double2, const S *, double2, S *, long long);                  \
  template lqcd_status blas_zero<S>(lqcd_ctx *, S *, long long);                                                \
  template lqcd_status blas_norms<S>(lqcd_ctx *, const S *, long long, int, double *);                          \
  template lqcd_status blas_invscale<S>(lqcd_ctx *, S *, const double *, long long, int);
#define LQCD_BLAS_INSTANTIATE2(SV, SW)                                                                         \
  template lqcd_status blas_multidot<SV, SW>(lqcd_ctx *, const SV *, long long, long long, int, const SW *,     \
                                             long long, int, double2 *);                                       \
  template lqcd_status blas_multiaxpy<SV, SW>(lqcd_ctx *, const SV *, long long, long long, int, const double2 *, \
                                              double, SW *, long long, int);                                   \
  template lqcd_status blas_combine<SV, SW>(lqcd_ctx *, const SV *, long long, long long, int, const double2 *,  \
                                            int, SW *, long long, long long, int);
LQCD_BLAS_INSTANTIATE(double2)
LQCD_BLAS_INSTANTIATE(float2)
LQCD_BLAS_INSTANTIATE(__half2)
LQCD_BLAS_INSTANTIATE(__nv_bfloat162)
LQCD_BLAS_INSTANTIATE2(double2, double2)
LQCD_BLAS_INSTANTIATE2(float2, float2)
LQCD_BLAS_INSTANTIATE2(__half2, __half2)
LQCD_BLAS_INSTANTIATE2(__half2, float2)
LQCD_BLAS_INSTANTIATE2(__nv_bfloat162, __nv_bfloat162)
LQCD_BLAS_INSTANTIATE2(__nv_bfloat162, float2)
template lqcd_status blas_copy<float2, __half2>(lqcd_ctx *, const float2 *, __half2 *, long long);
template lqcd_status blas_copy<float2, __nv_bfloat162>(lqcd_ctx *, const float2 *, __nv_bfloat162 *, long long);

lqcd_status noise_launch(lqcd_ctx *ctx, uint64_t seed, uint32_t first, int nrhs, double2 *out) {
  kbegin(ctx);
  noise_kernel<<<dim3(ceil_div(ctx->V, BT), nrhs), BT, 0, ctx->stream>>>((uint32_t)(seed & 0xffffffffu),
                                                                          (uint32_t)(seed >> 32), first, ctx->V, out);
  return launch_check(ctx, "noise_kernel", K_NOISE, (double)ctx->V * nrhs);
}

// ---- input check: NaN / Inf anywhere in an FP64 array ------------------------------------------
namespace {
__global__ void nonfinite_kernel(const double *__restrict__ x, long long n, unsigned *__restrict__ count) {
  unsigned bad = 0;
  for (long long e = (long long)blockIdx.x * BT + threadIdx.x; e < n; e += (long long)gridDim.x * BT)
    bad += isfinite(x[e]) ? 0u : 1u;
  bad = __reduce_add_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd(count, bad);
}
}  // namespace

lqcd_status check_finite(lqcd_ctx *ctx, const double *x, long long n, const char *what) {
  unsigned *cnt;
  LQCD_TRY(ws_get(ctx, WS_SCAL, sizeof(double) * 2, (void **)&cnt));
  LQCD_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(unsigned), ctx->stream));
  kbegin(ctx);
  nonfinite_kernel<<<std::min(blocks_for(n), 8 * ctx->sms), BT, 0, ctx->stream>>>(x, n, cnt);
  LQCD_TRY(launch_check(ctx, "nonfinite_kernel", K_BLAS1, (double)n / 2));
  unsigned h = 0;
  LQCD_CUDA(ctx, cudaMemcpyAsync(&h, cnt, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
  LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (h) return set_err(ctx, LQCD_ERR_NONFINITE, "%s: %u non-finite values", what, h);
  return LQCD_OK;
}

extern "C" lqcd_status lqcd_noise_z4(lqcd_ctx *ctx, uint64_t seed, uint32_t first_noise, int nrhs, double *out) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_full(ctx, "noise_z4"));
  if (!out || nrhs <= 0 || nrhs > 65535) return set_err(ctx, LQCD_ERR_INVALID_ARG, "noise_z4: bad arguments");
  return noise_launch(ctx, seed, first_noise, nrhs, (double2 *)out);
}
