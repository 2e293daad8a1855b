// FP64-accurate deflation contractions on the tcgen05 tensor cores (split-precision emulation).
//
// The HFES projection of Sec. 5.4, x' = gamma_5 V' Lambda'^-1 V'^dag eta, is two dense products
// with the k deflation vectors E (k x 12V complex):
//
//   G = E^dag X     (k x nrhs; the reduction runs over the 24 V reals of a field)
//   Y = E C         (nrhs fields; the reduction runs over the k vectors)
//
// Both are computed to FP64 accuracy with bf16 tensor-core products (Ozaki's error-free splitting,
// Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59 (2012)):
//
//  * every row of the left operand (over the reduction index) is scaled by a power of two 2^e so
//    that its entries are below 1/2, and written as seven balanced base-256 digits,
//    x 2^-e = sum_s d_s 2^(-8(s+1)) with |d_s| <= 128 (truncated after 56 bits, an error below
//    2^-54 of the row's largest entry): each slice d_s 2^(-8(s+1)) is exact in bf16.  The rows are
//    the vectors E_q for G and the real components m of the fields for Y, so the two products
//    use two slice copies of E, each with its own scales;
//  * the right operand is split the same way per column (seven slices), or, when every entry of
//    the block is a small integer times a common power of two (Z(4) noise: 0, +-1), kept as one
//    exact slice;
//  * slice products d_s d'_t carry the unit 2^(-8(s+t+c)); products of one "group" g = s + t
//    share a unit, so their FP32 sums in TMEM are exact integers as long as they stay within 2^24
//    units (every partial sum is then an integer of at most 24 bits).  Every group g <= 7 has its
//    own accumulator (TMEM columns g NP .. (g+1) NP - 1): stacking the slices of the right operand
//    along N, one MMA of left slice s against right slices t0..t1 writes A_s B_t straight into the
//    columns of group s + t, so TMEM does the grouping.  Groups 0..4 are read out (and combined as
//    an exact 64-bit integer, then FP64) often enough to stay within the 2^24 bound; groups 5..7,
//    at least 2^-40 below the leading group, are added in FP32 (rounding below 2^-60 of the
//    leading term).  Pairs with s + t > 7 are not formed (below 2^-62 of the leading term).
//  Per entry of the result the error is thus below about 2^-52 (max_i |a_i| sum_i |b_i| +
//  sum_i |a_i| max_i |b_i|) plus the FP64 rounding of the folds, the bound of the splitting
//  (an FP64 dot product has 2^-53 n sum_i |a_i||b_i| in the worst case).
//
// The tensor-core kernel (tc_gemm_kernel) is a persistent, warp-specialised tcgen05 GEMM:
//   warp 8 (one lane)  moves pre-tiled slice blocks global -> shared with cp.async.bulk into a
//                      ring of stages guarded by mbarriers (full / empty);
//   warp 9 (one lane)  issues tcgen05.mma.cta_group::1.kind::f16 (bf16 x bf16 -> FP32, M = 128,
//                      N = (slices stacked) x NP <= 256, K = 16) into TMEM: 7 (Z(4) right operand)
//                      to 11 MMAs per 16 reduction elements, an unrolled sequence with constant
//                      descriptor offsets; tcgen05.commit frees a stage / hands an accumulator set
//                      to the epilogue;
//   warps 0-7          read the accumulators with tcgen05.ld (warp w owns TMEM lanes 32 (w % 4) ..
//                      32 (w % 4) + 31, i.e. output rows; warps 0-3 take the first half of the
//                      columns, warps 4-7 the second), fold the slice groups into FP64 and write
//                      the result, then zero the accumulator set (tcgen05.st) for its next use.
//                      Eight warps hide the latency of the integer / FP64 folds.
// Two accumulator sets in TMEM (when they fit in 512 columns) let the MMAs of the next group run
// while the epilogue drains the previous one.
//
// Operand storage (K-major, no swizzle): a block of R rows x 32 K elements (bf16) is made of
// 8 x 8 "core matrices" of 128 contiguous bytes (8 rows of 16 bytes), core matrix (i, j) (row
// group i, K group j) at byte (4 i + j) * 128.  In the tcgen05 shared-memory descriptor the K
// direction stride between core matrices (leading byte offset) is 128 and the row-group stride
// (stride byte offset) is 512.  The slicing kernels write the slices in exactly this order, so a
// pipeline stage is filled by plain bulk copies.
//
// Every mbarrier wait is bounded in time: after about two seconds the kernel records
// LQCD_ERR_TIMEOUT in a device flag, stops issuing work, waits (again bounded) for the copies and
// MMAs it has in flight, frees its TMEM and returns.
#include <algorithm>

#include "common.cuh"

namespace {

constexpr int TC_M = 128;                  // rows per tile = TMEM lanes
constexpr int TC_KCH = 32;                 // K elements per pipeline chunk (64 bytes per row)
constexpr int TC_SA = 7;                   // slices of the row-scaled operand (7 x 8 bits)
constexpr int TC_NGRP = 8;                 // accumulated slice groups g = s + t <= 7
constexpr int TC_NEXACT = 5;               // groups 0..4 are exact integers; 5..7 are summed in FP32
constexpr int TC_THREADS = 320;            // warps 0-7 epilogue, 8 loader, 9 MMA issuer
constexpr int TC_EPI_WARPS = 8;
constexpr int TC_BLK = TC_M * TC_KCH * 2;  // bytes of a full 128-row slice block (8 KB)
constexpr int TC_SMEM_MAX = 227 * 1024;
constexpr int TC_SMEM_MIN = 120 * 1024;    // forces one CTA per SM (TMEM is allocated per CTA)
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;  // default bound of a pipeline wait; fixed bound of a drain

// byte offset of element (row, k) of an R x 32 block in the core-matrix order above
__host__ __device__ __forceinline__ int tile_off(int row, int k) {
  return ((((row >> 3) << 2) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}
__host__ __device__ __forceinline__ int round8(int x) { return (x + 7) & ~7; }

// ---------------------------------------------------------------------------------------------
// Digits of the splitting
// ---------------------------------------------------------------------------------------------

// Scale exponent of a row / column whose largest magnitude has the bit pattern mb: e such that
// every entry satisfies |x| < 2^(e-1) (0 for an all-zero vector).
__host__ __device__ __forceinline__ int scale_exp(unsigned long long mb) {
  const int be = (int)((mb >> 52) & 0x7ff);
  return be == 0 ? 0 : be - 1021;
}

// Balanced base-256 digits of x 2^-e truncated after 56 bits: x 2^-e ~= sum_s d[s] 2^(-8(s+1)),
// |d[s]| <= 128, error below 2^-56.  Requires |x| < 2^(e-1).  Zeros and subnormals give 0
// digits (the scales used here are far above the subnormal range).
__device__ __forceinline__ void split_digits(double x, int e, int d[TC_SA]) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int be = (int)((u >> 52) & 0x7ff);
  long long F = 0;
  if (be != 0 && be != 0x7ff) {
    const unsigned long long mant = (u & 0xfffffffffffffull) | (1ull << 52);
    const int sh = be - 1075 + 8 * TC_SA - e;  // |x| < 2^(e-1) => F < 2^55
    if (sh >= 0) F = (long long)(mant << sh);
    else if (sh > -64) F = (long long)(mant >> (-sh));
  }
#pragma unroll
  for (int s = TC_SA - 1; s >= 1; --s) {
    int dd = (int)(F & 255);
    if (dd >= 128) dd -= 256;
    d[s] = dd;
    F = (F - dd) >> 8;
  }
  d[0] = (int)F;
  if (u >> 63) {
#pragma unroll
    for (int s = 0; s < TC_SA; ++s) d[s] = -d[s];
  }
}

// bf16 bits of d 2^(-8(s+1)) (exact: |d| <= 256 has at most 8 significant bits)
__device__ __forceinline__ unsigned short slice_bits(int d, int s) {
  const float f = (float)d * __int_as_float((127 - 8 * (s + 1)) << 23);
  return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}
// bf16 bits of a small integer d (|d| < 256)
__device__ __forceinline__ unsigned short int_bits(int d) {
  return __bfloat16_as_ushort(__float2bfloat16_rn((float)d));
}

// ---------------------------------------------------------------------------------------------
// Statistics and slicing kernels
// ---------------------------------------------------------------------------------------------

// Per vector v (nvec vectors of len doubles, stride len): maxbits[v] = bit pattern of max |x|,
// minlsb[v] = smallest exponent of a lowest set bit over the nonzero entries; *flag |= 1 on a
// NaN / Inf.  maxbits / minlsb must be initialised (0 / INT_MAX).
__global__ void vec_stats_kernel(const double *__restrict__ x, long long len, unsigned long long *maxbits,
                                 int *minlsb, int *flag) {
  const int v = blockIdx.y;
  const double *xv = x + (long long)v * len;
  unsigned long long mb = 0;
  int lsb = 0x7fffffff, bad = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(xv[i]) & 0x7fffffffffffffffull;
    const int be = (int)(u >> 52);
    if (be == 0x7ff) { bad = 1; continue; }
    if (u > mb) mb = u;
    if (be != 0) {
      const unsigned long long mant = (u & 0xfffffffffffffull) | (1ull << 52);
      lsb = min(lsb, be - 1075 + __ffsll((long long)mant) - 1);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mb = max(mb, (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)mb, o));
    lsb = min(lsb, __shfl_xor_sync(0xffffffffu, lsb, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (mb) atomicMax(&maxbits[v], mb);
    if (lsb != 0x7fffffff) atomicMin(&minlsb[v], lsb);
    if (bad) atomicOr(flag, 1);
  }
}

__global__ void stats_init_kernel(unsigned long long *maxbits, int *minlsb, int n, int *flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) { maxbits[i] = 0; minlsb[i] = 0x7fffffff; }
  if (i == 0) *flag = 0;
}

// Slices of the k deflation vectors as the left operand of G = E^dag X (rows q, K = real index m
// of L = 24 V reals): tile mt = q / 128, chunk c = m / 32, slice s at
//        Ag + mt * kcg * 7 * 8192 + (c * 7 + s) * rows8(mt) * 64 + tile_off(q % 128, m % 32)
// where rows8 is 128 except for the last tile (its valid rows rounded up to 8).  eexp[q] = the
// row's scale exponent.  One thread per (q, 8 consecutive reals).  Padding must be zero already.
__global__ void slice_ag_kernel(const double *__restrict__ E, int k, long long L, const unsigned long long *maxbits,
                                int kcg, unsigned short *__restrict__ Ag, int *eexp) {
  const int q = blockIdx.y;
  const long long m0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 8;
  if (m0 >= L) return;
  const int e = scale_exp(maxbits[q]);
  if (m0 == 0) eexp[q] = e;
  const double *src = E + (long long)q * L + m0;
  int dg[8][TC_SA];
#pragma unroll
  for (int j = 0; j < 8; ++j) split_digits(src[j], e, dg[j]);
  const int mt = q / TC_M, row = q % TC_M;
  const int r8 = min(TC_M, round8(k - mt * TC_M));
  const long long c = m0 / TC_KCH;
  unsigned char *base = (unsigned char *)Ag + (size_t)mt * kcg * TC_SA * TC_BLK;
#pragma unroll
  for (int s = 0; s < TC_SA; ++s) {
    uint4 w;
    w.x = slice_bits(dg[0][s], s) | ((unsigned)slice_bits(dg[1][s], s) << 16);
    w.y = slice_bits(dg[2][s], s) | ((unsigned)slice_bits(dg[3][s], s) << 16);
    w.z = slice_bits(dg[4][s], s) | ((unsigned)slice_bits(dg[5][s], s) << 16);
    w.w = slice_bits(dg[6][s], s) | ((unsigned)slice_bits(dg[7][s], s) << 16);
    *(uint4 *)(base + (size_t)(c * TC_SA + s) * r8 * (TC_KCH * 2) + tile_off(row, (int)(m0 % TC_KCH))) = w;
  }
}

// Row scale of the left operand of Y = E C: rowexp[m] = scale exponent of max_q |E_q[m]| for
// every real component m (one thread each); *flag |= 1 on a NaN / Inf.
__global__ void rowexp_kernel(const double *__restrict__ E, int k, long long L, int *rowexp, int *flag) {
  const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= L) return;
  unsigned long long mb = 0;
  for (int q = 0; q < k; ++q) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(E[(long long)q * L + m]) & 0x7fffffffffffffffull;
    if ((u >> 52) == 0x7ff) atomicOr(flag, 1);
    else if (u > mb) mb = u;
  }
  rowexp[m] = scale_exp(mb);
}

// Slices of E as the left operand of Y = E C (rows = real components m, K = vector index q, row
// scale rowexp[m]): tile mt = m / 128, chunk c = q / 32, slice s at
//        Ac + mt * kcc * 7 * 8192 + (c * 7 + s) * rows8(mt) * 64 + tile_off(m % 128, q % 32).
// One thread per (m, 8 consecutive q: one 16-byte core-matrix row).  Padding must be zero already.
__global__ void slice_ac_kernel(const double *__restrict__ E, int k, long long L, const int *rowexp, int kcc,
                                unsigned short *__restrict__ Ac) {
  const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int q0 = blockIdx.y * 8;
  if (m >= L || q0 >= k) return;
  const int e = rowexp[m];
  int dg[8][TC_SA];
#pragma unroll
  for (int j = 0; j < 8; ++j) split_digits(q0 + j < k ? E[(long long)(q0 + j) * L + m] : 0.0, e, dg[j]);
  const long long mt = m / TC_M;
  const int r8 = (int)min((long long)TC_M, (long long)round8((int)min(L - mt * TC_M, (long long)TC_M)));
  const int c = q0 / TC_KCH;
  unsigned char *base = (unsigned char *)Ac + (size_t)mt * kcc * TC_SA * TC_BLK;
#pragma unroll
  for (int s = 0; s < TC_SA; ++s) {
    uint4 w;
    w.x = slice_bits(dg[0][s], s) | ((unsigned)slice_bits(dg[1][s], s) << 16);
    w.y = slice_bits(dg[2][s], s) | ((unsigned)slice_bits(dg[3][s], s) << 16);
    w.z = slice_bits(dg[4][s], s) | ((unsigned)slice_bits(dg[5][s], s) << 16);
    w.w = slice_bits(dg[6][s], s) | ((unsigned)slice_bits(dg[7][s], s) << 16);
    *(uint4 *)(base + (size_t)(c * TC_SA + s) * r8 * (TC_KCH * 2) + tile_off((int)(m % TC_M), q0 % TC_KCH)) = w;
  }
}

// Right operand of G = E^dag X: column n = 2r is field r of X read as L reals, column 2r + 1 is
// i conj-rotated field r (entries (Im, -Re) per complex number), so that the real products give
// Re and Im of conj(E) . X.  small != 0: one exact slice x 2^-lsb[r] (integers below 256);
// otherwise seven slices with the column scale.  colexp[r] receives the exponent to undo.
// Layout: B + (c * SB + t) * NP * 64 + tile_off(n, m % 32).  One thread per (r, 8 reals), writing
// both columns of r; integer arithmetic only.
__device__ __forceinline__ int small_digit(double x, int e) {
  // x = +-mant 2^(be - 1075) is an integer multiple of 2^e below 2^(e + 8): shift the significand
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int be = (int)((u >> 52) & 0x7ff);
  if (be == 0) return 0;
  const unsigned long long mant = (u & 0xfffffffffffffull) | (1ull << 52);
  const int sh = be - 1075 - e;
  const int d = sh >= 0 ? (int)(mant << sh) : (sh > -64 ? (int)(mant >> (-sh)) : 0);
  return (u >> 63) ? -d : d;
}
__device__ __forceinline__ uint4 pack8(const unsigned short h[8]) {
  uint4 w;
  w.x = h[0] | ((unsigned)h[1] << 16);
  w.y = h[2] | ((unsigned)h[3] << 16);
  w.z = h[4] | ((unsigned)h[5] << 16);
  w.w = h[6] | ((unsigned)h[7] << 16);
  return w;
}
__global__ void slice_x_kernel(const double *__restrict__ X, int nrhs, long long L, const unsigned long long *maxbits,
                               const int *minlsb, int small, int SB, int NP, unsigned short *__restrict__ B,
                               int *colexp) {
  const int r = blockIdx.y;
  const long long m0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 8;
  if (m0 >= L || r >= nrhs) return;
  const int e = small ? (maxbits[r] ? minlsb[r] : 0) : scale_exp(maxbits[r]);
  if (m0 == 0) colexp[r] = e;
  const double *src = X + (long long)r * L + m0;
  double v[2][8];
#pragma unroll
  for (int j = 0; j < 8; j += 2) {
    const double re = src[j], im = src[j + 1];
    v[0][j] = re; v[0][j + 1] = im;     // column 2r
    v[1][j] = im; v[1][j + 1] = -re;    // column 2r + 1
  }
  const long long c = m0 / TC_KCH;
  unsigned char *base = (unsigned char *)B + (size_t)c * SB * NP * (TC_KCH * 2);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    unsigned char *row = base + tile_off(2 * r + h, (int)(m0 % TC_KCH));
    if (small) {
      unsigned short b[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) b[j] = int_bits(small_digit(v[h][j], e));
      *(uint4 *)row = pack8(b);
    } else {
      int dg[8][TC_SA];
#pragma unroll
      for (int j = 0; j < 8; ++j) split_digits(v[h][j], e, dg[j]);
#pragma unroll
      for (int s = 0; s < TC_SA; ++s) {
        unsigned short b[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) b[j] = slice_bits(dg[j][s], s);
        *(uint4 *)(row + (size_t)s * NP * (TC_KCH * 2)) = pack8(b);
      }
    }
  }
}

// Right operand of Y = E C: row q of the reduction carries d_q C[q][r], column n = 2r its real
// part and 2r + 1 its imaginary part, seven slices per column with the column scale colexp[n].
// d may be NULL (all ones).  One block per r.
// Layout: B + (c * 7 + t) * NP * 64 + tile_off(n, q % 32), c = q / 32.
__global__ void slice_c_kernel(const double2 *__restrict__ Cm, const double2 *__restrict__ d, int k,
                               int ldc, int NP, unsigned short *__restrict__ B, int *colexp) {
  const int r = blockIdx.x;
  __shared__ unsigned long long smax[2];
  if (threadIdx.x < 2) smax[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long m0 = 0, m1 = 0;
  for (int q = threadIdx.x; q < k; q += blockDim.x) {
    double2 c = Cm[(size_t)q * ldc + r];
    if (d) c = cmul(d[q], c);
    const double re = c.x, im = c.y;
    m0 = max(m0, (unsigned long long)__double_as_longlong(fabs(re)));
    m1 = max(m1, (unsigned long long)__double_as_longlong(fabs(im)));
  }
  atomicMax(&smax[0], m0);
  atomicMax(&smax[1], m1);
  __syncthreads();
  const int e0 = scale_exp(smax[0]), e1 = scale_exp(smax[1]);
  if (threadIdx.x == 0) { colexp[2 * r] = e0; colexp[2 * r + 1] = e1; }
  for (int q = threadIdx.x; q < k; q += blockDim.x) {
    double2 c = Cm[(size_t)q * ldc + r];
    if (d) c = cmul(d[q], c);
    const double re = c.x, im = c.y;
    int d0[TC_SA], d1[TC_SA];
    split_digits(re, e0, d0);
    split_digits(im, e1, d1);
    const int c32 = q / TC_KCH, kk = q % TC_KCH;
#pragma unroll
    for (int t = 0; t < TC_SA; ++t) {
      unsigned char *blk = (unsigned char *)B + (size_t)(c32 * TC_SA + t) * NP * (TC_KCH * 2);
      *(unsigned short *)(blk + tile_off(2 * r, kk)) = slice_bits(d0[t], t);
      *(unsigned short *)(blk + tile_off(2 * r + 1, kk)) = slice_bits(d1[t], t);
    }
  }
}

// G[q * ldg + r] = 2^(eexp[q] + colexp[r]) sum over splits of the two partial columns, r < nb
__global__ void vhx_reduce_kernel(const double *__restrict__ part, int nsplit, int NP, long long Mtot, int k, int nb,
                                  const int *eexp, const int *colexp, double2 *G, int ldg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k * nb) return;
  const int q = i / nb, r = i % nb;
  double re = 0.0, im = 0.0;
  for (int sp = 0; sp < nsplit; ++sp) {
    re += part[((size_t)sp * NP + 2 * r) * Mtot + q];
    im += part[((size_t)sp * NP + 2 * r + 1) * Mtot + q];
  }
  const int e = eexp[q] + colexp[r];
  G[(size_t)q * ldg + r] = make_double2(scalbn(re, e), scalbn(im, e));
}

// ---------------------------------------------------------------------------------------------
// PTX wrappers (tcgen05, TMEM, bulk copies, mbarriers)
// ---------------------------------------------------------------------------------------------

// x 2^e: one multiplication by a power of two built from its bits (scalbn outside the normal range)
__device__ __forceinline__ double mul_pow2(double x, int e) {
  if (e >= -1022 && e <= 1023) return x * __longlong_as_double((long long)(e + 1023) << 52);
  return scalbn(x, e);
}

// (T 2^-(8 (TC_NEXACT - 1) + unit_shift) + tail) 2^e for the exact integer part T and the FP32
// tail: both power-of-two scales are applied exactly before one conversion and one FMA; outside
// the normal ranges the slower general form is used
__device__ __forceinline__ double fold_scaled(long long T, float tail, int e, int unit_shift) {
  const int e1 = e - 8 * (TC_NEXACT - 1) - unit_shift;
  if (e1 >= -1022 && e1 <= 1023 && e >= -126 && e <= 127) {
    const double s1 = __longlong_as_double((long long)(e1 + 1023) << 52);
    const float tf = tail * __int_as_float((e + 127) << 23);
    return fma((double)T, s1, (double)tf);
  }
  const double unitx = __longlong_as_double((long long)(1023 - 8 * (TC_NEXACT - 1) - unit_shift) << 52);
  return mul_pow2((double)T * unitx + (double)tail, e);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase of the given parity; false if the CTA aborted or the wait ran out of time
// (after wait_ns; then the abort flag and the device error flag are set).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, int *err,
                                          unsigned long long wait_ns) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  for (unsigned it = 1;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255) == 0) {
      if (*abort_flag) return false;
      if (gtimer() - t0 > wait_ns) {
        *abort_flag = 1;
        atomicExch(err, (int)LQCD_ERR_TIMEOUT);
        return false;
      }
    }
  }
}
// bounded wait used only while draining after an abort (its own fixed bound, independent of the
// configurable one, so that copies and MMAs in flight always land before the CTA exits)
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = gtimer();
  while (!mbar_try(bar, parity) && gtimer() - t0 < TC_WAIT_NS) {
  }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: no swizzle, K-direction core-matrix stride 128 B (leading
// byte offset), row-group stride 512 B (stride byte offset), descriptor version 1 (bits 46-47).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3ffff) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B bf16 (bits 7-9,
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ __forceinline__ uint32_t mma_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// zero 8 consecutive TMEM columns of the warp's 32 lanes
__device__ __forceinline__ void tmem_zero8(uint32_t taddr) {
  const uint32_t z = 0;
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr), "r"(z)
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------------------------------------
// The tcgen05 GEMM
// ---------------------------------------------------------------------------------------------

struct TcArgs {
  const unsigned char *A;  // row-scaled operand, pre-tiled (see slice_ag_kernel, slice_ac_kernel)
  const unsigned char *B;  // column operand, pre-tiled [chunk][slice][NP x 32]
  int mt_count;            // row tiles
  int m_valid;             // valid rows (rows >= m_valid are neither loaded from HBM nor written)
  int kc_count;            // K chunks of 32
  int ksplit;              // K splits per row tile (work items = mt_count * ksplit)
  int kcr;                 // chunks per accumulator read-out (keeps the exact groups within 2^24 units)
  int unit_shift;          // exact group g holds integers in units of 2^-(8 g + unit_shift)
  double *part;            // mode 0: part[(split * NP + n) * Mtot + m]
  long long Mtot;
  const int *colexp;       // mode 1: scale exponent per column
  const int *rowexp;       // mode 1: scale exponent per row
  int nb;                  // mode 1: complex columns (column 2r real part, 2r + 1 imaginary part)
  double *out;             // mode 1: out[r * m_valid + m]
  int *err;
  unsigned long long wait_ns;  // bound of every pipeline wait (the context's setting)
  int stop_after;          // failure injection: the loader stops after this many chunks (-1: never)
};

__host__ __device__ constexpr int tc_stage_bytes(int SB, int NP) { return TC_SA * TC_BLK + SB * NP * TC_KCH * 2; }
__host__ __device__ constexpr int tc_nbuf(int NP) { return 2 * TC_NGRP * NP <= 512 ? 2 : 1; }
// TMEM columns to allocate: a power of two >= 32 holding every accumulator set
__host__ __device__ constexpr uint32_t tc_tmem_cols(int NP) {
  return tc_nbuf(NP) * TC_NGRP * NP <= 32    ? 32u
         : tc_nbuf(NP) * TC_NGRP * NP <= 64  ? 64u
         : tc_nbuf(NP) * TC_NGRP * NP <= 128 ? 128u
         : tc_nbuf(NP) * TC_NGRP * NP <= 256 ? 256u
                                             : 512u;
}
// right slices per MMA: N = slices x NP <= 256
__host__ __device__ constexpr int tc_tch(int NP) { return 256 / NP < TC_SA ? 256 / NP : TC_SA; }

__device__ __forceinline__ void work_range(const TcArgs &p, int w, int &mt, int &sp, int &c0, int &c1) {
  mt = w / p.ksplit;
  sp = w % p.ksplit;
  c0 = (int)((long long)p.kc_count * sp / p.ksplit);
  c1 = (int)((long long)p.kc_count * (sp + 1) / p.ksplit);
}

// MODE 0: partial sums of G = E^dag X; MODE 1: fields of Y = E C (see TcArgs)
template <int NP, int SB, int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm_kernel(const __grid_constant__ TcArgs p, int stages) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int sbytes = tc_stage_bytes(SB, NP);
  unsigned long long *bars = (unsigned long long *)(smem + (size_t)stages * sbytes);
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * stages, accf0 = full0 + 16 * stages,
                 acce0 = accf0 + 16, drain = acce0 + 16;
  uint32_t *tmem_slot = (uint32_t *)(bars + 2 * stages + 5);
  volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NBUF = tc_nbuf(NP);
  constexpr uint32_t NCOLS = tc_tmem_cols(NP);
  const int nwork = p.mt_count * p.ksplit;

  // stage buffers start as zeros: rows that a partial tile does not load then hold finite values
  for (int i = threadIdx.x; i < stages * sbytes / 16; i += TC_THREADS) ((uint4 *)smem)[i] = make_uint4(0, 0, 0, 0);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, TC_EPI_WARPS * 32);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // every accumulator column starts at zero: the MMAs only ever accumulate
  if (warp < TC_EPI_WARPS) {
    const uint32_t tq = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    for (int c = (warp >> 2) * 8; c < NBUF * TC_NGRP * NP; c += 16) tmem_zero8(tq + (uint32_t)c);
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (warp == TC_EPI_WARPS) {
    // ---- loader ----
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t filled = 0;  // stages armed at least once (for the drain after an abort)
      constexpr uint32_t bbytes = (uint32_t)(SB * NP * TC_KCH * 2);
      bool ok = true;
      int narmed = 0;
      for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
        int mt, sp, c0, c1;
        work_range(p, w, mt, sp, c0, c1);
        const int r8 = min(TC_M, round8(p.m_valid - mt * TC_M));
        const uint32_t ablk = (uint32_t)(r8 * TC_KCH * 2);
        const unsigned char *abase = p.A + (size_t)mt * p.kc_count * TC_SA * TC_BLK;
        (void)sp;
        for (int c = c0; c < c1; ++c) {
          // injected stall: stop arming stages, so the MMA warp waits on one that nothing fills
          if (narmed == p.stop_after) { ok = false; break; }
          if (!mbar_wait(empty0 + 8 * stage, phase ^ 1, abort_flag, p.err, p.wait_ns)) { ok = false; break; }
          const uint32_t sA = smem_u32(smem + (size_t)stage * sbytes);
          mbar_expect_tx(full0 + 8 * stage, TC_SA * ablk + bbytes);
          bulk_g2s(sA, abase + (size_t)c * TC_SA * ablk, TC_SA * ablk, full0 + 8 * stage);
          bulk_g2s(sA + TC_SA * TC_BLK, p.B + (size_t)c * bbytes, bbytes, full0 + 8 * stage);
          filled |= 1u << stage;
          ++narmed;
          if (++stage == stages) { stage = 0; phase ^= 1; }
        }
      }
      if (!ok) {
        // let every armed copy land before the CTA exits: stage s was last armed in the lap
        // before the current position if s >= stage, else in the current lap
        for (int s = 0; s < stages; ++s)
          if (filled >> s & 1) mbar_drain(full0 + 8 * s, s < stage ? phase : phase ^ 1);
      }
    }
  } else if (warp == TC_EPI_WARPS + 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      int stage = 0, buf = 0;
      uint32_t phase = 0, accph[2] = {0, 0};
      bool ok = true, issued = false;
      for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
        int mt, sp, c0, c1;
        work_range(p, w, mt, sp, c0, c1);
        const int r8 = min(TC_M, round8(p.m_valid - mt * TC_M));
        const uint32_t ablk = (uint32_t)(r8 * TC_KCH * 2);
        for (int g0 = c0; g0 < c1 && ok; g0 += p.kcr) {
          const int g1 = min(c1, g0 + p.kcr);
          if (!mbar_wait(acce0 + 8 * buf, accph[buf] ^ 1, abort_flag, p.err, p.wait_ns)) { ok = false; break; }
          tc_fence_after();
          const uint32_t dbase = tmem + (uint32_t)(buf * TC_NGRP * NP);
          for (int c = g0; c < g1; ++c) {
            if (!mbar_wait(full0 + 8 * stage, phase, abort_flag, p.err, p.wait_ns)) { ok = false; break; }
            tc_fence_after();
            const uint32_t sA = smem_u32(smem + (size_t)stage * sbytes), sB = sA + TC_SA * TC_BLK;
            // descriptors of the stage's first K step; later operands differ only in the start
            // address field (bits 0-13, units of 16 bytes)
            const uint64_t a0 = smem_desc(sA), b0 = smem_desc(sB);
            const uint32_t ab16 = ablk >> 4;
#pragma unroll
            for (int j = 0; j < TC_KCH / 16; ++j) {
#pragma unroll
              for (int sl = 0; sl < TC_SA; ++sl) {
                // right slices t with sl + t <= 7, in MMAs of at most tc_tch(NP) stacked slices
                constexpr int TCH = tc_tch(NP);
                const int tmax = (SB - 1 < TC_NGRP - 1 - sl) ? SB - 1 : TC_NGRP - 1 - sl;
#pragma unroll
                for (int t0 = 0; t0 <= tmax; t0 += TCH) {
                  const int t1 = (t0 + TCH - 1 < tmax) ? t0 + TCH - 1 : tmax;
                  mma_bf16(dbase + (uint32_t)((sl + t0) * NP),
                           a0 + (uint64_t)(sl * ab16 + 16 * j),
                           b0 + (uint64_t)(t0 * (NP * TC_KCH * 2 / 16) + 16 * j),
                           mma_idesc((t1 - t0 + 1) * NP), 1u);
                }
              }
            }
            issued = true;
            mma_commit(empty0 + 8 * stage);
            if (++stage == stages) { stage = 0; phase ^= 1; }
          }
          if (!ok) break;
          mma_commit(accf0 + 8 * buf);
          accph[buf] ^= 1;
          buf ^= NBUF - 1;
        }
      }
      if (!ok && issued) {
        mma_commit(drain);
        mbar_drain(drain, 0);
      }
    }
  } else {
    // ---- epilogue: warps 0-7; thread = TMEM lane = output row, half of the columns per warp ----
    constexpr int NH = NP / 2;                   // columns of this warp
    const int quad = warp & 3, half = warp >> 2;
    const int row = quad * 32 + lane;
    const int cb = half * NH;                    // first column of this warp
    int buf = 0;
    uint32_t accph[2] = {0, 0};
    bool ok = true;
    const float sc0 = __int_as_float((127 + p.unit_shift) << 23);       // 2^unit_shift
    // unit of the last exact group: 2^-(8 (TC_NEXACT - 1) + unit_shift)
    const double unitx = __longlong_as_double((long long)(1023 - 8 * (TC_NEXACT - 1) - p.unit_shift) << 52);
    int ce[NH];                                  // column scale exponents (mode 1)
#pragma unroll
    for (int j = 0; j < NH; ++j) ce[j] = (MODE == 1 && cb + j < 2 * p.nb) ? p.colexp[cb + j] : 0;
    for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
      int mt, sp, c0, c1;
      work_range(p, w, mt, sp, c0, c1);
      const long long m = (long long)mt * TC_M + row;
      const int rexp = (MODE == 1 && m < p.m_valid) ? p.rowexp[m] : 0;   // issued before the waits
      // MODE 0 folds every read-out into FP64; MODE 1 (a few read-outs per tile, bounded on the
      // host) keeps the exact part as a 64-bit integer and the FP32 tail until the final write
      double acc[MODE == 0 ? NH : 1];
      long long Ti[MODE == 1 ? NH : 1];
      float tl[MODE == 1 ? NH : 1];
#pragma unroll
      for (int j = 0; j < NH; ++j) {
        if constexpr (MODE == 0) acc[j] = 0.0;
        else { Ti[j] = 0; tl[j] = 0.f; }
      }
      for (int g0 = c0; g0 < c1; g0 += p.kcr) {
        // the whole warp leaves together (tcgen05.ld and the shuffles below are warp-collective)
        if (!__all_sync(0xffffffffu, mbar_wait(accf0 + 8 * buf, accph[buf], abort_flag, p.err, p.wait_ns))) {
          ok = false;
          break;
        }
        accph[buf] ^= 1;
        tc_fence_after();
        const uint32_t tb = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * TC_NGRP * NP + cb);
#pragma unroll
        for (int n0 = 0; n0 < NH; n0 += 8) {
          float v[TC_NGRP][8];
#pragma unroll
          for (int a = 0; a < TC_NGRP; ++a) tmem_ld8(tb + (uint32_t)(a * NP + n0), v[a]);
          tmem_wait_ld();
#pragma unroll
          for (int a = 0; a < TC_NGRP; ++a) tmem_zero8(tb + (uint32_t)(a * NP + n0));   // ready for reuse
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            // exact groups: integers n_g = v_g 2^(8 g + unit_shift) of at most 2^24, combined
            // exactly into T = sum_g n_g 2^(8 (4 - g)) < 2^57
            long long T = 0;
            float sc = sc0;
#pragma unroll
            for (int g = 0; g < TC_NEXACT; ++g) {
              T = T * 256 + (long long)__float2int_rn(v[g][i] * sc);
              sc *= 256.0f;
            }
            const float tail = (v[7][i] + v[6][i]) + v[5][i];
            if constexpr (MODE == 0) acc[n0 + i] += (double)T * unitx + (double)tail;
            else { Ti[n0 + i] += T; tl[n0 + i] += tail; }
          }
        }
        tmem_wait_st();
        tc_fence_before();
        mbar_arrive(acce0 + 8 * buf);
        buf ^= NBUF - 1;
      }
      if (!ok) break;
      if constexpr (MODE == 0) {
        if (m < p.m_valid) {
#pragma unroll
          for (int j = 0; j < NH; ++j) p.part[((size_t)sp * NP + cb + j) * p.Mtot + m] = acc[j];
        }
      } else {
        // rows 2i (real part) and 2i + 1 (imaginary part) of a complex entry are lanes 2i, 2i + 1;
        // column pair (2r, 2r + 1) holds the real and imaginary parts of coefficient column r
#pragma unroll
        for (int j = 0; j < NH; j += 2) {
          const int r = (cb + j) >> 1;
          const double p1 = r < p.nb ? fold_scaled(Ti[j], tl[j], rexp + ce[j], p.unit_shift) : 0.0;
          const double p2 = r < p.nb ? fold_scaled(Ti[j + 1], tl[j + 1], rexp + ce[j + 1], p.unit_shift) : 0.0;
          const double p2o = __shfl_xor_sync(0xffffffffu, p2, 1);
          if (r < p.nb && m < p.m_valid) p.out[(size_t)r * p.m_valid + m] = (row & 1) ? p2o + p1 : p1 - p2o;
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS) : "memory");
}

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------

struct TcSlices {
  int k;
  long long L;                 // reals per vector (24 V)
  int mtg, kcg;                // G = E^dag X operand: row tiles over q, K chunks over the reals
  int mtc, kcc;                // Y = E C operand: row tiles over the reals, K chunks over q
  unsigned char *Ag, *Ac;      // pre-tiled slices
  int *eexp;                   // per-vector scale exponent (device)
  int *rowexp;                 // per-real-component scale exponent of the Y = E C operand (device)
  unsigned long long *maxbits; // per-vector maximum (device)
  int *minlsb, *flag;
};

size_t tc_bytes_g(int k, long long L) {
  const int mt = (k + TC_M - 1) / TC_M;
  const long long kc = (L + TC_KCH - 1) / TC_KCH;
  return (size_t)mt * kc * TC_SA * TC_BLK;
}
size_t tc_bytes_c(int k, long long L) {
  const long long mt = (L + TC_M - 1) / TC_M;
  const int kc = (k + TC_KCH - 1) / TC_KCH;
  return (size_t)mt * kc * TC_SA * TC_BLK;
}

template <int NP, int SB, int MODE> lqcd_status tc_gemm_launch(lqcd_ctx *ctx, const TcArgs &args, double units) {
  TcArgs a = args;
  a.wait_ns = ctx->tc_wait_ns;
  a.stop_after = ctx->tc_stop_after;
  ctx->tc_stop_after = -1;  // the injection is one-shot
  constexpr int sbytes = tc_stage_bytes(SB, NP);
  const int bar_bytes = 8 * (2 * 4 + 8) + 64;  // room for up to 4 stages of barriers + slot + flag
  int stages = std::min(4, (TC_SMEM_MAX - bar_bytes - 64) / sbytes);
  if (stages < 2) return set_err(ctx, LQCD_ERR_INVALID_ARG, "tensor-core contraction: stage does not fit");
  const int smem = std::max(TC_SMEM_MIN, stages * sbytes + 8 * (2 * stages + 5) + 64);
  LQCD_CUDA(ctx, cudaFuncSetAttribute(tc_gemm_kernel<NP, SB, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int nwork = a.mt_count * a.ksplit;
  const int grid = std::min(nwork, ctx->sms);
  kbegin(ctx);
  tc_gemm_kernel<NP, SB, MODE><<<grid, TC_THREADS, smem, ctx->stream>>>(a, stages);
  return launch_check(ctx, "tc_gemm_kernel", K_TENSOR, units);
}

// MODE 0 (G = E^dag X partial sums) with SB = 1 (small-integer right operand) or 7 slices;
// MODE 1 (Y = E C fields) with SB = 7
lqcd_status tc_gemm(lqcd_ctx *ctx, int NP, int SB, int mode, const TcArgs &a, double units) {
#define TC_NP_CASES(SBV, MV)                                              \
  switch (NP) {                                                           \
    case 16: return tc_gemm_launch<16, SBV, MV>(ctx, a, units);          \
    case 32: return tc_gemm_launch<32, SBV, MV>(ctx, a, units);          \
    case 48: return tc_gemm_launch<48, SBV, MV>(ctx, a, units);          \
    case 64: return tc_gemm_launch<64, SBV, MV>(ctx, a, units);          \
  }
  if (mode == 0 && SB == 1) TC_NP_CASES(1, 0)
  if (mode == 0 && SB == TC_SA) TC_NP_CASES(TC_SA, 0)
  if (mode == 1 && SB == TC_SA) TC_NP_CASES(TC_SA, 1)
#undef TC_NP_CASES
  return set_err(ctx, LQCD_ERR_INVALID_ARG, "tensor-core contraction: bad shape NP %d SB %d mode %d", NP, SB, mode);
}

// chunks per read-out such that an exact group (at most P pairs of products of at most dA * dB
// units each) stays within 2^24 units: kcr * 32 * P * dA * dB <= 2^24
int tc_kcr(int SB, double dB) {
  const double P = std::min(TC_NEXACT, SB);
  const double kc = std::floor(16777216.0 / (P * 128.0 * dB * TC_KCH));
  return (int)std::max(1.0, std::min(kc, 1e6));
}

lqcd_status tc_slices_fill(lqcd_ctx *ctx, const double2 *E, TcSlices *S, size_t bg, size_t bc);

lqcd_status check_flag(lqcd_ctx *ctx, int *flag_dev, const char *what) {
  int f = 0;
  LQCD_CUDA(ctx, cudaMemcpyAsync(&f, flag_dev, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (f == LQCD_ERR_TIMEOUT) return set_err(ctx, LQCD_ERR_TIMEOUT, "%s: a tensor-core pipeline wait timed out", what);
  if (f) return set_err(ctx, LQCD_ERR_NONFINITE, "%s: non-finite input", what);
  return LQCD_OK;
}

}  // namespace

// Slices of the k vectors E (device, k x N complex, vector-major) for both contractions; the
// buffers are allocated here and released by tc_slices_free.
lqcd_status tc_slices_make(lqcd_ctx *ctx, const double2 *E, int k, void **out) {
  *out = nullptr;
  if (k <= 0 || k > 4096) return set_err(ctx, LQCD_ERR_INVALID_ARG, "tensor-core slices: 1 <= k <= 4096");
  TcSlices *S = new TcSlices();
  S->k = k;
  S->L = 2 * ctx->N;
  S->mtg = (k + TC_M - 1) / TC_M;
  S->kcg = (int)((S->L + TC_KCH - 1) / TC_KCH);
  S->mtc = (int)((S->L + TC_M - 1) / TC_M);
  S->kcc = (k + TC_KCH - 1) / TC_KCH;
  const size_t bg = tc_bytes_g(k, S->L), bc = tc_bytes_c(k, S->L);
  cudaError_t e1 = cudaMalloc(&S->Ag, bg), e2 = cudaMalloc(&S->Ac, bc);
  cudaError_t e3 = cudaMalloc(&S->eexp, sizeof(int) * (k + 2) + sizeof(unsigned long long) * k + sizeof(int) * (k + 1));
  cudaError_t e4 = cudaMalloc(&S->rowexp, sizeof(int) * S->L);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess) {
    cudaGetLastError();
    if (e1 == cudaSuccess) cudaFree(S->Ag);
    if (e2 == cudaSuccess) cudaFree(S->Ac);
    if (e3 == cudaSuccess) cudaFree(S->eexp);
    if (e4 == cudaSuccess) cudaFree(S->rowexp);
    delete S;
    return set_err(ctx, LQCD_ERR_OOM, "tensor-core slices: %.1f GB not available", (bg + bc) / 1e9);
  }
  S->maxbits = (unsigned long long *)(S->eexp + k + (k & 1));
  S->minlsb = (int *)(S->maxbits + k);
  S->flag = S->minlsb + k;
  // the object is handed out only once every slice is written: a failure (non-finite input, CUDA
  // error) releases it, so a deflation object never keeps half-built slices
  const lqcd_status st = tc_slices_fill(ctx, E, S, bg, bc);
  if (st != LQCD_OK) {
    tc_slices_free(S);  // cudaFree waits for the kernels still using the buffers
    return st;
  }
  *out = S;
  return LQCD_OK;
}

namespace {
lqcd_status tc_slices_fill(lqcd_ctx *ctx, const double2 *E, TcSlices *S, size_t bg, size_t bc) {
  const int k = S->k;
  LQCD_CUDA(ctx, cudaMemsetAsync(S->Ag, 0, bg, ctx->stream));
  LQCD_CUDA(ctx, cudaMemsetAsync(S->Ac, 0, bc, ctx->stream));
  kbegin(ctx);
  stats_init_kernel<<<ceil_div(k, 256), 256, 0, ctx->stream>>>(S->maxbits, S->minlsb, k, S->flag);
  LQCD_TRY(launch_check(ctx, "stats_init_kernel", K_SLICE, (double)k));
  kbegin(ctx);
  vec_stats_kernel<<<dim3(std::min(ceil_div(S->L, 256), 64), k), 256, 0, ctx->stream>>>((const double *)E, S->L,
                                                                                           S->maxbits, S->minlsb, S->flag);
  LQCD_TRY(launch_check(ctx, "vec_stats_kernel", K_SLICE, (double)k * S->L));
  LQCD_TRY(check_flag(ctx, S->flag, "tensor-core slices"));
  kbegin(ctx);
  rowexp_kernel<<<ceil_div(S->L, 256), 256, 0, ctx->stream>>>((const double *)E, k, S->L, S->rowexp, S->flag);
  LQCD_TRY(launch_check(ctx, "rowexp_kernel", K_SLICE, (double)k * S->L));
  LQCD_TRY(check_flag(ctx, S->flag, "tensor-core slices"));
  kbegin(ctx);
  slice_ag_kernel<<<dim3(ceil_div(S->L / 8, 128), k), 128, 0, ctx->stream>>>(
      (const double *)E, k, S->L, S->maxbits, S->kcg, (unsigned short *)S->Ag, S->eexp);
  LQCD_TRY(launch_check(ctx, "slice_ag_kernel", K_SLICE, (double)k * S->L));
  kbegin(ctx);
  slice_ac_kernel<<<dim3(ceil_div(S->L, 128), S->kcc * (TC_KCH / 8)), 128, 0, ctx->stream>>>(
      (const double *)E, k, S->L, S->rowexp, S->kcc, (unsigned short *)S->Ac);
  return launch_check(ctx, "slice_ac_kernel", K_SLICE, (double)k * S->L);
}
}  // namespace

void tc_slices_free(void *p) {
  TcSlices *S = (TcSlices *)p;
  if (!S) return;
  cudaFree(S->Ag);
  cudaFree(S->Ac);
  cudaFree(S->eexp);
  cudaFree(S->rowexp);
  delete S;
}

// G[q * nrhs + r] = <E_q, X_r> (device output, k x nrhs complex)
lqcd_status tc_vhx(lqcd_ctx *ctx, const void *slices, const double2 *X, int nrhs, double2 *G) {
  const TcSlices *S = (const TcSlices *)slices;
  const int k = S->k;
  for (int r0 = 0; r0 < nrhs; r0 += 32) {
    const int nb = std::min(32, nrhs - r0);
    const int NP = std::max(16, ((2 * nb + 15) / 16) * 16);
    const double2 *Xb = X + (size_t)r0 * ctx->N;
    unsigned long long *mb;
    int *lsb, *flag, *colexp;
    unsigned char *Bsl;
    double *part;
    void *p;
    LQCD_TRY(ws_get(ctx, WS_TC_STAT, 64 * (sizeof(unsigned long long) + 2 * sizeof(int)) + 64, &p));
    mb = (unsigned long long *)p;
    lsb = (int *)(mb + 64);
    colexp = lsb + 64;
    flag = colexp + 64;
    kbegin(ctx);
    stats_init_kernel<<<1, 64, 0, ctx->stream>>>(mb, lsb, 64, flag);
    LQCD_TRY(launch_check(ctx, "stats_init_kernel", K_SLICE, 64.0));
    kbegin(ctx);
    vec_stats_kernel<<<dim3(std::min(ceil_div(S->L, 256), 64), nb), 256, 0, ctx->stream>>>((const double *)Xb, S->L,
                                                                                              mb, lsb, flag);
    LQCD_TRY(launch_check(ctx, "vec_stats_kernel", K_SLICE, (double)nb * S->L));
    // the read-out schedule depends on the operand's value range: read it back
    std::vector<unsigned long long> hmb(nb);
    std::vector<int> hl(nb);
    int hflag = 0;
    LQCD_CUDA(ctx, cudaMemcpyAsync(hmb.data(), mb, sizeof(unsigned long long) * nb, cudaMemcpyDeviceToHost, ctx->stream));
    LQCD_CUDA(ctx, cudaMemcpyAsync(hl.data(), lsb, sizeof(int) * nb, cudaMemcpyDeviceToHost, ctx->stream));
    LQCD_CUDA(ctx, cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (hflag) return set_err(ctx, LQCD_ERR_NONFINITE, "tensor-core V^dag X: non-finite input");
    // small-integer operand: every column is integers below 256 times one power of two
    bool small = true;
    int span = 0;
    for (int r = 0; r < nb; ++r) {
      if (!hmb[r]) continue;
      const int mexp = (int)((hmb[r] >> 52) & 0x7ff) - 1023;
      span = std::max(span, mexp - hl[r]);
      if (mexp - hl[r] > 7) small = false;
    }
    TcArgs a{};
    const int SB = small ? 1 : TC_SA;
    const double dB = small ? std::ldexp(1.0, span + 1) : 128.0;
    a.kcr = tc_kcr(SB, dB);
    a.unit_shift = small ? 8 : 16;
    const size_t bbytes = (size_t)S->kcg * SB * NP * TC_KCH * 2;
    LQCD_TRY(ws_get(ctx, WS_TC_B, bbytes, &p));
    Bsl = (unsigned char *)p;
    LQCD_CUDA(ctx, cudaMemsetAsync(Bsl, 0, bbytes, ctx->stream));
    kbegin(ctx);
    slice_x_kernel<<<dim3(ceil_div(S->L / 8, 128), nb), 128, 0, ctx->stream>>>(
        (const double *)Xb, nb, S->L, mb, lsb, small ? 1 : 0, SB, NP, (unsigned short *)Bsl, colexp);
    LQCD_TRY(launch_check(ctx, "slice_x_kernel", K_SLICE, (double)nb * S->L));
    a.A = S->Ag;
    a.B = Bsl;
    a.mt_count = S->mtg;
    a.m_valid = k;
    a.kc_count = S->kcg;
    a.ksplit = std::max(1, std::min(S->kcg, ctx->sms / S->mtg));
    a.Mtot = (long long)S->mtg * TC_M;
    LQCD_TRY(ws_get(ctx, WS_TC_PART, sizeof(double) * (size_t)a.ksplit * NP * a.Mtot + 64, &p));
    part = (double *)p;
    a.part = part;
    a.err = flag;
    LQCD_TRY(tc_gemm(ctx, NP, SB, 0, a, (double)k * nb * ctx->N));
    kbegin(ctx);
    vhx_reduce_kernel<<<ceil_div(k * nb, 128), 128, 0, ctx->stream>>>(part, a.ksplit, NP, a.Mtot, k, nb, S->eexp,
                                                                       colexp, G + r0, nrhs);
    LQCD_TRY(launch_check(ctx, "vhx_reduce_kernel", K_SLICE, (double)k * nb));
    LQCD_TRY(check_flag(ctx, flag, "tensor-core V^dag X"));
  }
  return LQCD_OK;
}

// Y_r = sum_q E_q d_q C[q * nrhs + r] (device in / out; d: device k complex or NULL)
lqcd_status tc_vc(lqcd_ctx *ctx, const void *slices, const double2 *Cm, const double2 *d, int nrhs, double2 *Y) {
  const TcSlices *S = (const TcSlices *)slices;
  const int k = S->k;
  for (int r0 = 0; r0 < nrhs; r0 += 32) {
    const int nb = std::min(32, nrhs - r0);
    const int NP = std::max(16, ((2 * nb + 15) / 16) * 16);
    void *p;
    LQCD_TRY(ws_get(ctx, WS_TC_STAT, 64 * (sizeof(unsigned long long) + 2 * sizeof(int)) + 64, &p));
    int *colexp = (int *)((unsigned long long *)p + 64) + 64;
    int *flag = colexp + 64;
    const size_t bbytes = (size_t)S->kcc * TC_SA * NP * TC_KCH * 2;
    LQCD_TRY(ws_get(ctx, WS_TC_B, bbytes, &p));
    unsigned char *Bsl = (unsigned char *)p;
    LQCD_CUDA(ctx, cudaMemsetAsync(Bsl, 0, bbytes, ctx->stream));
    LQCD_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
    kbegin(ctx);
    slice_c_kernel<<<nb, 128, 0, ctx->stream>>>(Cm + r0, d, k, nrhs, NP, (unsigned short *)Bsl, colexp);
    LQCD_TRY(launch_check(ctx, "slice_c_kernel", K_SLICE, (double)k * nb));
    TcArgs a{};
    a.kcr = tc_kcr(TC_SA, 128.0);
    a.unit_shift = 16;
    a.A = S->Ac;
    a.B = Bsl;
    a.mt_count = S->mtc;
    a.m_valid = (int)S->L;
    a.kc_count = S->kcc;
    a.ksplit = 1;
    a.colexp = colexp;
    a.rowexp = S->rowexp;
    a.nb = nb;
    a.out = (double *)(Y + (size_t)r0 * ctx->N);
    a.err = flag;
        // the exact parts of all read-outs of a tile are summed as 64-bit integers (each < 2^57)
    if ((S->kcc + a.kcr - 1) / a.kcr > 63)
      return set_err(ctx, LQCD_ERR_INVALID_ARG, "tensor-core V C: too many read-outs per tile");
    LQCD_TRY(tc_gemm(ctx, NP, TC_SA, 1, a, (double)k * nb * ctx->N));
    LQCD_TRY(check_flag(ctx, flag, "tensor-core V C"));
  }
  return LQCD_OK;
}

// Y = E C (ncol output fields; E: k fields of N, vector-major; C: device, k x ncol) on the tensor
// cores with only the operand slices of this product, built in context workspace (kept for the next
// call of the same or smaller size): the restart rotation V_{k+1} = V_{m+1} P_{k+1} of GMRES-DR /
// MINRES-DR and its Ritz vectors, a new basis every call.
lqcd_status tc_vc_oneshot(lqcd_ctx *ctx, const double2 *E, int k, const double2 *C, int ncol, double2 *Y) {
  if (k <= 0 || k > 4096 || ncol <= 0) return set_err(ctx, LQCD_ERR_INVALID_ARG, "tensor-core V C: bad sizes");
  TcSlices S{};
  S.k = k;
  S.L = 2 * ctx->N;
  S.mtc = (int)((S.L + TC_M - 1) / TC_M);
  S.kcc = (k + TC_KCH - 1) / TC_KCH;
  const size_t bc = tc_bytes_c(k, S.L);
  void *p;
  LQCD_TRY(ws_get(ctx, WS_TC_AC, bc, &p));
  S.Ac = (unsigned char *)p;
  LQCD_TRY(ws_get(ctx, WS_TC_REXP, sizeof(int) * (size_t)S.L + 64, &p));
  S.rowexp = (int *)p;
  int *flag = S.rowexp + S.L;
  LQCD_CUDA(ctx, cudaMemsetAsync(S.Ac, 0, bc, ctx->stream));
  LQCD_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
  kbegin(ctx);
  rowexp_kernel<<<ceil_div(S.L, 256), 256, 0, ctx->stream>>>((const double *)E, k, S.L, S.rowexp, flag);
  LQCD_TRY(launch_check(ctx, "rowexp_kernel", K_SLICE, (double)k * S.L));
  LQCD_TRY(check_flag(ctx, flag, "tensor-core V C"));
  kbegin(ctx);
  slice_ac_kernel<<<dim3(ceil_div(S.L, 128), S.kcc * (TC_KCH / 8)), 128, 0, ctx->stream>>>(
      (const double *)E, k, S.L, S.rowexp, S.kcc, (unsigned short *)S.Ac);
  LQCD_TRY(launch_check(ctx, "slice_ac_kernel", K_SLICE, (double)k * S.L));
  return tc_vc(ctx, &S, C, nullptr, ncol, Y);
}

extern "C" lqcd_status lqcd_tc_slice_bytes(const int dims[4], int k, size_t *bytes) {
  if (!dims || !bytes || k < 1 || k > 4096) return LQCD_ERR_INVALID_ARG;
  long long V = 1;
  for (int i = 0; i < 4; ++i) {
    // the same limits as a context: extents 2..1024 and at most 2^28 sites, so no product overflows
    if (dims[i] < 2 || dims[i] > 1024) return LQCD_ERR_INVALID_ARG;
    V *= dims[i];
    if (V > (1LL << 28)) return LQCD_ERR_INVALID_ARG;
  }
  const long long L = 24 * V;  // reals per field
  *bytes = tc_bytes_g(k, L) + tc_bytes_c(k, L) + sizeof(int) * (size_t)L +
           sizeof(int) * (k + 2) + sizeof(unsigned long long) * k + sizeof(int) * (k + 1);
  return LQCD_OK;
}

extern "C" lqcd_status lqcd_set_wait_limit(lqcd_ctx *ctx, double seconds) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  if (!(seconds >= 1e-3 && seconds <= 60.0))
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "set_wait_limit: seconds must be in [1e-3, 60]");
  ctx->tc_wait_ns = (unsigned long long)(seconds * 1e9);
  return LQCD_OK;
}

extern "C" lqcd_status lqcd_inject_tc_stall(lqcd_ctx *ctx, int chunks) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  ctx->tc_stop_after = chunks < 0 ? -1 : chunks;
  return LQCD_OK;
}

extern "C" lqcd_status lqcd_set_defl_engine(lqcd_ctx *ctx, int engine) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  if (engine != LQCD_DEFL_FP64 && engine != LQCD_DEFL_TENSOR)
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "set_defl_engine: unknown engine %d", engine);
  ctx->defl_engine = engine;
  return LQCD_OK;
}

namespace {
// slices of caller vectors for one call, released on every exit path
struct ScopedSlices {
  void *p = nullptr;
  ~ScopedSlices() { tc_slices_free(p); }
};
}  // namespace

extern "C" lqcd_status lqcd_tc_vdag_x(lqcd_ctx *ctx, const double *E, int k, const double *X, int nrhs, double *G) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  if (!E || !X || !G || k <= 0 || nrhs <= 0 || nrhs > 65535)
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "tc_vdag_x: bad arguments");
  ScopedSlices sl;
  LQCD_TRY(tc_slices_make(ctx, (const double2 *)E, k, &sl.p));
  return tc_vhx(ctx, sl.p, (const double2 *)X, nrhs, (double2 *)G);
}

extern "C" lqcd_status lqcd_tc_v_c(lqcd_ctx *ctx, const double *E, int k, const double *C, int nrhs, double *Y) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  if (!E || !C || !Y || k <= 0 || nrhs <= 0 || nrhs > 65535)
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "tc_v_c: bad arguments");
  ScopedSlices sl;
  LQCD_TRY(tc_slices_make(ctx, (const double2 *)E, k, &sl.p));
  return tc_vc(ctx, sl.p, (const double2 *)C, nullptr, nrhs, (double2 *)Y);
}
