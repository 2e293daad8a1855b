// Shared definitions of the liblqcd CUDA sources: context, status plumbing, complex helpers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <memory>
#include <string>
#include <vector>

#include "lqcd.h"
#include <nvtx3/nvToolsExt.h>

// NVTX range of one stage of the path (visible to profilers; a no-op without one attached)
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// kernel classes for the optional per-class device timing (values of LQCD_K_* in lqcd.h)
enum KClass { K_WILSON = 0, K_DOT, K_AXPY, K_COMBINE, K_NORM, K_CONTRACT, K_BLAS1, K_NOISE, K_PROBE, K_TENSOR, K_SLICE,
              K_NCLASS };

struct TimedLaunch {
  int start, end, cls;  // indices into lqcd_ctx::ev_pool
  double units;         // work units of the launch (see lqcd_timing_read)
  double bytes;         // compulsory device-memory bytes of the launch (0 where not tracked)
};

struct lqcd_ctx {
  int dims[4];          // Lx, Ly, Lz, Lt
  int V;                // sites
  long long N;          // complex unknowns per field, 12 V
  int device;
  int recon;            // 12 or 18: link storage of the packed FP32 inner operator
  int sms;
  cudaStream_t stream;
  std::string err;
  long launches;
  // named, growable device workspace (slot -> buffer); freed by lqcd_ctx_destroy
  std::vector<void *> ws_ptr;
  std::vector<size_t> ws_size;
  double *host_pinned;  // small pinned host staging buffer
  size_t host_pinned_size;
  // optional kernel timing: events bracket every launch while enabled
  bool timing;
  int pending_start;
  std::vector<cudaEvent_t> ev_pool;
  int ev_used;
  std::vector<TimedLaunch> timed;
  double t_ms[K_NCLASS];
  long t_count[K_NCLASS];
  double t_units[K_NCLASS];
  double t_bytes[K_NCLASS];
  // CUDA graphs of fixed launch sequences (the Arnoldi steps of a Krylov cycle), keyed by every
  // pointer and parameter they bake in; dropped whenever a workspace buffer is reallocated
  bool graphs;
  cudaStream_t cap_stream;   // private stream used only to capture
  cudaStream_t run_stream;   // private stream for concurrent batched runs
  struct GraphEntry {
    std::string key;
    cudaGraphExec_t exec;
    long nlaunch;            // kernels per replay
  };
  std::vector<GraphEntry> graph_cache;
  int packed_nr;             // tuned right-hand sides per thread of the packed FP32 operator (0 = built in)
  int defl_engine;           // LQCD_DEFL_FP64 or LQCD_DEFL_TENSOR (deflation projections)
  unsigned long long tc_wait_ns;  // bound of every tensor-core pipeline wait (lqcd_set_wait_limit)
  int tc_stop_after;         // injected stall of the next tensor-core launch (-1: none)
  int inner_gs_passes;       // Gram-Schmidt passes of the reduced-precision inner Arnoldi (0 = by storage)
  int probe_depth;           // full applications of P per probe in the hopping traces (0 = by cost)
  int inner_window;          // Lanczos window of Hermitian mixed-precision inner cycles (0 = full Gram-Schmidt)
  // even/odd reduced context (lqcd_ctx_create_evenodd): fields hold the even sites only (V above is
  // half the lattice), the operator is hat M = 1 - kappa^2 P_eo P_oe, eo_dims the full extents
  int eo;
  int eo_dims[4];
};

namespace dense { struct QRFact; }

struct lqcd_defl {
  lqcd_ctx *ctx;
  int k;
  int hermitian;
  long long N;
  double2 *V;           // (k+1) vectors of N (device), NULL when imported
  double2 *E;           // k eigenvectors of N (device)
  std::vector<double2> Hbar;  // (k+1) x k row-major (host)
  std::vector<double2> lam;   // k eigenvalues (host)
  std::vector<double> eres;   // k eigen residual norms (host)
  double2 *Hbar_dev;    // (k+1) x k row-major (device), NULL when imported
  void *tc;             // bf16 slices of E for the tensor-core contractions (made on first use)
  void *Vf32;           // packed FP32 copy of V for mixed-precision solves (made on first use)
  // Householder factorisation of Hbar for the GMRES-Proj projections (made on first use)
  std::shared_ptr<dense::QRFact> hqr;
};

// ----- status plumbing ------------------------------------------------------------------
lqcd_status set_err(lqcd_ctx *ctx, lqcd_status st, const char *fmt, ...);

#define LQCD_CUDA(ctx, call)                                                               \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return set_err((ctx), LQCD_ERR_CUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call,      \
                     cudaGetErrorString(e_));                                              \
  } while (0)

#define LQCD_TRY(expr)                                                                     \
  do {                                                                                     \
    lqcd_status s_ = (expr);                                                               \
    if (s_ != LQCD_OK) return s_;                                                          \
  } while (0)

// record the start event of the next launch (when timing is enabled)
void kbegin(lqcd_ctx *ctx);
// check the launch that was just enqueued, count it, and record its end event when timing
lqcd_status launch_check(lqcd_ctx *ctx, const char *what, int cls, double units);
// the same, also recording the launch's compulsory bytes (each operand element read or written once)
lqcd_status launch_check_bytes(lqcd_ctx *ctx, const char *what, int cls, double units, double bytes);

// growable workspace slot (device memory owned by the context)
enum WsSlot {
  WS_PARTIAL = 0, WS_SCAL, WS_TMP0, WS_TMP1, WS_TMP2, WS_TMP3, WS_BASIS, WS_HESS, WS_COEF,
  WS_BASIS2, WS_TMP4, WS_TMP5, WS_EST0, WS_EST1, WS_EST2, WS_PROBE,
  WS_MIX_U, WS_MIX_V, WS_MIX_R32, WS_MIX_E32, WS_MIX_R, WS_MIX_S, WS_COUNT, WS_TUNE, WS_SPEC, WS_NBLK, WS_TC_STAT, WS_TC_B, WS_TC_PART, WS_TC_D,
  WS_POLY1, WS_POLY2, WS_POLY3, WS_EO, WS_TC_AC, WS_TC_REXP, WS_PROBE_OFF, WS_HOST_LINKS, WS_NSLOTS
};
lqcd_status ws_get(lqcd_ctx *ctx, int slot, size_t bytes, void **ptr);
void graph_cache_clear(lqcd_ctx *ctx);
// Append the raw bytes of v to a graph key
template <typename T> inline void key_add(std::string &k, const T &v) { k.append((const char *)&v, sizeof(T)); }
// Run enqueue(arg) (a function that only enqueues work on ctx->stream: no synchronisation and no
// workspace growth) through a cached CUDA graph under key, capturing it on first use; with graphs
// off or device timing on, enqueue(arg) runs directly.
lqcd_status graph_cached(lqcd_ctx *ctx, const std::string &key, lqcd_status (*enqueue)(void *), void *arg);
// Reserve the workspace of blas_multidot / blas_norms for vectors of length n, nrhs right-hand
// sides and up to max_nvec basis vectors (so graph capture never grows a buffer).
lqcd_status blas_reserve(lqcd_ctx *ctx, long long n, int nrhs, int max_nvec);
lqcd_status host_stage(lqcd_ctx *ctx, size_t bytes, double **ptr);

// ----- complex helpers (device) -----------------------------------------------------------
__host__ __device__ __forceinline__ double2 cmake(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// conj(a) * b
__host__ __device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
// i * a and -i * a
__host__ __device__ __forceinline__ double2 cmuli(double2 a) { return make_double2(-a.y, a.x); }
__host__ __device__ __forceinline__ double2 cmulmi(double2 a) { return make_double2(a.y, -a.x); }
// acc += a * b
__device__ __forceinline__ void cfma(double2 &acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfma_conj(double2 &acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

// Neumaier compensated accumulation of one double
struct KSum {
  double s, c;
  __device__ __forceinline__ void init() { s = 0.0; c = 0.0; }
  __device__ __forceinline__ void add(double v) {
    double t = s + v;
    if (fabs(s) >= fabs(v)) c += (s - t) + v; else c += (v - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return s + c; }
};

static inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// ----- kernel launchers shared between translation units ---------------------------------
// Wilson operator on nrhs fields (see lqcd_wilson_apply); in and out must not overlap.
lqcd_status wilson_launch(lqcd_ctx *ctx, const double2 *U, double kappa, const double2 *in,
                          double2 *out, int nrhs, int prec, int flags);
// Reduced (even/odd) operator of an eo context: hat M, hat M gamma_5, hat M^dag or P_eo P_oe
lqcd_status eo_schur_launch(lqcd_ctx *ctx, const double2 *U, double kappa, const double2 *in, double2 *out, int nrhs,
                            int prec, int flags);
// reserve the odd-site scratch of eo_schur_launch for nrhs fields (no-op on a full context)
lqcd_status eo_reserve(lqcd_ctx *ctx, int nrhs);
// LQCD_ERR_INVALID_ARG on an even/odd reduced context (entry points that need the full lattice)
lqcd_status require_full(lqcd_ctx *ctx, const char *what);
// b_e + kappa P_eo b_o (b full, be reduced) and the full solution from x_e (x_o = b_o + kappa P_oe x_e)
lqcd_status eo_rhs_launch(lqcd_ctx *ctx, const double2 *U, double kappa, const double2 *b, double2 *be, int nrhs);
lqcd_status eo_reconstruct_launch(lqcd_ctx *ctx, const double2 *U, double kappa, const double2 *xe, const double2 *b,
                                  double2 *x, int nrhs);
// FP64, right-hand side r gets M gamma_5 when bit r of g5mask is set and M otherwise (nrhs <= 64)
lqcd_status wilson_launch_masked(lqcd_ctx *ctx, const double2 *U, double kappa, const double2 *in, double2 *out,
                                 int nrhs, unsigned long long g5mask);
// Packed FP32 operator (layout in wilson.cu): links packed by pack_links_f32 (recon 12 or 18),
// nr right-hand sides per thread (0 = automatic)
lqcd_status wilson_launch_packed(lqcd_ctx *ctx, const float4 *U, int recon, double kappa, const float4 *in, float4 *out,
                                 int nrhs, int flags, int nr);
lqcd_status pack_f32(lqcd_ctx *ctx, const double2 *x, const double *scale, float4 *y, int nrhs);
lqcd_status unpack_f32(lqcd_ctx *ctx, const float4 *c, const double *scale, double2 *x, int nrhs);
lqcd_status pack_links_f32(lqcd_ctx *ctx, const double2 *U, float4 *P, int recon);
// The same operator and packing with FP16 / BF16 fields (S = __half2 or __nv_bfloat162; FP32 links
// and arithmetic): the packed layout keeps the FP32 element order, each float4 chunk becoming an
// 8-byte pair of S, so FP32 and reduced-precision vectors of one solve index alike.
template <typename S>
lqcd_status wilson_launch_packed_lp(lqcd_ctx *ctx, const float4 *U, int recon, double kappa, const S *in, S *out,
                                   int nrhs, int flags);
template <typename S> lqcd_status pack_lp(lqcd_ctx *ctx, const double2 *x, const double *scale, S *y, int nrhs);
template <typename S> lqcd_status unpack_lp(lqcd_ctx *ctx, const S *c, const double *scale, double2 *x, int nrhs);
// FP32 storage and arithmetic (links converted to FP32 by the caller)
lqcd_status wilson_launch_f32(lqcd_ctx *ctx, const float2 *U, double kappa, const float2 *in, float2 *out,
                              int nrhs, int flags);
// ----- reduced-precision storage -----------------------------------------------------------
// Complex storage types of the inner solver: float2 (FP32), __half2 (FP16) and __nv_bfloat162
// (BF16); arithmetic on all three is FP32.  A field stored in FP16 or BF16 holds sigma * value with
// sigma = 2^floor(log2(sqrt(N))) for fields of N = 12 V components, so the entries of a unit
// vector are of order one: far from the FP16 overflow (65504) and subnormal (6e-5) ranges.  Every
// level-1/2 kernel and the packing kernels account for sigma; the operator, being linear, ignores it.
template <typename S> struct StoreScaled { static constexpr bool value = false; };
template <> struct StoreScaled<__half2> { static constexpr bool value = true; };
template <> struct StoreScaled<__nv_bfloat162> { static constexpr bool value = true; };
static inline double half_sigma(long long N) { return std::ldexp(1.0, (int)std::floor(0.5 * std::log2((double)N))); }
template <typename S> inline double store_sigma(long long N) { return StoreScaled<S>::value ? half_sigma(N) : 1.0; }
// distinct tag per storage type (graph keys: FP16 and BF16 have the same size)
template <typename S> struct StoreTag;
template <> struct StoreTag<double2> { static constexpr int value = 0; };
template <> struct StoreTag<float2> { static constexpr int value = 1; };
template <> struct StoreTag<__half2> { static constexpr int value = 2; };
template <> struct StoreTag<__nv_bfloat162> { static constexpr int value = 3; };

// Batched level-1/level-2 kernels (blas.cu).  Templates are instantiated for double2 (FP64 path)
// and for the inner-solver storage types float2, __half2, __nv_bfloat162 (two-type forms mix a
// reduced-precision basis with FP32 vectors); coefficients and cross-thread reductions are FP64.
// Vectors of __half2 / __nv_bfloat162 are fields of ctx->N components scaled by store_sigma.
template <typename SX, typename SY> lqcd_status blas_copy(lqcd_ctx *ctx, const SX *x, SY *y, long long n);
template <typename S> lqcd_status blas_zero(lqcd_ctx *ctx, S *y, long long n);
lqcd_status blas_g5(lqcd_ctx *ctx, const double2 *x, double2 *y, int nrhs);
// t = b - t
lqcd_status blas_bminus(lqcd_ctx *ctx, double2 *t, const double2 *b, long long n);
// norms[r] = ||x_r||_2 for nrhs vectors of length n (device output)
template <typename S> lqcd_status blas_norms(lqcd_ctx *ctx, const S *x, long long n, int nrhs, double *norms);
// Basis vector i of right-hand side r is V_i^r = V + i*vstride + r*vrs (vrs = 0: one basis shared
// by every right-hand side); w^r = w + r*n.
// h[i*nrhs + r] = <V_i^r, w^r> for i < nvec
template <typename SV, typename SW>
lqcd_status blas_multidot(lqcd_ctx *ctx, const SV *V, long long vstride, long long vrs, int nvec, const SW *w,
                          long long n, int nrhs, double2 *h);
// w^r += sign * sum_i V_i^r h[i*nrhs + r]
template <typename SV, typename SW>
lqcd_status blas_multiaxpy(lqcd_ctx *ctx, const SV *V, long long vstride, long long vrs, int nvec, const double2 *h,
                           double sign, SW *w, long long n, int nrhs);
// out_c^r = out + c*ostride + r*n = sum_i V_i^r C[(i*ncol + c)*nrhs + r] for c < ncol (no aliasing)
template <typename SV, typename SO>
lqcd_status blas_combine(lqcd_ctx *ctx, const SV *V, long long vstride, long long vrs, int nvec, const double2 *C,
                         int ncol, SO *out, long long ostride, long long n, int nrhs);
// x^r *= 1 / s[r] (s device); zero vector if s[r] == 0
template <typename S> lqcd_status blas_invscale(lqcd_ctx *ctx, S *x, const double *s, long long n, int nrhs);
// y += a x with a host scalar a
lqcd_status blas_axpy(lqcd_ctx *ctx, double2 a, const double2 *x, double2 *y, long long n);
// y = a x + b y with host scalars (any storage type)
template <typename S> lqcd_status blas_axpby(lqcd_ctx *ctx, double2 a, const S *x, double2 b, S *y, long long n);
// y^r = float(x^r / s[r])  and  x^r += s[r] * double(c^r)  (mixed-precision defect correction)
lqcd_status blas_demote(lqcd_ctx *ctx, const double2 *x, const double *s, float2 *y, long long n, int nrhs);
lqcd_status blas_promote_acc(lqcd_ctx *ctx, const float2 *c, const double *s, double2 *x, long long n, int nrhs);
lqcd_status blas_to_f32(lqcd_ctx *ctx, const double2 *x, float2 *y, long long n);
// contraction densities summed per timeslice (loops.cu); out device [nrhs][9][Lt]
lqcd_status contract_launch(lqcd_ctx *ctx, const double2 *U, double kappa, const double2 *eta,
                            const double2 *w, int nrhs, double2 *out_dev);
lqcd_status noise_launch(lqcd_ctx *ctx, uint64_t seed, uint32_t first, int nrhs, double2 *out);
// LQCD_ERR_NONFINITE (with a message naming what) when any of the n doubles at x is NaN or Inf;
// synchronises the stream
lqcd_status check_finite(lqcd_ctx *ctx, const double *x, long long n, const char *what);
// Tensor-core split-precision contractions with k vectors E (tcdefl.cu): slices of E made once
// (tc_slices_make, released by tc_slices_free), then G[q * nrhs + r] = <E_q, X_r> (tc_vhx) and
// Y_r = sum_q E_q d_q C[q * nrhs + r] (tc_vc; d device k complex or NULL); all device pointers.
lqcd_status tc_slices_make(lqcd_ctx *ctx, const double2 *E, int k, void **out);
void tc_slices_free(void *slices);
lqcd_status tc_vhx(lqcd_ctx *ctx, const void *slices, const double2 *X, int nrhs, double2 *G);
lqcd_status tc_vc(lqcd_ctx *ctx, const void *slices, const double2 *C, const double2 *d, int nrhs, double2 *Y);
// Y = E C for a basis used once (E: k fields, C: k x ncol device): only this product's slices, in
// context workspace
lqcd_status tc_vc_oneshot(lqcd_ctx *ctx, const double2 *E, int k, const double2 *C, int ncol, double2 *Y);
// right-hand-side block width autotuner (batch.cu); see lqcd_autotune_block
lqcd_status autotune_block(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_defl *defl,
                           const lqcd_krylov_opts *o, const int *cand, int ncand, int *best, double *seconds);
