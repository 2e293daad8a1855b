/*
 * lqcd.h -- C ABI of the GB300 (sm_103a) library for disconnected-loop noise estimation with
 * deflation, perturbative and polynomial subtraction (Baral, Whyte, Wilcox, Morgan,
 * "Disconnected Loop Subtraction Methods in Lattice QCD").
 *
 * Conventions shared by every call
 * --------------------------------
 *  Complex numbers are interleaved FP64 pairs (re, im) ("complex128").  A spinor field of one
 *  right-hand side is 12 V complex numbers in the canonical order
 *        [T][Z][Y][X][spin 4][colour 3],  site s = x + Lx (y + Ly (z + Lz t)),
 *  and a block of nrhs fields is nrhs such fields back to back.  Gauge links are
 *        [mu 4][T][Z][Y][X][3][3]  complex128, mu = x, y, z, t, row-major colour matrices.
 *  Gamma matrices: Euclidean Hermitian, Dirac representation,
 *        gamma_k = [[0, -i sigma_k], [i sigma_k, 0]], gamma_4 = diag(1, 1, -1, -1),
 *        gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4.
 *  Boundary conditions are periodic in all four directions (Sec. 7).
 *
 *  Unless a parameter says "host", every array argument is a caller-owned DEVICE pointer on the
 *  device that was current when the context was created, 16-byte aligned.  The library owns only
 *  its internal workspace (held by the context) and the deflation-space objects it returns.
 *  Calls are enqueued on the context's stream; a call that returns host data synchronises that
 *  stream before returning.  No call aborts the process: every call returns an lqcd_status and,
 *  on failure, lqcd_last_error_string(ctx) describes the first problem found.
 */
#ifndef LQCD_H
#define LQCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LQCD_OK = 0,
  LQCD_ERR_INVALID_ARG = 1,   /* bad size, NULL pointer, unsupported option            */
  LQCD_ERR_NONFINITE = 2,     /* NaN or Inf found in an input or a solver iterate      */
  LQCD_ERR_NOT_CONVERGED = 3, /* solver stopped at max_cycles above its tolerance      */
  LQCD_ERR_TIMEOUT = 4,       /* a bounded device wait ran out                         */
  LQCD_ERR_CUDA = 5,          /* a CUDA runtime call failed (message has the details)  */
  LQCD_ERR_OOM = 6            /* workspace allocation failed                           */
} lqcd_status;

/* Precision of an operator application or of the inner solver of a mixed-precision solve.  F64 is
 * the plain FP64 path; F32 is FP32 storage and arithmetic; F16 and BF16 are FP16 / BF16 storage of
 * the fields and Krylov vectors with FP32 arithmetic. */
typedef enum { LQCD_PREC_F64 = 0, LQCD_PREC_F32 = 1, LQCD_PREC_F16 = 2, LQCD_PREC_BF16 = 3 } lqcd_prec;

/* lqcd_wilson_apply flags (may be OR-ed only where stated) */
#define LQCD_APPLY_M 0     /* out = M in,  M = 1 - kappa P                      (Eq. xyz556) */
#define LQCD_APPLY_G5R 1   /* out = M gamma_5 in  (M' of Sec. 5.4, Hermitian)                */
#define LQCD_APPLY_DAG 2   /* out = M^dagger in = gamma_5 M gamma_5 in                      */
#define LQCD_APPLY_HOP 3   /* out = P in  (the hopping matrix below Eq. xyz556)              */

/* Which linear system a solver works on */
#define LQCD_SYS_M 0       /* M x = b                                                       */
#define LQCD_SYS_MG5 1     /* M gamma_5 y = b  (then x = gamma_5 y solves M x = b)          */

/* Subtraction modes of Sec. 5 (bit mask for lqcd_loop_estimate) */
#define LQCD_SUB_NONE (1 << 0)      /* NS                                                   */
#define LQCD_SUB_PERT (1 << 1)      /* PS, Sec. 5.1                                         */
#define LQCD_SUB_POLY (1 << 2)      /* POLY, Sec. 5.2                                       */
#define LQCD_SUB_DEFL (1 << 3)      /* HFES, Sec. 5.4                                       */
#define LQCD_SUB_DEFL_PERT (1 << 4) /* HFPS, Sec. 5.5                                       */
#define LQCD_SUB_DEFL_POLY (1 << 5) /* HFPOLY, Sec. 5.5                                     */
#define LQCD_SUB_ES (1 << 6)        /* ES, Sec. 5.3: Ritz pairs of M on the GMRES-DR space,
                                       left vectors e_L(lambda) = gamma_5 e_R(lambda*) / conj(e_R(lambda*)^dag
                                       gamma_5 e_R(lambda)); a mode whose conjugate partner is not
                                       among the pairs is not subtracted; with LQCD_SYS_MG5 there is
                                       no space of M and ES subtracts nothing (equals NS)        */
#define LQCD_SUB_ALL 127
#define LQCD_NMODES 7
#define LQCD_NOPS 9 /* 0 scalar, 1-4 local vector mu = x,y,z,t, 5-8 point-split mu = x,y,z,t */

typedef struct lqcd_ctx lqcd_ctx;
typedef struct lqcd_defl lqcd_defl;

typedef struct {
  int m;             /* Krylov subspace size per cycle (GMRES-DR(m, k))                      */
  int k;             /* deflation size: harmonic Ritz vectors kept at restart (0 = GMRES(m)) */
  double tol;        /* stop when ||b - A x|| <= tol ||b|| (relative true residual)          */
  int max_cycles;    /* restart cycles before LQCD_ERR_NOT_CONVERGED                         */
  int system;        /* LQCD_SYS_M or LQCD_SYS_MG5                                           */
  int prec;          /* lqcd_prec of the inner operator; LQCD_PREC_F64 for the plain path    */
  double inner_tol;  /* mixed precision: relative residual of each inner solve (0 = default:
                        5e-6 F32, 2e-2 F16, 5e-2 BF16)                                        */
  double eig_tol;    /* GMRES-DR / MINRES-DR: with eig_tol > 0 the cycles also continue until
                        every Rayleigh-Ritz residual ||A e - lambda e|| of the restart space is
                        <= eig_tol ("super-convergence" of the first right-hand side, which
                        converges the eigenvectors, Sec. 5.4, 7); 0 = residual criterion only */
  int poly_degree;   /* polynomial right preconditioner (the Min-Res polynomial of Sec. 5.2 used
                        inside the solver): the Krylov method works on B = A p(A) with
                        p(A) = sum_j a_j A^j (A = M or M gamma_5 by the system), returns
                        x = p(A) y (the solution of A x = b, same residual); deflation spaces
                        made or used by the call are spaces of B.  0 = none, at most 32      */
  const double *poly_coeffs; /* host, poly_degree + 1 complex a_j (read during the call)      */
} lqcd_krylov_opts;

typedef struct {
  int cycles;        /* restart cycles used (largest over the right-hand sides)              */
  long matvecs;      /* operator applications, summed over right-hand sides                  */
  int converged;     /* 1 when every right-hand side met tol                                 */
  double true_resid; /* largest relative true residual over the right-hand sides (FP64)      */
  double seconds;    /* wall time of the call                                                */
} lqcd_solve_info;

/* ---- context --------------------------------------------------------------------------- */

/* Create a context for an Lx x Ly x Lz x Lt lattice (dims[0..3] = Lx, Ly, Lz, Lt, each >= 2) on
 * the current CUDA device.  link_recon is 18 (general links) or 12 (the caller declares the links
 * special unitary: the FP32 inner operator of the mixed-precision solver then stores two rows per
 * link and rebuilds the third; FP64 operators always read all nine entries).  stream is a
 * cudaStream_t (NULL = legacy default stream).  Returns LQCD_ERR_INVALID_ARG for bad dims or
 * link_recon, LQCD_ERR_CUDA if no device is usable. */
lqcd_status lqcd_ctx_create(lqcd_ctx **ctx, const int dims[4], int link_recon, void *stream);
lqcd_status lqcd_ctx_destroy(lqcd_ctx *ctx);
lqcd_status lqcd_set_stream(lqcd_ctx *ctx, void *stream);
/* Message of the last failure on this context ("" if none); valid until the next call. */
const char *lqcd_last_error_string(const lqcd_ctx *ctx);
/* Library version string (static storage). */
const char *lqcd_version(void);
/* Number of kernels this context has launched since creation (diagnostics). */
long lqcd_kernel_launches(const lqcd_ctx *ctx);

/* Per-kernel-class device timing (diagnostics; the paper has no counterpart).  While enabled,
 * every kernel launched through this context is bracketed by CUDA events on the context's stream
 * (a small per-launch cost).  lqcd_timing_read synchronises the stream and returns, for one class
 * since the last reset, the summed device milliseconds, the launch count and the summed work
 * units (may be NULL): site x right-hand-side pairs for WILSON, CONTRACT, NOISE and PROBE;
 * complex multiply-adds for DOT, AXPY and COMBINE; complex elements for NORM and BLAS1. */
#define LQCD_K_WILSON 0   /* Wilson operator (Eq. xyz556)                               */
#define LQCD_K_DOT 1      /* batched inner products (Gram-Schmidt, projections)          */
#define LQCD_K_AXPY 2     /* batched multi-vector updates                                */
#define LQCD_K_COMBINE 3  /* basis rotations V P (restarts, Ritz vectors)                */
#define LQCD_K_NORM 4     /* batched norms                                               */
#define LQCD_K_CONTRACT 5 /* operator contractions (Sec. 6)                              */
#define LQCD_K_BLAS1 6    /* copies, scalings, gamma_5, axpy                             */
#define LQCD_K_NOISE 7    /* Z(4) noise generation                                       */
#define LQCD_K_PROBE 8    /* probe-vector generation for the hopping traces              */
#define LQCD_K_TENSOR 9   /* tcgen05 split-precision contractions (units: complex MACs)   */
#define LQCD_K_SLICE 10   /* operand statistics and bf16 slicing for them (units: elements) */
#define LQCD_K_NCLASS 11
lqcd_status lqcd_timing_enable(lqcd_ctx *ctx, int enable);
lqcd_status lqcd_timing_reset(lqcd_ctx *ctx);
lqcd_status lqcd_timing_read(lqcd_ctx *ctx, int cls, double *total_ms, long *launches, double *units);
/* Compulsory device-memory bytes (every operand element read or written once) summed over the
 * timed launches of one class since the last reset, for the launches that record them (Wilson
 * operators, DOT, AXPY, COMBINE, NORM and the basis scaling of BLAS1; other launches add 0).
 * Synchronises the stream like lqcd_timing_read. */
lqcd_status lqcd_timing_bytes(lqcd_ctx *ctx, int cls, double *bytes);

/* ---- Z(4) noise (Sec. 2, 3) ------------------------------------------------------- */

/* out[n] = Z(4) noise number first_noise + n, n < nrhs: entry (s, spin, colour) is
 * {1, i, -1, -i}[(w >> 2c) & 3] with c = 3 spin + colour and w word 0 of Philox-4x32-10
 * (Salmon et al., SC'11) with key (seed mod 2^32, seed >> 32) and counter (noise, s, 0, 0).
 * out: device, nrhs * 12 V complex128.  Bit-exact. */
lqcd_status lqcd_noise_z4(lqcd_ctx *ctx, uint64_t seed, uint32_t first_noise, int nrhs, double *out);

/* ---- Wilson operator (Eq. xyz556; Sec. 5.4) --------------------------------------- */

/* out = A in for nrhs fields, A selected by flags (LQCD_APPLY_*).  links: device gauge field;
 * in/out: device, nrhs * 12 V complex128, must not overlap.  prec must be LQCD_PREC_F64 or
 * LQCD_PREC_F32 (FP32 arithmetic on FP64 data, for testing the inner operator). */
lqcd_status lqcd_wilson_apply(lqcd_ctx *ctx, const double *links, double kappa, const double *in,
                              double *out, int nrhs, int prec, int flags);

/* The inner operator of the mixed-precision solver: the same operator on FP32 storage with FP32
 * arithmetic.  links32: device gauge field as interleaved float pairs, same layout as the FP64
 * links; in/out: device, nrhs * 12 V float pairs, must not overlap.  flags as above. */
lqcd_status lqcd_wilson_apply_f32(lqcd_ctx *ctx, const float *links32, double kappa, const float *in, float *out,
                                  int nrhs, int flags);
/* Convert n complex numbers from FP64 to FP32 storage on the device (e.g. links for the call above). */
lqcd_status lqcd_to_f32(lqcd_ctx *ctx, const double *in, float *out, long long n);

/* Packed FP32 layout of the mixed-precision inner solver: per right-hand side, the 24 reals of a
 * site form six float4 chunks (chunk q = complex components 2q, 2q+1 of the canonical spin-colour
 * order), stored chunk-major: float4 (r, q, s) at index (r * 6 + q) * V + s.  Packed links: per
 * direction, recon 12 stores rows 0 and 1 as three float4 chunks ((u00,u01), (u02,u10), (u11,u12))
 * and rebuilds row 2 = conj(row0 x row1) (exact for SU(3) links); recon 18 stores all nine entries
 * in five float4 chunks (last half zero).  Buffers: packed fields nrhs * 24 V floats, packed links
 * 4 * 12 V (recon 12) or 4 * 20 V (recon 18) floats, device. */
lqcd_status lqcd_pack_f32(lqcd_ctx *ctx, const double *in, float *out, int nrhs);
lqcd_status lqcd_unpack_f32(lqcd_ctx *ctx, const float *in, double *out, int nrhs);
lqcd_status lqcd_pack_links_f32(lqcd_ctx *ctx, const double *links, float *out, int recon);
/* Packed FP32 operator (flags as lqcd_wilson_apply).  rhs_per_thread: 1 = one thread per site and
 * right-hand side; 2 = two right-hand sides per thread in the two lanes of packed FP32 arithmetic
 * (links loaded and rebuilt once for both); 3 = the same with the neighbour spinors and links of
 * the next directions staged asynchronously in shared memory (cp.async) while the current one is
 * computed; 4 = four per thread, scalar; 0 = the context's setting (lqcd_set_rhs_per_thread, or the
 * autotuner's pick), else 2. */
lqcd_status lqcd_wilson_apply_packed(lqcd_ctx *ctx, const float *links_packed, int recon, double kappa,
                                     const float *in, float *out, int nrhs, int flags, int rhs_per_thread);

/* FP16 / BF16 fields (prec LQCD_PREC_F16 or LQCD_PREC_BF16) of the mixed-precision inner solver:
 * the packed FP32 layout above with each float4 chunk stored as two FP16 or BF16 complex numbers
 * (8 bytes), holding sigma * value with sigma = 2^floor(log2(sqrt(12 V))) so that the entries of a
 * unit-norm field are of order one.  Buffers: nrhs * 24 V halves (2 bytes each), device.
 * lqcd_pack_half / lqcd_unpack_half convert from / to canonical complex128 (sigma applied and
 * removed); lqcd_wilson_apply_half applies the operator (flags as lqcd_wilson_apply) with packed
 * FP32 links (lqcd_pack_links_f32) and FP32 arithmetic, in and out must not overlap. */
lqcd_status lqcd_pack_half(lqcd_ctx *ctx, int prec, const double *in, void *out, int nrhs);
lqcd_status lqcd_unpack_half(lqcd_ctx *ctx, int prec, const void *in, double *out, int nrhs);
lqcd_status lqcd_wilson_apply_half(lqcd_ctx *ctx, int prec, const float *links_packed, int recon, double kappa,
                                   const void *in, void *out, int nrhs, int flags);
/* Right-hand sides per thread of the packed operators used by this context when a call does not
 * choose (0 = built-in choice, paired lanes; 1; 2 = paired lanes, also for FP16 / BF16 fields;
 * 3 = paired lanes with asynchronous staging, also for FP16 / BF16; 4 = FP32 only).
 * The mixed-precision solvers use it; lqcd_autotune_block sets it. */
lqcd_status lqcd_set_rhs_per_thread(lqcd_ctx *ctx, int nr);

/* ---- GMRES-DR and MINRES-DR (Sec. 5.3, 7, 8) --------------------------------- */

/* GMRES-DR(m, k) for nrhs independent right-hand sides (each with its own Krylov basis).
 * b, x: device, nrhs * 12 V complex128 (x is overwritten; the initial guess is zero).
 * opts->system selects M or M gamma_5.  If defl_out is not NULL and nrhs == 1, *defl_out
 * receives the deflation space of the final cycle: V_{k+1} (12 V x (k+1)), Hbar_k
 * ((k+1) x k) with A V_k = V_{k+1} Hbar_k, and the Rayleigh-Ritz eigenpairs of A on V_k;
 * free it with lqcd_defl_destroy.  Host info may be NULL. */
lqcd_status lqcd_gmresdr_solve(lqcd_ctx *ctx, const double *links, double kappa, const double *b,
                               double *x, int nrhs, const lqcd_krylov_opts *opts,
                               lqcd_solve_info *info, lqcd_defl **defl_out);

/* MINRES-DR: the same cycle for the Hermitian M' = M gamma_5 (opts->system is ignored and taken
 * as LQCD_SYS_MG5); the harmonic Ritz problem is solved in its Hermitian-definite form and the
 * returned eigenpairs (lambda'_q, e'_q) are real / orthonormal (Sec. 5.4, 8). */
lqcd_status lqcd_minresdr_solve(lqcd_ctx *ctx, const double *links, double kappa, const double *b,
                                double *x, int nrhs, const lqcd_krylov_opts *opts,
                                lqcd_solve_info *info, lqcd_defl **defl_out);

/* ---- deflated multi-RHS solves (GMRES-Proj, Sec. 5.3, 7) --------------------------- */

/* Solve A x = b for nrhs right-hand sides with GMRES-Proj over defl (made by one of the two
 * solvers above on the same A): each cycle is a minimum-residual projection over V_{k+1} and
 * Hbar_k followed by GMRES(opts->m).  opts->k is ignored.  b, x: device (nrhs * 12 V).
 * opts->prec = LQCD_PREC_F32, LQCD_PREC_F16 or LQCD_PREC_BF16 selects mixed precision: an FP64
 * defect-correction loop around the same GMRES-Proj run in that storage precision with FP32
 * arithmetic (Krylov basis in that precision; deflation space, inner solution and residual in
 * FP32; inner relative residual opts->inner_tol), stopping on the FP64 true residual
 * ||b - A x|| <= tol ||b||; opts->max_cycles bounds the inner cycles. */
lqcd_status lqcd_proj_solve(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_defl *defl,
                            const double *b, double *x, int nrhs, const lqcd_krylov_opts *opts,
                            lqcd_solve_info *info);

/* ---- deflation-space objects ------------------------------------------------------------ */

lqcd_status lqcd_defl_destroy(lqcd_defl *defl);
/* k and whether it came from the Hermitian solver (host outputs). */
lqcd_status lqcd_defl_info(const lqcd_defl *defl, int *k, int *hermitian);
/* Copy out, each optional (NULL skips):  V (device, (k+1) x 12V, vector-major), Hbar (host,
 * (k+1) x k complex row-major), lam (host, k complex eigenvalues, increasing |lam|),
 * E (device, k x 12V eigenvectors, vector-major), eig_resid (host, k doubles ||A e - lam e||). */
lqcd_status lqcd_defl_export(const lqcd_defl *defl, double *V, double *Hbar, double *lam, double *E,
                             double *eig_resid);
/* Build a deflation object from caller data (e.g. eigenvectors from elsewhere): E (device,
 * k x 12V orthonormal eigenvectors of M' = M gamma_5), lam (host, k complex).  Only usable for
 * lqcd_deflate_project / lqcd_xi_inverse / lqcd_loop_estimate subtraction (no projection data). */
lqcd_status lqcd_defl_import(lqcd_ctx *ctx, int k, const double *E, const double *lam,
                             lqcd_defl **defl_out);
/* Build a full deflation space from caller data (a checkpointed solver space, or one made
 * elsewhere): V (device, (k+1) x 12V, vector-major, orthonormal) and Hbar (host, (k+1) x k complex
 * row-major) with A V_k = V_{k+1} Hbar_k for A = M (hermitian = 0) or M' = M gamma_5 (hermitian = 1).
 * The Rayleigh-Ritz eigenpairs are computed as for a solver-made space, so the object serves
 * lqcd_proj_solve, lqcd_deflate_project and lqcd_loop_setup_from alike.  The data are copied.
 * LQCD_ERR_NONFINITE for a NaN / Inf in Hbar, LQCD_ERR_OOM if the copies do not fit. */
lqcd_status lqcd_defl_import_space(lqcd_ctx *ctx, int k, const double *V, const double *Hbar, int hermitian,
                                   lqcd_defl **defl_out);

/* ---- deflation projection (HFES, Sec. 5.4) ----------------------------------------- */

/* out = gamma_5 V' diag(d) V'^dagger eta for nrhs fields, V' the k eigenvectors of defl and d a
 * host array of k complex weights (1/lambda' for HFES, 1/lambda' - 1/xi' for HFPS/HFPOLY).
 * eta, out: device, nrhs * 12 V. */
lqcd_status lqcd_deflate_project(lqcd_ctx *ctx, const lqcd_defl *defl, const double *eta,
                                 double *out, int nrhs, const double *d);

/* ---- FP64 deflation contractions on the tensor cores (Sec. 5.4) ------------------------ */

/* The two dense products of the HFES projection, V'^dagger eta and V' C, can run on the tcgen05
 * tensor cores with FP64 accuracy by split-precision emulation: each FP64 operand row / column is
 * scaled by a power of two and cut into seven bf16 slices of 8 bits (balanced digits), the slice
 * products are accumulated in FP32 tensor memory in groups that stay exact integers, and the groups
 * are folded into FP64 (error below 2^-53 of sum_i |a_i||b_i| plus FP64 rounding of the folds).
 * A right-hand side made of small integers times one power of two (Z(4) noise) is a single exact
 * slice.  The slices of a deflation space take 28 bytes per complex entry of device memory. */
#define LQCD_DEFL_FP64 0   /* FP64 CUDA-core kernels (default)                                */
#define LQCD_DEFL_TENSOR 1 /* split-precision tensor-core kernels                             */
/* Select the engine of lqcd_deflate_project and of the HFES / HFPS / HFPOLY projections inside
 * lqcd_loop_estimate for this context.  With LQCD_DEFL_TENSOR the slices of a deflation object
 * are made on its first projection and kept until lqcd_defl_destroy.  LQCD_ERR_INVALID_ARG for an
 * unknown engine. */
lqcd_status lqcd_set_defl_engine(lqcd_ctx *ctx, int engine);
/* Bound, in seconds, of every device-side wait of the tensor-core kernels (their mbarrier pipeline
 * waits): a wait that runs out makes the kernel record LQCD_ERR_TIMEOUT, stop issuing work, let the
 * copies and MMAs it has in flight land (under a fixed 2 s bound of its own), free its tensor
 * memory and return, so the call returns LQCD_ERR_TIMEOUT with the context still usable.  Default
 * 2; LQCD_ERR_INVALID_ARG outside [1e-3, 60]. */
lqcd_status lqcd_set_wait_limit(lqcd_ctx *ctx, double seconds);
/* Failure injection for tests of that timeout path (it faults nothing): the next tensor-core
 * contraction launched on this context has every CTA's loader stop issuing copies after `chunks`
 * pipeline chunks, so its MMA warp waits on a stage that nothing fills until the wait limit runs
 * out.  One-shot; chunks < 0 cancels. */
lqcd_status lqcd_inject_tc_stall(lqcd_ctx *ctx, int chunks);
/* G[q * nrhs + r] = E_q^dagger X_r on the tensor cores (one-shot: E is sliced on every call).
 * E: device, k x 12V complex128 vectors (vector-major); X: device, nrhs fields; G: device output,
 * k x nrhs complex128.  1 <= k <= 4096.  Returns LQCD_ERR_NONFINITE for a NaN / Inf input,
 * LQCD_ERR_OOM if the slices do not fit, LQCD_ERR_TIMEOUT if a pipeline wait ran out. */
lqcd_status lqcd_tc_vdag_x(lqcd_ctx *ctx, const double *E, int k, const double *X, int nrhs, double *G);
/* Y_r = sum_q E_q C[q * nrhs + r] on the tensor cores (one-shot).  E as above; C: device,
 * k x nrhs complex128; Y: device output, nrhs fields (must not overlap E or C).  Errors as above. */
lqcd_status lqcd_tc_v_c(lqcd_ctx *ctx, const double *E, int k, const double *C, int nrhs, double *Y);
/* Device bytes the tensor-core slices of k vectors take on an Lx x Ly x Lz x Lt lattice (dims[0..3],
 * each >= 2): the two slice copies kept per deflation object with LQCD_DEFL_TENSOR (and made for
 * the duration of one lqcd_tc_vdag_x / lqcd_tc_v_c call), plus their per-row exponents.  Host
 * only: needs no GPU and no context.  LQCD_ERR_INVALID_ARG for bad dims (an extent outside 2..1024,
 * or more than 2^28 sites, the limits of lqcd_ctx_create), k outside 1..4096 or a NULL bytes. */
lqcd_status lqcd_tc_slice_bytes(const int dims[4], int k, size_t *bytes);

/* ---- perturbative and polynomial series (Sec. 5.1, 5.2) ---------------------- */

/* out = sum_{k=0}^{K-1} c_k (kappa P)^k eta; c: host K complex, or NULL for all ones (PS). */
lqcd_status lqcd_hop_series(lqcd_ctx *ctx, const double *links, double kappa, const double *eta,
                            double *out, int nrhs, int K, const double *c);
/* out = sum_{j=0}^{n} a_j M^j eta; a: host n+1 complex (POLY). */
lqcd_status lqcd_poly_apply(lqcd_ctx *ctx, const double *links, double kappa, const double *eta,
                            double *out, int nrhs, int n, const double *a);
/* Min-Res coefficients a_0..a_n (host out, n+1 complex) minimising ||b - M P_n(M) b|| for
 * b = Z(4) noise number 2^32 - 1 of the given seed (Sec. 5.2, "one single noise vector"). */
lqcd_status lqcd_poly_coeffs(lqcd_ctx *ctx, const double *links, double kappa, uint64_t seed, int n,
                             double *a);

/* ---- hopping traces (Sec. 5.1) ------------------------------------------------------ */

/* t[k][op][t] = sum over the timeslice t of the exact diagonal density of Tr(Theta_op P^k),
 * k < K, by probing with colour classes whose members are more than K hops apart (host out,
 * K x 9 x Lt complex).  kappa enters only the point-split operators' own prefactor.
 * Meet in the middle (Sec. 5.1 add-back): P is applied to the whole probe field only up to a depth
 * h (lqcd_set_probe_depth; by default the h with the fewest site updates, e.g. 2 of the 6 orders at
 * K = 7 with 512 classes); each higher order k is evaluated only within K - k hops of the class
 * members, where the contraction and the later orders read it.  The result is the same trace. */
lqcd_status lqcd_hop_traces(lqcd_ctx *ctx, const double *links, double kappa, int K, double *t);

/* Full-lattice applications of P per probe in lqcd_hop_traces and in the setup of loop estimates:
 * depth in 1..64 fixes it, capped at K - 1 (every order a full application) and raised where an
 * order would otherwise be completed more than 8 hops around the members; 0 = chosen per call to
 * minimise the site updates (default).  LQCD_ERR_INVALID_ARG for values outside 0..64. */
lqcd_status lqcd_set_probe_depth(lqcd_ctx *ctx, int depth);

/* The depth lqcd_hop_traces uses (host only; needs no GPU and no context): for an Lx x Ly x Lz x Lt
 * torus (dims[0..3], each in 2..1024), K terms and a fixed depth as lqcd_set_probe_depth sets it
 * (0 = by cost), *depth receives the number of full applications of P per probe.
 * LQCD_ERR_INVALID_ARG for bad arguments. */
lqcd_status lqcd_probe_depth(const int dims[4], int K, int fixed, int *depth);

/* The colour classes lqcd_hop_traces probes with (host only; needs no GPU and no context): for an
 * Lx x Ly x Lz x Lt torus (dims[0..3], each >= 2) and K >= 1 terms, *nclasses receives the class
 * count and, when classes is not NULL, classes[s] (host, V ints; s = x + Lx (y + Ly (z + Lz t)))
 * the class of every site.  Any two sites of one class are more than K hops apart.  Returns
 * LQCD_ERR_INVALID_ARG for bad arguments. */
lqcd_status lqcd_probe_classes(const int dims[4], int K, int *nclasses, int *classes);

/* ---- 1/xi' for HFPS / HFPOLY (Sec. 5.5) ------------------------------------------- */

/* xi[q] = e'_q^dagger gamma_5 tilde M^{-1} e'_q (host out, k complex) with tilde M^{-1} the PS
 * series of K terms (sub = LQCD_SUB_PERT, coeffs ignored) or the POLY polynomial with the n+1 =
 * K host coefficients coeffs (sub = LQCD_SUB_POLY). */
lqcd_status lqcd_xi_inverse(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_defl *defl,
                            int sub, int K, const double *coeffs, double *xi);

/* ---- operator contractions (Sec. 6, Table Table903) ------------------------------ */

/* out[n][op][t] = sum over timeslice t of the density of eta_n^dagger Theta_op w_n (host out,
 * nrhs x 9 x Lt complex), compensated FP64 sums.  Densities: scalar eta^dag w; local
 * eta^dag gamma_mu w; point-split kappa [eta(x+mu)^dag (1+gamma_mu) U_mu(x)^dag w(x)
 * - eta(x)^dag (1-gamma_mu) U_mu(x) w(x+mu)] at base site x. */
lqcd_status lqcd_contract(lqcd_ctx *ctx, const double *links, double kappa, const double *eta,
                          const double *w, int nrhs, double *out);

/* Allocation-free variant of lqcd_contract (the paper has no counterpart; it exists for callers).
 * Some callers cannot allocate device memory: plug-ins whose host application owns every device
 * byte through its own allocator, code running under a hard memory budget, and latency-critical
 * paths where a cudaMalloc (which may synchronise the device) is not acceptable.  This entry point
 * allocates nothing and needs no context:
 * the caller passes the lattice dims (Lx, Ly, Lz, Lt), the device links, eta, w (nrhs fields) and
 * a device output buffer out (nrhs x 9 x Lt complex128, same layout as lqcd_contract), and a
 * cudaStream_t (NULL = legacy default stream).  Partial sums go to a fixed 1 MiB scratch array
 * compiled into the library, which every GPU that loads the library holds until the process exits;
 * it requires nrhs * Lt * 9 <= 65536 and returns LQCD_ERR_INVALID_ARG otherwise (or for bad
 * dims: an extent outside 2..1024 or more than 2^28 sites, the limits of lqcd_ctx_create; or NULL
 * pointers; there is no context, hence no error string).  The first call on each device looks up
 * the scratch array's device address in the current CUDA context, so make it before any stream
 * capture; a call in a new context of that device (after cudaDeviceReset, for instance) looks it up
 * again, so make the first call after a reset before any capture too.  All calls
 * share the one array, which keeps the last call's contents (every entry read is written first by
 * the same call): calls that overlap on the GPU, from any stream or thread, race and must be
 * serialised by the caller.  Asynchronous on the stream; no other call of this library is made. */
lqcd_status lqcd_contract_noalloc(const int dims[4], const double *links, double kappa, const double *eta,
                                  const double *w, int nrhs, double *out, void *stream);

/* ---- whole path: loop estimate on one gauge configuration ----------------------------- */

typedef struct {
  uint64_t seed;      /* noise seed (noises 0 .. nnoise-1; specials 2^32-2 and 2^32-1)       */
  int nnoise;         /* N                                                                   */
  int block;          /* right-hand sides solved together (multi-RHS block width b); 0 = pick
                         it with lqcd_autotune_block among 8, 16, 32, 64 (those <= nnoise)    */
  int m, k;           /* GMRES-DR(m, k) / MINRES-DR(m, k) for the special right-hand side    */
  int m_inner;        /* GMRES cycle length inside GMRES-Proj (m - k if 0)                   */
  int K;              /* PS terms: I .. (kappa P)^{K-1}  ("seventh order" = 7)               */
  int npoly;          /* POLY degree n (n + 1 coefficients)                                  */
  double tol;         /* noise solves: relative true residual                                */
  double tol_special; /* super-convergence tolerance of the special right-hand side         */
  int max_cycles;
  int modes;          /* LQCD_SUB_* bit mask                                                 */
  int prec;           /* LQCD_PREC_F64 (plain) or LQCD_PREC_F32 / F16 / BF16 (mixed-precision
                         noise solves; special solves, series, projections and contractions
                         stay FP64)                                                         */
  double inner_tol;   /* mixed precision: inner relative residual (0 = default, see above)   */
  double eig_tol;     /* special solves: also stop only when the Rayleigh-Ritz residuals of
                         both deflation spaces are <= eig_tol (0 = off; see lqcd_krylov_opts)  */
  int system;         /* LQCD_SYS_M (0): GMRES-DR on M for the noise solves' GMRES-Proj space
                         and MINRES-DR on M' for the HFES eigenpairs; LQCD_SYS_MG5: the Hermitian
                         path, one MINRES-DR on M' for both, every noise solved as
                         M' y = eta by GMRES-Proj over that space and x = gamma_5 y (for fields
                         whose spectrum of M surrounds the origin, where GMRES on M stagnates) */
  int prec_degree;    /* > 0: polynomial preconditioning of the noise solves (and of the special
                         solve that makes their space): the Min-Res polynomial p of degree
                         prec_degree of the solver's operator A (M, or M' on the Hermitian path,
                         real coefficients there) on the polynomial noise; the Krylov methods
                         work on A p(A) (lqcd_krylov_opts.poly_degree).  HFES eigenvalues are then
                         Rayleigh quotients of M' on the Ritz vectors; ES is off.  0 = none     */
  int evenodd;        /* 1: the noise solves run on the even/odd reduced system (Sec. 7; every
                         extent even, plain FP64 only, prec_degree 0): a reduced context of the
                         lattice, its own GMRES-DR (MINRES-DR on hat M gamma_5 on the Hermitian
                         path) space of the special right-hand side for GMRES-Proj, per noise
                         hat M x_e = eta_e + kappa P_eo eta_o to a tolerance that bounds the full
                         relative residual by tol, x_o = eta_o + kappa P_oe x_e, and the full FP64
                         true residual checked.  ES then uses the full eigenpairs of M built from
                         the reduced ones (lqcd_eo_full_eigenpairs).  HFES keeps the MINRES-DR
                         eigenpairs of the full M'.  lqcd_loop_derivs rejects 1.  0 = full system */
} lqcd_est_opts;

typedef struct {
  /* host arrays supplied by the caller (any may be NULL):                                   */
  double *per_noise;  /* [7 modes][nnoise][9 ops] complex: eta^dag Theta (x - tilde x), summed */
  double *per_t;      /* [7][9][Lt] complex: per-timeslice mean over noises of the noise term */
  double *addback;    /* [7][9][Lt] complex: Tr(Theta tilde M^{-1}) per timeslice            */
  double *mean;       /* [7][9] complex: estimate of Tr(Theta M^{-1})                         */
  double *stderr_;    /* [7][9] double: error bar of the signal part (Re scalar, Im vectors)  */
  double *lam;        /* [k] complex: eigenvalues lambda'_q of M' used for deflation          */
  double *poly_a;     /* [npoly+1] complex: Min-Res coefficients                              */
  /* filled by the library:                                                                  */
  long matvecs_setup, matvecs_noise;
  double seconds_setup, seconds_noise;
  double max_true_resid;
  int converged;
  int block;          /* right-hand-side block width used (the autotuner's pick when opts->block == 0) */
} lqcd_estimate;

/* Tr(Theta M^{-1}) for the nine operators and the requested subtraction modes (Sec. 5-7): the
 * setup below, then the noise phase over noises 0 .. nnoise-1, then the summary (mean, error bar). */
lqcd_status lqcd_loop_estimate(lqcd_ctx *ctx, const double *links, double kappa,
                               const lqcd_est_opts *opts, lqcd_estimate *out);

/* ---- the same in two phases: per-configuration setup, then batches of noises ---------------------- */

/* The setup of one gauge configuration (Sec. 5-7, done once and amortised over the noises): the
 * special right-hand side (Z(4) noise 2^32-2) solved by GMRES-DR(m, k) on M (the GMRES-Proj space of
 * the noise solves) and MINRES-DR(m, k) on M' (the Q = k eigenpairs of HFES), the Min-Res
 * coefficients, the hopping traces t_k, 1/xi' for HFPS and HFPOLY, and every add-back.  A setup is
 * also the natural checkpoint: with the counter-based noise, noises can be run in any batches and
 * in any order, on this setup or on one rebuilt with lqcd_loop_setup_from. */
typedef struct lqcd_loop lqcd_loop;
typedef struct {
  /* host arrays supplied by the caller (any may be NULL):                                   */
  double *addback;    /* [7][9][Lt] complex: Tr(Theta tilde M^{-1}) per timeslice            */
  double *lam;        /* [Q] complex: eigenvalues lambda'_q of M' used for deflation          */
  double *poly_a;     /* [npoly+1] complex: Min-Res coefficients                              */
  double *xi_pert;    /* [Q] complex: 1/xi'_q = e'_q^dag gamma_5 tilde M^{-1}_pert e'_q       */
  double *xi_poly;    /* [Q] complex: the same with the POLY polynomial                      */
  /* filled by the library:                                                                  */
  int Q;              /* deflation eigenpairs                                                 */
  int block;          /* right-hand-side block width of the noise solves (autotuned if 0 was asked) */
  long matvecs_setup;
  double seconds_setup;
  double eig_resid_max; /* largest ||M' e - lambda e|| of the deflation eigenpairs (0 if unknown) */
} lqcd_loop_info;
typedef struct {
  long matvecs;        /* operator applications of the noise solves and series               */
  double seconds;      /* wall time of the call                                              */
  double max_true_resid;
  int converged;
  int block;
} lqcd_noise_info;
/* opts as lqcd_loop_estimate (nnoise only bounds the autotuner's candidates).  *out: free with
 * lqcd_loop_destroy.  Returns LQCD_ERR_NOT_CONVERGED only when no deflation space could be made. */
lqcd_status lqcd_loop_setup(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_est_opts *opts,
                            lqcd_loop **out);
/* The same setup from given spaces instead of the special solves: proj, a Krylov space of M
 * (solver-made or lqcd_defl_import_space) for GMRES-Proj; eig, eigenpairs of M' for HFES (any
 * deflation object); a, host npoly+1 complex Min-Res coefficients, or NULL to compute them.  proj
 * and eig are borrowed: they must outlive the setup. */
lqcd_status lqcd_loop_setup_from(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_est_opts *opts,
                                 const lqcd_defl *proj, const lqcd_defl *eig, const double *a, lqcd_loop **out);
/* Noise phase for Z(4) noises first .. first+count-1 of opts->seed (first + count <= 2^32-2):
 * per_noise_t (host, [7][count][9][Lt] complex) receives eta^dag Theta (x - tilde x) summed per
 * timeslice for the modes in opts->modes (zero for the others; add the add-back for the estimate).
 * links: the same gauge field as the setup.  info may be NULL.  LQCD_ERR_NOT_CONVERGED (results
 * still written) when a noise solve stopped at max_cycles above tol. */
lqcd_status lqcd_loop_noises(lqcd_loop *loop, const double *links, uint32_t first, int count, double *per_noise_t,
                             lqcd_noise_info *info);
/* lqcd_loop_noises with the gauge field in host memory (links_host: 4 x V x 3 x 3 complex, the
 * canonical layout; pinned memory makes the copy asynchronous): the call copies it to a device
 * buffer of the context on the context's stream, then runs the noise phase on it.  The end-to-end
 * form of a noise block for callers whose data lives on the host. */
lqcd_status lqcd_loop_noises_host(lqcd_loop *loop, const double *links_host, uint32_t first, int count,
                                  double *per_noise_t, lqcd_noise_info *info);
/* Solver precision of the noise phase from now on (prec, inner_tol as in lqcd_est_opts; the setup
 * itself is FP64 whatever the precision), and its block width (0 keeps the current one). */
lqcd_status lqcd_loop_set_noise_opts(lqcd_loop *loop, int prec, double inner_tol, int block);
/* Cycle length of the noise solves' GMRES-Proj from now on (as lqcd_est_opts.m_inner: 0 = m - k).
 * LQCD_ERR_INVALID_ARG outside 0..1024. */
lqcd_status lqcd_loop_set_inner_restart(lqcd_loop *loop, int m_inner);
/* Outputs of a setup (host), see lqcd_loop_info. */
lqcd_status lqcd_loop_get(const lqcd_loop *loop, lqcd_loop_info *out);
lqcd_status lqcd_loop_destroy(lqcd_loop *loop);

/* ---- batching -------------------------------------------------------------------------- */

/* Autotuner of the right-hand-side block width of the noise solves: for each candidate width b in
 * cand[0..ncand-1] it times, on b Z(4) noises, the marginal cost of one more GMRES-Proj(opts->m)
 * cycle over defl (a call limited to two cycles minus one limited to one, CUDA events on the
 * context's stream, after an untimed warm-up of each width), and picks the width with the least
 * time per right-hand side and cycle.  opts->prec selects the path (plain FP64 or mixed
 * precision); with a mixed precision it then also picks the packed inner operator's right-hand
 * sides per thread (1, 2 or 4 for FP32 fields, 1 or 2 for FP16 / BF16) for that width and keeps it
 * in the context (as lqcd_set_rhs_per_thread).  Outputs (host): *best;
 * seconds[i] = seconds per right-hand side and cycle of cand[i] (may be NULL).  Candidates must be
 * in 1..4096.  Uses the context's stream and synchronises with it. */
lqcd_status lqcd_autotune_block(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_defl *defl,
                                const lqcd_krylov_opts *opts, const int *cand, int ncand, int *best,
                                double *seconds);

/* Replay the fixed launch sequence of each Krylov cycle (its Arnoldi steps) from a CUDA graph,
 * captured on first use and cached per context (default on).  Off, or with device timing on, the
 * same kernels are launched one by one. */
lqcd_status lqcd_set_graphs(lqcd_ctx *ctx, int enable);

/* Gram-Schmidt passes per Arnoldi step of the inner GMRES-Proj cycles of mixed-precision solves
 * (FP32, FP16 or BF16 basis): 2 = classical Gram-Schmidt twice, 1 = once, 0 = by storage (default:
 * one pass for FP16 / BF16 bases, two for FP32).  One pass halves the basis traffic of the inner
 * cycles; the orthogonality it gives up is of the order of the storage rounding of a half-precision
 * basis anyway, and the outer FP64 defect correction still stops on the FP64 true residual, so only
 * the inner convergence rate can change (measured on 24^3 x 32 at kappa 0.157: the same matvecs
 * per noise, 1.4 x faster).  FP64 Krylov solves always use two passes.  LQCD_ERR_INVALID_ARG for
 * other values. */
lqcd_status lqcd_set_inner_gs_passes(lqcd_ctx *ctx, int passes);

/* Lanczos window of the inner GMRES-Proj cycles of mixed-precision solves on the Hermitian operator
 * M' = M gamma_5 (the Hermitian path; other operators ignore it): window w >= 2 orthogonalises each
 * new basis vector only against the last w vectors.  For a Hermitian operator the Arnoldi
 * recurrence is the three-term Lanczos one (MINRES-DR on M', Sec. 8), so w = 2 drops only inner
 * products that vanish in exact arithmetic; the Arnoldi relation A V_m = V_{m+1} Hbar_m still holds
 * by construction, the cycle's least-squares step becomes quasi-minimal where the reduced-precision
 * basis loses orthogonality, and the outer FP64 defect correction still stops on the FP64 true
 * residual.  0 = every vector (default).  LQCD_ERR_INVALID_ARG for 1 or values above 1024. */
lqcd_status lqcd_set_inner_window(lqcd_ctx *ctx, int window);

/* Loop estimates of n independent problems (lattices of any, uneven, sizes), run concurrently: each
 * context (all distinct) works on its own private stream from its own host thread, ordered after
 * the work already queued on its stream (links ready there) and before the work queued there
 * later.  links[i], kappas[i], opts[i], out[i] as lqcd_loop_estimate on ctxs[i]; status[i]
 * receives each problem's status (host array).  Returns LQCD_OK when every problem returned
 * LQCD_OK, otherwise the first failing status. */
lqcd_status lqcd_batch_loop_estimate(int n, lqcd_ctx *const *ctxs, const double *const *links, const double *kappas,
                                     const lqcd_est_opts *opts, lqcd_estimate *out, int *status);

/* ---- derivatives (an addition: the paper has no derivatives) ------------ */

/* Link gradient of scalar noise estimates T_n = eta_n^dag M^{-1} eta_n from x_n = M^{-1} eta_n and
 * z_n = M^{-dag} eta_n (device, nrhs fields each).  Accumulates (+=) scale * sum_n into
 *   grad[mu][s][a]  (device, 4 x V x 8 complex): dT/dw_a under U_mu(s) -> exp(i w lambda_a/2) U_mu(s),
 *                   lambda_a the Gell-Mann matrices: (i kappa / 2) tr(lambda_a B) with
 *                   B = sum_spin [(1-g_mu) U x(s+mu)] z(s)^dag - [(1+g_mu) x(s)] (U z(s+mu))^dag;
 *   grad_links (device, 4 x V x 3 x 3 complex, may be NULL): dT/dU* + conj(dT/dU), the gradient of
 *                   Re T with respect to the complex link entries in torch's convention. */
lqcd_status lqcd_link_grad(lqcd_ctx *ctx, const double *links, double kappa, const double *z, const double *x,
                           int nrhs, double scale, double *grad, double *grad_links);

typedef struct {
  double grad_scale;  /* in: factor applied to link_grad / grad_links (e.g. an upstream gradient)   */
  double *dkappa;     /* host [2 modes: NS, PS][9 ops] complex: mean d Tr(Theta M^{-1}) / dkappa   */
  double *dkappa_err; /* host [2][9]: error bar of the signal part (Re scalar, Im vectors)          */
  double *per_noise;  /* host [2][nnoise][9] complex                                                 */
  double *link_grad;  /* device [4][V][8] complex, or NULL: mean over noises of the NS scalar dT/dw  */
  double *grad_links; /* device [4][V][3][3] complex, or NULL (needs link_grad): torch-convention   */
  long matvecs;
  double seconds;
  double max_true_resid;
  int converged;
} lqcd_derivs;

/* d Tr(Theta M^{-1}) / dkappa for the nine operators with no subtraction (NS) and with
 * perturbative subtraction (PS, opts->K terms, differentiated term by term), and the gradient of
 * the NS scalar estimate with respect to every link.  Per noise three solves run (x = M^{-1} eta,
 * y = M^{-1} P x, and the adjoint w = M^{-1} g5 eta, z = g5 w) with GMRES-Proj over a GMRES-DR
 * space of the special right-hand side (or, with opts->system = LQCD_SYS_MG5, over a MINRES-DR
 * space of M' with every solve done as M' y = b, x = gamma_5 y), to opts->tol (opts->prec selects
 * plain FP64 or mixed precision); nothing is kept from a previous call.  Uses opts seed, nnoise,
 * block, m, k, m_inner, K, tol, tol_special, max_cycles, prec, eig_tol, system. */
lqcd_status lqcd_loop_derivs(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_est_opts *opts,
                             lqcd_derivs *out);

/* ---- even/odd preconditioning (Sec. 7) ------------------------------------------------------
 * With every extent even and a site's parity (x + y + z + t) mod 2, P couples only opposite
 * parities; eliminating the odd sites leaves the reduced matrix on the even sites
 *   hat M = 1 - kappa^2 P_eo P_oe,  hat M x_e = b_e + kappa P_eo b_o,  x_o = b_o + kappa P_oe x_e.
 * A reduced field holds the sites of one parity in lexicographic order of the full site index
 * (compact index s >> 1): [nrhs][V/2][spin 4][colour 3] complex128.  Links stay the full
 * [mu][V][3][3] array. */

/* Create a reduced context for the even sites of an Lx x Ly x Lz x Lt lattice (every extent even,
 * 2..1024, at most 2^28 sites).  Its fields have 12 V/2 complex entries, and on it
 * lqcd_wilson_apply applies hat M (LQCD_APPLY_M), hat M gamma_5 (LQCD_APPLY_G5R; Hermitian),
 * hat M^dag = gamma_5 hat M gamma_5 (LQCD_APPLY_DAG) or P_eo P_oe (LQCD_APPLY_HOP), in FP64 or FP32
 * arithmetic, and lqcd_gmresdr_solve / lqcd_minresdr_solve / lqcd_proj_solve (plain precision) and
 * lqcd_deflate_project solve and deflate the reduced system.  Entry points that need the full
 * lattice (noise, contractions, traces, loop estimates, packed and mixed-precision operators)
 * return LQCD_ERR_INVALID_ARG on it.  Destroy with lqcd_ctx_destroy. */
lqcd_status lqcd_ctx_create_evenodd(lqcd_ctx **ctx, const int dims[4], int link_recon, void *stream);

/* Split nrhs full fields into their even and odd halves (either output may be NULL), or join them
 * back.  Device pointers; outputs must not overlap inputs. */
lqcd_status lqcd_eo_split(lqcd_ctx *ctx, const double *full, double *even, double *odd, int nrhs);
lqcd_status lqcd_eo_join(lqcd_ctx *ctx, const double *even, const double *odd, double *full, int nrhs);

/* out = P_eo in (parity_out = 0: in odd, out even) or P_oe in (parity_out = 1), reduced fields. */
lqcd_status lqcd_eo_hop(lqcd_ctx *ctx, const double *links, const double *in, double *out, int nrhs, int parity_out);

/* Reduced right-hand side be = b_e + kappa P_eo b_o of nrhs full fields b. */
lqcd_status lqcd_eo_rhs(lqcd_ctx *ctx, const double *links, double kappa, const double *b, double *be, int nrhs);

/* Full solution x (nrhs full fields) from the reduced one: x_e = xe, x_o = b_o + kappa P_oe x_e. */
lqcd_status lqcd_eo_reconstruct(lqcd_ctx *ctx, const double *links, double kappa, const double *xe, const double *b,
                                double *x, int nrhs);

/* Full eigenpairs of M from Q reduced eigenpairs (mu_q, v_e^(q)) of hat M: if M v = lambda v then
 * hat M v_e = mu v_e with mu = 1 - (1 - lambda)^2, so each reduced pair gives the two full pairs
 * 1 - lambda = +-sqrt(1 - mu) (principal root; + first), v = (v_e, kappa P_oe v_e / (1 - lambda))
 * normalised to unit length.  mu: host Q complex; Ve: device Q reduced fields; lam: host 2Q
 * complex out; E: device 2Q full fields out.  LQCD_ERR_INVALID_ARG when some |sqrt(1 - mu)| <= tol
 * (lambda = 1: the odd half is undefined).  Synchronises the context's stream. */
lqcd_status lqcd_eo_full_eigenpairs(lqcd_ctx *ctx, const double *links, double kappa, const double *mu,
                                    const double *Ve, int Q, double tol, double *lam, double *E);


#ifdef __cplusplus
}
#endif
#endif /* LQCD_H */
