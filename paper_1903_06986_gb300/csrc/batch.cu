// Batching: the autotuner of the right-hand-side block width (and of the packed operator's
// right-hand sides per thread), and concurrent loop estimates of several lattices of uneven size.
//
// Within one problem the multi-right-hand-side kernels already batch the noises of a block, and
// the Arnoldi steps of a Krylov cycle run as one cached CUDA graph (krylov.cu).  Across problems
// each context runs on its own private stream from its own host thread, so the small kernels of
// small lattices overlap on the GPU instead of queueing behind each other.
#include <algorithm>
#include <thread>

#include "common.cuh"

lqcd_status proj_core_entry(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_defl *defl, const double2 *b,
                            double2 *x, int nrhs, const lqcd_krylov_opts *o, lqcd_solve_info *info);

namespace {

// device seconds of f() on the context's stream
template <typename F>
lqcd_status timed(lqcd_ctx *ctx, F &&f, double *sec) {
  cudaEvent_t e0, e1;
  LQCD_CUDA(ctx, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    cudaEventDestroy(e0);
    return set_err(ctx, LQCD_ERR_CUDA, "autotune: event creation failed");
  }
  struct G {
    cudaEvent_t a, b;
    ~G() { cudaEventDestroy(a); cudaEventDestroy(b); }
  } g{e0, e1};
  LQCD_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
  LQCD_TRY(f());
  LQCD_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
  LQCD_CUDA(ctx, cudaEventSynchronize(e1));
  float ms = 0.f;
  LQCD_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
  *sec = ms * 1e-3;
  return LQCD_OK;
}

// one GMRES-Proj call limited to `cycles` cycles; not converging is the expected outcome
lqcd_status proj_cycles(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_defl *defl, const double2 *b,
                        double2 *x, int nb, const lqcd_krylov_opts *o, int cycles) {
  lqcd_krylov_opts c = *o;
  c.tol = 1e-300;
  c.max_cycles = cycles;
  lqcd_solve_info si{};
  const lqcd_status st = proj_core_entry(ctx, links, kappa, defl, b, x, nb, &c, &si);
  return st == LQCD_ERR_NOT_CONVERGED ? LQCD_OK : st;
}

}  // namespace

lqcd_status autotune_block(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_defl *defl,
                           const lqcd_krylov_opts *o, const int *cand, int ncand, int *best, double *seconds) {
  int bmax = 0;
  for (int i = 0; i < ncand; ++i) {
    if (cand[i] < 1 || cand[i] > 4096) return set_err(ctx, LQCD_ERR_INVALID_ARG, "autotune: candidate %d out of range", cand[i]);
    bmax = std::max(bmax, cand[i]);
  }
  double2 *b, *x;
  LQCD_TRY(ws_get(ctx, WS_TUNE, sizeof(double2) * (size_t)ctx->N * bmax * 2, (void **)&b));
  x = b + (size_t)ctx->N * bmax;
  LQCD_TRY(noise_launch(ctx, 0x5eedULL, 0u, bmax, b));
  double best_t = 0.0;
  for (int i = 0; i < ncand; ++i) {
    const int nb = cand[i];
    double t1 = 0.0, t2 = 0.0;
    LQCD_TRY(proj_cycles(ctx, links, kappa, defl, b, x, nb, o, 2));  // warm-up: workspace, graphs
    LQCD_TRY(timed(ctx, [&] { return proj_cycles(ctx, links, kappa, defl, b, x, nb, o, 1); }, &t1));
    LQCD_TRY(timed(ctx, [&] { return proj_cycles(ctx, links, kappa, defl, b, x, nb, o, 2); }, &t2));
    // marginal cost of a cycle; the one-cycle time where timing noise made the difference negative
    const double per = (t2 > t1 ? t2 - t1 : t1) / nb;
    if (seconds) seconds[i] = per;
    if (i == 0 || per < best_t) {
      best_t = per;
      *best = nb;
    }
  }
  if (o->prec != LQCD_PREC_F64) {
    // right-hand sides per thread of the packed inner operator at the chosen width: 1, 2 (paired
    // lanes), 3 (paired lanes, asynchronously staged) or 4 for FP32 fields, 1, 2 or 3 for FP16 / BF16
    float4 *Up, *in, *out;
    const int recon = ctx->recon, nb = *best;
    const size_t fl = (size_t)ctx->V * 24 * nb;  // floats of nb packed FP32 fields
    LQCD_TRY(ws_get(ctx, WS_MIX_U, sizeof(float) * (size_t)ctx->V * 4 * (recon == 12 ? 12 : 20), (void **)&Up));
    LQCD_TRY(ws_get(ctx, WS_TMP2, sizeof(float) * fl * 2, (void **)&in));
    out = in + fl / 4;
    LQCD_TRY(pack_links_f32(ctx, (const double2 *)links, Up, recon));
    if (o->prec == LQCD_PREC_F32) {
      LQCD_TRY(pack_f32(ctx, b, nullptr, in, nb));
    } else if (o->prec == LQCD_PREC_F16) {
      LQCD_TRY(pack_lp(ctx, b, nullptr, (__half2 *)in, nb));
    } else {
      LQCD_TRY(pack_lp(ctx, b, nullptr, (__nv_bfloat162 *)in, nb));
    }
    const int saved = ctx->packed_nr;
    double tb = 0.0;
    int nr_best = 1;
    for (int nr : {1, 2, 3, 4}) {
      if ((nr > 1 && nb < 2) || (nr == 4 && (nb < 4 || o->prec != LQCD_PREC_F32))) continue;
      ctx->packed_nr = nr;
      auto f = [&] {
        for (int rep = 0; rep < 3; ++rep) {
          if (o->prec == LQCD_PREC_F32) {
            LQCD_TRY(wilson_launch_packed(ctx, Up, recon, kappa, in, out, nb, LQCD_APPLY_M, nr));
          } else if (o->prec == LQCD_PREC_F16) {
            LQCD_TRY(wilson_launch_packed_lp(ctx, Up, recon, kappa, (const __half2 *)in, (__half2 *)out, nb, LQCD_APPLY_M));
          } else {
            LQCD_TRY(wilson_launch_packed_lp(ctx, Up, recon, kappa, (const __nv_bfloat162 *)in, (__nv_bfloat162 *)out, nb,
                                             LQCD_APPLY_M));
          }
        }
        return LQCD_OK;
      };
      double t = 0.0;
      lqcd_status st = f();
      if (st == LQCD_OK) st = timed(ctx, f, &t);
      if (st != LQCD_OK) {
        ctx->packed_nr = saved;
        return st;
      }
      if (nr == 1 || t < tb) {
        tb = t;
        nr_best = nr;
      }
    }
    if (nr_best != saved) graph_cache_clear(ctx);
    ctx->packed_nr = nr_best;
  }
  return LQCD_OK;
}

extern "C" lqcd_status lqcd_autotune_block(lqcd_ctx *ctx, const double *links, double kappa, const lqcd_defl *defl,
                                           const lqcd_krylov_opts *opts, const int *cand, int ncand, int *best,
                                           double *seconds) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(require_full(ctx, "autotune_block"));
  if (!links || !defl || !opts || !cand || ncand < 1 || !best)
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "autotune_block: bad arguments");
  if (!defl->V || !defl->Hbar_dev) return set_err(ctx, LQCD_ERR_INVALID_ARG, "autotune_block: needs a solver-made deflation space");
  return autotune_block(ctx, links, kappa, defl, opts, cand, ncand, best, seconds);
}

extern "C" lqcd_status lqcd_batch_loop_estimate(int n, lqcd_ctx *const *ctxs, const double *const *links,
                                                const double *kappas, const lqcd_est_opts *opts, lqcd_estimate *out,
                                                int *status) {
  if (n < 1 || !ctxs || !links || !kappas || !opts || !out || !status) return LQCD_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return LQCD_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return set_err(ctxs[i], LQCD_ERR_INVALID_ARG, "batch_loop_estimate: contexts must be distinct");
  }
  // move every problem onto its private stream, after the work already queued on its own
  std::vector<cudaStream_t> user(n);
  std::vector<cudaEvent_t> ev(n, nullptr);
  for (int i = 0; i < n; ++i) {
    lqcd_ctx *c = ctxs[i];
    user[i] = c->stream;
    if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ev[i], c->stream) != cudaSuccess || cudaStreamWaitEvent(c->run_stream, ev[i], 0) != cudaSuccess) {
      cudaGetLastError();
      for (int j = 0; j <= i; ++j) {
        if (ev[j]) cudaEventDestroy(ev[j]);
        ctxs[j]->stream = user[j];
      }
      return set_err(c, LQCD_ERR_CUDA, "batch_loop_estimate: stream ordering failed");
    }
    c->stream = c->run_stream;
  }
  std::vector<std::thread> th;
  th.reserve(n);
  for (int i = 0; i < n; ++i)
    th.emplace_back([&, i] {
      cudaSetDevice(ctxs[i]->device);
      status[i] = lqcd_loop_estimate(ctxs[i], links[i], kappas[i], &opts[i], &out[i]);
    });
  for (auto &t : th) t.join();
  lqcd_status first = LQCD_OK;
  for (int i = 0; i < n; ++i) {
    lqcd_ctx *c = ctxs[i];
    // work queued later on the caller's stream waits for this problem
    if (cudaEventRecord(ev[i], c->run_stream) != cudaSuccess || cudaStreamWaitEvent(user[i], ev[i], 0) != cudaSuccess) {
      cudaGetLastError();
      cudaStreamSynchronize(c->run_stream);
    }
    cudaEventDestroy(ev[i]);
    c->stream = user[i];
    if (first == LQCD_OK && status[i] != LQCD_OK) first = (lqcd_status)status[i];
  }
  return first;
}
