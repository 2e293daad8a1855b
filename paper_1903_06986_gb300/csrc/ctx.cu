// Context lifetime, error reporting and workspace management of liblqcd.
#include <cstdarg>
#include <cstring>

#include "common.cuh"

lqcd_status set_err(lqcd_ctx *ctx, lqcd_status st, const char *fmt, ...) {
  if (ctx) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return st;
}

static lqcd_status timing_collect(lqcd_ctx *ctx);

static int next_event(lqcd_ctx *ctx) {
  if (ctx->ev_used == (int)ctx->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    ctx->ev_pool.push_back(e);
  }
  return ctx->ev_used++;
}

void kbegin(lqcd_ctx *ctx) {
  ctx->pending_start = -1;
  if (!ctx->timing) return;
  const int i = next_event(ctx);
  if (i >= 0 && cudaEventRecord(ctx->ev_pool[i], ctx->stream) == cudaSuccess) ctx->pending_start = i;
}

lqcd_status launch_check(lqcd_ctx *ctx, const char *what, int cls, double units) {
  return launch_check_bytes(ctx, what, cls, units, 0.0);
}

lqcd_status launch_check_bytes(lqcd_ctx *ctx, const char *what, int cls, double units, double bytes) {
  ctx->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_err(ctx, LQCD_ERR_CUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
  if (ctx->timing && ctx->pending_start >= 0) {
    const int j = next_event(ctx);
    if (j >= 0 && cudaEventRecord(ctx->ev_pool[j], ctx->stream) == cudaSuccess)
      ctx->timed.push_back(TimedLaunch{ctx->pending_start, j, cls, units, bytes});
    ctx->pending_start = -1;
    if (ctx->timed.size() >= 16384) return timing_collect(ctx);  // bound the event pool
  }
  return LQCD_OK;
}

// fold recorded launch times into the per-class totals and recycle the events
static lqcd_status timing_collect(lqcd_ctx *ctx) {
  if (ctx->timed.empty()) {
    ctx->ev_used = 0;
    return LQCD_OK;
  }
  LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (const TimedLaunch &t : ctx->timed) {
    float ms = 0.f;
    LQCD_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev_pool[t.start], ctx->ev_pool[t.end]));
    ctx->t_ms[t.cls] += ms;
    ctx->t_count[t.cls] += 1;
    ctx->t_units[t.cls] += t.units;
    ctx->t_bytes[t.cls] += t.bytes;
  }
  ctx->timed.clear();
  ctx->ev_used = 0;
  return LQCD_OK;
}

lqcd_status ws_get(lqcd_ctx *ctx, int slot, size_t bytes, void **ptr) {
  if (slot < 0 || slot >= WS_NSLOTS) return set_err(ctx, LQCD_ERR_INVALID_ARG, "bad workspace slot %d", slot);
  if (bytes == 0) bytes = 16;
  if (ctx->ws_size[slot] < bytes) {
    graph_cache_clear(ctx);  // captured graphs hold the old addresses
    if (ctx->ws_ptr[slot]) {
      // the old buffer may still be read by queued work
      cudaError_t e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) return set_err(ctx, LQCD_ERR_CUDA, "sync before workspace growth: %s", cudaGetErrorString(e));
      cudaFree(ctx->ws_ptr[slot]);
      ctx->ws_ptr[slot] = nullptr;
      ctx->ws_size[slot] = 0;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_err(ctx, LQCD_ERR_OOM, "workspace slot %d: cudaMalloc(%zu) failed: %s", slot, bytes, cudaGetErrorString(e));
    }
    ctx->ws_ptr[slot] = p;
    ctx->ws_size[slot] = bytes;
  }
  *ptr = ctx->ws_ptr[slot];
  return LQCD_OK;
}

void graph_cache_clear(lqcd_ctx *ctx) {
  if (ctx->graph_cache.empty()) return;
  cudaStreamSynchronize(ctx->stream);
  for (auto &g : ctx->graph_cache) cudaGraphExecDestroy(g.exec);
  ctx->graph_cache.clear();
}

lqcd_status graph_cached(lqcd_ctx *ctx, const std::string &key, lqcd_status (*enqueue)(void *), void *arg) {
  if (!ctx->graphs || ctx->timing) return enqueue(arg);
  for (auto &g : ctx->graph_cache)
    if (g.key == key) {
      LQCD_CUDA(ctx, cudaGraphLaunch(g.exec, ctx->stream));
      ctx->launches += g.nlaunch;
      return LQCD_OK;
    }
  cudaStream_t user = ctx->stream;
  LQCD_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
  ctx->stream = ctx->cap_stream;
  const long l0 = ctx->launches;
  const lqcd_status st = enqueue(arg);
  ctx->stream = user;
  const long nl = ctx->launches - l0;
  ctx->launches = l0;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
  if (st != LQCD_OK) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return st;
  }
  if (e != cudaSuccess || !g) {
    cudaGetLastError();
    return set_err(ctx, LQCD_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
  }
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, LQCD_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
  }
  if (ctx->graph_cache.size() >= 32) {
    cudaStreamSynchronize(ctx->stream);
    cudaGraphExecDestroy(ctx->graph_cache.front().exec);
    ctx->graph_cache.erase(ctx->graph_cache.begin());
  }
  ctx->graph_cache.push_back(lqcd_ctx::GraphEntry{key, ex, nl});
  LQCD_CUDA(ctx, cudaGraphLaunch(ex, ctx->stream));
  ctx->launches += nl;
  return LQCD_OK;
}

lqcd_status host_stage(lqcd_ctx *ctx, size_t bytes, double **ptr) {
  if (ctx->host_pinned_size < bytes) {
    if (ctx->host_pinned) {
      cudaError_t e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) return set_err(ctx, LQCD_ERR_CUDA, "sync before staging growth: %s", cudaGetErrorString(e));
      cudaFreeHost(ctx->host_pinned);
      ctx->host_pinned = nullptr;
      ctx->host_pinned_size = 0;
    }
    void *p = nullptr;
    cudaError_t e = cudaMallocHost(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_err(ctx, LQCD_ERR_OOM, "pinned staging of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    ctx->host_pinned = (double *)p;
    ctx->host_pinned_size = bytes;
  }
  *ptr = ctx->host_pinned;
  return LQCD_OK;
}

extern "C" {

const char *lqcd_version(void) { return "lqcd-gb300 0.1 (sm_103a)"; }

lqcd_status lqcd_ctx_create(lqcd_ctx **out, const int dims[4], int link_recon, void *stream) {
  if (!out || !dims) return LQCD_ERR_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < 4; ++i)
    if (dims[i] < 2 || dims[i] > 1024) return LQCD_ERR_INVALID_ARG;
  if (link_recon != 18 && link_recon != 12) return LQCD_ERR_INVALID_ARG;
  long long V = (long long)dims[0] * dims[1] * dims[2] * dims[3];
  if (V > (1LL << 28)) return LQCD_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return LQCD_ERR_CUDA; }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) { cudaGetLastError(); return LQCD_ERR_CUDA; }
  lqcd_ctx *c = new lqcd_ctx();
  memcpy(c->dims, dims, sizeof(int) * 4);
  c->V = (int)V;
  c->N = 12 * V;
  c->device = dev;
  c->recon = link_recon;
  c->sms = prop.multiProcessorCount;
  c->stream = (cudaStream_t)stream;
  c->launches = 0;
  c->ws_ptr.assign(WS_NSLOTS, nullptr);
  c->ws_size.assign(WS_NSLOTS, 0);
  c->host_pinned = nullptr;
  c->host_pinned_size = 0;
  c->timing = false;
  c->pending_start = -1;
  c->ev_used = 0;
  for (int k = 0; k < K_NCLASS; ++k) {
    c->t_ms[k] = 0.0;
    c->t_count[k] = 0;
    c->t_units[k] = 0.0;
    c->t_bytes[k] = 0.0;
  }
  c->graphs = true;
  c->packed_nr = 0;
  c->defl_engine = LQCD_DEFL_FP64;
  c->tc_wait_ns = 2000000000ull;
  c->tc_stop_after = -1;
  c->inner_gs_passes = 0;
  c->probe_depth = 0;
  c->inner_window = 0;
  c->eo = 0;
  for (int i = 0; i < 4; ++i) c->eo_dims[i] = dims[i];
  c->cap_stream = nullptr;
  c->run_stream = nullptr;
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->run_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
    return LQCD_ERR_CUDA;
  }
  *out = c;
  return LQCD_OK;
}

lqcd_status lqcd_ctx_destroy(lqcd_ctx *ctx) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  cudaStreamSynchronize(ctx->stream);
  graph_cache_clear(ctx);
  cudaStreamSynchronize(ctx->run_stream);
  cudaStreamDestroy(ctx->cap_stream);
  cudaStreamDestroy(ctx->run_stream);
  for (void *p : ctx->ws_ptr)
    if (p) cudaFree(p);
  if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  delete ctx;
  return LQCD_OK;
}

lqcd_status lqcd_set_stream(lqcd_ctx *ctx, void *stream) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  ctx->stream = (cudaStream_t)stream;
  return LQCD_OK;
}

const char *lqcd_last_error_string(const lqcd_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

lqcd_status lqcd_set_graphs(lqcd_ctx *ctx, int enable) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  ctx->graphs = enable != 0;
  if (!ctx->graphs) graph_cache_clear(ctx);
  return LQCD_OK;
}

lqcd_status lqcd_set_inner_gs_passes(lqcd_ctx *ctx, int passes) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  if (passes < 0 || passes > 2) return set_err(ctx, LQCD_ERR_INVALID_ARG, "set_inner_gs_passes: passes must be 0, 1 or 2");
  if (passes != ctx->inner_gs_passes) graph_cache_clear(ctx);
  ctx->inner_gs_passes = passes;
  return LQCD_OK;
}

lqcd_status lqcd_set_inner_window(lqcd_ctx *ctx, int window) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  if (window != 0 && (window < 2 || window > 1024))
    return set_err(ctx, LQCD_ERR_INVALID_ARG, "set_inner_window: window must be 0 or in 2..1024");
  if (window != ctx->inner_window) graph_cache_clear(ctx);
  ctx->inner_window = window;
  return LQCD_OK;
}

lqcd_status lqcd_set_probe_depth(lqcd_ctx *ctx, int depth) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  if (depth < 0 || depth > 64) return set_err(ctx, LQCD_ERR_INVALID_ARG, "set_probe_depth: depth must be in 0..64");
  ctx->probe_depth = depth;
  return LQCD_OK;
}

long lqcd_kernel_launches(const lqcd_ctx *ctx) { return ctx ? ctx->launches : -1; }

lqcd_status lqcd_timing_enable(lqcd_ctx *ctx, int enable) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  if (!enable) LQCD_TRY(timing_collect(ctx));
  ctx->timing = enable != 0;
  return LQCD_OK;
}

lqcd_status lqcd_timing_reset(lqcd_ctx *ctx) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  LQCD_TRY(timing_collect(ctx));
  for (int k = 0; k < K_NCLASS; ++k) {
    ctx->t_ms[k] = 0.0;
    ctx->t_count[k] = 0;
    ctx->t_units[k] = 0.0;
    ctx->t_bytes[k] = 0.0;
  }
  return LQCD_OK;
}

lqcd_status lqcd_timing_read(lqcd_ctx *ctx, int cls, double *total_ms, long *launches, double *units) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  if (cls < 0 || cls >= K_NCLASS || !total_ms || !launches) return set_err(ctx, LQCD_ERR_INVALID_ARG, "timing_read: bad class");
  LQCD_TRY(timing_collect(ctx));
  *total_ms = ctx->t_ms[cls];
  *launches = ctx->t_count[cls];
  if (units) *units = ctx->t_units[cls];
  return LQCD_OK;
}

lqcd_status lqcd_timing_bytes(lqcd_ctx *ctx, int cls, double *bytes) {
  if (!ctx) return LQCD_ERR_INVALID_ARG;
  if (cls < 0 || cls >= K_NCLASS || !bytes) return set_err(ctx, LQCD_ERR_INVALID_ARG, "timing_bytes: bad class");
  LQCD_TRY(timing_collect(ctx));
  *bytes = ctx->t_bytes[cls];
  return LQCD_OK;
}

}  // extern "C"
