// ctx.cu -- context, workspace and status handling of the libslqr C ABI.
#include "slqr_internal.cuh"

#include <vector>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <new>

namespace slqr {

slqr_status fail(slqr_ctx *ctx, slqr_status st, const char *fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->last_error = buf;
  }
  return st;
}

slqr_status check_launch(slqr_ctx *ctx, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  return SLQR_OK;
}

static slqr_status grow(slqr_ctx *ctx, Workspace &ws, size_t bytes);

#ifdef SLQR_CHECKED
// Checked build: every workspace is followed by a guard zone of this byte
// pattern, and its contents are NaN bytes (0xFF) each time an entry point
// takes it, so that a read of anything not written first shows up as NaN
// in the results and a write past the end shows up at the next check.
constexpr size_t kGuardBytes = 64 * 1024;
constexpr unsigned char kGuardByte = 0xA5;

static slqr_status check_guard(slqr_ctx *ctx, const Workspace &ws) {
  if (!ws.ptr) return SLQR_OK;
  std::vector<unsigned char> g(kGuardBytes);
  cudaError_t e = cudaMemcpy(g.data(), (char *)ws.ptr + ws.bytes, kGuardBytes, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "guard zone: %s", cudaGetErrorString(e));
  for (size_t i = 0; i < kGuardBytes; ++i)
    if (g[i] != kGuardByte)
      return fail(ctx, SLQR_ECHECK, "workspace guard zone overwritten at byte %zu past the end", i);
  return SLQR_OK;
}

static slqr_status poison(slqr_ctx *ctx, Workspace &ws) {
  cudaError_t e = cudaDeviceSynchronize();             // (work still using it)
  if (e == cudaSuccess) e = cudaMemset(ws.ptr, 0xFF, ws.bytes);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "poison: %s", cudaGetErrorString(e));
  return SLQR_OK;
}
#endif

slqr_status ensure_workspace(slqr_ctx *ctx, size_t bytes) { return grow(ctx, ctx->ws, bytes); }
slqr_status ensure_workspace2(slqr_ctx *ctx, size_t bytes) { return grow(ctx, ctx->ws2, bytes); }

slqr_status check_workspaces(slqr_ctx *ctx) {
#ifdef SLQR_CHECKED
  slqr_status st = check_guard(ctx, ctx->ws);
  if (st == SLQR_OK) st = check_guard(ctx, ctx->ws2);
  return st;
#else
  (void)ctx;
  return SLQR_OK;
#endif
}

static slqr_status grow(slqr_ctx *ctx, Workspace &ws, size_t bytes) {
#ifdef SLQR_CHECKED
  if (bytes <= ws.bytes) {
    slqr_status st = check_guard(ctx, ws);
    return st == SLQR_OK ? poison(ctx, ws) : st;
  }
  if (ws.ptr) {
    slqr_status st = check_guard(ctx, ws);
    if (st != SLQR_OK) return st;
  }
#else
  if (bytes <= ws.bytes) return SLQR_OK;
#endif
  bytes = align_up(bytes, (size_t)1 << 20);
  if (ctx->hbm_budget && bytes > ctx->hbm_budget)
    return fail(ctx, SLQR_EBUSY, "workspace of %zu bytes exceeds the HBM budget %zu", bytes,
                ctx->hbm_budget);
  if (ws.ptr) {
    // the old workspace may still be in use by enqueued work
    cudaDeviceSynchronize();
    cudaFree(ws.ptr);
    ws.ptr = nullptr;
    ws.bytes = 0;
  }
  void *p = nullptr;
#ifdef SLQR_CHECKED
  cudaError_t e = cudaMalloc(&p, bytes + kGuardBytes);
#else
  cudaError_t e = cudaMalloc(&p, bytes);
#endif
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, SLQR_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  ws.ptr = p;
  ws.bytes = bytes;
#ifdef SLQR_CHECKED
  e = cudaMemset((char *)p + bytes, kGuardByte, kGuardBytes);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "guard zone: %s", cudaGetErrorString(e));
  return poison(ctx, ws);
#else
  return SLQR_OK;
#endif
}

static cudaEvent_t take_event(slqr_ctx *ctx) {
  if (!ctx->prof.free_events.empty()) {
    cudaEvent_t e = ctx->prof.free_events.back();
    ctx->prof.free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

int prof_begin(slqr_ctx *ctx, cudaStream_t stream) {
  if (!ctx->prof.on) return -1;
  ProfRecord r;
  r.start = take_event(ctx);
  r.stop = take_event(ctx);
  r.kid = -1;
  r.flops = 0;
  if (!r.start || !r.stop) return -1;
  cudaEventRecord(r.start, stream);
  ctx->prof.pending.push_back(r);
  return (int)ctx->prof.pending.size() - 1;
}

void prof_end(slqr_ctx *ctx, cudaStream_t stream, int slot, int kid, double flops) {
  ++ctx->launch_count;
  if (slot < 0) return;
  ProfRecord &r = ctx->prof.pending[slot];
  cudaEventRecord(r.stop, stream);
  r.kid = kid;
  r.flops = flops;
}

// Fold finished records into the totals (waits for their stop events).
static void prof_collect(slqr_ctx *ctx) {
  for (ProfRecord &r : ctx->prof.pending) {
    float ms = 0.f;
    if (r.kid >= 0 && cudaEventSynchronize(r.stop) == cudaSuccess &&
        cudaEventElapsedTime(&ms, r.start, r.stop) == cudaSuccess) {
      ctx->prof.ms[r.kid] += ms;
      ctx->prof.launches[r.kid] += 1;
      ctx->prof.flops[r.kid] += r.flops;
    }
    cudaGetLastError();
    ctx->prof.free_events.push_back(r.start);
    ctx->prof.free_events.push_back(r.stop);
  }
  ctx->prof.pending.clear();
}

}  // namespace slqr

using namespace slqr;

extern "C" int slqr_profile(slqr_ctx *ctx, int enable) {
  if (!ctx) return SLQR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  prof_collect(ctx);
  if (enable) {
    for (int k = 0; k < kNumKernelIds; ++k) {
      ctx->prof.ms[k] = 0;
      ctx->prof.launches[k] = 0;
      ctx->prof.flops[k] = 0;
    }
  }
  ctx->prof.on = enable != 0;
  return SLQR_OK;
}

extern "C" slqr_status slqr_profile_read(slqr_ctx *ctx, int kernel, double *ms,
                                         long long *launches, double *flops) {
  if (!ctx || kernel < 0 || kernel >= kNumKernelIds) return SLQR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  prof_collect(ctx);
  if (ms) *ms = ctx->prof.ms[kernel];
  if (launches) *launches = ctx->prof.launches[kernel];
  if (flops) *flops = ctx->prof.flops[kernel];
  return SLQR_OK;
}

extern "C" long long slqr_launch_count(slqr_ctx *ctx) {
  if (!ctx) return -1;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  return ctx->launch_count;
}

extern "C" slqr_status slqr_create(slqr_ctx **out, int device, size_t hbm_budget_bytes) {
  if (!out) return SLQR_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return SLQR_EINVAL;
  }
  slqr_ctx *ctx = new (std::nothrow) slqr_ctx();
  if (!ctx) return SLQR_ENOMEM;
  ctx->device = device;
  ctx->hbm_budget = hbm_budget_bytes;
  cudaError_t e = cudaSetDevice(device);
  int sms = 0, optin = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_start, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_panel, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (ctx->d_status) cudaFree(ctx->d_status);
    delete ctx;
    return SLQR_ECUDA;
  }
  ctx->num_sms = sms;
  ctx->smem_optin = (size_t)optin;
  if (init_kernel_attrs(ctx) != SLQR_OK || init_batch_attrs(ctx) != SLQR_OK ||
      init_tc_attrs(ctx) != SLQR_OK || init_bf16_attrs(ctx) != SLQR_OK ||
      init_cluster_attrs(ctx) != SLQR_OK || init_lookahead_attrs(ctx) != SLQR_OK) {
    cudaEventDestroy(ctx->ev_start);
    cudaEventDestroy(ctx->ev_ready);
    cudaEventDestroy(ctx->ev_panel);
    cudaStreamDestroy(ctx->aux_stream);
    cudaFree(ctx->d_status);
    delete ctx;
    return SLQR_ECUDA;
  }
  *out = ctx;
  return SLQR_OK;
}

extern "C" void slqr_destroy(slqr_ctx *ctx) {
  if (!ctx) return;
  server_stop(ctx);
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  prof_collect(ctx);
  for (cudaEvent_t e : ctx->prof.free_events) cudaEventDestroy(e);
  if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
  if (ctx->ev_ready) cudaEventDestroy(ctx->ev_ready);
  if (ctx->ev_panel) cudaEventDestroy(ctx->ev_panel);
  if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
  if (ctx->ws.ptr) cudaFree(ctx->ws.ptr);
  if (ctx->ws2.ptr) cudaFree(ctx->ws2.ptr);
  if (ctx->d_status) cudaFree(ctx->d_status);
  delete ctx;
}

namespace slqr {

// A wait on a word that nothing sets, bounded by `polls`: the same give-up
// path as the kernels' barrier and mbarrier waits (record SLQR_ETIMEOUT in
// the status word, return).
__global__ void wait_probe_kernel(const unsigned *word, unsigned polls, int *status) {
  if (threadIdx.x != 0) return;
  for (unsigned it = 0; ld_acquire_u32(word) == 0u; ++it) {
    if (it >= polls) {
      record_status(status, SLQR_ETIMEOUT);
      return;
    }
    if (it > 64) __nanosleep(256);
  }
}

}  // namespace slqr

extern "C" slqr_status slqr_check_bounded_wait(slqr_ctx *ctx, unsigned polls, void *stream) {
  if (!ctx || polls == 0 || polls > (1u << 20)) return SLQR_EINVAL;
  NvtxRange nvtx_range("slqr_check_bounded_wait");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaError_t e = cudaSetDevice(ctx->device);
  unsigned *word = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&word, sizeof(unsigned));
  cudaStream_t s = (cudaStream_t)stream;
  if (e == cudaSuccess) e = cudaMemsetAsync(word, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) {
    wait_probe_kernel<<<1, 32, 0, s>>>(word, polls, ctx->d_status);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int st = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
  if (word) cudaFree(word);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "bounded-wait check: %s", cudaGetErrorString(e));
  return st;
}

extern "C" slqr_status slqr_set_spin_limit(slqr_ctx *ctx, unsigned polls) {
  if (!ctx || polls > kSpinLimit) return SLQR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  ctx->spin_limit = polls == 0 ? kSpinLimit : polls;
  return SLQR_OK;
}

namespace slqr {

// FP64 FMA peak probe: register-resident DFMA chains, 8 independent ones per
// thread (enough to cover the pipe's latency), 4 CTAs of 256 threads per SM.
__global__ void __launch_bounds__(256)
dfma_peak_kernel(double *out, int iters, double a, double b) {
  double acc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = fma(acc[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += acc[i];
  if (s == 12345.678) out[0] = s;       // keeps the chains live; never true in practice
}

slqr_status measure_tf32_peak(slqr_ctx *ctx, double *tflops);

static slqr_status measure_fp64_peak(slqr_ctx *ctx, double *tflops) {
  const int iters = 1 << 14, threads = 256, grid = 4 * ctx->num_sms;
  double *out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, 0);
    dfma_peak_kernel<<<grid, threads>>>(out, iters, 0.999999, 1e-7);
    cudaEventRecord(e1, 0);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "FP64 peak probe: %s", cudaGetErrorString(e));
  *tflops = 2.0 * 8.0 * iters * (double)threads * grid / (best * 1e-3) / 1e12;
  return SLQR_OK;
}

}  // namespace slqr

extern "C" slqr_status slqr_measure_peak(slqr_ctx *ctx, int kind, double *tflops) {
  if (!ctx || !tflops) return SLQR_EINVAL;
  NvtxRange nvtx_range("slqr_measure_peak");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "peak probe: %s", cudaGetErrorString(e));
  if (kind == SLQR_PEAK_FP64_FMA) return measure_fp64_peak(ctx, tflops);
  if (kind == SLQR_PEAK_TF32_TC) return measure_tf32_peak(ctx, tflops);
  return fail(ctx, SLQR_EINVAL, "peak kind %d", kind);
}

extern "C" const char *slqr_last_error(slqr_ctx *ctx) {
  if (!ctx) return "NULL context";
  return ctx->last_error.c_str();
}

extern "C" slqr_status slqr_sync(slqr_ctx *ctx, void *stream) {
  if (!ctx) return SLQR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "stream: %s", cudaGetErrorString(e));
  int st = 0;
  e = cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "status word: %s", cudaGetErrorString(e));
  if (st != 0) {
    if (st == SLQR_ERANK) fail(ctx, st, "R has an exact zero on its diagonal");
    else if (st == SLQR_ETIMEOUT) fail(ctx, st, "a bounded device wait gave up");
    else if (st == SLQR_ECHECK) fail(ctx, st, "a device bounds or invariant check failed");
  }
  if (st == 0) {
    const slqr_status g = check_workspaces(ctx);        // (checked build only)
    if (g != SLQR_OK) return g;
  }
  return st;
}

// The checked build's self test: an index one past a 64-entry buffer, which
// the check must catch (the access is skipped).
__global__ void check_selftest_kernel(double *buf, int n, int *status) {
  const int i = threadIdx.x;                           // 0 .. n (one past the end)
  if (slqr_check(i < n, status)) buf[i] = (double)i;
}

extern "C" int slqr_is_checked(void) {
#ifdef SLQR_CHECKED
  return 1;
#else
  return 0;
#endif
}

extern "C" slqr_status slqr_check_selftest(slqr_ctx *ctx) {
  if (!ctx) return SLQR_EINVAL;
#ifndef SLQR_CHECKED
  return SLQR_EINVAL;
#else
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaError_t e = cudaSetDevice(ctx->device);
  double *buf = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&buf, 64 * sizeof(double));
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "selftest: %s", cudaGetErrorString(e));
  check_selftest_kernel<<<1, 65>>>(buf, 64, ctx->d_status);
  e = cudaDeviceSynchronize();
  cudaFree(buf);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "selftest: %s", cudaGetErrorString(e));
  int st = 0;
  e = cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "selftest: %s", cudaGetErrorString(e));
  return st;
#endif
}
