// serve.cu -- continuous-batching request loop (slqr_submit / slqr_poll).
//
// SLSQP solves one least-squares subproblem per iteration and reuses the
// stored factorization for its back-substitution (paper, Section 1 and the
// abstract).  Many concurrent SLSQP runs make a stream of such subproblems;
// this file serves them on one GPU.
//
// A worker thread inside the library owns the loop:
//  * admission: requests are taken in arrival order while the HBM budget of
//    the context allows; the library copies A (and b) into memory it owns,
//    allocated stream-ordered from its own pool (no device-wide
//    synchronisation);
//  * batching: every admitted small problem (m <= slqr_batch_max_rows()) of
//    one precision goes into one persistent batched launch; a launch is made
//    as soon as the previous one of that precision has been issued, so
//    requests that arrive while others run join the next launch;
//  * larger problems run one per stream from a pool of streams (each with its
//    own context and workspace), so they overlap with each other and with
//    the batched launches;
//  * latency routing: one CTA of the batched launch factors a problem at the
//    FP64 rate of a single SM, while the stream path spreads it over many
//    SMs; so while at most half of the streams are busy, a small problem with
//    m * n >= kRouteMN takes the stream path (lower latency on an idle GPU),
//    and under load it joins the batch (higher throughput);
//  * residency: a FACTOR request keeps its factorization (A in H12 form, up,
//    compact-WY store) on the device under a handle until RELEASE; SOLVE
//    requests reuse it (Q^T b, back-substitution);
//  * mixed precision: FP32 requests of the batch size class join the batched
//    FP32 launch; every other mixed-precision request (SLQR_FP32 with
//    m > 512, SLQR_TF32, SLQR_BF16X3, and SOLVE on a mixed-precision handle)
//    goes to a mixed lane: a helper thread with its own context and stream
//    that runs the synchronous mixed-precision solve (low-precision
//    factorization, refinement against the FP64 A, the FP64 fallback when the
//    refinement fails, flagged as SLQR_FALLBACK).  A mixed FACTOR keeps the
//    library's FP64 copy of A and the low-precision factorization resident
//    (both counted in the HBM budget) for later SOLVE requests;
//  * completion is observed with CUDA events (with a host flag for the mixed
//    lanes); the solution is copied into the caller's host buffer and the
//    request's latency recorded.
#include "slqr_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

namespace slqr {

using Clock = std::chrono::steady_clock;

struct Resident {
  int m = 0, n = 0;
  bool stacked = false;          // [L^T; C] factorization (slqr_factor_stacked)
  bool mixed = false;            // low-precision factorization: dA is the FP64 copy of A and
  MixedFactorState fs;           //   fs the state of its factorization (mixed_factor_into)
  double *dA = nullptr, *dup = nullptr, *dwy = nullptr;
  size_t bytes = 0;
  cudaEvent_t ready = nullptr;   // the factorization is complete after this
  int users = 0;                 // SOLVE requests in flight on it
  bool release = false;
};

struct Req {
  uint64_t ticket = 0;
  slqr_request r{};
  int state = 0;                 // 0 pending, 1 in flight, 2 done
  slqr_result res{};
  Clock::time_point t_submit;
  double *dA = nullptr, *dup = nullptr, *dwy = nullptr, *db = nullptr;
  size_t bytes = 0;              // owned bytes (freed when done, unless resident)
  uint64_t handle = 0;           // SOLVE/RELEASE: the handle used; FACTOR: the one made
  bool small = false;
  bool mixed = false;            // runs on a mixed lane
  double *dx = nullptr;          // mixed lanes: the solution (n doubles)
  MixedFactorState fs;           // mixed FACTOR: the state made (in the request's block)
};

struct Unit {                    // one launch sequence whose completion is watched
  std::vector<Req *> reqs;
  cudaEvent_t done = nullptr;
  std::shared_ptr<std::atomic<int>> host_done;   // mixed lanes: set by the helper thread
  cudaStream_t stream = nullptr;
  int *d_status = nullptr;       // batch: per-problem status
  double *d_err = nullptr;
};

struct Server {
  slqr_ctx *owner = nullptr;
  int device = 0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv;
  bool stopping = false;
  std::deque<uint64_t> incoming;
  std::unordered_map<uint64_t, Req> reqs;
  std::unordered_map<uint64_t, Resident> handles;
  uint64_t next_ticket = 1, next_handle = 1;
  // worker-owned state
  std::deque<Req *> pending;
  std::atomic<size_t> used_bytes{0};
  int nstreams = 0, rr = 0;
  std::vector<cudaStream_t> streams;
  std::vector<slqr_ctx *> sub;
  cudaStream_t bstream[2] = {nullptr, nullptr};   // batched launches per precision
  slqr_ctx *bctx[2] = {nullptr, nullptr};
  cudaMemPool_t pool = nullptr;
  std::vector<Unit> inflight;
  std::vector<Req *> small_ready[2];              // admitted small requests, per precision
  // mixed lanes: helper threads, each with a context, a stream and a job queue
  struct Lane {
    slqr_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    std::thread thread;
    std::deque<std::pair<Req *, std::shared_ptr<std::atomic<int>>>> jobs;
    int busy = 0;                                  // jobs queued or running (worker's view)
  };
  std::vector<Lane> lanes;
  std::mutex lane_mu;
  std::condition_variable lane_cv;
  bool lanes_stopping = false;
};

// A request served on a mixed lane: every mixed-precision request except the
// FP32 FACTOR_SOLVE of the batch size class, and SOLVE on a mixed handle.
static bool is_mixed_lane(const slqr_request &r) {
  if (r.kind != SLQR_REQ_FACTOR && r.kind != SLQR_REQ_FACTOR_SOLVE) return false;
  if (r.prec == SLQR_FP64) return false;
  return !(r.prec == SLQR_FP32 && r.kind == SLQR_REQ_FACTOR_SOLVE && r.m <= slqr_batch_max_rows());
}

static const size_t kAlign = 256;
// Smallest m * n a batch-sized problem needs to be sent down the stream path
// when the streams are idle: about where one SM's FP64 time for the
// factorization (2 m n^2 flops at ~8 GFLOP/s) overtakes the stream path's
// per-column latency (~8-10 us per column plus launches).
static const long long kRouteMN = 60000;

static double *pool_alloc(Server *S, size_t bytes, cudaStream_t s) {
  void *p = nullptr;
  if (cudaMallocFromPoolAsync(&p, std::max(bytes, kAlign), S->pool, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (double *)p;
}

static void pool_free(double *p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

static size_t request_bytes(const slqr_request &r) {
  if (is_mixed_lane(r)) {
    // the FP64 copy of A, the low-precision state, b and x
    size_t b = align_up((size_t)r.m * r.n * 8, kAlign) + align_up(mixed_state_bytes(r.m, r.n), kAlign);
    if (r.kind == SLQR_REQ_FACTOR_SOLVE)
      b += align_up((size_t)r.m * 8, kAlign) + align_up((size_t)r.n * 8, kAlign);
    return b;
  }
  switch (r.kind) {
    case SLQR_REQ_FACTOR:
    case SLQR_REQ_FACTOR_SOLVE: {
      size_t b = align_up((size_t)r.m * r.n * 8, kAlign) + align_up((size_t)r.n * 8, kAlign) +
                 align_up(slqr_wy_size(r.m, r.n), kAlign);
      if (r.kind == SLQR_REQ_FACTOR_SOLVE) b += align_up((size_t)r.m * 8, kAlign);
      return b;
    }
    case SLQR_REQ_SOLVE: return 0;   // set at admission from the handle's m
    default: return 0;
  }
}

// Called with S->mu held: after this the request belongs to slqr_poll.
static void finish(Server *S, Req &q, int status) {
  (void)S;
  q.res.status = status;
  q.res.latency_ms =
      std::chrono::duration<double, std::milli>(Clock::now() - q.t_submit).count();
  q.state = 2;
}

// Copy the solution (and the residual norm) of a finished solve to the host.
// FP64: the residual is ||(Q^T b)[n:m]||.  FP32 (refined): ||b - A x|| with
// the caller's A and b, which stay valid until the request is done.
static void deliver_solution(Req &q, int m, int n) {
  std::vector<double> hb(m);
  if (cudaMemcpy(hb.data(), q.db, sizeof(double) * m, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    q.res.status = SLQR_ECUDA;
    return;
  }
  if (q.r.x) std::memcpy(q.r.x, hb.data(), sizeof(double) * n);
  if (q.mixed) return;            // the mixed lane has set the residual norm
  double s = 0.0;
  if (q.r.prec != SLQR_FP64 && !q.r.A) {
    q.res.residual_norm = std::nan("");            // mixed SOLVE: A is not at hand
    return;
  }
  if (q.r.prec != SLQR_FP64) {
    for (int i = 0; i < m; ++i) {
      double ri = q.r.b[i];
      for (int j = 0; j < n; ++j) ri -= q.r.A[(size_t)i + (size_t)j * q.r.lda] * hb[j];
      s += ri * ri;
    }
  } else {
    for (int i = n; i < m; ++i) s += hb[i] * hb[i];
  }
  q.res.residual_norm = std::sqrt(s);
}

// Body of one mixed-lane job (runs in the lane's helper thread): the
// low-precision factorization and/or the refinement, synchronous on the lane's
// stream; the solution ends in q.db[0:n] for deliver_solution.
static void run_mixed_job(Server *S, Server::Lane &L, Req &q) {
  const slqr_request &r = q.r;
  slqr_mixed_opts o{};
  o.fp64_fallback = 1;
  slqr_mixed_info info{};
  info.err = HUGE_VAL;
  slqr_status st = SLQR_OK;
  int m = r.m, n = r.n;
  if (r.kind == SLQR_REQ_SOLVE) {
    Resident *h = nullptr;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      h = &S->handles[q.handle];     // kept alive by its user count
    }
    m = h->m;
    n = h->n;
    cudaStreamWaitEvent(L.stream, h->ready, 0);
    st = mixed_solve_with(L.ctx, h->fs, h->dA, h->m, q.db, q.dx, o, &info, L.stream);
  } else {
    void *state = (char *)q.dA + align_up((size_t)m * n * 8, kAlign);
    const int ntop = (r.structure == SLQR_STACKED) ? n : 0;
    st = mixed_factor_into(L.ctx, m, n, q.dA, m, r.prec, ntop, state, &q.fs, L.stream);
    if (st == SLQR_OK && r.kind == SLQR_REQ_FACTOR_SOLVE)
      st = mixed_solve_with(L.ctx, q.fs, q.dA, m, q.db, q.dx, o, &info, L.stream);
  }
  const bool solved = q.db && (st == SLQR_OK || st == SLQR_FALLBACK || st == SLQR_ERANK);
  if (solved)
    cudaMemcpyAsync(q.db, q.dx, sizeof(double) * n, cudaMemcpyDeviceToDevice, L.stream);
  if (cudaStreamSynchronize(L.stream) != cudaSuccess) {
    cudaGetLastError();
    st = SLQR_ECUDA;
  }
  // ||b - A x|| from the caller's host arrays (here, not in the worker loop);
  // a SOLVE request has no A at hand
  double res = std::nan("");
  if (solved && st != SLQR_ECUDA && r.A) {
    std::vector<double> x(n);
    if (cudaMemcpy(x.data(), q.dx, sizeof(double) * n, cudaMemcpyDeviceToHost) == cudaSuccess) {
      double acc = 0.0;
      for (int i = 0; i < m; ++i) {
        double ri = r.b[i];
        for (int j = 0; j < n; ++j) ri -= r.A[(size_t)i + (size_t)j * r.lda] * x[j];
        acc += ri * ri;
      }
      res = std::sqrt(acc);
    } else {
      cudaGetLastError();
    }
  }
  std::lock_guard<std::mutex> lk(S->mu);
  q.res.status = st;
  q.res.err = info.err;
  q.res.residual_norm = res;
}

static void lane_main(Server *S, int li) {
  cudaSetDevice(S->device);
  Server::Lane &L = S->lanes[li];
  for (;;) {
    std::pair<Req *, std::shared_ptr<std::atomic<int>>> job;
    {
      std::unique_lock<std::mutex> lk(S->lane_mu);
      S->lane_cv.wait(lk, [&] { return S->lanes_stopping || !L.jobs.empty(); });
      if (L.jobs.empty()) break;                   // stopping, nothing left
      job = L.jobs.front();
      L.jobs.pop_front();
    }
    run_mixed_job(S, L, *job.first);
    job.second->store(1);
  }
}

// Hand a request to the least busy mixed lane (its copies in are already
// enqueued on that lane's stream).
static void dispatch_mixed(Server *S, Req &q, int li) {
  Unit u;
  u.reqs.push_back(&q);
  u.stream = S->lanes[li].stream;
  u.host_done = std::make_shared<std::atomic<int>>(0);
  S->lanes[li].busy++;
  {
    std::lock_guard<std::mutex> lk(S->lane_mu);
    S->lanes[li].jobs.emplace_back(&q, u.host_done);
  }
  S->lane_cv.notify_all();
  S->inflight.push_back(u);
}

static int least_busy_lane(Server *S) {
  int best = 0;
  for (int i = 1; i < (int)S->lanes.size(); ++i)
    if (S->lanes[i].busy < S->lanes[best].busy) best = i;
  return best;
}

// Admit pending requests in arrival order while the budget allows.
static void admit(Server *S) {
  const size_t budget = S->owner->hbm_budget;
  while (!S->pending.empty()) {
    Req &q = *S->pending.front();
    const slqr_request &r = q.r;
    if (r.kind == SLQR_REQ_RELEASE) {
      std::lock_guard<std::mutex> lk(S->mu);
      auto it = S->handles.find(r.handle);
      if (it == S->handles.end() || it->second.release) {
        finish(S, q, SLQR_ENOTFOUND);
      } else {
        it->second.release = true;   // freed once no SOLVE uses it
        finish(S, q, SLQR_OK);
      }
      S->pending.pop_front();
      continue;
    }
    if (r.kind == SLQR_REQ_SOLVE) {
      Resident *h = nullptr;
      {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->handles.find(r.handle);
        if (it != S->handles.end() && !it->second.release) h = &it->second;
        if (!h) {
          finish(S, q, SLQR_ENOTFOUND);
          S->pending.pop_front();
          continue;
        }
      }
      if (h->mixed) {
        // b and x of a refinement with the resident low-precision factorization
        const size_t bytes = align_up((size_t)h->m * 8, kAlign) + align_up((size_t)h->n * 8, kAlign);
        if (budget && S->used_bytes + bytes > budget) break;
        const int li = least_busy_lane(S);
        cudaStream_t s = S->lanes[li].stream;
        q.db = pool_alloc(S, bytes, s);
        if (!q.db) break;
        q.dx = (double *)((char *)q.db + align_up((size_t)h->m * 8, kAlign));
        q.bytes = bytes;
        q.mixed = true;
        S->used_bytes += bytes;
        cudaMemcpyAsync(q.db, r.b, sizeof(double) * h->m, cudaMemcpyHostToDevice, s);
        {
          std::lock_guard<std::mutex> lk(S->mu);
          h->users++;
          q.handle = r.handle;
          q.state = 1;
          q.res.status = SLQR_OK;
        }
        dispatch_mixed(S, q, li);
        S->pending.pop_front();
        continue;
      }
      const size_t bytes = align_up((size_t)h->m * 8, kAlign);
      if (budget && S->used_bytes + bytes > budget) break;
      const int si = S->rr++ % S->nstreams;
      cudaStream_t s = S->streams[si];
      q.db = pool_alloc(S, bytes, s);
      if (!q.db) break;   // pool exhausted: retry later
      q.bytes = bytes;
      S->used_bytes += bytes;
      cudaMemcpyAsync(q.db, r.b, sizeof(double) * h->m, cudaMemcpyHostToDevice, s);
      cudaStreamWaitEvent(s, h->ready, 0);
      slqr_ctx *c = S->sub[si];
      slqr_status st =
          h->stacked
              ? slqr_apply_qt_stacked(c, h->n, h->m - h->n, h->dA, h->m, h->dup, h->dwy, 1, q.db,
                                      h->m, s)
              : slqr_apply_qt(c, h->m, h->n, h->dA, h->m, h->dup, h->dwy, 1, q.db, h->m, s);
      if (st == SLQR_OK) st = slqr_solve_r(c, h->n, h->dA, h->m, 1, q.db, h->m, s);
      Unit u;
      u.reqs.push_back(&q);
      u.stream = s;
      cudaEventCreateWithFlags(&u.done, cudaEventDisableTiming);
      cudaEventRecord(u.done, s);
      S->inflight.push_back(u);
      {
        std::lock_guard<std::mutex> lk(S->mu);
        h->users++;
        q.handle = r.handle;
        q.state = 1;
        q.res.status = st;
      }
      S->pending.pop_front();
      continue;
    }
    // FACTOR / FACTOR_SOLVE
    const size_t bytes = request_bytes(r);
    if (budget && bytes > budget) {
      std::lock_guard<std::mutex> lk(S->mu);
      finish(S, q, SLQR_EBUSY);
      S->pending.pop_front();
      continue;
    }
    if (budget && S->used_bytes + bytes > budget) break;   // wait for memory to free up
    if (is_mixed_lane(r)) {
      const int li = least_busy_lane(S);
      cudaStream_t s = S->lanes[li].stream;
      char *blk = (char *)pool_alloc(S, bytes, s);
      if (!blk) break;
      const size_t a_b = align_up((size_t)r.m * r.n * 8, kAlign);
      const size_t s_b = align_up(mixed_state_bytes(r.m, r.n), kAlign);
      q.mixed = true;
      q.dA = (double *)blk;
      if (r.kind == SLQR_REQ_FACTOR_SOLVE) {
        q.db = (double *)(blk + a_b + s_b);
        q.dx = (double *)(blk + a_b + s_b + align_up((size_t)r.m * 8, kAlign));
      }
      q.bytes = bytes;
      S->used_bytes += bytes;
      cudaMemcpy2DAsync(q.dA, sizeof(double) * r.m, r.A, sizeof(double) * r.lda,
                        sizeof(double) * r.m, r.n, cudaMemcpyHostToDevice, s);
      if (q.db) cudaMemcpyAsync(q.db, r.b, sizeof(double) * r.m, cudaMemcpyHostToDevice, s);
      {
        std::lock_guard<std::mutex> lk(S->mu);
        q.state = 1;
        q.res.status = SLQR_OK;
      }
      dispatch_mixed(S, q, li);
      S->pending.pop_front();
      continue;
    }
    bool small = (r.m <= slqr_batch_max_rows());
    if (small && (long long)r.m * r.n >= kRouteMN) {
      int busy = 0;                                  // units in flight on the stream pool
      for (const Unit &u : S->inflight)
        if (!u.host_done && u.stream != S->bstream[0] && u.stream != S->bstream[1]) ++busy;
      if (2 * busy < S->nstreams) small = false;
    }
    const int pi = (r.prec == SLQR_FP32) ? 1 : 0;
    const int si = small ? -1 : (S->rr++ % S->nstreams);
    cudaStream_t s = small ? S->bstream[pi] : S->streams[si];
    const size_t a_b = align_up((size_t)r.m * r.n * 8, kAlign);
    const size_t u_b = align_up((size_t)r.n * 8, kAlign);
    const size_t w_b = align_up(slqr_wy_size(r.m, r.n), kAlign);
    char *blk = (char *)pool_alloc(S, bytes, s);
    if (!blk) break;
    q.small = small;
    q.dA = (double *)blk;
    q.dup = (double *)(blk + a_b);
    q.dwy = (double *)(blk + a_b + u_b);
    q.db = (r.kind == SLQR_REQ_FACTOR_SOLVE) ? (double *)(blk + a_b + u_b + w_b) : nullptr;
    q.bytes = bytes;
    S->used_bytes += bytes;
    // copy A in (column-major, leading dimension m on the device)
    cudaMemcpy2DAsync(q.dA, sizeof(double) * r.m, r.A, sizeof(double) * r.lda,
                      sizeof(double) * r.m, r.n, cudaMemcpyHostToDevice, s);
    if (q.db) cudaMemcpyAsync(q.db, r.b, sizeof(double) * r.m, cudaMemcpyHostToDevice, s);
    slqr_status st = SLQR_OK;
    if (small) {
      S->small_ready[pi].push_back(&q);
    } else {
      slqr_ctx *c = S->sub[si];
      const bool stacked = (r.structure == SLQR_STACKED);
      st = stacked ? slqr_factor_stacked(c, r.n, r.m - r.n, q.dA, r.m, q.dup, q.dwy, s)
                   : slqr_factor(c, r.m, r.n, q.dA, r.m, q.dup, q.dwy, s);
      if (st == SLQR_OK && q.db) {
        st = stacked ? slqr_apply_qt_stacked(c, r.n, r.m - r.n, q.dA, r.m, q.dup, q.dwy, 1, q.db,
                                             r.m, s)
                     : slqr_apply_qt(c, r.m, r.n, q.dA, r.m, q.dup, q.dwy, 1, q.db, r.m, s);
        if (st == SLQR_OK) st = slqr_solve_r(c, r.n, q.dA, r.m, 1, q.db, r.m, s);
      }
      Unit u;
      u.reqs.push_back(&q);
      u.stream = s;
      cudaEventCreateWithFlags(&u.done, cudaEventDisableTiming);
      cudaEventRecord(u.done, s);
      S->inflight.push_back(u);
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      q.state = 1;
      q.res.status = st;
    }
    S->pending.pop_front();
  }
}

// One batched launch per precision for the admitted small requests.
static void launch_batches(Server *S) {
  for (int pi = 0; pi < 2; ++pi) {
    auto &ready = S->small_ready[pi];
    if (ready.empty()) continue;
    const int cnt = (int)ready.size();
    std::vector<int> m(cnt), n(cnt), ntop(cnt), lda(cnt);
    std::vector<double *> A(cnt), up(cnt), b(cnt);
    bool any_b = false;
    for (int i = 0; i < cnt; ++i) {
      const Req &q = *ready[i];
      m[i] = q.r.m;
      n[i] = q.r.n;
      ntop[i] = (q.r.structure == SLQR_STACKED) ? q.r.n : 0;
      lda[i] = q.r.m;
      A[i] = q.dA;
      up[i] = q.dup;
      b[i] = q.db;
      any_b |= (q.db != nullptr);
    }
    cudaStream_t s = S->bstream[pi];
    Unit u;
    u.stream = s;
    u.d_status = (int *)pool_alloc(S, sizeof(int) * cnt, s);
    u.d_err = pool_alloc(S, sizeof(double) * cnt, s);
    slqr_status st = batch_factor_locked(S->bctx[pi], cnt, m.data(), n.data(), ntop.data(),
                                         A.data(), lda.data(), up.data(),
                                         any_b ? b.data() : nullptr, pi ? SLQR_FP32 : SLQR_FP64,
                                         u.d_status, u.d_err, s);
    u.reqs = ready;
    cudaEventCreateWithFlags(&u.done, cudaEventDisableTiming);
    cudaEventRecord(u.done, s);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (Req *q : ready) q->res.status = st;
    }
    S->inflight.push_back(u);
    ready.clear();
  }
}

// Retire finished launches: deliver solutions, create handles, free memory.
static void retire(Server *S) {
  for (size_t ui = 0; ui < S->inflight.size();) {
    Unit &u = S->inflight[ui];
    cudaError_t e = cudaSuccess;
    if (u.host_done) {
      if (!u.host_done->load()) {
        ++ui;
        continue;
      }
      for (auto &ln : S->lanes)
        if (ln.stream == u.stream) ln.busy--;
    } else {
      e = cudaEventQuery(u.done);
      if (e == cudaErrorNotReady) {
        ++ui;
        continue;
      }
    }
    std::vector<int> st_host;
    std::vector<double> err_host;
    if (u.d_status) {
      st_host.resize(u.reqs.size());
      err_host.resize(u.reqs.size());
      cudaMemcpy(st_host.data(), u.d_status, sizeof(int) * st_host.size(), cudaMemcpyDeviceToHost);
      cudaMemcpy(err_host.data(), u.d_err, sizeof(double) * err_host.size(),
                 cudaMemcpyDeviceToHost);
    }
    cudaStream_t s = u.stream;
    for (size_t k = 0; k < u.reqs.size(); ++k) {
      std::lock_guard<std::mutex> lk(S->mu);
      Req &q = *u.reqs[k];
      int status = (e == cudaSuccess) ? q.res.status : SLQR_ECUDA;
      if (status == SLQR_OK && u.d_status) status = st_host[k];
      if (u.d_status) q.res.err = err_host[k];
      const slqr_request &r = q.r;
      q.res.status = status;
      if (r.kind == SLQR_REQ_SOLVE) {
        Resident &h = S->handles[q.handle];
        if (status == SLQR_OK || status == SLQR_ERANK || status == SLQR_FALLBACK)
          deliver_solution(q, h.m, h.n);
        pool_free(q.db, s);
        S->used_bytes -= q.bytes;
        h.users--;
      } else {
        if (q.db && (status == SLQR_OK || status == SLQR_ERANK || status == SLQR_ENOCONV ||
                     status == SLQR_FALLBACK))
          deliver_solution(q, r.m, r.n);
        if (r.kind == SLQR_REQ_FACTOR && status == SLQR_OK) {
          const uint64_t id = S->next_handle++;
          Resident h;
          h.m = r.m;
          h.n = r.n;
          h.mixed = q.mixed;
          h.fs = q.fs;
          h.stacked = (r.structure == SLQR_STACKED) && !q.mixed;
          h.dA = q.dA;
          h.dup = q.dup;
          h.dwy = q.small ? nullptr : q.dwy;   // the batched kernel keeps no WY store
          h.bytes = q.bytes;
          cudaEventCreateWithFlags(&h.ready, cudaEventDisableTiming);
          cudaEventRecord(h.ready, s);
          S->handles[id] = h;
          q.res.handle = id;
        } else {
          pool_free(q.dA, s);   // one block holds A, up, wy and b
          S->used_bytes -= q.bytes;
        }
      }
      finish(S, q, q.res.status);
    }
    if (u.d_status) {
      pool_free((double *)u.d_status, s);
      pool_free(u.d_err, s);
    }
    if (u.done) cudaEventDestroy(u.done);
    S->inflight.erase(S->inflight.begin() + ui);
  }
  // free released handles nobody uses any more
  std::lock_guard<std::mutex> lk(S->mu);
  for (auto it = S->handles.begin(); it != S->handles.end();) {
    if (it->second.release && it->second.users == 0) {
      cudaStreamWaitEvent(S->streams[0], it->second.ready, 0);
      pool_free(it->second.dA, S->streams[0]);
      S->used_bytes -= it->second.bytes;
      cudaEventDestroy(it->second.ready);
      it = S->handles.erase(it);
    } else {
      ++it;
    }
  }
}

static void worker_main(Server *S) {
  cudaSetDevice(S->device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->incoming.empty() && S->inflight.empty() && S->pending.empty()) {
        if (S->stopping) break;
        S->cv.wait_for(lk, std::chrono::milliseconds(5));
      }
      while (!S->incoming.empty()) {
        S->pending.push_back(&S->reqs[S->incoming.front()]);
        S->incoming.pop_front();
      }
      if (S->stopping && S->pending.empty() && S->inflight.empty()) break;
    }
    admit(S);
    launch_batches(S);
    retire(S);
    if (!S->inflight.empty() || !S->pending.empty())
      std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

static slqr_status server_start(slqr_ctx *ctx) {
  if (ctx->server) return SLQR_OK;
  Server *S = new (std::nothrow) Server();
  if (!S) return SLQR_ENOMEM;
  S->owner = ctx;
  S->device = ctx->device;
  S->nstreams = 8;   // measured: about 8% more mid-size requests per second than 4; 16 no better
  cudaSetDevice(ctx->device);
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = ctx->device;
  if (cudaMemPoolCreate(&S->pool, &props) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return fail(ctx, SLQR_ECUDA, "cudaMemPoolCreate failed");
  }
  uint64_t keep = UINT64_MAX;
  cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  // on a failed set-up, release what was made so far
  auto undo = [&]() {
    for (slqr_ctx *c : S->sub) slqr_destroy(c);
    for (cudaStream_t st : S->streams) cudaStreamDestroy(st);
    for (int pi = 0; pi < 2; ++pi) {
      if (S->bctx[pi]) slqr_destroy(S->bctx[pi]);
      if (S->bstream[pi]) cudaStreamDestroy(S->bstream[pi]);
    }
    cudaMemPoolDestroy(S->pool);
    delete S;
  };
  for (int i = 0; i < S->nstreams; ++i) {
    cudaStream_t s = nullptr;
    slqr_ctx *c = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        slqr_create(&c, ctx->device, 0) != SLQR_OK) {
      cudaGetLastError();
      if (s) cudaStreamDestroy(s);
      undo();
      return fail(ctx, SLQR_ECUDA, "server stream set-up failed");
    }
    S->streams.push_back(s);
    S->sub.push_back(c);
  }
  for (int pi = 0; pi < 2; ++pi) {
    if (cudaStreamCreateWithFlags(&S->bstream[pi], cudaStreamNonBlocking) != cudaSuccess ||
        slqr_create(&S->bctx[pi], ctx->device, 0) != SLQR_OK) {
      cudaGetLastError();
      undo();
      return fail(ctx, SLQR_ECUDA, "server batch stream set-up failed");
    }
  }
  const int nlanes = 8;   // as many as the FP64 stream pool: a mixed solve is synchronous per lane
  S->lanes.resize(nlanes);
  for (int i = 0; i < nlanes; ++i) {
    Server::Lane &L = S->lanes[i];
    if (cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess ||
        slqr_create(&L.ctx, ctx->device, 0) != SLQR_OK) {
      cudaGetLastError();
      for (auto &l2 : S->lanes) {
        if (l2.ctx) slqr_destroy(l2.ctx);
        if (l2.stream) cudaStreamDestroy(l2.stream);
      }
      undo();
      return fail(ctx, SLQR_ECUDA, "server mixed-lane set-up failed");
    }
  }
  for (int i = 0; i < nlanes; ++i) S->lanes[i].thread = std::thread(lane_main, S, i);
  S->worker = std::thread(worker_main, S);
  ctx->server = S;
  return SLQR_OK;
}

void server_stop(slqr_ctx *ctx) {
  Server *S = ctx->server;
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  {
    std::lock_guard<std::mutex> lk(S->lane_mu);
    S->lanes_stopping = true;
  }
  S->lane_cv.notify_all();
  for (auto &L : S->lanes)
    if (L.thread.joinable()) L.thread.join();
  cudaSetDevice(S->device);
  cudaDeviceSynchronize();
  for (auto &kv : S->handles) {
    pool_free(kv.second.dA, S->streams[0]);
    cudaEventDestroy(kv.second.ready);
  }
  cudaStreamSynchronize(S->streams[0]);
  for (slqr_ctx *c : S->sub) slqr_destroy(c);
  for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
  for (int pi = 0; pi < 2; ++pi) {
    slqr_destroy(S->bctx[pi]);
    cudaStreamDestroy(S->bstream[pi]);
  }
  for (auto &L : S->lanes) {
    slqr_destroy(L.ctx);
    cudaStreamDestroy(L.stream);
  }
  cudaMemPoolDestroy(S->pool);
  delete S;
  ctx->server = nullptr;
}

}  // namespace slqr

using namespace slqr;

extern "C" slqr_status slqr_submit(slqr_ctx *ctx, const slqr_request *req, uint64_t *ticket) {
  if (!ctx || !req || !ticket) return SLQR_EINVAL;
  const slqr_request &r = *req;
  switch (r.kind) {
    case SLQR_REQ_FACTOR:
    case SLQR_REQ_FACTOR_SOLVE:
      if (r.m < 1 || r.n < 1 || r.m < r.n || r.lda < r.m || !r.A)
        return fail(ctx, SLQR_EINVAL, "request: need m >= n >= 1, lda >= m, A");
      if (r.kind == SLQR_REQ_FACTOR_SOLVE && (!r.b || !r.x))
        return fail(ctx, SLQR_EINVAL, "request: FACTOR_SOLVE needs b and x");
      if (r.prec != SLQR_FP64 && r.prec != SLQR_FP32 && r.prec != SLQR_TF32 &&
          r.prec != SLQR_BF16X3)
        return fail(ctx, SLQR_EINVAL, "request: unknown precision %d", r.prec);
      if (r.m > slqr_max_rows()) return fail(ctx, SLQR_EINVAL, "request: m above slqr_max_rows()");
      if (r.structure != SLQR_DENSE && r.structure != SLQR_STACKED)
        return fail(ctx, SLQR_EINVAL, "request: unknown structure %d", r.structure);
      break;
    case SLQR_REQ_SOLVE:
      if (!r.b || !r.x) return fail(ctx, SLQR_EINVAL, "request: SOLVE needs b and x");
      break;
    case SLQR_REQ_RELEASE:
      break;
    default:
      return fail(ctx, SLQR_EINVAL, "request: unknown kind %d", r.kind);
  }
  {
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    slqr_status st = server_start(ctx);
    if (st != SLQR_OK) return st;
  }
  Server *S = ctx->server;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    const uint64_t t = S->next_ticket++;
    Req &q = S->reqs[t];
    q.ticket = t;
    q.r = r;
    q.t_submit = Clock::now();
    S->incoming.push_back(t);
    *ticket = t;
  }
  S->cv.notify_one();
  return SLQR_OK;
}

extern "C" slqr_status slqr_poll(slqr_ctx *ctx, uint64_t ticket, slqr_result *out) {
  if (!ctx || !out) return SLQR_EINVAL;
  Server *S = ctx->server;
  if (!S) return SLQR_ENOTFOUND;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return SLQR_ENOTFOUND;
  if (it->second.state != 2) return SLQR_PENDING;
  *out = it->second.res;
  S->reqs.erase(it);
  return SLQR_OK;
}

extern "C" size_t slqr_server_bytes_in_use(slqr_ctx *ctx) {
  if (!ctx || !ctx->server) return 0;
  return ctx->server->used_bytes;
}
