// batch.cu -- host side of the batched H12 least squares (slqr_batch_factor,
// slqr_batch_factor_stacked, batch plans) and the batch autotuner.
//
// Each problem is the factorization of Alg. 2 (update_pivot_row, then
// update_trailing_non_pivot_row on every later column; Task 1 skip rule),
// optionally followed by Q^T b and the back-substitution (Section 1: the
// stored reflectors are reused by the solve); the kernels are in
// batch_core.cuh.  Problems are independent, so one CTA owns one problem at a
// time; persistent CTAs take the next problem from a device-side atomic
// counter over a list ordered costliest first (longest-processing-time
// first), the GPU descendant of the paper's shared main_queue of ready tasks
// (Alg. 5).
//
// Settings.  The panel width NB and the tile width TC of the kernels are
// chosen per size class of the problems (m <= 64, <= 128, <= 256, <= 512) and
// per precision, the batch form of the paper's alpha/beta task sizes
// (Section 4.1); for FP64 the classes m <= 64 and m <= 128 may also take the
// shared-memory-resident kernel (the whole problem in shared memory).
// slqr_batch_autotune searches them on a sample of the caller's shapes; by
// default every class uses NB = 16, TC = 32.  The problems of the classes that share a setting go into
// one persistent launch (with its own costliest-first order and work
// counter); the launches of a batch follow each other on the caller's stream,
// costliest group first.
#include "batch_core.cuh"

#include <algorithm>
#include <mutex>
#include <numeric>
#include <vector>

namespace slqr {

BatchKernels batch_kernels_nb16(int tc) {
  switch (tc) {
    case 16: return batch_kernels_of<16, 16>();
    case 32: return batch_kernels_of<16, 32>();
    case 64: return batch_kernels_of<16, 64>();
    default: return BatchKernels{};
  }
}

// kernels of a setting (null pointers when not valid); rm > 0: the
// shared-memory-resident FP64 kernel for problems of at most rm rows
static BatchKernels batch_kernels(int nb, int tc, int rm = 0) {
  if (rm > 0) {
    if (nb != 16 || tc != 32) return BatchKernels{};
    if (rm == 64) return batch_resident_kernels_of<16, 32, 64>();
    if (rm == 128) return batch_resident_kernels_of<16, 32, 128>();
    return BatchKernels{};
  }
  switch (nb) {
    case 8: return batch_kernels_nb8(tc);
    case 16: return batch_kernels_nb16(tc);
    case 32: return batch_kernels_nb32(tc);
    default: return BatchKernels{};
  }
}

// size classes of the problems by their row count
constexpr int kBClasses = 4;
static const int kBClassHi[kBClasses] = {64, 128, 256, kBMaxRows};
static int batch_class(int m) {
  for (int c = 0; c < kBClasses; ++c)
    if (m <= kBClassHi[c]) return c;
  return kBClasses - 1;
}

struct BatchSetting {
  int nb = kBNBDefault, tc = kBTCDefault;
  int rm = 0;                   // > 0: the resident FP64 kernel for m <= rm
  bool operator==(const BatchSetting &o) const { return nb == o.nb && tc == o.tc && rm == o.rm; }
};
// per precision (0: SLQR_FP64, 1: SLQR_FP32) and size class
static BatchSetting g_batch_setting[2][kBClasses];
static std::mutex g_batch_mu;

static BatchSetting batch_setting(int prec, int cls) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  return g_batch_setting[prec == SLQR_FP32 ? 1 : 0][cls];
}

static const BatchSetting kBSettings[] = {{8, 32}, {8, 64}, {16, 16}, {16, 32}, {16, 64},
                                          {32, 16}, {32, 32}, {32, 64}};

// the resident setting a size class may take (FP64 only): its row bound
static BatchSetting resident_setting(int cls) {
  BatchSetting s;
  s.rm = (cls <= 1) ? kBClassHi[cls] : 0;
  return s;
}

slqr_status init_batch_attrs(slqr_ctx *ctx) {
  cudaError_t e = cudaSuccess;
  for (const BatchSetting &s : kBSettings) {
    BatchKernels k = batch_kernels(s.nb, s.tc);
    if (!k.fp64 || !k.mixed) return fail(ctx, SLQR_ECUDA, "batch kernels (%d, %d) missing", s.nb, s.tc);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k.fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem_fp64);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k.mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)k.smem_mixed);
  }
  for (int c = 0; c < 2 && e == cudaSuccess; ++c) {
    const BatchSetting r = resident_setting(c);
    BatchKernels k = batch_kernels(r.nb, r.tc, r.rm);
    if (!k.fp64) return fail(ctx, SLQR_ECUDA, "resident batch kernel (%d rows) missing", r.rm);
    e = cudaFuncSetAttribute(k.fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem_fp64);
  }
  if (e != cudaSuccess)
    return fail(ctx, SLQR_ECUDA, "cudaFuncSetAttribute(batch): %s", cudaGetErrorString(e));
  return SLQR_OK;
}

}  // namespace slqr

using namespace slqr;

extern "C" int slqr_batch_max_rows(void) { return kBMaxRows; }

namespace slqr {

// One persistent launch of a batch: the problems of the classes that share
// one setting, at [begin, begin + count) of the order array.
struct BatchGroup {
  BatchSetting set;
  int begin = 0, count = 0, grid = 0;
  double cost = 0.0;
};

// A batch as the kernels see it: the problem table (in the order given), the
// order (per group, longest first), the groups and the algorithmic flops.
struct BatchSetup {
  std::vector<BatchProblem> probs;
  std::vector<int> order;
  std::vector<BatchGroup> groups;
  bool mixed = false;
  int max_grid = 0;
  double flops = 0.0;
  size_t table_bytes = 0, head = 0, af_bytes = 0, gt_bytes = 0;   // device layout
};

constexpr int kBMaxGroups = 64;   // work counters in the first 256 bytes of the layout

// Validate the arguments and build the setup (no device work).
static slqr_status batch_build(slqr_ctx *ctx, int count, const int *m, const int *n,
                               const int *ntop, double *const *A, const int *lda,
                               double *const *up, double *const *b, int prec, BatchSetup &bs) {
  if (count <= 0) return fail(ctx, SLQR_EINVAL, "count=%d must be > 0", count);
  if (!m || !n || !A || !lda) return fail(ctx, SLQR_EINVAL, "NULL size or pointer array");
  if (prec != SLQR_FP64 && prec != SLQR_FP32)
    return fail(ctx, SLQR_EINVAL, "precision %d not available for batches", prec);
  if (prec == SLQR_FP64 && !up) return fail(ctx, SLQR_EINVAL, "SLQR_FP64 needs the up arrays");
  if (prec == SLQR_FP32 && !b) return fail(ctx, SLQR_EINVAL, "SLQR_FP32 needs the b arrays");
  bs.probs.resize(count);
  std::vector<double> cost(count);
  for (int i = 0; i < count; ++i) {
    if (n[i] < 0 || m[i] < n[i] || m[i] > kBMaxRows)
      return fail(ctx, SLQR_EINVAL, "problem %d: need %d >= m >= n >= 0 (m=%d n=%d)", i,
                  kBMaxRows, m[i], n[i]);
    if (n[i] > 0 && (lda[i] < std::max(1, m[i]) || !A[i] ||
                     (prec == SLQR_FP64 && !up[i]) || (prec == SLQR_FP32 && !b[i])))
      return fail(ctx, SLQR_EINVAL, "problem %d: bad lda or NULL pointer", i);
    const int nt = ntop ? ntop[i] : 0;
    bs.probs[i] = BatchProblem{A[i], up ? up[i] : nullptr, b ? b[i] : nullptr, m[i], n[i], lda[i], nt};
    // flops of the factorization as this launch performs it (the stacked form
    // touches the m - n rows of C and one diagonal row per reflector)
    cost[i] = (nt > 0 ? 2.0 * (m[i] - n[i] + 1) * (double)n[i] * n[i]
                      : 2.0 * m[i] * (double)n[i] * n[i] - 2.0 * (double)n[i] * n[i] * n[i] / 3.0) +
              (b && b[i] ? 6.0 * m[i] * (double)n[i] : 0.0);
  }
  bs.flops = 0.0;
  for (int i = 0; i < count; ++i) bs.flops += cost[i];
  bs.mixed = (prec == SLQR_FP32);
  // group the problems by the setting of their size class
  std::vector<BatchSetting> cls_set(kBClasses);
  for (int c = 0; c < kBClasses; ++c) cls_set[c] = batch_setting(prec, c);
  std::vector<int> gidx(kBClasses, -1);            // class -> group
  for (int c = 0; c < kBClasses; ++c) {
    for (int c2 = 0; c2 < c; ++c2)
      if (cls_set[c2] == cls_set[c]) { gidx[c] = gidx[c2]; break; }
    if (gidx[c] < 0) {
      gidx[c] = (int)bs.groups.size();
      BatchGroup g;
      g.set = cls_set[c];
      bs.groups.push_back(g);
    }
  }
  std::vector<std::vector<int>> members(bs.groups.size());
  for (int i = 0; i < count; ++i) {
    const int g = gidx[batch_class(m[i])];
    members[g].push_back(i);
    bs.groups[g].cost += cost[i];
  }
  // costliest group first; longest problem first inside each group
  std::vector<int> gorder(bs.groups.size());
  std::iota(gorder.begin(), gorder.end(), 0);
  std::stable_sort(gorder.begin(), gorder.end(),
                   [&](int a, int c) { return bs.groups[a].cost > bs.groups[c].cost; });
  std::vector<BatchGroup> groups;
  bs.order.clear();
  for (int g : gorder) {
    if (members[g].empty()) continue;
    std::stable_sort(members[g].begin(), members[g].end(),
                     [&](int a, int c) { return cost[a] > cost[c]; });
    BatchGroup grp = bs.groups[g];
    grp.begin = (int)bs.order.size();
    grp.count = (int)members[g].size();
    bs.order.insert(bs.order.end(), members[g].begin(), members[g].end());
    BatchKernels k = batch_kernels(grp.set.nb, grp.set.tc, grp.set.rm);
    if (bs.mixed ? !k.mixed : !k.fp64)
      return fail(ctx, SLQR_EINVAL, "batch setting (%d, %d, resident %d) has no kernel here",
                  grp.set.nb, grp.set.tc, grp.set.rm);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, bs.mixed ? k.mixed : k.fp64, kThreads, bs.mixed ? k.smem_mixed : k.smem_fp64);
    if (e != cudaSuccess || per_sm < 1)
      return fail(ctx, SLQR_ECUDA, "batch occupancy: %s", cudaGetErrorString(e));
    grp.grid = std::min(grp.count, per_sm * ctx->num_sms);
    bs.max_grid = std::max(bs.max_grid, grp.grid);
    groups.push_back(grp);
  }
  bs.groups = groups;
  // device layout: [work counters 256 B][problem table][order][per-CTA scratch (mixed)]
  bs.table_bytes = align_up(sizeof(BatchProblem) * count, 256);
  bs.head = align_up(256 + bs.table_bytes + sizeof(int) * count, 256);
  bs.af_bytes = bs.mixed ? (size_t)bs.max_grid * kBMaxRows * kBMaxRows * sizeof(float) : 0;
  bs.gt_bytes = bs.mixed ? (size_t)bs.max_grid * kBGtDoubles * sizeof(double) : 0;
  return SLQR_OK;
}

// The kernel launches of a batch whose table and order are already at `base`
// (one per group, in order, each with its own work counter).
static void batch_kernel_launch(const BatchSetup &bs, char *base, int *status, double *err,
                                cudaStream_t s) {
  unsigned *counters = (unsigned *)base;
  BatchProblem *d_probs = (BatchProblem *)(base + 256);
  int *d_order = (int *)(base + 256 + bs.table_bytes);
  for (size_t gi = 0; gi < bs.groups.size(); ++gi) {
    const BatchGroup &g = bs.groups[gi];
    BatchKernels k = batch_kernels(g.set.nb, g.set.tc, g.set.rm);
    if (!bs.mixed) {
      BatchParams bp{d_probs, d_order + g.begin, g.count, counters + gi, status};
      void *args[] = {&bp};
      cudaLaunchKernel(k.fp64, dim3(g.grid), dim3(kThreads), args, k.smem_fp64, s);
    } else {
      BatchMixedParams mp{d_probs, d_order + g.begin, g.count, counters + gi, status, err,
                          (float *)(base + bs.head), (double *)(base + bs.head + bs.af_bytes),
                          kBMaxRefine, kBRefineTol};
      void *args[] = {&mp};
      cudaLaunchKernel(k.mixed, dim3(g.grid), dim3(kThreads), args, k.smem_mixed, s);
    }
  }
}

// The launch behind slqr_batch_factor and slqr_batch_factor_stacked (ntop:
// NULL, or per problem the rows of its upper-triangular top block, 0 for a
// dense problem).  The context mutex is held by the caller.
slqr_status batch_launch(slqr_ctx *ctx, int count, const int *m, const int *n, const int *ntop,
                         double *const *A, const int *lda, double *const *up, double *const *b,
                         int prec, int *status, double *err, void *stream) {
  if (count < 0) return fail(ctx, SLQR_EINVAL, "count=%d < 0", count);
  if (count == 0) return SLQR_OK;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  BatchSetup bs;
  slqr_status st = batch_build(ctx, count, m, n, ntop, A, lda, up, b, prec, bs);
  if (st != SLQR_OK) return st;
  st = ensure_workspace(ctx, bs.head + bs.af_bytes + bs.gt_bytes);
  if (st != SLQR_OK) return st;
  char *base = (char *)ctx->ws.ptr;
  cudaStream_t s = (cudaStream_t)stream;
  e = cudaMemsetAsync(base, 0, 256, s);
  // (copies from pageable host memory return once the source has been staged)
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + 256, bs.probs.data(), sizeof(BatchProblem) * count,
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + 256 + bs.table_bytes, bs.order.data(), sizeof(int) * count,
                        cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "batch set-up: %s", cudaGetErrorString(e));
  int slot = prof_begin(ctx, s);
  batch_kernel_launch(bs, base, status, err, s);
  prof_end(ctx, s, slot, kBatch, bs.flops);
  ctx->launch_count += (long long)bs.groups.size() - 1;
  return check_launch(ctx, "batch_factor");
}

slqr_status batch_factor_locked(slqr_ctx *ctx, int count, const int *m, const int *n,
                                const int *ntop, double *const *A, const int *lda,
                                double *const *up, double *const *b, int prec, int *status,
                                double *err, void *stream) {
  if (!ctx) return SLQR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  return batch_launch(ctx, count, m, n, ntop, A, lda, up, b, prec, status, err, stream);
}

// Generic scratch entries in (-1, 1) from a hash of the index (the timing does
// not depend on the values, only on their being generic).
__global__ void batch_tune_fill_kernel(double *A, size_t count, unsigned long long salt) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x) {
    unsigned long long h = (i + 1 + salt) * 0x9E3779B97F4A7C15ull;
    h ^= h >> 31;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 27;
    A[i] = (double)(h >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

}  // namespace slqr

extern "C" slqr_status slqr_batch_factor(slqr_ctx *ctx, int count, const int *m, const int *n,
                                         double *const *A, const int *lda, double *const *up,
                                         double *const *b, int prec, int *status, double *err,
                                         void *stream) {
  NvtxRange nvtx_range("slqr_batch_factor");
  if (!ctx) return SLQR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  return batch_launch(ctx, count, m, n, nullptr, A, lda, up, b, prec, status, err, stream);
}

extern "C" slqr_status slqr_batch_factor_stacked(slqr_ctx *ctx, int count, const int *n,
                                                 const int *m_eq, double *const *A,
                                                 const int *lda, double *const *up,
                                                 double *const *b, int prec, int *status,
                                                 double *err, void *stream) {
  NvtxRange nvtx_range("slqr_batch_factor_stacked");
  if (!ctx) return SLQR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (count < 0) return fail(ctx, SLQR_EINVAL, "count=%d < 0", count);
  if (count > 0 && (!n || !m_eq)) return fail(ctx, SLQR_EINVAL, "NULL size array");
  std::vector<int> m(std::max(count, 0));
  for (int i = 0; i < count; ++i) {
    if (n[i] < 0 || m_eq[i] < 0)
      return fail(ctx, SLQR_EINVAL, "problem %d: need n, m_eq >= 0 (n=%d m_eq=%d)", i, n[i],
                  m_eq[i]);
    m[i] = n[i] + m_eq[i];
  }
  return batch_launch(ctx, count, m.data(), n, n, A, lda, up, b, prec, status, err, stream);
}

extern "C" int slqr_batch_classes(void) { return kBClasses; }

extern "C" int slqr_batch_class_rows(int m_class) {
  return (m_class >= 0 && m_class < kBClasses) ? kBClassHi[m_class] : 0;
}

extern "C" slqr_status slqr_batch_set_tuning(int prec, int m_class, int panel_width,
                                             int tile_cols, int resident) {
  if (prec != SLQR_FP64 && prec != SLQR_FP32) return SLQR_EINVAL;
  if (m_class < -1 || m_class >= kBClasses) return SLQR_EINVAL;
  BatchSetting s;
  if (resident) {
    // the resident kernel: FP64, one size class of at most 128 rows, (16, 32)
    if (prec != SLQR_FP64 || m_class < 0 || m_class > 1) return SLQR_EINVAL;
    if (!((panel_width == 16 && tile_cols == 32) || (panel_width == 0 && tile_cols == 0)))
      return SLQR_EINVAL;
    s = resident_setting(m_class);
  } else if (panel_width != 0 || tile_cols != 0) {
    bool ok = false;
    for (const BatchSetting &v : kBSettings) ok |= (v.nb == panel_width && v.tc == tile_cols);
    if (!ok) return SLQR_EINVAL;
    s.nb = panel_width;
    s.tc = tile_cols;
  }
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (int c = 0; c < kBClasses; ++c)
    if (m_class < 0 || c == m_class) g_batch_setting[prec == SLQR_FP32 ? 1 : 0][c] = s;
  return SLQR_OK;
}

extern "C" slqr_status slqr_batch_get_tuning(int prec, int m_class, int *panel_width,
                                             int *tile_cols, int *resident) {
  if ((prec != SLQR_FP64 && prec != SLQR_FP32) || m_class < 0 || m_class >= kBClasses)
    return SLQR_EINVAL;
  BatchSetting s = batch_setting(prec, m_class);
  if (panel_width) *panel_width = s.nb;
  if (tile_cols) *tile_cols = s.tc;
  if (resident) *resident = s.rm > 0 ? 1 : 0;
  return SLQR_OK;
}

extern "C" slqr_status slqr_batch_autotune(slqr_ctx *ctx, int prec, int count, const int *m,
                                           const int *n, int sample, int *panel_width,
                                           int *tile_cols, int *resident, double *ms_out) {
  NvtxRange nvtx_range("slqr_batch_autotune");
  if (!ctx) return SLQR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (prec != SLQR_FP64 && prec != SLQR_FP32)
    return fail(ctx, SLQR_EINVAL, "precision %d not available for batches", prec);
  if (count < 0 || (count > 0 && (!m || !n)))
    return fail(ctx, SLQR_EINVAL, "autotune: bad shape list (count=%d)", count);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  // the scratch batch: `sample` problems, every (count / sample)-th of the
  // caller's shapes, or drawn from the default law (m ~ U{16..512},
  // n ~ U{ceil(m/4)..m}, the 20,000-problem workload) with a fixed LCG
  const int ns_ = sample > 0 ? sample : (count > 0 ? std::min(count, 3000) : 3000);
  std::vector<int> mv, nv;
  if (count > 0) {
    for (int i = 0; i < ns_ && i < count; ++i) {
      const int k = (int)((long long)i * count / std::min(ns_, count));
      if (n[k] < 0 || m[k] < n[k] || m[k] > kBMaxRows)
        return fail(ctx, SLQR_EINVAL, "autotune: problem %d: need %d >= m >= n >= 0", k, kBMaxRows);
      if (n[k] == 0) continue;
      mv.push_back(m[k]);
      nv.push_back(n[k]);
    }
  } else {
    unsigned long long r = 0x2545F4914F6CDD1Dull;
    auto next = [&](int a, int b) {
      r = r * 6364136223846793005ull + 1442695040888963407ull;
      return a + (int)((r >> 33) % (unsigned long long)(b - a + 1));
    };
    for (int i = 0; i < ns_; ++i) {
      mv.push_back(next(16, kBMaxRows));
      nv.push_back(next((mv.back() + 3) / 4, mv.back()));
    }
  }
  const int cnt = (int)mv.size();
  if (cnt == 0) return fail(ctx, SLQR_EINVAL, "autotune: no problem with n > 0");
  std::vector<int> ldv(mv);
  size_t a_total = 0, b_total = 0, n_total = 0;
  std::vector<double> cls_cost(kBClasses, 0.0);
  for (int i = 0; i < cnt; ++i) {
    a_total += (size_t)mv[i] * nv[i];
    b_total += mv[i];
    n_total += nv[i];
    cls_cost[batch_class(mv[i])] += 2.0 * mv[i] * (double)nv[i] * nv[i];
  }
  const int pi = prec == SLQR_FP32 ? 1 : 0;
  BatchSetting cur[kBClasses];
  {
    std::lock_guard<std::mutex> lk2(g_batch_mu);
    for (int c = 0; c < kBClasses; ++c) cur[c] = g_batch_setting[pi][c];
  }
  const BatchSetting saved[kBClasses] = {cur[0], cur[1], cur[2], cur[3]};
  auto apply = [&](const BatchSetting *set) {
    std::lock_guard<std::mutex> lk2(g_batch_mu);
    for (int c = 0; c < kBClasses; ++c) g_batch_setting[pi][c] = set[c];
  };
  double *A0 = nullptr, *Aw = nullptr, *B0 = nullptr, *Bw = nullptr, *UP = nullptr, *derr = nullptr;
  int *dstat = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&A0, a_total * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&Aw, a_total * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&B0, b_total * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&Bw, b_total * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&UP, n_total * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&dstat, cnt * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&derr, cnt * sizeof(double));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  std::vector<double *> Ap(cnt), Bp(cnt), Up(cnt);
  {
    size_t ao = 0, bo = 0, no = 0;
    for (int i = 0; i < cnt; ++i) {
      Ap[i] = Aw + ao;
      Bp[i] = Bw + bo;
      Up[i] = UP + no;
      ao += (size_t)mv[i] * nv[i];
      bo += mv[i];
      no += nv[i];
    }
  }
  if (e == cudaSuccess) {
    batch_tune_fill_kernel<<<4 * ctx->num_sms, 256, 0, s>>>(A0, a_total, 0);
    batch_tune_fill_kernel<<<4 * ctx->num_sms, 256, 0, s>>>(B0, b_total, a_total);
    e = cudaGetLastError();
  }
  slqr_status st = SLQR_OK;
  // the sample batch under the settings now in the table: best of two runs
  // after a warm-up
  auto time_it = [&]() -> double {
    float tmin = 1e30f;
    for (int rep = 0; rep < 3 && st == SLQR_OK && e == cudaSuccess; ++rep) {
      cudaMemcpyAsync(Aw, A0, a_total * sizeof(double), cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(Bw, B0, b_total * sizeof(double), cudaMemcpyDeviceToDevice, s);
      cudaEventRecord(e0, s);
      st = batch_launch(ctx, cnt, mv.data(), nv.data(), nullptr, Ap.data(), ldv.data(), Up.data(),
                        Bp.data(), prec, dstat, derr, s);
      cudaEventRecord(e1, s);
      e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tmin = std::min(tmin, ms);
    }
    return tmin;
  };
  const double t_before = time_it();
  double t_best = t_before;
  // greedy coordinate search: the classes costliest first, each trying every
  // setting with the others held, a change kept only when the whole sample
  // batch gets faster (so a split into several launches must pay for itself)
  std::vector<int> corder(kBClasses);
  std::iota(corder.begin(), corder.end(), 0);
  std::stable_sort(corder.begin(), corder.end(),
                   [&](int a, int c) { return cls_cost[a] > cls_cost[c]; });
  for (int c : corder) {
    if (cls_cost[c] == 0.0) continue;
    std::vector<BatchSetting> cands(std::begin(kBSettings), std::end(kBSettings));
    if (prec == SLQR_FP64 && c <= 1) cands.push_back(resident_setting(c));
    for (const BatchSetting &cand : cands) {
      if (st != SLQR_OK || e != cudaSuccess) break;
      if (cand == cur[c]) continue;
      BatchSetting trial[kBClasses] = {cur[0], cur[1], cur[2], cur[3]};
      trial[c] = cand;
      apply(trial);
      const double t = time_it();
      if (t < 0.99 * t_best) {              // a clear gain, not timing noise
        t_best = t;
        cur[c] = cand;
      }
    }
    apply(cur);
  }
  cudaFree(A0);
  cudaFree(Aw);
  cudaFree(B0);
  cudaFree(Bw);
  cudaFree(UP);
  cudaFree(dstat);
  cudaFree(derr);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (e != cudaSuccess || st != SLQR_OK) {
    apply(saved);
    if (st != SLQR_OK) return st;
    cudaGetLastError();
    return fail(ctx, SLQR_ENOMEM, "batch autotune: %s", cudaGetErrorString(e));
  }
  apply(cur);
  for (int c = 0; c < kBClasses; ++c) {
    if (panel_width) panel_width[c] = cur[c].nb;
    if (tile_cols) tile_cols[c] = cur[c].tc;
    if (resident) resident[c] = cur[c].rm > 0 ? 1 : 0;
  }
  if (ms_out) {
    ms_out[0] = t_before;
    ms_out[1] = t_best;
  }
  return SLQR_OK;
}

// --------------------------------------------------------------------------
// Batch plans: the same batch launched many times (an SLSQP loop refactors
// problems of unchanged shapes at every iteration).  The problem table and
// the order go to the device once; the launch (reset of the work counter and
// the persistent kernel) is captured into a CUDA graph and replayed.
// --------------------------------------------------------------------------
struct slqr_batch_plan {
  slqr_ctx *ctx = nullptr;
  slqr::BatchSetup bs;
  int count = 0;
  char *dev = nullptr;               // counter, table, order, mixed scratch
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" void slqr_batch_plan_destroy(slqr_batch_plan *plan) {
  if (!plan) return;
  cudaSetDevice(plan->ctx->device);
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  if (plan->dev) cudaFree(plan->dev);
  delete plan;
}

extern "C" slqr_status slqr_batch_plan_create(slqr_ctx *ctx, int count, const int *m,
                                              const int *n, const int *ntop, double *const *A,
                                              const int *lda, double *const *up,
                                              double *const *b, int prec, int *status,
                                              double *err, slqr_batch_plan **out) {
  if (!ctx || !out) return SLQR_EINVAL;
  NvtxRange nvtx_range("slqr_batch_plan_create");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  *out = nullptr;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  slqr_batch_plan *plan = new (std::nothrow) slqr_batch_plan();
  if (!plan) return SLQR_ENOMEM;
  plan->ctx = ctx;
  plan->count = count;
  slqr_status st = batch_build(ctx, count, m, n, ntop, A, lda, up, b, prec, plan->bs);
  if (st != SLQR_OK) {
    delete plan;
    return st;
  }
  const size_t bytes = plan->bs.head + plan->bs.af_bytes + plan->bs.gt_bytes;
  if (ctx->hbm_budget && bytes > ctx->hbm_budget) {
    delete plan;
    return fail(ctx, SLQR_EBUSY, "batch plan of %zu bytes exceeds the HBM budget", bytes);
  }
  e = cudaMalloc(&plan->dev, bytes);
  if (e == cudaSuccess)
    e = cudaMemcpy(plan->dev + 256, plan->bs.probs.data(), sizeof(BatchProblem) * count,
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(plan->dev + 256 + plan->bs.table_bytes, plan->bs.order.data(),
                   sizeof(int) * count, cudaMemcpyHostToDevice);
  cudaStream_t cs = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemsetAsync(plan->dev, 0, 256, cs);
    batch_kernel_launch(plan->bs, plan->dev, status, err, cs);
    e = cudaStreamEndCapture(cs, &plan->graph);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&plan->exec, plan->graph, 0);
  if (cs) cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    slqr_batch_plan_destroy(plan);
    return fail(ctx, SLQR_ECUDA, "batch plan: %s", cudaGetErrorString(e));
  }
  *out = plan;
  return SLQR_OK;
}

extern "C" slqr_status slqr_batch_plan_launch(slqr_batch_plan *plan, void *stream) {
  if (!plan) return SLQR_EINVAL;
  NvtxRange nvtx_range("slqr_batch_plan_launch");
  slqr_ctx *ctx = plan->ctx;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaError_t e = cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  int slot = prof_begin(ctx, s);
  if (e == cudaSuccess) e = cudaGraphLaunch(plan->exec, s);
  prof_end(ctx, s, slot, kBatch, plan->bs.flops);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "batch plan launch: %s", cudaGetErrorString(e));
  return SLQR_OK;
}
