// slqr_internal.cuh -- shared declarations of the libslqr CUDA sources.
//
// Layout conventions: matrices are FP64, column-major, element (i, j) of a
// matrix with leading dimension ld at p[i + j*ld].  The factorization runs in
// panels of NB reflectors (compact-WY form, see factor.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <string>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/slqr.h"

#define SLQR_IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

namespace slqr {

constexpr int kThreads = 256;          // threads per CTA of the tiled kernels
constexpr int kMaxPanelRowsPerCta = 384;  // rows of a panel one CTA holds in smem (NB=64)

// Upper bound on spin iterations of a device-side wait (each iteration sleeps
// ~100 ns), after which the kernel records SLQR_ETIMEOUT and returns.  The
// default of a context's limit (slqr_set_spin_limit), and the fixed limit of
// the tensor-core kernels' mbarrier waits.
constexpr unsigned kSpinLimit = 1u << 24;

// Device status word codes (same values as the C ABI).
constexpr int kStatusOk = 0;

struct Workspace {
  void *ptr = nullptr;
  size_t bytes = 0;
};

// Kernel families timed by the optional profiler (slqr_profile).
enum KernelId {
  kPanel = 0, kVtx = 1, kTw = 2, kUpd = 3, kWyRebuild = 4, kTrsm = 5, kBatch = 6,
  kNumKernelIds = 7
};

struct ProfRecord {
  cudaEvent_t start, stop;
  int kid;
  double flops;
};

struct Profiler {
  bool on = false;
  std::vector<ProfRecord> pending;
  std::vector<cudaEvent_t> free_events;
  double ms[kNumKernelIds] = {0};
  long long launches[kNumKernelIds] = {0};
  double flops[kNumKernelIds] = {0};
};

}  // namespace slqr

namespace slqr { struct Server; }

struct slqr_ctx {
  int device = 0;
  int num_sms = 0;
  size_t hbm_budget = 0;
  size_t smem_optin = 0;
  int *d_status = nullptr;             // device status word
  slqr::Workspace ws;                  // grown on demand
  slqr::Workspace ws2;                 // buffers of the mixed-precision driver
  slqr::Profiler prof;                 // optional CUDA-event timing per kernel family
  cudaStream_t aux_stream = nullptr;   // look-ahead panels run here
  cudaEvent_t ev_start = nullptr, ev_ready = nullptr, ev_panel = nullptr;
  long long launch_count = 0;          // kernels launched by this context
  slqr::Server *server = nullptr;      // request loop (slqr_submit), started lazily
  // FP32 factorization: trailing update on tcgen05 (0: FMA pipe, 1: TF32,
  // 2: BF16 split in hi + lo, with the BF16 shadows of the matrix below)
  int tc_mode = 0;
  void *sh_hi = nullptr, *sh_lo = nullptr;
  // limit of the polled exchanges and grid barriers of the cooperative kernels
  unsigned spin_limit = slqr::kSpinLimit;
  std::string last_error;
  // serialises the entry points of one context; recursive so that a driver
  // (the mixed-precision solve's FP64 fallback) can call other entry points
  std::recursive_mutex mu;
};

namespace slqr {

// NVTX range over one entry point (visible in Nsight timelines; free when no
// tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Record an error message in the context and return the status.
slqr_status fail(slqr_ctx *ctx, slqr_status st, const char *fmt, ...);

// Make sure the workspace holds at least `bytes`; returns SLQR_OK or an error.
slqr_status ensure_workspace(slqr_ctx *ctx, size_t bytes);
slqr_status ensure_workspace2(slqr_ctx *ctx, size_t bytes);
// Checked build: verify the workspaces' guard zones (SLQR_ECHECK when one was
// overwritten); SLQR_OK otherwise and in the normal build.
slqr_status check_workspaces(slqr_ctx *ctx);

// Check the last launch; returns SLQR_OK or SLQR_ECUDA with the message set.
slqr_status check_launch(slqr_ctx *ctx, const char *what);

// Profiling around one launch: begin returns a slot (or -1 when off); end
// records the stop event and the algorithmic flops of that launch.  Both also
// count the launch.
int prof_begin(slqr_ctx *ctx, cudaStream_t stream);
void prof_end(slqr_ctx *ctx, cudaStream_t stream, int slot, int kid, double flops);

// Stop the request loop of a context (waits for its requests to finish).
void server_stop(slqr_ctx *ctx);

// Opt kernels into large dynamic shared memory (once per device).
slqr_status init_kernel_attrs(slqr_ctx *ctx);
slqr_status init_batch_attrs(slqr_ctx *ctx);
slqr_status init_tc_attrs(slqr_ctx *ctx);

// X -= V W' for a full 64-wide panel on a 128 x 64 tile grid with tcgen05
// (TF32 operands, FP32 accumulation in tensor memory), X = columns
// [xcol0, xcol0 + N) of A from row k0; Wt = W'^T ([column][64]); Vr: scratch
// of M x 64 floats for the row-major V.  Returns false (nothing launched) when
// a tensor map cannot be encoded; see tc_update.cu.
bool launch_upd_tc(const float *A, int lda, const double *Vtop, int k0, int M, int xcol0, int N,
                   const float *Wt, float *Vr, int *status, cudaStream_t stream);
// The BF16-split (hi + lo) variants (tc_bf16.cu): shadows of a region of the
// FP32 matrix, and the two products reading / writing those shadows.
slqr_status init_bf16_attrs(slqr_ctx *ctx);
void split_bf16_region(const float *A, int lda, int r0, int r1, int c0, int c1, void *hi,
                       void *lo, int num_sms, cudaStream_t stream);
int launch_vtx_bf16(const float *A, int lda, const void *sh_hi, const void *sh_lo,
                    const double *Vtop, int k0, int M, int xcol0, int N, float *Wp,
                    size_t work_elems, int num_sms, int *status, cudaStream_t stream,
                    void (*vtop_part)(const float *, int, const double *, int, int, const float *,
                                      int, int, float *, cudaStream_t));
bool launch_upd_bf16(const float *A, int lda, void *sh_hi, void *sh_lo, const double *Vtop,
                     int k0, int M, int xcol0, int N, const float *Wt, void *scratch,
                     int num_sms, int *status, cudaStream_t stream);
// W = V^T X partials with TMA + tcgen05 for a full 64-wide panel; returns the
// number of partial slices written to Wp (0: not applicable).
int launch_vtx_tc(const float *A, int lda, const double *Vtop, int k0, int M, int xcol0, int N,
                  float *Wp, size_t work_elems, int num_sms, int *status, cudaStream_t stream,
                  void (*vtop_part)(const float *, int, const double *, int, int, const float *, int,
                                    int, float *, cudaStream_t));

// slqr_batch_factor with a per-problem stacked top block (ntop[i] rows, 0 for a
// dense problem; ntop may be NULL); takes the context mutex.
slqr_status batch_factor_locked(slqr_ctx *ctx, int count, const int *m, const int *n,
                                const int *ntop, double *const *A, const int *lda,
                                double *const *up, double *const *b, int prec, int *status,
                                double *err, void *stream);

// --------------------------------------------------------------------------
// device helpers shared by the cooperative kernels
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void record_status(int *status, int code) {
  atomicCAS(status, kStatusOk, code);
}

// Checked build (SLQR_CHECKED): a condition that must hold for an access or
// a launch; when it fails the first failure is recorded as SLQR_ECHECK and
// the caller skips the access.  Normal build: always true, no code.
#ifdef SLQR_CHECKED
__device__ __forceinline__ bool slqr_check(bool ok, int *status) {
  if (!ok) atomicCAS(status, kStatusOk, SLQR_ECHECK);
  return ok;
}
#else
__device__ __forceinline__ bool slqr_check(bool ok, int *) { return true; }
#endif

// Arrive at a grid barrier (a monotonic arrival counter) and wait, bounded by
// `limit` polls, until it reaches `target`.  Returns false after recording
// SLQR_ETIMEOUT.  Cooperative launches only (every CTA resident).
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned target, int *status,
                                             int *s_ok, unsigned limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    unsigned it = 0;
    int ok = 1;
    while (ld_acquire_u32(bar) < target) {
      if (++it > limit) { ok = 0; break; }
      if (it > 256) __nanosleep(64);
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  if (!*s_ok) {
    if (threadIdx.x == 0) record_status(status, SLQR_ETIMEOUT);
    return false;
  }
  return true;
}

// Panel width used for an m x n factorization.
int panel_width(int m, int n);

// The panel factored by one thread-block cluster (panel_cluster.cu): the
// panel's M = m - k0 - skip rows split over `ctas` CTAs of R rows each
// (R >= nbw), each slice in shared memory, the per-column sums exchanged
// through distributed shared memory.
struct ClusterPanelParams {
  void *A;             // T * (float or double), column-major, leading dimension lda
  double *up;          // global up array
  double *wy;          // this panel's compact-WY block (Vtop | G | tau)
  int m, lda, k0, nbw;
  int skip;            // rows skipped after the panel's top nbw rows (stacked [L^T; C])
  int stacked;         // stacked [L^T; C]: the diagonal block's strict lower part is zero
  int R;               // rows per CTA
  int *status;         // device status word (SLQR_ETIMEOUT when a wait gives up)
  unsigned spin;       // polls of a bounded wait before it gives up
};
size_t cluster_panel_smem_bytes(int nb, int R, size_t elem);
// largest R for panel width nb and element size elem (0: no cluster panel)
int cluster_panel_rows_max(const slqr_ctx *ctx, int nb, size_t elem);
slqr_status init_cluster_attrs(slqr_ctx *ctx);
// whether a cluster of `ctas` CTAs of R rows each can be resident on the device
bool cluster_panel_fits(slqr_ctx *ctx, bool f32, int nb, int ctas, int R);
// the register-resident FP32 panel of width 64 (panel_cluster_reg.cu): rows
// per lane for R rows per CTA (0: too tall), its shared memory, its kernel
int cluster_reg_rows_per_lane(int R);
size_t cluster_reg_smem_bytes(int R);
const void *cluster_reg_kernel(int rpl);
int cluster_panel_variant();
void set_cluster_panel_variant(int v);
// the setting of slqr_set_panel_cluster (-1: no cluster kernels at all)
int panel_cluster_setting();
// Q^T f (trans) or Q f for one vector by a cluster of CTAs (qvec_cluster.cu),
// for the FP32 factorization A32 with the explicit T of each panel (Tm);
// false when the cluster does not fit (nothing launched), else *st is the
// launch status.
bool apply_q_cluster(slqr_ctx *ctx, const float *A32, int lda32, const double *up, int m, int K,
                     int nb, int np, const float *Tm, float *f, bool trans, cudaStream_t s,
                     slqr_status *st);
bool apply_q_cluster(slqr_ctx *ctx, const float *A32, int lda32, const double *up, int m, int K,
                     int nb, int np, const double *Tm, double *f, bool trans, cudaStream_t s,
                     slqr_status *st);
// R y = c (upper) or R^T y = c for the FP32 R by a cluster of CTAs
// (trsv_cluster.cu), with the inverses of R's 64 x 64 diagonal blocks; false
// when it does not apply (n not a multiple of 64 or above 4096, alignment),
// nothing launched, else *st is the launch status.
bool trsv_cluster(slqr_ctx *ctx, bool upper, const float *R, int lda, int n, const float *Rinv,
                  const int *zblk, float *y, int *zero_flag, cudaStream_t s, slqr_status *st);
bool trsv_cluster(slqr_ctx *ctx, bool upper, const float *R, int lda, int n, const double *Rinv,
                  const int *zblk, double *y, int *zero_flag, cudaStream_t s, slqr_status *st);
slqr_status launch_cluster_panel(slqr_ctx *ctx, bool f32, int nb, const ClusterPanelParams &pp,
                                 int ctas, cudaStream_t stream);
// Cluster size of the panel for a panel of M rows (0: the cooperative panel)
// under the setting of slqr_set_panel_cluster.
int panel_cluster_ctas(slqr_ctx *ctx, bool f32, int nb, int M, int nbw);

// Look-ahead update of the next panel's columns (at most 64) of an FP32
// factorization with panels of width 64, in one cooperative launch
// (lookahead.cu): false when it does not apply (setting off, rows per CTA
// above its limit, workspace) or the launch was refused, nothing launched;
// else *st = SLQR_OK and bar_base advanced past its two grid barriers.
bool lookahead_update_f32(slqr_ctx *ctx, int m, int k0, int nbw, float *A, int lda,
                          const double *wy_panel, int cb, int N, float *work, size_t work_elems,
                          unsigned *bar, unsigned &bar_base, cudaStream_t stream,
                          slqr_status *st);
slqr_status init_lookahead_attrs(slqr_ctx *ctx);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// --------------------------------------------------------------------------
// Compact-WY store: per panel p, at offset p * wy_panel_doubles(nb):
//   [0, nb*nb)          Vtop: top nb x nb block of V (column-major, ld nb):
//                       0 above the diagonal, up on it, reflector tails below
//   [nb*nb, 2*nb*nb)    G: strict upper triangle of V^T V (column-major, ld nb)
//   [2*nb*nb, +nb)      tau_j = -1/b_j (0 for a skipped or absent reflector)
// --------------------------------------------------------------------------
__host__ __device__ inline size_t wy_panel_doubles(int nb) { return 2 * (size_t)nb * nb + nb; }
__host__ __device__ inline int num_panels(int K, int nb) { return (K + nb - 1) / nb; }

// Number of reflectors min(m-1, n).
__host__ __device__ inline int num_reflectors(int m, int n) {
  int k = m - 1 < n ? m - 1 : n;
  return k < 0 ? 0 : k;
}

// --- launchers (defined in factor.cu / apply.cu / solve.cu) -------------
// Trailing update of columns [c0, c0+N) of the matrix X (rows [k0, m), leading
// dimension ldx) by the panel (V from A/Vtop, G, tau) at offset k0 of width nbw.
// skip: rows left out after the panel's top nbw rows (stacked [L^T; C], see
// panel_row in factor.cu); 0 for a dense matrix.
slqr_status apply_panel_update(slqr_ctx *ctx, int m, int k0, int nbw, int nb,
                               const double *A, int lda, const double *wy_panel,
                               double *X, int ldx, int N, double *work, size_t work_doubles,
                               cudaStream_t stream, int skip = 0);
size_t panel_update_work_doubles(int m, int N, int nb, int num_sms);

// Persistent state of one low-precision factorization of the mixed-precision
// path (mixed.cu): the FP32 copy of A D, up, the compact-WY store, the column
// scales D and the explicit T of every panel, in memory the caller owns
// (mixed_state_bytes(m, n) bytes).  The request loop keeps one per resident
// mixed-precision handle.
struct MixedFactorState {
  int m = 0, n = 0, prec = 0, nb = 0, K = 0, np = 0, lda32 = 0;
  int ntop = 0;                        // > 0: stacked [L^T; C], top block of ntop rows
  float *A32 = nullptr;
  double *up = nullptr, *wy = nullptr, *colscale = nullptr;
  float *Tm32 = nullptr;
};
size_t mixed_state_bytes(int m, int n);
// Factor A (FP64, lda) in precision prec into state_mem; asynchronous on s.
slqr_status mixed_factor_into(slqr_ctx *ctx, int m, int n, const double *A, int lda, int prec,
                              int ntop, void *state_mem, MixedFactorState *fs, cudaStream_t s);
// The refinement (and optional FP64 fallback) of x for b with that state and
// the same FP64 A; synchronous, as slqr_lstsq_mixed_ex.
slqr_status mixed_solve_with(slqr_ctx *ctx, const MixedFactorState &fs, const double *A, int lda,
                             const double *b, double *x, const slqr_mixed_opts &o,
                             slqr_mixed_info *info, cudaStream_t s);

// FP32 factorization (up and the compact-WY store in FP64) used by the
// mixed-precision driver.
// ntop > 0: A = [L^T; C] with an upper-triangular top block of ntop rows (the
// structure-aware factorization, as factor_impl).
slqr_status factor_f32(slqr_ctx *ctx, int m, int n, float *A, int lda, double *up, double *wy,
                       cudaStream_t stream, int ntop = 0);

}  // namespace slqr
