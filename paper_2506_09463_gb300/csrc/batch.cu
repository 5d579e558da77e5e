// batch.cu -- many independent H12 least-squares problems in one persistent
// launch (slqr_batch_factor).
//
// Each problem is the factorization of Alg. 2 (update_pivot_row, then
// update_trailing_non_pivot_row on every later column; Task 1 skip rule),
// optionally followed by Q^T b and the back-substitution (Section 1: the
// stored reflectors are reused by the solve).  Problems are independent, so
// one CTA owns one problem at a time; persistent CTAs take the next problem
// from a device-side atomic counter over a list ordered costliest first
// (longest-processing-time first), the GPU descendant of the paper's shared
// main_queue of ready tasks (Alg. 5).
//
// Inside a CTA a problem is factored in panels of kBNB reflectors:
//  * the panel (rows k0..m-1, kBNB columns) sits in shared memory; each column
//    is one block-level reduction (scaled norm, dots of the column tail with
//    the other panel columns, which also give striu(V^T V)), then the update
//    of the later panel columns;
//  * the trailing columns (and b, as one more column) are updated in tiles of
//    32 columns: W = V^T C (8 lanes per column, each over every 8th row),
//    then W' = T^T W by forward substitution (one lane per column), then
//    C -= V W' (the same lanes as W).
// All arithmetic is FP64 (DFMA).
#include "slqr_internal.cuh"

#include <math_constants.h>

#include <algorithm>
#include <numeric>
#include <vector>

namespace slqr {

constexpr int kBNB = 16;          // reflectors per panel
constexpr int kBMaxRows = 512;    // rows of a batched problem (panel slice in smem)
constexpr int kBCols = 32;        // trailing columns per tile
constexpr int kBWarps = kThreads / 32;
constexpr int kBRowGroups = 8;                  // lanes of a column in the tile phases
constexpr int kBGroupCols = 32 / kBRowGroups;   // columns of one warp in the tile phases
static_assert(kBGroupCols * kBWarps == kBCols, "one column group per warp covers the tile");
constexpr int kBMaxRefine = 12;        // refinement sweeps of the mixed path
constexpr double kBRefineTol = 1e-14;  // stop when ||dx||_inf <= tol ||x||_inf
constexpr double kBStallOk = 1e-10;    // a stalled refinement is accepted below this

struct BatchProblem {
  double *A;
  double *up;
  double *b;
  int m, n, lda;
  int ntop;          // > 0: stacked [L^T; C] with an upper-triangular top block of ntop rows
};

struct BatchParams {
  const BatchProblem *probs;
  const int *order;
  int count;
  unsigned *counter;
  int *status;
};

// Exponent bits of |x| (as a double): the integer order of these bit patterns
// is the numeric order, so a max over them finds the largest magnitude.
template <typename T>
__device__ __forceinline__ unsigned b_abs_hi(T x) {
  return (unsigned)((unsigned long long)__double_as_longlong((double)x) >> 32) & 0x7fffffffu;
}

// 2^e as a double for e in [-1022, 1023] (exact; built from the exponent bits)
__device__ __forceinline__ double b_pow2(int e) {
  return __longlong_as_double((long long)(e + 1023) << 52);
}

// Sum of 16 per-lane values acc[0..15] over the 8 lanes g = lane & 7 of one
// column group by a halving exchange: at each of three levels a lane keeps
// half of its values and adds the other half received from its partner (14
// shuffles and adds per lane instead of 48 for 16 separate butterflies).
// Afterwards lane g holds the totals of values 2g and 2g + 1 in acc[0], acc[1].
template <typename T>
__device__ __forceinline__ void b_group8_sum16(T (&acc)[kBNB], int g) {
  static_assert(kBNB == 16, "three halving levels over 8 lanes");
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const bool hi = (g & 4) != 0;
    const T send = hi ? acc[i] : acc[i + 8];
    const T keep = hi ? acc[i + 8] : acc[i];
    acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const bool hi = (g & 2) != 0;
    const T send = hi ? acc[i] : acc[i + 4];
    const T keep = hi ? acc[i + 4] : acc[i];
    acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool hi = (g & 1) != 0;
    const T send = hi ? acc[i] : acc[i + 2];
    const T keep = hi ? acc[i + 2] : acc[i];
    acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
  }
}

__device__ __forceinline__ float b_warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double b_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Shared-memory layout of the batched kernels.  The panel slice Ps and the
// W tile are of the working type T (double for SLQR_FP64, float for the
// mixed-precision path); the small per-panel quantities are double.
__host__ __device__ constexpr size_t align_up_c(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <typename T>
struct BatchSmem {
  static constexpr int kPanel = kBNB * kBMaxRows;       // Ps[c][r]
  static constexpr int kW = kBNB * (kBCols + 1);        // Wt[a][col]
  static constexpr int kG = kBNB * kBNB;                // G[q][j] (ld kBNB)
  // T copies of the panel's G and tau for W' = T^T W (phase B)
  static constexpr size_t kBytesT = (size_t)(kPanel + kW + kG + kBNB) * sizeof(T);
  static constexpr int kMisc = 7 * kBNB + 8;  // dots, sigma, tau, up, scale, 1/scale, fast, norm
  static constexpr size_t kBytes = align_up_c(kBytesT, 16) + (size_t)(kG + kMisc) * sizeof(double);
};

// The H12 factorization of one m x n problem by one CTA (see the file
// header).  T == double: all FP64.  T == float: dot products, updates, the
// norm, cl, up, b and sigma in FP32 (FP64 for a column whose power-of-two
// scale is extreme for FP32), up, tau and G stored in FP64.  When
// G_out/tau_out are given, each panel's
// striu(V^T V) and tau are kept there (the mixed path reuses them to apply Q).
// Bcol (T == double only) is an extra right-hand-side column updated with the
// trailing columns, giving Q^T b.
//
// ntop > 0: A = [L^T; C] with an upper-triangular top block of ntop rows.  A
// panel at k0 then uses its own nbw diagonal rows and the rows of C only (row
// r of the panel is matrix row k0 + r for r < nbw, k0 + skip + r below, with
// skip = ntop - k0 - nbw): the rows between are zero in every reflector and
// untouched by the update.
template <typename T>
__device__ void batch_factor_core(T *A, int lda, int m, int n, double *up_out, double *Bcol,
                                  double *G_out, double *tau_out, char *smraw, int ntop) {
  using SM = BatchSmem<T>;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g8 = lane & (kBRowGroups - 1);
  T *Ps = (T *)smraw;
  T *Wt = Ps + SM::kPanel;
  T *Gt = Wt + SM::kW;              // G and tau of the panel in T (phase B)
  T *taut = Gt + SM::kG;
  double *Gs = (double *)(smraw + align_up_c(SM::kBytesT, 16));
  double *dots = Gs + SM::kG;
  double *sig = dots + kBNB;
  double *tau = sig + kBNB;
  double *ups = tau + kBNB;
  double *scl = ups + kBNB;         // per-column scale 2^-E of the panel
  double *sinv = scl + kBNB;        // and its inverse 2^E
  double *fst = sinv + kBNB;        // 1: FP32 pivot for this column (T == float, |E| <= 60)
  double *misc = fst + kBNB;        // [0] = norm
  // An FP32 factorization (T == float) forms the norm, the pivot and the
  // multipliers in FP32 (its per-column chain then stays off the FP64 pipe);
  // a column whose power-of-two scale is extreme for FP32 forms its pivot in
  // FP64.  T == double: everything FP64.
  constexpr bool kF32 = std::is_same<T, float>::value;
  const int K = num_reflectors(m, n);
  for (int k = K + tid; k < n; k += kThreads) up_out[k] = 0.0;

  for (int k0 = 0; k0 < K; k0 += kBNB) {
    const int nbw = min(kBNB, K - k0);
    const int skip = ntop > 0 ? ntop - k0 - nbw : 0;
    const int M = m - k0 - skip;
    // matrix row (relative to k0) of panel row r
    auto prow = [&](int r) { return r + (r >= nbw ? skip : 0); };
    // (stacked: the strictly lower part of the diagonal block is zero, not read)
    for (int idx = tid; idx < kBNB * M; idx += kThreads) {
      int c = idx / M, r = idx - c * M;
      const bool zero = c >= nbw || (ntop > 0 && r < nbw && r > c);
      Ps[c * kBMaxRows + r] = zero ? T(0) : A[SLQR_IDX(k0 + prow(r), k0 + c, lda)];
    }
    __syncthreads();
    // Per-column scale of the panel for the overflow-safe norm: 2^-E with E the
    // exponent of the column's largest |entry| from its diagonal down (an exact
    // power of two; entries that earlier reflectors of the panel add stay
    // within a factor sqrt(M) of it).
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int c = warp + kBWarps * t;
      if (c < nbw) {
        unsigned mx = 0;
        for (int r = c + lane; r < M; r += 32) mx = max(mx, b_abs_hi(Ps[c * kBMaxRows + r]));
        mx = __reduce_max_sync(0xffffffffu, mx);
        if (lane == 0) {
          int E = (int)((mx >> 20) & 0x7ff) - 1023;
          // (FP32: 2^-E and 2^E both normal floats)
          E = kF32 ? min(max(E, -126), 126) : min(max(E, -1000), 1022);
          scl[c] = b_pow2(-E);
          sinv[c] = b_pow2(E);
          fst[c] = (kF32 && E >= -60 && E <= 60) ? 1.0 : 0.0;
        }
      }
    }
    __syncthreads();
    for (int j = 0; j < nbw; ++j) {
      const T *x = Ps + j * kBMaxRows;
      // phase 1: warp w takes panel columns w and w + 8
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int c = warp + kBWarps * t;
        if (c >= nbw) continue;
        if (c == j) {
          const T sc = (T)scl[j];
          T S = T(0), S1 = T(0);                       // two chains
          int r = j + lane;
          for (; r + 32 < M; r += 64) {
            const T xs = x[r] * sc, xs1 = x[r + 32] * sc;
            S = fma(xs, xs, S);
            S1 = fma(xs1, xs1, S1);
          }
          if (r < M) {
            const T xs = x[r] * sc;
            S = fma(xs, xs, S);
          }
          S = b_warp_sum(S + S1);
          if (lane == 0) {                             // exact rescale by 2^E
            if (S == T(0)) misc[0] = 0.0;
            else if (kF32 && fst[j] != 0.0) misc[0] = (double)(sqrt(S) * (T)sinv[j]);
            else misc[0] = sqrt((double)S) * sinv[j];
          }
        } else {
          const T *col = Ps + c * kBMaxRows;
          T acc = T(0), acc1 = T(0);                   // two chains
          int r = j + 1 + lane;
          for (; r + 32 < M; r += 64) {
            acc = fma(x[r], col[r], acc);
            acc1 = fma(x[r + 32], col[r + 32], acc1);
          }
          if (r < M) acc = fma(x[r], col[r], acc);
          acc += acc1;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
          if (lane == 0) dots[c] = (double)acc;
        }
      }
      __syncthreads();
      const double s = misc[0];
      const bool defined = (s != 0.0);
      double cl = 0.0, upk = 0.0, tk = 0.0;
      if (kF32 && fst[j] != 0.0) {                     // FP32 pivot and multipliers
        const T sT = (T)s, x0 = x[j];
        T clT = T(0), upT = T(0), tkT = T(0);
        if (defined) {
          clT = (x0 > T(0)) ? -sT : sT;
          upT = x0 - clT;
          if (warp == 0) tkT = T(-1) / (upT * clT);    // tau = -1/b (warp 0 uses it)
        }
        if (tid < nbw) {
          const int c = tid;
          const T pr_c = Ps[c * kBMaxRows + j];
          if (c > j) sig[c] = defined ? (double)(-(upT * pr_c + (T)dots[c]) * tkT) : 0.0;
          else if (c < j) Gs[c + j * kBNB] = (double)(pr_c * upT + (T)dots[c]);
        }
        cl = clT;
        upk = upT;
        tk = tkT;
      } else {
        const double x0 = (double)x[j];
        if (defined) {
          cl = (x0 > 0.0) ? -s : s;
          upk = x0 - cl;
          if (warp == 0) tk = -1.0 / (upk * cl);      // tau = -1/b (warp 0 uses it)
        }
        if (tid < nbw) {
          const int c = tid;
          const double pr_c = (double)Ps[c * kBMaxRows + j];
          // sigma_c = (up p_c + D_c) / b = -(up p_c + D_c) tau
          if (c > j) sig[c] = defined ? -(upk * pr_c + dots[c]) * tk : 0.0;
          else if (c < j) Gs[c + j * kBNB] = pr_c * upk + dots[c];
        }
      }
      __syncthreads();
      if (defined) {
        const T upT = (T)upk;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const int c = warp + kBWarps * t;
          if (c > j && c < nbw) {
            T *col = Ps + c * kBMaxRows;
            const T sg = (T)sig[c];
            for (int r = j + 1 + lane; r < M; r += 32) col[r] = fma(sg, x[r], col[r]);
            if (lane == 0) col[j] = fma(sg, upT, col[j]);
          }
        }
      }
      __syncthreads();
      if (tid == 0) {
        if (defined) Ps[j * kBMaxRows + j] = (T)cl;
        tau[j] = tk;
        ups[j] = upk;
      }
      __syncthreads();
    }
    // write the panel back; keep G and tau if asked; then turn the slice into
    // V (zero above the diagonal, up on it) for the trailing update
    for (int idx = tid; idx < nbw * M; idx += kThreads) {
      int c = idx / M, r = idx - c * M;
      if (!(ntop > 0 && r < nbw && r > c)) A[SLQR_IDX(k0 + prow(r), k0 + c, lda)] = Ps[c * kBMaxRows + r];
    }
    if (tid < nbw) up_out[k0 + tid] = ups[tid];
    if (G_out) {
      double *Gp = G_out + (size_t)(k0 / kBNB) * kBNB * kBNB;
      for (int idx = tid; idx < kBNB * kBNB; idx += kThreads) {
        int jj = idx / kBNB, q = idx - jj * kBNB;
        Gp[idx] = (q < jj && jj < nbw) ? Gs[idx] : 0.0;
      }
      if (tid < kBNB) tau_out[k0 + tid] = (tid < nbw) ? tau[tid] : 0.0;
    }
    __syncthreads();
    for (int idx = tid; idx < kBNB * kBNB; idx += kThreads) {
      int c = idx / kBNB, r = idx - c * kBNB;
      if (r <= c && r < M) Ps[c * kBMaxRows + r] = (r == c && c < nbw) ? (T)ups[c] : T(0);
      Gt[idx] = (T)Gs[idx];
    }
    if (tid < kBNB) taut[tid] = (T)tau[tid];
    __syncthreads();

    // trailing columns [k0 + nbw, n), plus Bcol as one more column
    const int NT = n - (k0 + nbw);
    const int NC = NT + (Bcol ? 1 : 0);
    for (int t0 = 0; t0 < NC; t0 += kBCols) {
      // phase A: W[a][col] = sum_r V[a][r] C[r][col].  Warp w takes the four
      // columns 4w .. 4w+3 of the tile; lane = 8 * (column - 4w) + g walks
      // the rows r = g (mod 8), so a column's 16 partial sums are combined
      // over 8 lanes only (14 adds per lane) and a ragged M leaves at most
      // 7 lanes of a column idle on its last row step.
      if (t0 + kBGroupCols * warp < NC) {
        const int cc = kBGroupCols * warp + (lane >> 3);
        const int col = t0 + cc;
        T acc[kBNB];
#pragma unroll
        for (int a = 0; a < kBNB; ++a) acc[a] = T(0);
        if (col < NC) {
          const T *C = (col < NT) ? A + SLQR_IDX(k0, k0 + nbw + col, lda) : (const T *)(Bcol + k0);
#pragma unroll 4
          for (int r = g8; r < M; r += kBRowGroups) {
            const T cv = C[prow(r)];
#pragma unroll
            for (int a = 0; a < kBNB; ++a)
              if (a < nbw) acc[a] = fma(Ps[a * kBMaxRows + r], cv, acc[a]);
          }
        }
        b_group8_sum16(acc, g8);                // lane g holds W[2g], W[2g + 1]
        if (col < NC) {
          Wt[(2 * g8) * (kBCols + 1) + cc] = acc[0];
          Wt[(2 * g8 + 1) * (kBCols + 1) + cc] = acc[1];
        }
      }
      __syncthreads();
      // phase B: W' = T^T W, one lane per column, in T (an FP32
      // factorization keeps this chain off the slow FP64 pipe)
      if (warp == 0 && t0 + lane < NC) {
        T w[kBNB];
#pragma unroll
        for (int jj = 0; jj < kBNB; ++jj) {
          if (jj < nbw) {
            T t = Wt[jj * (kBCols + 1) + lane];
#pragma unroll
            for (int q = 0; q < jj; ++q) t = fma(-Gt[q + jj * kBNB], w[q], t);
            w[jj] = taut[jj] * t;
            Wt[jj * (kBCols + 1) + lane] = w[jj];
          }
        }
      }
      __syncthreads();
      // phase C: C -= V W', the same lane layout as phase A
      {
        const int cc = kBGroupCols * warp + (lane >> 3);
        const int col = t0 + cc;
        if (col < NC) {
          T *C = (col < NT) ? A + SLQR_IDX(k0, k0 + nbw + col, lda) : (T *)(Bcol + k0);
          T w[kBNB];
#pragma unroll
          for (int a = 0; a < kBNB; ++a) w[a] = (a < nbw) ? Wt[a * (kBCols + 1) + cc] : T(0);
#pragma unroll 4
          for (int r = g8; r < M; r += kBRowGroups) {
            const int pr = prow(r);
            T cv = C[pr];
#pragma unroll
            for (int a = 0; a < kBNB; ++a)
              if (a < nbw) cv = fma(-Ps[a * kBMaxRows + r], w[a], cv);
            C[pr] = cv;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Back-substitution R x = (Q^T b)[0:n] of the FP64 path, column-oriented.
__device__ void batch_solve_fp64(const double *A, int lda, int n, double *b, double *xs,
                                 int *status_out) {
  const int tid = threadIdx.x;
  for (int i = tid; i < n; i += kThreads) xs[i] = b[i];
  __syncthreads();
  bool rank_def = false;
  for (int i = n - 1; i >= 0; --i) {
    const double d = A[SLQR_IDX(i, i, lda)];
    if (tid == 0) xs[i] = (d != 0.0) ? xs[i] / d : 0.0;
    if (d == 0.0) rank_def = true;
    __syncthreads();
    const double xi = xs[i];
    for (int l = tid; l < i; l += kThreads) xs[l] = fma(-A[SLQR_IDX(l, i, lda)], xi, xs[l]);
    __syncthreads();
  }
  for (int i = tid; i < n; i += kThreads) b[i] = xs[i];
  if (tid == 0) *status_out = rank_def ? SLQR_ERANK : SLQR_OK;
  __syncthreads();
}

constexpr size_t kBSmemBytes = BatchSmem<double>::kBytes;

__global__ void __launch_bounds__(kThreads, 2)   // two CTAs per SM
batch_factor_fp64_kernel(BatchParams bp) {
  extern __shared__ __align__(16) char smraw[];
  __shared__ int s_item;
  __shared__ int s_status;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(bp.counter, 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= bp.count) break;
    const int p = bp.order[item];
    const BatchProblem pr = bp.probs[p];
    if (pr.n > 0) {
      batch_factor_core<double>(pr.A, pr.lda, pr.m, pr.n, pr.up, pr.b, nullptr, nullptr, smraw,
                                pr.ntop);
      if (pr.b) {
        batch_solve_fp64(pr.A, pr.lda, pr.n, pr.b, (double *)smraw, &s_status);
      } else if (threadIdx.x == 0) {
        s_status = SLQR_OK;
      }
      __syncthreads();
      if (threadIdx.x == 0 && bp.status) bp.status[p] = s_status;
    } else if (threadIdx.x == 0 && bp.status) {
      bp.status[p] = SLQR_OK;
    }
  }
}

// --------------------------------------------------------------------------
// Mixed precision (SLQR_FP32): the factorization runs in FP32 on a scratch
// copy of A (up, tau and G stored in FP64), and the LS solution is recovered by
// iterative refinement of the augmented system [I A; A^T 0][r; x] = [b; 0]
// (Bjorck): residuals f = b - r - A x and g = -A^T r in FP64 from the
// original A, the correction through the FP32 QR:
//   h = R^-T g,  d = Q^T f,  dx = R^-1 (d[0:n] - h),  dr = Q [h; d[n:m]].
// This converges to the FP64 LS solution when kappa times the backward error
// of the FP32 factorization (a modest multiple of u_fp32) is below 1, for
// consistent and inconsistent right-hand sides alike.
// --------------------------------------------------------------------------
struct BatchMixedParams {
  const BatchProblem *probs;
  const int *order;
  int count;
  unsigned *counter;
  int *status;
  double *err;
  float *af;            // per CTA: kBMaxRows * kBMaxRows floats
  double *gt;           // per CTA: G (kMaxPanels * kBNB^2) + tau (kBMaxRows) + up (kBMaxRows)
  int max_it;
  double tol;
};

constexpr int kBMaxPanels = kBMaxRows / kBNB;
// per-CTA global scratch of the mixed kernel: G of every panel, tau, up and
// the column scales d_j of the equilibration
constexpr size_t kBGtDoubles = (size_t)kBMaxPanels * kBNB * kBNB + 3 * kBMaxRows;

// V(i, a) of panel p from the FP32 factorization (rows relative to k0 = p*kBNB)
__device__ __forceinline__ float mixed_v(const float *Af, int m, const double *up, int k0,
                                         int nbw, int i, int a) {
  if (a >= nbw || i < a) return 0.f;
  if (i == a) return (float)up[k0 + a];
  return Af[SLQR_IDX(k0 + i, k0 + a, m)];
}

// y <- Q^T y (forward = true) or y <- Q y, panel by panel, FP32 arithmetic.
// Per panel each thread loads the V entries of its rows (at most two: m <=
// 512) once, all in flight, and keeps them in registers for both products:
// w = V^T y (per-thread partials, a halving exchange over the warp, then the
// 8 warp totals), w' = T^T w or T w on warp 0, then y -= V w'.  red holds
// kBWarps * kBNB floats.
constexpr int kBRowsPerThread = kBMaxRows / kThreads;
static_assert(kBRowsPerThread * kThreads == kBMaxRows, "rows per thread");

__device__ void mixed_apply_q(const float *Af, int m, int n, const double *G, const double *tau,
                              const double *up, float *y, float *red, bool forward) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = num_reflectors(m, n);
  const int np = num_panels(K, kBNB);
  for (int s = 0; s < np; ++s) {
    const int pnl = forward ? s : np - 1 - s;
    const int k0 = pnl * kBNB;
    const int nbw = min(kBNB, K - k0);
    const int M = m - k0;
    float vr[kBRowsPerThread][kBNB];
    float yv[kBRowsPerThread];
    float acc[kBNB];
#pragma unroll
    for (int a = 0; a < kBNB; ++a) acc[a] = 0.f;
#pragma unroll
    for (int t = 0; t < kBRowsPerThread; ++t) {
      const int i = tid + t * kThreads;
      const bool in = i < M;
#pragma unroll
      for (int a = 0; a < kBNB; ++a) {
        float v = 0.f;
        if (in && a < nbw && i >= a)
          v = (i == a) ? (float)up[k0 + a] : Af[SLQR_IDX(k0 + i, k0 + a, m)];
        vr[t][a] = v;
      }
      yv[t] = in ? y[k0 + i] : 0.f;
#pragma unroll
      for (int a = 0; a < kBNB; ++a) acc[a] = fmaf(vr[t][a], yv[t], acc[a]);
    }
    // halving exchange: lanes 2a, 2a + 1 end with the warp's total of acc[a]
#pragma unroll
    for (int h = 8, mask = 16; h >= 1; h >>= 1, mask >>= 1) {
      const bool hi = (lane & mask) != 0;
#pragma unroll
      for (int i = 0; i < h; ++i) {
        const float send = hi ? acc[i] : acc[i + h];
        const float keep = hi ? acc[i + h] : acc[i];
        acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
      }
    }
    acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
    if ((lane & 1) == 0) red[warp * kBNB + (lane >> 1)] = acc[0];
    __syncthreads();
    // T^T w (forward) or T w, right-looking in FP32 on warp 0: lane j holds
    // w_j and its column (forward) or row of G; at step q lane q's value is
    // final and the lanes still open subtract its contribution
    if (warp == 0) {
      const double *Gp = G + (size_t)pnl * kBNB * kBNB;
      const int j = lane;
      const bool act = j < nbw;
      float t = 0.f;
      if (act) {
#pragma unroll
        for (int w8 = 0; w8 < kBWarps; ++w8) t += red[w8 * kBNB + j];
      }
      const float tj = act ? (float)tau[k0 + j] : 0.f;
      float gl[kBNB];
#pragma unroll
      for (int q = 0; q < kBNB; ++q)
        gl[q] = (act && q < nbw) ? (float)(forward ? Gp[q + j * kBNB] : Gp[j + q * kBNB]) : 0.f;
      float wf = 0.f;
#pragma unroll
      for (int s2 = 0; s2 < kBNB; ++s2) {
        const int q = forward ? s2 : kBNB - 1 - s2;
        if (q < nbw) {                                 // uniform over the warp
          const float fin = __shfl_sync(0xffffffffu, t * tj, q);
          if (forward ? (j > q) : (j < q)) t = fmaf(-gl[q], fin, t);
          if (j == q) wf = fin;
        }
      }
      __syncwarp();
      if (act) red[j] = wf;                           // (every lane has read red)
    }
    __syncthreads();
    float wv[kBNB];
#pragma unroll
    for (int a = 0; a < kBNB; ++a) wv[a] = (a < nbw) ? red[a] : 0.f;
#pragma unroll
    for (int t = 0; t < kBRowsPerThread; ++t) {
      const int i = tid + t * kThreads;
      if (i < M) {
        float v = yv[t];
#pragma unroll
        for (int a = 0; a < kBNB; ++a) v = fmaf(-vr[t][a], wv[a], v);
        y[k0 + i] = v;
      }
    }
    __syncthreads();
  }
}

// Triangular solves with R = triu(Af[0:n, 0:n]) in FP32, in blocks of 32
// rows.  upper == true: R x = y (back); false: R^T x = y (forward).  y is
// replaced; a zero diagonal gives x_i = 0 and returns true.  Per block, warp
// 0 solves the 32 x 32 diagonal block with the block's entries of R in
// registers (lane l = row; at each step one lane's x is final and is
// broadcast), then every thread updates the rows not yet solved.
__device__ bool mixed_trsv(const float *Af, int m, int n, float *y, bool upper) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  bool zero = false;
  const int nblk = (n + 31) / 32;
  for (int bi = 0; bi < nblk; ++bi) {
    const int i0 = upper ? max(0, n - 32 * (bi + 1)) : 32 * bi;
    const int nb = upper ? (n - 32 * bi) - i0 : min(32, n - i0);
    if (warp == 0) {
      const int i = i0 + lane;
      const bool act = lane < nb;
      float rv[32];
#pragma unroll
      for (int s = 0; s < 32; ++s) {
        // upper: R[i, i0+s] for s > lane; lower: R^T[i, i0+s] = R[i0+s, i] for s < lane
        const bool need = act && s < nb && (upper ? s > lane : s < lane);
        rv[s] = need ? (upper ? Af[SLQR_IDX(i, i0 + s, m)] : Af[SLQR_IDX(i0 + s, i, m)]) : 0.f;
      }
      const float d = act ? Af[SLQR_IDX(i, i, m)] : 1.f;
      float yl = act ? y[i] : 0.f;
      if (__any_sync(0xffffffffu, act && d == 0.f)) zero = true;
      float xl = 0.f;
#pragma unroll
      for (int s2 = 0; s2 < 32; ++s2) {
        const int s = upper ? 31 - s2 : s2;
        if (s < nb) {                                  // uniform over the warp
          const float xs = __shfl_sync(0xffffffffu, (d != 0.f) ? yl / d : 0.f, s);
          if (lane == s) xl = xs;
          if (upper ? lane < s : lane > s) yl = fmaf(-rv[s], xs, yl);
        }
      }
      if (act) y[i] = xl;
    }
    __syncthreads();
    // rows not yet solved: upper -> [0, i0), lower -> [i0 + nb, n)
    const int r0 = upper ? 0 : i0 + nb, r1 = upper ? i0 : n;
    for (int l = r0 + tid; l < r1; l += kThreads) {
      float v = y[l];
#pragma unroll 8
      for (int s = 0; s < nb; ++s)
        v = fmaf(-(upper ? Af[SLQR_IDX(l, i0 + s, m)] : Af[SLQR_IDX(i0 + s, l, m)]), y[i0 + s], v);
      y[l] = v;
    }
    __syncthreads();
  }
  return __syncthreads_or(zero);
}

__device__ double block_max_abs(double v, double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = fabs(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = 0.0;
  for (int w = 0; w < kBWarps; ++w) r = fmax(r, red[w]);
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kThreads, 2)   // two CTAs per SM
batch_factor_mixed_kernel(BatchMixedParams bp) {
  extern __shared__ __align__(16) char smraw[];
  __shared__ int s_item;
  __shared__ double red[kBWarps];
  float *Af = bp.af + (size_t)blockIdx.x * kBMaxRows * kBMaxRows;
  double *G = bp.gt + (size_t)blockIdx.x * kBGtDoubles;
  double *tau = G + (size_t)kBMaxPanels * kBNB * kBNB;
  double *up = tau + kBMaxRows;
  double *dcol = up + kBMaxRows;       // d_j = 2^-e_j: the FP32 copy is of A D
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (;;) {
    if (tid == 0) s_item = (int)atomicAdd(bp.counter, 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= bp.count) break;
    const int p = bp.order[item];
    const BatchProblem pr = bp.probs[p];
    const int m = pr.m, n = pr.n;
    if (n == 0) {
      if (tid == 0) {
        if (bp.status) bp.status[p] = SLQR_OK;
        if (bp.err) bp.err[p] = 0.0;
      }
      continue;
    }
    // column equilibration by exact powers of two (the largest entry of each
    // column of A D in [1/2, 1): no FP32 overflow or underflow of products for
    // any column scale), the FP32 working copy of A D (ld = m), then its FP32
    // factorization; the refinement solves for y with x = D y
    for (int j = warp; j < n; j += kBWarps) {
      double mx = 0.0;
      for (int i = lane; i < m; i += 32) mx = fmax(mx, fabs(pr.A[SLQR_IDX(i, j, pr.lda)]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) {
        int ex = 0;
        if (mx > 0.0 && isfinite(mx)) {
          frexp(mx, &ex);
          ex = max(-1000, min(1000, ex));
        }
        dcol[j] = ldexp(1.0, -ex);
      }
    }
    __syncthreads();
    for (int idx = tid; idx < m * n; idx += kThreads) {
      int c = idx / m, r = idx - c * m;
      Af[idx] = (float)(pr.A[SLQR_IDX(r, c, pr.lda)] * dcol[c]);
    }
    __syncthreads();
    batch_factor_core<float>(Af, m, m, n, up, nullptr, G, tau, smraw, pr.ntop);
    __syncthreads();
    // refinement vectors in shared memory (the panel area is free now)
    double *x = (double *)smraw;          // n
    double *r = x + kBMaxRows;            // m
    double *dx = r + kBMaxRows;           // n (FP64 copy of the correction)
    float *f = (float *)(dx + kBMaxRows); // m   f, then d = Q^T f, then dr
    float *g = f + kBMaxRows;             // n   g, then h
    float *e = g + kBMaxRows;             // m
    float *w = e + kBMaxRows;             // kBWarps * kBNB (apply_q reductions)
    // r = 0, x = 0: the first sweep is the plain QR solve (see mixed.cu)
    for (int i = tid; i < m; i += kThreads) r[i] = 0.0;
    for (int i = tid; i < n; i += kThreads) x[i] = 0.0;
    __syncthreads();
    int status = SLQR_ENOCONV;
    double err = 1.0, prev = 1e300;
    for (int it = 0; it < bp.max_it; ++it) {
      // f = b - r - A x (FP64), one thread per row
      // (four partial sums: the dependent FP64 chain is a quarter as long)
      for (int i = tid; i < m; i += kThreads) {
        double a0 = pr.b[i] - r[i], a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int j = 0;
        for (; j + 3 < n; j += 4) {
          a0 = fma(-pr.A[SLQR_IDX(i, j, pr.lda)], x[j], a0);
          a1 = fma(-pr.A[SLQR_IDX(i, j + 1, pr.lda)], x[j + 1], a1);
          a2 = fma(-pr.A[SLQR_IDX(i, j + 2, pr.lda)], x[j + 2], a2);
          a3 = fma(-pr.A[SLQR_IDX(i, j + 3, pr.lda)], x[j + 3], a3);
        }
        for (; j < n; ++j) a0 = fma(-pr.A[SLQR_IDX(i, j, pr.lda)], x[j], a0);
        f[i] = (float)((a0 + a1) + (a2 + a3));
      }
      // g = -D A^T r (FP64), one warp per column
      for (int j = warp; j < n; j += kBWarps) {
        double acc = 0.0;
        for (int i = lane; i < m; i += 32) acc = fma(pr.A[SLQR_IDX(i, j, pr.lda)], r[i], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) g[j] = (float)(-acc * dcol[j]);
      }
      __syncthreads();
      bool zero = mixed_trsv(Af, m, n, g, false);            // h = R^-T g (in g)
      mixed_apply_q(Af, m, n, G, tau, up, f, w, true);        // d = Q^T f (in f)
      for (int i = tid; i < m; i += kThreads) e[i] = (i < n) ? f[i] - g[i] : f[i];
      __syncthreads();
      zero |= mixed_trsv(Af, m, n, e, true);                 // dx = R^-1 (d1 - h) (in e[0:n])
      for (int i = tid; i < n; i += kThreads) dx[i] = (double)e[i] * dcol[i];
      for (int i = tid; i < m; i += kThreads) f[i] = (i < n) ? g[i] : f[i];   // [h; d2]
      __syncthreads();
      mixed_apply_q(Af, m, n, G, tau, up, f, w, false);       // dr = Q [h; d2] (in f)
      double dmax = 0.0, xmax = 0.0;
      for (int i = tid; i < n; i += kThreads) {
        x[i] += dx[i];
        // a non-finite entry (an FP32 overflow) counts as +inf: never "converged"
        dmax = fmax(dmax, isfinite(dx[i]) ? fabs(dx[i]) : CUDART_INF);
        xmax = fmax(xmax, isfinite(x[i]) ? fabs(x[i]) : CUDART_INF);
      }
      for (int i = tid; i < m; i += kThreads) r[i] += (double)f[i];
      dmax = block_max_abs(dmax, red);
      xmax = block_max_abs(xmax, red);
      // an exact zero on the diagonal of R is a rank statement whatever the
      // step looks like, so it is reported before the non-finite guard
      if (zero) {
        status = SLQR_ERANK;
        err = (isfinite(dmax) && isfinite(xmax) && xmax > 0.0) ? dmax / xmax : CUDART_INF;
        break;
      }
      if (!isfinite(dmax) || !isfinite(xmax)) {
        status = SLQR_ENOCONV;
        err = CUDART_INF;
        break;
      }
      err = (xmax > 0.0) ? dmax / xmax : 0.0;
      if (err <= bp.tol) { status = SLQR_OK; break; }
      if (it >= 2 && err > 0.5 * prev) {        // no longer contracting: FP64 noise level
        status = (err <= kBStallOk) ? SLQR_OK : SLQR_ENOCONV;
        break;
      }
      prev = err;
    }
    for (int i = tid; i < n; i += kThreads) pr.b[i] = x[i];
    if (tid == 0) {
      if (bp.status) bp.status[p] = status;
      if (bp.err) bp.err[p] = err;
    }
    __syncthreads();
  }
}

constexpr size_t kBMixedSmemBytes = BatchSmem<float>::kBytes > 6 * kBMaxRows * sizeof(double)
                                        ? BatchSmem<float>::kBytes
                                        : 6 * kBMaxRows * sizeof(double);

slqr_status init_batch_attrs(slqr_ctx *ctx) {
  cudaError_t e = cudaFuncSetAttribute(batch_factor_fp64_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kBSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_factor_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kBMixedSmemBytes);
  if (e != cudaSuccess)
    return fail(ctx, SLQR_ECUDA, "cudaFuncSetAttribute(batch): %s", cudaGetErrorString(e));
  return SLQR_OK;
}

}  // namespace slqr

using namespace slqr;

extern "C" int slqr_batch_max_rows(void) { return kBMaxRows; }

namespace slqr {

// The launch behind slqr_batch_factor and slqr_batch_factor_stacked (ntop:
// NULL, or per problem the rows of its upper-triangular top block, 0 for a
// dense problem).  The context mutex is held by the caller.
// A batch as the kernels see it: the problem table (in the order given), the
// longest-first order, the grid and the algorithmic flops.
struct BatchSetup {
  std::vector<BatchProblem> probs;
  std::vector<int> order;
  bool mixed = false;
  int grid = 0;
  double flops = 0.0;
  size_t table_bytes = 0, head = 0, af_bytes = 0, gt_bytes = 0;   // device layout
};

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
  bs.order.resize(count);
  std::iota(bs.order.begin(), bs.order.end(), 0);
  std::stable_sort(bs.order.begin(), bs.order.end(),
                   [&](int a, int c) { return cost[a] > cost[c]; });
  bs.flops = 0.0;
  for (int i = 0; i < count; ++i) bs.flops += cost[i];
  bs.mixed = (prec == SLQR_FP32);
  int per_sm = 0;
  cudaError_t e;
  if (bs.mixed)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_factor_mixed_kernel, kThreads,
                                                      kBMixedSmemBytes);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_factor_fp64_kernel, kThreads,
                                                      kBSmemBytes);
  if (e != cudaSuccess || per_sm < 1)
    return fail(ctx, SLQR_ECUDA, "batch occupancy: %s", cudaGetErrorString(e));
  bs.grid = std::min(count, per_sm * ctx->num_sms);
  // device layout: [counter 256 B][problem table][order][per-CTA scratch (mixed)]
  bs.table_bytes = align_up(sizeof(BatchProblem) * count, 256);
  bs.head = align_up(256 + bs.table_bytes + sizeof(int) * count, 256);
  bs.af_bytes = bs.mixed ? (size_t)bs.grid * kBMaxRows * kBMaxRows * sizeof(float) : 0;
  bs.gt_bytes = bs.mixed ? (size_t)bs.grid * kBGtDoubles * sizeof(double) : 0;
  return SLQR_OK;
}

// The kernel launch of a batch whose table and order are already at `base`.
static void batch_kernel_launch(const BatchSetup &bs, char *base, int count, int *status,
                                double *err, cudaStream_t s) {
  unsigned *counter = (unsigned *)base;
  BatchProblem *d_probs = (BatchProblem *)(base + 256);
  int *d_order = (int *)(base + 256 + bs.table_bytes);
  if (!bs.mixed) {
    BatchParams bp{d_probs, d_order, count, counter, status};
    batch_factor_fp64_kernel<<<bs.grid, kThreads, kBSmemBytes, s>>>(bp);
  } else {
    BatchMixedParams mp{d_probs, d_order, count, counter, status, err,
                        (float *)(base + bs.head), (double *)(base + bs.head + bs.af_bytes),
                        kBMaxRefine, kBRefineTol};
    batch_factor_mixed_kernel<<<bs.grid, kThreads, kBMixedSmemBytes, s>>>(mp);
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
  batch_kernel_launch(bs, base, count, status, err, s);
  prof_end(ctx, s, slot, kBatch, bs.flops);
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
    batch_kernel_launch(plan->bs, plan->dev, count, status, err, cs);
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
