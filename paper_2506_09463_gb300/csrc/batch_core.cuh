// batch_core.cuh -- device code of the batched H12 least squares
// (slqr_batch_factor): many independent problems in one persistent launch.
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
// Inside a CTA a problem is factored in panels of NB reflectors (NB = 8, 16
// or 32, a setting of the batch autotuner; 16 by default):
//  * the panel (rows k0..m-1, NB columns) sits in shared memory; each column
//    is one block-level reduction (scaled norm, dots of the column tail with
//    the other panel columns, which also give striu(V^T V)), then the update
//    of the later panel columns;
//  * the trailing columns (and b, as one more column) are updated in tiles of
//    TC columns (16, 32 or 64; 32 by default): W = V^T C (256 / TC lanes per
//    column, each over every (256 / TC)-th row), then W' = T^T W by forward
//    substitution (one thread per column), then C -= V W' (the same lanes as
//    W).
// The FP64 kernel does all arithmetic in FP64 (DFMA).
#pragma once
#include "slqr_internal.cuh"

#include <math_constants.h>

#include <type_traits>

namespace slqr {

constexpr int kBMaxRows = 512;    // rows of a batched problem (panel slice in smem)
constexpr int kBWarps = kThreads / 32;
constexpr int kBNBMax = 32;       // widest panel of the batched kernels
// Settings of the batched kernels (the batch autotuner's search space): NB
// reflectors per panel (8, 16, 32) and TC trailing columns per tile (16, 32,
// 64).  In the tile phases every warp takes CPW = TC / 8 columns and RG =
// 256 / TC lanes work on one column (each over every RG-th row); the NB
// partial sums of a column are then combined over those RG lanes by a halving
// exchange, which leaves NB / RG sums per lane (so NB >= RG).
constexpr int kBNBDefault = 16, kBTCDefault = 32;
template <int NB, int TC>
struct BTile {
  static constexpr int RG = kThreads / TC;    // lanes of one column
  static constexpr int CPW = 32 / RG;         // columns of one warp
  static constexpr int VPL = NB / RG;         // W entries a lane holds after the exchange
  static constexpr int NBW8 = (NB + kBWarps - 1) / kBWarps;   // panel columns per warp
  static_assert(NB == 8 || NB == 16 || NB == 32, "panel width 8, 16 or 32");
  static_assert(TC == 16 || TC == 32 || TC == 64, "tile of 16, 32 or 64 columns");
  static_assert(NB % RG == 0, "at least one W entry per lane after the exchange");
};
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

// Sum of NB per-lane values acc[0..NB-1] over the RG lanes g = lane % RG of
// one column group by a halving exchange: at each of log2(RG) levels a lane
// keeps half of its values and adds the other half received from its partner
// (for NB = 16 over 8 lanes: 14 shuffles and adds per lane instead of 48 for 16
// separate butterflies).  Afterwards lane g holds the totals of values
// (NB/RG) g + i in acc[i], i < NB/RG.
template <typename T, int NB, int RG>
__device__ __forceinline__ void b_group_sum(T (&acc)[NB], int g) {
#pragma unroll
  for (int mask = RG / 2, half = NB / 2; mask >= 1; mask >>= 1, half >>= 1) {
    const bool hi = (g & mask) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const T send = hi ? acc[i] : acc[i + half];
      const T keep = hi ? acc[i + half] : acc[i];
      acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
    }
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

// PR: rows the panel slice holds (kBMaxRows, or the row bound of the
// shared-memory-resident kernels)
template <typename T, int NB, int TC, int PR = kBMaxRows>
struct BatchSmem {
  static constexpr int kPanel = NB * PR;                // Ps[c][r]
  static constexpr int kW = NB * (TC + 1);              // Wt[a][col]
  static constexpr int kG = NB * NB;                    // G[q][j] (ld NB)
  // T copies of the panel's G and tau for W' = T^T W (phase B)
  static constexpr size_t kBytesT = (size_t)(kPanel + kW + kG + NB) * sizeof(T);
  static constexpr int kMisc = 7 * NB + 8;    // dots, sigma, tau, up, scale, 1/scale, fast, norm
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
//
// A and Bcol may point to global or to shared memory (the resident kernels
// factor a shared-memory copy of the problem); PR is the panel's row capacity.
template <typename T, int NB, int TC, int PR = kBMaxRows>
__device__ void batch_factor_core(T *A, int lda, int m, int n, double *up_out, double *Bcol,
                                  double *G_out, double *tau_out, char *smraw, int ntop) {
  using SM = BatchSmem<T, NB, TC, PR>;
  using TL = BTile<NB, TC>;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g8 = lane & (TL::RG - 1);          // this lane's row group in the tile phases
  T *Ps = (T *)smraw;
  T *Wt = Ps + SM::kPanel;
  T *Gt = Wt + SM::kW;              // G and tau of the panel in T (phase B)
  T *taut = Gt + SM::kG;
  double *Gs = (double *)(smraw + align_up_c(SM::kBytesT, 16));
  double *dots = Gs + SM::kG;
  double *sig = dots + NB;
  double *tau = sig + NB;
  double *ups = tau + NB;
  double *scl = ups + NB;           // per-column scale 2^-E of the panel
  double *sinv = scl + NB;          // and its inverse 2^E
  double *fst = sinv + NB;          // 1: FP32 pivot for this column (T == float, |E| <= 60)
  double *misc = fst + NB;          // [0] = norm
  // An FP32 factorization (T == float) forms the norm, the pivot and the
  // multipliers in FP32 (its per-column chain then stays off the FP64 pipe);
  // a column whose power-of-two scale is extreme for FP32 forms its pivot in
  // FP64.  T == double: everything FP64.
  constexpr bool kF32 = std::is_same<T, float>::value;
  const int K = num_reflectors(m, n);
  for (int k = K + tid; k < n; k += kThreads) up_out[k] = 0.0;

  for (int k0 = 0; k0 < K; k0 += NB) {
    const int nbw = min(NB, K - k0);
    const int skip = ntop > 0 ? ntop - k0 - nbw : 0;
    const int M = m - k0 - skip;
    // matrix row (relative to k0) of panel row r
    auto prow = [&](int r) { return r + (r >= nbw ? skip : 0); };
    // (stacked: the strictly lower part of the diagonal block is zero, not read)
    for (int idx = tid; idx < NB * M; idx += kThreads) {
      int c = idx / M, r = idx - c * M;
      const bool zero = c >= nbw || (ntop > 0 && r < nbw && r > c);
      Ps[c * PR + r] = zero ? T(0) : A[SLQR_IDX(k0 + prow(r), k0 + c, lda)];
    }
    __syncthreads();
    // Per-column scale of the panel for the overflow-safe norm: 2^-E with E the
    // exponent of the column's largest |entry| from its diagonal down (an exact
    // power of two; entries that earlier reflectors of the panel add stay
    // within a factor sqrt(M) of it).
#pragma unroll
    for (int t = 0; t < TL::NBW8; ++t) {
      const int c = warp + kBWarps * t;
      if (c < nbw) {
        unsigned mx = 0;
        for (int r = c + lane; r < M; r += 32) mx = max(mx, b_abs_hi(Ps[c * PR + r]));
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
      const T *x = Ps + j * PR;
      // phase 1: warp w takes panel columns w, w + 8, ...
#pragma unroll
      for (int t = 0; t < TL::NBW8; ++t) {
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
          const T *col = Ps + c * PR;
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
          const T pr_c = Ps[c * PR + j];
          if (c > j) sig[c] = defined ? (double)(-(upT * pr_c + (T)dots[c]) * tkT) : 0.0;
          else if (c < j) Gs[c + j * NB] = (double)(pr_c * upT + (T)dots[c]);
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
          const double pr_c = (double)Ps[c * PR + j];
          // sigma_c = (up p_c + D_c) / b = -(up p_c + D_c) tau
          if (c > j) sig[c] = defined ? -(upk * pr_c + dots[c]) * tk : 0.0;
          else if (c < j) Gs[c + j * NB] = pr_c * upk + dots[c];
        }
      }
      __syncthreads();
      if (defined) {
        const T upT = (T)upk;
#pragma unroll
        for (int t = 0; t < TL::NBW8; ++t) {
          const int c = warp + kBWarps * t;
          if (c > j && c < nbw) {
            T *col = Ps + c * PR;
            const T sg = (T)sig[c];
            for (int r = j + 1 + lane; r < M; r += 32) col[r] = fma(sg, x[r], col[r]);
            if (lane == 0) col[j] = fma(sg, upT, col[j]);
          }
        }
      }
      __syncthreads();
      if (tid == 0) {
        if (defined) Ps[j * PR + j] = (T)cl;
        tau[j] = tk;
        ups[j] = upk;
      }
      __syncthreads();
    }
    // write the panel back; keep G and tau if asked; then turn the slice into
    // V (zero above the diagonal, up on it) for the trailing update
    for (int idx = tid; idx < nbw * M; idx += kThreads) {
      int c = idx / M, r = idx - c * M;
      if (!(ntop > 0 && r < nbw && r > c)) A[SLQR_IDX(k0 + prow(r), k0 + c, lda)] = Ps[c * PR + r];
    }
    if (tid < nbw) up_out[k0 + tid] = ups[tid];
    if (G_out) {
      double *Gp = G_out + (size_t)(k0 / NB) * NB * NB;
      for (int idx = tid; idx < NB * NB; idx += kThreads) {
        int jj = idx / NB, q = idx - jj * NB;
        Gp[idx] = (q < jj && jj < nbw) ? Gs[idx] : 0.0;
      }
      if (tid < NB) tau_out[k0 + tid] = (tid < nbw) ? tau[tid] : 0.0;
    }
    __syncthreads();
    for (int idx = tid; idx < NB * NB; idx += kThreads) {
      int c = idx / NB, r = idx - c * NB;
      if (r <= c && r < M) Ps[c * PR + r] = (r == c && c < nbw) ? (T)ups[c] : T(0);
      Gt[idx] = (T)Gs[idx];
    }
    if (tid < NB) taut[tid] = (T)tau[tid];
    __syncthreads();

    // trailing columns [k0 + nbw, n), plus Bcol as one more column
    const int NT = n - (k0 + nbw);
    const int NC = NT + (Bcol ? 1 : 0);
    for (int t0 = 0; t0 < NC; t0 += TC) {
      // phase A: W[a][col] = sum_r V[a][r] C[r][col].  Warp w takes the CPW
      // columns CPW w .. CPW w + CPW - 1 of the tile; lane = RG (column -
      // CPW w) + g walks the rows r = g (mod RG), so a column's NB partial
      // sums are combined over RG lanes only (for NB = 16, TC = 32: 14 adds
      // per lane) and a ragged M leaves at most RG - 1 lanes of a column idle
      // on its last row step.
      if (t0 + TL::CPW * warp < NC) {
        const int cc = TL::CPW * warp + lane / TL::RG;
        const int col = t0 + cc;
        T acc[NB];
#pragma unroll
        for (int a = 0; a < NB; ++a) acc[a] = T(0);
        if (col < NC) {
          const T *C = (col < NT) ? A + SLQR_IDX(k0, k0 + nbw + col, lda) : (const T *)(Bcol + k0);
#pragma unroll 4
          for (int r = g8; r < M; r += TL::RG) {
            const T cv = C[prow(r)];
#pragma unroll
            for (int a = 0; a < NB; ++a)
              if (a < nbw) acc[a] = fma(Ps[a * PR + r], cv, acc[a]);
          }
        }
        b_group_sum<T, NB, TL::RG>(acc, g8);    // lane g holds W[VPL g + i], i < VPL
        if (col < NC) {
#pragma unroll
          for (int i = 0; i < TL::VPL; ++i) Wt[(TL::VPL * g8 + i) * (TC + 1) + cc] = acc[i];
        }
      }
      __syncthreads();
      // phase B: W' = T^T W, one thread per column, in T (an FP32
      // factorization keeps this chain off the slow FP64 pipe)
      if (tid < TC && t0 + tid < NC) {
        T w[NB];
#pragma unroll
        for (int jj = 0; jj < NB; ++jj) {
          if (jj < nbw) {
            T t = Wt[jj * (TC + 1) + tid];
#pragma unroll
            for (int q = 0; q < jj; ++q) t = fma(-Gt[q + jj * NB], w[q], t);
            w[jj] = taut[jj] * t;
            Wt[jj * (TC + 1) + tid] = w[jj];
          }
        }
      }
      __syncthreads();
      // phase C: C -= V W', the same lane layout as phase A
      {
        const int cc = TL::CPW * warp + lane / TL::RG;
        const int col = t0 + cc;
        if (col < NC) {
          T *C = (col < NT) ? A + SLQR_IDX(k0, k0 + nbw + col, lda) : (T *)(Bcol + k0);
          T w[NB];
#pragma unroll
          for (int a = 0; a < NB; ++a) w[a] = (a < nbw) ? Wt[a * (TC + 1) + cc] : T(0);
#pragma unroll 4
          for (int r = g8; r < M; r += TL::RG) {
            const int pr = prow(r);
            T cv = C[pr];
#pragma unroll
            for (int a = 0; a < NB; ++a)
              if (a < nbw) cv = fma(-Ps[a * PR + r], w[a], cv);
            C[pr] = cv;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Back-substitution R x = (Q^T b)[0:n] of the FP64 path, column-oriented.
static __device__ void batch_solve_fp64(const double *A, int lda, int n, double *b, double *xs,
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

// Two CTAs per SM, except for panels of 32 reflectors (their FP64 panel alone
// takes 131 KB of shared memory, and their 32 partial sums per lane need the
// registers of one CTA per SM).
template <int NB>
constexpr int batch_min_ctas() { return NB >= 32 ? 1 : 2; }

template <int NB, int TC>
__global__ void __launch_bounds__(kThreads, batch_min_ctas<NB>())
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
      batch_factor_core<double, NB, TC>(pr.A, pr.lda, pr.m, pr.n, pr.up, pr.b, nullptr, nullptr,
                                        smraw, pr.ntop);
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

// Shared-memory-resident FP64 kernel for problems of at most RM rows: the
// problem (A, ld m) and b are copied into shared memory once, factored and
// back-substituted there by the same code, and written back once, so the
// trailing updates and the solve never touch global memory.
template <int NB, int TC, int RM>
struct BatchResident {
  static constexpr size_t kCore = align_up_c(BatchSmem<double, NB, TC, RM>::kBytes, 16);
  static constexpr size_t kBytes = kCore + (size_t)(RM * RM + 2 * RM) * sizeof(double);
};

template <int NB, int TC, int RM>
__global__ void __launch_bounds__(kThreads, RM <= 64 ? 2 : 1)
batch_factor_resident_kernel(BatchParams bp) {
  extern __shared__ __align__(16) char smraw[];
  __shared__ int s_item;
  __shared__ int s_status;
  using RS = BatchResident<NB, TC, RM>;
  double *As = (double *)(smraw + RS::kCore);      // [RM][RM], ld m
  double *bs = As + RM * RM;                       // RM
  double *xs = bs + RM;                            // RM (the solve's scratch)
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(bp.counter, 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= bp.count) break;
    const int p = bp.order[item];
    const BatchProblem pr = bp.probs[p];
    const int m = pr.m, n = pr.n;
    if (n > 0) {
      for (int idx = threadIdx.x; idx < m * n; idx += kThreads) {
        const int c = idx / m, r = idx - c * m;
        // (stacked: the strictly lower part of the top block is not read)
        As[idx] = (pr.ntop > 0 && c < pr.ntop && r > c && r < pr.ntop) ? 0.0
                                                                       : pr.A[SLQR_IDX(r, c, pr.lda)];
      }
      if (pr.b)
        for (int i = threadIdx.x; i < m; i += kThreads) bs[i] = pr.b[i];
      __syncthreads();
      batch_factor_core<double, NB, TC, RM>(As, m, m, n, pr.up, pr.b ? bs : nullptr, nullptr,
                                            nullptr, smraw, pr.ntop);
      if (pr.b) {
        batch_solve_fp64(As, m, n, bs, xs, &s_status);
      } else if (threadIdx.x == 0) {
        s_status = SLQR_OK;
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < m * n; idx += kThreads) {
        const int c = idx / m, r = idx - c * m;
        if (!(pr.ntop > 0 && c < pr.ntop && r > c && r < pr.ntop)) pr.A[SLQR_IDX(r, c, pr.lda)] = As[idx];
      }
      if (pr.b)
        for (int i = threadIdx.x; i < m; i += kThreads) pr.b[i] = bs[i];
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
  double *gt;           // per CTA: kBGtDoubles (G, tau, up, column scales)
  int max_it;
  double tol;
};

// per-CTA global scratch of the mixed kernel: G of every panel ((m / NB)
// panels of NB^2, at most kBMaxRows kBNBMax doubles for any NB), tau, up and
// the column scales d_j of the equilibration
constexpr size_t kBGDoubles = (size_t)kBMaxRows * kBNBMax;
constexpr size_t kBGtDoubles = kBGDoubles + 3 * kBMaxRows;

// V(i, a) of panel p from the FP32 factorization (rows relative to k0 = p*NB)
static __device__ __forceinline__ float mixed_v(const float *Af, int m, const double *up, int k0,
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
// kBWarps * NB floats.
constexpr int kBRowsPerThread = kBMaxRows / kThreads;
static_assert(kBRowsPerThread * kThreads == kBMaxRows, "rows per thread");

template <int NB>
__device__ void mixed_apply_q(const float *Af, int m, int n, const double *G, const double *tau,
                              const double *up, float *y, float *red, bool forward) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = num_reflectors(m, n);
  const int np = num_panels(K, NB);
  // lanes sharing one W entry after the halving levels (32 / NB)
  constexpr int kShare = 32 / NB;
  for (int s = 0; s < np; ++s) {
    const int pnl = forward ? s : np - 1 - s;
    const int k0 = pnl * NB;
    const int nbw = min(NB, K - k0);
    const int M = m - k0;
    float vr[kBRowsPerThread][NB];
    float yv[kBRowsPerThread];
    float acc[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a) acc[a] = 0.f;
#pragma unroll
    for (int t = 0; t < kBRowsPerThread; ++t) {
      const int i = tid + t * kThreads;
      const bool in = i < M;
#pragma unroll
      for (int a = 0; a < NB; ++a) {
        float v = 0.f;
        if (in && a < nbw && i >= a)
          v = (i == a) ? (float)up[k0 + a] : Af[SLQR_IDX(k0 + i, k0 + a, m)];
        vr[t][a] = v;
      }
      yv[t] = in ? y[k0 + i] : 0.f;
#pragma unroll
      for (int a = 0; a < NB; ++a) acc[a] = fmaf(vr[t][a], yv[t], acc[a]);
    }
    // halving exchange over the warp (log2 NB levels from mask 16 down), then
    // plain butterflies over the kShare lanes left: lanes kShare a .. kShare a
    // + kShare - 1 end with the warp's total of acc[a]
#pragma unroll
    for (int h = NB / 2, mask = 16; h >= 1; h >>= 1, mask >>= 1) {
      const bool hi = (lane & mask) != 0;
#pragma unroll
      for (int i = 0; i < h; ++i) {
        const float send = hi ? acc[i] : acc[i + h];
        const float keep = hi ? acc[i + h] : acc[i];
        acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
      }
    }
#pragma unroll
    for (int mask = kShare / 2; mask >= 1; mask >>= 1)
      acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], mask);
    if ((lane & (kShare - 1)) == 0) red[warp * NB + lane / kShare] = acc[0];
    __syncthreads();
    // T^T w (forward) or T w, right-looking in FP32 on warp 0: lane j holds
    // w_j and its column (forward) or row of G; at step q lane q's value is
    // final and the lanes still open subtract its contribution
    if (warp == 0) {
      const double *Gp = G + (size_t)pnl * NB * NB;
      const int j = lane;
      const bool act = j < nbw;
      float t = 0.f;
      if (act) {
#pragma unroll
        for (int w8 = 0; w8 < kBWarps; ++w8) t += red[w8 * NB + j];
      }
      const float tj = act ? (float)tau[k0 + j] : 0.f;
      float gl[NB];
#pragma unroll
      for (int q = 0; q < NB; ++q)
        gl[q] = (act && q < nbw) ? (float)(forward ? Gp[q + j * NB] : Gp[j + q * NB]) : 0.f;
      float wf = 0.f;
#pragma unroll
      for (int s2 = 0; s2 < NB; ++s2) {
        const int q = forward ? s2 : NB - 1 - s2;
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
    float wv[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a) wv[a] = (a < nbw) ? red[a] : 0.f;
#pragma unroll
    for (int t = 0; t < kBRowsPerThread; ++t) {
      const int i = tid + t * kThreads;
      if (i < M) {
        float v = yv[t];
#pragma unroll
        for (int a = 0; a < NB; ++a) v = fmaf(-vr[t][a], wv[a], v);
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
static __device__ bool mixed_trsv(const float *Af, int m, int n, float *y, bool upper) {
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

static __device__ double block_max_abs(double v, double *red) {
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

template <int NB, int TC>
__global__ void __launch_bounds__(kThreads, batch_min_ctas<NB>())
batch_factor_mixed_kernel(BatchMixedParams bp) {
  extern __shared__ __align__(16) char smraw[];
  __shared__ int s_item;
  __shared__ double red[kBWarps];
  float *Af = bp.af + (size_t)blockIdx.x * kBMaxRows * kBMaxRows;
  double *G = bp.gt + (size_t)blockIdx.x * kBGtDoubles;
  double *tau = G + kBGDoubles;
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
    batch_factor_core<float, NB, TC>(Af, m, m, n, up, nullptr, G, tau, smraw, pr.ntop);
    __syncthreads();
    // refinement vectors in shared memory (the panel area is free now)
    double *x = (double *)smraw;          // n
    double *r = x + kBMaxRows;            // m
    double *dx = r + kBMaxRows;           // n (FP64 copy of the correction)
    float *f = (float *)(dx + kBMaxRows); // m   f, then d = Q^T f, then dr
    float *g = f + kBMaxRows;             // n   g, then h
    float *e = g + kBMaxRows;             // m
    float *w = e + kBMaxRows;             // kBWarps * NB (apply_q reductions)
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
      mixed_apply_q<NB>(Af, m, n, G, tau, up, f, w, true);    // d = Q^T f (in f)
      for (int i = tid; i < m; i += kThreads) e[i] = (i < n) ? f[i] - g[i] : f[i];
      __syncthreads();
      zero |= mixed_trsv(Af, m, n, e, true);                 // dx = R^-1 (d1 - h) (in e[0:n])
      for (int i = tid; i < n; i += kThreads) dx[i] = (double)e[i] * dcol[i];
      for (int i = tid; i < m; i += kThreads) f[i] = (i < n) ? g[i] : f[i];   // [h; d2]
      __syncthreads();
      mixed_apply_q<NB>(Af, m, n, G, tau, up, f, w, false);   // dr = Q [h; d2] (in f)
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


template <int NB, int TC>
constexpr size_t batch_mixed_smem_bytes() {
  return BatchSmem<float, NB, TC>::kBytes > 6 * kBMaxRows * sizeof(double)
             ? BatchSmem<float, NB, TC>::kBytes
             : 6 * kBMaxRows * sizeof(double);
}

// The two persistent kernels of one setting and their dynamic shared memory
// (the resident settings have an FP64 kernel only).
struct BatchKernels {
  const void *fp64 = nullptr, *mixed = nullptr;
  size_t smem_fp64 = 0, smem_mixed = 0;
};

template <int NB, int TC>
BatchKernels batch_kernels_of() {
  BatchKernels k;
  k.fp64 = (const void *)batch_factor_fp64_kernel<NB, TC>;
  k.mixed = (const void *)batch_factor_mixed_kernel<NB, TC>;
  k.smem_fp64 = BatchSmem<double, NB, TC>::kBytes;
  k.smem_mixed = batch_mixed_smem_bytes<NB, TC>();
  return k;
}

template <int NB, int TC, int RM>
BatchKernels batch_resident_kernels_of() {
  BatchKernels k;
  k.fp64 = (const void *)batch_factor_resident_kernel<NB, TC, RM>;
  k.smem_fp64 = BatchResident<NB, TC, RM>::kBytes;
  return k;
}

// The kernels of setting (nb, tc), instantiated in batch.cu (nb = 16, and the
// resident ones), batch_nb8.cu and batch_nb32.cu; null pointers for a setting
// that is not valid (nb < 256 / tc).
BatchKernels batch_kernels_nb8(int tc);
BatchKernels batch_kernels_nb16(int tc);
BatchKernels batch_kernels_nb32(int tc);

}  // namespace slqr
