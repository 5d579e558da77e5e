// factor.cu -- in-place H12 Householder QR on the GPU (FP64), blocked in
// panels of NB reflectors with a compact-WY trailing update.
//
// What it computes is Alg. 2 of the paper (Section 3): for each pivot k the
// kernel update_pivot_row builds reflector k from column k (its pivot entry
// `up` kept apart, Task 1 / Alg. 3), then update_trailing_non_pivot_row
// applies it to every later column.  The paper runs those two kernels as a
// DAG of CPU tasks; here the same arithmetic is regrouped for the GPU:
//
//  * panel kernel (cooperative, one CTA per slice of rows): for each of the NB
//    columns of the panel it does update_pivot_row (scaled norm, sign rule,
//    up) and update_trailing_non_pivot_row on the remaining panel columns.
//    One grid-wide reduction per column carries the partial column norm, the
//    dot products of the column tail with every other panel column, and the
//    pivot row.  The same dot products give the strict upper triangle of the
//    Gram matrix G = V^T V of the panel, so the compact-WY factor needs no
//    extra pass.
//  * trailing update of the columns right of the panel by all NB reflectors
//    at once: X <- (H_0 ... H_{NB-1})^T X = X - V T^T (V^T X), with
//    T^{-1} = striu(G) + diag(-b) (the identity T^{-1} + T^{-T} = V^T V of
//    the compact-WY form, with H_j = I - tau_j v_j v_j^T, tau_j = -1/b_j):
//      gemm_vtx   W_s = V_s^T X_s on row slices s (partials),
//      tw         W' = T^T W by forward substitution with striu(G), tau,
//      gemm_upd   X -= V W'.
//    All three run on the FP64 pipe (DFMA); on GB300 FP64 DMMA issues slower
//    than DFMA, so these are register-tiled DFMA kernels.
//
// Rounding differs from the sequential order (blocked sums, power-of-two
// scaled norms), so results agree with the sequential H12 to a tolerance,
// not bitwise.
#include "slqr_internal.cuh"

#include <cstdio>
#include <cstdarg>
#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>

namespace slqr {

// --------------------------------------------------------------------------
// small device helpers
// --------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// --------------------------------------------------------------------------
// panel kernel
// --------------------------------------------------------------------------
constexpr int kMaxPanelCtas = 160;
// The panel kernel sized for at most 64 CTAs holds fewer partials per thread
// (fewer registers), which lets trailing-update CTAs share the SMs it uses.
constexpr int kSmallPanelCtas = 64;

struct PanelParams {
  void *A;             // T * (the storage type of the factorization)
  double *up;          // global up array (n doubles)
  double *wy;          // this panel's compact-WY block (Vtop | G | tau)
  double *rec;         // NB * P * NB doubles: per column j the records [j][cta][entry]
  double *srec;        // P * NB doubles: per-CTA column scales (panel start)
  double *gpart;       // P * NB*(NB-1)/2 doubles: per-CTA partial Gram terms
  double *prow;        // NB * NB doubles: per column j the pivot row [j][entry]
  unsigned *bar;       // monotonic arrival counter
  int *status;
  int m, lda, k0, nbw;
  int skip;            // rows skipped after the panel's top nbw rows (stacked [L^T; C])
  int stacked;         // stacked [L^T; C]: the diagonal block's strict lower part is zero
  int P, R;            // CTAs, rows per CTA
  unsigned bar_base;   // counter value when this panel starts
  unsigned spin;       // polls of a bounded wait before it gives up
};

// Row map of a panel: row i of the panel (0 <= i < m - k0 - skip) is matrix
// row k0 + i for i < nbw and k0 + skip + i below.  skip = 0 for a dense
// matrix; for a stacked [L^T; C] (upper-triangular top block of n rows) the
// rows between the panel's diagonal block and C are zero in every reflector
// and untouched by the update, so they are left out.
__host__ __device__ __forceinline__ int panel_row(int k0, int nbw, int skip, int i) {
  return k0 + i + (i >= nbw ? skip : 0);
}

// Bits of |x| as an unsigned 64-bit integer: for non-negative doubles the
// integer order of the bit patterns is the numeric order.
template <typename T>
__device__ __forceinline__ unsigned abs_hi_bits(T x) {
  return (unsigned)((unsigned long long)__double_as_longlong((double)x) >> 32) & 0x7fffffffu;
}

// 2^e as a double for e in [-1022, 1023] (exact; built from the exponent bits)
__device__ __forceinline__ double pow2(int e) {
  return __longlong_as_double((long long)(e + 1023) << 52);
}

// Per-column records are exchanged without a grid barrier: every slot is
// written once per panel, and until then it holds kUnset, a signalling-NaN
// bit pattern that no arithmetic result has (FP operations return the
// canonical quiet NaN).  A reader polls the slot until it holds a value, so
// the value itself is the message (one 8-byte store, single-copy atomic).
constexpr unsigned long long kUnset = 0x7ff0dead5a5a5a5aull;

__device__ __forceinline__ bool is_unset(double v) {
  return (unsigned long long)__double_as_longlong(v) == kUnset;
}

// Publish v (relaxed, GPU scope); a copied input that happens to carry the
// kUnset pattern goes out as the canonical quiet NaN instead.
__device__ __forceinline__ void publish(double *p, double v) {
  if (is_unset(v)) v = __longlong_as_double(0x7fffffffffffffffll);
  asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

__device__ __forceinline__ double ld_relaxed_f64(const double *p) {
  double v;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
  return v;
}

// One CTA per slice of R rows of the panel (rows [k0, m), NB columns); the
// slice stays in shared memory for the whole panel.
//
// Panel start: each column c gets a power-of-two scale 2^-E_c from the
// largest |entry| of the column (one grid max-reduction of exponent bits, on
// the integer pipe).  The in-panel reflectors are orthogonal on rows
// [k0, m), so the column's tail never outgrows that scale: sum (x_i 2^-E_c)^2
// neither overflows nor, for any column that still carries weight,
// underflows.  The norm of each column is then a plain scaled sum reduced
// like the dot products (no exponent bookkeeping per column).
//
// Per column j:
//   phase 1  local partials: the scaled sum of squares of the column (from
//            the pivot down) and the dots of its tail with the later panel
//            columns (published); the dots with the earlier columns (Gram
//            terms of V^T V) are kept in a CTA-local accumulator.  Lane
//            partials are reduced through shared memory (every FP64
//            instruction works on 32 useful lanes).
//   phase 2  every CTA waits until each CTA's record of column j has arrived
//            (one warp polls the records; no grid barrier per column), then
//            reduces the published partials: thread (g, c) sums entry c over
//            its slice g of the CTAs (all loads in flight), the slices are
//            added in a fixed order (the same in every CTA);
//   pivot    one thread forms s, cl, up, b and 1/b; sigma_c = (up p_c + D_c)/b;
//   phase 3  update of the later panel columns.
// At the end the local Gram terms are published and reduced once, each CTA
// reducing its share of the entries into the compact-WY store.
template <typename T, int NB, int PMAX>
__global__ void __launch_bounds__(kThreads)
panel_kernel(PanelParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NW = kThreads / 32;
  constexpr int CPW = (NB + NW - 1) / NW;     // columns per warp
  constexpr int RECW = NB;                    // record: entry c (c == j: norm, c > j: dot)
  constexpr int GROUPS = kThreads / NB;       // CTA slices of the reduction
  constexpr int LQ = kThreads / NB;           // lane quarters in the phase-1 reduction
  T *Ps = (T *)smem_raw;                      // [NB][R] column-major panel slice
  double *Gloc = (double *)(smem_raw + ((size_t)NB * p.R * sizeof(T) + 15) / 16 * 16);
                                              // [NB][NB] local Gram terms
  // Per-column arithmetic (partial sums, norm, reduction, pivot, multipliers)
  // runs in the storage precision: an FP32 factorization keeps these chains
  // on the FP32 pipe (an FP64 operation waits tens of cycles on GB300, and
  // the chain of one column is the panel's critical path).  The norm stays
  // overflow-safe through the power-of-two column scale; a column whose scale
  // is extreme for FP32 (|E| > 60: s^2 or b could leave the FP32 range) forms
  // its pivot and multipliers in FP64.
  using Acc = typename std::conditional<std::is_same<T, float>::value, float, double>::type;
  constexpr bool kF32 = std::is_same<T, float>::value;
  __shared__ Acc s_lane[NB][33];
  __shared__ Acc s_nlane[32];
  __shared__ Acc s_part[GROUPS][NB];
  __shared__ unsigned s_mx[GROUPS][NB];       // column-scale reduction
  __shared__ Acc s_pivc[3];                   // cl, up, 1/b in Acc (FP32 pivot)
  __shared__ double s_sig[NB];                // sigma per column
  __shared__ double s_up[NB];
  __shared__ double s_prow[NB];               // pivot row of the current column
  __shared__ double s_sc[NB];                 // column scales 2^-E_c
  __shared__ int s_E[NB];
  __shared__ double s_piv[4];                 // cl, up, 1/b, tau
  __shared__ int s_defined;
  __shared__ int s_ok;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cta = blockIdx.x;
  const int R = p.R;
  const int row0 = cta * R;                        // first panel row of this slice
  const int RO = min(R, p.m - p.k0 - p.skip - row0);   // rows owned
  const int nbw = p.nbw;
  T *A = (T *)p.A;
  const int lda = p.lda;

  for (int idx = tid; idx < nbw * R; idx += kThreads) {
    int c = idx / R, r = idx - c * R;
    // (stacked: the strictly lower part of the diagonal block is zero, not read)
    const bool zero = r >= RO || (p.stacked && row0 + r < nbw && row0 + r > c) ||
                      !slqr_check(panel_row(p.k0, nbw, p.skip, row0 + r) < p.m, p.status);
    Ps[c * R + r] =
        zero ? T(0) : A[SLQR_IDX(panel_row(p.k0, nbw, p.skip, row0 + r), p.k0 + c, lda)];
  }
  for (int idx = tid; idx < NB * NB; idx += kThreads) Gloc[idx] = 0.0;
  // this CTA's record slots of every column (and CTA 0: the pivot rows) back
  // to kUnset; the grid barrier below orders this before any publish or poll
  for (int idx = tid; idx < nbw * NB; idx += kThreads) {
    const int jj = idx / NB, c = idx - jj * NB;
    p.rec[((size_t)jj * p.P + cta) * NB + c] = __longlong_as_double((long long)kUnset);
    if (cta == 0) p.prow[idx] = __longlong_as_double((long long)kUnset);
  }
  double *G = p.wy + (size_t)NB * NB;
  double *tau = p.wy + 2 * (size_t)NB * NB;
  __syncthreads();

  // ---- panel start: column scales ------------------------------------------
  {
    double *rec = p.srec;
#pragma unroll
    for (int t = 0; t < CPW; ++t) {
      const int c = warp + t * NW;
      unsigned mx = 0;
      if (c < nbw) {
        const int r_from = (cta == 0) ? c : 0;
        for (int r = r_from + lane; r < RO; r += 32) mx = max(mx, abs_hi_bits(Ps[c * R + r]));
      }
      mx = __reduce_max_sync(0xffffffffu, mx);
      if (lane == 0 && c < nbw) rec[(size_t)cta * RECW + c] = (double)mx;
    }
  }
  if (!grid_barrier(p.bar, p.bar_base + (unsigned)p.P, p.status, &s_ok, p.spin)) return;
  {
    constexpr int QMAX = (PMAX + GROUPS - 1) / GROUPS;
    const double *rec = p.srec;
    const int g = tid / NB, c = tid - g * NB;
    const int per = (p.P + GROUPS - 1) / GROUPS;
    const int q0 = g * per, q1 = min(p.P, q0 + per);
    unsigned v[QMAX];
#pragma unroll
    for (int t = 0; t < QMAX; ++t)
      v[t] = (c < nbw && q0 + t < q1) ? (unsigned)__ldcg(rec + (size_t)(q0 + t) * RECW + c) : 0u;
    unsigned mx = 0;
#pragma unroll
    for (int t = 0; t < QMAX; ++t) mx = max(mx, v[t]);
    s_mx[g][c] = mx;
  }
  __syncthreads();
  if (tid < NB) {
    unsigned mx = 0;
    for (int g = 0; g < GROUPS; ++g) mx = max(mx, s_mx[g][tid]);
    int E = (int)((mx >> 20) & 0x7ff) - 1023;        // exponent of the largest |entry|
    // (FP32: 2^-E and 2^E must both be normal floats)
    E = kF32 ? min(max(E, -126), 126) : min(max(E, -1000), 1022);
    s_E[tid] = E;
    s_sc[tid] = pow2(-E);
  }
  __syncthreads();

  for (int j = 0; j < nbw; ++j) {
    const double *rec = p.rec + (size_t)j * p.P * RECW;   // records of column j
    double *myrec = p.rec + ((size_t)j * p.P + cta) * RECW;
    double *prow = p.prow + (size_t)j * NB;
    const int r_tail = (cta == 0) ? j + 1 : 0;       // rows strictly below the pivot
    const T *x = Ps + j * R;

    // ---- phase 1 ---------------------------------------------------------
    {
      // dots in the storage type T, the norm on scaled entries
      T acc[CPW];
#pragma unroll
      for (int t = 0; t < CPW; ++t) acc[t] = T(0);
      Acc nacc = Acc(0);
      const bool norm_warp = (warp == (j % NW));
      const Acc sc = (Acc)s_sc[j];
      for (int r = r_tail + lane; r < RO; r += 32) {
        const T xv = x[r];
#pragma unroll
        for (int t = 0; t < CPW; ++t) {
          const int c = warp + t * NW;
          if (c < nbw && c != j) acc[t] = fma(xv, Ps[c * R + r], acc[t]);
        }
        if (norm_warp) {
          const Acc xs = (Acc)xv * sc;
          nacc = fma(xs, xs, nacc);
        }
      }
      if (cta == 0 && norm_warp && lane == 0) {     // the pivot entry joins the norm
        const Acc xs = (Acc)x[j] * sc;
        nacc = fma(xs, xs, nacc);
      }
#pragma unroll
      for (int t = 0; t < CPW; ++t) {
        const int c = warp + t * NW;
        if (c < NB && c != j) s_lane[c][lane] = (Acc)acc[t];
      }
      if (norm_warp) s_nlane[lane] = nacc;
      if (cta == 0 && tid < nbw) publish(prow + tid, (double)Ps[tid * R + j]);
    }
    __syncthreads();
    {
      // thread (c, quarter) sums 32 / LQ lane partials; then one thread per c
      const int c = tid / LQ, qq = tid - c * LQ;
      constexpr int LPQ = 32 / LQ;
      Acc v = Acc(0);
      if (c == j) {
#pragma unroll
        for (int l = 0; l < LPQ; ++l) v += s_nlane[qq * LPQ + l];
      } else {
#pragma unroll
        for (int l = 0; l < LPQ; ++l) v += s_lane[c][qq * LPQ + l];
      }
      s_part[qq][c] = v;
    }
    __syncthreads();
    if (tid < nbw) {
      const int c = tid;
      Acc v = s_part[0][c];
#pragma unroll
      for (int qq = 1; qq < LQ; ++qq) v += s_part[qq][c];
      if (c >= j) publish(myrec + c, (double)v);      // norm (c == j) and dots
      else Gloc[c + j * NB] = (double)v;              // Gram term: kept
    }

    // ---- phase 2 ---------------------------------------------------------
    {
      constexpr int QMAX = (PMAX + GROUPS - 1) / GROUPS;
      static_assert(QMAX <= 64, "one pending bit per polled record");
      const int g = tid / NB, c = tid - g * NB;
      const int per = (p.P + GROUPS - 1) / GROUPS;
      const int q0 = g * per, q1 = min(p.P, q0 + per);
      const bool sums = c >= j && c < nbw;
      // warp 0 waits until the norm entry of every CTA's record has arrived
      // (a record's entries are stored together, so the rest follow at once):
      // each lane loads its CTAs' entries together, then polls the missing
      bool ok = true;
      if (warp == 0) {
        constexpr int PW = (PMAX + 31) / 32;
        unsigned pend = 0;
#pragma unroll
        for (int t = 0; t < PW; ++t) {
          const int q = lane + 32 * t;
          if (q < p.P && is_unset(ld_relaxed_f64(rec + (size_t)q * RECW + j))) pend |= 1u << t;
        }
        unsigned it = 0;
        while (pend != 0) {                           // bounded
          if (++it > p.spin) { ok = false; break; }
          if (it > 8) __nanosleep(32);
#pragma unroll
          for (int t = 0; t < PW; ++t) {
            if (((pend >> t) & 1u) && !is_unset(ld_relaxed_f64(rec + (size_t)(lane + 32 * t) * RECW + j)))
              pend &= ~(1u << t);
          }
        }
      }
      if (!__syncthreads_and(ok)) {
        if (tid == 0) record_status(p.status, SLQR_ETIMEOUT);
        return;
      }
      // every thread loads its entries (all in flight, from L2) and sums them
      // in a fixed order; an entry not yet visible (rare: it still reads as
      // kUnset) sends the thread through a bounded re-poll of its slots in
      // the same order
      double v[QMAX];
#pragma unroll
      for (int t = 0; t < QMAX; ++t)
        v[t] = (sums && q0 + t < q1) ? __ldcg(rec + (size_t)(q0 + t) * RECW + c) : 0.0;
      double pv = (tid < nbw) ? __ldcg(prow + tid) : 0.0;
      Acc acc = Acc(0);
      bool miss = false;
#pragma unroll
      for (int t = 0; t < QMAX; ++t) {
        miss |= is_unset(v[t]);
        acc += (Acc)v[t];
      }
      if (miss) {
        acc = Acc(0);
        for (int t = 0; t < QMAX && ok; ++t) {
          if (!(sums && q0 + t < q1)) continue;
          double x;
          unsigned it = 0;
          while (is_unset(x = ld_relaxed_f64(rec + (size_t)(q0 + t) * RECW + c))) {
            if (++it > p.spin) { ok = false; break; }
            __nanosleep(32);
          }
          acc += (Acc)x;
        }
      }
      if (tid < nbw) {
        unsigned it = 0;
        while (is_unset(pv)) {
          if (++it > p.spin) { ok = false; break; }
          __nanosleep(32);
          pv = ld_relaxed_f64(prow + tid);
        }
      }
      if (sums) s_part[g][c] = acc;
      if (tid < nbw) s_prow[tid] = pv;
      if (!__syncthreads_and(ok)) {
        if (tid == 0) record_status(p.status, SLQR_ETIMEOUT);
        return;
      }
    }
    // FP32 pivot unless the column's scale is extreme (uniform over the CTA)
    const bool fast = kF32 && abs(s_E[j]) <= 60;
    if (tid == 0) {
      Acc Sa = s_part[0][j];
      for (int g = 1; g < GROUPS; ++g) Sa += s_part[g][j];
      const bool defined = (Sa != Acc(0));
      double cl = 0.0, upk = 0.0, rb = 0.0;
      if (defined && fast) {
        const Acc sn = sqrt(Sa) * (Acc)pow2(s_E[j]);
        const Acc x0 = (Acc)s_prow[j];
        const Acc clc = (x0 > Acc(0)) ? -sn : sn;
        const Acc upc = x0 - clc;
        const Acc rbc = Acc(1) / (upc * clc);         // 1 / b
        s_pivc[0] = clc;
        s_pivc[1] = upc;
        s_pivc[2] = rbc;
        cl = clc;
        upk = upc;
        rb = rbc;
      } else if (defined) {
        const double sn = sqrt((double)Sa) * pow2(s_E[j]);
        const double x0 = s_prow[j];
        cl = (x0 > 0.0) ? -sn : sn;
        upk = x0 - cl;
        rb = 1.0 / (upk * cl);                        // 1 / b
      }
      s_piv[0] = cl;
      s_piv[1] = upk;
      s_piv[2] = rb;
      s_piv[3] = -rb;                                 // tau = -1 / b
      s_defined = defined;
    }
    __syncthreads();

    const bool defined = s_defined != 0;
    const double cl = s_piv[0], upk = s_piv[1], rb = s_piv[2];
    if (tid < nbw) {
      const int c = tid;
      if (c > j) {
        Acc D = s_part[0][c];
#pragma unroll
        for (int g = 1; g < GROUPS; ++g) D += s_part[g][c];
        if (!defined) s_sig[c] = 0.0;
        else if (fast) s_sig[c] = (double)((s_pivc[1] * (Acc)s_prow[c] + D) * s_pivc[2]);
        else s_sig[c] = (upk * s_prow[c] + (double)D) * rb;
      } else if (c < j && cta == 0) {
        // G[c, j] = v_c^T v_j = v_c[k] up_j + sum_{r > k} v_c[r] x_r: the first
        // term is added once, by CTA 0
        Gloc[c + j * NB] += s_prow[c] * upk;
      }
    }
    if (cta == 0 && tid == 0) {
      s_up[j] = upk;
      p.up[p.k0 + j] = upk;
      tau[j] = s_piv[3];
    }
    __syncthreads();

    // ---- phase 3: apply the reflector to the remaining panel columns -------
    if (defined) {
      for (int t = 0; t < CPW; ++t) {
        int c = warp + t * NW;
        if (c > j && c < nbw) {
          const T sg = (T)s_sig[c];
          T *col = Ps + c * R;
          for (int r = r_tail + lane; r < RO; r += 32) col[r] = fma(sg, x[r], col[r]);
        }
      }
      if (cta == 0) {
        int c = tid;
        if (c > j && c < nbw) Ps[c * R + j] = (T)fma(s_sig[c], upk, (double)Ps[c * R + j]);
        if (tid == 0) Ps[j * R + j] = (T)cl;
      }
    }
    __syncthreads();
  }

  // write the slice back
  for (int idx = tid; idx < nbw * R; idx += kThreads) {
    int c = idx / R, r = idx - c * R;
    if (r < RO && !(p.stacked && row0 + r < nbw && row0 + r > c))
      A[SLQR_IDX(panel_row(p.k0, nbw, p.skip, row0 + r), p.k0 + c, lda)] = Ps[c * R + r];
  }
  // publish the local Gram terms and reduce them: CTA q owns entries q, q+P, ..
  constexpr int NT = NB * (NB - 1) / 2;       // strict upper triangle, packed by column
  {
    double *mine = p.gpart + (size_t)cta * NT;
    for (int idx = tid; idx < NB * NB; idx += kThreads) {
      const int jj = idx / NB, c = idx - jj * NB;
      if (c < jj) mine[jj * (jj - 1) / 2 + c] = Gloc[idx];
    }
  }
  if (!grid_barrier(p.bar, p.bar_base + 2u * (unsigned)p.P, p.status, &s_ok, p.spin)) return;
  for (int idx = cta + tid * p.P; idx < NB * NB; idx += kThreads * p.P) {
    const int jj = idx / NB, c = idx - jj * NB;
    double v = 0.0;
    if (c < jj && jj < nbw) {
      const int pos = jj * (jj - 1) / 2 + c;
      for (int q = 0; q < p.P; ++q) v += __ldcg(p.gpart + (size_t)q * NT + pos);
    }
    G[idx] = v;
  }
  if (cta == 0) {
    // Vtop (ld NB): zero above the diagonal, up on it, tails below
    double *Vtop = p.wy;
    for (int idx = tid; idx < NB * NB; idx += kThreads) {
      int c = idx / NB, r = idx - c * NB;
      double v = 0.0;
      if (c < nbw && r < nbw) {
        if (r == c) v = s_up[c];
        else if (r > c) v = (double)Ps[c * R + r];
      }
      Vtop[idx] = v;
    }
    for (int c = nbw + tid; c < NB; c += kThreads) tau[c] = 0.0;
  }
}

// --------------------------------------------------------------------------
// tiled kernels of the trailing update (T = double: the FP64 path; T = float:
// the FP32 factorization of the mixed-precision path)
// --------------------------------------------------------------------------
// V(i, a) for the panel at row offset k0: rows i < nbw from Vtop, the rest
// straight from the reflector tails in A.  Columns a >= nbw read as 0.
template <typename T>
__device__ __forceinline__ T v_at(const T *A, int lda, const double *Vtop, int NB, int k0,
                                  int nbw, int i, int a, int skip) {
  if (a >= nbw) return T(0);
  if (i < nbw) return (T)Vtop[i + a * NB];
  return A[SLQR_IDX(k0 + skip + i, k0 + a, lda)];
}

constexpr int kBK = 32;   // rows per chunk of the V^T X reduction
constexpr int kBN = 64;   // columns per tile
constexpr int kBM = 64;   // rows per tile of the update

// W_part[s][c][a] = sum_{i in slice s} V(i, a) X(i, c)
// grid: (ceil(N / kBN), S); rows of slice s: [s*RS, min((s+1)*RS, M))
template <typename T, int NB, bool X_IS_V>
__global__ void __launch_bounds__(kThreads)
gemm_vtx_kernel(const T *__restrict__ A, int lda, const double *__restrict__ Vtop, int k0,
                int nbw, int M, const T *__restrict__ X, int ldx, int N, int RS,
                T *__restrict__ Wp, int skip = 0) {
  __shared__ T Vs[NB][kBK + 1];
  __shared__ T Xs[kBN][kBK + 1];
  constexpr int TP = NB / 16;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int c0 = blockIdx.x * kBN;
  const int s = blockIdx.y;
  const int i_begin = s * RS, i_end = min(M, i_begin + RS);
  T acc[TP][4];
#pragma unroll
  for (int a = 0; a < TP; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[a][q] = T(0);

  for (int i0 = i_begin; i0 < i_end; i0 += kBK) {
    for (int idx = tid; idx < NB * kBK; idx += kThreads) {
      int a = idx / kBK, ii = idx - a * kBK;
      int i = i0 + ii;
      Vs[a][ii] = (i < i_end) ? v_at<T>(A, lda, Vtop, NB, k0, nbw, i, a, skip) : T(0);
    }
    for (int idx = tid; idx < kBN * kBK; idx += kThreads) {
      int c = idx / kBK, ii = idx - c * kBK;
      int i = i0 + ii, cc = c0 + c;
      T v = T(0);
      if (i < i_end && cc < N) {
        if (X_IS_V) v = v_at<T>(A, lda, Vtop, NB, k0, nbw, i, cc, skip);
        else v = X[SLQR_IDX(panel_row(k0, nbw, skip, i), cc, ldx)];
      }
      Xs[c][ii] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kBK; ++kk) {
      T va[TP], xc[4];
#pragma unroll
      for (int a = 0; a < TP; ++a) va[a] = Vs[tx + 16 * a][kk];
#pragma unroll
      for (int q = 0; q < 4; ++q) xc[q] = Xs[ty + 16 * q][kk];
#pragma unroll
      for (int a = 0; a < TP; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[a][q] = fma(va[a], xc[q], acc[a][q]);
    }
    __syncthreads();
  }
  T *out = Wp + (size_t)s * N * NB;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int cc = c0 + ty + 16 * q;
    if (cc < N) {
#pragma unroll
      for (int a = 0; a < TP; ++a) out[(size_t)cc * NB + tx + 16 * a] = acc[a][q];
    }
  }
}

// W'[a][c] = (T^T W)[a][c] (TRANS) or (T W)[a][c].  Each CTA owns kThreads / NB
// columns and each thread one (column, reflector) entry: it sums that
// entry's S partials in a fixed order (coalesced loads, all of a thread's
// loads independent).  Then one warp does the substitution with
// T^{-1} = striu(G) + diag(1/tau):
//   T^T w:  w'_j = tau_j (w_j - sum_{q<j} G[q,j] w'_q),  j = 0 .. nbw-1
//   T w:    w'_j = tau_j (w_j - sum_{q>j} G[j,q] w'_q),  j = nbw-1 .. 0
// (in the storage precision: FP64 for the FP64 factorization, FP32 for the
// FP32 one).
template <typename T, int NB, bool TRANS, int COLS, bool CMAJOR = false>
__global__ void __launch_bounds__(kThreads)
tw_kernel(const T *__restrict__ Wp, int S, int N, const double *__restrict__ wy, int nbw,
          T *__restrict__ Wt) {
  static_assert(COLS * NB <= kThreads, "one entry needs at least one thread");
  constexpr int TPE = kThreads / (COLS * NB);   // threads per entry (split over s)
  // arithmetic in the storage precision: FP64 for the FP64 factorization,
  // FP32 for the FP32 one (G and tau converted once per CTA), so that the
  // substitution chain of an FP32 update stays off the FP64 pipe
  using AT = T;
  __shared__ AT w[NB][COLS + 1];
  __shared__ AT part[TPE][COLS * NB];
  // striu(V^T V) of the panel, row-major with row stride NB + 1: the
  // substitution reads a row (TRANS) or a column of it across the lanes, and
  // both are conflict-free in this layout (the store is column-major)
  constexpr int GLD = NB + 1;
  __shared__ AT G[NB * GLD];
  __shared__ AT tau[NB];
  const int tid = threadIdx.x;
  {
    // all loads of G issued before the first store (one round trip to L2)
    constexpr int GPER = NB * NB / kThreads;
    static_assert(GPER * kThreads == NB * NB, "G splits evenly over the threads");
    double gv[GPER];
#pragma unroll
    for (int u = 0; u < GPER; ++u) gv[u] = wy[(size_t)NB * NB + tid + u * kThreads];
#pragma unroll
    for (int u = 0; u < GPER; ++u) {
      const int idx = tid + u * kThreads, r = idx % NB, c = idx / NB;
      G[r * GLD + c] = (AT)gv[u];
    }
  }
  if (tid < NB) tau[tid] = (AT)wy[2 * (size_t)NB * NB + tid];
  const int c0 = blockIdx.x * COLS;
  {
    const int e = tid % (COLS * NB), h = tid / (COLS * NB);
    const int c = e / NB, a = e - c * NB;        // entry (column c0 + c, reflector a)
    AT acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
    if (c0 + c < N) {
      const T *src = Wp + (size_t)(c0 + c) * NB + a;
      const size_t stride = (size_t)N * NB;
      int s = h;
      for (; s + 3 * TPE < S; s += 4 * TPE) {
        acc0 += (AT)src[(size_t)s * stride];
        acc1 += (AT)src[(size_t)(s + TPE) * stride];
        acc2 += (AT)src[(size_t)(s + 2 * TPE) * stride];
        acc3 += (AT)src[(size_t)(s + 3 * TPE) * stride];
      }
      for (; s < S; s += TPE) acc0 += (AT)src[(size_t)s * stride];
    }
    part[h][e] = (acc0 + acc1) + (acc2 + acc3);
  }
  __syncthreads();
  if (tid < COLS * NB) {
    AT v = part[0][tid];
#pragma unroll
    for (int h = 1; h < TPE; ++h) v += part[h][tid];
    const int c = tid / NB, a = tid - c * NB;
    w[a][c] = v;
  }
  __syncthreads();
  // Substitution, right-looking, one warp per column with the column's NB
  // entries in registers (lane l holds rows l and l + 32): at step j the
  // owner's entry becomes w'_j = tau_j w_j, which is broadcast and folded into
  // every row still to come (TRANS: k > j with G[j, k]; else k < j with
  // G[k, j]).  The chain per step is one shuffle, one multiply and one FMA.
  static_assert(COLS <= kThreads / 32, "one warp per column");
  const int warp = tid >> 5, lane = tid & 31;
  if (warp < COLS) {
    const int c = warp;
    AT r0 = w[lane][c];
    AT r1 = (NB > 32) ? w[(lane + 32) & (NB - 1)][c] : AT(0);
    for (int s = 0; s < nbw; ++s) {
      const int j = TRANS ? s : nbw - 1 - s;
      const AT wj = __shfl_sync(0xffffffffu, (j < 32) ? r0 : r1, j & 31);
      const AT wpj = tau[j] * wj;
      if (TRANS) {
        if (lane > j) r0 = fma(-G[j * GLD + lane], wpj, r0);
        if (NB > 32 && lane + 32 > j) r1 = fma(-G[j * GLD + ((lane + 32) & (NB - 1))], wpj, r1);
      } else {
        if (lane < j) r0 = fma(-G[lane * GLD + j], wpj, r0);
        if (NB > 32 && lane + 32 < j) r1 = fma(-G[(lane + 32) * GLD + j], wpj, r1);
      }
      if (lane == (j & 31)) {
        if (j < 32) r0 = wpj;
        else r1 = wpj;
      }
    }
    w[lane][c] = r0;
    if (NB > 32) w[(lane + 32) & (NB - 1)][c] = r1;
  }
  __syncthreads();
  if (CMAJOR) {                                 // W'^T: [column][reflector] (tensor-core path)
    for (int idx = tid; idx < NB * COLS; idx += kThreads) {
      const int c = idx / NB, a = idx - c * NB;
      if (c0 + c < N) Wt[(size_t)(c0 + c) * NB + a] = (a < nbw) ? (T)w[a][c] : T(0);
    }
  } else {                                      // W': [reflector][column]
    for (int idx = tid; idx < NB * COLS; idx += kThreads) {
      const int a = idx / COLS, c = idx - a * COLS;
      if (c0 + c < N) Wt[(size_t)a * N + c0 + c] = (a < nbw) ? (T)w[a][c] : T(0);
    }
  }
}

// Launch W' = T^T W (TRANS) or T W: one column per CTA (4 threads per entry)
// while there are few columns, kThreads / NB columns per CTA otherwise.
template <typename T, int NB, bool TRANS, bool CMAJOR = false>
static void launch_tw(const T *Wp, int S, int N, const double *wy, int nbw, T *Wt,
                      cudaStream_t stream) {
  constexpr int WIDE = kThreads / NB;
  if (N <= 4 * 152) {
    tw_kernel<T, NB, TRANS, 1, CMAJOR><<<N, kThreads, 0, stream>>>(Wp, S, N, wy, nbw, Wt);
  } else {
    tw_kernel<T, NB, TRANS, WIDE, CMAJOR><<<(N + WIDE - 1) / WIDE, kThreads, 0, stream>>>(
        Wp, S, N, wy, nbw, Wt);
  }
}

// X(i, c) -= sum_a V(i, a) W'[a][c] on a kBM x kBN tile; grid (ceil(M/kBM), ceil(N/kBN))
template <typename T, int NB>
__global__ void __launch_bounds__(kThreads)
gemm_upd_kernel(const T *__restrict__ A, int lda, const double *__restrict__ Vtop, int k0,
                int nbw, int M, T *__restrict__ X, int ldx, int N, const T *__restrict__ Wt,
                int skip = 0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Vs = (T *)smem_raw;             // [NB][kBM]
  T *Ws = Vs + NB * kBM;             // [NB][kBN]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * kBM, c0 = blockIdx.y * kBN;
  for (int idx = tid; idx < NB * kBM; idx += kThreads) {
    int a = idx / kBM, ii = idx - a * kBM;
    int i = i0 + ii;
    Vs[idx] = (i < M) ? v_at<T>(A, lda, Vtop, NB, k0, nbw, i, a, skip) : T(0);
  }
  for (int idx = tid; idx < NB * kBN; idx += kThreads) {
    int a = idx / kBN, cc = idx - a * kBN;
    Ws[idx] = (c0 + cc < N) ? Wt[(size_t)a * N + c0 + cc] : T(0);
  }
  __syncthreads();
  T acc[4][4];
#pragma unroll
  for (int pp = 0; pp < 4; ++pp)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[pp][q] = T(0);
#pragma unroll 4
  for (int a = 0; a < nbw; ++a) {
    T v[4], ww[4];
#pragma unroll
    for (int pp = 0; pp < 4; ++pp) v[pp] = Vs[a * kBM + tx + 16 * pp];
#pragma unroll
    for (int q = 0; q < 4; ++q) ww[q] = Ws[a * kBN + ty + 16 * q];
#pragma unroll
    for (int pp = 0; pp < 4; ++pp)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[pp][q] = fma(v[pp], ww[q], acc[pp][q]);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int cc = c0 + ty + 16 * q;
    if (cc >= N) continue;
#pragma unroll
    for (int pp = 0; pp < 4; ++pp) {
      int i = i0 + tx + 16 * pp;
      if (i < M) {
        T *dst = X + SLQR_IDX(panel_row(k0, nbw, skip, i), cc, ldx);
        *dst -= acc[pp][q];
      }
    }
  }
}

// FP32 forms of the two products for panels of width 64.  The FP64 kernels
// above read one value per shared-memory load, which leaves the FP32 pipe
// waiting on shared memory (8 loads per 16 FMAs, at about twice the FMA
// time); these read four values per 16-byte load and stage each tile with
// every global load issued before the first store.  Each output sums its
// terms in the same order as the FP64-form kernels, so results are
// identical.
constexpr int kF32Ld = kBK + 4;   // row stride of a staged chunk (= 4 mod 32)

// W_part[s][c][a] = sum_{i in slice s} V(i, a) X(i, c), chunks of kBK rows
// staged [column][row]; thread (tx, ty) owns a = tx + 16 i, c = ty + 16 j and
// reads four consecutive rows of each with one load (V: 16 distinct addresses
// per half-warp, two wavefronts; X: two, one wavefront).
__global__ void __launch_bounds__(kThreads, 3)
gemm_vtx_f32_kernel(const float *__restrict__ A, int lda, const double *__restrict__ Vtop,
                    int k0, int nbw, int M, const float *__restrict__ X, int ldx, int N, int RS,
                    float *__restrict__ Wp, int skip) {
  constexpr int NB = 64;
  __shared__ __align__(16) float Vs[NB * kF32Ld];
  __shared__ __align__(16) float Xs[kBN * kF32Ld];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int c0 = blockIdx.x * kBN;
  const int s = blockIdx.y;
  const int i_begin = s * RS, i_end = min(M, i_begin + RS);
  constexpr int PER = NB * kBK / kThreads;     // entries of V (and of X) per thread: 8
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int i0 = i_begin; i0 < i_end; i0 += kBK) {
    float vv[PER], xv[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int idx = tid + u * kThreads, a = idx / kBK, kk = idx % kBK;
      const int i = i0 + kk, cc = c0 + a;
      vv[u] = (i < i_end) ? v_at<float>(A, lda, Vtop, NB, k0, nbw, i, a, skip) : 0.f;
      xv[u] = (i < i_end && cc < N) ? X[SLQR_IDX(panel_row(k0, nbw, skip, i), cc, ldx)] : 0.f;
    }
    __syncthreads();                           // the previous chunk has been read
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int idx = tid + u * kThreads, a = idx / kBK, kk = idx % kBK;
      Vs[a * kF32Ld + kk] = vv[u];
      Xs[a * kF32Ld + kk] = xv[u];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; kk += 4) {
      float4 va[4], xc[4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
        va[i] = *reinterpret_cast<const float4 *>(Vs + (tx + 16 * i) * kF32Ld + kk);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        xc[j] = *reinterpret_cast<const float4 *>(Xs + (ty + 16 * j) * kF32Ld + kk);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j] = fmaf(va[i].x, xc[j].x, acc[i][j]);
          acc[i][j] = fmaf(va[i].y, xc[j].y, acc[i][j]);
          acc[i][j] = fmaf(va[i].z, xc[j].z, acc[i][j]);
          acc[i][j] = fmaf(va[i].w, xc[j].w, acc[i][j]);
        }
    }
  }
  float *out = Wp + (size_t)s * N * NB;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int cc = c0 + ty + 16 * j;
    if (cc < N) {
#pragma unroll
      for (int i = 0; i < 4; ++i) out[(size_t)cc * NB + tx + 16 * i] = acc[i][j];
    }
  }
}

// X(i, c) -= sum_a V(i, a) W'[a][c] on a kBM x kBN tile; thread (tx, ty) owns
// rows 4 tx .. 4 tx + 3 and columns 4 ty .. 4 ty + 3 and reads each with one
// 16-byte load per reflector; X is read and written four rows at a time where
// the row map and the alignment allow (vec).
__global__ void __launch_bounds__(kThreads)
gemm_upd_f32_kernel(const float *__restrict__ A, int lda, const double *__restrict__ Vtop,
                    int k0, int nbw, int M, float *__restrict__ X, int ldx, int N,
                    const float *__restrict__ Wt, int skip, int vec) {
  constexpr int NB = 64;
  __shared__ __align__(16) float Vs[NB * kBM];   // [a][row]
  __shared__ __align__(16) float Ws[NB * kBN];   // [a][column]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * kBM, c0 = blockIdx.y * kBN;
  {
    constexpr int PER = NB * kBM / kThreads;    // 16
    float vv[PER], wv[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int idx = tid + u * kThreads, a = idx / kBM, ii = idx % kBM;
      const int i = i0 + ii;
      vv[u] = (i < M) ? v_at<float>(A, lda, Vtop, NB, k0, nbw, i, a, skip) : 0.f;
      wv[u] = (c0 + ii < N) ? Wt[(size_t)a * N + c0 + ii] : 0.f;   // (kBN == kBM)
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int idx = tid + u * kThreads;
      Vs[idx] = vv[u];
      Ws[idx] = wv[u];
    }
  }
  __syncthreads();
  float acc[4][4];                              // [row p][column q]
#pragma unroll
  for (int pp = 0; pp < 4; ++pp)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[pp][q] = 0.f;
#pragma unroll 4
  for (int a = 0; a < nbw; ++a) {
    const float4 v = *reinterpret_cast<const float4 *>(Vs + a * kBM + 4 * tx);
    const float4 w = *reinterpret_cast<const float4 *>(Ws + a * kBN + 4 * ty);
    const float vr[4] = {v.x, v.y, v.z, v.w}, wr[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int pp = 0; pp < 4; ++pp)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[pp][q] = fmaf(vr[pp], wr[q], acc[pp][q]);
  }
  const int ib = i0 + 4 * tx;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int cc = c0 + 4 * ty + q;
    if (cc >= N) continue;
    if (vec && ib + 3 < M && (ib >= nbw || ib + 3 < nbw)) {
      float4 *dst = reinterpret_cast<float4 *>(X + SLQR_IDX(panel_row(k0, nbw, skip, ib), cc, ldx));
      float4 x = *dst;
      x.x -= acc[0][q]; x.y -= acc[1][q]; x.z -= acc[2][q]; x.w -= acc[3][q];
      *dst = x;
    } else {
#pragma unroll
      for (int pp = 0; pp < 4; ++pp) {
        const int i = ib + pp;
        if (i < M) X[SLQR_IDX(panel_row(k0, nbw, skip, i), cc, ldx)] -= acc[pp][q];
      }
    }
  }
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
// Tuning knobs (slqr_set_tuning): panel width override and the smallest
// slice of rows a panel CTA holds (which sets how many CTAs share a panel).
static int g_tune_nb = 0;
static int g_tune_rows_min = 0;        // 0: chosen from the panel height (rows_min_auto)

// Per-shape settings found by slqr_autotune, keyed by (m, n); the global
// overrides of slqr_set_tuning take precedence.
struct TuneEntry { int nb, rows_min; };
static std::map<std::pair<int, int>, TuneEntry> g_tune_cache;
static std::mutex g_tune_mu;

static bool tune_lookup(int m, int n, TuneEntry *e) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune_cache.find({m, n});
  if (it == g_tune_cache.end()) return false;
  *e = it->second;
  return true;
}

// The rows-per-CTA minimum for an m x n factorization (0: by panel height).
static int rows_min_for(int m, int n) {
  if (g_tune_rows_min > 0) return g_tune_rows_min;
  TuneEntry e;
  return tune_lookup(m, n, &e) ? e.rows_min : 0;
}

// Smallest row slice per panel CTA when not set: small panels get more CTAs
// (each column step then does less FP64 work per SM), tall ones fewer (they
// share the SMs with the concurrent trailing update).  Measured on GB300:
// 600 x 500 and 1200 x 1000 are 20-25% faster with 64 rows than with 192,
// 2500..5000 rows best with 128, 8192 rows and up with 192.  The FP32 panel
// (mixed precision) does little arithmetic per row: 128 rows stay best at
// 8192 rows (the 8192 x 4096 mixed solves 3-5% faster than with 192).
static int rows_min_auto(int M, size_t elem) {
  if (elem == sizeof(float)) return M < 1536 ? 64 : 128;
  return M < 1536 ? 64 : (M < 6144 ? 128 : 192);
}

// Panel by a thread-block cluster (panel_cluster.cu): 0 chosen per panel,
// -1 never, 2..16 clusters of that many CTAs wherever the panel fits.
static int g_panel_cluster = 0;

// Automatic choice: the FP32 panel whenever it fits a cluster (its column
// steps are latency-bound: an exchange through distributed shared memory
// instead of polled records in L2).  FP64 panels stay cooperative: their
// column steps carry the slow FP64 FMAs of a slice, which the cooperative
// panel spreads over more SMs (on GB300 the 256 x 128 problem takes 1.56 ms
// with it and 2.4 ms with a cluster of 4 to 16 CTAs).  At least
// kClusterRowsMin rows per CTA.
constexpr int kClusterRowsMin = 64;
constexpr int kClusterMaxCtas = 16;

int panel_cluster_ctas(slqr_ctx *ctx, bool f32, int nb, int M, int nbw) {
  const int mode = g_panel_cluster;
  if (mode < 0 || M <= 0) return 0;
  const size_t elem = f32 ? sizeof(float) : sizeof(double);
  const int rmax = cluster_panel_rows_max(ctx, nb, elem);
  int ctas;
  if (mode > 0) {
    ctas = mode;
  } else {
    if (!f32) return 0;
    ctas = std::min(kClusterMaxCtas, (M + kClusterRowsMin - 1) / kClusterRowsMin);
  }
  ctas = std::max(1, ctas);
  const int R = std::max(nbw, (M + ctas - 1) / ctas);
  if (R > rmax) return 0;
  ctas = (M + R - 1) / R;                        // no CTA without rows
  if (!cluster_panel_fits(ctx, f32, nb, ctas, R)) return 0;
  return ctas;
}

int panel_width(int m, int n) {
  if (g_tune_nb == 32 || g_tune_nb == 64) return g_tune_nb;
  TuneEntry e;
  if (tune_lookup(m, n, &e)) return e.nb;
  return n <= 256 ? 32 : 64;
}

static int split_count(int M, int ntiles, int num_sms) {
  const int slots = 3 * num_sms;
  int S = (4 * slots + ntiles - 1) / ntiles;
  int maxS = std::max(1, M / 64);
  return std::max(1, std::min(S, maxS));
}

// Upper bound of the partial-sum workspace over every trailing width N' <= N:
// S * N' <= (4 * slots / ntiles' + 1) * ntiles' * kBN <= (4 * slots + ntiles) * kBN.
size_t panel_update_work_doubles(int m, int N, int nb, int num_sms) {
  (void)m;
  size_t ntiles = (size_t)(N + kBN - 1) / kBN;
  size_t slots = 3 * (size_t)num_sms;
  return (4 * slots + ntiles + 1) * kBN * nb + (size_t)nb * N;
}

// Partial slice 0 of W = V^T X over the top 64 rows of a panel (where V is
// the Vtop triangle), on the FP32 FMA pipe; the tensor-core kernel does the
// remaining rows.
static void vtop_part_f32(const float *A, int lda, const double *Vtop, int k0, int rows,
                          const float *X, int ldx, int N, float *Wp, cudaStream_t stream) {
  gemm_vtx_f32_kernel<<<dim3((N + kBN - 1) / kBN, 1), kThreads, 0, stream>>>(
      A, lda, Vtop, k0, 64, rows, X, ldx, N, rows, Wp, 0);
}

// lookahead: the update of the next panel's columns only (FP32: on the FMA
// pipe, three short launches instead of the tensor-core chain, and no BF16
// shadows to refresh: those columns are split again once they are factored)
template <typename T, int NB, bool TRANS = true>
static slqr_status panel_update_impl(slqr_ctx *ctx, int m, int k0, int nbw, const T *A, int lda,
                                     const double *wy_panel, T *X, int ldx, int N, T *work,
                                     size_t work_elems, cudaStream_t stream, int skip = 0,
                                     bool lookahead = false) {
  if (N <= 0) return SLQR_OK;
  const int M = m - k0 - skip;                     // rows of the panel (row map: panel_row)
  const int ntiles = (N + kBN - 1) / kBN;
  const int S = split_count(M, ntiles, ctx->num_sms);
  int RS = (M + S - 1) / S;
  RS = (RS + kBK - 1) / kBK * kBK;
  const int Seff = (M + RS - 1) / RS;
  if ((size_t)Seff * N * NB + (size_t)NB * N > work_elems)
    return fail(ctx, SLQR_ENOMEM, "internal: trailing-update workspace too small");
  T *Wp = work;
  T *Wt = work + (size_t)Seff * N * NB;
  const double *Vtop = wy_panel;
  const double gemm_flops = 2.0 * M * nbw * (double)N;
  int slot = prof_begin(ctx, stream);
  int slices = 0;
  bool tc = false;
  // tensor-core mode of an FP32 factorization (0 FMA, 1 TF32, 2 BF16 hi + lo)
  const int mode = (std::is_same<T, float>::value && !lookahead) ? ctx->tc_mode : 0;
  // BF16 mode: an update done on the FMA pipe refreshes the shadows it changed
  auto refresh_shadows = [&]() {
    if constexpr (std::is_same<T, float>::value) {
      if (ctx->tc_mode == 2 && !lookahead && ldx == lda && X >= A + (size_t)lda * (k0 + nbw)) {
        const int xcol0 = (int)((X - A) / lda);
        split_bf16_region((const float *)A, lda, k0, m, xcol0, xcol0 + N, ctx->sh_hi, ctx->sh_lo,
                          ctx->num_sms, stream);
      }
    }
  };
  // the FMA-pipe products (FP32 panels of width 64: the 16-byte-load forms)
  auto launch_vtx_fma = [&](int S_, int RS_) {
    if constexpr (std::is_same<T, float>::value && NB == 64)
      gemm_vtx_f32_kernel<<<dim3(ntiles, S_), kThreads, 0, stream>>>(A, lda, Vtop, k0, nbw, M, X,
                                                                      ldx, N, RS_, Wp, skip);
    else
      gemm_vtx_kernel<T, NB, false><<<dim3(ntiles, S_), kThreads, 0, stream>>>(
          A, lda, Vtop, k0, nbw, M, X, ldx, N, RS_, Wp, skip);
  };
  auto launch_upd_fma = [&](const T *Wt_) {
    if constexpr (std::is_same<T, float>::value && NB == 64) {
      const int vec = (ldx % 4 == 0 && ((uintptr_t)X & 15) == 0 && k0 % 4 == 0 && skip % 4 == 0 &&
                       nbw % 4 == 0) ? 1 : 0;
      gemm_upd_f32_kernel<<<dim3((M + kBM - 1) / kBM, ntiles), kThreads, 0, stream>>>(
          A, lda, Vtop, k0, nbw, M, X, ldx, N, Wt_, skip, vec);
    } else {
      gemm_upd_kernel<T, NB><<<dim3((M + kBM - 1) / kBM, ntiles), kThreads,
                               (size_t)NB * (kBM + kBN) * sizeof(T), stream>>>(
          A, lda, Vtop, k0, nbw, M, X, ldx, N, Wt_, skip);
    }
  };
  if constexpr (std::is_same<T, float>::value && NB == 64) {
    // tensor-core path: both products on the tensor cores for a full panel
    // whose X lies in A (the factorization); W'^T and a row-major V follow
    // the partials
    if (mode != 0 && TRANS && skip == 0 && nbw == 64 && ldx == lda &&
        X >= A + (size_t)lda * (k0 + nbw)) {
      const int xcol0 = (int)((X - A) / lda);
      if (mode == 2)
        slices = launch_vtx_bf16(A, lda, ctx->sh_hi, ctx->sh_lo, Vtop, k0, M, xcol0, N, Wp,
                                 work_elems, ctx->num_sms, ctx->d_status, stream, &vtop_part_f32);
      else
        slices = launch_vtx_tc(A, lda, Vtop, k0, M, xcol0, N, Wp, work_elems, ctx->num_sms,
                               ctx->d_status, stream, &vtop_part_f32);
      if (slices > 0) {
        Wt = work + (size_t)slices * N * NB;
        // scratch after W'^T: the row-major V (TF32), or the hi / lo pairs of V and W'
        const size_t scratch = (mode == 2) ? (size_t)(M + N) * NB : (size_t)M * NB;
        tc = (size_t)slices * N * NB + (size_t)NB * N + scratch <= work_elems;
        if (!tc) {                                  // partials only: finish on the FMA pipe
          prof_end(ctx, stream, slot, kVtx, gemm_flops);
          slot = prof_begin(ctx, stream);
          launch_tw<T, NB, TRANS>(Wp, slices, N, wy_panel, nbw, Wt, stream);
          prof_end(ctx, stream, slot, kTw, (double)nbw * nbw * N);
          slot = prof_begin(ctx, stream);
          launch_upd_fma(Wt);
          refresh_shadows();
          prof_end(ctx, stream, slot, kUpd, gemm_flops);
          return check_launch(ctx, "trailing update");
        }
      }
    }
  }
  if (slices == 0) {
    slices = Seff;
    launch_vtx_fma(Seff, RS);
  }
  prof_end(ctx, stream, slot, kVtx, gemm_flops);
  slot = prof_begin(ctx, stream);
  if (tc) launch_tw<T, NB, TRANS, true>(Wp, slices, N, wy_panel, nbw, Wt, stream);
  else launch_tw<T, NB, TRANS>(Wp, slices, N, wy_panel, nbw, Wt, stream);
  prof_end(ctx, stream, slot, kTw, (double)nbw * nbw * N);
  slot = prof_begin(ctx, stream);
  bool done = false;
  if constexpr (std::is_same<T, float>::value) {
    if (tc) {
      const int xcol0 = (int)((X - A) / lda);
      if (mode == 2)
        done = launch_upd_bf16((const float *)A, lda, ctx->sh_hi, ctx->sh_lo, Vtop, k0, M, xcol0,
                               N, (const float *)Wt, (void *)(Wt + (size_t)NB * N), ctx->num_sms,
                               ctx->d_status, stream);
      else
        done = launch_upd_tc((const float *)A, lda, Vtop, k0, M, xcol0, N, (const float *)Wt,
                             (float *)(Wt + (size_t)NB * N), ctx->d_status, stream);
      if (!done)                                    // no tensor map: W' again in FMA layout
        launch_tw<T, NB, TRANS>(Wp, slices, N, wy_panel, nbw, Wt, stream);
    }
  }
  if (!done) {
    launch_upd_fma(Wt);
    refresh_shadows();
  }
  prof_end(ctx, stream, slot, kUpd, gemm_flops);
  return check_launch(ctx, "trailing update");
}

slqr_status apply_panel_update(slqr_ctx *ctx, int m, int k0, int nbw, int nb, const double *A,
                               int lda, const double *wy_panel, double *X, int ldx, int N,
                               double *work, size_t work_doubles, cudaStream_t stream, int skip) {
  if (nb == 32)
    return panel_update_impl<double, 32>(ctx, m, k0, nbw, A, lda, wy_panel, X, ldx, N, work,
                                         work_doubles, stream, skip);
  return panel_update_impl<double, 64>(ctx, m, k0, nbw, A, lda, wy_panel, X, ldx, N, work,
                                       work_doubles, stream, skip);
}

// Opt the kernels that use more than 48 KB of dynamic shared memory in; run
// once per device (slqr_create) with that device current.
slqr_status init_kernel_attrs(slqr_ctx *ctx) {
  const int max_smem = 200 * 1024;
  cudaError_t e = cudaSuccess;
  e = cudaFuncSetAttribute(panel_kernel<double, 32, kSmallPanelCtas>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(panel_kernel<double, 32, kMaxPanelCtas>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(panel_kernel<double, 64, kSmallPanelCtas>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(panel_kernel<double, 64, kMaxPanelCtas>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(panel_kernel<float, 32, kSmallPanelCtas>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(panel_kernel<float, 32, kMaxPanelCtas>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(panel_kernel<float, 64, kSmallPanelCtas>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(panel_kernel<float, 64, kMaxPanelCtas>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_upd_kernel<double, 64>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * (kBM + kBN) * 8);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_upd_kernel<double, 32>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 32 * (kBM + kBN) * 8);
  if (e != cudaSuccess)
    return fail(ctx, SLQR_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
  return SLQR_OK;
}

// rows per CTA of the panel kernel
// Rows per panel CTA: at least the tuning minimum, and enough that the panel
// fits the small-grid kernel (at most 64 CTAs, fewer registers) whenever the
// slice still fits shared memory (max_rows).
static int panel_rows_per_cta(int M, int nbw, int num_sms, int max_rows, int rows_min,
                              size_t elem = sizeof(double)) {
  const int ctas = std::min(num_sms, kMaxPanelCtas);
  int R = (M + ctas - 1) / ctas;
  R = std::max(R, nbw);
  R = std::max(R, rows_min > 0 ? rows_min : rows_min_auto(M, elem));
  const int r_small = (M + kSmallPanelCtas - 1) / kSmallPanelCtas;
  if (r_small <= max_rows) R = std::max(R, r_small);
  return R;
}

template <typename T, int NB>
static const void *panel_kernel_for(int P) {
  return P <= kSmallPanelCtas ? (const void *)panel_kernel<T, NB, kSmallPanelCtas>
                              : (const void *)panel_kernel<T, NB, kMaxPanelCtas>;
}

static int max_rows_per_cta(int nb, size_t elem = sizeof(double)) {
  return (200 * 1024 - nb * nb * (int)sizeof(double) - 16) / (nb * (int)elem);
}

// dynamic shared memory of the panel kernel: the slice (T) then the local
// Gram terms (double), 16-byte aligned
static size_t panel_smem_bytes(int nb, int R, size_t elem) {
  return ((size_t)nb * R * elem + 15) / 16 * 16 + (size_t)nb * nb * sizeof(double);
}

// ntop > 0: A = [L^T; C] with an upper-triangular top block of ntop = n rows
// (the structure-aware factorization: each panel skips the zero rows between
// its diagonal block and C).
template <typename T, int NB>
static slqr_status factor_impl(slqr_ctx *ctx, int m, int n, T *A, int lda, double *up,
                               double *wy, cudaStream_t stream, int ntop = 0) {
  const int K = num_reflectors(m, n);
  auto skip_of = [&](int k0, int nbw) { return ntop > 0 ? ntop - (k0 + nbw) : 0; };
  const int np = num_panels(K, NB);
  const int rmin = rows_min_for(m, n);
  // workspace: [bar (256 B)] [records] [scale records] [Gram partials] [prow]
  // [wy if none given] [trailing work]
  const int Pmax = ctx->num_sms;
  const size_t rec_doubles = (size_t)NB * NB * Pmax;
  const size_t srec_doubles = (size_t)NB * Pmax;
  const size_t gpart_doubles = (size_t)Pmax * NB * (NB - 1) / 2;
  const size_t prow_doubles = (size_t)NB * NB;
  const size_t wy_doubles = wy ? 0 : wy_panel_doubles(NB) * (size_t)std::max(np, 1);
  // (the FP32 path also keeps a row-major copy of V for the tensor-core update)
  // (the FP32 path also keeps a row-major V, or the BF16 pairs of V and W')
  const size_t work_doubles = panel_update_work_doubles(m, n, NB, ctx->num_sms) +
                              (std::is_same<T, float>::value ? (size_t)(m + n) * NB : 0);
  const size_t bytes = 256 +
                       (rec_doubles + srec_doubles + gpart_doubles + prow_doubles + wy_doubles) * 8 +
                       work_doubles * sizeof(T) + 256;
  slqr_status st = ensure_workspace(ctx, bytes);
  if (st != SLQR_OK) return st;
  char *base = (char *)ctx->ws.ptr;
  unsigned *bar = (unsigned *)base;
  double *rec = (double *)(base + 256);
  double *srec = rec + rec_doubles;
  double *gpart = srec + srec_doubles;
  double *prow = gpart + gpart_doubles;
  double *wy_store = wy ? wy : prow + prow_doubles;
  // 256-byte aligned (vector stores and TMA maps of the trailing update)
  T *work = (T *)align_up((size_t)(prow + prow_doubles + wy_doubles), 256);

  cudaError_t e = cudaMemsetAsync(bar, 0, 256, stream);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  // up[k] for k >= K is 0 (no reflector)
  if (n > K) {
    e = cudaMemsetAsync(up + K, 0, sizeof(double) * (n - K), stream);
    if (e != cudaSuccess)
      return fail(ctx, SLQR_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  }
  if (np == 0) return SLQR_OK;

  // Look-ahead: after panel p, the columns of panel p+1 are updated first;
  // panel p+1 is then factored while the rest of the trailing update of
  // panel p runs on the other stream (the GPU form of running the critical
  // path T_{i,i} early).
  cudaStream_t aux = ctx->aux_stream;
  unsigned bar_base = 0;
  auto launch_panel = [&](int pnl, cudaStream_t s) -> slqr_status {
    const int k0 = pnl * NB;
    const int nbw = std::min(NB, K - k0);
    const int skip = skip_of(k0, nbw);
    const int M = m - k0 - skip;
    // algorithmic flops of the panel: per column j a norm over M-j entries and,
    // for each later panel column, a dot and an axpy over M-j entries
    double pflops = 0.0;
    for (int j = 0; j < nbw; ++j) pflops += 2.0 * (M - j) * (1 + 2 * (nbw - 1 - j));
    const int cs = panel_cluster_ctas(ctx, std::is_same<T, float>::value, NB, M, nbw);
    if (cs > 0) {
      ClusterPanelParams cp;
      cp.A = A; cp.up = up; cp.wy = wy_store + (size_t)pnl * wy_panel_doubles(NB);
      cp.m = m; cp.lda = lda; cp.k0 = k0; cp.nbw = nbw; cp.skip = skip; cp.stacked = ntop > 0;
      cp.R = std::max(nbw, (M + cs - 1) / cs);
      cp.status = ctx->d_status; cp.spin = ctx->spin_limit;
      int slot = prof_begin(ctx, s);
      slqr_status cst = launch_cluster_panel(ctx, std::is_same<T, float>::value, NB, cp, cs, s);
      prof_end(ctx, s, slot, kPanel, pflops);
      if (cst != SLQR_OK) return cst;
      if constexpr (std::is_same<T, float>::value) {
        if (ctx->tc_mode == 2)
          split_bf16_region((const float *)A, lda, k0, m, k0, k0 + nbw, ctx->sh_hi, ctx->sh_lo,
                            ctx->num_sms, s);
      }
      return SLQR_OK;                             // (no grid barrier used)
    }
    const int R = panel_rows_per_cta(M, nbw, Pmax, max_rows_per_cta(NB, sizeof(T)), rmin,
                                     sizeof(T));
    if (R > max_rows_per_cta(NB, sizeof(T)))
      return fail(ctx, SLQR_EINVAL, "m = %d is too large for the shared-memory panel", m);
    const int P = (M + R - 1) / R;
    double *wy_panel = wy_store + (size_t)pnl * wy_panel_doubles(NB);
    PanelParams pp;
    pp.A = A; pp.up = up; pp.wy = wy_panel; pp.rec = rec; pp.srec = srec; pp.gpart = gpart;
    pp.prow = prow; pp.bar = bar;
    pp.status = ctx->d_status; pp.m = m; pp.lda = lda; pp.k0 = k0; pp.nbw = nbw;
    pp.skip = skip; pp.stacked = ntop > 0; pp.P = P; pp.R = R; pp.bar_base = bar_base;
    pp.spin = ctx->spin_limit;
    void *args[] = {&pp};
    size_t smem = panel_smem_bytes(NB, R, sizeof(T));
    int slot = prof_begin(ctx, s);
    cudaError_t le = cudaLaunchCooperativeKernel(panel_kernel_for<T, NB>(P), dim3(P),
                                                 dim3(kThreads), args, smem, s);
    prof_end(ctx, s, slot, kPanel, pflops);
    if (le != cudaSuccess)
      return fail(ctx, SLQR_ECUDA, "panel launch (P=%d, smem=%zu): %s", P, smem,
                  cudaGetErrorString(le));
    if constexpr (std::is_same<T, float>::value) {
      // BF16 mode: the panel's columns (the reflectors) into the shadows
      if (ctx->tc_mode == 2)
        split_bf16_region((const float *)A, lda, k0, m, k0, k0 + nbw, ctx->sh_hi, ctx->sh_lo,
                          ctx->num_sms, s);
    }
    bar_base += 2u * (unsigned)P;                 // two grid barriers per panel
    return SLQR_OK;
  };
  // the fused look-ahead kernel's grid barriers count on their own counter
  // (bar[32], another cache line than the panels' bar[0])
  unsigned la_base = 0;
  auto update = [&](int pnl, int c_begin, int c_end, bool lookahead,
                    cudaStream_t us) -> slqr_status {
    const int k0 = pnl * NB;
    const int nbw = std::min(NB, K - k0);
    if (c_end <= c_begin) return SLQR_OK;
    if constexpr (std::is_same<T, float>::value && NB == 64) {
      slqr_status lst = SLQR_OK;
      if (lookahead && ntop == 0 &&
          lookahead_update_f32(ctx, m, k0, nbw, A, lda,
                               wy_store + (size_t)pnl * wy_panel_doubles(NB), c_begin,
                               c_end - c_begin, work, work_doubles, bar + 32, la_base, us,
                               &lst))
        return lst;
    }
    return panel_update_impl<T, NB>(ctx, m, k0, nbw, A, lda,
                                 wy_store + (size_t)pnl * wy_panel_doubles(NB),
                                 A + (size_t)c_begin * lda, lda, c_end - c_begin, work,
                                 work_doubles, us, skip_of(k0, nbw), lookahead);
  };
  // order the auxiliary stream after everything already on the caller's stream
  e = cudaEventRecord(ctx->ev_start, stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ctx->ev_start, 0);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "event: %s", cudaGetErrorString(e));
  st = launch_panel(0, stream);
  if (st != SLQR_OK) return st;
  // FP64: the panels on the auxiliary stream, the updates (the longer chain)
  // back to back on the caller's stream.  FP32: the panels (the longer chain)
  // right behind the look-ahead on the caller's stream, so that a panel is
  // never queued behind the first kernel of the rest of the update and has
  // its SMs before the update fills the GPU, and the rest of each update on
  // the auxiliary stream.
  constexpr bool kPanelsOnCaller = std::is_same<T, float>::value;
  for (int pnl = 0; pnl < np; ++pnl) {
    const int k0 = pnl * NB;
    const int nbw = std::min(NB, K - k0);
    const int c0 = k0 + nbw;                       // first trailing column
    if (pnl + 1 < np) {
      const int next_w = std::min(NB, K - (k0 + NB));
      st = update(pnl, c0, c0 + next_w, true, stream);   // columns of panel p+1
      if (st != SLQR_OK) return st;
      e = cudaEventRecord(ctx->ev_ready, stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ctx->ev_ready, 0);
      if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "event: %s", cudaGetErrorString(e));
      if (kPanelsOnCaller) {
        // rest of the update of panel p (aux) || panel p+1 (caller's stream)
        st = update(pnl, c0 + next_w, n, false, aux);
        if (st != SLQR_OK) return st;
        e = cudaEventRecord(ctx->ev_panel, aux);
        if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "event: %s", cudaGetErrorString(e));
        st = launch_panel(pnl + 1, stream);
        if (st != SLQR_OK) return st;
        e = cudaStreamWaitEvent(stream, ctx->ev_panel, 0);
      } else {
        st = launch_panel(pnl + 1, aux);
        if (st != SLQR_OK) return st;
        e = cudaEventRecord(ctx->ev_panel, aux);
        if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "event: %s", cudaGetErrorString(e));
        st = update(pnl, c0 + next_w, n, false, stream);  // concurrently with the panel
        if (st != SLQR_OK) return st;
        e = cudaStreamWaitEvent(stream, ctx->ev_panel, 0);
      }
      if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "event: %s", cudaGetErrorString(e));
    } else {
      st = update(pnl, c0, n, false, stream);
      if (st != SLQR_OK) return st;
    }
  }
  return check_launch(ctx, "factor");
}

slqr_status factor_f32(slqr_ctx *ctx, int m, int n, float *A, int lda, double *up, double *wy,
                       cudaStream_t stream, int ntop) {
  if (panel_width(m, n) == 32)
    return factor_impl<float, 32>(ctx, m, n, A, lda, up, wy, stream, ntop);
  return factor_impl<float, 64>(ctx, m, n, A, lda, up, wy, stream, ntop);
}


}  // namespace slqr

using namespace slqr;

extern "C" int slqr_panel_width(int m, int n) { return panel_width(m, n); }

extern "C" void slqr_set_tuning(int panel_width, int panel_rows_min) {
  g_tune_nb = (panel_width == 32 || panel_width == 64) ? panel_width : 0;
  g_tune_rows_min = panel_rows_min > 0 ? std::min(panel_rows_min, 1024) : 0;
  if (g_tune_nb == 0 && g_tune_rows_min == 0) {      // back to the defaults
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache.clear();
  }
}

extern "C" slqr_status slqr_set_panel_cluster(int ctas) {
  if (!(ctas == 0 || ctas == -1 || (ctas >= 1 && ctas <= kClusterMaxCtas))) return SLQR_EINVAL;
  g_panel_cluster = ctas;
  return SLQR_OK;
}

extern "C" int slqr_get_panel_cluster(void) { return g_panel_cluster; }

namespace slqr {
int panel_cluster_setting() { return g_panel_cluster; }
}  // namespace slqr

extern "C" slqr_status slqr_set_panel_cluster_variant(int variant) {
  if (variant < 0 || variant > 3) return SLQR_EINVAL;
  set_cluster_panel_variant(variant);
  return SLQR_OK;
}

namespace slqr {

// Deterministic scratch matrix for the autotuner: entries in (-1, 1) from a
// hash of the index (the timing does not depend on the values, only on their
// being generic).
__global__ void tune_fill_kernel(double *A, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x) {
    unsigned long long h = (i + 1) * 0x9E3779B97F4A7C15ull;
    h ^= h >> 31;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 27;
    A[i] = (double)(h >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

}  // namespace slqr

extern "C" slqr_status slqr_autotune(slqr_ctx *ctx, int m, int n, double *best_ms,
                                     int *best_panel_width, int *best_rows_min) {
  NvtxRange nvtx_range("slqr_autotune");
  if (!ctx) return SLQR_EINVAL;
  if (m < 1 || n < 1 || m < n || m > slqr_max_rows())
    return fail(ctx, SLQR_EINVAL, "autotune: need 1 <= n <= m <= %d (m=%d n=%d)", slqr_max_rows(),
                m, n);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  // measure without a previous entry for this shape (candidate 0 is "by panel height")
  TuneEntry old_entry;
  bool had_entry = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find({m, n});
    if (it != g_tune_cache.end()) {
      old_entry = it->second;
      had_entry = true;
      g_tune_cache.erase(it);
    }
  }
  const size_t count = (size_t)m * n;
  double *A0 = nullptr, *A = nullptr, *up = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&A0, count * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&A, count * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&up, (size_t)n * sizeof(double));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  auto cleanup = [&]() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(A0);
    cudaFree(A);
    cudaFree(up);
  };
  if (e != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    if (had_entry) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_cache[{m, n}] = old_entry;
    }
    return fail(ctx, SLQR_ENOMEM, "autotune scratch: %s", cudaGetErrorString(e));
  }
  tune_fill_kernel<<<4 * ctx->num_sms, 256, 0, s>>>(A0, count);
  const int saved_nb = g_tune_nb, saved_rows = g_tune_rows_min;
  const int widths[2] = {32, 64};
  const int rows[6] = {0, 64, 96, 128, 192, 256};
  double best = 1e300;
  int bw = 0, br = 0;
  slqr_status st = SLQR_OK;
  for (int wi = 0; wi < 2 && st == SLQR_OK; ++wi) {
    if (widths[wi] == 64 && n <= 32) continue;      // one panel either way
    for (int ri = 0; ri < 6 && st == SLQR_OK; ++ri) {
      g_tune_nb = widths[wi];
      g_tune_rows_min = rows[ri];
      float ms_min = 1e30f;
      for (int rep = 0; rep < 2 && st == SLQR_OK; ++rep) {
        cudaMemcpyAsync(A, A0, count * sizeof(double), cudaMemcpyDeviceToDevice, s);
        cudaEventRecord(e0, s);
        st = slqr_factor(ctx, m, n, A, m, up, nullptr, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = SLQR_ECUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms_min = std::min(ms_min, ms);
      }
      if (st == SLQR_EINVAL) {                      // setting outside the kernel limits
        st = SLQR_OK;
        continue;
      }
      if (st == SLQR_OK && ms_min < best) {
        best = ms_min;
        bw = widths[wi];
        br = rows[ri];
      }
    }
  }
  cleanup();
  g_tune_nb = saved_nb;
  g_tune_rows_min = saved_rows;
  if (st != SLQR_OK || best >= 1e300) {
    if (had_entry) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_cache[{m, n}] = old_entry;
    }
    return st != SLQR_OK ? st : fail(ctx, SLQR_ECUDA, "autotune: no setting ran");
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[{m, n}] = TuneEntry{bw, br};
  }
  if (best_ms) *best_ms = best;
  if (best_panel_width) *best_panel_width = bw;
  if (best_rows_min) *best_rows_min = br;
  return SLQR_OK;
}

extern "C" size_t slqr_wy_size(int m, int n) {
  if (m <= 0 || n <= 0) return 0;
  int nb = panel_width(m, n);
  int K = num_reflectors(m, n);
  return wy_panel_doubles(nb) * (size_t)num_panels(K, nb) * sizeof(double);
}

extern "C" int slqr_max_rows(void) { return 49152; }

extern "C" slqr_status slqr_factor(slqr_ctx *ctx, int m, int n, double *A, int lda, double *up,
                                   double *wy, void *stream) {
  NvtxRange nvtx_range("slqr_factor");
  if (!ctx) return SLQR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (m < 0 || n < 0 || m < n) return fail(ctx, SLQR_EINVAL, "need m >= n >= 0 (m=%d n=%d)", m, n);
  if (n == 0) return SLQR_OK;
  if (lda < std::max(1, m)) return fail(ctx, SLQR_EINVAL, "lda=%d < m=%d", lda, m);
  if (!A || !up) return fail(ctx, SLQR_EINVAL, "NULL A or up");
  if (m > slqr_max_rows()) return fail(ctx, SLQR_EINVAL, "m=%d above slqr_max_rows()", m);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  cudaStream_t s = (cudaStream_t)stream;
  if (panel_width(m, n) == 32) return factor_impl<double, 32>(ctx, m, n, A, lda, up, wy, s);
  return factor_impl<double, 64>(ctx, m, n, A, lda, up, wy, s);
}

extern "C" slqr_status slqr_factor_stacked(slqr_ctx *ctx, int n, int m_eq, double *A, int lda,
                                           double *up, double *wy, void *stream) {
  NvtxRange nvtx_range("slqr_factor_stacked");
  if (!ctx) return SLQR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (n < 0 || m_eq < 0) return fail(ctx, SLQR_EINVAL, "need n, m_eq >= 0 (n=%d m_eq=%d)", n, m_eq);
  if (n == 0) return SLQR_OK;
  const int m = n + m_eq;
  if (lda < m) return fail(ctx, SLQR_EINVAL, "lda=%d < n + m_eq=%d", lda, m);
  if (!A || !up) return fail(ctx, SLQR_EINVAL, "NULL A or up");
  if (m > slqr_max_rows()) return fail(ctx, SLQR_EINVAL, "m=%d above slqr_max_rows()", m);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  cudaStream_t s = (cudaStream_t)stream;
  if (panel_width(m, n) == 32) return factor_impl<double, 32>(ctx, m, n, A, lda, up, wy, s, n);
  return factor_impl<double, 64>(ctx, m, n, A, lda, up, wy, s, n);
}

// ==========================================================================
// slqr_factor_noalloc: the same factorization for callers that cannot
// allocate device memory.  Its scratch (barrier counter, reduction records,
// compact-WY store, partial sums) lives in one file-scope __device__ array of
// fixed size instead of a context workspace.  It has no counterpart in the
// paper.
// ==========================================================================
namespace slqr {

constexpr int kNoAllocMaxRows = 8192;
constexpr int kNoAllocMaxCols = 1024;
constexpr int kNoAllocMaxSms = 256;
constexpr int kNoAllocMaxDevices = 64;
constexpr size_t kNoAllocHeadDoubles = 32;                       // 256 B: counter + status
constexpr size_t kNoAllocRecDoubles = (size_t)64 * 64 * kMaxPanelCtas;
constexpr size_t kNoAllocSrecDoubles = (size_t)64 * kMaxPanelCtas;
constexpr size_t kNoAllocGpartDoubles = (size_t)kMaxPanelCtas * 64 * 63 / 2;
constexpr size_t kNoAllocProwDoubles = 64 * 64;
constexpr size_t kNoAllocWyDoubles = (kNoAllocMaxCols / 64) * (2 * 64 * 64 + 64);
constexpr size_t kNoAllocWorkDoubles = 384 * 1024;
constexpr size_t kNoAllocScratchDoubles = kNoAllocHeadDoubles + kNoAllocRecDoubles +
                                          kNoAllocSrecDoubles + kNoAllocGpartDoubles +
                                          kNoAllocProwDoubles +
                                          kNoAllocWyDoubles + kNoAllocWorkDoubles;

// kNoAllocScratchDoubles doubles, about 12.1 MB, on every device that loads the
// library, held until exit.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

static std::mutex g_noalloc_mu;
static double *g_noalloc_ptr[kNoAllocMaxDevices];
static int g_noalloc_sms[kNoAllocMaxDevices];

// Once per device, with that device current: the device address of the
// scratch array (its name in host code is only a host-side stand-in) and the
// shared-memory opt-in of the kernels.
static slqr_status noalloc_setup(int dev, double **ptr, int *sms) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_ptr[dev]) {
    *ptr = g_noalloc_ptr[dev];
    *sms = g_noalloc_sms[dev];
    return SLQR_OK;
  }
  double *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return SLQR_ECUDA;
  }
  int n_sms = 0;
  e = cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess || n_sms <= 0 || n_sms > kNoAllocMaxSms) {
    cudaGetLastError();
    return SLQR_ECUDA;
  }
  const int max_smem = 200 * 1024;
  e = cudaFuncSetAttribute(panel_kernel<double, 32, kSmallPanelCtas>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(panel_kernel<double, 32, kMaxPanelCtas>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(panel_kernel<double, 64, kSmallPanelCtas>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(panel_kernel<double, 64, kMaxPanelCtas>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(panel_kernel<float, 32, kSmallPanelCtas>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(panel_kernel<float, 32, kMaxPanelCtas>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(panel_kernel<float, 64, kSmallPanelCtas>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(panel_kernel<float, 64, kMaxPanelCtas>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_upd_kernel<double, 64>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * (kBM + kBN) * 8);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_upd_kernel<double, 32>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 32 * (kBM + kBN) * 8);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SLQR_ECUDA;
  }
  g_noalloc_ptr[dev] = p;
  g_noalloc_sms[dev] = n_sms;
  *ptr = p;
  *sms = n_sms;
  return SLQR_OK;
}

// Trailing update with the row-split count capped so the partial sums fit
// the fixed scratch.
template <int NB>
static slqr_status noalloc_update(int num_sms, int m, int k0, int nbw, const double *A, int lda,
                                  const double *wy_panel, double *X, int ldx, int N,
                                  double *work, size_t work_doubles, cudaStream_t stream) {
  const int M = m - k0;
  const int ntiles = (N + kBN - 1) / kBN;
  int S = split_count(M, ntiles, num_sms);
  const long long maxS = ((long long)(work_doubles / NB) - N) / N;
  if (maxS < 1) return SLQR_EINVAL;
  S = (int)std::max(1LL, std::min((long long)S, maxS));
  int RS = (M + S - 1) / S;
  RS = (RS + kBK - 1) / kBK * kBK;
  const int Seff = (M + RS - 1) / RS;
  if ((size_t)Seff * N * NB + (size_t)NB * N > work_doubles) return SLQR_EINVAL;
  double *Wp = work;
  double *Wt = work + (size_t)Seff * N * NB;
  gemm_vtx_kernel<double, NB, false><<<dim3(ntiles, Seff), kThreads, 0, stream>>>(
      A, lda, wy_panel, k0, nbw, M, X, ldx, N, RS, Wp);
  launch_tw<double, NB, true>(Wp, Seff, N, wy_panel, nbw, Wt, stream);
  size_t smem = (size_t)NB * (kBM + kBN) * sizeof(double);
  gemm_upd_kernel<double, NB><<<dim3((M + kBM - 1) / kBM, ntiles), kThreads, smem, stream>>>(
      A, lda, wy_panel, k0, nbw, M, X, ldx, N, Wt);
  return cudaGetLastError() == cudaSuccess ? SLQR_OK : SLQR_ECUDA;
}

template <int NB>
static slqr_status noalloc_factor_impl(double *scratch, int num_sms, int m, int n, double *A,
                                       int lda, double *up, double *wy, int *status,
                                       cudaStream_t stream) {
  const int K = num_reflectors(m, n);
  const int np = num_panels(K, NB);
  const int rmin = rows_min_for(m, n);
  unsigned *bar = (unsigned *)scratch;
  if (!status) status = (int *)(scratch + 16);
  double *rec = scratch + kNoAllocHeadDoubles;
  double *srec = rec + kNoAllocRecDoubles;
  double *gpart = srec + kNoAllocSrecDoubles;
  double *prow = gpart + kNoAllocGpartDoubles;
  double *wy_store = wy ? wy : prow + kNoAllocProwDoubles;
  double *work = prow + kNoAllocProwDoubles + kNoAllocWyDoubles;
  // the array keeps the previous call's contents: clear the counter and status
  cudaError_t e = cudaMemsetAsync(scratch, 0, kNoAllocHeadDoubles * sizeof(double), stream);
  if (e == cudaSuccess && n > K) e = cudaMemsetAsync(up + K, 0, sizeof(double) * (n - K), stream);
  if (e != cudaSuccess) return SLQR_ECUDA;
  unsigned bar_base = 0;
  for (int pnl = 0; pnl < np; ++pnl) {
    const int k0 = pnl * NB;
    const int nbw = std::min(NB, K - k0);
    const int M = m - k0;
    const int R = panel_rows_per_cta(M, nbw, num_sms, max_rows_per_cta(NB), rmin);
    if (R > max_rows_per_cta(NB)) return SLQR_EINVAL;
    const int P = (M + R - 1) / R;
    double *wy_panel = wy_store + (size_t)pnl * wy_panel_doubles(NB);
    PanelParams pp;
    pp.A = A; pp.up = up; pp.wy = wy_panel; pp.rec = rec; pp.srec = srec; pp.gpart = gpart;
    pp.prow = prow; pp.bar = bar;
    pp.status = status; pp.m = m; pp.lda = lda; pp.k0 = k0; pp.nbw = nbw;
    pp.skip = 0; pp.stacked = 0; pp.P = P; pp.R = R; pp.bar_base = bar_base;
    pp.spin = kSpinLimit;
    void *args[] = {&pp};
    size_t smem = panel_smem_bytes(NB, R, sizeof(double));
    e = cudaLaunchCooperativeKernel(panel_kernel_for<double, NB>(P), dim3(P), dim3(kThreads), args,
                                    smem, stream);
    if (e != cudaSuccess) return SLQR_ECUDA;
    bar_base += 2u * (unsigned)P;
    const int N = n - (k0 + nbw);
    if (N > 0) {
      slqr_status st = noalloc_update<NB>(num_sms, m, k0, nbw, A, lda, wy_panel,
                                          A + (size_t)(k0 + nbw) * lda, lda, N, work,
                                          kNoAllocWorkDoubles, stream);
      if (st != SLQR_OK) return st;
    }
  }
  return cudaGetLastError() == cudaSuccess ? SLQR_OK : SLQR_ECUDA;
}

}  // namespace slqr

extern "C" int slqr_noalloc_max_rows(void) { return kNoAllocMaxRows; }
extern "C" int slqr_noalloc_max_cols(void) { return kNoAllocMaxCols; }

extern "C" slqr_status slqr_factor_noalloc(int m, int n, double *A, int lda, double *up,
                                           double *wy, int *status, void *stream) {
  NvtxRange nvtx_range("slqr_factor_noalloc");
  if (m < 0 || n < 0 || m < n) return SLQR_EINVAL;
  if (n == 0) return SLQR_OK;
  if (m > kNoAllocMaxRows || n > kNoAllocMaxCols) return SLQR_EINVAL;
  if (lda < std::max(1, m) || !A || !up) return SLQR_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
    cudaGetLastError();
    return SLQR_ECUDA;
  }
  double *scratch = nullptr;
  int sms = 0;
  slqr_status st = noalloc_setup(dev, &scratch, &sms);
  if (st != SLQR_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (panel_width(m, n) == 32)
    return noalloc_factor_impl<32>(scratch, sms, m, n, A, lda, up, wy, status, s);
  return noalloc_factor_impl<64>(scratch, sms, m, n, A, lda, up, wy, status, s);
}
