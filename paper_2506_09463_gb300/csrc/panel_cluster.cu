// panel_cluster.cu -- the panel of NB columns factored by one thread-block
// cluster: the panel's rows are split over the cluster's CTAs (up to 16),
// each slice resident in its CTA's shared memory, and the per-column
// reductions travel through distributed shared memory.
//
// The arithmetic is that of the cooperative panel kernel of factor.cu (Alg. 2
// of the paper on one panel: per column the scaled norm, the sign rule and up
// of Alg. 3, then the reflector applied to the later panel columns), with the
// same power-of-two column scales and the same compact-WY outputs (Vtop, the
// Gram terms of V^T V, tau).  What changes is how a column step is organised:
//
//  * one pass over the slice per column: the pass of column j applies
//    reflector j-1 to the columns right of it and, in the same sweep over the
//    rows, forms the partial sums of column j (its scaled norm from the
//    pivot down, the dots of its tail with the later columns, the Gram terms
//    with the earlier ones).  The updated column j is computed by every warp
//    from the old column and reflector j-1 (one FMA), so no warp waits for
//    another within the pass; the warp that owns column j keeps the result in
//    a column buffer (three, by j mod 3) and writes it into the slice while
//    the next column's records travel;
//  * the partial sums are reduced within each warp by shuffles (a butterfly:
//    every lane ends with the same bits) into a per-CTA record, which is
//    pushed to every CTA of the cluster in 16-byte pieces with st.async
//    (only the live entries); each store also counts its bytes on the
//    receiver's mbarrier (double-buffered by column parity), so the receiver
//    waits on its own barrier and no CTA waits for the others' stores to
//    drain.  CTA 0 pushes the pivot row (updated first, at the start of the
//    column step) entry by entry, counted on the same barriers;
//  * every warp then sums the received records from its own shared memory in
//    a fixed lane order: every warp of every CTA computes the same pivot and
//    multipliers bit for bit.  An FP32 panel keeps this chain on the FP32
//    pipe (a column whose scale is extreme for FP32 forms its pivot in FP64).
//    The writes nothing waits for (the previous column's final copy into the
//    slice, the R entries of the previous pivot row) run while the records
//    travel.
//
// Waits are bounded: past the context's spin limit a wait records
// SLQR_ETIMEOUT once and keeps waiting up to a fixed limit, so that no store
// of the column is still in flight when the kernel moves on.  Every thread of
// every CTA reaches every barrier (the checked build's launch-invariant check
// returns from every CTA at once, before the first barrier), and all CTAs of
// a cluster are co-scheduled by the hardware.  FP32 panels of at most 16 x 512 rows use
// the register-resident variant of panel_cluster_reg.cu instead.
#include "cluster_common.cuh"

#include <type_traits>

namespace slqr {

using namespace cl;

template <typename T, int NB, int NWARPS>
__global__ void __launch_bounds__(NWARPS * 32, 1)
cluster_panel_kernel(ClusterPanelParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NW = NWARPS;
  constexpr int NT = NWARPS * 32;
  constexpr int CPW = NB / NW;                 // columns per warp: c = warp + t * NW
  static_assert(NB % NW == 0, "whole columns per warp");
  constexpr bool kF32 = std::is_same<T, float>::value;
  const int R = p.R;
  T *Ps = (T *)smem_raw;                       // [NB][R] column-major slice
  T *xb = Ps + (size_t)NB * R;                 // [3][R] column j by j % 3
  T *Gl = xb + (size_t)3 * R;                  // [NB][NB] local Gram terms (c < j at c + j NB)
  // records received from every CTA of the cluster, by column parity:
  // entry j the partial norm of column j, c > j the partial dot with column c
  __shared__ __align__(16) T s_recv[2][kClMaxCtas][NB];
  __shared__ __align__(16) T s_prow[2][NB];    // pivot row, pushed by CTA 0
  __shared__ __align__(16) T s_rec[2][2][NB];  // this CTA's record and (CTA 0) pivot row
  __shared__ unsigned s_mx[NB];                // column-scale exchange
  __shared__ int s_E[NB];
  __shared__ T s_upT[NB], s_rbT[NB];           // up and 1/b per column (FP32 pivots)
  __shared__ double s_upD[NB], s_rbD[NB];      // (FP64 pivots)
  __shared__ int s_fast[NB];
  __shared__ __align__(8) unsigned long long s_mbar[2];   // receive barriers, by column parity
  __shared__ int s_ok;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int q = cluster_rank(), CS = cluster_ctas();
  const int row0 = q * R;
  const int RO = max(0, min(R, p.m - p.k0 - p.skip - row0));   // rows owned
  const int nbw = p.nbw;
  T *A = (T *)p.A;
  const int lda = p.lda;
  // checked build: the launch's invariants (uniform: every CTA returns here
  // together, before any barrier)
  if (!slqr_check(CS <= kClMaxCtas && R >= nbw && nbw >= 1 && nbw <= NB &&
                      p.m - p.k0 - p.skip <= CS * R && lda >= p.m, p.status))
    return;

  for (int idx = tid; idx < NB * R; idx += NT) {
    const int c = idx / R, r = idx - c * R;
    // (stacked: the strictly lower part of the diagonal block is zero, not read)
    const bool zero = c >= nbw || r >= RO || (p.stacked && row0 + r < nbw && row0 + r > c);
    Ps[idx] = zero ? T(0) : A[SLQR_IDX(cpanel_row(p.k0, nbw, p.skip, row0 + r), p.k0 + c, lda)];
  }
  for (int idx = tid; idx < 3 * R + NB * NB; idx += NT) xb[idx] = T(0);   // (and Gl)
  __syncthreads();

  // Bytes every CTA receives for column j: each CTA's record from the piece
  // holding entry j to nbw (16-byte pieces of V entries), and CTA 0's pivot
  // row entries [j, nbw).
  constexpr int V = 16 / (int)sizeof(T);
  auto step_bytes = [&](int jj) -> unsigned {
    const int npc = (nbw - (jj & ~(V - 1)) + V - 1) / V;
    return (unsigned)(CS * npc * 16 + (nbw - jj) * (int)sizeof(T));
  };
  if (tid == 0) {
    mbar_init1(&s_mbar[0]);
    mbar_init1(&s_mbar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // the phases of columns 0 and 1; column j + 2's is announced once column
    // j's has completed (before this CTA pushes anything for column j + 1,
    // so no byte of column j + 2 can arrive first)
    if (nbw > 0) mbar_expect(&s_mbar[0], step_bytes(0));
    if (nbw > 1) mbar_expect(&s_mbar[1], step_bytes(1));
    s_ok = 1;
  }
  // the pushes: thread tid sends pieces tid / CS, + stride, ... to CTA tid % CS
  const int push_stride = NT / CS;
  const int push_dest = tid % CS, push_piece = tid < push_stride * CS ? tid / CS : NB;

  // ---- panel start: power-of-two column scales (max over the cluster) -------
#pragma unroll
  for (int t = 0; t < CPW; ++t) {
    const int c = warp + t * NW;
    unsigned mx = 0;
    if (c < nbw) {
      const int r_from = (q == 0) ? c : 0;
      for (int r = r_from + lane; r < RO; r += 32) mx = max(mx, abs_bits_hi(Ps[c * R + r]));
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) s_mx[c] = mx;
  }
  cluster_sync_all();
  if (tid < NB) {
    unsigned mx = 0;
    for (int r = 0; r < CS; ++r) mx = max(mx, cluster_ld_u32(cluster_addr(&s_mx[tid], r)));
    int E = (int)((mx >> 20) & 0x7ff) - 1023;          // exponent of the largest |entry|
    // (FP32: 2^-E and 2^E must both be normal floats)
    E = kF32 ? min(max(E, -126), 126) : min(max(E, -1000), 1022);
    s_E[tid] = E;
  }
  __syncthreads();

  // per-thread state carried from one column step to the next (the same in
  // every thread of the cluster, except sig: the multipliers of the warp's
  // own columns, 0 for every column left of the pivot)
  T sig[CPW];
#pragma unroll
  for (int t = 0; t < CPW; ++t) sig[t] = T(0);
  T sig_next = T(0);          // multiplier of column j (reflector j-1)
  T upT_prev = T(0), clT_prev = T(0);
  double upD_prev = 0.0, clD_prev = 0.0;
  bool def_prev = false, fast_prev = true;
  bool reported = false;      // this thread has recorded a wait past the spin limit

  for (int j = 0; j < nbw; ++j) {
    const int buf = j & 1;
    const bool upd = j > 0;                      // reflector j-1 to apply
    const T *xo_col = xb + (size_t)((j + 2) % 3) * R;   // column j-1 (zero before the first)
    T *xn_col = xb + (size_t)(j % 3) * R;        // column j, updated (written by its owner)
    const T *colj = Ps + (size_t)j * R;
    const int r_main = (q == 0) ? j + 1 : 0;     // rows strictly below the pivot
    const int Ej = s_E[j];
    const T sc = pow2_t<T>(-Ej);
    const bool owner_j = warp == (j % NW);
    // Every own column runs the same instructions in the pass: v = old +
    // sig * x_{j-1} (sig = 0 left of the pivot), then the dot with column j.
    // Columns right of the pivot store v back (the update); left of it the
    // dot is a Gram term (column j-1 read from the column buffer, its slice
    // copy being written one step later); column j's own and those past nbw
    // are ignored.
    const T *src[CPW];
    bool st_ok[CPW];
#pragma unroll
    for (int t = 0; t < CPW; ++t) {
      const int c = warp + t * NW;
      src[t] = (c == j - 1) ? xo_col : Ps + (size_t)c * R;
      st_ok[t] = upd && c > j && c < nbw;
    }
    T acc[CPW];
#pragma unroll
    for (int t = 0; t < CPW; ++t) acc[t] = T(0);
    T nacc = T(0);

    // ---- CTA 0: the pivot row j (row j updated by reflector j-1), pushed to
    // every CTA first; the pivot entry joins the norm -------------------------
    if (q == 0) {
      T pv[CPW];
      if (lane == (j & 31)) {
        const T xo = xo_col[j];
#pragma unroll
        for (int t = 0; t < CPW; ++t) {
          const int c = warp + t * NW;
          T *col = Ps + (size_t)c * R;
          const T v = fma_t(c == j ? sig_next : sig[t], xo, col[j]);
          pv[t] = v;
          if (st_ok[t]) col[j] = v;
          if (c == j) {
            const T xs = v * sc;
            nacc = fma_t(xs, xs, nacc);
          }
        }
      }
#pragma unroll
      for (int t = 0; t < CPW; ++t) {
        const int c = warp + t * NW;
        if (c >= j && c < nbw) {
          const T v = __shfl_sync(0xffffffffu, pv[t], j & 31);
          if (lane < CS)
            st_async1(cluster_addr(&s_prow[buf][c], lane), v, cluster_addr(&s_mbar[buf], lane));
        }
      }
    }

    // ---- the pass: rows strictly below the pivot (lane r % 32 owns row r) ---
    // U rows per lane per iteration, every load issued before any store
    constexpr int U = 4;
    for (int base = (r_main & ~31) + lane; base < RO; base += 32 * U) {
      bool ok[U];
      T xo[U], xn[U], v[CPW][U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int r = base + 32 * u;
        ok[u] = r >= r_main && r < RO;
        xo[u] = ok[u] ? xo_col[r] : T(0);
        xn[u] = ok[u] ? colj[r] : T(0);
      }
#pragma unroll
      for (int t = 0; t < CPW; ++t)
#pragma unroll
        for (int u = 0; u < U; ++u) v[t][u] = ok[u] ? src[t][base + 32 * u] : T(0);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        xn[u] = fma_t(sig_next, xo[u], xn[u]);
        const T xs = xn[u] * sc;
        nacc = fma_t(xs, xs, nacc);
      }
#pragma unroll
      for (int t = 0; t < CPW; ++t)
#pragma unroll
        for (int u = 0; u < U; ++u) {
          v[t][u] = fma_t(sig[t], xo[u], v[t][u]);
          acc[t] = fma_t(xn[u], v[t][u], acc[t]);
        }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int r = base + 32 * u;
        if (ok[u] && owner_j) xn_col[r] = xn[u];
#pragma unroll
        for (int t = 0; t < CPW; ++t)
          if (ok[u] && st_ok[t]) Ps[(size_t)(warp + t * NW) * R + r] = v[t][u];
      }
    }
    // ---- warp sums (the butterfly leaves the same bits in every lane) ---------
#pragma unroll
    for (int t = 0; t < CPW; ++t) acc[t] = lanes_sum(acc[t]);
    if (owner_j) nacc = lanes_sum(nacc);
    if (lane == 0) {
#pragma unroll
      for (int t = 0; t < CPW; ++t) {
        const int c = warp + t * NW;
        if (c > j && c < nbw) s_rec[buf][0][c] = acc[t];
        else if (c < j) Gl[c + j * NB] = acc[t];
      }
      if (owner_j) s_rec[buf][0][j] = nacc;
    }
    __syncthreads();
    // this CTA's record pushed to every CTA of the cluster in 16-byte pieces,
    // only the live entries (from the piece holding j to nbw)
    {
      const int c0 = j & ~(V - 1);
      const int npc = (nbw - c0 + V - 1) / V;
      for (int pc = push_piece; pc < npc; pc += push_stride) {
        const int c = c0 + pc * V;
        st_async16(cluster_addr(&s_recv[buf][q][c], push_dest), &s_rec[buf][0][c],
                   cluster_addr(&s_mbar[buf], push_dest));
      }
    }

    // ---- while the records travel: the writes nothing waits for --------------
    if (upd) {
      // column j-1 is final: its tail from the column buffer (rows > j-1)
      if (warp == (j - 1) % NW) {
        T *col = Ps + (size_t)(j - 1) * R;
        const int r_from = (q == 0) ? j : 0;
        for (int r = (r_from & ~31) + lane; r < RO; r += 32)
          if (r >= r_from) col[r] = xo_col[r];
      }
      // CTA 0, row j-1 (the pivot row of reflector j-1): R entries of the
      // later columns, the diagonal entry cl of column j-1
      if (q == 0 && lane == ((j - 1) & 31)) {
#pragma unroll
        for (int t = 0; t < CPW; ++t) {
          const int c = warp + t * NW;
          T *col = Ps + (size_t)c * R;
          if (c < nbw && c >= j) {
            const T s = (c == j) ? sig_next : sig[t];
            if (fast_prev) col[j - 1] = fma_t(s, upT_prev, col[j - 1]);
            else col[j - 1] = (T)fma_t((double)s, upD_prev, (double)col[j - 1]);
          } else if (c == j - 1 && def_prev) {
            col[j - 1] = fast_prev ? clT_prev : (T)clD_prev;
          }
        }
      }
    }
    // ---- every record of column j has arrived (bounded wait; after a wait
    // that ran out completely the later ones are skipped) ---------------------
    bool got = false;
    if (s_ok) got = mbar_wait_bounded(&s_mbar[buf], (unsigned)(j >> 1) & 1u, p.spin, p.status,
                                      &reported);
    if (!got) {
      if (s_ok) record_status(p.status, SLQR_ETIMEOUT);
      s_ok = 0;
    }
    if (tid == 0 && got && j + 2 < nbw) mbar_expect(&s_mbar[buf], step_bytes(j + 2));

    // ---- every warp: the cluster sums, the pivot and the multipliers ----------
    // entry e: 0 the norm of column j, 1 the dot of column j + 1, 2 + t the dot
    // of own column t; lane l sums CTA (l & 15)'s record for the entries of
    // parity l >> 4, then each half-warp adds over the CTAs
    constexpr int NE = 2 + CPW;
    constexpr int NH = (NE + 1) / 2;
    const int rq = lane & 15, half = lane >> 4;
    T part[NH];
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      const int e = 2 * i + half;
      int c = -1;
      if (e == 0) c = j;
      else if (e == 1) c = j + 1;
      else if (e < NE) c = warp + (e - 2) * NW;
      const bool valid = rq < CS && c >= 0 && c < nbw && (e == 0 || c > j);
      part[i] = valid ? s_recv[buf][rq][c] : T(0);
    }
#pragma unroll
    for (int i = 0; i < NH; ++i) part[i] = half_sum(part[i]);
    T sum[NE];
#pragma unroll
    for (int e = 0; e < NE; ++e) sum[e] = __shfl_sync(0xffffffffu, part[e / 2], (e & 1) ? 16 : 0);
    const T x0 = s_prow[buf][j];
    const T p_next = (j + 1 < nbw) ? s_prow[buf][j + 1] : T(0);

    const bool fast = kF32 && abs(Ej) <= 60;    // FP32 pivot unless the scale is extreme
    const T S = sum[0];
    const bool defined = S != T(0);
    if (fast) {
      T clT = T(0), upT = T(0), rbT = T(0);
      if (defined) {
        const T sn = sqrt_t(S) * pow2_t<T>(Ej);
        clT = (x0 > T(0)) ? -sn : sn;
        upT = x0 - clT;
        rbT = T(1) / (upT * clT);                // 1 / b
      }
      // sigma_c = (up p_c + D_c) / b
#pragma unroll
      for (int t = 0; t < CPW; ++t) {
        const int c = warp + t * NW;
        sig[t] = (defined && c > j && c < nbw) ? (upT * s_prow[buf][c] + sum[2 + t]) * rbT : T(0);
      }
      sig_next = (defined && j + 1 < nbw) ? (upT * p_next + sum[1]) * rbT : T(0);
      upT_prev = upT;
      clT_prev = clT;
      if (q == 0 && tid == 0) {
        s_upT[j] = upT;
        s_rbT[j] = rbT;
        s_fast[j] = 1;
      }
    } else {
      double cl = 0.0, upk = 0.0, rb = 0.0;
      if (defined) {
        const double sn = sqrt_t((double)S) * exp2i(Ej);
        cl = ((double)x0 > 0.0) ? -sn : sn;
        upk = (double)x0 - cl;
        rb = 1.0 / (upk * cl);
      }
#pragma unroll
      for (int t = 0; t < CPW; ++t) {
        const int c = warp + t * NW;
        sig[t] = (defined && c > j && c < nbw)
                     ? (T)((upk * (double)s_prow[buf][c] + (double)sum[2 + t]) * rb) : T(0);
      }
      sig_next = (defined && j + 1 < nbw) ? (T)((upk * (double)p_next + (double)sum[1]) * rb) : T(0);
      upD_prev = upk;
      clD_prev = cl;
      if (q == 0 && tid == 0) {
        s_upD[j] = upk;
        s_rbD[j] = rb;
        s_fast[j] = 0;
      }
    }
    def_prev = defined;
    fast_prev = fast;
  }

  // ---- the last column: its tail from the column buffer, cl on the diagonal --
  if (nbw > 0) {
    const int jl = nbw - 1;
    if (warp == jl % NW) {
      const T *xl = xb + (size_t)(jl % 3) * R;
      T *col = Ps + (size_t)jl * R;
      const int r_from = (q == 0) ? jl + 1 : 0;
      for (int r = (r_from & ~31) + lane; r < RO; r += 32)
        if (r >= r_from) col[r] = xl[r];
      if (q == 0 && lane == (jl & 31) && def_prev) col[jl] = fast_prev ? clT_prev : (T)clD_prev;
    }
  }
  __syncthreads();

  // write the slice back
  for (int idx = tid; idx < nbw * R; idx += NT) {
    const int c = idx / R, r = idx - c * R;
    if (r < RO && !(p.stacked && row0 + r < nbw && row0 + r > c))
      A[SLQR_IDX(cpanel_row(p.k0, nbw, p.skip, row0 + r), p.k0 + c, lda)] = Ps[c * R + r];
  }
  double *tau = p.wy + 2 * (size_t)NB * NB;
  if (q == 0 && tid < NB) {
    double upk = 0.0, rb = 0.0;
    if (tid < nbw) {
      upk = s_fast[tid] ? (double)s_upT[tid] : s_upD[tid];
      rb = s_fast[tid] ? (double)s_rbT[tid] : s_rbD[tid];
      p.up[p.k0 + tid] = upk;
    }
    s_upD[tid] = upk;                            // (now for every column)
    tau[tid] = tid < nbw ? -rb : 0.0;            // tau = -1 / b
  }
  cluster_sync_all();
  // G[c, j] = v_c^T v_j = v_c[j] up_j + sum_{r > j} v_c[r] x_r: the partial
  // sums of every CTA, plus the first term from CTA 0 (which holds rows
  // 0..nbw-1); entry idx reduced by CTA idx % CS
  {
    double *G = p.wy + (size_t)NB * NB;
    for (int idx = q + tid * CS; idx < NB * NB; idx += NT * CS) {
      const int jj = idx / NB, c = idx - jj * NB;
      double v = 0.0;
      if (c < jj && jj < nbw) {
        for (int r = 0; r < CS; ++r) v += (double)cluster_ld(cluster_addr(&Gl[idx], r), T(0));
        v += (double)cluster_ld(cluster_addr(&Ps[c * R + jj], 0), T(0)) *
             cluster_ld(cluster_addr(&s_upD[jj], 0), 0.0);
      }
      G[idx] = v;
    }
  }
  if (q == 0) {
    // Vtop (ld NB): zero above the diagonal, up on it, tails below
    double *Vtop = p.wy;
    for (int idx = tid; idx < NB * NB; idx += NT) {
      const int c = idx / NB, r = idx - c * NB;
      double v = 0.0;
      if (c < nbw && r < nbw) {
        if (r == c) v = s_upD[c];
        else if (r > c) v = (double)Ps[c * R + r];
      }
      Vtop[idx] = v;
    }
  }
  // no CTA leaves while its shared memory may still be read
  cluster_sync_all();
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
// dynamic shared memory: the slice, three column buffers, the Gram terms
size_t cluster_panel_smem_bytes(int nb, int R, size_t elem) {
  return ((size_t)(nb + 3) * R + (size_t)nb * nb) * elem;
}

// Kernel variant (slqr_set_panel_cluster_variant): 0 chosen per panel (the
// register panel for FP32 panels of width 64 and at most 512 rows per CTA,
// else the shared-memory panel with 16 warps), 1 shared memory with 16 warps,
// 2 shared memory with 8 warps, 3 the register panel where it applies.
static int g_cluster_variant = 0;

template <typename T, int NB>
static const void *cluster_kernel(int warps) {
  return warps == 8 ? (const void *)cluster_panel_kernel<T, NB, 8>
                    : (const void *)cluster_panel_kernel<T, NB, 16>;
}

static const void *cluster_kernel_for(bool f32, int nb, int warps) {
  if (f32) return nb == 64 ? cluster_kernel<float, 64>(warps) : cluster_kernel<float, 32>(warps);
  return nb == 64 ? cluster_kernel<double, 64>(warps) : cluster_kernel<double, 32>(warps);
}

int cluster_panel_variant() { return g_cluster_variant; }
void set_cluster_panel_variant(int v) { g_cluster_variant = (v >= 0 && v <= 3) ? v : 0; }

struct ClusterLaunch {
  const void *kernel;
  int threads;
  size_t smem;
};

// The kernel, block size and dynamic shared memory of a cluster panel of R
// rows per CTA under the current variant.
static ClusterLaunch cluster_launch_for(bool f32, int nb, int R) {
  const int v = g_cluster_variant;
  if (f32 && nb == 64 && (v == 0 || v == 3)) {
    const int rpl = cluster_reg_rows_per_lane(R);
    if (rpl > 0) return {cluster_reg_kernel(rpl), 512, cluster_reg_smem_bytes(R)};
  }
  const int warps = v == 2 ? 8 : 16;
  return {cluster_kernel_for(f32, nb, warps), warps * 32,
          cluster_panel_smem_bytes(nb, R, f32 ? sizeof(float) : sizeof(double))};
}

// Dynamic shared memory a cluster-panel CTA may use (the static arrays and a
// reserve come off the opt-in maximum).
static size_t cluster_smem_cap(const slqr_ctx *ctx) {
  const size_t reserve = 24 * 1024;           // static arrays (at most ~21 KB) and slack
  return ctx->smem_optin > reserve ? ctx->smem_optin - reserve : 0;
}

int cluster_panel_rows_max(const slqr_ctx *ctx, int nb, size_t elem) {
  const size_t cap = cluster_smem_cap(ctx);
  const size_t fixed = (size_t)nb * nb * elem;
  if (cap <= fixed) return 0;
  return (int)((cap - fixed) / ((size_t)(nb + 3) * elem));
}

slqr_status init_cluster_attrs(slqr_ctx *ctx) {
  const int cap = (int)cluster_smem_cap(ctx);
  std::vector<const void *> ks;
  for (int f = 0; f < 2; ++f)
    for (int nb : {32, 64})
      for (int w : {8, 16}) ks.push_back(cluster_kernel_for(f == 1, nb, w));
  for (int rpl : {4, 8, 12, 16}) ks.push_back(cluster_reg_kernel(rpl));
  for (const void *k : ks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess)
      return fail(ctx, SLQR_ECUDA, "cluster panel attributes: %s", cudaGetErrorString(e));
  }
  return SLQR_OK;
}

static cudaLaunchConfig_t cluster_config(const ClusterLaunch &L, int ctas, cudaStream_t stream,
                                         cudaLaunchAttribute *attr) {
  cudaLaunchConfig_t cfg = {};
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)ctas);
  cfg.blockDim = dim3((unsigned)L.threads);
  cfg.dynamicSmemBytes = L.smem;
  cfg.stream = stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Can the cluster of `ctas` CTAs of R rows each be resident on this device?
// (Cached per kernel, cluster size and shared memory.)
bool cluster_panel_fits(slqr_ctx *ctx, bool f32, int nb, int ctas, int R) {
  const ClusterLaunch L = cluster_launch_for(f32, nb, R);
  if (L.smem > cluster_smem_cap(ctx)) return false;
  struct Key { const void *k; int ctas; size_t smem; int dev; int ok; };
  static std::mutex mu;
  static std::vector<Key> cache;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (const Key &k : cache)
      if (k.k == L.kernel && k.ctas == ctas && k.smem == L.smem && k.dev == ctx->device)
        return k.ok != 0;
  }
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cluster_config(L, ctas, 0, attr);
  int n = 0;
  cudaError_t e = cudaOccupancyMaxActiveClusters(&n, L.kernel, &cfg);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    n = 0;
  }
  std::lock_guard<std::mutex> lk(mu);
  cache.push_back({L.kernel, ctas, L.smem, ctx->device, n > 0 ? 1 : 0});
  return n > 0;
}

slqr_status launch_cluster_panel(slqr_ctx *ctx, bool f32, int nb, const ClusterPanelParams &pp,
                                 int ctas, cudaStream_t stream) {
  const ClusterLaunch L = cluster_launch_for(f32, nb, pp.R);
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cluster_config(L, ctas, stream, attr);
  ClusterPanelParams arg = pp;
  void *args[] = {&arg};
  cudaError_t e = cudaLaunchKernelExC(&cfg, L.kernel, args);
  if (e != cudaSuccess)
    return fail(ctx, SLQR_ECUDA, "cluster panel launch (%d CTAs, %d threads, smem=%zu): %s",
                ctas, L.threads, L.smem, cudaGetErrorString(e));
  return SLQR_OK;
}

}  // namespace slqr
