// panel_cluster_reg.cu -- the FP32 panel of 64 columns by one thread-block
// cluster with the panel held in registers.
//
// Same arithmetic and outputs as the shared-memory cluster panel of
// panel_cluster.cu (Alg. 2 of the paper on one panel: the scaled norm, the
// sign rule and up of Alg. 3, the reflector applied to the later panel
// columns; Vtop, the Gram terms of V^T V and tau for the compact-WY update),
// and the same exchange (records pushed with st.async into every CTA's
// receive buffer, counted on an mbarrier there).  What differs is where the
// slice lives: warp w of the 16 holds columns w, w + 16, w + 32, w + 48, lane
// l rows l, l + 32, ... of the CTA's slice, in registers (RPL rows per lane),
// so the per-column pass does no shared-memory traffic for the columns it
// updates.  Only two columns travel through shared memory each step: the
// reflector's column x_{j-1} (written by its owner when it is formed) and
// column j before its last update (written by its owner one pass earlier),
// from which every warp forms x_j itself with one FMA per row.
//
// The pass has no row masks.  The two shared columns are stored with zeros
// on the rows above the pivot (CTA 0) and past the slice, so those rows get a
// zero multiplier input and a zero x_j: every own column runs the same FMAs
// on every row.  The pivot row j is updated inside the pass like the rows
// below it and joins every sum; its term is taken back out algebraically
// (with up = x_0 - cl):
//     v^T a_c = up p_c + sum_{r>j} x_r a_rc = D'_c - cl p_c,
//     G[c, j] = v_c[j] up_j + sum_{r>j} v_c[r] x_r = G'_cj - cl_j v_c[j],
// where D'_c and G'_cj are the sums from the pivot row down.  CTA 0 reads the
// pivot row out of the registers for the exchange.  The R entries of each
// pivot row (row j of the later columns: + sigma_c up_j) and the diagonal
// entries cl_j are applied at the end of the panel from a table of the
// multipliers, so no step waits for them.
#include "cluster_common.cuh"

#include <type_traits>

namespace slqr {
using namespace cl;

template <int RPL>
__global__ void __launch_bounds__(512, 1)
cluster_panel_reg_kernel(ClusterPanelParams p) {
  using T = float;
  constexpr int NB = 64, NW = 16, NT = 512, CPW = NB / NW, V = 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int RP = 32 * RPL;           // rows per lane times 32 (>= R)
  const int R = p.R;
  T *xb = (T *)smem_raw;                 // [2][RP] x_j by j & 1 (zero above the pivot, past RO)
  T *cb = xb + 2 * RP;                   // [2][RP] column j before reflector j-1, by j & 1 (same)
  T *Gl = cb + 2 * RP;                   // [NB][NB] at c + j NB: Gram terms (c < j), multipliers (c > j)
  T *top = Gl + NB * NB;                 // [NB][NB] CTA 0: panel rows 0..NB-1, column-major
  __shared__ __align__(16) T s_recv[2][kClMaxCtas][NB];
  __shared__ __align__(16) T s_prow[2][NB];
  __shared__ __align__(16) T s_rec[2][2][NB];
  __shared__ unsigned s_mx[NB];
  __shared__ int s_E[NB];
  __shared__ T s_upT[NB], s_rbT[NB], s_clT[NB];
  __shared__ double s_upD[NB], s_rbD[NB], s_clD[NB];
  __shared__ int s_fast[NB], s_def[NB];
  __shared__ T s_sig[NB];                // multipliers of the current step
  __shared__ __align__(8) unsigned long long s_mbar[2];
  __shared__ int s_ok;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int q = cluster_rank(), CS = cluster_ctas();
  const int row0 = q * R;
  const int RO = max(0, min(R, p.m - p.k0 - p.skip - row0));   // rows owned
  const int nbw = p.nbw;
  T *A = (T *)p.A;
  const int lda = p.lda;
  // checked build: the launch's invariants (the same in every CTA, so every
  // CTA returns here together, before any barrier)
  if (!slqr_check(CS <= kClMaxCtas && R >= nbw && R <= RP && nbw >= 1 && nbw <= NB &&
                      p.m - p.k0 - p.skip <= CS * R && lda >= p.m, p.status))
    return;

  // ---- the slice into registers --------------------------------------------
  T v[CPW][RPL];
#pragma unroll
  for (int t = 0; t < CPW; ++t) {
    const int c = warp + t * NW;
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
      const int r = lane + 32 * i;
      // (stacked: the strictly lower part of the diagonal block is zero, not read)
      const bool zero = c >= nbw || r >= RO || (p.stacked && row0 + r < nbw && row0 + r > c);
      v[t][i] = zero ? T(0) : A[SLQR_IDX(cpanel_row(p.k0, nbw, p.skip, row0 + r), p.k0 + c, lda)];
    }
  }
  for (int idx = tid; idx < 4 * RP + NB * NB; idx += NT) xb[idx] = T(0);   // xb, cb, Gl
  __syncthreads();
  if (warp == 0) {                       // column 0 for the first pass
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
      const int r = lane + 32 * i;
      if (r < RO) cb[r] = v[0][i];
    }
  }

  // Bytes every CTA receives for column j: each CTA's record and CTA 0's
  // pivot row, each from the piece holding entry j to nbw (pieces of V).
  auto step_bytes = [&](int jj) -> unsigned {
    const int npc = (nbw - (jj & ~(V - 1)) + V - 1) / V;
    return (unsigned)((CS + 1) * npc * 16);
  };
  if (tid == 0) {
    mbar_init1(&s_mbar[0]);
    mbar_init1(&s_mbar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // the phases of columns 0 and 1; column j + 2's is announced once column
    // j's has completed (before this CTA pushes anything for column j + 1)
    if (nbw > 0) mbar_expect(&s_mbar[0], step_bytes(0));
    if (nbw > 1) mbar_expect(&s_mbar[1], step_bytes(1));
    s_ok = 1;
  }
  const int push_stride = NT / CS;
  const int push_dest = tid % CS, push_piece = tid < push_stride * CS ? tid / CS : 2 * NB;

  // ---- power-of-two column scales (max over the cluster) --------------------
#pragma unroll
  for (int t = 0; t < CPW; ++t) {
    const int c = warp + t * NW;
    const int r_from = (q == 0) ? c : 0;
    unsigned mx = 0;
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
      const int r = lane + 32 * i;
      if (c < nbw && r >= r_from && r < RO) mx = max(mx, abs_bits_hi(v[t][i]));
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) s_mx[c] = mx;
  }
  cluster_sync_all();
  if (tid < NB) {
    unsigned mx = 0;
    for (int r = 0; r < CS; ++r) mx = max(mx, cluster_ld_u32(cluster_addr(&s_mx[tid], r)));
    int E = (int)((mx >> 20) & 0x7ff) - 1023;
    s_E[tid] = min(max(E, -126), 126);   // 2^-E and 2^E normal floats
  }
  __syncthreads();

  T sig[CPW];                            // multipliers of the own columns (0 left of the pivot)
#pragma unroll
  for (int t = 0; t < CPW; ++t) sig[t] = T(0);
  T sig_next = T(0);                     // multiplier of column j (reflector j-1)
  bool reported = false;

  for (int j = 0; j < nbw; ++j) {
    const int buf = j & 1;
    const T *xo_c = xb + (size_t)(buf ^ 1) * RP;   // x_{j-1} (zero before the first)
    T *xn_o = xb + (size_t)buf * RP;               // x_j, by its owner
    const T *cj = cb + (size_t)buf * RP;           // column j before reflector j-1
    T *cn_o = cb + (size_t)(buf ^ 1) * RP;         // column j + 1 before reflector j, by its owner
    const int Ej = s_E[j];
    const T sc = pow2_t<T>(-Ej);
    const bool owner_j = warp == (j % NW);
    const int t1 = (j + 1) / NW;
    const bool owner_1 = (j + 1 < nbw) && warp == ((j + 1) % NW);
    T acc[CPW];
#pragma unroll
    for (int t = 0; t < CPW; ++t) acc[t] = T(0);
    T nacc = T(0);

    // ---- the pass: every row, the same FMAs (x_j is zero above the pivot) --
    // Rows 0..63 of CTA 0 are the only ones above a pivot: there the owners
    // store zeros above it into the shared columns.
    auto pass = [&](auto owner) {
      constexpr bool kOwner = decltype(owner)::value;
#pragma unroll
      for (int i = 0; i < RPL; ++i) {
        const int r = lane + 32 * i;
        const T xo = xo_c[r];
        const T xn = fma_t(sig_next, xo, cj[r]);   // x_j (the pivot entry on row j)
#pragma unroll
        for (int t = 0; t < CPW; ++t) {
          v[t][i] = fma_t(sig[t], xo, v[t][i]);
          acc[t] = fma_t(xn, v[t][i], acc[t]);
        }
        if constexpr (kOwner) {
          const T xs = xn * sc;
          nacc = fma_t(xs, xs, nacc);
          // the tail of x_j (rows > j) for the next pass
          xn_o[r] = (i < 2 && q == 0 && r <= j) ? T(0) : xn;
        }
      }
    };
    if (owner_j) pass(std::true_type{});
    else pass(std::false_type{});
    // ---- CTA 0: the pivot row, read out of the registers ----------------------
    if (q == 0 && lane == (j & 31)) {      // (row j < 64: register row 0 or 1)
#pragma unroll
      for (int t = 0; t < CPW; ++t) {
        const int c = warp + t * NW;
        const T w = (j < 32) ? v[t][0] : v[t][1];
        if (c >= j && c < nbw) s_rec[buf][1][c] = w;
      }
    }
    // ---- warp sums into this CTA's record (the butterfly leaves the same bits
    // in every lane) -------------------------------------------------------------
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
    // the record (CTA 0: and the pivot row) pushed to every CTA in 16-byte
    // pieces, from the piece holding entry j
    {
      const int c0 = j & ~(V - 1);
      const int npc = (nbw - c0 + V - 1) / V;
      const int items = npc * (q == 0 ? 2 : 1);
      for (int pc = push_piece; pc < items; pc += push_stride) {
        const int which = pc >= npc ? 1 : 0;
        const int c = c0 + (pc - which * npc) * V;
        const unsigned dst = which ? cluster_addr(&s_prow[buf][c], push_dest)
                                   : cluster_addr(&s_recv[buf][q][c], push_dest);
        st_async16(dst, &s_rec[buf][which][c], cluster_addr(&s_mbar[buf], push_dest));
      }
    }
    // column j + 1 before reflector j (rows >= j + 1) for the next pass,
    // written while the records travel (the barrier below orders it before
    // the next pass)
    if (owner_1) {
#pragma unroll
      for (int t = 0; t < CPW; ++t) {
        if (t != t1) continue;
#pragma unroll
        for (int i = 0; i < RPL; ++i) {
          const int r = lane + 32 * i;
          cn_o[r] = (i < 2 && q == 0 && r <= j) ? T(0) : v[t][i];
        }
      }
    }
    // ---- warp 0: every record of column j has arrived (bounded wait; after a
    // wait that ran out completely the later ones are skipped), then the
    // cluster sums, the pivot and the multiplier of every column ---------------
    if (warp == 0) {
      bool got = false;
      if (s_ok) got = mbar_wait_bounded(&s_mbar[buf], (unsigned)(j >> 1) & 1u, p.spin, p.status,
                                        &reported);
      if (!got) {
        if (s_ok) record_status(p.status, SLQR_ETIMEOUT);
        s_ok = 0;
      }
      if (lane == 0 && got && j + 2 < nbw) mbar_expect(&s_mbar[buf], step_bytes(j + 2));
      // lane l: columns l and l + 32 (a pairwise sum over the CTAs in a fixed
      // order, the same in every CTA); every lane: the norm
      T Dc[2], Sn;
      {
        T a0[kClMaxCtas], a1[kClMaxCtas], an[kClMaxCtas];
#pragma unroll
        for (int r = 0; r < kClMaxCtas; ++r) {
          a0[r] = r < CS ? s_recv[buf][r][lane] : T(0);
          a1[r] = r < CS ? s_recv[buf][r][lane + 32] : T(0);
          an[r] = r < CS ? s_recv[buf][r][j] : T(0);
        }
#pragma unroll
        for (int w = kClMaxCtas / 2; w > 0; w >>= 1)
#pragma unroll
          for (int r = 0; r < w; ++r) {
            a0[r] += a0[r + w];
            a1[r] += a1[r + w];
            an[r] += an[r + w];
          }
        Dc[0] = a0[0];
        Dc[1] = a1[0];
        Sn = an[0];
      }
      const T x0 = s_prow[buf][j];
      const bool fast = abs(Ej) <= 60;         // FP32 pivot unless the scale is extreme
      const bool defined = Sn != T(0);
      if (fast) {
        T clT = T(0), upT = T(0), rbT = T(0);
        if (defined) {
          const T sn = sqrt_t(Sn) * pow2_t<T>(Ej);
          clT = (x0 > T(0)) ? -sn : sn;
          upT = x0 - clT;
          rbT = T(1) / (upT * clT);            // 1 / b
        }
        // sigma_c = v^T a_c / b = (D'_c - cl p_c) / b
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = lane + 32 * h;
          const T sg = (defined && c > j && c < nbw) ? fma_t(-clT, s_prow[buf][c], Dc[h]) * rbT : T(0);
          s_sig[c] = sg;
          if (q == 0 && c > j && c < nbw) Gl[c + j * NB] = sg;   // for the R entries of row j
        }
        if (q == 0 && lane == 0) {
          s_upT[j] = upT;
          s_rbT[j] = rbT;
          s_clT[j] = clT;
          s_fast[j] = 1;
          s_def[j] = defined;
        }
      } else {
        double cl = 0.0, upk = 0.0, rb = 0.0;
        if (defined) {
          const double sn = sqrt_t((double)Sn) * exp2i(Ej);
          cl = ((double)x0 > 0.0) ? -sn : sn;
          upk = (double)x0 - cl;
          rb = 1.0 / (upk * cl);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = lane + 32 * h;
          const T sg = (defined && c > j && c < nbw)
                           ? (T)(((double)Dc[h] - cl * (double)s_prow[buf][c]) * rb) : T(0);
          s_sig[c] = sg;
          if (q == 0 && c > j && c < nbw) Gl[c + j * NB] = sg;
        }
        if (q == 0 && lane == 0) {
          s_upD[j] = upk;
          s_rbD[j] = rb;
          s_clD[j] = cl;
          s_fast[j] = 0;
          s_def[j] = defined;
        }
      }
    }
    __syncthreads();
    // the multipliers of this step for every warp
#pragma unroll
    for (int t = 0; t < CPW; ++t) sig[t] = s_sig[warp + t * NW];   // (0 left of the pivot)
    sig_next = (j + 1 < nbw) ? s_sig[j + 1] : T(0);
  }

  // ---- registers back: CTA 0's rows 0..NB-1 into `top` for the fix-ups, the
  // rest straight to the matrix -------------------------------------------------
#pragma unroll
  for (int t = 0; t < CPW; ++t) {
    const int c = warp + t * NW;
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
      const int r = lane + 32 * i;
      if (c < nbw && r < RO) {
        if (q == 0 && r < NB) top[c * NB + r] = v[t][i];
        else if (!(p.stacked && row0 + r < nbw && row0 + r > c))
          A[SLQR_IDX(cpanel_row(p.k0, nbw, p.skip, row0 + r), p.k0 + c, lda)] = v[t][i];
      }
    }
  }
  double *tau = p.wy + 2 * (size_t)NB * NB;
  __syncthreads();
  if (q == 0) {
    // row jj of column c > jj: + sigma_c^(jj) up_jj; the diagonal entry cl_jj
    for (int idx = tid; idx < NB * NB; idx += NT) {
      const int c = idx / NB, jj = idx - c * NB;
      if (jj < nbw && c < nbw && jj < RO) {
        if (c > jj) {
          const T s = Gl[c + jj * NB];
          top[idx] = s_fast[jj] ? fma_t(s, s_upT[jj], top[idx])
                                : (T)fma_t((double)s, s_upD[jj], (double)top[idx]);
        } else if (c == jj && s_def[jj]) {
          top[idx] = s_fast[jj] ? s_clT[jj] : (T)s_clD[jj];
        }
      }
    }
    if (tid < NB) {
      double upk = 0.0, rb = 0.0, cl = 0.0;
      if (tid < nbw) {
        upk = s_fast[tid] ? (double)s_upT[tid] : s_upD[tid];
        rb = s_fast[tid] ? (double)s_rbT[tid] : s_rbD[tid];
        cl = s_fast[tid] ? (double)s_clT[tid] : s_clD[tid];
        p.up[p.k0 + tid] = upk;
      }
      s_upD[tid] = upk;                        // (now for every column)
      s_clD[tid] = cl;
      tau[tid] = tid < nbw ? -rb : 0.0;        // tau = -1 / b
    }
  }
  __syncthreads();
  if (q == 0) {
    for (int idx = tid; idx < NB * NB; idx += NT) {
      const int c = idx / NB, r = idx - c * NB;
      if (c < nbw && r < RO && !(p.stacked && r < nbw && r > c))
        A[SLQR_IDX(cpanel_row(p.k0, nbw, p.skip, r), p.k0 + c, lda)] = top[idx];
    }
  }
  cluster_sync_all();
  // G[c, j] = v_c^T v_j = G'_cj - cl_j v_c[j] (G' summed from the pivot row
  // down): every CTA's partial sums plus the correction from CTA 0; entry idx
  // by CTA idx % CS
  {
    double *G = p.wy + (size_t)NB * NB;
    for (int idx = q + tid * CS; idx < NB * NB; idx += NT * CS) {
      const int jj = idx / NB, c = idx - jj * NB;
      double g = 0.0;
      if (c < jj && jj < nbw) {
        for (int r = 0; r < CS; ++r) g += (double)cluster_ld(cluster_addr(&Gl[idx], r), T(0));
        g -= (double)cluster_ld(cluster_addr(&top[c * NB + jj], 0), T(0)) *
             cluster_ld(cluster_addr(&s_clD[jj], 0), 0.0);
      }
      G[idx] = g;
    }
  }
  if (q == 0) {
    // Vtop (ld NB): zero above the diagonal, up on it, tails below
    double *Vtop = p.wy;
    for (int idx = tid; idx < NB * NB; idx += NT) {
      const int c = idx / NB, r = idx - c * NB;
      double g = 0.0;
      if (c < nbw && r < nbw) {
        if (r == c) g = s_upD[c];
        else if (r > c) g = (double)top[c * NB + r];
      }
      Vtop[idx] = g;
    }
  }
  // no CTA leaves while its shared memory may still be read
  cluster_sync_all();
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
int cluster_reg_rows_per_lane(int R) {
  const int need = (R + 31) / 32;
  for (int rpl : {4, 8, 12, 16})
    if (need <= rpl) return rpl;
  return 0;                              // too tall for the register panel
}

size_t cluster_reg_smem_bytes(int R) {
  const int rpl = cluster_reg_rows_per_lane(R);
  return (4 * 32 * (size_t)rpl + 2 * 64 * 64) * sizeof(float);
}

const void *cluster_reg_kernel(int rpl) {
  switch (rpl) {
    case 4: return (const void *)cluster_panel_reg_kernel<4>;
    case 8: return (const void *)cluster_panel_reg_kernel<8>;
    case 12: return (const void *)cluster_panel_reg_kernel<12>;
    case 16: return (const void *)cluster_panel_reg_kernel<16>;
    default: return nullptr;
  }
}

}  // namespace slqr
