// qvec_cluster.cu -- Q^T f and Q f for one vector by one thread-block cluster
// (the Q applications of the mixed-precision refinement).
//
// Same operation and the same block reflectors as the cooperative qvec
// kernel of mixed.cu: each panel's block reflector is applied as
// f <- f - V (T^T (V^T f)) (Q^T, panels in order) or f - V (T (V^T f)) (Q,
// panels in reverse), the product of the reflectors H_k of Alg. 2 taken as
// the stored reflectors of Section 1 are reused.  The panels are applied one
// after the other (each needs the previous one's result), so the time per
// panel is the latency of one global reduction plus the time to stream the
// panel's reflectors.  Here the reduction is exchanged inside a cluster of up
// to 16 CTAs, each owning a slice of rows of f (kept in shared memory):
//
//   load    warp w takes columns w, w + 16, ... of the panel, lane l the rows
//           l, l + 32, ... of the slice: the panel's entries go straight from
//           the FP32 factorization into registers, every load issued at once
//           (the triangle of the panel's top rows is 0 above the diagonal and
//           up on it); the next panel's slice is then prefetched into L2
//           (one bulk prefetch per column);
//   dot     V^T f partials from those registers, then a warp sum;
//   push    the CTA's partials go to every CTA (st.async, 16-byte pieces,
//           counted on the receiver's mbarrier, double-buffered by panel
//           parity);
//   W'      warps 0-1 wait for the records and sum them in a fixed order
//           (the same bits in every CTA); then every thread takes part in
//           W' = T^T W (or T W) with the panel's T, fetched into shared
//           memory during the dot (eight threads per entry);
//   update  f -= V W' from the same registers: each warp's part of every row
//           through shared memory, the 16 parts of a row added in a fixed
//           order.
// Where shared memory allows, the next panel's slice comes into shared memory
// by TMA bulk copies (one per column, counted on an mbarrier) while the
// current panel is processed, and moves to registers at the start of its
// step.  The copies are issued by the warps that would otherwise wait for the
// exchange.  The slice of V in registers limits a CTA to 512 rows (m <= 8192 with
// 16 CTAs); taller problems keep the cooperative kernel.
//
// Waits are bounded as in the cluster panel: past the context's spin limit a
// wait records SLQR_ETIMEOUT and keeps waiting up to a fixed limit.  Every
// thread reaches every barrier (the checked build's launch-invariant check
// returns from every CTA at once, before the first barrier).
#include "cluster_common.cuh"

namespace slqr {
using namespace cl;

template <typename VT>
struct QvecClusterParams {
  const float *A;        // FP32 factorization (H12 form), ld lda
  const double *up;      // pivot entries of the reflectors
  const VT *Tm;          // explicit T of each panel, nb x nb, ld nb + 1
  VT *f;                 // the vector, m entries, updated in place
  int *status;
  int lda, m, K, np;
  int trans;             // 1: Q^T f, 0: Q f
  int R;                 // rows of f per CTA
  unsigned spin;
};

template <typename VT>
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}

template <typename VT, int NB, int RPL, bool TMA>
__global__ void __launch_bounds__(512, 1)
qvec_cluster_kernel(QvecClusterParams<VT> p) {
  constexpr int NW = 16, NT = 512, CPW = NB / NW;
  constexpr int V = 16 / (int)sizeof(VT);              // entries per 16-byte piece
  constexpr int TSZ = NB * (NB + 1);                   // one T (a multiple of 16 bytes)
  constexpr int RP = 32 * RPL;                         // rows per lane times 32 (>= R)
  extern __shared__ __align__(16) unsigned char qraw[];
  VT *Ts = (VT *)qraw;                                 // [NB][NB + 1] T of the current panel
  VT *sp = Ts + TSZ;                                   // [NW][RP] per-warp parts of V W'
  VT *fs = sp + NW * RP;                               // [2 RP] the CTA's slice of f, zero past it
  float *Vs = (float *)(fs + 2 * RP);                  // TMA: [NB][RP] the next panel's slice
  __shared__ __align__(16) VT s_recv[2][kClMaxCtas][NB];
  __shared__ __align__(16) VT s_rec[2][NB];
  __shared__ VT s_w[NB], s_wt[NB];
  __shared__ float s_upf[NB];                          // the panel's pivot entries, as floats
  __shared__ __align__(8) unsigned long long s_mbar[2];
  __shared__ __align__(8) unsigned long long s_vbar;   // TMA: the panel slice has landed
  __shared__ int s_ok;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int q = cluster_rank(), CS = cluster_ctas();
  const int R = p.R;
  const int r0 = q * R, r1 = min(p.m, r0 + R);
  const float *A = p.A;
  const size_t lda = (size_t)p.lda;
  // checked build: the launch's invariants (uniform: every CTA returns here
  // together, before any barrier)
  if (!slqr_check(CS <= kClMaxCtas && R <= RP && (long long)CS * R >= p.m && p.lda >= p.m &&
                      (!TMA || (R % 64 == 0 && p.lda % 4 == 0 && p.m % 4 == 0)), p.status))
    return;

  for (int r = tid; r < 2 * RP; r += NT) fs[r] = r < r1 - r0 ? p.f[r0 + r] : VT(0);
  // (TMA: every entry of Vs is finite before the first copy lands; entries
  // outside a panel's slice meet zeros of f or of W')
  if (TMA) {
    for (int r = tid; r < NB * RP; r += NT) Vs[r] = 0.f;
    // (these generic writes before the copies of the async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  const unsigned step_bytes = (unsigned)(CS * NB * (int)sizeof(VT));
  if (tid == 0) {
    mbar_init1(&s_mbar[0]);
    mbar_init1(&s_mbar[1]);
    if (TMA) mbar_init1(&s_vbar);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (p.np > 0) mbar_expect(&s_mbar[0], step_bytes);
    if (p.np > 1) mbar_expect(&s_mbar[1], step_bytes);
    s_ok = 1;
  }
  bool reported = false;
  cluster_sync_all();

  auto panel_of = [&](int step) { return p.trans ? step : p.np - 1 - step; };
  // a panel's slice of V into L2 (one bulk prefetch per column, by the
  // first NB threads) and its pivot entries into s_upf as floats (the
  // conversion runs once per panel, not per entry)
  auto prefetch = [&](int step) {
    if (step >= p.np || tid >= NB) return;
    const int pnl = panel_of(step), k0 = pnl * NB, nbw = min(NB, p.K - k0);
    const int lo = max(r0, k0), rows = r1 - lo;
    const int c = tid;
    if (c < nbw && rows > 0) {
      const float *col = A + (size_t)lo + (size_t)(k0 + c) * lda;
      const unsigned bytes = (unsigned)(rows * 4) & ~15u;
      if (bytes > 0 && (((size_t)col) & 15) == 0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(col), "r"(bytes) : "memory");
    }
  };
  auto load_up = [&](int step) {
    if (step >= p.np || tid >= NB) return;
    const int k0 = panel_of(step) * NB;
    s_upf[tid] = k0 + tid < p.K ? (float)p.up[k0 + tid] : 0.f;
  };
  // TMA: threads [t0, t0 + nth) (whole warps) copy each column of a panel's
  // slice, the first of them announcing the bytes
  auto rows_of = [&](int step, int *lo_, int *rows_) {
    const int k0 = panel_of(step) * NB;
    *lo_ = max(r0, k0);
    *rows_ = max(0, r1 - *lo_);
  };
  auto tma_issue = [&](int step, int t0, int nth) {
    if (!TMA || step >= p.np || tid < t0 || tid >= t0 + nth) return;
    const int pnl = panel_of(step), k0 = pnl * NB, nbw = min(NB, p.K - k0);
    int lo, rows;
    rows_of(step, &lo, &rows);
    const unsigned bytes = (unsigned)rows * 4u;         // (rows % 4 == 0)
    if (tid == t0) mbar_expect(&s_vbar, bytes * (unsigned)nbw);
    if (nth == 32) __syncwarp();
    else asm volatile("bar.sync 2, %0;" ::"r"(nth) : "memory");
    if (bytes == 0) return;
    const unsigned bar = (unsigned)__cvta_generic_to_shared(&s_vbar);
    for (int c = tid - t0; c < nbw; c += nth) {
      const float *src = A + (size_t)lo + (size_t)(k0 + c) * lda;
      const unsigned dst = (unsigned)__cvta_generic_to_shared(Vs + (size_t)c * RP);
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
          ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
    }
  };
  if (TMA) {
    __syncthreads();                                    // (the barrier's init before its use)
    tma_issue(0, 0, 32);
  } else {
    prefetch(0);
  }
  load_up(0);
  __syncthreads();

  for (int s = 0; s < p.np; ++s) {
    const int buf = s & 1;
    const int pnl = panel_of(s);
    const int k0 = pnl * NB, nbw = min(NB, p.K - k0);
    const int lo = max(r0, k0), rows = max(0, r1 - lo);   // this CTA's rows of the panel
    // first of them in the slice; a CTA with none of the panel's rows reads
    // the zeros past its slice instead (fs holds 2 RP entries, zero from R on)
    const int off = rows > 0 ? lo - r0 : R;
    // the panel's T into shared memory while the dot runs
    {
      const VT *src = p.Tm + (size_t)pnl * TSZ;
      for (int c = tid; c < TSZ / V; c += NT) cp_async16<VT>(Ts + V * c, src + V * c);
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    // ---- the slice of V into registers (every load issued at once): 0 above
    // the diagonal, up on it, the stored tail below; 0 past the slice -----------
    float vr[CPW][RPL];
    if (TMA) {
      if (s_ok && !mbar_wait_bounded(&s_vbar, (unsigned)s & 1u, p.spin, p.status, &reported))
        s_ok = 0;
      // every row of the slice came by TMA (m % 4 == 0); past the slice the
      // entries are stale but finite and meet zeros of f
#pragma unroll
      for (int t = 0; t < CPW; ++t)
#pragma unroll
        for (int i = 0; i < RPL; ++i) vr[t][i] = Vs[(size_t)(warp + t * NW) * RP + lane + 32 * i];
      if (lo == k0) {                                     // the panel's top rows are in this slice
#pragma unroll
        for (int t = 0; t < CPW; ++t) {
          const int c = warp + t * NW;
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            const int d = lane + 32 * i - c;              // 0 above the diagonal, up on it
            if (d < 0) vr[t][i] = 0.f;
            else if (d == 0) vr[t][i] = s_upf[c];
          }
        }
      }
      __syncthreads();                                    // every thread is done with Vs
    } else {
#pragma unroll
      for (int t = 0; t < CPW; ++t) {
        const int c = warp + t * NW;
#pragma unroll
        for (int i = 0; i < RPL; ++i) {
          const int rr = lane + 32 * i, g = lo + rr, d = g - k0 - c;
          vr[t][i] = (c < nbw && rr < rows && d > 0) ? __ldg(A + (size_t)g + (size_t)(k0 + c) * lda)
                                                      : 0.f;
          if (c < nbw && rr < rows && d == 0) vr[t][i] = s_upf[c];
        }
      }
      prefetch(s + 1);                                    // the next panel, into L2
    }
    // ---- dot: V^T f on the slice ----------------------------------------------
    VT acc[CPW];
#pragma unroll
    for (int t = 0; t < CPW; ++t) acc[t] = VT(0);
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
      const int rr = lane + 32 * i;
      const VT fv = slqr_check(off + rr < 2 * RP, p.status) ? fs[off + rr] : VT(0);   // (zero past the slice)
#pragma unroll
      for (int t = 0; t < CPW; ++t) acc[t] = fma_t((VT)vr[t][i], fv, acc[t]);
    }
#pragma unroll
    for (int t = 0; t < CPW; ++t) acc[t] = lanes_sum(acc[t]);
    if (lane == 0) {
#pragma unroll
      for (int t = 0; t < CPW; ++t) s_rec[buf][warp + t * NW] = acc[t];   // (0 past nbw)
    }
    asm volatile("cp.async.wait_all;" ::: "memory");    // this thread's part of T has landed
    __syncthreads();
    // ---- push the partials to every CTA ------------------------------------------
    for (int it = tid; it < (NB / V) * CS; it += NT) {
      const int dest = it % CS, c = (it / CS) * V;
      st_async16(cluster_addr(&s_recv[buf][q][c], dest), &s_rec[buf][c],
                 cluster_addr(&s_mbar[buf], dest));
    }
    // ---- warps 2-15 start the next panel's copies (an issuing warp can stall
    // until the copy engine accepts them) while warps 0-1 wait for the
    // cluster's records and sum them ----------------------------------------------
    tma_issue(s + 1, 64, NT - 64);
    if (warp < 2) {
      bool got = false;
      if (s_ok) got = mbar_wait_bounded(&s_mbar[buf], (unsigned)(s >> 1) & 1u, p.spin, p.status,
                                        &reported);
      if (!got) {
        if (s_ok) record_status(p.status, SLQR_ETIMEOUT);
        s_ok = 0;
      }
      if (tid == 0 && got && s + 2 < p.np) mbar_expect(&s_mbar[buf], step_bytes);
      // thread c < NB: W_c, a pairwise sum over the CTAs in a fixed order
      if (tid < NB) {
        VT a[kClMaxCtas];
#pragma unroll
        for (int r = 0; r < kClMaxCtas; ++r) a[r] = r < CS ? s_recv[buf][r][tid] : VT(0);
#pragma unroll
        for (int w = kClMaxCtas / 2; w > 0; w >>= 1)
#pragma unroll
          for (int r = 0; r < w; ++r) a[r] += a[r + w];
        s_w[tid] = a[0];
      }
    }
    __syncthreads();
    // ---- W' = T^T W (or T W): eight threads per entry j, thread l of the
    // eight taking the terms qq = l, l + 8, ..; the eight parts summed by a
    // butterfly in a fixed order -----------------------------------------------
    {
      constexpr int TPJ = NT / NB;                      // threads per entry (8)
      static_assert(TPJ * NB == NT && (TPJ & (TPJ - 1)) == 0, "threads per entry");
      const int j = tid / TPJ, l = tid % TPJ;
      VT v = VT(0);
      if (j < nbw) {
#pragma unroll
        for (int i = 0; i < NB / TPJ; ++i) {
          const int qq = l + TPJ * i;
          if (p.trans) {
            if (qq <= j) v = fma_t(Ts[qq + j * (NB + 1)], s_w[qq], v);
          } else {
            if (qq >= j && qq < nbw) v = fma_t(Ts[j + qq * (NB + 1)], s_w[qq], v);
          }
        }
      }
#pragma unroll
      for (int w = TPJ / 2; w > 0; w >>= 1) v += __shfl_xor_sync(0xffffffffu, v, w);
      if (l == 0) s_wt[j] = v;
    }
    __syncthreads();
    // ---- update: f -= V W' on the slice: each warp its columns' part of every
    // row, then the parts of a row added in a fixed order ----------------------
    {
      VT wt[CPW];
#pragma unroll
      for (int t = 0; t < CPW; ++t) wt[t] = s_wt[warp + t * NW];   // (0 past nbw)
#pragma unroll
      for (int i = 0; i < RPL; ++i) {
        VT v = VT(0);
#pragma unroll
        for (int t = 0; t < CPW; ++t) v = fma_t((VT)vr[t][i], wt[t], v);
        sp[warp * RP + lane + 32 * i] = v;
      }
    }
    __syncthreads();
    for (int rr = tid; rr < rows; rr += NT) {
      VT v = VT(0);
#pragma unroll
      for (int w = 0; w < NW; ++w) v += sp[w * RP + rr];
      if (slqr_check(rr < RP && off + rr < 2 * RP, p.status)) fs[off + rr] -= v;
    }
    load_up(s + 1);                                       // (read after the barrier)
    __syncthreads();
  }
  for (int r = tid; r < r1 - r0; r += NT) p.f[r0 + r] = fs[r];
  // no CTA leaves while a store to its shared memory may be in flight
  cluster_sync_all();
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
template <typename VT, int NB, bool TMA>
static const void *qvec_cluster_kernel_of(int rpl) {
  switch (rpl) {
    case 4: return (const void *)qvec_cluster_kernel<VT, NB, 4, TMA>;
    case 8: return (const void *)qvec_cluster_kernel<VT, NB, 8, TMA>;
    case 16: return (const void *)qvec_cluster_kernel<VT, NB, 16, TMA>;
    default: return nullptr;
  }
}

static const void *qvec_cluster_kernel_for(bool dbl, int nb, int rpl, bool tma) {
  if (dbl) {
    if (nb == 64) return tma ? qvec_cluster_kernel_of<double, 64, true>(rpl)
                             : qvec_cluster_kernel_of<double, 64, false>(rpl);
    return tma ? qvec_cluster_kernel_of<double, 32, true>(rpl)
               : qvec_cluster_kernel_of<double, 32, false>(rpl);
  }
  if (nb == 64) return tma ? qvec_cluster_kernel_of<float, 64, true>(rpl)
                           : qvec_cluster_kernel_of<float, 64, false>(rpl);
  return tma ? qvec_cluster_kernel_of<float, 32, true>(rpl)
             : qvec_cluster_kernel_of<float, 32, false>(rpl);
}

// rows per lane for R rows per CTA (0: too tall for the register slice)
static int qvec_cluster_rpl(int R) {
  const int need = (R + 31) / 32;
  for (int rpl : {4, 8, 16})
    if (need <= rpl) return rpl;
  return 0;
}

// T, the per-warp parts, the slice of f (twice its rows, zero past them);
// with TMA also a panel slice of V
static size_t qvec_cluster_smem(bool dbl, int nb, int rpl, bool tma) {
  const size_t e = dbl ? sizeof(double) : sizeof(float);
  return e * ((size_t)nb * (nb + 1) + 18 * 32 * (size_t)rpl) +
         (tma ? sizeof(float) * (size_t)nb * 32 * rpl : 0);
}

// Launch one Q application on a cluster; false (nothing launched) when the
// cluster does not fit this device.
template <typename VT>
static bool qvec_cluster_launch(slqr_ctx *ctx, const QvecClusterParams<VT> &pp0, int nb,
                                cudaStream_t stream, slqr_status *st) {
  const bool dbl = sizeof(VT) == sizeof(double);
  QvecClusterParams<VT> pp = pp0;
  const int ctas = std::max(1, std::min(kClMaxCtas, (pp.m + 63) / 64));
  // slices of a multiple of 64 rows: they start on 256-byte boundaries, and
  // a panel's top triangle (rows k0..k0+nb-1) never straddles two slices
  pp.R = ((pp.m + ctas - 1) / ctas + 63) / 64 * 64;
  const int rpl = qvec_cluster_rpl(pp.R);
  if (rpl == 0) return false;
  const size_t cap = ctx->smem_optin > 24576 ? ctx->smem_optin - 24576 : 0;   // (static arrays)
  // the panel slices by TMA when they fit shared memory and the columns of
  // the factorization start on 16-byte boundaries
  const bool tma = qvec_cluster_smem(dbl, nb, rpl, true) <= cap && (pp.lda % 4) == 0 &&
                   (pp.m % 4) == 0 && (((size_t)pp.A) & 15) == 0;
  const size_t smem = qvec_cluster_smem(dbl, nb, rpl, tma);
  if (smem > cap) return false;
  const void *k = qvec_cluster_kernel_for(dbl, nb, rpl, tma);
  static std::mutex mu;
  static std::vector<std::pair<const void *, int>> ready;   // (kernel, device) with attributes set
  {
    std::lock_guard<std::mutex> lk(mu);
    bool have = false;
    for (auto &r : ready) have |= (r.first == k && r.second == ctx->device);
    if (!have) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
      }
      ready.push_back({k, ctx->device});
    }
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)ctas);
  cfg.blockDim = dim3(512);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess || n <= 0) {
    (void)cudaGetLastError();
    return false;
  }
  void *args[] = {&pp};
  cudaError_t e = cudaLaunchKernelExC(&cfg, k, args);
  ++ctx->launch_count;
  *st = e == cudaSuccess ? SLQR_OK
                         : fail(ctx, SLQR_ECUDA, "Q application (cluster): %s", cudaGetErrorString(e));
  return true;
}

bool apply_q_cluster(slqr_ctx *ctx, const float *A32, int lda32, const double *up, int m, int K,
                     int nb, int np, const float *Tm, float *f, bool trans, cudaStream_t s,
                     slqr_status *st) {
  QvecClusterParams<float> pp;
  pp.A = A32; pp.up = up; pp.Tm = Tm; pp.f = f; pp.status = ctx->d_status; pp.lda = lda32;
  pp.m = m; pp.K = K; pp.np = np; pp.trans = trans ? 1 : 0; pp.R = 0; pp.spin = ctx->spin_limit;
  return qvec_cluster_launch<float>(ctx, pp, nb, s, st);
}

// The FP64 application (the GMRES-IR preconditioner) stays on the cooperative
// kernel for panels of more than 256 rows per CTA: its arithmetic runs on the
// FP64 pipe, which 16 SMs make the bound (on GB300, 8192 x 4096: 2x slower
// than the cooperative kernel's 128 CTAs), and its slices no longer fit
// shared memory for the TMA copies.
bool apply_q_cluster(slqr_ctx *ctx, const float *A32, int lda32, const double *up, int m, int K,
                     int nb, int np, const double *Tm, double *f, bool trans, cudaStream_t s,
                     slqr_status *st) {
  if (m > 16 * 256) return false;
  QvecClusterParams<double> pp;
  pp.A = A32; pp.up = up; pp.Tm = Tm; pp.f = f; pp.status = ctx->d_status; pp.lda = lda32;
  pp.m = m; pp.K = K; pp.np = np; pp.trans = trans ? 1 : 0; pp.R = 0; pp.spin = ctx->spin_limit;
  return qvec_cluster_launch<double>(ctx, pp, nb, s, st);
}

}  // namespace slqr
