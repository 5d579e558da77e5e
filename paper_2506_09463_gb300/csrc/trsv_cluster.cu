// trsv_cluster.cu -- triangular solves with the FP32 R of the mixed-precision
// factorization by one thread-block cluster (the back-substitution of the
// paper's LS solve, Section 1, applied inside the refinement).
//
// Same operation and the same blocking as trsv_coop_kernel in mixed.cu:
// UPPER solves R y = c with 64-row blocks from the bottom, otherwise R^T y = c
// from the top; each diagonal block is one product with its precomputed
// inverse (diag_inv_kernel, an exact zero on the diagonal gives 0 there and
// raises *zero_flag).  Block t is owned by CTA t mod CS of a cluster of up to
// 16 CTAs, which keeps its part of the vector in shared memory.  Step k:
//
//   tiles   every CTA fetches (cp.async) the tiles of R it needs with x_b,
//           b = the k-th block solved, for each of its blocks still to be
//           solved, and the owner of the next block that block's inverse;
//   wait    every CTA waits for x_b, which the owner of b pushed into a
//           receive slot of its own for step k (st.async, counted on that
//           step's mbarrier: the slots are never reused, so no CTA can be
//           overrun however far ahead the others are);
//   update  c_t -= R_tb x_b (or R_bt^T x_b) for each of its blocks t, the
//           partial sums of a row added in a fixed order;
//   solve   the owner of the next block forms x = Rinv c, writes it to y and
//           pushes it to every CTA.
//
// Waits are bounded as in the other cluster kernels.  Every thread reaches
// every barrier (the checked build's launch-invariant check returns from
// every CTA at once, before the first barrier).
#include "cluster_common.cuh"

namespace slqr {
using namespace cl;

constexpr int kTsBlocks = 64;          // at most 64 blocks (n <= 4096)
constexpr int kTsLocal = 4;            // at most 4 blocks per CTA (16 CTAs)
constexpr int kTsLd = 68;              // tile column stride in shared memory (16-byte multiple)

template <typename VT>
struct TrsvClusterParams {
  const float *R;        // FP32 factorization; R = its upper triangle, ld lda
  const VT *Rinv;        // inverses of R's 64 x 64 diagonal blocks, [block][col][row]
  const int *zblk;       // per block, 1 when it has a zero diagonal
  VT *y;                 // right-hand side in, solution out
  int *zero_flag;
  int *status;
  int lda, n, nblk;
  unsigned spin;
};

__device__ __forceinline__ void cp16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}

template <bool UPPER, typename VT>
__global__ void __launch_bounds__(512, 1)
trsv_cluster_kernel(TrsvClusterParams<VT> p) {
  constexpr int NT = 512;
  extern __shared__ __align__(16) unsigned char traw[];
  float *Rt = (float *)traw;                                   // [kTsLocal][64][kTsLd] tiles
  VT *Ri = (VT *)(Rt + kTsLocal * 64 * kTsLd);                 // [64][64] the next block's inverse
  VT *sx = Ri + 64 * 64;                                       // [kTsBlocks][64] receive slots
  VT *red = sx + kTsBlocks * 64;                               // [kTsLocal][8][64] row parts
  __shared__ VT cs[kTsLocal][64];                              // this CTA's blocks of the vector
  __shared__ __align__(8) unsigned long long s_mb[kTsBlocks];  // one per step
  __shared__ int s_ok;

  const int tid = threadIdx.x;
  const int q = cluster_rank(), CS = cluster_ctas();
  const int nblk = p.nblk, n = p.n;
  const size_t lda = (size_t)p.lda;
  const float *R = p.R;
  constexpr int V = 16 / (int)sizeof(VT);
  auto blk = [&](int k) { return UPPER ? nblk - 1 - k : k; };    // the k-th block solved
  auto owner = [&](int b) { return b % CS; };
  auto slot = [&](int b) { return b / CS; };                     // its place in cs
  const int nloc = (nblk - q + CS - 1) / CS;                     // blocks of this CTA
  // checked build: the launch's invariants (uniform: every CTA returns here
  // together, before any barrier)
  if (!slqr_check(CS <= kClMaxCtas && nblk >= 1 && nblk <= kTsBlocks && n == 64 * nblk &&
                      (nblk + CS - 1) / CS <= kTsLocal && p.lda >= n, p.status))
    return;

  // this CTA's blocks of the right-hand side
  for (int idx = tid; idx < kTsLocal * 64; idx += NT) {
    const int i = idx >> 6, r = idx & 63, b = q + i * CS, g = b * 64 + r;
    cs[i][r] = (i < nloc && g < n) ? p.y[g] : VT(0);
  }
  if (tid == 0) {
    for (int k = 0; k < nblk; ++k) mbar_init1(&s_mb[k]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int k = 0; k < nblk; ++k) mbar_expect(&s_mb[k], 64 * (unsigned)sizeof(VT));
    s_ok = 1;
  }
  bool reported = false;
  cluster_sync_all();

  // the inverse of block b into Ri
  auto fetch_inv = [&](int b) {
    const VT *src = p.Rinv + (size_t)b * 4096;
    for (int c = tid; c < 4096 / V; c += NT) cp16(Ri + V * c, src + V * c);
  };
  // x_b = Rinv_b c_b (UPPER) or Rinv_b^T c_b by the owner of b (its inverse
  // in Ri, landed), then to y and to every CTA's receive slot of step k
  auto solve_push = [&](int k) {
    const int b = blk(k), i = slot(b);
    const int r = tid & 63, kg = tid >> 6;
    VT acc = VT(0);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = 8 * kg + j;
      acc = fma_t(UPPER ? Ri[c * 64 + r] : Ri[r * 64 + c], cs[i][c], acc);
    }
    red[kg * 64 + r] = acc;                               // (slot 0 of red)
    __syncthreads();
    if (tid < 64) {
      VT v = VT(0);
#pragma unroll
      for (int g = 0; g < 8; ++g) v += red[g * 64 + tid];
      const int row = b * 64 + tid;
      if (row < n) p.y[row] = v;
      cs[i][tid] = v;                                     // (the block is solved)
      sx[k * 64 + tid] = v;                               // staging for the push
    }
    if (tid == 0 && p.zblk[b]) atomicExch(p.zero_flag, 1);
    __syncthreads();
    for (int it = tid; it < (64 / V) * CS; it += NT) {
      const int dest = it % CS, c = (it / CS) * V;
      st_async16(cluster_addr(&sx[k * 64 + c], dest), &sx[k * 64 + c],
                 cluster_addr(&s_mb[k], dest));
    }
  };

  // the first block: its owner solves it at once
  if (owner(blk(0)) == q) {
    fetch_inv(blk(0));
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_all;" ::: "memory");
    __syncthreads();
    solve_push(0);
  }

  for (int k = 0; k < nblk; ++k) {
    const int b = blk(k), b0 = b * 64;
    const bool has_next = k + 1 < nblk;
    const int bn = has_next ? blk(k + 1) : -1;
    const bool own_next = has_next && owner(bn) == q;
    // ---- tiles for this step: blocks t of this CTA still to be solved -----------
    for (int i = 0; i < nloc; ++i) {
      const int t = q + i * CS;
      if (UPPER ? t >= b : t <= b) continue;
      const int t0 = t * 64;
      float *dst = Rt + (size_t)i * 64 * kTsLd;
      // UPPER: tile column c = R[t0 .. t0+63, b0 + c]; else column r = R[b0 .. b0+63, t0 + r]
      for (int e = tid; e < 64 * 16; e += NT) {
        const int col = e >> 4, piece = e & 15;
        const float *src = UPPER ? R + (size_t)(t0 + 4 * piece) + (size_t)(b0 + col) * lda
                                 : R + (size_t)(b0 + 4 * piece) + (size_t)(t0 + col) * lda;
        cp16(dst + col * kTsLd + 4 * piece, src);
      }
    }
    if (own_next) fetch_inv(bn);
    asm volatile("cp.async.commit_group;" ::: "memory");
    // ---- x_b ------------------------------------------------------------------------
    if (s_ok && !mbar_wait_bounded(&s_mb[k], 0u, p.spin, p.status, &reported)) {
      record_status(p.status, SLQR_ETIMEOUT);
      s_ok = 0;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    // ---- c_t -= R_tb x_b for every block t of this CTA still to be solved ---------
    {
      const VT *x = sx + k * 64;
      const int r = tid & 63, kg = tid >> 6;
      for (int i = 0; i < nloc; ++i) {
        const int t = q + i * CS;
        if (UPPER ? t >= b : t <= b) continue;
        const float *tile = Rt + (size_t)i * 64 * kTsLd;
        VT acc = VT(0);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int c = 8 * kg + j;
          // UPPER: R[t0 + r, b0 + c] = tile[c][r]; else R[b0 + c, t0 + r] = tile[r][c]
          acc = fma_t((VT)(UPPER ? tile[c * kTsLd + r] : tile[r * kTsLd + c]), x[c], acc);
        }
        red[(i * 8 + kg) * 64 + r] = acc;
      }
    }
    __syncthreads();
    for (int idx = tid; idx < nloc * 64; idx += NT) {
      const int i = idx >> 6, r = idx & 63, t = q + i * CS;
      if (UPPER ? t >= b : t <= b) continue;
      VT v = VT(0);
#pragma unroll
      for (int g = 0; g < 8; ++g) v += red[(i * 8 + g) * 64 + r];
      cs[i][r] -= v;
    }
    __syncthreads();
    // ---- the next block, by its owner ---------------------------------------------------
    if (own_next) solve_push(k + 1);
  }
  // no CTA leaves while a store to its shared memory may be in flight (every
  // step's slot was waited for above)
  cluster_sync_all();
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
template <bool UPPER, typename VT>
static size_t trsv_cluster_smem() {
  return sizeof(float) * (size_t)kTsLocal * 64 * kTsLd +
         sizeof(VT) * ((size_t)64 * 64 + (size_t)kTsBlocks * 64 + (size_t)kTsLocal * 8 * 64);
}

template <bool UPPER, typename VT>
static bool trsv_cluster_launch(slqr_ctx *ctx, const TrsvClusterParams<VT> &pp, cudaStream_t s,
                                slqr_status *st) {
  const int ctas = std::min(kClMaxCtas, pp.nblk);
  if (pp.nblk > kTsBlocks || (pp.nblk + ctas - 1) / ctas > kTsLocal) return false;
  if ((pp.lda % 4) != 0 || (((size_t)pp.R) & 15) != 0 || (((size_t)pp.Rinv) & 15) != 0)
    return false;
  const size_t smem = trsv_cluster_smem<UPPER, VT>();
  const size_t cap = ctx->smem_optin > 8192 ? ctx->smem_optin - 8192 : 0;   // (static arrays)
  if (smem > cap) return false;
  const void *k = (const void *)trsv_cluster_kernel<UPPER, VT>;
  static std::mutex mu;
  static std::vector<std::pair<const void *, int>> ready;
  {
    std::lock_guard<std::mutex> lk(mu);
    bool have = false;
    for (auto &r : ready) have |= (r.first == k && r.second == ctx->device);
    if (!have) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  static std::vector<std::pair<const void *, int>> fits;     // (kernel, ctas) known to fit
  {
    std::lock_guard<std::mutex> lk(mu);
    bool known = false;
    for (auto &f : fits) known |= (f.first == k && f.second == ctas);
    if (!known) {
      int nc = 0;
      if (cudaOccupancyMaxActiveClusters(&nc, k, &cfg) != cudaSuccess || nc <= 0) {
        (void)cudaGetLastError();
        return false;
      }
      fits.push_back({k, ctas});
    }
  }
  TrsvClusterParams<VT> arg = pp;
  void *args[] = {&arg};
  cudaError_t e = cudaLaunchKernelExC(&cfg, k, args);
  ++ctx->launch_count;
  *st = e == cudaSuccess ? SLQR_OK
                         : fail(ctx, SLQR_ECUDA, "triangular solve (cluster): %s", cudaGetErrorString(e));
  return true;
}

template <typename VT>
static bool trsv_cluster_any(slqr_ctx *ctx, bool upper, const float *R, int lda, int n,
                             const VT *Rinv, const int *zblk, VT *y, int *zero_flag,
                             cudaStream_t s, slqr_status *st) {
  if (Rinv == nullptr || zblk == nullptr || n <= 0) return false;
  TrsvClusterParams<VT> pp;
  pp.R = R; pp.Rinv = Rinv; pp.zblk = zblk; pp.y = y; pp.zero_flag = zero_flag;
  pp.status = ctx->d_status; pp.lda = lda; pp.n = n; pp.nblk = (n + 63) / 64;
  pp.spin = ctx->spin_limit;
  // the tiles are copied in whole 16-byte pieces of 64-row blocks
  if ((n % 64) != 0) return false;
  return upper ? trsv_cluster_launch<true, VT>(ctx, pp, s, st)
               : trsv_cluster_launch<false, VT>(ctx, pp, s, st);
}

bool trsv_cluster(slqr_ctx *ctx, bool upper, const float *R, int lda, int n, const float *Rinv,
                  const int *zblk, float *y, int *zero_flag, cudaStream_t s, slqr_status *st) {
  return trsv_cluster_any<float>(ctx, upper, R, lda, n, Rinv, zblk, y, zero_flag, s, st);
}

bool trsv_cluster(slqr_ctx *ctx, bool upper, const float *R, int lda, int n, const double *Rinv,
                  const int *zblk, double *y, int *zero_flag, cudaStream_t s, slqr_status *st) {
  return trsv_cluster_any<double>(ctx, upper, R, lda, n, Rinv, zblk, y, zero_flag, s, st);
}

}  // namespace slqr
