// apply.cu -- B <- Q^T B with the reflectors of an H12 factorization.
//
// Section 1 and the abstract of the paper: SLSQP keeps the Householder
// reflectors of its in-place QR and reuses them to apply Q^T to vectors
// before the back-substitution.  In the sequential H12 form the reflectors are
// applied one by one in the order they were built (each one an
// update_trailing_non_pivot_row on every right-hand side, Alg. 2).  Here they
// are applied NB at a time in compact-WY form, B <- B - V T^T (V^T B), using
// the same tiled DFMA kernels as the trailing update of the factorization.
//
// The compact-WY store (Vtop, strict upper V^T V, tau per panel) comes from
// slqr_factor when the caller kept it, or is rebuilt here from (A, up): Vtop
// and tau by one kernel, the Gram matrices by a row-split partial product and
// a fixed-order reduction.
#include "slqr_internal.cuh"

#include <algorithm>

namespace slqr {

// Vtop and tau of every panel from the stored form (A, up).  A reflector with
// b_k = up[k] * R_kk >= 0 is skipped: tau_k = 0.
template <int NB>
__global__ void wy_prep_kernel(const double *__restrict__ A, int lda, const double *__restrict__ up,
                               int K, double *__restrict__ wy) {
  const int pnl = blockIdx.x;
  const int k0 = pnl * NB;
  const int nbw = min(NB, K - k0);
  double *Vtop = wy + (size_t)pnl * wy_panel_doubles(NB);
  double *G = Vtop + (size_t)NB * NB;
  double *tau = Vtop + 2 * (size_t)NB * NB;
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
    int c = idx / NB, r = idx - c * NB;
    double v = 0.0;
    if (c < nbw && r < nbw) {
      if (r == c) v = up[k0 + c];
      else if (r > c) v = A[SLQR_IDX(k0 + r, k0 + c, lda)];
    }
    Vtop[idx] = v;
    G[idx] = 0.0;
  }
  for (int c = threadIdx.x; c < NB; c += blockDim.x) {
    double t = 0.0;
    if (c < nbw) {
      double b = up[k0 + c] * A[SLQR_IDX(k0 + c, k0 + c, lda)];
      if (b < 0.0) t = -1.0 / b;
    }
    tau[c] = t;
  }
}

// Partial Gram matrices: Gp[pnl][s][a][b] = sum over rows i of slice s of
// V(i, a) V(i, b), V of panel pnl (rows relative to its offset k0).
template <int NB>
__global__ void __launch_bounds__(kThreads)
gram_partial_kernel(const double *__restrict__ A, int lda, int m, int K,
                    const double *__restrict__ wy, int S, double *__restrict__ Gp) {
  constexpr int BK = 32;
  constexpr int TP = NB / 16;
  __shared__ double Vs[NB][BK + 1];
  const int pnl = blockIdx.x, s = blockIdx.y;
  const int k0 = pnl * NB;
  const int nbw = min(NB, K - k0);
  const int M = m - k0;
  int RS = (M + S - 1) / S;
  RS = (RS + BK - 1) / BK * BK;
  const int i_begin = s * RS, i_end = min(M, i_begin + RS);
  const double *Vtop = wy + (size_t)pnl * wy_panel_doubles(NB);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[TP][TP];
#pragma unroll
  for (int a = 0; a < TP; ++a)
#pragma unroll
    for (int b = 0; b < TP; ++b) acc[a][b] = 0.0;
  for (int i0 = i_begin; i0 < i_end; i0 += BK) {
    for (int idx = tid; idx < NB * BK; idx += kThreads) {
      int a = idx / BK, ii = idx - a * BK;
      int i = i0 + ii;
      double v = 0.0;
      if (i < i_end && a < nbw) v = (i < nbw) ? Vtop[i + a * NB] : A[SLQR_IDX(k0 + i, k0 + a, lda)];
      Vs[a][ii] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      double va[TP], vb[TP];
#pragma unroll
      for (int a = 0; a < TP; ++a) va[a] = Vs[tx + 16 * a][kk];
#pragma unroll
      for (int b = 0; b < TP; ++b) vb[b] = Vs[ty + 16 * b][kk];
#pragma unroll
      for (int a = 0; a < TP; ++a)
#pragma unroll
        for (int b = 0; b < TP; ++b) acc[a][b] = fma(va[a], vb[b], acc[a][b]);
    }
    __syncthreads();
  }
  double *out = Gp + ((size_t)pnl * S + s) * NB * NB;
#pragma unroll
  for (int a = 0; a < TP; ++a)
#pragma unroll
    for (int b = 0; b < TP; ++b) out[(tx + 16 * a) + (ty + 16 * b) * NB] = acc[a][b];
}

// G (strict upper part) of each panel = sum of its S partials, fixed order.
template <int NB>
__global__ void gram_reduce_kernel(const double *__restrict__ Gp, int S, int K,
                                   double *__restrict__ wy) {
  const int pnl = blockIdx.x;
  const int nbw = min(NB, K - pnl * NB);
  double *G = wy + (size_t)pnl * wy_panel_doubles(NB) + (size_t)NB * NB;
  const double *src = Gp + (size_t)pnl * S * NB * NB;
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
    int b = idx / NB, a = idx - b * NB;
    double v = 0.0;
    if (a < b && b < nbw) {
      for (int s = 0; s < S; ++s) v += src[(size_t)s * NB * NB + idx];
    }
    G[idx] = v;
  }
}

// ntop > 0: A holds the factorization of a stacked [L^T; C] (upper-triangular
// top block of ntop = n rows), whose reflectors are zero between each panel's
// diagonal block and C: those rows are skipped.
template <int NB>
static slqr_status apply_qt_impl(slqr_ctx *ctx, int m, int n, const double *A, int lda,
                                 const double *up, const double *wy, int nrhs, double *B,
                                 int ldb, cudaStream_t stream, int ntop = 0) {
  const int K = num_reflectors(m, n);
  const int np = num_panels(K, NB);
  if (np == 0) return SLQR_OK;
  const int slots = 3 * ctx->num_sms;
  const int Sg = std::max(1, std::min((4 * slots + np - 1) / np, std::max(1, m / 64)));
  const size_t wy_doubles = wy ? 0 : wy_panel_doubles(NB) * (size_t)np;
  const size_t gp_doubles = wy ? 0 : (size_t)np * Sg * NB * NB;
  const size_t work_doubles = panel_update_work_doubles(m, nrhs, NB, ctx->num_sms);
  slqr_status st = ensure_workspace(ctx, (wy_doubles + gp_doubles + work_doubles) * 8 + 256);
  if (st != SLQR_OK) return st;
  double *base = (double *)ctx->ws.ptr;
  double *wy_store = base;
  double *Gp = base + wy_doubles;
  double *work = Gp + gp_doubles;
  if (!wy) {
    double gflops = 0.0;
    for (int pnl = 0; pnl < np; ++pnl) gflops += 2.0 * (m - pnl * NB) * NB * NB;
    int slot = prof_begin(ctx, stream);
    wy_prep_kernel<NB><<<np, kThreads, 0, stream>>>(A, lda, up, K, wy_store);
    prof_end(ctx, stream, slot, kWyRebuild, 0.0);
    slot = prof_begin(ctx, stream);
    gram_partial_kernel<NB><<<dim3(np, Sg), kThreads, 0, stream>>>(A, lda, m, K, wy_store, Sg, Gp);
    prof_end(ctx, stream, slot, kWyRebuild, gflops);
    slot = prof_begin(ctx, stream);
    gram_reduce_kernel<NB><<<np, kThreads, 0, stream>>>(Gp, Sg, K, wy_store);
    prof_end(ctx, stream, slot, kWyRebuild, 0.0);
    st = check_launch(ctx, "compact-WY rebuild");
    if (st != SLQR_OK) return st;
  }
  const double *wys = wy ? wy : wy_store;
  for (int pnl = 0; pnl < np; ++pnl) {
    const int k0 = pnl * NB;
    const int nbw = std::min(NB, K - k0);
    const int skip = ntop > 0 ? ntop - (k0 + nbw) : 0;
    st = apply_panel_update(ctx, m, k0, nbw, NB, A, lda, wys + (size_t)pnl * wy_panel_doubles(NB),
                            B, ldb, nrhs, work, work_doubles, stream, skip);
    if (st != SLQR_OK) return st;
  }
  return SLQR_OK;
}

}  // namespace slqr

using namespace slqr;

extern "C" slqr_status slqr_apply_qt(slqr_ctx *ctx, int m, int n, const double *A, int lda,
                                     const double *up, const double *wy, int nrhs, double *B,
                                     int ldb, void *stream) {
  NvtxRange nvtx_range("slqr_apply_qt");
  if (!ctx) return SLQR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (m < 0 || n < 0 || m < n) return fail(ctx, SLQR_EINVAL, "need m >= n >= 0 (m=%d n=%d)", m, n);
  if (nrhs < 0) return fail(ctx, SLQR_EINVAL, "nrhs=%d < 0", nrhs);
  if (n == 0 || nrhs == 0 || m == 0) return SLQR_OK;
  if (lda < std::max(1, m)) return fail(ctx, SLQR_EINVAL, "lda=%d < m=%d", lda, m);
  if (ldb < std::max(1, m)) return fail(ctx, SLQR_EINVAL, "ldb=%d < m=%d", ldb, m);
  if (!A || !up || !B) return fail(ctx, SLQR_EINVAL, "NULL A, up or B");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  cudaStream_t s = (cudaStream_t)stream;
  if (panel_width(m, n) == 32) return apply_qt_impl<32>(ctx, m, n, A, lda, up, wy, nrhs, B, ldb, s);
  return apply_qt_impl<64>(ctx, m, n, A, lda, up, wy, nrhs, B, ldb, s);
}

extern "C" slqr_status slqr_apply_qt_stacked(slqr_ctx *ctx, int n, int m_eq, const double *A,
                                             int lda, const double *up, const double *wy,
                                             int nrhs, double *B, int ldb, void *stream) {
  NvtxRange nvtx_range("slqr_apply_qt_stacked");
  if (!ctx) return SLQR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (n < 0 || m_eq < 0) return fail(ctx, SLQR_EINVAL, "need n, m_eq >= 0 (n=%d m_eq=%d)", n, m_eq);
  if (nrhs < 0) return fail(ctx, SLQR_EINVAL, "nrhs=%d < 0", nrhs);
  const int m = n + m_eq;
  if (n == 0 || nrhs == 0) return SLQR_OK;
  if (lda < m) return fail(ctx, SLQR_EINVAL, "lda=%d < n + m_eq=%d", lda, m);
  if (ldb < m) return fail(ctx, SLQR_EINVAL, "ldb=%d < n + m_eq=%d", ldb, m);
  if (!A || !up || !B) return fail(ctx, SLQR_EINVAL, "NULL A, up or B");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  cudaStream_t s = (cudaStream_t)stream;
  if (panel_width(m, n) == 32)
    return apply_qt_impl<32>(ctx, m, n, A, lda, up, wy, nrhs, B, ldb, s, n);
  return apply_qt_impl<64>(ctx, m, n, A, lda, up, wy, nrhs, B, ldb, s, n);
}
