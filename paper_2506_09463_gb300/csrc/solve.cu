// solve.cu -- back-substitution R X = C with the R of an H12 factorization.
//
// The paper (Section 1, abstract) names the back-substitution that SLSQP runs
// on the stored factorization at each iteration; it is the textbook
// substitution x_i = (c_i - sum_{j>i} R_ij x_j) / R_ii, i = n-1 .. 0.  An
// exact zero on the diagonal sets x_i = 0 and records SLQR_ERANK.
//
// GPU form: blocks of kTB rows from the bottom.  One launch first inverts
// every diagonal block (independent, one CTA each).  Launch b then updates
// every row block above block b with the now known x of block b (a tiled FP64
// GEMV or GEMM over the right-hand sides), and the CTA of the row block just
// above multiplies its updated right-hand sides by its block's inverse, so
// each launch advances the substitution by one block with no sequential chain
// inside it.  An exact zero R_ii gets a zero row and column in the block
// inverse, which sets x_i = 0 and leaves c_i unused: the same result as the
// substitution that sets x_i = 0 and carries on.
#include "slqr_internal.cuh"

#include <algorithm>

namespace slqr {

constexpr int kTB = 64;    // rows per block of R
constexpr int kRC = 16;    // right-hand sides per CTA

// Rinv[b] = inverse of the upper-triangular diagonal block b (kTB x kTB,
// column-major, zero-padded).  Thread j computes column j by back-substitution
// of R y = e_j with the diagonal reciprocals (0 for an exact zero R_ii).
__global__ void __launch_bounds__(kTB)
trsm_inv_kernel(const double *__restrict__ A, int lda, int n, double *__restrict__ Rinv,
                int *status) {
  __shared__ double Rs[kTB][kTB + 1];
  __shared__ double rd[kTB];
  const int b = blockIdx.x, j = threadIdx.x;
  const int row_begin = b * kTB;
  const int rows = min(kTB, n - row_begin);
  for (int c = 0; c < kTB; ++c)
    Rs[j][c] = (j < rows && c < rows && j <= c) ? A[SLQR_IDX(row_begin + j, row_begin + c, lda)]
                                                : 0.0;
  __syncthreads();
  const double d = Rs[j][j];
  rd[j] = (j < rows && d != 0.0) ? 1.0 / d : 0.0;
  const bool zero = (j < rows && d == 0.0);
  __syncthreads();
  double *out = Rinv + (size_t)b * kTB * kTB + (size_t)j * kTB;   // column j
  double y[kTB];
#pragma unroll
  for (int i = 0; i < kTB; ++i) y[i] = 0.0;
  if (j < rows) {
#pragma unroll
    for (int i = kTB - 1; i >= 0; --i) {
      if (i <= j) {
        double t = (i == j) ? 1.0 : 0.0;
#pragma unroll
        for (int k = i + 1; k < kTB; ++k)
          if (k <= j) t = fma(-Rs[i][k], y[k], t);
        y[i] = t * rd[i];
      }
    }
  }
#pragma unroll
  for (int i = 0; i < kTB; ++i) out[i] = y[i];
  if (zero) atomicCAS(status, 0, SLQR_ERANK);
}

// grid: (blocks, ceil(nrhs / kRC)), row block t = t_first + blockIdx.x.
// CTA t updates row block t with the x of block b_src (when b_src >= 0), and
// CTA t == b_diag then replaces its right-hand sides by Rinv[t] times them.
__global__ void __launch_bounds__(kThreads)
trsm_step_kernel(const double *__restrict__ A, int lda, int n, int nrhs, double *__restrict__ B,
                 int ldb, int t_first, int b_src, int b_diag, const double *__restrict__ Rinv) {
  __shared__ double Rs[kTB][kTB + 1];   // R tile (or the block inverse) [row][col]
  __shared__ double Xs[kRC][kTB + 1];   // x of block b_src, or the rhs being solved
  const int t = t_first + blockIdx.x;
  const int r0 = blockIdx.y * kRC;
  const int nr = min(kRC, nrhs - r0);
  const int tid = threadIdx.x;
  const int row_begin = t * kTB;
  const int rows = min(kTB, n - row_begin);
  // thread -> (row r, rhs group g): 64 rows x 4 groups of 4 rhs
  const int r = tid & (kTB - 1);
  const int g = tid >> 6;

  if (b_src >= 0) {
    const int col_begin = b_src * kTB;
    const int cols = min(kTB, n - col_begin);
    for (int idx = tid; idx < kTB * kTB; idx += kThreads) {
      int c = idx / kTB, rr = idx - c * kTB;
      Rs[rr][c] = (rr < rows && c < cols) ? A[SLQR_IDX(row_begin + rr, col_begin + c, lda)] : 0.0;
    }
    for (int idx = tid; idx < kRC * kTB; idx += kThreads) {
      int q = idx / kTB, c = idx - q * kTB;
      Xs[q][c] = (q < nr && c < cols) ? B[SLQR_IDX(col_begin + c, r0 + q, ldb)] : 0.0;
    }
    __syncthreads();
    if (r < rows) {
      double acc[kRC / 4];
#pragma unroll
      for (int q = 0; q < kRC / 4; ++q) acc[q] = 0.0;
      for (int c = 0; c < cols; ++c) {
        double rv = Rs[r][c];
#pragma unroll
        for (int q = 0; q < kRC / 4; ++q) acc[q] = fma(rv, Xs[g * (kRC / 4) + q][c], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < kRC / 4; ++q) {
        int rr = g * (kRC / 4) + q;
        if (rr < nr) B[SLQR_IDX(row_begin + r, r0 + rr, ldb)] -= acc[q];
      }
    }
    __syncthreads();
  }
  if (t != b_diag) return;

  // x of the diagonal block = Rinv[t] * (its updated right-hand sides)
  const double *Ri = Rinv + (size_t)t * kTB * kTB;
  for (int idx = tid; idx < kTB * kTB; idx += kThreads) {
    int c = idx / kTB, rr = idx - c * kTB;
    Rs[rr][c] = Ri[idx];
  }
  for (int idx = tid; idx < kRC * kTB; idx += kThreads) {
    int q = idx / kTB, rr = idx - q * kTB;
    Xs[q][rr] = (q < nr && rr < rows) ? B[SLQR_IDX(row_begin + rr, r0 + q, ldb)] : 0.0;
  }
  __syncthreads();
  if (r < rows) {
    double acc[kRC / 4];
#pragma unroll
    for (int q = 0; q < kRC / 4; ++q) acc[q] = 0.0;
    for (int c = r; c < rows; ++c) {                 // the inverse is upper triangular
      double rv = Rs[r][c];
#pragma unroll
      for (int q = 0; q < kRC / 4; ++q) acc[q] = fma(rv, Xs[g * (kRC / 4) + q][c], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < kRC / 4; ++q) {
      int rr = g * (kRC / 4) + q;
      if (rr < nr) B[SLQR_IDX(row_begin + r, r0 + rr, ldb)] = acc[q];
    }
  }
}

}  // namespace slqr

using namespace slqr;

extern "C" slqr_status slqr_solve_r(slqr_ctx *ctx, int n, const double *A, int lda, int nrhs,
                                    double *B, int ldb, void *stream) {
  NvtxRange nvtx_range("slqr_solve_r");
  if (!ctx) return SLQR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (n < 0 || nrhs < 0) return fail(ctx, SLQR_EINVAL, "n=%d nrhs=%d must be >= 0", n, nrhs);
  if (n == 0 || nrhs == 0) return SLQR_OK;
  if (lda < std::max(1, n)) return fail(ctx, SLQR_EINVAL, "lda=%d < n=%d", lda, n);
  if (ldb < std::max(1, n)) return fail(ctx, SLQR_EINVAL, "ldb=%d < n=%d", ldb, n);
  if (!A || !B) return fail(ctx, SLQR_EINVAL, "NULL A or B");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  cudaStream_t s = (cudaStream_t)stream;
  const int nblk = (n + kTB - 1) / kTB;
  const int gy = (nrhs + kRC - 1) / kRC;
  slqr_status st = ensure_workspace(ctx, (size_t)nblk * kTB * kTB * sizeof(double));
  if (st != SLQR_OK) return st;
  double *Rinv = (double *)ctx->ws.ptr;
  auto rows_of = [&](int blk) { return std::min(kTB, n - blk * kTB); };
  int slot = prof_begin(ctx, s);
  trsm_inv_kernel<<<nblk, kTB, 0, s>>>(A, lda, n, Rinv, ctx->d_status);
  prof_end(ctx, s, slot, kTrsm, 0.0);
  // first launch: only the last diagonal block
  double fl = (double)rows_of(nblk - 1) * rows_of(nblk - 1) * nrhs;
  slot = prof_begin(ctx, s);
  trsm_step_kernel<<<dim3(1, gy), kThreads, 0, s>>>(A, lda, n, nrhs, B, ldb, nblk - 1, -1,
                                                     nblk - 1, Rinv);
  prof_end(ctx, s, slot, kTrsm, fl);
  for (int b = nblk - 1; b >= 1; --b) {
    // update of rows [0, b*kTB) by block b, then the diagonal block b-1
    fl = 2.0 * b * kTB * rows_of(b) * nrhs + (double)kTB * kTB * nrhs;
    slot = prof_begin(ctx, s);
    trsm_step_kernel<<<dim3(b, gy), kThreads, 0, s>>>(A, lda, n, nrhs, B, ldb, 0, b, b - 1, Rinv);
    prof_end(ctx, s, slot, kTrsm, fl);
  }
  return check_launch(ctx, "solve_r");
}
