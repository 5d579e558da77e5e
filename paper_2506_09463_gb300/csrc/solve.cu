// solve.cu -- back-substitution R X = C with the R of an H12 factorization.
//
// The paper (Section 1, abstract) names the back-substitution that SLSQP runs
// on the stored factorization at each iteration; it is the textbook
// substitution x_i = (c_i - sum_{j>i} R_ij x_j) / R_ii, i = n-1 .. 0.  An
// exact zero on the diagonal sets x_i = 0 and records SLQR_ERANK.
//
// GPU form: blocks of kTB rows from the bottom.  Launch b updates every row
// block above block b with the now known x of block b (a tiled FP64 GEMV or
// GEMM over the right-hand sides) and the CTA of the row block just above
// then solves its diagonal block, so each launch advances the substitution by
// one block.  Launch count = number of row blocks.
#include "slqr_internal.cuh"

#include <algorithm>

namespace slqr {

constexpr int kTB = 64;    // rows per block of R
constexpr int kRC = 16;    // right-hand sides per CTA

// grid: (blocks, ceil(nrhs / kRC)), row block t = t_first + blockIdx.x.
// CTA t updates row block t with the x
// of block b_src (when b_src >= 0), and CTA t == b_diag then solves its
// diagonal block.
__global__ void __launch_bounds__(kThreads)
trsm_step_kernel(const double *__restrict__ A, int lda, int n, int nrhs, double *__restrict__ B,
                 int ldb, int t_first, int b_src, int b_diag, int *status) {
  __shared__ double Rs[kTB][kTB + 1];   // R tile [row][col]
  __shared__ double Xs[kRC][kTB + 1];   // x of block b_src, or the rhs being solved
  const int t = t_first + blockIdx.x;
  const int r0 = blockIdx.y * kRC;
  const int nr = min(kRC, nrhs - r0);
  const int tid = threadIdx.x;
  const int row_begin = t * kTB;
  const int rows = min(kTB, n - row_begin);

  if (b_src >= 0) {
    const int col_begin = b_src * kTB;
    const int cols = min(kTB, n - col_begin);
    for (int idx = tid; idx < kTB * kTB; idx += kThreads) {
      int c = idx / kTB, r = idx - c * kTB;
      Rs[r][c] = (r < rows && c < cols) ? A[SLQR_IDX(row_begin + r, col_begin + c, lda)] : 0.0;
    }
    for (int idx = tid; idx < kRC * kTB; idx += kThreads) {
      int q = idx / kTB, c = idx - q * kTB;
      Xs[q][c] = (q < nr && c < cols) ? B[SLQR_IDX(col_begin + c, r0 + q, ldb)] : 0.0;
    }
    __syncthreads();
    // thread -> (row r, rhs group): 64 rows x 4 groups of 4 rhs
    const int r = tid & (kTB - 1);
    const int g = tid >> 6;
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

  // solve the diagonal block: R_tt x = c (column-oriented, one warp per rhs)
  for (int idx = tid; idx < kTB * kTB; idx += kThreads) {
    int c = idx / kTB, r = idx - c * kTB;
    Rs[r][c] = (r < rows && c < rows && r <= c) ? A[SLQR_IDX(row_begin + r, row_begin + c, lda)] : 0.0;
  }
  for (int idx = tid; idx < kRC * kTB; idx += kThreads) {
    int q = idx / kTB, r = idx - q * kTB;
    Xs[q][r] = (q < nr && r < rows) ? B[SLQR_IDX(row_begin + r, r0 + q, ldb)] : 0.0;
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  bool rank_def = false;
  for (int q = warp; q < nr; q += kThreads / 32) {
    double c0 = Xs[q][lane], c1 = Xs[q][lane + 32];
    for (int i = rows - 1; i >= 0; --i) {
      double ci = __shfl_sync(0xffffffffu, i < 32 ? c0 : c1, i & 31);
      double d = Rs[i][i];
      double xi = 0.0;
      if (d != 0.0) xi = ci / d;
      else rank_def = true;
      if (lane == (i & 31)) {
        if (i < 32) c0 = xi; else c1 = xi;
      }
      // rows l < i: c_l -= R[l][i] x_i
      if (lane < i) c0 = fma(-Rs[lane][i], xi, c0);
      if (lane + 32 < i) c1 = fma(-Rs[lane + 32][i], xi, c1);
    }
    Xs[q][lane] = c0;
    Xs[q][lane + 32] = c1;
  }
  __syncthreads();
  for (int idx = tid; idx < kRC * kTB; idx += kThreads) {
    int q = idx / kTB, r = idx - q * kTB;
    if (q < nr && r < rows) B[SLQR_IDX(row_begin + r, r0 + q, ldb)] = Xs[q][r];
  }
  if (rank_def) atomicCAS(status, 0, SLQR_ERANK);
}

}  // namespace slqr

using namespace slqr;

extern "C" slqr_status slqr_solve_r(slqr_ctx *ctx, int n, const double *A, int lda, int nrhs,
                                    double *B, int ldb, void *stream) {
  if (!ctx) return SLQR_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
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
  auto rows_of = [&](int blk) { return std::min(kTB, n - blk * kTB); };
  // first launch: only the last diagonal block
  double fl = (double)rows_of(nblk - 1) * rows_of(nblk - 1) * nrhs;
  int slot = prof_begin(ctx, s);
  trsm_step_kernel<<<dim3(1, gy), kThreads, 0, s>>>(A, lda, n, nrhs, B, ldb, nblk - 1, -1,
                                                     nblk - 1, ctx->d_status);
  prof_end(ctx, s, slot, kTrsm, fl);
  for (int b = nblk - 1; b >= 1; --b) {
    // update of rows [0, b*kTB) by block b, then the diagonal block b-1
    fl = 2.0 * b * kTB * rows_of(b) * nrhs + (double)kTB * kTB * nrhs;
    slot = prof_begin(ctx, s);
    trsm_step_kernel<<<dim3(b, gy), kThreads, 0, s>>>(A, lda, n, nrhs, B, ldb, 0, b, b - 1,
                                                       ctx->d_status);
    prof_end(ctx, s, slot, kTrsm, fl);
  }
  return check_launch(ctx, "solve_r");
}
