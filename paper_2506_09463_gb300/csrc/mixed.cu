// mixed.cu -- mixed-precision least squares for large matrices
// (slqr_lstsq_mixed).
//
// The factorization (Alg. 2, H12 storage) runs on an FP32 copy of A: the
// trailing-update products and the panel's per-column arithmetic (norm, up, b,
// multipliers) in FP32, up and the compact-WY coefficients stored in FP64
// (SLQR_FP32: FP32 FMA pipe).  The LS solution is then refined
// against the FP64 A with the augmented system [I A; A^T 0][r; x] = [b; 0]
// (Bjorck): residuals f = b - r - A x and g = -A^T r in FP64, the correction
// through the FP32 QR, h = R^-T g, d = Q^T f, dx = R^-1 (d[0:n] - h),
// dr = Q [h; d[n:m]].  This converges to the FP64 LS solution when kappa times
// the backward error of the low-precision factorization (a modest multiple of
// u_low) is below 1, for consistent and inconsistent right-hand sides.
#include "slqr_internal.cuh"

#include <math_constants.h>
#include <cmath>

#include <algorithm>
#include <cmath>
#include <vector>

namespace slqr {

constexpr int kRowsPerCta = 256;

// fused multiply-add in the vector type of a kernel (FP32 or FP64)
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
// A refinement whose steps stop contracting is accepted when its last step is
// below this (the 1e-10 solution-error target): the step then measures the
// FP64 noise level kappa * eps of an ill-conditioned problem.
constexpr double kStallOk = 1e-10;
constexpr int kColChunk = 256;

// Column equilibration by exact powers of two: D = diag(d_j), d_j = 2^-e_j
// with 2^(e_j - 1) <= max_i |a_ij| < 2^e_j, so that every column of A D has
// its largest entry in [1/2, 1).  The low-precision factorization is of A D
// (no FP32 overflow or underflow of products for any column scale); the
// refinement solves for y with x = D y, its residuals still in FP64 from A.
// One warp per column.
__global__ void col_scale_kernel(const double *__restrict__ A, int lda, int m, int n,
                                 double *__restrict__ d) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  double mx = 0.0;
  for (int i = lane; i < m; i += 32) mx = fmax(mx, fabs(A[SLQR_IDX(i, warp, lda)]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) {
    int e = 0;
    if (mx > 0.0 && isfinite(mx)) {
      frexp(mx, &e);
      e = max(-1000, min(1000, e));     // d_j stays a finite power of two
    }
    d[warp] = ldexp(1.0, -e);
  }
}

// A32 = (float) (A D)
__global__ void to_f32_kernel(const double *__restrict__ A, int lda, int m, int n,
                              const double *__restrict__ d, float *__restrict__ A32, int lda32) {
  const size_t total = (size_t)lda32 * n;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx / lda32), i = (int)(idx - (size_t)j * lda32);
    A32[idx] = (i < m) ? (float)(A[SLQR_IDX(i, j, lda)] * d[j]) : 0.f;
  }
}

// partial row sums of A (D x) over column chunks: part[chunk][i] (d NULL: D = I)
__global__ void __launch_bounds__(kRowsPerCta)
ax_partial_kernel(const double *__restrict__ A, int lda, int m, int n,
                  const double *__restrict__ x, const double *__restrict__ d,
                  double *__restrict__ part) {
  const int i = blockIdx.x * kRowsPerCta + threadIdx.x;
  const int j0 = blockIdx.y * kColChunk, j1 = min(n, j0 + kColChunk);
  __shared__ double xs[kColChunk];
  for (int j = j0 + threadIdx.x; j < j1; j += kRowsPerCta) xs[j - j0] = d ? x[j] * d[j] : x[j];
  __syncthreads();
  if (i >= m) return;
  double acc = 0.0;
  for (int j = j0; j < j1; ++j) acc = fma(A[SLQR_IDX(i, j, lda)], xs[j - j0], acc);
  part[(size_t)blockIdx.y * m + i] = acc;
}

// f = b - r - sum_chunks part (fixed order); f32 = (float) f
__global__ void resid_f_kernel(const double *__restrict__ b, const double *__restrict__ r,
                               const double *__restrict__ part, int chunks, int m,
                               float *__restrict__ f32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double ax = 0.0;
  for (int c = 0; c < chunks; ++c) ax += part[(size_t)c * m + i];
  f32[i] = (float)(b[i] - r[i] - ax);
}

// g = -(A D)^T r (one warp per column), g32 = (float) g
__global__ void resid_g_kernel(const double *__restrict__ A, int lda, int m, int n,
                               const double *__restrict__ r, const double *__restrict__ d,
                               float *__restrict__ g32) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  double acc = 0.0;
  for (int i = lane; i < m; i += 32) acc = fma(A[SLQR_IDX(i, warp, lda)], r[i], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) g32[warp] = (float)(-acc * d[warp]);
}

// e[0:n] = d[0:n] - h ; keep d[n:m] in e (e aliases nothing)
__global__ void form_e_kernel(const float *__restrict__ d, const float *__restrict__ h, int m,
                              int n, float *__restrict__ e) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) e[i] = (i < n) ? d[i] - h[i] : d[i];
}

// d[0:n] = h (so that d = [h; d2]); x += D dy (FP64); per-CTA maxima of |D dy|, |x|
__global__ void update_kernel(float *__restrict__ d, const float *__restrict__ h,
                              const float *__restrict__ dx, const double *__restrict__ cs,
                              double *__restrict__ x, int n, double *__restrict__ maxima) {
  __shared__ double s_dx[256], s_x[256];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double a = 0.0, c = 0.0;
  if (i < n) {
    d[i] = h[i];
    const double v = (double)dx[i] * cs[i];
    const double xn = x[i] + v;
    x[i] = xn;
    // a non-finite entry (an FP32 overflow in the factorization) becomes +inf,
    // which the max below keeps and the driver reports as non-convergence
    a = isfinite(v) ? fabs(v) : CUDART_INF;
    c = isfinite(xn) ? fabs(xn) : CUDART_INF;
  }
  s_dx[threadIdx.x] = a;
  s_x[threadIdx.x] = c;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s_dx[threadIdx.x] = fmax(s_dx[threadIdx.x], s_dx[threadIdx.x + o]);
      s_x[threadIdx.x] = fmax(s_x[threadIdx.x], s_x[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    maxima[2 * blockIdx.x] = s_dx[0];
    maxima[2 * blockIdx.x + 1] = s_x[0];
  }
}

// r += dr (FP64)
__global__ void add_r_kernel(double *__restrict__ r, const float *__restrict__ dr, int m) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) r[i] += (double)dr[i];
}

// r = 0, x = 0: the first sweep (f = b, g = 0) is then the plain QR solve
// x = R^-1 (Q^T b)[0:n], r = Q [0; (Q^T b)[n:m]].  Starting from r = b
// instead would route the first correction through R^-T A^T b, whose error
// grows like kappa^2 u_fp32.
__global__ void init_kernel(double *__restrict__ r, int m, double *__restrict__ x, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) r[i] = 0.0;
  if (i < n) x[i] = 0.0;
}

// --------------------------------------------------------------------------
// Q^T f and Q f for one FP32 vector in a single cooperative launch.
//
// Each panel's block reflector is applied as f <- f - V (T^T (V^T f)) (Q^T)
// or f - V (T (V^T f)) (Q), with the panels taken in order (Q^T) or in
// reverse (Q).  T is formed once per factorization (tmat_kernel) from
// T^-1 = striu(V^T V) + diag(1/tau).  A CTA owns a fixed slice of R rows of f:
// per panel it stages its slice of V in shared memory, publishes its 64
// partial dot products, and after one grid barrier every CTA sums the
// partials of all CTAs in the same fixed order, forms W' = T^T W (or T W) and
// updates its own rows.  One barrier per panel instead of three launches.
// --------------------------------------------------------------------------
constexpr int kQvRows = 128;     // rows of f per CTA (more when m exceeds 128 per SM)
constexpr int kQvRows64 = 64;    // the same for the FP64 application (GMRES-IR): twice the
                                 // CTAs, half the FP64 arithmetic per CTA and panel

// T of panel p (VT = float or double, ld nb + 1): column j solves U y = e_j by
// back substitution with U = striu(G) + diag(1/tau), i.e. y_j = tau_j and
// y_i = -tau_i sum_{k=i+1..j} G[i,k] y_k (tau = 0: a zero row and column).
template <typename VT>
__global__ void __launch_bounds__(64)
tmat_kernel(const double *__restrict__ wy, int nb, int K, VT *__restrict__ Tm) {
  __shared__ double ys[64][65];
  const int pnl = blockIdx.x, j = threadIdx.x;
  const int nbw = min(nb, K - pnl * nb);
  const double *G = wy + (size_t)pnl * wy_panel_doubles(nb) + (size_t)nb * nb;
  const double *tau = G + (size_t)nb * nb;
  VT *T = Tm + (size_t)pnl * nb * (nb + 1);
  if (j < nb) {
    for (int i = 0; i < nb; ++i) ys[i][j] = 0.0;
    if (j < nbw) {
      ys[j][j] = tau[j];
      for (int i = j - 1; i >= 0; --i) {
        double t = 0.0;
        for (int k = i + 1; k <= j; ++k) t = fma(G[i + (size_t)k * nb], ys[k][j], t);
        ys[i][j] = -tau[i] * t;
      }
    }
    for (int i = 0; i < nb; ++i) T[i + (size_t)j * (nb + 1)] = (VT)ys[i][j];
  }
}

// VT: the type of the vector and of the arithmetic (float for the Bjorck
// sweeps, double for the preconditioner of GMRES-IR, which must be one fixed
// linear operator); the reflectors are read from the FP32 factorization.
template <typename VT>
struct QvecParams {
  const float *A;        // FP32 factorization (H12 form), ld lda
  const double *up;      // pivot entries of the reflectors
  const VT *Tm;          // explicit T of each panel, nb x nb, ld nb + 1
  VT *f;                 // the vector, m entries, updated in place
  VT *part;              // 2 buffers x P CTAs x nb partial sums
  unsigned *bar;         // monotonic arrival counter
  int *status;
  int lda, m, K, nb, np;
  int trans;             // 1: Q^T f, 0: Q f
  int R, P;
  unsigned bar_base;
  unsigned spin;         // polls of the grid barrier before it gives up
};

template <typename VT>
__global__ void __launch_bounds__(kThreads)
qvec_kernel(QvecParams<VT> p) {
  extern __shared__ __align__(16) unsigned char qv_raw[];
  const int nb = p.nb, R = p.R;
  const int tsz = nb * (nb + 1);                // one T (a multiple of 16 bytes)
  VT *Ts2 = (VT *)qv_raw;                       // [2][nb][nb + 1], 16-byte aligned
  float *Vs = (float *)(Ts2 + 2 * tsz);         // [nb][R + 1]
  VT *fs = (VT *)(Vs + (size_t)nb * (R + 1));   // [R] (R + 1 odd: 8-byte aligned)
  VT *red = fs + R;                             // [kThreads / nb][nb]
  VT *ws = red + kThreads;                      // [nb]
  VT *wt = ws + nb;                             // [nb]
  __shared__ int s_ok;
  const int tid = threadIdx.x, cta = blockIdx.x;
  const int r0 = cta * R, r1 = min(p.m, r0 + R);
  // T of a panel into buffer `buf` with asynchronous 16-byte copies
  auto fetch_t = [&](int step, int buf) {
    if (step >= p.np) return;
    const int pnl = p.trans ? step : p.np - 1 - step;
    constexpr int kPer16 = 16 / (int)sizeof(VT);
    const VT *src = p.Tm + (size_t)pnl * tsz;
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(Ts2 + buf * tsz);
    for (int c = tid; c < tsz / kPer16; c += kThreads)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(dst + 16 * c),
                   "l"(src + kPer16 * c) : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  fetch_t(0, 0);
  for (int step = 0; step < p.np; ++step) {
    const int pnl = p.trans ? step : p.np - 1 - step;
    VT *Ts = Ts2 + (step & 1) * tsz;
    const int k0 = pnl * nb, nbw = min(nb, p.K - k0);
    const int lo = max(r0, k0), rows = max(0, r1 - lo);
    VT *mypart = p.part + ((size_t)(step & 1) * p.P + cta) * nb;
    // phase A: stage V and f of the slice, partial dots V^T f.  The slice
    // starts on a multiple of 64 rows and the columns of A are 128-byte
    // aligned, so whole rows of four go in one 16-byte load (8 in flight per
    // thread); the panel's top rows are then fixed up (0 above the diagonal, up on it).
    {
      const int rows4 = rows >> 2, n4 = nbw * rows4;
      for (int base = tid; base < n4; base += 8 * kThreads) {
        float4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int idx = base + u * kThreads;
          if (idx < n4) {
            const int a = idx / rows4, q = idx - a * rows4;
            v[u] = __ldcs((const float4 *)(p.A + SLQR_IDX(lo + 4 * q, k0 + a, p.lda)));
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int idx = base + u * kThreads;
          if (idx < n4) {
            const int a = idx / rows4, q = idx - a * rows4;
            float *dst = Vs + a * (R + 1) + 4 * q;
            dst[0] = v[u].x; dst[1] = v[u].y; dst[2] = v[u].z; dst[3] = v[u].w;
          }
        }
      }
      for (int idx = tid; idx < nbw * (rows - 4 * rows4); idx += kThreads) {   // ragged rows
        const int tail = rows - 4 * rows4, a = idx / tail, rr = 4 * rows4 + idx - a * tail;
        Vs[a * (R + 1) + rr] = p.A[SLQR_IDX(lo + rr, k0 + a, p.lda)];
      }
    }
    for (int rr = tid; rr < rows; rr += kThreads) fs[rr] = p.f[lo + rr];
    __syncthreads();
    if (lo < k0 + nbw) {
      // the panel's top rows: V is 0 above the diagonal and up on it (the
      // tails below are the staged entries of A)
      const int top = min(k0 + nbw, r1) - lo;
      for (int idx = tid; idx < nbw * top; idx += kThreads) {
        const int a = idx / top, rr = idx - a * top, ii = lo + rr - k0;
        if (ii < a) Vs[a * (R + 1) + rr] = 0.f;
        else if (ii == a) Vs[a * (R + 1) + rr] = (float)p.up[k0 + a];
      }
    }
    __syncthreads();
    {
      const int a = tid % nb, g = tid / nb, G = kThreads / nb;
      VT acc = 0;
      if (a < nbw)
        for (int rr = g; rr < rows; rr += G) acc = fma_t((VT)Vs[a * (R + 1) + rr], fs[rr], acc);
      red[g * nb + a] = acc;
      __syncthreads();
      if (tid < nb) {
        VT v = 0;
        for (int q = 0; q < G; ++q) v += red[q * nb + tid];
        mypart[tid] = v;
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");      // this panel's T has landed
    if (!grid_barrier(p.bar, p.bar_base + (unsigned)(step + 1) * (unsigned)p.P, p.status, &s_ok,
                      p.spin))
      return;
    fetch_t(step + 1, (step + 1) & 1);                   // the next panel's T, in flight
    // phase B: W (all CTAs, fixed order: thread (a, g) sums the partials of
    // CTAs g, g + G, .. with four loads in flight, then the G sums are added),
    // then W' = T^T W or T W
    {
      const int a = tid % nb, g = tid / nb, G = kThreads / nb;
      const VT *src = p.part + (size_t)(step & 1) * p.P * nb + a;
      VT v0 = 0, v1 = 0, v2 = 0, v3 = 0;
      int q = g;
      for (; q + 3 * G < p.P; q += 4 * G) {
        v0 += __ldcg(src + (size_t)q * nb);
        v1 += __ldcg(src + (size_t)(q + G) * nb);
        v2 += __ldcg(src + (size_t)(q + 2 * G) * nb);
        v3 += __ldcg(src + (size_t)(q + 3 * G) * nb);
      }
      for (; q < p.P; q += G) v0 += __ldcg(src + (size_t)q * nb);
      red[g * nb + a] = (v0 + v1) + (v2 + v3);
      __syncthreads();
      if (tid < nb) {
        VT v = 0;
        for (int gg = 0; gg < G; ++gg) v += red[gg * nb + tid];
        ws[tid] = v;
      }
    }
    __syncthreads();
    {
      // W' entry j: four threads take every fourth term of its dot product
      const int j = tid >> 2, part = tid & 3;
      VT v = 0;
      if (j < nbw) {
        if (p.trans) {
          for (int q = part; q <= j; q += 4) v = fma_t(Ts[q + j * (nb + 1)], ws[q], v);
        } else {
          for (int q = j + part; q < nbw; q += 4) v = fma_t(Ts[j + q * (nb + 1)], ws[q], v);
        }
      }
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      if (part == 0 && j < nb) wt[j] = v;
    }
    __syncthreads();
    // phase C: f -= V W' on the slice
    if (2 * rows <= kThreads) {                  // two threads per row, half the terms each
      const int rr = tid >> 1, half = tid & 1;
      VT v = 0;
      if (rr < rows)
        for (int a = half; a < nbw; a += 2) v = fma_t(-(VT)Vs[a * (R + 1) + rr], wt[a], v);
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      if (rr < rows && half == 0) p.f[lo + rr] = fs[rr] + v;
    } else {
      for (int rr = tid; rr < rows; rr += kThreads) {
        VT v = fs[rr];
        for (int a = 0; a < nbw; ++a) v = fma_t(-(VT)Vs[a * (R + 1) + rr], wt[a], v);
        p.f[lo + rr] = v;
      }
    }
    __syncthreads();
  }
}

template <typename VT>
static size_t qvec_smem_bytes(int nb, int R) {
  return sizeof(VT) * (2 * (size_t)nb * (nb + 1) + R + kThreads + 2 * (size_t)nb) +
         sizeof(float) * (size_t)nb * (R + 1);
}

// FP32 triangular solve with R = triu(A32[0:n, 0:n]) (ld lda) in one
// cooperative launch.  UPPER: R y = c, 64-row blocks from the bottom; else
// R^T y = c, blocks from the top.  CTA q owns the row blocks t = q (mod P).
// Step b: the owner of block b solves its diagonal block (one warp, the
// updates of every earlier step already applied to it), one grid barrier
// publishes x_b, and every CTA subtracts R_tb x_b (or R_bt^T x_b) from each of
// its blocks t still to be solved.  An exact zero on the diagonal sets that
// entry of y to 0 and raises *zero_flag.
template <typename VT>
struct TrsvParams {
  const float *R;        // FP32 factorization; the solve runs in VT arithmetic
  const VT *Rinv;        // NULL, or the inverses of R's 64 x 64 diagonal blocks
                         // (diag_inv_kernel): each block is then one product
  const int *zblk;       // with Rinv: per block, 1 when it has a zero diagonal
  VT *y;
  int *zero_flag;
  unsigned *bar;
  int *status;
  int lda, n, nblk, P;
  unsigned bar_base;
  unsigned spin;         // polls of the grid barrier before it gives up
};

template <bool UPPER, typename VT>
__global__ void __launch_bounds__(kThreads)
trsv_coop_kernel(TrsvParams<VT> p) {
  __shared__ float Rs[64][65];      // diagonal block being solved
  __shared__ float Tu[64][65];      // update tile, [c][r]: R[t r, b c] (UPPER) or R[b c, t r]
  __shared__ VT rdiag[64];
  __shared__ VT xs[64];
  __shared__ VT red[4][64];
  __shared__ int s_ok;
  const int tid = threadIdx.x, cta = blockIdx.x, lane = tid & 31;
  // with one block per CTA the diagonal block stays in shared memory throughout
  const bool one = (p.P == p.nblk);
  auto load_diag = [&](int b) {
    const int b0 = b * 64, rows = min(64, p.n - b0);
    for (int idx = tid; idx < 64 * 64; idx += kThreads) {
      const int c = idx >> 6, r = idx & 63;
      float v = 0.f;
      if (r < rows && c < rows) {
        if (UPPER && r <= c) v = p.R[SLQR_IDX(b0 + r, b0 + c, p.lda)];
        if (!UPPER && r >= c) v = p.R[SLQR_IDX(b0 + c, b0 + r, p.lda)];
      }
      Rs[r][c] = v;
    }
    __syncthreads();
    if (tid < 64)
      rdiag[tid] = (tid < rows && Rs[tid][tid] != 0.f) ? (VT)1 / (VT)Rs[tid][tid] : (VT)0;
    __syncthreads();
  };
  auto load_update = [&](int t, int b) {
    const int t0 = t * 64, b0 = b * 64;
    const int trows = min(64, p.n - t0), rows = min(64, p.n - b0);
    for (int idx = tid; idx < 64 * 64; idx += kThreads) {
      int r, c;
      if (UPPER) { r = idx & 63; c = idx >> 6; } else { c = idx & 63; r = idx >> 6; }
      float v = 0.f;
      if (r < trows && c < rows)
        v = UPPER ? p.R[SLQR_IDX(t0 + r, b0 + c, p.lda)] : p.R[SLQR_IDX(b0 + c, t0 + r, p.lda)];
      Tu[c][r] = v;
    }
  };
  if (one && !p.Rinv) load_diag(cta);
  for (int step = 0; step < p.nblk; ++step) {
    const int b = UPPER ? p.nblk - 1 - step : step;
    const int b0 = b * 64, rows = min(64, p.n - b0);
    if (b % p.P == cta && p.Rinv) {
      // x_b = Rinv_b c_b (UPPER) or Rinv_b^T c_b: thread (r, q) sums 16 terms
      // of row r, the four partials of a row are added in a fixed order
      if (tid < 64) xs[tid] = (tid < rows) ? p.y[b0 + tid] : (VT)0;
      __syncthreads();
      const VT *Ri = p.Rinv + (size_t)b * 64 * 64;
      const int r = tid & 63, q = tid >> 6;
      VT acc = 0;
      for (int c = q * 16; c < q * 16 + 16; ++c)
        acc = fma_t(UPPER ? Ri[r + 64 * c] : Ri[c + 64 * r], xs[c], acc);
      red[q][r] = acc;
      __syncthreads();
      if (tid < rows) p.y[b0 + tid] = (red[0][tid] + red[1][tid]) + (red[2][tid] + red[3][tid]);
      if (tid == 0 && p.zblk[b]) atomicExch(p.zero_flag, 1);
    } else if (b % p.P == cta) {
      if (!one) load_diag(b);
      if (tid < 64) xs[tid] = (tid < rows) ? p.y[b0 + tid] : (VT)0;
      __syncthreads();
      if (tid < 32) {
        VT c0 = xs[lane], c1 = xs[lane + 32];
        bool zero = false;
        for (int s = 0; s < rows; ++s) {
          const int i = UPPER ? rows - 1 - s : s;
          const VT ci = __shfl_sync(0xffffffffu, i < 32 ? c0 : c1, i & 31);
          const VT rd = rdiag[i];
          const VT xi = ci * rd;
          zero |= (rd == (VT)0);
          if (lane == (i & 31)) {
            if (i < 32) c0 = xi; else c1 = xi;
          }
          if (UPPER) {
            if (lane < i) c0 = fma_t(-(VT)Rs[lane][i], xi, c0);
            if (lane + 32 < i) c1 = fma_t(-(VT)Rs[lane + 32][i], xi, c1);
          } else {
            if (lane > i) c0 = fma_t(-(VT)Rs[lane][i], xi, c0);
            if (lane + 32 > i && lane + 32 < rows) c1 = fma_t(-(VT)Rs[lane + 32][i], xi, c1);
          }
        }
        if (lane < rows) p.y[b0 + lane] = c0;
        if (lane + 32 < rows) p.y[b0 + lane + 32] = c1;
        if (zero && lane == 0) atomicExch(p.zero_flag, 1);
      }
    }
    // one block per CTA: its update tile does not depend on x_b, so it is
    // loaded while the owner of block b solves
    const bool upd_one = one && (UPPER ? cta < b : cta > b);
    if (upd_one) load_update(cta, b);
    if (!grid_barrier(p.bar, p.bar_base + (unsigned)(step + 1) * (unsigned)p.P, p.status, &s_ok,
                      p.spin))
      return;
    if (tid < 64) xs[tid] = (tid < rows) ? __ldcg(p.y + b0 + tid) : (VT)0;
    __syncthreads();
    for (int t = cta; t < p.nblk; t += p.P) {
      if (UPPER ? t >= b : t <= b) continue;
      if (!one) {
        load_update(t, b);
        __syncthreads();
      }
      const int t0 = t * 64, trows = min(64, p.n - t0);
      const int r = tid & 63, q = tid >> 6;
      VT acc = 0;
      for (int c = q; c < rows; c += 4) acc = fma_t((VT)Tu[c][r], xs[c], acc);
      red[q][r] = acc;
      __syncthreads();
      if (tid < trows) p.y[t0 + tid] -= (red[0][tid] + red[1][tid]) + (red[2][tid] + red[3][tid]);
      __syncthreads();
    }
  }
}

}  // namespace slqr

namespace slqr {

// --------------------------------------------------------------------------
// GMRES-based iterative refinement (GMRES-IR) of the augmented system
//   Aaug [r; x] = [b; 0],  Aaug = [I A; A^T 0],
// left-preconditioned by M^-1, where M is the augmented matrix of the FP32
// factorization (A ~ Q R in low precision): M^-1 [f; g] is exactly one Bjorck
// correction, h = R^-T g, d = Q^T f, dx = R^-1 (d[0:n] - h), dr = Q [h; d[n:m]],
// here applied in FP64 arithmetic to the FP32 factors so that it is one fixed
// linear operator.  Each refinement step computes the residual [f; g] of the
// current (r, x) in FP64 from the FP64 A, solves Aaug z = [f; g] by GMRES on
// M^-1 Aaug z = M^-1 [f; g] (Krylov basis in FP64, classical Gram-Schmidt
// applied twice, Givens rotations on the host) and adds z.  This is the
// method of Carson, Higham and Pranesh (three-precision GMRES-IR for least
// squares, SIAM J. Sci. Comput. 42(6), 2020) with the working and residual
// precisions both FP64.  It needs far more work per step than the Bjorck
// sweep, but it converges where kappa times the factorization's backward
// error is above 1, where the Bjorck iteration diverges.
// --------------------------------------------------------------------------

// part[chunk][i] of A v (ax_partial_kernel), then
//   out_s[i] = sgn_v * v_s[i] + sgn_a * sum_chunks part   (fixed order)
// (Aaug v: sgn_v = 1, sgn_a = 1 with v_s the r-part; the residual b - r - A x:
// computed by resid64_f_kernel below)
__global__ void aug_s_kernel(const double *__restrict__ vs, const double *__restrict__ part,
                             int chunks, int m, double *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double ax = 0.0;
  for (int c = 0; c < chunks; ++c) ax += part[(size_t)c * m + i];
  out[i] = vs[i] + ax;
}

// f = b - r - sum_chunks part (FP64 output)
__global__ void resid64_f_kernel(const double *__restrict__ b, const double *__restrict__ r,
                                 const double *__restrict__ part, int chunks, int m,
                                 double *__restrict__ f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double ax = 0.0;
  for (int c = 0; c < chunks; ++c) ax += part[(size_t)c * m + i];
  f[i] = b[i] - r[i] - ax;
}

// out[j] = sgn * d_j * (A^T v)[j], one warp per column
__global__ void atv_kernel(const double *__restrict__ A, int lda, int m, int n,
                           const double *__restrict__ v, double sgn, const double *__restrict__ d,
                           double *__restrict__ out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  double acc = 0.0;
  for (int i = lane; i < m; i += 32) acc = fma(A[SLQR_IDX(i, warp, lda)], v[i], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[warp] = sgn * acc * d[warp];
}

// middle of M^-1 [f; g] in place on w = [w_s (m); w_x (n)] after h = R^-T g
// (in w_x) and d = Q^T f (in w_s): w_x = d[0:n] - h (then solved with R),
// w_s[0:n] = h (so that w_s = [h; d[n:m]] for the final Q application)
__global__ void prec_mid_kernel(double *__restrict__ ws, double *__restrict__ wx, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double h = wx[i], d = ws[i];
  wx[i] = d - h;
  ws[i] = h;
}

// block-wide sum of one double per thread (fixed order), result in thread 0
__device__ __forceinline__ double block_sum_256(double v, double *red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  return red[0];
}

// out[q] = V[:, q]^T w for q < k (one CTA per basis vector; V column-major,
// ld = N)
__global__ void __launch_bounds__(256)
basis_dots_kernel(const double *__restrict__ V, size_t N, int k, const double *__restrict__ w,
                  double *__restrict__ out) {
  __shared__ double red[256];
  const int q = blockIdx.x;
  if (q >= k) return;
  const double *vq = V + (size_t)q * N;
  double a0 = 0.0, a1 = 0.0;
  size_t i = threadIdx.x;
  for (; i + 256 < N; i += 512) {
    a0 = fma(vq[i], w[i], a0);
    a1 = fma(vq[i + 256], w[i + 256], a1);
  }
  if (i < N) a0 = fma(vq[i], w[i], a0);
  const double t = block_sum_256(a0 + a1, red);
  if (threadIdx.x == 0) out[q] = t;
}

// w -= V[:, 0:k] h  (h: k doubles, k <= kMaxKrylov + 1)
constexpr int kMaxKrylov = 512;
__global__ void __launch_bounds__(256)
basis_axpy_kernel(const double *__restrict__ V, size_t N, int k, const double *__restrict__ h,
                  double *__restrict__ w) {
  __shared__ double hs[kMaxKrylov + 1];
  for (int q = threadIdx.x; q < k; q += blockDim.x) hs[q] = h[q];
  __syncthreads();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q < k; ++q) acc = fma(V[i + (size_t)q * N], hs[q], acc);
    w[i] -= acc;
  }
}

// out[0] = ||w||_2 (one CTA, fixed order)
__global__ void __launch_bounds__(256)
vec_norm_kernel(const double *__restrict__ w, size_t N, double *__restrict__ out) {
  __shared__ double red[256];
  double a = 0.0;
  for (size_t i = threadIdx.x; i < N; i += 256) a = fma(w[i], w[i], a);
  const double t = block_sum_256(a, red);
  if (threadIdx.x == 0) out[0] = sqrt(t);
}

// w *= s
__global__ void vec_scale_kernel(double *__restrict__ w, size_t N, double s) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x)
    w[i] *= s;
}

// z = V[:, 0:k] y; r += z[0:m], x += D z[m:m+n]; per-CTA maxima of |dx| and |x|
// (a non-finite entry counts as +inf, so that it is never taken as converged)
__global__ void __launch_bounds__(256)
gmres_update_kernel(const double *__restrict__ V, size_t N, int k, const double *__restrict__ y,
                    double *__restrict__ r, int m, double *__restrict__ x, int n,
                    const double *__restrict__ d, double *__restrict__ maxima) {
  __shared__ double ys[kMaxKrylov];
  __shared__ double s_dx[256], s_x[256];
  for (int q = threadIdx.x; q < k; q += blockDim.x) ys[q] = y[q];
  __syncthreads();
  double a = 0.0, c = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x) {
    double z = 0.0;
    for (int q = 0; q < k; ++q) z = fma(V[i + (size_t)q * N], ys[q], z);
    if (i < (size_t)m) {
      r[i] += z;
    } else {
      const size_t j = i - m;
      const double dz = z * d[j];
      const double xn = x[j] + dz;
      x[j] = xn;
      a = fmax(a, isfinite(dz) ? fabs(dz) : CUDART_INF);
      c = fmax(c, isfinite(xn) ? fabs(xn) : CUDART_INF);
    }
  }
  s_dx[threadIdx.x] = a;
  s_x[threadIdx.x] = c;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s_dx[threadIdx.x] = fmax(s_dx[threadIdx.x], s_dx[threadIdx.x + o]);
      s_x[threadIdx.x] = fmax(s_x[threadIdx.x], s_x[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    maxima[2 * blockIdx.x] = s_dx[0];
    maxima[2 * blockIdx.x + 1] = s_x[0];
  }
}

// out = [max |R_ii|, min |R_ii|] over the diagonal of the FP32 R (one CTA):
// their ratio is the condition estimate that sets the FP64 noise level below
__global__ void __launch_bounds__(256)
diag_range_kernel(const float *__restrict__ R, int lda, int n, double *__restrict__ out) {
  __shared__ double smax[256], smin[256];
  double hi = 0.0, lo = CUDART_INF;
  for (int i = threadIdx.x; i < n; i += 256) {
    const double d = fabs((double)R[SLQR_IDX(i, i, lda)]);
    hi = fmax(hi, d);
    lo = fmin(lo, d);
  }
  smax[threadIdx.x] = hi;
  smin[threadIdx.x] = lo;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = smax[0];
    out[1] = smin[0];
  }
}

// Inverse of the upper-triangular 64 x 64 diagonal block b of the FP32 R, in
// FP64 (one CTA per block, thread j builds column j right-looking: at step k
// its y_k = acc_k / R_kk is final and is subtracted from the rows above).  An
// exact zero R_kk gives y_k = 0, the substitution's x_k = 0, and marks the
// block in zblk.  Rinv: [block][col][row], ld 64.
template <typename OT>
__global__ void __launch_bounds__(64)
diag_inv_kernel(const float *__restrict__ R, int lda, int n, OT *__restrict__ Rinv,
                int *__restrict__ zblk) {
  __shared__ double Rs[64][65];
  const int b = blockIdx.x, j = threadIdx.x, b0 = b * 64, rows = min(64, n - b0);
  for (int c = 0; c < 64; ++c)
    Rs[j][c] = (j < rows && c < rows && j <= c) ? (double)R[SLQR_IDX(b0 + j, b0 + c, lda)] : 0.0;
  __syncthreads();
  double acc[64];
#pragma unroll
  for (int i = 0; i < 64; ++i) acc[i] = (i == j) ? 1.0 : 0.0;
  bool zero = false;
#pragma unroll
  for (int k = 63; k >= 0; --k) {
    const double d = Rs[k][k];
    const double yk = (k < rows && d != 0.0) ? acc[k] / d : 0.0;
    zero |= (k < rows && d == 0.0);
    acc[k] = yk;
#pragma unroll
    for (int i = 0; i < k; ++i) acc[i] = fma(-Rs[i][k], yk, acc[i]);
  }
#pragma unroll
  for (int i = 0; i < 64; ++i) Rinv[(size_t)b * 4096 + (size_t)j * 64 + i] = (OT)acc[i];
  if (j == 0) zblk[b] = zero ? 1 : 0;
}

template <bool UPPER, typename VT>
static slqr_status trsv_vec(slqr_ctx *ctx, const float *R, int lda, int n, VT *y, int *zero_flag,
                            unsigned *bar, unsigned &bar_base, cudaStream_t s,
                            const VT *Rinv = nullptr, const int *zblk = nullptr) {
  // a cluster of CTAs (the solved blocks pushed through distributed shared
  // memory) unless cluster kernels are switched off or it does not apply
  if (panel_cluster_setting() >= 0 && Rinv != nullptr) {
    slqr_status cst;
    if (trsv_cluster(ctx, UPPER, R, lda, n, Rinv, zblk, y, zero_flag, s, &cst)) return cst;
  }
  TrsvParams<VT> tp;
  tp.R = R; tp.Rinv = Rinv; tp.zblk = zblk;
  tp.y = y; tp.zero_flag = zero_flag; tp.bar = bar; tp.status = ctx->d_status;
  tp.lda = lda; tp.n = n; tp.nblk = (n + 63) / 64;
  tp.P = std::min(tp.nblk, ctx->num_sms);
  tp.bar_base = bar_base;
  tp.spin = ctx->spin_limit;
  void *args[] = {&tp};
  cudaError_t e = cudaLaunchCooperativeKernel((const void *)trsv_coop_kernel<UPPER, VT>,
                                              dim3(tp.P), dim3(kThreads), args, 0, s);
  ++ctx->launch_count;
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "triangular solve: %s", cudaGetErrorString(e));
  bar_base += (unsigned)tp.nblk * (unsigned)tp.P;
  return SLQR_OK;
}

// Everything one mixed-precision solve holds on the device.
struct MixedSolve {
  slqr_ctx *ctx;
  cudaStream_t s;
  int m, n, lda, lda32, nb, K, np, chunks, ublocks;
  const double *A, *b;
  double *x;
  float *A32;
  double *up, *wy, *r, *part, *maxima;
  double *colscale;                    // D: powers of two, x = D y
  int *zero_flag;
  float *f32, *g32, *e32, *Tm32, *qpart32;
  double *Tm64, *qpart64;
  unsigned *qbar;
  unsigned qbar_base = 0;
  int qv_R, qv_P;                      // FP32 Q application: rows per CTA, CTAs
  int qv_R64, qv_P64;                  // FP64 Q application
  // GMRES-IR: Krylov basis (restart + 1 vectors of m + n) and small buffers
  double *Vk = nullptr, *hdev = nullptr, *ydev = nullptr, *drange = nullptr;
  double *Rinv = nullptr;              // FP64 inverses of R's diagonal blocks
  int *zblk = nullptr;
  float *Rinv32 = nullptr;             // the same in FP32 (the Bjorck sweeps' solves)
  int *zblk32 = nullptr;
  int restart = 0;
};

template <typename VT>
static slqr_status apply_q_vec(MixedSolve &ms, VT *f, const VT *Tm, VT *qpart, bool trans) {
  if (ms.np == 0) return SLQR_OK;
  // a cluster of CTAs (the exchange of each panel's partial sums through
  // distributed shared memory) unless cluster kernels are switched off or
  // the cluster does not fit
  if (panel_cluster_setting() >= 0) {
    slqr_status cst;
    if (apply_q_cluster(ms.ctx, ms.A32, ms.lda32, ms.up, ms.m, ms.K, ms.nb, ms.np, Tm, f, trans,
                        ms.s, &cst))
      return cst;
  }
  QvecParams<VT> qp;
  qp.A = ms.A32; qp.up = ms.up; qp.Tm = Tm; qp.f = f; qp.part = qpart; qp.bar = ms.qbar;
  qp.status = ms.ctx->d_status; qp.lda = ms.lda32; qp.m = ms.m; qp.K = ms.K; qp.nb = ms.nb;
  const bool dbl = sizeof(VT) == sizeof(double);
  const int R = dbl ? ms.qv_R64 : ms.qv_R, P = dbl ? ms.qv_P64 : ms.qv_P;
  qp.np = ms.np; qp.trans = trans ? 1 : 0; qp.R = R; qp.P = P;
  qp.bar_base = ms.qbar_base;
  qp.spin = ms.ctx->spin_limit;
  void *args[] = {&qp};
  cudaError_t le = cudaLaunchCooperativeKernel((const void *)qvec_kernel<VT>, dim3(P),
                                               dim3(kThreads), args,
                                               qvec_smem_bytes<VT>(ms.nb, R), ms.s);
  ++ms.ctx->launch_count;
  if (le != cudaSuccess)
    return fail(ms.ctx, SLQR_ECUDA, "Q application: %s", cudaGetErrorString(le));
  ms.qbar_base += (unsigned)ms.np * (unsigned)P;
  return SLQR_OK;
}

// Read back the per-CTA maxima of |dx| and |x| and the zero-diagonal flag.
static slqr_status read_step(MixedSolve &ms, int nblocks, double *dmax, double *xmax, int *zflag) {
  std::vector<double> hmax(2 * (size_t)nblocks);
  cudaError_t e = cudaMemcpyAsync(hmax.data(), ms.maxima, sizeof(double) * 2 * nblocks,
                                  cudaMemcpyDeviceToHost, ms.s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(zflag, ms.zero_flag, sizeof(int), cudaMemcpyDeviceToHost, ms.s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ms.s);
  if (e != cudaSuccess) return fail(ms.ctx, SLQR_ECUDA, "refinement: %s", cudaGetErrorString(e));
  *dmax = 0.0;
  *xmax = 0.0;
  for (int k = 0; k < nblocks; ++k) {
    *dmax = std::max(*dmax, hmax[2 * k]);
    *xmax = std::max(*xmax, hmax[2 * k + 1]);
  }
  return SLQR_OK;
}

// Bjorck sweeps (FP32 corrections, FP64 residuals) from r = 0, x = 0.
// Returns the refinement status; *it sweeps done, *e_out the last step.
static slqr_status bjorck(MixedSolve &ms, int max_iter, double tol, int *it_out, double *e_out) {
  slqr_ctx *ctx = ms.ctx;
  cudaStream_t s = ms.s;
  const int m = ms.m, n = ms.n;
  init_kernel<<<(m + 255) / 256, 256, 0, s>>>(ms.r, m, ms.x, n);
  // the inverses of R's diagonal blocks (computed in FP64, kept in FP32), once
  // for all the sweeps' triangular solves
  diag_inv_kernel<float><<<(n + 63) / 64, 64, 0, s>>>(ms.A32, ms.lda32, n, ms.Rinv32, ms.zblk32);
  ctx->launch_count += 2;
  // the two solves of a sweep that do not depend on each other run at once
  // when both are cluster kernels (their size limits)
  const bool overlap = panel_cluster_setting() >= 0 && n % 64 == 0 && n <= 4096 && m <= 8192 &&
                       m % 4 == 0 && ms.lda32 % 4 == 0;
  int it = 0, status = SLQR_ENOCONV;
  double e_cur = 1.0, e_prev = 1e300;
  slqr_status st;
  for (it = 1; it <= max_iter; ++it) {
    ax_partial_kernel<<<dim3((m + kRowsPerCta - 1) / kRowsPerCta, ms.chunks), kRowsPerCta, 0, s>>>(
        ms.A, ms.lda, m, n, ms.x, nullptr, ms.part);
    resid_f_kernel<<<(m + 255) / 256, 256, 0, s>>>(ms.b, ms.r, ms.part, ms.chunks, m, ms.f32);
    resid_g_kernel<<<(n * 32 + 255) / 256, 256, 0, s>>>(ms.A, ms.lda, m, n, ms.r, ms.colscale,
                                                         ms.g32);
    ctx->launch_count += 3;
    if (overlap) {
      // h = R^-T g on the auxiliary stream while d = Q^T f runs here: both
      // are clusters of 16 CTAs and share no buffer or barrier counter
      cudaError_t oe = cudaEventRecord(ctx->ev_ready, s);
      if (oe == cudaSuccess) oe = cudaStreamWaitEvent(ctx->aux_stream, ctx->ev_ready, 0);
      if (oe != cudaSuccess) return fail(ctx, SLQR_ECUDA, "event: %s", cudaGetErrorString(oe));
      st = trsv_vec<false>(ctx, ms.A32, ms.lda32, n, ms.g32, ms.zero_flag, ms.qbar, ms.qbar_base,
                           ctx->aux_stream, (const float *)ms.Rinv32, ms.zblk32);
      if (st != SLQR_OK) return st;                                     // h = R^-T g
      st = apply_q_vec(ms, ms.f32, ms.Tm32, ms.qpart32, true);          // d = Q^T f
      if (st != SLQR_OK) return st;
      oe = cudaEventRecord(ctx->ev_panel, ctx->aux_stream);
      if (oe == cudaSuccess) oe = cudaStreamWaitEvent(s, ctx->ev_panel, 0);
      if (oe != cudaSuccess) return fail(ctx, SLQR_ECUDA, "event: %s", cudaGetErrorString(oe));
    } else {
      st = trsv_vec<false>(ctx, ms.A32, ms.lda32, n, ms.g32, ms.zero_flag, ms.qbar, ms.qbar_base,
                           s, (const float *)ms.Rinv32, ms.zblk32);
      if (st != SLQR_OK) return st;                                     // h = R^-T g
      st = apply_q_vec(ms, ms.f32, ms.Tm32, ms.qpart32, true);          // d = Q^T f
      if (st != SLQR_OK) return st;
    }
    form_e_kernel<<<(m + 255) / 256, 256, 0, s>>>(ms.f32, ms.g32, m, n, ms.e32);
    ++ctx->launch_count;
    st = trsv_vec<true>(ctx, ms.A32, ms.lda32, n, ms.e32, ms.zero_flag, ms.qbar, ms.qbar_base, s,
                        (const float *)ms.Rinv32, ms.zblk32);
    if (st != SLQR_OK) return st;                                       // dx = R^-1 (d1 - h)
    update_kernel<<<ms.ublocks, 256, 0, s>>>(ms.f32, ms.g32, ms.e32, ms.colscale, ms.x, n,
                                             ms.maxima);
    ++ctx->launch_count;                                                // d = [h; d2], x += dx
    st = apply_q_vec(ms, ms.f32, ms.Tm32, ms.qpart32, false);           // dr = Q [h; d2]
    if (st != SLQR_OK) return st;
    add_r_kernel<<<(m + 255) / 256, 256, 0, s>>>(ms.r, ms.f32, m);
    ++ctx->launch_count;
    double dmax, xmax;
    int zflag = 0;
    st = read_step(ms, ms.ublocks, &dmax, &xmax, &zflag);
    if (st != SLQR_OK) return st;
    // an exact zero on the diagonal of R is reported first (a rank statement,
    // whatever the step looks like), then a non-finite step (an overflow:
    // never "converged")
    if (zflag) {
      e_cur = (std::isfinite(dmax) && std::isfinite(xmax) && xmax > 0.0) ? dmax / xmax : HUGE_VAL;
      status = SLQR_ERANK;
      break;
    }
    if (!std::isfinite(dmax) || !std::isfinite(xmax)) {
      e_cur = HUGE_VAL;
      status = SLQR_ENOCONV;
      break;
    }
    e_cur = (xmax > 0.0) ? dmax / xmax : 0.0;
    if (e_cur <= tol) { status = SLQR_OK; break; }
    if (it >= 3 && e_cur > 0.5 * e_prev) {      // no longer contracting
      status = (e_cur <= kStallOk) ? SLQR_OK : SLQR_ENOCONV;
      break;
    }
    e_prev = e_cur;
  }
  *it_out = std::min(it, max_iter);
  *e_out = e_cur;
  return status;
}

// w <- M^-1 w in place, w = [w_s (m); w_x (n)] in FP64 (see above)
static slqr_status precondition64(MixedSolve &ms, double *w) {
  slqr_ctx *ctx = ms.ctx;
  double *ws = w, *wx = w + ms.m;
  slqr_status st = trsv_vec<false>(ctx, ms.A32, ms.lda32, ms.n, wx, ms.zero_flag, ms.qbar,
                                   ms.qbar_base, ms.s, (const double *)ms.Rinv,
                                   ms.zblk);                            // h = R^-T g
  if (st != SLQR_OK) return st;
  st = apply_q_vec(ms, ws, ms.Tm64, ms.qpart64, true);                  // d = Q^T f
  if (st != SLQR_OK) return st;
  prec_mid_kernel<<<(ms.n + 255) / 256, 256, 0, ms.s>>>(ws, wx, ms.n);
  ++ctx->launch_count;
  st = trsv_vec<true>(ctx, ms.A32, ms.lda32, ms.n, wx, ms.zero_flag, ms.qbar, ms.qbar_base,
                      ms.s, (const double *)ms.Rinv, ms.zblk);          // dx = R^-1 (d1 - h)
  if (st != SLQR_OK) return st;
  return apply_q_vec(ms, ws, ms.Tm64, ms.qpart64, false);               // Q [h; d2]
}

// y = Aaug v = [v_s + A D v_x; D A^T v_s] (the augmented matrix of A D)
static void aug_matvec(MixedSolve &ms, const double *v, double *y) {
  const int m = ms.m, n = ms.n;
  ax_partial_kernel<<<dim3((m + kRowsPerCta - 1) / kRowsPerCta, ms.chunks), kRowsPerCta, 0, ms.s>>>(
      ms.A, ms.lda, m, n, v + m, ms.colscale, ms.part);
  aug_s_kernel<<<(m + 255) / 256, 256, 0, ms.s>>>(v, ms.part, ms.chunks, m, y);
  atv_kernel<<<(n * 32 + 255) / 256, 256, 0, ms.s>>>(ms.A, ms.lda, m, n, v, 1.0, ms.colscale,
                                                     y + m);
  ms.ctx->launch_count += 3;
}

struct GmresResult {
  int steps = 0, iters = 0;
  double err = 1.0;
};

// GMRES-IR from the current (r, x).  Returns the refinement status.
static slqr_status gmres_ir(MixedSolve &ms, double tol, int max_iters, double inner_tol,
                            double noise, GmresResult *res) {
  slqr_ctx *ctx = ms.ctx;
  cudaStream_t s = ms.s;
  const int m = ms.m, n = ms.n;
  const size_t N = (size_t)m + n;
  const int k_max = ms.restart;
  const int gblocks = std::min(4 * ctx->num_sms, (int)((N + 255) / 256));
  std::vector<double> H((size_t)(k_max + 1) * k_max), cs(k_max), sn(k_max), gv(k_max + 1),
      y(k_max), hh(2 * (size_t)(k_max + 2));
  const int max_steps = 20;
  int status = SLQR_ENOCONV;
  double e_prev = HUGE_VAL;
  slqr_status st;
  for (int step = 1; step <= max_steps && res->iters < max_iters; ++step) {
    // residual of the augmented system in FP64: f = b - r - A x, g = -D A^T r
    double *V0 = ms.Vk;
    ax_partial_kernel<<<dim3((m + kRowsPerCta - 1) / kRowsPerCta, ms.chunks), kRowsPerCta, 0, s>>>(
        ms.A, ms.lda, m, n, ms.x, nullptr, ms.part);
    resid64_f_kernel<<<(m + 255) / 256, 256, 0, s>>>(ms.b, ms.r, ms.part, ms.chunks, m, V0);
    atv_kernel<<<(n * 32 + 255) / 256, 256, 0, s>>>(ms.A, ms.lda, m, n, ms.r, -1.0, ms.colscale,
                                                    V0 + m);
    ctx->launch_count += 3;
    st = precondition64(ms, V0);
    if (st != SLQR_OK) return st;
    vec_norm_kernel<<<1, 256, 0, s>>>(V0, N, ms.hdev);
    ++ctx->launch_count;
    double beta = 0.0;
    cudaError_t e = cudaMemcpyAsync(&beta, ms.hdev, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "GMRES-IR: %s", cudaGetErrorString(e));
    if (!std::isfinite(beta)) { res->err = HUGE_VAL; return SLQR_ENOCONV; }
    if (beta == 0.0) { res->err = 0.0; return SLQR_OK; }    // (r, x) solves the system
    vec_scale_kernel<<<gblocks, 256, 0, s>>>(V0, N, 1.0 / beta);
    ++ctx->launch_count;
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int k = 0;
    bool inner_ok = false, hopeless = false;
    const int iters_left = max_iters - res->iters;
    for (int j = 0; j < k_max && res->iters < max_iters; ++j) {
      double *vj = ms.Vk + (size_t)j * N, *w = ms.Vk + (size_t)(j + 1) * N;
      aug_matvec(ms, vj, w);                                   // w = Aaug v_j
      st = precondition64(ms, w);                              // w = M^-1 Aaug v_j
      if (st != SLQR_OK) return st;
      // classical Gram-Schmidt, twice
      basis_dots_kernel<<<j + 1, 256, 0, s>>>(ms.Vk, N, j + 1, w, ms.hdev);
      basis_axpy_kernel<<<gblocks, 256, 0, s>>>(ms.Vk, N, j + 1, ms.hdev, w);
      basis_dots_kernel<<<j + 1, 256, 0, s>>>(ms.Vk, N, j + 1, w, ms.hdev + (k_max + 2));
      basis_axpy_kernel<<<gblocks, 256, 0, s>>>(ms.Vk, N, j + 1, ms.hdev + (k_max + 2), w);
      vec_norm_kernel<<<1, 256, 0, s>>>(w, N, ms.hdev + (j + 1));
      ctx->launch_count += 5;
      e = cudaMemcpyAsync(hh.data(), ms.hdev, sizeof(double) * 2 * (k_max + 2),
                          cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "GMRES-IR: %s", cudaGetErrorString(e));
      ++res->iters;
      double *hc = &H[(size_t)j * (k_max + 1)];
      for (int q = 0; q <= j; ++q) hc[q] = hh[q] + hh[(k_max + 2) + q];
      const double hnext = hh[j + 1];
      hc[j + 1] = hnext;
      if (!std::isfinite(hnext)) { res->err = HUGE_VAL; return SLQR_ENOCONV; }
      // previous rotations, then a new one that zeroes H[j+1, j]
      for (int q = 0; q < j; ++q) {
        const double a = hc[q], c = hc[q + 1];
        hc[q] = cs[q] * a + sn[q] * c;
        hc[q + 1] = -sn[q] * a + cs[q] * c;
      }
      const double rho = std::hypot(hc[j], hc[j + 1]);
      cs[j] = rho > 0.0 ? hc[j] / rho : 1.0;
      sn[j] = rho > 0.0 ? hc[j + 1] / rho : 0.0;
      hc[j] = rho;
      hc[j + 1] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      k = j + 1;
      const double rel = std::fabs(gv[j + 1]) / beta;
      if (rel <= inner_tol) { inner_ok = true; break; }
      if (hnext <= 1e-300 * beta) { inner_ok = true; break; }   // invariant subspace: exact
      // give up early when the residual's rate so far predicts far more
      // iterations than the budget has left (the caller's fallback, if any,
      // then starts at once): after 32 iterations, a geometric rate
      // rel^(1/(j+1)) would need (j+1) log(inner_tol) / log(rel) iterations
      if (j + 1 >= 32) {
        const double need = (rel < 1.0) ? (j + 1) * std::log(inner_tol) / std::log(rel) : HUGE_VAL;
        if (need > 2.0 * iters_left) { hopeless = true; break; }
      }
      vec_scale_kernel<<<gblocks, 256, 0, s>>>(w, N, 1.0 / hnext);
      ++ctx->launch_count;
    }
    if (hopeless) { res->err = HUGE_VAL; return SLQR_ENOCONV; }
    // y = H[0:k, 0:k]^-1 g[0:k] (upper triangular after the rotations)
    for (int q = k - 1; q >= 0; --q) {
      double t = gv[q];
      for (int c = q + 1; c < k; ++c) t -= H[(size_t)c * (k_max + 1) + q] * y[c];
      const double d = H[(size_t)q * (k_max + 1) + q];
      y[q] = d != 0.0 ? t / d : 0.0;
    }
    e = cudaMemcpyAsync(ms.ydev, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "GMRES-IR: %s", cudaGetErrorString(e));
    const int ub = std::min(4 * ctx->num_sms, (int)((N + 255) / 256));
    gmres_update_kernel<<<ub, 256, 0, s>>>(ms.Vk, N, k, ms.ydev, ms.r, m, ms.x, n, ms.colscale,
                                           ms.maxima);
    ++ctx->launch_count;
    ++res->steps;
    double dmax, xmax;
    int zflag = 0;
    st = read_step(ms, ub, &dmax, &xmax, &zflag);
    if (st != SLQR_OK) return st;
    if (zflag) { res->err = HUGE_VAL; return SLQR_ERANK; }
    if (!std::isfinite(dmax) || !std::isfinite(xmax)) { res->err = HUGE_VAL; return SLQR_ENOCONV; }
    const double e_cur = (xmax > 0.0) ? dmax / xmax : 0.0;
    res->err = e_cur;
    // converged: the step is below tol, or it is at the FP64 noise level of
    // this problem after an inner solve that reached its tolerance (the
    // remaining error is then a small fraction of that step)
    if (e_cur <= tol || (inner_ok && e_cur <= noise)) { status = SLQR_OK; break; }
    if (step >= 3 && e_cur > 0.5 * e_prev) {           // no longer contracting
      status = (e_cur <= noise) ? SLQR_OK : SLQR_ENOCONV;
      break;
    }
    e_prev = e_cur;
  }
  return status;
}

// FP64 solve of the same problem (slqr_factor, slqr_apply_qt, slqr_solve_r on
// a copy of A): the opt-in fallback when the mixed-precision refinement fails.
static slqr_status fp64_fallback(slqr_ctx *ctx, int m, int n, const double *A, int lda,
                                 const double *b, double *x, cudaStream_t s) {
  const size_t a_bytes = align_up((size_t)m * n * sizeof(double), 256);
  const size_t up_bytes = align_up((size_t)n * sizeof(double), 256);
  const size_t wy_bytes = align_up(slqr_wy_size(m, n), 256);
  const size_t b_bytes = align_up((size_t)m * sizeof(double), 256);
  cudaError_t e = cudaStreamSynchronize(s);   // the mixed buffers are no longer in use
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "fallback: %s", cudaGetErrorString(e));
  slqr_status st = ensure_workspace2(ctx, a_bytes + up_bytes + wy_bytes + b_bytes);
  if (st != SLQR_OK) return st;
  char *base = (char *)ctx->ws2.ptr;
  double *A64 = (double *)base;
  double *up = (double *)(base + a_bytes);
  double *wy = (double *)(base + a_bytes + up_bytes);
  double *B = (double *)(base + a_bytes + up_bytes + wy_bytes);
  int st_before = 0;
  e = cudaMemcpy2DAsync(A64, (size_t)m * sizeof(double), A, (size_t)lda * sizeof(double),
                        (size_t)m * sizeof(double), n, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B, b, (size_t)m * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&st_before, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "fallback: %s", cudaGetErrorString(e));
  st = slqr_factor(ctx, m, n, A64, m, up, wy, s);
  if (st == SLQR_OK) st = slqr_apply_qt(ctx, m, n, A64, m, up, wy, 1, B, m, s);
  if (st == SLQR_OK) st = slqr_solve_r(ctx, n, A64, m, 1, B, m, s);
  if (st != SLQR_OK) return st;
  int st_after = 0;
  e = cudaMemcpyAsync(x, B, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&st_after, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "fallback: %s", cudaGetErrorString(e));
  if (st_before == 0 && st_after != 0) {      // raised by this solve: report it here
    cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
    return st_after;
  }
  return SLQR_OK;
}

// Bytes of the persistent state of one low-precision factorization (kept by
// the request loop for resident mixed-precision handles): the FP32 copy of
// A D (columns padded to 128 bytes), up, the compact-WY store, the column
// scales D and the explicit T of every panel.
size_t mixed_state_bytes(int m, int n) {
  const int nb = panel_width(m, n), K = num_reflectors(m, n), np = num_panels(K, nb);
  const int lda32 = (m + 31) / 32 * 32;
  size_t b = 0;
  b += align_up((size_t)lda32 * n * sizeof(float), 256);
  b += align_up((size_t)n * sizeof(double), 256);
  b += align_up(wy_panel_doubles(nb) * (size_t)std::max(np, 1) * sizeof(double), 256);
  b += align_up((size_t)n * sizeof(double), 256);
  b += align_up((size_t)std::max(np, 1) * nb * (nb + 1) * sizeof(float), 256);
  return b;
}

static void mixed_state_carve(char *mem, int m, int n, int prec, MixedFactorState *fs) {
  fs->m = m; fs->n = n; fs->prec = prec;
  fs->nb = panel_width(m, n); fs->K = num_reflectors(m, n); fs->np = num_panels(fs->K, fs->nb);
  fs->lda32 = (m + 31) / 32 * 32;
  size_t off = 0;
  auto take = [&](size_t bytes) { char *p = mem + off; off += align_up(bytes, 256); return p; };
  fs->A32 = (float *)take((size_t)fs->lda32 * n * sizeof(float));
  fs->up = (double *)take((size_t)n * sizeof(double));
  fs->wy = (double *)take(wy_panel_doubles(fs->nb) * (size_t)std::max(fs->np, 1) * sizeof(double));
  fs->colscale = (double *)take((size_t)n * sizeof(double));
  fs->Tm32 = (float *)take((size_t)std::max(fs->np, 1) * fs->nb * (fs->nb + 1) * sizeof(float));
}

static size_t factor_scratch_bytes(int m, int n, int prec) {
  const int lda32 = (m + 31) / 32 * 32;
  return (prec == SLQR_BF16X3) ? 2 * align_up((size_t)lda32 * n * 2, 256) : 0;
}

// The low-precision factorization of A D into the state `fs` (memory carved
// already); `scratch` holds the BF16 shadows of SLQR_BF16X3.
static slqr_status factor_phase(slqr_ctx *ctx, const double *A, int lda, MixedFactorState &fs,
                                char *scratch, cudaStream_t s) {
  const int m = fs.m, n = fs.n, prec = fs.prec;
  col_scale_kernel<<<(n * 32 + 255) / 256, 256, 0, s>>>(A, lda, m, n, fs.colscale);
  to_f32_kernel<<<4 * ctx->num_sms, 256, 0, s>>>(A, lda, m, n, fs.colscale, fs.A32, fs.lda32);
  ctx->launch_count += 2;
  ctx->tc_mode = (prec == SLQR_TF32) ? 1 : (prec == SLQR_BF16X3) ? 2 : 0;
  if (prec == SLQR_BF16X3) {
    ctx->sh_hi = scratch;
    ctx->sh_lo = scratch + align_up((size_t)fs.lda32 * n * 2, 256);
    split_bf16_region(fs.A32, fs.lda32, 0, m, 0, n, ctx->sh_hi, ctx->sh_lo, ctx->num_sms, s);
  }
  slqr_status st = factor_f32(ctx, m, n, fs.A32, fs.lda32, fs.up, fs.wy, s, fs.ntop);
  ctx->tc_mode = 0;
  ctx->sh_hi = ctx->sh_lo = nullptr;
  if (st != SLQR_OK) return st;
  if (fs.np > 0) {
    tmat_kernel<float><<<fs.np, 64, 0, s>>>(fs.wy, fs.nb, fs.K, fs.Tm32);
    ++ctx->launch_count;
  }
  return check_launch(ctx, "mixed factorization");
}

// Layout of the refinement's scratch (carved from `base` when not NULL).
static size_t refine_scratch(slqr_ctx *ctx, const MixedFactorState &fs, bool use_gmres,
                             int restart, char *base, MixedSolve *ms) {
  const int m = fs.m, n = fs.n, nb = fs.nb, np = fs.np;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t of = off; off = align_up(off + bytes, 256); return of; };
  const int chunks = (n + kColChunk - 1) / kColChunk, ublocks = (n + 255) / 256;
  const size_t N = (size_t)m + n;
  const int max_blocks = std::max(ublocks, std::min(4 * ctx->num_sms, (int)((N + 255) / 256)));
  const int qv_R = std::max(kQvRows, ((m + ctx->num_sms - 1) / ctx->num_sms + 63) / 64 * 64);
  const int qv_P = (m + qv_R - 1) / qv_R;
  const int qv_R64 = std::max(kQvRows64, ((m + ctx->num_sms - 1) / ctx->num_sms + 63) / 64 * 64);
  const int qv_P64 = (m + qv_R64 - 1) / qv_R64;
  const size_t t_elems = (size_t)std::max(np, 1) * nb * (nb + 1);
  const int nblk64 = (n + 63) / 64;
  const size_t o_r = take((size_t)m * sizeof(double));
  const size_t o_f = take((size_t)m * sizeof(float));
  const size_t o_g = take((size_t)n * sizeof(float));
  const size_t o_e = take((size_t)m * sizeof(float));
  const size_t o_part = take((size_t)chunks * m * sizeof(double));
  const size_t o_max = take((size_t)2 * max_blocks * sizeof(double));
  const size_t o_flag = take(sizeof(int));
  const size_t o_qpart = take((size_t)2 * qv_P * nb * sizeof(float));
  const size_t o_bar = take(256);
  const size_t o_dr = take(2 * sizeof(double));
  const size_t o_tm64 = use_gmres ? take(t_elems * sizeof(double)) : 0;
  const size_t o_qpart64 = use_gmres ? take((size_t)2 * qv_P64 * nb * sizeof(double)) : 0;
  const size_t o_vk = use_gmres ? take((size_t)(restart + 1) * N * sizeof(double)) : 0;
  const size_t o_h = use_gmres ? take((size_t)2 * (restart + 2) * sizeof(double)) : 0;
  const size_t o_y = use_gmres ? take((size_t)restart * sizeof(double)) : 0;
  const size_t o_rinv = use_gmres ? take((size_t)nblk64 * 4096 * sizeof(double)) : 0;
  const size_t o_zblk = use_gmres ? take((size_t)nblk64 * sizeof(int)) : 0;
  const size_t o_rinv32 = take((size_t)nblk64 * 4096 * sizeof(float));
  const size_t o_zblk32 = take((size_t)nblk64 * sizeof(int));
  if (base && ms) {
    ms->ctx = ctx; ms->m = m; ms->n = n; ms->nb = nb; ms->K = fs.K; ms->np = np;
    ms->lda32 = fs.lda32; ms->chunks = chunks; ms->ublocks = ublocks;
    ms->A32 = fs.A32; ms->up = fs.up; ms->wy = fs.wy; ms->colscale = fs.colscale;
    ms->Tm32 = fs.Tm32;
    ms->qv_R = qv_R; ms->qv_P = qv_P; ms->qv_R64 = qv_R64; ms->qv_P64 = qv_P64;
    ms->r = (double *)(base + o_r);
    ms->f32 = (float *)(base + o_f);
    ms->g32 = (float *)(base + o_g);
    ms->e32 = (float *)(base + o_e);
    ms->part = (double *)(base + o_part);
    ms->maxima = (double *)(base + o_max);
    ms->zero_flag = (int *)(base + o_flag);
    ms->qpart32 = (float *)(base + o_qpart);
    ms->qbar = (unsigned *)(base + o_bar);
    ms->drange = (double *)(base + o_dr);
    ms->Rinv32 = (float *)(base + o_rinv32);
    ms->zblk32 = (int *)(base + o_zblk32);
    if (use_gmres) {
      ms->Tm64 = (double *)(base + o_tm64);
      ms->qpart64 = (double *)(base + o_qpart64);
      ms->Vk = (double *)(base + o_vk);
      ms->hdev = (double *)(base + o_h);
      ms->ydev = (double *)(base + o_y);
      ms->Rinv = (double *)(base + o_rinv);
      ms->zblk = (int *)(base + o_zblk);
      ms->restart = restart;
    }
  }
  return off;
}

static int gmres_budget(const slqr_mixed_opts &o) {
  return o.gmres_max_iters > 0 ? o.gmres_max_iters : 300;
}
static int gmres_restart_len(const slqr_mixed_opts &o) {
  const int it = gmres_budget(o);
  const int r = o.gmres_restart > 0 ? o.gmres_restart : std::min(it, 200);
  return std::max(1, std::min(r, kMaxKrylov));
}

// The refinement of x for b with the low-precision factorization `fs` of the
// FP64 matrix A (Bjorck sweeps, then or instead GMRES-IR, then the optional
// FP64 fallback); `scratch` as laid out by refine_scratch.
static slqr_status refine_phase(slqr_ctx *ctx, const MixedFactorState &fs, const double *A,
                                int lda, const double *b, double *x, const slqr_mixed_opts &o,
                                slqr_mixed_info *info, char *scratch, cudaStream_t s) {
  const int m = fs.m, n = fs.n;
  const bool use_gmres = o.refine != SLQR_REFINE_BJORCK;
  const bool use_bjorck = o.refine != SLQR_REFINE_GMRES;
  MixedSolve ms;
  refine_scratch(ctx, fs, use_gmres, gmres_restart_len(o), scratch, &ms);
  ms.s = s; ms.lda = lda; ms.A = A; ms.b = b; ms.x = x;
  cudaError_t e = cudaFuncSetAttribute(qvec_kernel<float>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)qvec_smem_bytes<float>(fs.nb, ms.qv_R));
  if (e == cudaSuccess && use_gmres)
    e = cudaFuncSetAttribute(qvec_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)qvec_smem_bytes<double>(fs.nb, ms.qv_R64));
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "qvec attribute: %s", cudaGetErrorString(e));
  cudaMemsetAsync(ms.qbar, 0, 256, s);
  cudaMemsetAsync(ms.zero_flag, 0, sizeof(int), s);
  slqr_status st;
  info->method = SLQR_REFINE_BJORCK;
  int status = SLQR_ENOCONV;
  if (use_bjorck) {
    double e_cur = HUGE_VAL;
    status = bjorck(ms, o.max_sweeps, o.tol, &info->sweeps, &e_cur);
    info->err = e_cur;
  } else {
    init_kernel<<<(m + 255) / 256, 256, 0, s>>>(ms.r, m, x, n);
    ++ctx->launch_count;
  }
  if (status == SLQR_ENOCONV && use_gmres) {
    if (fs.np > 0) {
      tmat_kernel<double><<<fs.np, 64, 0, s>>>(fs.wy, fs.nb, fs.K, ms.Tm64);
      ++ctx->launch_count;
    }
    // condition estimate from the diagonal of R: the FP64 noise level that a
    // converged refinement stalls at is about kappa * u
    diag_range_kernel<<<1, 256, 0, s>>>(fs.A32, fs.lda32, n, ms.drange);
    ++ctx->launch_count;
    double dr[2] = {0.0, 0.0};
    e = cudaMemcpyAsync(dr, ms.drange, sizeof(dr), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "GMRES-IR: %s", cudaGetErrorString(e));
    const double kappa_est = (dr[1] > 0.0) ? dr[0] / dr[1] : HUGE_VAL;
    // the FP64 inverses of R's diagonal blocks, once for all the triangular
    // solves of the preconditioner
    diag_inv_kernel<double><<<(n + 63) / 64, 64, 0, s>>>(fs.A32, fs.lda32, n, ms.Rinv, ms.zblk);
    ++ctx->launch_count;
    info->kappa_est = kappa_est;
    const double noise = std::max(kStallOk, 100.0 * kappa_est * std::ldexp(1.0, -53));
    if (use_bjorck) {
      // the Bjorck iterate may have diverged: start again from the plain solve
      init_kernel<<<(m + 255) / 256, 256, 0, s>>>(ms.r, m, x, n);
      ++ctx->launch_count;
    }
    GmresResult gr;
    const double inner_tol = o.gmres_tol > 0.0 ? o.gmres_tol : 1e-10;
    status = gmres_ir(ms, o.tol, gmres_budget(o), inner_tol, noise, &gr);
    info->method = SLQR_REFINE_GMRES;
    info->gmres_steps = gr.steps;
    info->gmres_iters = gr.iters;
    info->err = gr.err;
  }
  st = check_launch(ctx, "lstsq_mixed");
  if (st != SLQR_OK) return st;
  // a bounded device wait that gave up leaves the factorization or a
  // correction incomplete: report it (it stays in the status word for
  // slqr_sync as well)
  {
    int dstat = 0;
    e = cudaMemcpyAsync(&dstat, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "status word: %s", cudaGetErrorString(e));
    if (dstat == SLQR_ETIMEOUT) return fail(ctx, SLQR_ETIMEOUT, "a bounded device wait gave up");
  }
  if (status == SLQR_ENOCONV && o.fp64_fallback) {
    st = fp64_fallback(ctx, m, n, A, lda, b, x, s);
    if (st != SLQR_OK) return st;
    info->method = SLQR_REFINE_FP64;
    return SLQR_FALLBACK;
  }
  if (status != SLQR_OK)
    fail(ctx, status, status == SLQR_ENOCONV ? "refinement did not reach its tolerance"
                                             : "R has an exact zero on its diagonal");
  return status;
}

static slqr_status lstsq_mixed_impl(slqr_ctx *ctx, int m, int n, const double *A, int lda,
                                    const double *b, double *x, int prec,
                                    const slqr_mixed_opts &o, slqr_mixed_info *info,
                                    cudaStream_t s) {
  // the state first, then the larger of the two phases' scratch, in one
  // workspace of the context (the factorization itself uses ctx->ws)
  const bool use_gmres = o.refine != SLQR_REFINE_BJORCK;
  const size_t sbytes = align_up(mixed_state_bytes(m, n), 256);
  MixedFactorState fs;
  mixed_state_carve(nullptr, m, n, prec, &fs);     // sizes only
  const size_t rbytes = refine_scratch(ctx, fs, use_gmres, gmres_restart_len(o), nullptr, nullptr);
  const size_t fbytes = factor_scratch_bytes(m, n, prec);
  slqr_status st = ensure_workspace2(ctx, sbytes + std::max(rbytes, fbytes));
  if (st != SLQR_OK) return st;
  char *base = (char *)ctx->ws2.ptr;
  mixed_state_carve(base, m, n, prec, &fs);
  fs.ntop = (o.structure == SLQR_STACKED) ? n : 0;
  st = factor_phase(ctx, A, lda, fs, base + sbytes, s);
  if (st != SLQR_OK) return st;
  return refine_phase(ctx, fs, A, lda, b, x, o, info, base + sbytes, s);
}

// Internal entry points for the request loop (resident mixed factorizations).
slqr_status mixed_factor_into(slqr_ctx *ctx, int m, int n, const double *A, int lda, int prec,
                              int ntop, void *state_mem, MixedFactorState *fs, cudaStream_t s) {
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  slqr_status st = ensure_workspace2(ctx, std::max<size_t>(factor_scratch_bytes(m, n, prec), 256));
  if (st != SLQR_OK) return st;
  mixed_state_carve((char *)state_mem, m, n, prec, fs);
  fs->ntop = ntop;
  return factor_phase(ctx, A, lda, *fs, (char *)ctx->ws2.ptr, s);
}

slqr_status mixed_solve_with(slqr_ctx *ctx, const MixedFactorState &fs, const double *A, int lda,
                             const double *b, double *x, const slqr_mixed_opts &o,
                             slqr_mixed_info *info, cudaStream_t s) {
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  const bool use_gmres = o.refine != SLQR_REFINE_BJORCK;
  const size_t rbytes = refine_scratch(ctx, fs, use_gmres, gmres_restart_len(o), nullptr, nullptr);
  slqr_status st = ensure_workspace2(ctx, rbytes);
  if (st != SLQR_OK) return st;
  return refine_phase(ctx, fs, A, lda, b, x, o, info, (char *)ctx->ws2.ptr, s);
}

static slqr_status check_mixed_args(slqr_ctx *ctx, int m, int n, const double *A, int lda,
                                    const double *b, double *x, int prec) {
  if (m < 1 || n < 1 || m < n) return fail(ctx, SLQR_EINVAL, "need m >= n >= 1 (m=%d n=%d)", m, n);
  if (lda < m || !A || !b || !x) return fail(ctx, SLQR_EINVAL, "bad lda or NULL pointer");
  if (m > slqr_max_rows()) return fail(ctx, SLQR_EINVAL, "m=%d above slqr_max_rows()", m);
  if (prec != SLQR_FP32 && prec != SLQR_TF32 && prec != SLQR_BF16X3)
    return fail(ctx, SLQR_EINVAL, "precision %d not available", prec);
  return SLQR_OK;
}

}  // namespace slqr

using namespace slqr;

extern "C" slqr_status slqr_lstsq_mixed(slqr_ctx *ctx, int m, int n, const double *A, int lda,
                                        const double *b, double *x, int prec, int max_iter,
                                        double tol, int *iters, double *err, void *stream) {
  NvtxRange nvtx_range("slqr_lstsq_mixed");
  if (!ctx) return SLQR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  slqr_status st = check_mixed_args(ctx, m, n, A, lda, b, x, prec);
  if (st != SLQR_OK) return st;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  slqr_mixed_opts o = {};
  o.refine = SLQR_REFINE_BJORCK;
  o.max_sweeps = max_iter >= 1 ? max_iter : 30;
  o.tol = tol > 0.0 ? tol : 1e-14;
  slqr_mixed_info info = {};
  st = lstsq_mixed_impl(ctx, m, n, A, lda, b, x, prec, o, &info, (cudaStream_t)stream);
  if (iters) *iters = info.sweeps;
  if (err) *err = info.err;
  return st;
}

extern "C" slqr_status slqr_lstsq_mixed_ex(slqr_ctx *ctx, int m, int n, const double *A, int lda,
                                           const double *b, double *x, int prec,
                                           const slqr_mixed_opts *opts, slqr_mixed_info *info,
                                           void *stream) {
  NvtxRange nvtx_range("slqr_lstsq_mixed_ex");
  if (!ctx) return SLQR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  slqr_status st = check_mixed_args(ctx, m, n, A, lda, b, x, prec);
  if (st != SLQR_OK) return st;
  slqr_mixed_opts o = {};
  if (opts) o = *opts;
  if (o.refine < SLQR_REFINE_AUTO || o.refine > SLQR_REFINE_GMRES)
    return fail(ctx, SLQR_EINVAL, "refine = %d is not a refinement method", o.refine);
  if (o.gmres_restart > kMaxKrylov)
    return fail(ctx, SLQR_EINVAL, "gmres_restart = %d above %d", o.gmres_restart, kMaxKrylov);
  if (o.structure != SLQR_DENSE && o.structure != SLQR_STACKED)
    return fail(ctx, SLQR_EINVAL, "structure = %d", o.structure);
  if (o.max_sweeps < 1) o.max_sweeps = 30;
  if (!(o.tol > 0.0)) o.tol = 1e-14;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  slqr_mixed_info inf = {};
  inf.err = HUGE_VAL;
  st = lstsq_mixed_impl(ctx, m, n, A, lda, b, x, prec, o, &inf, (cudaStream_t)stream);
  if (info) *info = inf;
  return st;
}
