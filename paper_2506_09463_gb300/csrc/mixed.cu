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
// A refinement whose steps stop contracting is accepted when its last step is
// below this (the 1e-10 solution-error target): the step then measures the
// FP64 noise level kappa * eps of an ill-conditioned problem.
constexpr double kStallOk = 1e-10;
constexpr int kColChunk = 256;

// A32 = (float) A
__global__ void to_f32_kernel(const double *__restrict__ A, int lda, int m, int n,
                              float *__restrict__ A32, int lda32) {
  const size_t total = (size_t)lda32 * n;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx / lda32), i = (int)(idx - (size_t)j * lda32);
    A32[idx] = (i < m) ? (float)A[SLQR_IDX(i, j, lda)] : 0.f;
  }
}

// partial row sums of A x over column chunks: part[chunk][i]
__global__ void __launch_bounds__(kRowsPerCta)
ax_partial_kernel(const double *__restrict__ A, int lda, int m, int n,
                  const double *__restrict__ x, double *__restrict__ part) {
  const int i = blockIdx.x * kRowsPerCta + threadIdx.x;
  const int j0 = blockIdx.y * kColChunk, j1 = min(n, j0 + kColChunk);
  __shared__ double xs[kColChunk];
  for (int j = j0 + threadIdx.x; j < j1; j += kRowsPerCta) xs[j - j0] = x[j];
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

// g = -A^T r (one warp per column), g32 = (float) g
__global__ void resid_g_kernel(const double *__restrict__ A, int lda, int m, int n,
                               const double *__restrict__ r, float *__restrict__ g32) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  double acc = 0.0;
  for (int i = lane; i < m; i += 32) acc = fma(A[SLQR_IDX(i, warp, lda)], r[i], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) g32[warp] = (float)(-acc);
}

// e[0:n] = d[0:n] - h ; keep d[n:m] in e (e aliases nothing)
__global__ void form_e_kernel(const float *__restrict__ d, const float *__restrict__ h, int m,
                              int n, float *__restrict__ e) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) e[i] = (i < n) ? d[i] - h[i] : d[i];
}

// d[0:n] = h (so that d = [h; d2]); x += dx (FP64); per-CTA maxima of |dx|, |x|
__global__ void update_kernel(float *__restrict__ d, const float *__restrict__ h,
                              const float *__restrict__ dx, double *__restrict__ x, int n,
                              double *__restrict__ maxima) {
  __shared__ double s_dx[256], s_x[256];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double a = 0.0, c = 0.0;
  if (i < n) {
    d[i] = h[i];
    const double v = (double)dx[i];
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

// T of panel p (float, ld nb + 1): column j solves U y = e_j by back
// substitution with U = striu(G) + diag(1/tau), i.e. y_j = tau_j and
// y_i = -tau_i sum_{k=i+1..j} G[i,k] y_k (tau = 0: a zero row and column).
__global__ void __launch_bounds__(64)
tmat_kernel(const double *__restrict__ wy, int nb, int K, float *__restrict__ Tm) {
  __shared__ double ys[64][65];
  const int pnl = blockIdx.x, j = threadIdx.x;
  const int nbw = min(nb, K - pnl * nb);
  const double *G = wy + (size_t)pnl * wy_panel_doubles(nb) + (size_t)nb * nb;
  const double *tau = G + (size_t)nb * nb;
  float *T = Tm + (size_t)pnl * nb * (nb + 1);
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
    for (int i = 0; i < nb; ++i) T[i + (size_t)j * (nb + 1)] = (float)ys[i][j];
  }
}

struct QvecParams {
  const float *A;        // FP32 factorization (H12 form), ld lda
  const double *up;      // pivot entries of the reflectors
  const float *Tm;       // explicit T of each panel, nb x nb, ld nb + 1
  float *f;              // the vector, m entries, updated in place
  float *part;           // 2 buffers x P CTAs x nb partial sums
  unsigned *bar;         // monotonic arrival counter
  int *status;
  int lda, m, K, nb, np;
  int trans;             // 1: Q^T f, 0: Q f
  int R, P;
  unsigned bar_base;
};

__global__ void __launch_bounds__(kThreads)
qvec_kernel(QvecParams p) {
  extern __shared__ __align__(16) float qv_smem[];
  const int nb = p.nb, R = p.R;
  const int tsz = nb * (nb + 1);                // one T (multiple of 4 floats)
  float *Ts2 = qv_smem;                         // [2][nb][nb + 1], 16-byte aligned
  float *Vs = Ts2 + 2 * tsz;                    // [nb][R + 1]
  float *fs = Vs + (size_t)nb * (R + 1);        // [R]
  float *red = fs + R;                          // [kThreads / nb][nb]
  float *ws = red + kThreads;                   // [nb]
  float *wt = ws + nb;                          // [nb]
  __shared__ int s_ok;
  const int tid = threadIdx.x, cta = blockIdx.x;
  const int r0 = cta * R, r1 = min(p.m, r0 + R);
  // T of a panel into buffer `buf` with asynchronous 16-byte copies
  auto fetch_t = [&](int step, int buf) {
    if (step >= p.np) return;
    const int pnl = p.trans ? step : p.np - 1 - step;
    const float *src = p.Tm + (size_t)pnl * tsz;
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(Ts2 + buf * tsz);
    for (int c = tid; c < tsz / 4; c += kThreads)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(dst + 16 * c), "l"(src + 4 * c)
                   : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  fetch_t(0, 0);
  for (int step = 0; step < p.np; ++step) {
    const int pnl = p.trans ? step : p.np - 1 - step;
    float *Ts = Ts2 + (step & 1) * tsz;
    const int k0 = pnl * nb, nbw = min(nb, p.K - k0);
    const int lo = max(r0, k0), rows = max(0, r1 - lo);
    float *mypart = p.part + ((size_t)(step & 1) * p.P + cta) * nb;
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
      float acc = 0.f;
      if (a < nbw)
        for (int rr = g; rr < rows; rr += G) acc = fmaf(Vs[a * (R + 1) + rr], fs[rr], acc);
      red[g * nb + a] = acc;
      __syncthreads();
      if (tid < nb) {
        float v = 0.f;
        for (int q = 0; q < G; ++q) v += red[q * nb + tid];
        mypart[tid] = v;
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");      // this panel's T has landed
    if (!grid_barrier(p.bar, p.bar_base + (unsigned)(step + 1) * (unsigned)p.P, p.status, &s_ok))
      return;
    fetch_t(step + 1, (step + 1) & 1);                   // the next panel's T, in flight
    // phase B: W (all CTAs, fixed order: thread (a, g) sums the partials of
    // CTAs g, g + G, .. with four loads in flight, then the G sums are added),
    // then W' = T^T W or T W
    {
      const int a = tid % nb, g = tid / nb, G = kThreads / nb;
      const float *src = p.part + (size_t)(step & 1) * p.P * nb + a;
      float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
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
        float v = 0.f;
        for (int gg = 0; gg < G; ++gg) v += red[gg * nb + tid];
        ws[tid] = v;
      }
    }
    __syncthreads();
    {
      // W' entry j: four threads take every fourth term of its dot product
      const int j = tid >> 2, part = tid & 3;
      float v = 0.f;
      if (j < nbw) {
        if (p.trans) {
          for (int q = part; q <= j; q += 4) v = fmaf(Ts[q + j * (nb + 1)], ws[q], v);
        } else {
          for (int q = j + part; q < nbw; q += 4) v = fmaf(Ts[j + q * (nb + 1)], ws[q], v);
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
      float v = 0.f;
      if (rr < rows)
        for (int a = half; a < nbw; a += 2) v = fmaf(-Vs[a * (R + 1) + rr], wt[a], v);
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      if (rr < rows && half == 0) p.f[lo + rr] = fs[rr] + v;
    } else {
      for (int rr = tid; rr < rows; rr += kThreads) {
        float v = fs[rr];
        for (int a = 0; a < nbw; ++a) v = fmaf(-Vs[a * (R + 1) + rr], wt[a], v);
        p.f[lo + rr] = v;
      }
    }
    __syncthreads();
  }
}

static size_t qvec_smem_bytes(int nb, int R) {
  return sizeof(float) * (2 * (size_t)nb * (nb + 1) + (size_t)nb * (R + 1) + R + kThreads + 2 * nb);
}

// FP32 triangular solve with R = triu(A32[0:n, 0:n]) (ld lda) in one
// cooperative launch.  UPPER: R y = c, 64-row blocks from the bottom; else
// R^T y = c, blocks from the top.  CTA q owns the row blocks t = q (mod P).
// Step b: the owner of block b solves its diagonal block (one warp, the
// updates of every earlier step already applied to it), one grid barrier
// publishes x_b, and every CTA subtracts R_tb x_b (or R_bt^T x_b) from each of
// its blocks t still to be solved.  An exact zero on the diagonal sets that
// entry of y to 0 and raises *zero_flag.
struct TrsvParams {
  const float *R;
  float *y;
  int *zero_flag;
  unsigned *bar;
  int *status;
  int lda, n, nblk, P;
  unsigned bar_base;
};

template <bool UPPER>
__global__ void __launch_bounds__(kThreads)
trsv_coop_kernel(TrsvParams p) {
  __shared__ float Rs[64][65];      // diagonal block being solved
  __shared__ float Tu[64][65];      // update tile, [c][r]: R[t r, b c] (UPPER) or R[b c, t r]
  __shared__ float rdiag[64];
  __shared__ float xs[64];
  __shared__ float red[4][64];
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
    if (tid < 64) rdiag[tid] = (tid < rows && Rs[tid][tid] != 0.f) ? 1.f / Rs[tid][tid] : 0.f;
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
  if (one) load_diag(cta);
  for (int step = 0; step < p.nblk; ++step) {
    const int b = UPPER ? p.nblk - 1 - step : step;
    const int b0 = b * 64, rows = min(64, p.n - b0);
    if (b % p.P == cta) {
      if (!one) load_diag(b);
      if (tid < 64) xs[tid] = (tid < rows) ? p.y[b0 + tid] : 0.f;
      __syncthreads();
      if (tid < 32) {
        float c0 = xs[lane], c1 = xs[lane + 32];
        bool zero = false;
        for (int s = 0; s < rows; ++s) {
          const int i = UPPER ? rows - 1 - s : s;
          const float ci = __shfl_sync(0xffffffffu, i < 32 ? c0 : c1, i & 31);
          const float rd = rdiag[i];
          const float xi = ci * rd;
          zero |= (rd == 0.f);
          if (lane == (i & 31)) {
            if (i < 32) c0 = xi; else c1 = xi;
          }
          if (UPPER) {
            if (lane < i) c0 = fmaf(-Rs[lane][i], xi, c0);
            if (lane + 32 < i) c1 = fmaf(-Rs[lane + 32][i], xi, c1);
          } else {
            if (lane > i) c0 = fmaf(-Rs[lane][i], xi, c0);
            if (lane + 32 > i && lane + 32 < rows) c1 = fmaf(-Rs[lane + 32][i], xi, c1);
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
    if (!grid_barrier(p.bar, p.bar_base + (unsigned)(step + 1) * (unsigned)p.P, p.status, &s_ok))
      return;
    if (tid < 64) xs[tid] = (tid < rows) ? __ldcg(p.y + b0 + tid) : 0.f;
    __syncthreads();
    for (int t = cta; t < p.nblk; t += p.P) {
      if (UPPER ? t >= b : t <= b) continue;
      if (!one) {
        load_update(t, b);
        __syncthreads();
      }
      const int t0 = t * 64, trows = min(64, p.n - t0);
      const int r = tid & 63, q = tid >> 6;
      float acc = 0.f;
      for (int c = q; c < rows; c += 4) acc = fmaf(Tu[c][r], xs[c], acc);
      red[q][r] = acc;
      __syncthreads();
      if (tid < trows) p.y[t0 + tid] -= (red[0][tid] + red[1][tid]) + (red[2][tid] + red[3][tid]);
      __syncthreads();
    }
  }
}

}  // namespace slqr

namespace slqr {

template <bool UPPER>
static slqr_status trsv_f32(slqr_ctx *ctx, const float *R, int lda, int n, float *y, int *zero_flag,
                            unsigned *bar, unsigned &bar_base, cudaStream_t s) {
  TrsvParams tp;
  tp.R = R; tp.y = y; tp.zero_flag = zero_flag; tp.bar = bar; tp.status = ctx->d_status;
  tp.lda = lda; tp.n = n; tp.nblk = (n + 63) / 64;
  tp.P = std::min(tp.nblk, ctx->num_sms);
  tp.bar_base = bar_base;
  void *args[] = {&tp};
  cudaError_t e = cudaLaunchCooperativeKernel((const void *)trsv_coop_kernel<UPPER>, dim3(tp.P),
                                              dim3(kThreads), args, 0, s);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "triangular solve: %s", cudaGetErrorString(e));
  bar_base += (unsigned)tp.nblk * (unsigned)tp.P;
  return SLQR_OK;
}

}  // namespace slqr

using namespace slqr;

extern "C" slqr_status slqr_lstsq_mixed(slqr_ctx *ctx, int m, int n, const double *A, int lda,
                                        const double *b, double *x, int prec, int max_iter,
                                        double tol, int *iters, double *err, void *stream) {
  NvtxRange nvtx_range("slqr_lstsq_mixed");
  if (!ctx) return SLQR_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (m < 1 || n < 1 || m < n) return fail(ctx, SLQR_EINVAL, "need m >= n >= 1 (m=%d n=%d)", m, n);
  if (lda < m || !A || !b || !x) return fail(ctx, SLQR_EINVAL, "bad lda or NULL pointer");
  if (m > slqr_max_rows()) return fail(ctx, SLQR_EINVAL, "m=%d above slqr_max_rows()", m);
  if (prec != SLQR_FP32 && prec != SLQR_TF32 && prec != SLQR_BF16X3)
    return fail(ctx, SLQR_EINVAL, "precision %d not available", prec);
  if (max_iter < 1) max_iter = 30;
  if (!(tol > 0.0)) tol = 1e-14;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = panel_width(m, n);
  const int K = num_reflectors(m, n);
  const int np = num_panels(K, nb);
  const int chunks = (n + kColChunk - 1) / kColChunk;
  const int ublocks = (n + 255) / 256;
  // mixed-path buffers (a workspace of their own: the factorization uses ctx->ws)
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  const int lda32 = (m + 31) / 32 * 32;   // 128-byte aligned columns (TMA-friendly)
  const size_t o_a32 = take((size_t)lda32 * n * sizeof(float));
  const size_t o_up = take((size_t)n * sizeof(double));
  const size_t o_wy = take(wy_panel_doubles(nb) * (size_t)std::max(np, 1) * sizeof(double));
  const size_t o_r = take((size_t)m * sizeof(double));
  const size_t o_f = take((size_t)m * sizeof(float));
  const size_t o_g = take((size_t)n * sizeof(float));
  const size_t o_e = take((size_t)m * sizeof(float));
  const size_t o_part = take((size_t)chunks * m * sizeof(double));
  const size_t o_max = take((size_t)2 * ublocks * sizeof(double));
  const size_t o_flag = take(sizeof(int));
  // fused Q application: rows per CTA, explicit T per panel, partials, barrier
  // (a multiple of 64 rows: every slice starts 16-byte aligned for the vector loads)
  const int qv_R = std::max(kQvRows, ((m + ctx->num_sms - 1) / ctx->num_sms + 63) / 64 * 64);
  const int qv_P = (m + qv_R - 1) / qv_R;
  const size_t o_tm = take((size_t)std::max(np, 1) * nb * (nb + 1) * sizeof(float));
  const size_t o_qpart = take((size_t)2 * qv_P * nb * sizeof(float));
  const size_t o_bar = take(256);
  // BF16 hi / lo shadows of the FP32 matrix (SLQR_BF16X3)
  const size_t sh_bytes = (prec == SLQR_BF16X3) ? (size_t)lda32 * n * 2 : 0;
  const size_t o_shh = take(sh_bytes);
  const size_t o_shl = take(sh_bytes);
  slqr_status st = ensure_workspace2(ctx, off);
  if (st != SLQR_OK) return st;
  char *base = (char *)ctx->ws2.ptr;
  float *A32 = (float *)(base + o_a32);
  double *up = (double *)(base + o_up);
  double *wy = (double *)(base + o_wy);
  double *r = (double *)(base + o_r);
  float *f32 = (float *)(base + o_f);
  float *g32 = (float *)(base + o_g);
  float *e32 = (float *)(base + o_e);
  double *part = (double *)(base + o_part);
  double *maxima = (double *)(base + o_max);
  int *zero_flag = (int *)(base + o_flag);
  float *Tm = (float *)(base + o_tm);
  float *qpart = (float *)(base + o_qpart);
  unsigned *qbar = (unsigned *)(base + o_bar);
  const size_t qv_smem = qvec_smem_bytes(nb, qv_R);
  e = cudaFuncSetAttribute(qvec_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qv_smem);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "qvec attribute: %s", cudaGetErrorString(e));
  unsigned qbar_base = 0;
  // f <- Q^T f (trans) or Q f with one cooperative launch
  auto apply_q = [&](bool trans) -> slqr_status {
    if (np == 0) return SLQR_OK;
    QvecParams qp;
    qp.A = A32; qp.up = up; qp.Tm = Tm; qp.f = f32; qp.part = qpart; qp.bar = qbar;
    qp.status = ctx->d_status; qp.lda = lda32; qp.m = m; qp.K = K; qp.nb = nb; qp.np = np;
    qp.trans = trans ? 1 : 0; qp.R = qv_R; qp.P = qv_P; qp.bar_base = qbar_base;
    void *args[] = {&qp};
    cudaError_t le = cudaLaunchCooperativeKernel((const void *)qvec_kernel, dim3(qv_P),
                                                 dim3(kThreads), args, qv_smem, s);
    if (le != cudaSuccess)
      return fail(ctx, SLQR_ECUDA, "Q application: %s", cudaGetErrorString(le));
    qbar_base += (unsigned)np * (unsigned)qv_P;
    return SLQR_OK;
  };

  to_f32_kernel<<<4 * ctx->num_sms, 256, 0, s>>>(A, lda, m, n, A32, lda32);
  ctx->tc_mode = (prec == SLQR_TF32) ? 1 : (prec == SLQR_BF16X3) ? 2 : 0;
  if (prec == SLQR_BF16X3) {
    ctx->sh_hi = base + o_shh;
    ctx->sh_lo = base + o_shl;
    split_bf16_region(A32, lda32, 0, m, 0, n, ctx->sh_hi, ctx->sh_lo, ctx->num_sms, s);
  }
  st = factor_f32(ctx, m, n, A32, lda32, up, wy, s);
  ctx->tc_mode = 0;
  ctx->sh_hi = ctx->sh_lo = nullptr;
  if (st != SLQR_OK) return st;
  if (np > 0) tmat_kernel<<<np, 64, 0, s>>>(wy, nb, K, Tm);
  cudaMemsetAsync(qbar, 0, 256, s);
  init_kernel<<<(m + 255) / 256, 256, 0, s>>>(r, m, x, n);
  cudaMemsetAsync(zero_flag, 0, sizeof(int), s);
  std::vector<double> hmax(2 * ublocks);
  int it = 0, status = SLQR_ENOCONV;
  double e_cur = 1.0, e_prev = 1e300;
  for (it = 1; it <= max_iter; ++it) {
    ax_partial_kernel<<<dim3((m + kRowsPerCta - 1) / kRowsPerCta, chunks), kRowsPerCta, 0, s>>>(
        A, lda, m, n, x, part);
    resid_f_kernel<<<(m + 255) / 256, 256, 0, s>>>(b, r, part, chunks, m, f32);
    resid_g_kernel<<<(n * 32 + 255) / 256, 256, 0, s>>>(A, lda, m, n, r, g32);
    st = trsv_f32<false>(ctx, A32, lda32, n, g32, zero_flag, qbar, qbar_base, s);  // h = R^-T g
    if (st != SLQR_OK) return st;
    st = apply_q(true);                                                 // d = Q^T f
    if (st != SLQR_OK) return st;
    form_e_kernel<<<(m + 255) / 256, 256, 0, s>>>(f32, g32, m, n, e32);
    st = trsv_f32<true>(ctx, A32, lda32, n, e32, zero_flag, qbar, qbar_base, s);   // dx = R^-1 (d1 - h)
    if (st != SLQR_OK) return st;
    update_kernel<<<ublocks, 256, 0, s>>>(f32, g32, e32, x, n, maxima);  // d = [h; d2], x += dx
    st = apply_q(false);                                                // dr = Q [h; d2]
    if (st != SLQR_OK) return st;
    add_r_kernel<<<(m + 255) / 256, 256, 0, s>>>(r, f32, m);
    int zflag = 0;
    e = cudaMemcpyAsync(hmax.data(), maxima, sizeof(double) * 2 * ublocks, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&zflag, zero_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "refinement: %s", cudaGetErrorString(e));
    double dmax = 0.0, xmax = 0.0;
    for (int k = 0; k < ublocks; ++k) {
      dmax = std::max(dmax, hmax[2 * k]);
      xmax = std::max(xmax, hmax[2 * k + 1]);
    }
    if (!std::isfinite(dmax) || !std::isfinite(xmax)) {   // overflow: never "converged"
      e_cur = HUGE_VAL;
      status = SLQR_ENOCONV;
      break;
    }
    e_cur = (xmax > 0.0) ? dmax / xmax : 0.0;
    if (zflag) { status = SLQR_ERANK; break; }
    if (e_cur <= tol) { status = SLQR_OK; break; }
    if (it >= 3 && e_cur > 0.5 * e_prev) {      // no longer contracting
      status = (e_cur <= kStallOk) ? SLQR_OK : SLQR_ENOCONV;
      break;
    }
    e_prev = e_cur;
  }
  if (iters) *iters = std::min(it, max_iter);
  if (err) *err = e_cur;
  st = check_launch(ctx, "lstsq_mixed");
  if (st != SLQR_OK) return st;
  if (status != SLQR_OK)
    fail(ctx, status, status == SLQR_ENOCONV ? "refinement did not reach its tolerance"
                                             : "R has an exact zero on its diagonal");
  return status;
}
