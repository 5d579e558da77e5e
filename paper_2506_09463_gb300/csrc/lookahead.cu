// Look-ahead update of an FP32 factorization in one cooperative launch.
//
// After panel p of Alg. 2 (compact-WY form Q_p = I - V T V^T), the columns of
// panel p+1 (at most 64) are updated first, X <- Q_p^T X = X - V T^T (V^T X),
// so that panel p+1 can be factored while the rest of the trailing matrix is
// updated.  These are two thin products (M x 64 by 64 x 64) and a 64-step
// triangular substitution; as three separate launches (partial V^T X, T^T W,
// X -= V W') each of them waited on its own launch and on a pass through HBM.
// Here one kernel on up to one CTA per SM does all of it:
//   1. CTA q stages its 32-row-aligned slice of V and X in shared memory and
//      forms the partial W_q = V_q^T X_q;
//   2. (grid barrier) CTA q sums columns q, q + P, .. of the partials in a
//      fixed order (so the result does not depend on timing) and forms those
//      columns of W' = T^T W by the substitution with
//      T^{-1} = striu(G) + diag(1 / tau) (G = striu(V^T V) and tau as stored
//      in the compact-WY panel);
//   3. (grid barrier) every CTA reads W' and updates its slice, X_q -= V_q W',
//      from the V and X still in its shared memory, and stores X_q.
// HBM traffic is the algorithmic minimum: V and X read once, X written once.
// The grid barriers are bounded (SLQR_ETIMEOUT after the spin limit).
#include "slqr_internal.cuh"

namespace slqr {
namespace {

constexpr int kLaNB = 64;          // panel width this kernel handles
constexpr int kLaThreads = 256;
constexpr int kLaRowsMax = 256;    // rows per CTA (shared memory: V and X slices)
constexpr int kGLd = kLaNB + 1;    // row stride of G in shared memory (row-major)

int g_fused_lookahead = 1;

struct LaParams {
  float *A;              // the FP32 matrix (column-major, leading dimension lda)
  int lda;
  const double *wy;      // compact-WY store of the panel: Vtop, G, tau
  int k0, nbw;           // panel offset and width
  int M;                 // rows of the panel, m - k0
  int cb, N;             // updated columns [cb, cb + N), N <= 64
  int RS, P;             // rows per CTA (multiple of 32), CTAs
  int vec;               // 16-byte loads of A allowed (alignment checked on the host)
  float *Wp;             // P x 64 x 64 partials [q][c][a]
  float *Wt;             // W' [a][c], 64 x 64
  unsigned *bar;         // grid-barrier counter (monotonic)
  unsigned bar_base;     // its value when this launch starts
  int *status;
  unsigned spin;
};

__host__ __device__ inline int la_ld(int RS) { return RS + 4; }   // = 4 (mod 32): LDS.128 at full rate

size_t la_smem_bytes(int RS) {
  return ((size_t)2 * kLaNB * la_ld(RS) + (size_t)kLaNB * kGLd + kLaNB + 4 * kLaNB) * sizeof(float);
}

__global__ void __launch_bounds__(kLaThreads) la_update_kernel(LaParams p) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_ok;
  const int LD = la_ld(p.RS);
  float *Vc = sm;                             // [a][r], stride LD
  float *Xc = Vc + (size_t)kLaNB * LD;        // [c][r], stride LD
  float *Ws = Xc + (size_t)kLaNB * LD;        // G row-major (stride 65), later W' [a][c]
  float *tau_s = Ws + kLaNB * kGLd;
  float *part = tau_s + kLaNB;                // [4][64]
  const int tid = threadIdx.x, q = blockIdx.x;
  if (!slqr_check(p.RS % 32 == 0 && p.RS <= kLaRowsMax && (long long)p.P * p.RS >= p.M &&
                      p.N >= 1 && p.N <= kLaNB && p.nbw >= 1 && p.nbw <= kLaNB &&
                      (int)gridDim.x == p.P,
                  p.status))
    return;                                   // (uniform: every CTA returns)
  const int r0 = q * p.RS;
  const int rows = min(p.RS, p.M - r0);
  const int rend = (rows + 31) & ~31;         // rows staged, zero-padded to 32

  // ---- stage V_q and X_q (and, for the CTAs that form a column of W', the
  // panel's G and tau) -----------------------------------------------------
  // Every thread stages the same number of 4-row pieces, K = rend / 16, in
  // batches of 4 whose loads are all issued before the first store.
  auto load_piece = [&](int idx, float4 &v4, float4 &x4) {
    const int quads = rend / 4;
    const int c = idx / quads, r = (idx - c * quads) * 4;
    const int gr = r0 + r;                    // panel row of the first of 4 rows
    float v[4] = {0.f, 0.f, 0.f, 0.f}, x[4] = {0.f, 0.f, 0.f, 0.f};
    if (c < p.nbw) {
      if (p.vec && gr >= p.nbw && gr + 3 < p.M) {
        const float4 t = *reinterpret_cast<const float4 *>(
            p.A + SLQR_IDX(p.k0 + gr, p.k0 + c, p.lda));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = gr + u;
          if (i < p.nbw) v[u] = (float)p.wy[i + c * kLaNB];      // Vtop: 0, up, tails
          else if (i < p.M) v[u] = p.A[SLQR_IDX(p.k0 + i, p.k0 + c, p.lda)];
        }
      }
    }
    if (c < p.N) {
      if (p.vec && gr + 3 < p.M) {
        const float4 t = *reinterpret_cast<const float4 *>(
            p.A + SLQR_IDX(p.k0 + gr, p.cb + c, p.lda));
        x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (gr + u < p.M) x[u] = p.A[SLQR_IDX(p.k0 + gr + u, p.cb + c, p.lda)];
      }
    }
    v4 = make_float4(v[0], v[1], v[2], v[3]);
    x4 = make_float4(x[0], x[1], x[2], x[3]);
  };
  {
    const bool has_col = q < p.N;
    double2 gv[kLaNB * kLaNB / 2 / kLaThreads];
    float tv = 0.f;
    if (has_col) {
      const double2 *g2 = reinterpret_cast<const double2 *>(p.wy + (size_t)kLaNB * kLaNB);
#pragma unroll
      for (int u = 0; u < kLaNB * kLaNB / 2 / kLaThreads; ++u) gv[u] = g2[tid + u * kLaThreads];
      if (tid < kLaNB) tv = (float)p.wy[2 * (size_t)kLaNB * kLaNB + tid];
    }
    const int quads = rend / 4;
    const int K = kLaNB * quads / kLaThreads;  // rend is a multiple of 32: exact
    for (int k = 0; k < K; k += 4) {
      float4 v4[4], x4[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (k + u < K) load_piece(tid + (k + u) * kLaThreads, v4[u], x4[u]);
      if (k == 0 && has_col) {
        // G (column-major in the store) into rows of stride 65
#pragma unroll
        for (int u = 0; u < kLaNB * kLaNB / 2 / kLaThreads; ++u) {
          const int e = 2 * (tid + u * kLaThreads);
          const int row = e & (kLaNB - 1), col = e >> 6;
          Ws[row * kGLd + col] = (float)gv[u].x;
          Ws[(row + 1) * kGLd + col] = (float)gv[u].y;
        }
        if (tid < kLaNB) tau_s[tid] = tv;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (k + u < K) {
          const int idx = tid + (k + u) * kLaThreads;
          const int c = idx / quads, r = (idx - c * quads) * 4;
          *reinterpret_cast<float4 *>(Vc + (size_t)c * LD + r) = v4[u];
          *reinterpret_cast<float4 *>(Xc + (size_t)c * LD + r) = x4[u];
        }
    }
  }
  __syncthreads();

  // ---- partial W_q[a][c] = sum_r V[r][a] X[r][c] (rows in order) -----------
  {
    const int tx = tid & 15, ty = tid >> 4;   // a = tx + 16 i, c = ty + 16 j
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int r = 0; r < rend; r += 4) {
      float4 va[4], xc[4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
        va[i] = *reinterpret_cast<const float4 *>(Vc + (size_t)(tx + 16 * i) * LD + r);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        xc[j] = *reinterpret_cast<const float4 *>(Xc + (size_t)(ty + 16 * j) * LD + r);
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
    float *out = p.Wp + (size_t)q * kLaNB * kLaNB;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int i = 0; i < 4; ++i) out[(ty + 16 * j) * kLaNB + tx + 16 * i] = acc[i][j];
  }
  if (!grid_barrier(p.bar, p.bar_base + (unsigned)p.P, p.status, &s_ok, p.spin)) return;

  // ---- columns of W = sum_q W_q, then W' = T^T W column by column ----------
  // CTA q owns the columns q, q + P, q + 2P, ..; it takes up to four of them
  // per round (one warp each for the substitution); the P partials of an
  // entry are summed by 4 / nc threads in a fixed order.
  {
    const int own = (q < p.N) ? (p.N - q + p.P - 1) / p.P : 0;
    const int nc = own >= 3 ? 4 : own;        // columns per round: 1, 2 or 4
    const int warp = tid >> 5, lane = tid & 31;
    for (int t0 = 0; t0 < own; t0 += nc) {
      const int TPE = 4 / nc;                 // threads per entry
      const int e = tid % (nc * kLaNB), h = tid / (nc * kLaNB);
      const int t = t0 + e / kLaNB, a = e % kLaNB;
      float sum = 0.f;
      if (t < own) {
        const float *src = p.Wp + (size_t)(q + t * p.P) * kLaNB + a;
        const size_t stride = (size_t)kLaNB * kLaNB * TPE;
        // partials h, h + TPE, h + 2 TPE, ..: sixteen independent loads per round
        float acc[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) acc[u] = 0.f;
        src += (size_t)h * kLaNB * kLaNB;
        for (int s = h; s < p.P; s += 16 * TPE, src += 16 * stride) {
          float v[16];
#pragma unroll
          for (int u = 0; u < 16; ++u)
            v[u] = (s + u * TPE < p.P) ? __ldcg(src + (size_t)u * stride) : 0.f;
#pragma unroll
          for (int u = 0; u < 16; ++u) acc[u] += v[u];
        }
#pragma unroll
        for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
          for (int u = 0; u < w; ++u) acc[u] += acc[u + w];
        sum = acc[0];
      }
      part[h * (nc * kLaNB) + e] = sum;       // [TPE][nc * 64]
      __syncthreads();
      if (warp < nc && t0 + warp < own) {
        // one warp per column, lane l holding entries l and l + 32; at step j
        // the entry w'_j = tau_j w_j is broadcast and folded into the
        // entries k > j with G[j, k] (the order of the FP32 tw_kernel)
        const int c = q + (t0 + warp) * p.P;
        float r0v = 0.f, r1v = 0.f;
        for (int hh = 0; hh < TPE; ++hh) {
          r0v += part[hh * (nc * kLaNB) + warp * kLaNB + lane];
          r1v += part[hh * (nc * kLaNB) + warp * kLaNB + lane + 32];
        }
        for (int j = 0; j < p.nbw; ++j) {
          const float wj = __shfl_sync(0xffffffffu, (j < 32) ? r0v : r1v, j & 31);
          const float wpj = tau_s[j] * wj;
          if (lane > j) r0v = fmaf(-Ws[j * kGLd + lane], wpj, r0v);
          if (lane + 32 > j) r1v = fmaf(-Ws[j * kGLd + lane + 32], wpj, r1v);
          if (lane == (j & 31)) {
            if (j < 32) r0v = wpj;
            else r1v = wpj;
          }
        }
        p.Wt[lane * kLaNB + c] = (lane < p.nbw) ? r0v : 0.f;
        p.Wt[(lane + 32) * kLaNB + c] = (lane + 32 < p.nbw) ? r1v : 0.f;
      }
      __syncthreads();                        // part, before the next round
    }
  }
  if (!grid_barrier(p.bar, p.bar_base + 2u * (unsigned)p.P, p.status, &s_ok, p.spin)) return;

  // ---- X_q -= V_q W' ---------------------------------------------------------
  {
    float4 t[kLaNB * kLaNB / 4 / kLaThreads];
#pragma unroll
    for (int u = 0; u < kLaNB * kLaNB / 4 / kLaThreads; ++u)
      t[u] = __ldcg(reinterpret_cast<const float4 *>(p.Wt) + tid + u * kLaThreads);
#pragma unroll
    for (int u = 0; u < kLaNB * kLaNB / 4 / kLaThreads; ++u)
      reinterpret_cast<float4 *>(Ws)[tid + u * kLaThreads] = t[u];
  }
  __syncthreads();
  {
    const int lane = tid & 31, cg = tid >> 5;  // rows lane (+32), columns 8 cg .. 8 cg + 7
    for (int rb = 0; rb < rend; rb += 64) {
      const bool two = rb + 32 < rend;        // (uniform)
      const int ra = rb + lane, rbb = rb + 32 + lane;
      float acc0[8], acc1[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) acc0[k] = acc1[k] = 0.f;
      for (int a = 0; a < p.nbw; ++a) {
        const float v0 = Vc[(size_t)a * LD + ra];
        const float v1 = two ? Vc[(size_t)a * LD + rbb] : 0.f;
        const float4 w0 = *reinterpret_cast<const float4 *>(Ws + a * kLaNB + cg * 8);
        const float4 w1 = *reinterpret_cast<const float4 *>(Ws + a * kLaNB + cg * 8 + 4);
        const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          acc0[k] = fmaf(v0, w[k], acc0[k]);
          acc1[k] = fmaf(v1, w[k], acc1[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int c = cg * 8 + k;
        if (c < p.N) {
          if (ra < rows)
            p.A[SLQR_IDX(p.k0 + r0 + ra, p.cb + c, p.lda)] = Xc[(size_t)c * LD + ra] - acc0[k];
          if (two && rbb < rows)
            p.A[SLQR_IDX(p.k0 + r0 + rbb, p.cb + c, p.lda)] = Xc[(size_t)c * LD + rbb] - acc1[k];
        }
      }
    }
  }
}

}  // namespace

slqr_status init_lookahead_attrs(slqr_ctx *ctx) {
  (void)ctx;
  cudaError_t e = cudaFuncSetAttribute(la_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)la_smem_bytes(kLaRowsMax));
  return e == cudaSuccess ? SLQR_OK : SLQR_ECUDA;
}

int fused_lookahead_setting() { return g_fused_lookahead; }
void set_fused_lookahead(int on) { g_fused_lookahead = on ? 1 : 0; }

bool lookahead_update_f32(slqr_ctx *ctx, int m, int k0, int nbw, float *A, int lda,
                          const double *wy_panel, int cb, int N, float *work, size_t work_elems,
                          unsigned *bar, unsigned &bar_base, cudaStream_t stream,
                          slqr_status *st) {
  if (!g_fused_lookahead || nbw < 1 || nbw > kLaNB || N < 1 || N > kLaNB) return false;
  const int M = m - k0;
  if (M < 1) return false;
  const int P0 = ctx->num_sms;
  int RS = (M + P0 - 1) / P0;
  RS = (RS + 31) / 32 * 32;
  if (RS > kLaRowsMax) return false;
  const int P = (M + RS - 1) / RS;
  const size_t need = (size_t)P * kLaNB * kLaNB + (size_t)kLaNB * kLaNB;
  if (need > work_elems || ((uintptr_t)work & 15) != 0 || ((uintptr_t)wy_panel & 15) != 0)
    return false;
  LaParams lp;
  lp.A = A; lp.lda = lda; lp.wy = wy_panel; lp.k0 = k0; lp.nbw = nbw; lp.M = M;
  lp.cb = cb; lp.N = N; lp.RS = RS; lp.P = P;
  lp.vec = (lda % 4 == 0 && ((uintptr_t)A & 15) == 0 && k0 % 4 == 0) ? 1 : 0;
  lp.Wp = work; lp.Wt = work + (size_t)P * kLaNB * kLaNB;
  lp.bar = bar; lp.bar_base = bar_base;
  lp.status = ctx->d_status; lp.spin = ctx->spin_limit;
  void *args[] = {&lp};
  const double flops = 4.0 * M * nbw * (double)N;
  int slot = prof_begin(ctx, stream);
  cudaError_t e = cudaLaunchCooperativeKernel((const void *)la_update_kernel, dim3(P),
                                              dim3(kLaThreads), args, la_smem_bytes(RS), stream);
  prof_end(ctx, stream, slot, kUpd, flops);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();                 // not launched: the caller takes the tiled path
    return false;
  }
  bar_base += 2u * (unsigned)P;
  *st = SLQR_OK;
  return true;
}

}  // namespace slqr

extern "C" slqr_status slqr_set_fused_lookahead(int enable) {
  if (enable != 0 && enable != 1) return SLQR_EINVAL;
  slqr::set_fused_lookahead(enable);
  return SLQR_OK;
}

extern "C" int slqr_get_fused_lookahead(void) { return slqr::fused_lookahead_setting(); }
