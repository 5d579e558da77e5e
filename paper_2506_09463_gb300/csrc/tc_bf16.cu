// tc_bf16.cu -- the two products of the compact-WY trailing update of the FP32
// factorization on the tensor cores with BF16 operands split in two
// (tcgen05 kind::f16, FP32 accumulation in tensor memory):
//   x = x_hi + x_lo,  x_hi = bf16(x),  x_lo = bf16(x - x_hi)
//   a . b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi
// Each BF16 value carries 8 significant bits, so the pair carries about 16
// and the dropped term a_lo b_lo is about 2^-16 |a b|: a product accurate to
// roughly 2^-15 relative instead of TF32's 2^-11, with three MMAs per product.
//
// The FP32 matrix keeps BF16 shadow copies of itself (hi and lo, same layout
// and leading dimension): the X -= V W' kernel writes the shadows of the tile
// it updates, the panel's columns are re-split after each panel, so W = V^T X
// reads both of its operands from the shadows with TMA and no conversion.
//   vtx_bf16_kernel  W = V^T X   (K = rows, 3-stage TMA ring, 12 MMAs a stage)
//   upd_bf16_kernel  X -= V W'   (K = 64 reflectors, 12 MMAs a tile)
#include "tc_common.cuh"

#include <cuda_bf16.h>
#include <algorithm>

namespace slqr {

typedef __nv_bfloat16 bf16;

constexpr int kBfTile = 128;                 // M side of the MMA
constexpr int kBfThreads = 128;
// D = F32, A = B = BF16, both K-major, M = 128, N = 64
constexpr uint32_t kIdescBf16N64 = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) |
                                   ((uint32_t)(kBfTile >> 4) << 24);

__device__ __forceinline__ void split_bf16(float x, bf16 &hi, bf16 &lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// hi/lo shadows of rows [r0, r1) x columns [c0, c1) of the FP32 matrix A
// (the shadows share A's leading dimension).
__global__ void split_bf16_kernel(const float *__restrict__ A, int lda, int r0, int r1, int c0,
                                  int c1, bf16 *__restrict__ hi, bf16 *__restrict__ lo) {
  const int rows = r1 - r0;
  const size_t total = (size_t)rows * (c1 - c0);
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int j = c0 + (int)(idx / rows), i = r0 + (int)(idx % rows);
    const size_t at = SLQR_IDX(i, j, lda);
    bf16 h, l;
    split_bf16(A[at], h, l);
    hi[at] = h;
    lo[at] = l;
  }
}

// Row-major V of the panel at k0 as hi/lo pairs (64 per row): rows i < 64 from
// Vtop (up on the diagonal, zeros above), the rest the reflector tails in A.
__global__ void __launch_bounds__(256)
vrow_bf16_kernel(const float *__restrict__ A, int lda, const double *__restrict__ Vtop, int k0,
                 int M, bf16 *__restrict__ Vh, bf16 *__restrict__ Vl) {
  __shared__ float t[64][33];
  const int tid = threadIdx.x, i0 = blockIdx.x * 32;
  const int r = tid & 31;
  for (int a = tid >> 5; a < 64; a += 8) {
    const int i = i0 + r;
    float v = 0.f;
    if (i < M) v = (i < 64) ? (float)Vtop[i + a * 64] : A[SLQR_IDX(k0 + i, k0 + a, lda)];
    t[a][r] = v;
  }
  __syncthreads();
  for (int idx = tid; idx < 32 * 64; idx += 256) {
    const int rr = idx >> 6, a = idx & 63;
    if (i0 + rr < M) {
      bf16 h, l;
      split_bf16(t[a][rr], h, l);
      Vh[(size_t)(i0 + rr) * 64 + a] = h;
      Vl[(size_t)(i0 + rr) * 64 + a] = l;
    }
  }
}

// W'^T ([column][64], FP32) as hi/lo pairs
__global__ void wt_split_kernel(const float *__restrict__ Wt, int count, bf16 *__restrict__ Wh,
                                bf16 *__restrict__ Wl) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < count; idx += gridDim.x * blockDim.x) {
    bf16 h, l;
    split_bf16(Wt[idx], h, l);
    Wh[idx] = h;
    Wl[idx] = l;
  }
}

// Twelve MMAs of K = 16: the three products of the split (hi hi, hi lo,
// lo hi), four K steps along a 128-byte (64-value) operand row each.
__device__ __forceinline__ void mma_split3(uint32_t taddr, uint32_t a_hi, uint32_t a_lo,
                                           uint32_t b_hi, uint32_t b_lo, bool first) {
  const uint32_t As[3] = {a_hi, a_hi, a_lo};
  const uint32_t Bs[3] = {b_hi, b_lo, b_hi};
#pragma unroll
  for (int pr = 0; pr < 3; ++pr) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint64_t ad = sw128_desc(As[pr] + k * 32), bd = sw128_desc(Bs[pr] + k * 32);
      const uint32_t accum = (first && pr == 0 && k == 0) ? 0u : 1u;
      asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                   " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                   :: "r"(taddr), "l"(ad), "l"(bd), "r"(kIdescBf16N64), "r"(accum) : "memory");
    }
  }
}

// --------------------------------------------------------------------------
// W = V^T X, computed transposed (D[c][a] = sum_i X[i][c] V[i][a]) over a row
// slice: 128 columns of X on the M side, the 64 reflectors on the N side,
// 64 rows of K per stage from the shadows (X and the panel's columns of A).
// grid: (ceil(N / 128), S); slice s covers rows [row_first + s*RS, ...) of the
// panel (relative to k0), RS a multiple of 64; partial s+1 of Wp ([s][c][a]).
// --------------------------------------------------------------------------
constexpr int kVbStages = 3;
constexpr int kVbChunk = 64;                          // rows (K) per stage
constexpr int kVbBytesX = kBfTile * kVbChunk * 2;     // 16 KB per half
constexpr int kVbBytesV = 64 * kVbChunk * 2;          // 8 KB per half
constexpr int kVbStageBytes = 2 * kVbBytesX + 2 * kVbBytesV;
constexpr size_t kVbSmem = (size_t)kVbStages * kVbStageBytes + 1024;

__global__ void __launch_bounds__(kBfThreads)
vtx_bf16_kernel(const __grid_constant__ CUtensorMap mapXh, const __grid_constant__ CUtensorMap mapXl,
                const __grid_constant__ CUtensorMap mapVh, const __grid_constant__ CUtensorMap mapVl,
                int k0, int row_first, int M, int xcol0, int N, int RS, float *__restrict__ Wp,
                int *status) {
  extern __shared__ __align__(1024) unsigned char bf_smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)bf_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint32_t s_taddr;
  __shared__ __align__(8) uint64_t s_full[kVbStages], s_empty[kVbStages], s_done;
  __shared__ int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c0 = blockIdx.x * kBfTile, s = blockIdx.y;
  const int i_begin = row_first + s * RS;
  const int i_end = min(M, i_begin + RS);
  const int T = (i_end > i_begin) ? (i_end - i_begin + kVbChunk - 1) / kVbChunk : 0;
  // stage layout: X hi | X lo | V hi | V lo
  auto stage = [&](int st) { return smem_u32(base + st * kVbStageBytes); };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;"
                 :: "r"(smem_u32(&s_taddr)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int st = 0; st < kVbStages; ++st) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&s_full[st])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&s_empty[st])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&s_done)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = s_taddr;

  if (tid == 0) {
    bool ok = true;
    int issued = 0;
    auto issue = [&](int t) {
      const int st = t % kVbStages;
      const uint32_t full = smem_u32(&s_full[st]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                   :: "r"(full), "r"(kVbStageBytes) : "memory");
      const int row = k0 + i_begin + t * kVbChunk;
      const uint32_t b = stage(st);
      tma_load_2d(b, &mapXh, row, xcol0 + c0, full);
      tma_load_2d(b + kVbBytesX, &mapXl, row, xcol0 + c0, full);
      tma_load_2d(b + 2 * kVbBytesX, &mapVh, row, k0, full);              // V: the panel's columns
      tma_load_2d(b + 2 * kVbBytesX + kVbBytesV, &mapVl, row, k0, full);
    };
    for (; issued < T && issued < kVbStages; ++issued) issue(issued);
    for (int t = 0; t < T && ok; ++t) {
      const int st = t % kVbStages;
      const uint32_t ph = (uint32_t)((t / kVbStages) & 1);
      if (!mbar_wait(smem_u32(&s_full[st]), ph)) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t b = stage(st);
      mma_split3(taddr, b, b + kVbBytesX, b + 2 * kVbBytesX, b + 2 * kVbBytesX + kVbBytesV, t == 0);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(&s_empty[st])) : "memory");
      if (issued < T) {                                // refill this stage once its MMAs are done
        if (!mbar_wait(smem_u32(&s_empty[st]), ph)) { ok = false; break; }
        issue(issued++);
      }
    }
    if (ok) {
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(&s_done)) : "memory");
      ok = mbar_wait(smem_u32(&s_done), 0);
    } else {
      for (int t = 0; t < issued; ++t) {               // let the copies in flight land
        const int st = t % kVbStages;
        mbar_wait(smem_u32(&s_full[st]), (uint32_t)((t / kVbStages) & 1));
      }
      atomicCAS(status, 0, SLQR_ETIMEOUT);
    }
    s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (s_ok && T > 0) {
    const int c = c0 + warp * 32 + lane;                 // TMEM lane = column of X
    float *out = Wp + ((size_t)(s + 1) * N + c) * 64;
#pragma unroll 1
    for (int a0 = 0; a0 < 64; a0 += 16) {
      uint32_t r[16];
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                   "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                   : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                     "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                     "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                   : "r"(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)a0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (c < N) {
#pragma unroll
        for (int q = 0; q < 16; q += 4)
          *(float4 *)(out + a0 + q) = make_float4(__uint_as_float(r[q]), __uint_as_float(r[q + 1]),
                                                  __uint_as_float(r[q + 2]), __uint_as_float(r[q + 3]));
      }
    }
  } else if (s_ok) {
    // an empty slice still owns its partial: zeros
    const int c = c0 + warp * 32 + lane;
    if (c < N)
      for (int a = 0; a < 64; ++a) Wp[((size_t)(s + 1) * N + c) * 64 + a] = 0.f;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" :: "r"(taddr));
}

// --------------------------------------------------------------------------
// X -= V W' on 128 x 64 tiles of X, K = 64 reflectors: V (row-major hi/lo)
// and W'^T (hi/lo) by TMA with 128-byte swizzle, the X tile (FP32, no
// swizzle) by TMA; 12 MMAs; the epilogue subtracts the accumulator from the
// X tile, splits the new values into the shadow tiles (in the space the
// operands used) and stores all three tiles back with TMA.
// --------------------------------------------------------------------------
constexpr int kUbN = 64;                               // columns of X per CTA
constexpr int kUbBytesA = kBfTile * 64 * 2;            // 16 KB per half
constexpr int kUbBytesB = kUbN * 64 * 2;               // 8 KB per half
constexpr int kUbBytesX = kBfTile * kUbN * 4;          // 32 KB
constexpr size_t kUbSmem = (size_t)2 * kUbBytesA + 2 * kUbBytesB + kUbBytesX + 1024;

__global__ void __launch_bounds__(kBfThreads)
upd_bf16_kernel(const __grid_constant__ CUtensorMap mapVh, const __grid_constant__ CUtensorMap mapVl,
                const __grid_constant__ CUtensorMap mapWh, const __grid_constant__ CUtensorMap mapWl,
                const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapXh,
                const __grid_constant__ CUtensorMap mapXl, int k0, int xcol0, int *status) {
  extern __shared__ __align__(1024) unsigned char bf_smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)bf_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sAh = base;
  unsigned char *sAl = base + kUbBytesA;
  unsigned char *sBh = base + 2 * kUbBytesA;
  unsigned char *sBl = sBh + kUbBytesB;
  float *sX = (float *)(sBl + kUbBytesB);
  bf16 *sXh = (bf16 *)sAh;                             // [column][row], after the MMAs
  bf16 *sXl = (bf16 *)sAl;
  __shared__ uint32_t s_taddr;
  __shared__ __align__(8) uint64_t s_full, s_mma;
  __shared__ int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.x * kBfTile, c0 = blockIdx.y * kUbN;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&s_taddr)), "r"(kUbN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&s_full)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&s_mma)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = s_taddr;

  if (tid == 0) {
    const uint32_t full = smem_u32(&s_full);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(full), "r"(2 * kUbBytesA + 2 * kUbBytesB + kUbBytesX) : "memory");
    tma_load_2d(smem_u32(sAh), &mapVh, 0, i0, full);
    tma_load_2d(smem_u32(sAl), &mapVl, 0, i0, full);
    tma_load_2d(smem_u32(sBh), &mapWh, 0, c0, full);
    tma_load_2d(smem_u32(sBl), &mapWl, 0, c0, full);
    tma_load_2d(smem_u32(sX), &mapX, k0 + i0, xcol0 + c0, full);
    bool ok = mbar_wait(full, 0);
    if (ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      mma_split3(taddr, smem_u32(sAh), smem_u32(sAl), smem_u32(sBh), smem_u32(sBl), true);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(&s_mma)) : "memory");
      ok = mbar_wait(smem_u32(&s_mma), 0);
    } else {
      mbar_wait(full, 0);                 // let the copies in flight land before leaving
    }
    if (!ok) atomicCAS(status, 0, SLQR_ETIMEOUT);
    s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool ok = s_ok != 0;
  if (ok) {
    const int row = warp * 32 + lane;                 // TMEM lane = row of the tile
#pragma unroll 1
    for (int cc = 0; cc < kUbN; cc += 16) {
      uint32_t r[16];
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                   "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                   : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                     "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                     "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                   : "r"(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int at = (cc + q) * kBfTile + row;
        const float v = sX[at] - __uint_as_float(r[q]);
        sX[at] = v;
        bf16 h, l;
        split_bf16(v, h, l);
        sXh[at] = h;
        sXl[at] = l;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0 && ok) {
    tma_store_2d(&mapX, k0 + i0, xcol0 + c0, smem_u32(sX));
    tma_store_2d(&mapXh, k0 + i0, xcol0 + c0, smem_u32(sXh));
    tma_store_2d(&mapXl, k0 + i0, xcol0 + c0, smem_u32(sXl));
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(kUbN));
}

slqr_status init_bf16_attrs(slqr_ctx *ctx) {
  cudaError_t e = cudaFuncSetAttribute(upd_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kUbSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(vtx_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kVbSmem);
  if (e != cudaSuccess)
    return fail(ctx, SLQR_ECUDA, "cudaFuncSetAttribute(bf16): %s", cudaGetErrorString(e));
  return SLQR_OK;
}

void split_bf16_region(const float *A, int lda, int r0, int r1, int c0, int c1, void *hi,
                       void *lo, int num_sms, cudaStream_t stream) {
  if (r1 <= r0 || c1 <= c0) return;
  split_bf16_kernel<<<4 * num_sms, 256, 0, stream>>>(A, lda, r0, r1, c0, c1, (bf16 *)hi,
                                                     (bf16 *)lo);
}

int launch_vtx_bf16(const float *A, int lda, const void *sh_hi, const void *sh_lo,
                    const double *Vtop, int k0, int M, int xcol0, int N, float *Wp,
                    size_t work_elems, int num_sms, int *status, cudaStream_t stream,
                    void (*vtop_part)(const float *, int, const double *, int, int, const float *,
                                      int, int, float *, cudaStream_t)) {
  if (lda % 8 != 0 || ((uintptr_t)sh_hi & 15) != 0 || ((uintptr_t)sh_lo & 15) != 0 || M <= 64 ||
      N <= 0)
    return 0;
  const int rows = M - 64;
  const int ntiles = (N + kBfTile - 1) / kBfTile;
  int S = std::max(1, (2 * num_sms + ntiles - 1) / ntiles);
  int RS = (rows + S - 1) / S;
  RS = std::max(kVbChunk * 2, (RS + kVbChunk - 1) / kVbChunk * kVbChunk);
  S = (rows + RS - 1) / RS;
  if ((size_t)(S + 1) * N * 64 + (size_t)64 * N > work_elems) return 0;
  CUtensorMap mapXh, mapXl;
  if (!make_map(&mapXh, (const bf16 *)sh_hi, k0 + M, xcol0 + N, lda, kVbChunk, kBfTile) ||
      !make_map(&mapXl, (const bf16 *)sh_lo, k0 + M, xcol0 + N, lda, kVbChunk, kBfTile))
    return 0;
  // the V boxes (the panel's 64 columns) with a 64-column box
  CUtensorMap mapVh, mapVl;
  if (!make_map(&mapVh, (const bf16 *)sh_hi, k0 + M, xcol0 + N, lda, kVbChunk, 64) ||
      !make_map(&mapVl, (const bf16 *)sh_lo, k0 + M, xcol0 + N, lda, kVbChunk, 64))
    return 0;
  vtop_part(A, lda, Vtop, k0, 64, A + (size_t)xcol0 * lda, lda, N, Wp, stream);
  vtx_bf16_kernel<<<dim3(ntiles, S), kBfThreads, kVbSmem, stream>>>(mapXh, mapXl, mapVh, mapVl, k0,
                                                                    64, M, xcol0, N, RS, Wp,
                                                                    status);
  return S + 1;
}

bool launch_upd_bf16(const float *A, int lda, void *sh_hi, void *sh_lo, const double *Vtop,
                     int k0, int M, int xcol0, int N, const float *Wt, void *scratch,
                     int num_sms, int *status, cudaStream_t stream) {
  if (lda % 8 != 0 || ((uintptr_t)A & 15) != 0 || ((uintptr_t)scratch & 15) != 0 || M <= 0 ||
      N <= 0)
    return false;
  bf16 *Vh = (bf16 *)scratch;
  bf16 *Vl = Vh + (size_t)M * 64;
  bf16 *Wh = Vl + (size_t)M * 64;
  bf16 *Wl = Wh + (size_t)N * 64;
  CUtensorMap mapVh, mapVl, mapWh, mapWl, mapX, mapXh, mapXl;
  if (!make_map(&mapVh, (const bf16 *)Vh, 64, M, 64, 64, kBfTile) ||
      !make_map(&mapVl, (const bf16 *)Vl, 64, M, 64, 64, kBfTile) ||
      !make_map(&mapWh, (const bf16 *)Wh, 64, N, 64, 64, kUbN) ||
      !make_map(&mapWl, (const bf16 *)Wl, 64, N, 64, 64, kUbN) ||
      !make_map(&mapX, A, k0 + M, xcol0 + N, lda, kBfTile, kUbN, false) ||
      !make_map(&mapXh, (const bf16 *)sh_hi, k0 + M, xcol0 + N, lda, kBfTile, kUbN, false) ||
      !make_map(&mapXl, (const bf16 *)sh_lo, k0 + M, xcol0 + N, lda, kBfTile, kUbN, false))
    return false;
  vrow_bf16_kernel<<<(M + 31) / 32, 256, 0, stream>>>(A, lda, Vtop, k0, M, Vh, Vl);
  wt_split_kernel<<<std::min(4 * num_sms, (N * 64 + 255) / 256), 256, 0, stream>>>(Wt, N * 64, Wh,
                                                                                   Wl);
  dim3 grid((M + kBfTile - 1) / kBfTile, (N + kUbN - 1) / kUbN);
  upd_bf16_kernel<<<grid, kBfThreads, kUbSmem, stream>>>(mapVh, mapVl, mapWh, mapWl, mapX, mapXh,
                                                         mapXl, k0, xcol0, status);
  return true;
}

}  // namespace slqr
