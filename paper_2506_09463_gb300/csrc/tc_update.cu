// tc_update.cu -- the two products of the compact-WY trailing update on the
// 5th-generation tensor cores (tcgen05, kind::tf32), for the FP32
// factorization of the mixed-precision path:
//   vtx_tc_kernel  W = V^T X   (K = rows, a 4-stage TMA ring)
//   upd_tc_kernel  X -= V W'   (K = 64 reflectors, one TMA batch per tile)
//
// Operands reach shared memory by TMA (cp.async.bulk.tensor) in the K-major,
// 128-byte-swizzled layout the MMA reads (8-row x 128-byte atoms, 16-byte
// chunks XOR-ed with the row), one elected thread issues the MMAs into an FP32
// accumulator in tensor memory and commits them to an mbarrier, and after a
// bounded wait the four warps read the accumulator back with tcgen05.ld (warp
// w owns TMEM lanes 32w..32w+31).  TF32 keeps 10 mantissa bits of each
// operand; the products accumulate in FP32.
#include "tc_common.cuh"

#include <algorithm>

namespace slqr {

constexpr int kTcTile = 128;              // M = N = 128
constexpr int kTcThreads = 128;

// --------------------------------------------------------------------------
// W = V^T X on the tensor cores: partial sums over row slices, TMA-fed.
//
// Computed transposed, D[c][a] = sum_i X[i][c] V[i][a], so that the 128
// columns of X fill the M = 128 side of the MMA and the NB = 64 reflectors
// its N side.  Both operands are K-major in global memory already (each
// column of X and of V is contiguous along the rows i), so 2-D TMA boxes of
// 32 rows (128 bytes) x 128 or 64 columns land in shared memory in the
// 128-byte-swizzled K-major layout the MMA reads.  A 4-stage ring of
// (X, V) chunks is refilled as soon as the MMAs of a chunk complete
// (tcgen05.commit -> mbarrier).  Rows below the panel's top NB rows only: V
// there is exactly the reflector tails stored in A.
// --------------------------------------------------------------------------
constexpr int kVxStages = 4;
constexpr int kVxChunk = 32;                        // rows (K) per stage
constexpr int kVxBytesA = kTcTile * kVxChunk * 4;   // 16 KB
constexpr int kVxBytesB = 64 * kVxChunk * 4;        // 8 KB
constexpr uint32_t kIdescTf32N64 = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) |
                                   ((uint32_t)(kTcTile >> 4) << 24);

// grid: (ceil(N / 128), S); slice s covers rows [row_first + s*RS, ...) of the
// panel (relative to k0), RS a multiple of 32; partial s+1 of Wp ([s][c][a]).
__global__ void __launch_bounds__(kTcThreads)
vtx_tc_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapV,
              int k0, int row_first, int M, int xcol0, int N, int RS, float *__restrict__ Wp,
              int *status) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint32_t s_taddr;
  __shared__ __align__(8) uint64_t s_full[kVxStages], s_empty[kVxStages], s_done;
  __shared__ int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c0 = blockIdx.x * kTcTile, s = blockIdx.y;
  const int i_begin = row_first + s * RS;
  const int i_end = min(M, i_begin + RS);
  const int T = (i_end > i_begin) ? (i_end - i_begin + kVxChunk - 1) / kVxChunk : 0;
  auto sA = [&](int st) { return smem_u32(base + st * (kVxBytesA + kVxBytesB)); };
  auto sB = [&](int st) { return smem_u32(base + st * (kVxBytesA + kVxBytesB) + kVxBytesA); };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;"
                 :: "r"(smem_u32(&s_taddr)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int st = 0; st < kVxStages; ++st) {
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
    int issued = 0;                                    // chunks whose loads were issued
    auto issue = [&](int t) {
      const int st = t % kVxStages;
      const uint32_t full = smem_u32(&s_full[st]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                   :: "r"(full), "r"(kVxBytesA + kVxBytesB) : "memory");
      const int row = k0 + i_begin + t * kVxChunk;
      tma_load_2d(sA(st), &mapX, row, xcol0 + c0, full);
      tma_load_2d(sB(st), &mapV, row, k0, full);
    };
    for (; issued < T && issued < kVxStages; ++issued) issue(issued);
    for (int t = 0; t < T && ok; ++t) {
      const int st = t % kVxStages;
      const uint32_t ph = (uint32_t)((t / kVxStages) & 1);
      if (!mbar_wait(smem_u32(&s_full[st]), ph)) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int k = 0; k < kVxChunk / 8; ++k) {
        const uint64_t ad = sw128_desc(sA(st) + k * 32), bd = sw128_desc(sB(st) + k * 32);
        const uint32_t accum = (t > 0 || k > 0) ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                     :: "r"(taddr), "l"(ad), "l"(bd), "r"(kIdescTf32N64), "r"(accum) : "memory");
      }
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
      // a wait gave up: let the copies already issued land before leaving
      for (int t = 0; t < issued; ++t) {
        const int st = t % kVxStages;
        mbar_wait(smem_u32(&s_full[st]), (uint32_t)((t / kVxStages) & 1));
      }
      atomicCAS(status, 0, SLQR_ETIMEOUT);
    }
    s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (s_ok) {
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
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" :: "r"(taddr));
}

constexpr size_t kVxSmem = (size_t)kVxStages * (kVxBytesA + kVxBytesB) + 1024;

// --------------------------------------------------------------------------
// X -= V W' on the tensor cores, one 128 x 64 tile of X per CTA:
// D[i][c] = sum_a V[i][a] W'[a][c] with M = 128 rows, N = 64 columns and
// K = 64 reflectors.  The MMA wants both operands K-major (the 64 reflector
// values of a row of V, or of a column of W', contiguous), so V is first
// copied row-major (vrow_kernel) and the forward substitution writes W' as
// [column][reflector].  One elected thread loads the two K-halves of each
// operand (128-byte swizzle) and the X tile (no swizzle, [column][row]) on one
// mbarrier, issues 8 MMAs of K = 8, and the four warps subtract the
// accumulator from the X tile in shared memory, which one TMA store writes
// back (rows beyond the matrix are clipped by the tensor map).
// --------------------------------------------------------------------------
constexpr int kUpN = 64;                              // columns of X per CTA
constexpr int kUpBytesA = kTcTile * 64 * 4;           // V tile: 32 KB
constexpr int kUpBytesB = kUpN * 64 * 4;              // W' tile: 16 KB
constexpr int kUpBytesX = kTcTile * kUpN * 4;         // X tile: 32 KB
constexpr size_t kUpSmem = (size_t)kUpBytesA + kUpBytesB + kUpBytesX + 1024;

// Vr[i][a] = V(i, a) of the panel at row offset k0 (64 floats per row): rows
// i < 64 from Vtop (up on the diagonal, zeros above), the rest the reflector
// tails in A.  32 rows per CTA, transposed through shared memory.
__global__ void __launch_bounds__(256)
vrow_kernel(const float *__restrict__ A, int lda, const double *__restrict__ Vtop, int k0, int M,
            float *__restrict__ Vr) {
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
    if (i0 + rr < M) Vr[(size_t)(i0 + rr) * 64 + a] = t[a][rr];
  }
}

__global__ void __launch_bounds__(kTcThreads)
upd_tc_kernel(const __grid_constant__ CUtensorMap mapV, const __grid_constant__ CUtensorMap mapW,
              const __grid_constant__ CUtensorMap mapX, int k0, int xcol0, int *status) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = base;
  unsigned char *sB = base + kUpBytesA;
  float *sX = (float *)(base + kUpBytesA + kUpBytesB);
  __shared__ uint32_t s_taddr;
  __shared__ __align__(8) uint64_t s_full, s_mma;
  __shared__ int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.x * kTcTile, c0 = blockIdx.y * kUpN;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&s_taddr)), "r"(kUpN));
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
                 :: "r"(full), "r"(kUpBytesA + kUpBytesB + kUpBytesX) : "memory");
    tma_load_2d(smem_u32(sA), &mapV, 0, i0, full);
    tma_load_2d(smem_u32(sA + kUpBytesA / 2), &mapV, 32, i0, full);
    tma_load_2d(smem_u32(sB), &mapW, 0, c0, full);
    tma_load_2d(smem_u32(sB + kUpBytesB / 2), &mapW, 32, c0, full);
    tma_load_2d(smem_u32(sX), &mapX, k0 + i0, xcol0 + c0, full);
    bool ok = mbar_wait(full, 0);
    if (ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint64_t ad = sw128_desc(a0 + (k >> 2) * (kUpBytesA / 2) + (k & 3) * 32);
        const uint64_t bd = sw128_desc(b0 + (k >> 2) * (kUpBytesB / 2) + (k & 3) * 32);
        const uint32_t accum = (k > 0) ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                     :: "r"(taddr), "l"(ad), "l"(bd), "r"(kIdescTf32N64), "r"(accum) : "memory");
      }
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
    for (int cc = 0; cc < kUpN; cc += 16) {
      uint32_t r[16];
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                   "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                   : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                     "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                     "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                   : "r"(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int q = 0; q < 16; ++q) sX[(cc + q) * kTcTile + row] -= __uint_as_float(r[q]);
    }
    // the generic-proxy writes must be visible to the TMA store
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0 && ok) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
                 :: "l"((uint64_t)&mapX), "r"(k0 + i0), "r"(xcol0 + c0), "r"(smem_u32(sX))
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(kUpN));
}

// W = V^T X partials for a full 64-reflector panel of the FP32 matrix A
// (column-major, rows [0, k0 + M), columns [0, xcol0 + N)): slice 0 (the top
// 64 rows, where V is the Vtop triangle) on the FMA pipe, the rest on the
// tensor cores.  Returns the number of partial slices written, or 0 when the
// tensor-core path does not apply (the caller then uses the FMA kernels).
int launch_vtx_tc(const float *A, int lda, const double *Vtop, int k0, int M, int xcol0, int N,
                  float *Wp, size_t work_elems, int num_sms, int *status, cudaStream_t stream,
                  void (*vtop_part)(const float *, int, const double *, int, int, const float *, int,
                                    int, float *, cudaStream_t)) {
  if (lda % 4 != 0 || ((uintptr_t)A & 15) != 0 || M <= 64 || N <= 0) return 0;
  const int rows = M - 64;
  const int ntiles = (N + kTcTile - 1) / kTcTile;
  int S = std::max(1, (2 * num_sms + ntiles - 1) / ntiles);
  int RS = (rows + S - 1) / S;
  RS = std::max(kVxChunk * 4, (RS + kVxChunk - 1) / kVxChunk * kVxChunk);
  S = (rows + RS - 1) / RS;
  if ((size_t)(S + 1) * N * 64 + (size_t)64 * N > work_elems) return 0;
  CUtensorMap mapX, mapV;
  if (!make_map(&mapX, A, k0 + M, xcol0 + N, lda, kVxChunk, kTcTile) ||
      !make_map(&mapV, A, k0 + M, xcol0 + N, lda, kVxChunk, 64))
    return 0;
  vtop_part(A, lda, Vtop, k0, 64, A + (size_t)xcol0 * lda, lda, N, Wp, stream);
  vtx_tc_kernel<<<dim3(ntiles, S), kTcThreads, kVxSmem, stream>>>(mapX, mapV, k0, 64, M, xcol0, N,
                                                                   RS, Wp, status);
  return S + 1;
}

// TF32 tensor-core peak probe (slqr_measure_peak): one CTA per SM issues the
// MMAs of upd_tc_kernel (M = 128, N = 64, K = 8 each; the same descriptors,
// instruction descriptor and 64-column accumulator) back to back on operand
// tiles filled by plain stores, `iters` times 8 MMAs (K = 64), then commits and
// waits, bounded, for them.  2 * 128 * 64 * 64 flops per iteration.
constexpr size_t kPeakSmem = (size_t)kUpBytesA + kUpBytesB + 1024;

__global__ void __launch_bounds__(kTcThreads)
tf32_peak_kernel(int iters, int *status) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = base;
  unsigned char *sB = base + kUpBytesA;
  __shared__ uint32_t s_taddr;
  __shared__ __align__(8) uint64_t s_mma;
  const int tid = threadIdx.x, warp = tid >> 5;
  // operands: small generic values (their layout does not matter here)
  float *fa = (float *)sA, *fb = (float *)sB;
  for (int i = tid; i < (kUpBytesA + kUpBytesB) / 4; i += kTcThreads) {
    const float v = 1.0f + (float)((i * 37) & 255) * (1.0f / 256.0f);
    if (i < kUpBytesA / 4) fa[i] = v;
    else fb[i - kUpBytesA / 4] = v;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&s_taddr)), "r"(kUpN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&s_mma)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = s_taddr;
  if (tid == 0) {
    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint64_t ad = sw128_desc(a0 + (k >> 2) * (kUpBytesA / 2) + (k & 3) * 32);
        const uint64_t bd = sw128_desc(b0 + (k >> 2) * (kUpBytesB / 2) + (k & 3) * 32);
        const uint32_t accum = (it > 0 || k > 0) ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                     :: "r"(taddr), "l"(ad), "l"(bd), "r"(kIdescTf32N64), "r"(accum) : "memory");
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(&s_mma)) : "memory");
    if (!mbar_wait(smem_u32(&s_mma), 0)) atomicCAS(status, 0, SLQR_ETIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(kUpN));
}

slqr_status measure_tf32_peak(slqr_ctx *ctx, double *tflops) {
  const int iters = 4096;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, 0);
    tf32_peak_kernel<<<ctx->num_sms, kTcThreads, kPeakSmem, 0>>>(iters, ctx->d_status);
    cudaEventRecord(e1, 0);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);         // the first launch warms up
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(ctx, SLQR_ECUDA, "TF32 peak probe: %s", cudaGetErrorString(e));
  const double flops = 2.0 * kTcTile * 64.0 * 64.0 * iters * ctx->num_sms;
  *tflops = flops / (best * 1e-3) / 1e12;
  return SLQR_OK;
}

slqr_status init_tc_attrs(slqr_ctx *ctx) {
  cudaError_t e = cudaFuncSetAttribute(upd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kUpSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tf32_peak_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kPeakSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(vtx_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kVxSmem);
  if (e != cudaSuccess)
    return fail(ctx, SLQR_ECUDA, "cudaFuncSetAttribute(tc): %s", cudaGetErrorString(e));
  return SLQR_OK;
}

// X -= V W' for a full 64-reflector panel: V in row-major form (Vr), then the
// tensor-core tiles.  Returns false (nothing launched) when a tensor map
// cannot be encoded.
bool launch_upd_tc(const float *A, int lda, const double *Vtop, int k0, int M, int xcol0, int N,
                   const float *Wt, float *Vr, int *status, cudaStream_t stream) {
  if (lda % 4 != 0 || ((uintptr_t)A & 15) != 0 || ((uintptr_t)Wt & 15) != 0 ||
      ((uintptr_t)Vr & 15) != 0 || M <= 0 || N <= 0)
    return false;
  CUtensorMap mapV, mapW, mapX;
  if (!make_map(&mapV, Vr, 64, M, 64, 32, kTcTile) ||
      !make_map(&mapW, Wt, 64, N, 64, 32, kUpN) ||
      !make_map(&mapX, A, k0 + M, xcol0 + N, lda, kTcTile, kUpN, false))
    return false;
  vrow_kernel<<<(M + 31) / 32, 256, 0, stream>>>(A, lda, Vtop, k0, M, Vr);
  dim3 grid((M + kTcTile - 1) / kTcTile, (N + kUpN - 1) / kUpN);
  upd_tc_kernel<<<grid, kTcThreads, kUpSmem, stream>>>(mapV, mapW, mapX, k0, xcol0, status);
  return true;
}

}  // namespace slqr
