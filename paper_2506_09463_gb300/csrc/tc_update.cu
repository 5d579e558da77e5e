// tc_update.cu -- the two products of the compact-WY trailing update on the
// 5th-generation tensor cores (tcgen05, kind::tf32), for the FP32
// factorization of the mixed-precision path:
//   upd_tc_kernel  X -= V W'   (K = NB: operands staged by the threads)
//   vtx_tc_kernel  W = V^T X   (K = rows: operands streamed by TMA)
//
// One CTA (128 threads) owns a 128 x 128 tile of X.  The two operands are
// staged in shared memory in the K-major, 128-byte-swizzled layout the MMA
// reads (8-row x 128-byte atoms, 16-byte chunks XOR-ed with the row):
//   A = V   (128 rows of the tile x NB reflectors),
//   B = W'^T (128 columns of the tile x NB reflectors),
// one elected thread issues NB/8 MMAs (M = 128, N = 128, K = 8 each) into a
// 128 x 128 FP32 accumulator in tensor memory, commits them to an mbarrier,
// and after a bounded wait the four warps read the accumulator back with
// tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = rows of the tile) and
// subtract it from X.  TF32 keeps 10 mantissa bits of each operand; the
// products accumulate in FP32.
#include "slqr_internal.cuh"

#include <cuda.h>   // CUtensorMap and its enums (types only: the encoder is fetched at run time)
#include <algorithm>
#include <cstdint>
#include <mutex>

namespace slqr {

constexpr int kTcTile = 128;              // M = N = 128
constexpr int kTcThreads = 128;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: K-major operand, SWIZZLE_128B, 8-row
// groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);   // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)2 << 61;                    // SWIZZLE_128B
  return d;
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major, M = N = 128.
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) |
                                ((uint32_t)(kTcTile >> 3) << 17) |
                                ((uint32_t)(kTcTile >> 4) << 24);

// byte offset of element (row, k) of a K-major SW128 operand tile of 128 rows
__device__ __forceinline__ uint32_t sw128_offset(int row, int k) {
  const int kb = k >> 5, kk = k & 31;
  return (uint32_t)(kb * (kTcTile * 128) + (row >> 3) * 1024 + (row & 7) * 128 +
                    ((((kk >> 2) ^ (row & 7)) & 7) << 4) + (kk & 3) * 4);
}

template <int NB>
__global__ void __launch_bounds__(kTcThreads)
upd_tc_kernel(const float *__restrict__ A, int lda, const double *__restrict__ Vtop, int k0,
              int nbw, int M, float *__restrict__ X, int ldx, int N,
              const float *__restrict__ Wt, int *status) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  // 1024-byte aligned operand tiles
  unsigned char *base = (unsigned char *)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = base;
  unsigned char *sB = base + kTcTile * NB * 4;
  __shared__ uint32_t s_taddr;
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ int s_done;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.x * kTcTile, c0 = blockIdx.y * kTcTile;

  // stage A = V rows [i0, i0+128) and B = W'^T columns [c0, c0+128)
  for (int idx = tid; idx < kTcTile * NB; idx += kTcThreads) {
    const int r = idx & (kTcTile - 1), a = idx >> 7;
    const int i = i0 + r;
    float v = 0.f;
    if (i < M && a < nbw) v = (i < nbw) ? (float)Vtop[i + a * NB] : A[SLQR_IDX(k0 + i, k0 + a, lda)];
    *(float *)(sA + sw128_offset(r, a)) = v;
    const int c = c0 + r;
    float w = 0.f;
    if (c < N && a < nbw) w = Wt[(size_t)a * N + c];
    *(float *)(sB + sw128_offset(r, a)) = w;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&s_taddr)), "r"(kTcTile));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&s_mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // the generic-proxy smem writes must be visible to the tensor core
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = s_taddr;

  if (tid == 0) {
    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
    for (int s = 0; s < NB / 8; ++s) {
      const uint32_t koff = (uint32_t)((s >> 2) * (kTcTile * 128) + (s & 3) * 32);
      const uint64_t ad = sw128_desc(a0 + koff), bd = sw128_desc(b0 + koff);
      const uint32_t accum = (s > 0) ? 1u : 0u;
      asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                   " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                   :: "r"(taddr), "l"(ad), "l"(bd), "r"(kIdescTf32), "r"(accum) : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(&s_mbar)) : "memory");
  }
  // bounded wait for the MMAs
  if (tid == 0) {
    uint32_t done = 0;
    for (unsigned it = 0; it < kSpinLimit && !done; ++it) {
      asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                   " selp.b32 %0, 1, 0, p;\n}"
                   : "=r"(done) : "r"(smem_u32(&s_mbar)), "r"(0) : "memory");
      if (!done && it > 64) __nanosleep(32);
    }
    s_done = (int)done;
    if (!done) atomicCAS(status, 0, SLQR_ETIMEOUT);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (s_done) {
    const int row = warp * 32 + lane;
    const int i = i0 + row;
#pragma unroll 1
    for (int cc = 0; cc < kTcTile; cc += 16) {
      uint32_t r[16];
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                   "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                   : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                     "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                     "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                   : "r"(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (i < M) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int c = c0 + cc + q;
          if (c < N) X[SLQR_IDX(k0 + i, c, ldx)] -= __uint_as_float(r[q]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(taddr), "r"(kTcTile));
}

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

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  uint32_t done = 0;
  for (unsigned it = 0; it < kSpinLimit; ++it) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.b32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
    if (done) return true;
    if (it > 64) __nanosleep(32);
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t mbar) {
  asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
               " [%0], [%1, {%2, %3}], [%4];"
               :: "r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(mbar) : "memory");
}

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

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn tensor_map_encoder() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    cudaGetLastError();
  });
  return fn;
}

// 2-D map of a column-major FP32 matrix (rows contiguous), 128-byte swizzle,
// zero fill outside the matrix.
static bool make_map(CUtensorMap *map, const float *base, int rows, int cols, int ld, int box_rows,
                     int box_cols) {
  EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)box_cols};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)base, dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
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

template <int NB>
static size_t upd_tc_smem() {
  return (size_t)2 * kTcTile * NB * 4 + 1024;
}

slqr_status init_tc_attrs(slqr_ctx *ctx) {
  cudaError_t e = cudaFuncSetAttribute(upd_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)upd_tc_smem<64>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(upd_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)upd_tc_smem<32>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(vtx_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kVxSmem);
  if (e != cudaSuccess)
    return fail(ctx, SLQR_ECUDA, "cudaFuncSetAttribute(tc): %s", cudaGetErrorString(e));
  return SLQR_OK;
}

void launch_upd_tc(int nb, const float *A, int lda, const double *Vtop, int k0, int nbw, int M,
                   float *X, int ldx, int N, const float *Wt, int *status, cudaStream_t stream) {
  dim3 grid((M + kTcTile - 1) / kTcTile, (N + kTcTile - 1) / kTcTile);
  if (nb == 32)
    upd_tc_kernel<32><<<grid, kTcThreads, upd_tc_smem<32>(), stream>>>(A, lda, Vtop, k0, nbw, M, X,
                                                                       ldx, N, Wt, status);
  else
    upd_tc_kernel<64><<<grid, kTcThreads, upd_tc_smem<64>(), stream>>>(A, lda, Vtop, k0, nbw, M, X,
                                                                       ldx, N, Wt, status);
}

}  // namespace slqr
