// tc_update.cu -- the rank-NB trailing update X -= V W' of the compact-WY
// factorization on the 5th-generation tensor cores (tcgen05, kind::tf32),
// for the FP32 factorization of the mixed-precision path.
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

#include <cstdint>

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
