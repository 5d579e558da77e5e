// cluster_common.cuh -- device helpers of the thread-block-cluster panel
// kernels (panel_cluster.cu, panel_cluster_reg.cu): cluster rank and size,
// cluster barriers, distributed-shared-memory addresses, loads and stores,
// stores that count their bytes on the receiver's mbarrier, bounded mbarrier
// waits, and small arithmetic helpers.
#pragma once

#include "slqr_internal.cuh"

#include <type_traits>

namespace slqr {

namespace cl {

__device__ __forceinline__ int cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return (int)r;
}

__device__ __forceinline__ int cluster_ctas() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return (int)r;
}

// Barrier over every thread of every CTA of the cluster; orders the shared
// memory writes before it (release) with the reads after it (acquire),
// cluster-wide.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address of the object at `p` (this CTA's shared memory) in the shared
// memory of CTA `rank` of the cluster.
__device__ __forceinline__ unsigned cluster_addr(const void *p, int rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

__device__ __forceinline__ float cluster_ld(unsigned a, float) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}

__device__ __forceinline__ double cluster_ld(unsigned a, double) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
  return v;
}

__device__ __forceinline__ unsigned cluster_ld_u32(unsigned a) {
  unsigned v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}

// 2^e as a double for e in [-1022, 1023] (exact; built from the exponent bits)
__device__ __forceinline__ double exp2i(int e) {
  return __longlong_as_double((long long)(e + 1023) << 52);
}

// High word of |x| as a double (for non-negative doubles the integer order of
// the bit patterns is the numeric order).  For a float it is formed from the
// float's own bits with integer operations (a conversion to double would run
// on the FP64 pipe): exponent rebiased, the top 20 mantissa bits; subnormal
// floats map below every normal one, Inf and NaN above.
__device__ __forceinline__ unsigned abs_bits_hi(double x) {
  return (unsigned)((unsigned long long)__double_as_longlong(x) >> 32) & 0x7fffffffu;
}
__device__ __forceinline__ unsigned abs_bits_hi(float x) {
  const unsigned b = __float_as_uint(x) & 0x7fffffffu;
  const unsigned ef = b >> 23;
  if (ef == 0) return b ? (896u << 20) : 0u;
  if (ef == 255) return 0x7ff00000u;
  return ((ef + 896u) << 20) | ((b & 0x7fffffu) >> 3);
}

// fused multiply-add and square root in the type T (explicitly the FP32
// forms for float)
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float sqrt_t(float a) { return sqrtf(a); }
__device__ __forceinline__ double sqrt_t(double a) { return sqrt(a); }

// Sum over the 32 lanes (butterfly); lane 0's result is the one used.
template <typename T>
__device__ __forceinline__ T lanes_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the 16 lanes of a half-warp (butterfly).
template <typename T>
__device__ __forceinline__ T half_sum(T v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}


// Row map of a panel (as in factor.cu): panel row i is matrix row k0 + i for
// i < nbw and k0 + skip + i below.
__device__ __forceinline__ int cpanel_row(int k0, int nbw, int skip, int i) {
  return k0 + i + (i >= nbw ? skip : 0);
}

constexpr int kClMaxCtas = 16;        // largest cluster (non-portable size)

// 2^e in the type T (exact for the clamped exponents of the column scales)
template <typename T>
__device__ __forceinline__ T pow2_t(int e) {
  if constexpr (std::is_same<T, float>::value) return __int_as_float((e + 127) << 23);
  else return exp2i(e);
}

// 16-byte store into another CTA's shared memory (4 floats or 2 doubles)
__device__ __forceinline__ void cluster_st16(unsigned a, const float *v) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v[0]), "f"(v[1]),
               "f"(v[2]), "f"(v[3]) : "memory");
}
__device__ __forceinline__ void cluster_st16(unsigned a, const double *v) {
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v[0]), "d"(v[1]) : "memory");
}

// Stores into another CTA's shared memory that also count their bytes on an
// mbarrier there (complete-tx): the receiver waits on its own barrier, the
// sender does not wait at all.
__device__ __forceinline__ void st_async16(unsigned a, const float *v, unsigned mbar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];"
      ::"r"(a), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "r"(mbar) : "memory");
}
__device__ __forceinline__ void st_async16(unsigned a, const double *v, unsigned mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];"
               ::"r"(a), "d"(v[0]), "d"(v[1]), "r"(mbar) : "memory");
}
__device__ __forceinline__ void st_async1(unsigned a, float v, unsigned mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];"
               ::"r"(a), "f"(v), "r"(mbar) : "memory");
}
__device__ __forceinline__ void st_async1(unsigned a, double v, unsigned mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];"
               ::"r"(a), "d"(v), "r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_init1(unsigned long long *mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((unsigned)__cvta_generic_to_shared(mbar))
               : "memory");
}
// the single arrival of a phase, announcing `bytes` of complete-tx stores
__device__ __forceinline__ void mbar_expect(unsigned long long *mbar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
               ::"r"((unsigned)__cvta_generic_to_shared(mbar)), "r"(bytes) : "memory");
}
// Bounded wait for the phase of the given parity.  Past `report` polls (the
// context's spin limit) it records SLQR_ETIMEOUT once but goes on waiting, up
// to kSpinLimit polls, so that normally no store of the column is still in
// flight when the kernel moves on (the stores come from CTAs of the same
// cluster, all resident); false only when even that limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *mbar, unsigned parity,
                                                  unsigned report, int *status, bool *reported) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(mbar);
  for (unsigned it = 0;; ++it) {
    unsigned done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.b32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(a), "r"(parity) : "memory");
    if (done) return true;
    if (it >= report && !*reported) {
      record_status(status, SLQR_ETIMEOUT);
      *reported = true;
    }
    if (it >= kSpinLimit) return false;
    if (it > 64) __nanosleep(32);
  }
}

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}


}  // namespace cl
}  // namespace slqr
