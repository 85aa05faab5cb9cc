// tc_ptx.cuh -- inline-PTX wrappers shared by the tensor-core kernels
// (k_tc.cu, k_tch.cu): shared-memory addresses, mbarriers with bounded
// waits, bulk asynchronous copies, tcgen05 MMA / commit / TMEM loads, and
// the bf16 hi + lo split of FP32 complex entries.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace mf {
namespace ptx {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// One poll: returns when the phase completes or after at most kSuspendNs
// nanoseconds of suspension (the hint lets a waiting thread sleep instead of
// spinning, which leaves the issue slots of its SM sub-partition to the
// warps that work: 7 % faster Hermitian tensor-core walk than the default
// suspension; a completed phase still returns at once).
constexpr uint32_t kSuspendNs = 5000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "n"(kSuspendNs)
      : "memory");
  return ok != 0;
}
// bounded wait of at most `limit` polls; false on time-out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Six MMAs of one K step of a BF16 hi + lo split product into one
// accumulator, issued from one asm block (one predicate for the first MMA's
// accumulate flag, the others accumulate): A descriptors a0 a0 a1 a2 a2 a3
// with B descriptors b0 b1 b0 b2 b3 b2, i.e. a0 (b0 + b1) + a1 b0 and
// a2 (b2 + b3) + a3 b2.
__device__ __forceinline__ void mma_bf16_x6(uint32_t d, uint64_t a0, uint64_t a1, uint64_t a2, uint64_t a3,
                                            uint64_t b0, uint64_t b1, uint64_t b2, uint64_t b3, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.b32 p, %10, 0;\n setp.eq.b32 q, %10, %10;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %5, %9, p;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %6, %9, q;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %2, %5, %9, q;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %3, %7, %9, q;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %3, %8, %9, q;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %4, %7, %9, q;\n}\n" ::"r"(d),
      "l"(a0), "l"(a1), "l"(a2), "l"(a3), "l"(b0), "l"(b1), "l"(b2), "l"(b3), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

template <int NCOL>
__device__ __forceinline__ void tmem_load(uint32_t taddr, float* v);

template <>
__device__ __forceinline__ void tmem_load<4>(uint32_t taddr, float* v) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
__device__ __forceinline__ void tmem_load<8>(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
__device__ __forceinline__ void tmem_load<16>(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
__device__ __forceinline__ void tmem_load<32>(uint32_t taddr, float* v) {
  tmem_load<16>(taddr, v);
  tmem_load<16>(taddr + 16, v + 16);
}

// Shared-memory matrix descriptor of a canonical no-swizzle layout: start
// address, leading-dimension byte offset (between core matrices adjacent in
// K) and stride byte offset (between core matrices adjacent in M or N).
__device__ __forceinline__ uint64_t smem_desc_nosw(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// kind::f16 instruction descriptor: D f32, A and B bf16, M = 128, N = n;
// a_mn = 1 reads A MN-major (the transpose of the K-major A).
__host__ __device__ constexpr uint32_t idesc_bf16_m128(int n, int a_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(a_mn & 1) << 15) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

// Split two complex entries into bf16 hi + lo of their real and imaginary
// parts; plane p of the pair is word[p] (lower address = first entry).  The
// two entries go through the packed conversions (each lane rounded to
// nearest like the scalar conversion) and the packed FP32 subtraction.
__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t*>(&v); }

__device__ __forceinline__ void split_pair(float2 h0, float2 h1, uint32_t* w) {
  const float2 re = make_float2(h0.x, h1.x), im = make_float2(h0.y, h1.y);
  const __nv_bfloat162 rh = __floats2bfloat162_rn(re.x, re.y), ih = __floats2bfloat162_rn(im.x, im.y);
  const float2 rhf = __bfloat1622float2(rh), ihf = __bfloat1622float2(ih);
  const float2 rd = __fadd2_rn(re, make_float2(-rhf.x, -rhf.y));
  const float2 id = __fadd2_rn(im, make_float2(-ihf.x, -ihf.y));
  w[0] = bf2_bits(rh);
  w[1] = bf2_bits(__floats2bfloat162_rn(rd.x, rd.y));
  w[2] = bf2_bits(ih);
  w[3] = bf2_bits(__floats2bfloat162_rn(id.x, id.y));
}

}  // namespace ptx
}  // namespace mf
