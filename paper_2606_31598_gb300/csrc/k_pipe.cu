// k_pipe.cu -- measured throughput of the instruction classes the entry
// generators execute, for the per-pipe roofline of generation (the runtime
// model of Sec. V.A takes the generation time as the slowest resource; for
// procedural entries that resource is one of the SM's execution pipes).
//
// Each class runs as register-only chains with no memory traffic: NA
// independent accumulators per thread, 8 unrolled rounds per iteration,
// 8 CTAs of 256 threads per SM, every operation's result feeding the next
// operation of its chain so that no instruction can be removed, hoisted or
// folded with its neighbours.  The rate is operations per second over three
// timed launches after one warm-up launch (CUDA events on the caller's
// stream).  Classes:
//   0 IMAD.HI  mul.hi.u32 (the Philox round's high products)
//   1 IMAD     mad.lo.u32 (the low products)
//   2 LOP3     three-input logic operation (the Philox round's XORs)
//   3 IADD3    integer add (the Philox key schedule)
//   4 FFMA     FP32 fused multiply-add (counted as one operation)
//   5 MUFU     rsqrt.approx.f32 (the reciprocal and reciprocal square root
//              of the FP32 form use the same unit)
//   6 I2F      cvt.rn.f32.u32 (integer-to-float conversion)
//   7 DFMA     FP64 fused multiply-add
// and, when the caller asks for them, the 5th-generation tensor cores:
//   8 MMA128   tcgen05.mma kind::f16 (bf16 operands, FP32 accumulator in
//              TMEM), M = 128, N = 128, K = 16, both operands in shared
//              memory (no-swizzle K-major), one issuing thread per SM,
//              back to back into one accumulator
//   9 MMA256   the same with N = 256
// reported as MMA instructions per second over the GPU.  One instruction of
// either shape takes the same time on GB300, so N = 128 products (64 complex
// vectors) reach at most half of the dense BF16 rate.
#include <cuda_runtime.h>

#include <cstdint>

#include "mf_internal.h"
#include "tc_ptx.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;
constexpr int kClasses = 8;

__device__ __forceinline__ float rsqrt_approx(float v) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

// One round of class C on accumulator i of NA (neighbours are read before
// they are updated in this round, so the chains stay independent enough to
// fill the pipe but no value is dead).
template <int C, int NA>
struct Chain;

template <int NA>
struct Chain<0, NA> {
  using T = uint32_t;
  __device__ static T init(int i) { return threadIdx.x * 2654435761u + 977u * i + 1u; }
  __device__ static void round(T* x, T m) {
#pragma unroll
    for (int i = 0; i < NA; ++i) x[i] = __umulhi(x[i], m);
  }
};

template <int NA>
struct Chain<1, NA> {
  using T = uint32_t;
  __device__ static T init(int i) { return threadIdx.x * 2654435761u + 977u * i + 1u; }
  __device__ static void round(T* x, T m) {
#pragma unroll
    for (int i = 0; i < NA; ++i) x[i] = x[i] * m + x[(i + 1) % NA];
  }
};

// LOP3: bitwise majority of three chains (one three-input logic operation
// with no cheaper decomposition, so it cannot be split or shared).
__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}

template <int NA>
struct Chain<2, NA> {
  using T = uint32_t;
  __device__ static T init(int i) { return threadIdx.x * 2654435761u + 977u * i + 1u; }
  __device__ static void round(T* x, T) {
#pragma unroll
    for (int i = 0; i < NA; ++i) x[i] = maj3(x[i], x[(i + 1) % NA], x[(i + 2) % NA]);
  }
};

// IADD3: one add per result; every intermediate feeds two later adds, so
// merging adds into three-input forms saves no instruction.
template <int NA>
struct Chain<3, NA> {
  using T = uint32_t;
  __device__ static T init(int i) { return threadIdx.x * 2654435761u + 977u * i + 1u; }
  __device__ static void round(T* x, T) {
#pragma unroll
    for (int i = 0; i < NA; ++i) x[i] = x[i] + x[(i + 1) % NA];
  }
};

template <int NA>
struct Chain<4, NA> {
  using T = float;
  __device__ static T init(int i) { return threadIdx.x * 1e-3f + i; }
  __device__ static void round(T* x, T m) {
#pragma unroll
    for (int i = 0; i < NA; ++i) x[i] = __fmaf_rn(x[i], m, 1e-4f);
  }
};

template <int NA>
struct Chain<5, NA> {
  using T = float;
  __device__ static T init(int i) { return 1.0f + threadIdx.x * 1e-3f + i; }
  __device__ static void round(T* x, T) {
#pragma unroll
    for (int i = 0; i < NA; ++i) x[i] = rsqrt_approx(x[i]);
  }
};

// I2F: the converted value's bits are the next integer (a reinterpretation,
// no instruction), so the chain is conversions only.
template <int NA>
struct Chain<6, NA> {
  using T = uint32_t;
  __device__ static T init(int i) { return threadIdx.x * 2654435761u + 977u * i + 1u; }
  __device__ static void round(T* x, T) {
#pragma unroll
    for (int i = 0; i < NA; ++i) x[i] = __float_as_uint(__uint2float_rn(x[i]));
  }
};

template <int NA>
struct Chain<7, NA> {
  using T = double;
  __device__ static T init(int i) { return threadIdx.x * 1e-3 + i; }
  __device__ static void round(T* x, T m) {
#pragma unroll
    for (int i = 0; i < NA; ++i) x[i] = __fma_rn(x[i], m, 1e-4);
  }
};

template <int C, int NA>
__global__ void __launch_bounds__(kThreads) k_pipe(typename Chain<C, NA>::T* out, int iters,
                                                  typename Chain<C, NA>::T m) {
  using T = typename Chain<C, NA>::T;
  T x[NA];
#pragma unroll
  for (int i = 0; i < NA; ++i) x[i] = Chain<C, NA>::init(i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r) Chain<C, NA>::round(x, m);
  }
  T s = x[0];
#pragma unroll
  for (int i = 1; i < NA; ++i) s = s + x[i];
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;  // keeps every chain live
}

// Tensor-core class: operands A (64 KB) and B (64 KB) at the start of the
// dynamic shared memory; instruction i reads K step i % 8 of a 128-wide K
// tile (A: 16 row groups of 2048 B, B: N / 8 column groups of 2048 B, so the
// last byte read is below 128 KB).  Every wait is bounded; a time-out sets
// *err and the CTA still frees its TMEM.
constexpr int kMmaSmem = 144 * 1024;  // one CTA per SM
constexpr int kMmaCols = 256;

template <int N>
__global__ void __launch_bounds__(128, 1) k_pipe_mma(int nmma, int* err) {
  using namespace mf::ptx;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x;
  for (int i = tid; i < 32768; i += 128) reinterpret_cast<uint32_t*>(smem)[i] = 0x3c003c00u ^ (i & 0x00ff00ffu);
  if (tid == 0) mbar_init(&bar, 1);
  fence_async_smem();
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kMmaCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  if (tid == 0) {
    const uint32_t A = smem_u32(smem), B = smem_u32(smem + 65536);
    constexpr uint32_t idesc = idesc_bf16_m128(N, 0);
    uint32_t commits = 0;
    for (int i = 0; i < nmma; ++i) {
      const uint32_t k = (uint32_t)(i & 7) * 256;
      mma_bf16(tmem, smem_desc_nosw(A + k, 128, 2048), smem_desc_nosw(B + k, 128, 2048), idesc, i > 0 ? 1u : 0u);
      if ((i & 31) == 31 || i + 1 == nmma) {
        mma_commit(&bar);
        ++commits;
      }
    }
    if (commits > 0 && !mbar_wait(&bar, (commits - 1) & 1u, 1u << 26)) atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMmaCols) : "memory");
}

template <int N>
cudaError_t time_mma(int sms, int* err, cudaStream_t s, cudaEvent_t a, cudaEvent_t e, double* mma_per_s) {
  auto k = k_pipe_mma<N>;
  cudaError_t r = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMmaSmem);
  if (r != cudaSuccess) return r;
  const int nmma = 1 << 14;
  k<<<sms, 128, kMmaSmem, s>>>(256, err);
  if ((r = cudaGetLastError()) != cudaSuccess) return r;
  if ((r = cudaEventRecord(a, s)) != cudaSuccess) return r;
  k<<<sms, 128, kMmaSmem, s>>>(nmma, err);
  if ((r = cudaEventRecord(e, s)) != cudaSuccess) return r;
  if ((r = cudaEventSynchronize(e)) != cudaSuccess) return r;
  float ms = 0.f;
  if ((r = cudaEventElapsedTime(&ms, a, e)) != cudaSuccess) return r;
  *mma_per_s = ms > 0.f ? (double)nmma * sms / (ms * 1e-3) : 0.0;
  return cudaSuccess;
}

template <int C, int NA>
cudaError_t time_class(void* out, int blocks, int iters, typename Chain<C, NA>::T m, cudaStream_t s,
                       cudaEvent_t a, cudaEvent_t e, double* ops_per_s) {
  using T = typename Chain<C, NA>::T;
  k_pipe<C, NA><<<blocks, kThreads, 0, s>>>((T*)out, iters, m);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const int reps = 3;
  if ((err = cudaEventRecord(a, s)) != cudaSuccess) return err;
  for (int r = 0; r < reps; ++r) k_pipe<C, NA><<<blocks, kThreads, 0, s>>>((T*)out, iters, m);
  if ((err = cudaEventRecord(e, s)) != cudaSuccess) return err;
  if ((err = cudaEventSynchronize(e)) != cudaSuccess) return err;
  float ms = 0.f;
  if ((err = cudaEventElapsedTime(&ms, a, e)) != cudaSuccess) return err;
  const double ops = (double)NA * 8.0 * iters * (double)blocks * kThreads * reps;
  *ops_per_s = ms > 0.f ? ops / (ms * 1e-3) : 0.0;
  return cudaSuccess;
}

mf_status measure(int32_t device, void* stream, double* ops_per_s, bool tensor) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return MF_ERR_CUDA;
  const int blocks = sms * kCtasPerSm;
  cudaStream_t s = (cudaStream_t)stream;
  void* out = nullptr;
  if (mf::dev_malloc(&out, (size_t)blocks * kThreads * sizeof(double)) != cudaSuccess) return MF_ERR_OOM;
  cudaEvent_t a = nullptr, e = nullptr;
  cudaError_t err = cudaEventCreate(&a);
  if (err == cudaSuccess) err = cudaEventCreate(&e);
  // iteration counts give each launch a few milliseconds at the GB300 rates
  if (err == cudaSuccess) err = time_class<0, 16>(out, blocks, 1024, 2654435761u, s, a, e, &ops_per_s[0]);
  if (err == cudaSuccess) err = time_class<1, 16>(out, blocks, 2048, 2654435761u, s, a, e, &ops_per_s[1]);
  if (err == cudaSuccess) err = time_class<2, 16>(out, blocks, 2048, 0u, s, a, e, &ops_per_s[2]);
  if (err == cudaSuccess) err = time_class<3, 16>(out, blocks, 2048, 0u, s, a, e, &ops_per_s[3]);
  if (err == cudaSuccess) err = time_class<4, 16>(out, blocks, 4096, 0.999f, s, a, e, &ops_per_s[4]);
  if (err == cudaSuccess) err = time_class<5, 16>(out, blocks, 512, 0.f, s, a, e, &ops_per_s[5]);
  if (err == cudaSuccess) err = time_class<6, 16>(out, blocks, 512, 0u, s, a, e, &ops_per_s[6]);
  if (err == cudaSuccess) err = time_class<7, 8>(out, blocks, 64, 0.999, s, a, e, &ops_per_s[7]);
  int timed_out = 0;
  if (tensor && err == cudaSuccess) {
    int* d_err = reinterpret_cast<int*>(out);
    err = cudaMemsetAsync(d_err, 0, sizeof(int), s);
    if (err == cudaSuccess) err = time_mma<128>(sms, d_err, s, a, e, &ops_per_s[8]);
    if (err == cudaSuccess) err = time_mma<256>(sms, d_err, s, a, e, &ops_per_s[9]);
    if (err == cudaSuccess) err = cudaMemcpy(&timed_out, d_err, sizeof(int), cudaMemcpyDeviceToHost);
  }
  if (a) cudaEventDestroy(a);
  if (e) cudaEventDestroy(e);
  cudaFree(out);
  if (err != cudaSuccess) return MF_ERR_CUDA;
  return timed_out ? MF_ERR_TIMEOUT : MF_OK;
}

}  // namespace

extern "C" mf_status mf_pipe_rates(int32_t device, void* stream, double* ops_per_s, int32_t n) {
  if (!ops_per_s || n < kClasses || device < 0) return MF_ERR_INVALID;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return MF_ERR_CUDA;
  const mf_status st = measure(device, stream, ops_per_s, n >= kClasses + 2);
  cudaSetDevice(prev);
  return st;
}
