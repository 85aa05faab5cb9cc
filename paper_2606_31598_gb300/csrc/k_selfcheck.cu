// k_selfcheck.cu -- exhaustive check of the generator's correctly rounded
// division and square root (gen.cuh) against the IEEE intrinsics on the GPU
// at hand, over every float of the ranges the generator feeds them.
#include <cuda_runtime.h>

#include "mf_internal.h"

namespace mf {
namespace {

// numerator m - 1 and denominator m + 1 for every float m in [0.5, 2)
// (a superset of the folded mantissas in (sqrt(1/2), sqrt(2)])
__global__ void k_check_div(unsigned long long* bad) {
  const uint32_t lo = 0x3F000000u, hi = 0x40000000u;
  unsigned long long cnt = 0;
  for (uint32_t i = lo + blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += gridDim.x * blockDim.x) {
    const float m = __uint_as_float(i);
    const float a = __fsub_rn(m, 1.0f), b = __fadd_rn(m, 1.0f);
    cnt += __float_as_uint(div_rn_narrow(a, b)) != __float_as_uint(__fdiv_rn(a, b));
  }
  if (cnt) atomicAdd(bad, cnt);
}

// x = 0 and every float x in [2^-33, 64) (the values of -2 ln u)
__global__ void k_check_sqrt(unsigned long long* bad) {
  const uint32_t lo = 0x2F000000u, hi = 0x42800000u;
  unsigned long long cnt = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0)
    cnt += __float_as_uint(sqrt_rn_narrow(0.0f)) != __float_as_uint(__fsqrt_rn(0.0f));
  for (uint32_t i = lo + blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += gridDim.x * blockDim.x) {
    const float x = __uint_as_float(i);
    cnt += __float_as_uint(sqrt_rn_narrow(x)) != __float_as_uint(__fsqrt_rn(x));
  }
  if (cnt) atomicAdd(bad, cnt);
}

}  // namespace
}  // namespace mf

extern "C" mf_status mf_selfcheck_generator(int64_t* div_mismatches, int64_t* sqrt_mismatches) {
  using namespace mf;
  if (!div_mismatches || !sqrt_mismatches) return MF_ERR_INVALID;
  unsigned long long* d = nullptr;
  if (cudaMalloc((void**)&d, 2 * sizeof(unsigned long long)) != cudaSuccess) return MF_ERR_OOM;
  unsigned long long h[2] = {0, 0};
  cudaError_t e = cudaMemset(d, 0, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) {
    k_check_div<<<1024, 256>>>(d);
    k_check_sqrt<<<1024, 256>>>(d + 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return MF_ERR_CUDA;
  *div_mismatches = (int64_t)h[0];
  *sqrt_mismatches = (int64_t)h[1];
  return MF_OK;
}
