// fma_ceiling.cu -- the FP32 FMA-pipe ceiling on this GPU, measured: chains
// of independent fused multiply-adds on register operands only (scalar FFMA
// and packed FFMA2), 8 CTAs of 256 threads per SM, timed with CUDA events.
// The FP32 kernels' roofline denominator is the unit-count peak
// (SMs x 128 lanes x 2 FLOP x SM clock); this probe shows how much of it a
// kernel with no memory traffic at all reaches.  Not part of libmf.so.
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fma_ceiling \
//        paper_2606_31598_gb300/probes/fma_ceiling.cu && ./fma_ceiling
//
// On GB300 at 2070 MHz (unit-count peak 80.5 TFLOP/s): FFMA 74.6-74.8,
// FFMA2 75.9-76.4 TFLOP/s.
#include <cstdio>
#include <cuda_runtime.h>
template <int NA>
__global__ void __launch_bounds__(256) k_ffma(float* out, int iters, float b, float c) {
  float acc[NA];
#pragma unroll
  for (int i = 0; i < NA; ++i) acc[i] = threadIdx.x * 1e-3f + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int i = 0; i < NA; ++i) acc[i] = fmaf(acc[i], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < NA; ++i) s += acc[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
template <int NA>
__global__ void __launch_bounds__(256) k_ffma2(float* out, int iters, float b, float c) {
  float2 acc[NA];
#pragma unroll
  for (int i = 0; i < NA; ++i) acc[i] = make_float2(threadIdx.x * 1e-3f + i, i * 0.5f);
  const float2 bb = make_float2(b, b), cc = make_float2(c, c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int i = 0; i < NA; ++i) acc[i] = __ffma2_rn(acc[i], bb, cc);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < NA; ++i) s += acc[i].x + acc[i].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
int main() {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const int blocks = sms * 8, threads = 256, iters = 4096;
  float* out;
  cudaMalloc(&out, (size_t)blocks * threads * sizeof(float));
  cudaEvent_t a, e;
  cudaEventCreate(&a);
  cudaEventCreate(&e);
  auto run = [&](const char* name, void (*k)(float*, int, float, float), double fma_per_thread_iter) {
    for (int w = 0; w < 3; ++w) k<<<blocks, threads>>>(out, iters, 0.999f, 1e-4f);
    cudaEventRecord(a);
    for (int w = 0; w < 5; ++w) k<<<blocks, threads>>>(out, iters, 0.999f, 1e-4f);
    cudaEventRecord(e);
    cudaEventSynchronize(e);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, e);
    const double flop = 5.0 * 2.0 * fma_per_thread_iter * iters * (double)blocks * threads;
    printf("%-10s %8.3f ms  %7.2f TFLOP/s  err=%s\n", name, ms / 5, flop / (ms * 1e-3) / 1e12,
           cudaGetErrorString(cudaGetLastError()));
  };
  run("ffma16", k_ffma<16>, 8 * 16);
  run("ffma32", k_ffma<32>, 8 * 32);
  run("ffma2_8", k_ffma2<8>, 8 * 8 * 2);
  run("ffma2_16", k_ffma2<16>, 8 * 16 * 2);
  cudaFree(out);
  return 0;
}
