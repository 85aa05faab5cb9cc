// k_noalloc.cu -- an apply entry point that allocates no memory.
//
// Some callers cannot allocate device memory once they are running: a
// service whose device memory is already fully reserved by another runtime's
// caching allocator, or a plugin inside a host application that forbids it
// to call cudaMalloc (which can synchronise the device and can fail under
// fragmentation).  mf_apply_dvr_noalloc gives them y = H x for the sinc-DVR
// operator with no allocation at all: the caller passes x and y, and the
// kernels' scratch (the FP32 copy of x and the partial-sum slots) lives in
// one file-scope device array of fixed size that every GPU loading this
// library holds until the process exits.
//
// CUDA loads a library's device code and arrays lazily by default, on first
// use: the first call on a device loads the three kernels and the array and
// may need device memory for that.  A caller makes that first call once, as
// a warm-up, before its memory is reserved (and before any stream capture);
// later calls load and allocate nothing.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "mf_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)40 << 20;  // 40 MiB
constexpr int64_t kNoAllocMaxD = 131072;
constexpr int kMaxDevices = 64;

// The scratch array itself.  In host code this name is only a stand-in for
// the device symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device with that device current and kept for the life of the process.
// A device reset (cudaDeviceReset, or the primary context destroyed and
// created again) makes the kept address stale; callers that reset a device
// must not call this entry point on it afterwards.
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = ptr;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

mf_status status_of(cudaError_t e) {
  if (e == cudaSuccess) return MF_OK;
  return e == cudaErrorMemoryAllocation ? MF_ERR_OOM : MF_ERR_CUDA;
}

}  // namespace

extern "C" mf_status mf_apply_dvr_noalloc(int64_t D, double dvr_L, const void* x, void* y, void* stream) {
  using namespace mf;
  if (D < 2 || D > kNoAllocMaxD || !x || !y || !(dvr_L >= 0.0) || !std::isfinite(dvr_L)) return MF_ERR_INVALID;
  const size_t bytes = (size_t)D * sizeof(double2);
  const char *xb = (const char*)x, *yb = (const char*)y;
  if (yb < xb + bytes && xb < yb + bytes) return MF_ERR_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MF_ERR_CUDA;

  // the constants and launch shape the plan path sets up for this D (FP32
  // form, procedural): the same helpers, so the two cannot drift apart
  Plan p;
  p.D = D;
  p.gen = MF_GEN_SINC_DVR_HO;
  p.prec = MF_PREC_FP32;
  p.stream = (cudaStream_t)stream;
  p.device = dev;
  if (cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MF_ERR_CUDA;
  dvr_setup(p.dvr, D, dvr_L);
  p.use_dvr_window = true;
  dvr_fp32_window_shape(p);

  const size_t xc_bytes = ((size_t)p.dpad * sizeof(float2) + 255) & ~(size_t)255;
  const size_t part_bytes = (size_t)p.nslot * (size_t)p.dpad * sizeof(float2);
  if (xc_bytes + part_bytes > kNoAllocScratchBytes) return MF_ERR_INVALID;

  void* base = nullptr;
  mf_status st = status_of(scratch_address(dev, &base));
  if (st != MF_OK) return st;
  void* xc = base;
  void* part = (char*)base + xc_bytes;
  // every partial slot row the reduction reads is written by the apply kernel
  // first, so no part of the scratch needs clearing between calls
  const VecShape sh{1, 1, p.nslot, p.dpad};
  if ((st = status_of(launch_to_compute(p, (const double2*)x, xc, D, sh))) != MF_OK) return st;
  if ((st = status_of(launch_dvr_apply(p, xc, part, 1))) != MF_OK) return st;
  return status_of(launch_reduce(p, part, (const double2*)x, (double2*)y, sh));
}
