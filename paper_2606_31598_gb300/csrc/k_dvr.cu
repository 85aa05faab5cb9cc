// k_dvr.cu -- DVR Toeplitz-window generate-and-apply kernel (SIMT, one
// vector).
//
// Sec. III.A ("analytic generation"): the sinc-DVR kinetic block
// H^[n,m]_{ab} = T(r - c) depends on r - c only, so a CTA covering rows
// [R0, R0+RB) and columns [C0, C0+KC) generates the RB + KC - 1 distinct
// entries of its tile once into shared memory and contracts the whole
// RB x KC tile from that window: the dense O(RB*KC) product runs on the FMA
// pipe with register-blocked 16 x 16 sub-tiles.
#include <cuda_runtime.h>

#include "mf_internal.h"

namespace mf {


template <typename T> __device__ __forceinline__ typename cplx<T>::t czero();
template <> __device__ __forceinline__ float2 czero<float>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 czero<double>() { return make_double2(0.0, 0.0); }

// ---------------------------------------------------------------------------
// DVR Toeplitz-window kernel.  8 warps share the CTA's RB = 32*P rows and
// split its KC columns; lane L owns rows R0 + P*L + [0,P).  For a block of U
// columns the P x U sub-tile needs the P+U-1 window entries T(r - c), loaded
// from shared memory once and reused from registers.  The window table is
// stored with one pad slot per P entries so the lane-strided loads are free of
// bank conflicts.
// ---------------------------------------------------------------------------
template <typename T, int P>
__global__ void __launch_bounds__(256, 2) dvr_window(int64_t D, int64_t dpad, int kc, dvr_consts dk,
                                                     const typename cplx<T>::t* __restrict__ xc,
                                                     typename cplx<T>::t* __restrict__ part) {
  using C = typename cplx<T>::t;
  constexpr int U = P;
  constexpr int RB = 32 * P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ntb = RB + kc - 1;
  const int ntb_pad = ((ntb + ntb / P + 1) + 3) & ~3;
  T* tb = reinterpret_cast<T*>(smem_raw);
  C* xs = reinterpret_cast<C*>(tb + ntb_pad);

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t R0 = (int64_t)blockIdx.x * RB;
  const int64_t C0 = (int64_t)blockIdx.y * kc;
  const long long kmin = (long long)(R0 - C0) - kc + 1;
  for (int j = tid; j < ntb; j += 256) tb[j + j / P] = dvr_T(dk, kmin + j, T());
  for (int c = tid; c < kc; c += 256) {
    const int64_t g = C0 + c;
    xs[c] = g < D ? xc[g] : czero<T>();
  }
  __syncthreads();

  T acc_r[P], acc_i[P];
#pragma unroll
  for (int a = 0; a < P; ++a) {
    acc_r[a] = T(0);
    acc_i[a] = T(0);
  }
  const int kw = kc / 8;
  const int cbeg = w * kw, cend = cbeg + kw;
#pragma unroll 1
  for (int cc0 = cbeg; cc0 < cend; cc0 += U) {
    // window start jb is a multiple of P, so padded offsets are compile-time
    const int jb = P * lane - cc0 + kc - 1 - (U - 1);
    const T* wp = tb + jb + jb / P;
    T win[P + U - 1];
#pragma unroll
    for (int m = 0; m < P + U - 1; ++m) win[m] = wp[m + m / P];
    C xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = xs[cc0 + u];
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int a = 0; a < P; ++a) {
        const T t = win[a - u + U - 1];
        acc_r[a] = fma(t, xv[u].x, acc_r[a]);
        acc_i[a] = fma(t, xv[u].y, acc_i[a]);
      }
    }
  }
  __syncthreads();
  // cross-warp sum in fixed warp order (reuses the x region)
  C* red = xs;  // [8][RB]
#pragma unroll
  for (int a = 0; a < P; ++a) {
    C v;
    v.x = acc_r[a];
    v.y = acc_i[a];
    red[w * RB + P * lane + a] = v;
  }
  __syncthreads();
  for (int r = tid; r < RB; r += 256) {
    C s = red[r];
#pragma unroll
    for (int g = 1; g < 8; ++g) {
      s.x += red[g * RB + r].x;
      s.y += red[g * RB + r].y;
    }
    part[(int64_t)blockIdx.y * dpad + R0 + r] = s;
  }
}

template <typename T, int P>
static size_t dvr_smem_bytes(int kc) {
  using C = typename cplx<T>::t;
  const int RB = 32 * P;
  const int ntb = RB + kc - 1;
  const int ntb_pad = ((ntb + ntb / P + 1) + 3) & ~3;
  const size_t xs = (size_t)kc * sizeof(C), red = (size_t)8 * RB * sizeof(C);
  return (size_t)ntb_pad * sizeof(T) + (xs > red ? xs : red);
}

cudaError_t launch_dvr_apply(const Plan& p, const void* xc, void* part, int64_t nvec) {
  if (nvec != 1) return cudaErrorNotSupported;
  const int kc = p.dvr_cols;
  const int64_t nslot = (p.D + kc - 1) / kc;
  if (p.prec == MF_PREC_FP64) {
    constexpr int P = 8;
    const size_t sm = dvr_smem_bytes<double, P>(kc);
    auto k = dvr_window<double, P>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 grid((unsigned)((p.D + 32 * P - 1) / (32 * P)), (unsigned)nslot);
    k<<<grid, 256, sm, p.stream>>>(p.D, p.dpad, kc, p.dvr, (const double2*)xc, (double2*)part);
  } else {
    constexpr int P = 16;
    const size_t sm = dvr_smem_bytes<float, P>(kc);
    auto k = dvr_window<float, P>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 grid((unsigned)((p.D + 32 * P - 1) / (32 * P)), (unsigned)nslot);
    k<<<grid, 256, sm, p.stream>>>(p.D, p.dpad, kc, p.dvr, (const float2*)xc, (float2*)part);
  }
  return cudaGetLastError();
}

}  // namespace mf
