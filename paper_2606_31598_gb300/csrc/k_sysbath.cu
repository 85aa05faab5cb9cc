// k_sysbath.cu -- the system-bath operator of Sec. VII as one plan:
//
//   H = H_S (x) I_B + I_S (x) H_B + g sum_{a=1}^{n_int} A_a (x) B_a
//
// on psi in C^{d_S} (x) C^{d_B}, stored bath-major as X[beta][s] (a [d_B][d_S]
// multi-vector, R = d_S, Sec. IV.A).  With M_0 = I and M_a = g A_a,
//
//   Phi = sum_{o=0}^{n_int} B_o (X M_o^T) + X H_S^T,   B_0 = H_B,
//
// so one kernel generates the n_op = 1 + n_int dense bath operators (Philox
// ensembles with their own seeds, never stored) chunk by chunk and contracts
// each with its mixed input X_o = X M_o^T into the same accumulators
// (Eq. generic_matvec_flops: 8 n_op d_B^2 d_S real operations); the small
// X H_S^T term is added in FP64 by the reduction epilogue.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "rows_body.cuh"

namespace mf {

// xo[o][row][v] = sum_s xc[row][s] M_o[v][s] for v < dS (zero padding up to
// nb), FP64 arithmetic, rounded once to the compute precision.
template <typename C>
__global__ void k_sb_mix(const C* __restrict__ xc, C* __restrict__ xo, const double2* __restrict__ M, int nop, int ds,
                         int64_t rows, int64_t nb, int64_t ostride) {
  const int64_t n = (int64_t)nop * rows * nb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = e / (rows * nb), rem = e - o * rows * nb;
    const int64_t row = rem / nb, v = rem % nb;
    double sr = 0.0, si = 0.0;
    if (v < ds) {
      const double2* m = M + ((int64_t)o * ds + v) * ds;
      for (int s = 0; s < ds; ++s) {
        const C x = xc[row * nb + s];
        const double xr = (double)x.x, xi = (double)x.y;
        sr += m[s].x * xr - m[s].y * xi;
        si += m[s].x * xi + m[s].y * xr;
      }
    }
    C out;
    out.x = (decltype(out.x))sr;
    out.y = (decltype(out.y))si;
    xo[o * ostride + row * nb + v] = out;
  }
}

cudaError_t launch_sb_mix(const Plan& p, const void* xc, void* xo, int64_t nb, int64_t rows) {
  const int64_t n = (int64_t)p.sb_nop * rows * nb;
  int64_t g = (n + 255) / 256;
  if (g > (1 << 20)) g = 1 << 20;
  if (p.prec == MF_PREC_FP64)
    k_sb_mix<double2><<<(unsigned)g, 256, 0, p.stream>>>((const double2*)xc, (double2*)xo, p.d_sb_M, p.sb_nop,
                                                         p.sb_dS, rows, nb, rows * nb);
  else
    k_sb_mix<float2><<<(unsigned)g, 256, 0, p.stream>>>((const float2*)xc, (float2*)xo, p.d_sb_M, p.sb_nop,
                                                        p.sb_dS, rows, nb, rows * nb);
  return cudaGetLastError();
}

// Split-K CTA (row tile, column range): for every 32-column chunk and every
// operator o, generate B_o[R0:R0+128, c0:c0+32] into shared memory and
// accumulate it times the chunk of X_o; one partial per CTA.
template <typename T, int NV, int TR, int TV, int NT>
__global__ void __launch_bounds__(NT, NT <= 256 ? 2 : 1)
    sb_rows(int64_t D, int64_t dpad, int64_t ksplit_cols, int nop, const uint64_t* __restrict__ seeds, T sigma,
            const typename cplx<T>::t* __restrict__ xo, int64_t ostride, typename cplx<T>::t* __restrict__ part) {
  using C = typename cplx<T>::t;
  static_assert((RT / TR) * (NV / TV) == NT, "thread blocking must cover the tile");
  constexpr int LD = KCH + HPAD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* hs = reinterpret_cast<C*>(smem_raw);
  C* xs = hs + RT * LD;
  T* win = reinterpret_cast<T*>(xs + KCH * NV);
  const int64_t R0 = (int64_t)blockIdx.x * RT;
  const int64_t cbeg = (int64_t)blockIdx.y * ksplit_cols;
  const int64_t cend = cbeg + ksplit_cols < D ? cbeg + ksplit_cols : D;
  const int tid = threadIdx.x;
  const int tv = tid % (NV / TV), tr = tid / (NV / TV);
  const int r0 = tr * TR;
  const dvr_consts dk{};
  C acc[TR][TV];
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int j = 0; j < TV; ++j) acc[i][j] = zc<T>();
  for (int64_t c0 = cbeg; c0 < cend; c0 += KCH) {
    for (int o = 0; o < nop; ++o) {
      fill_chunk<T, MF_GEN_PHILOX_GUE, NT>(hs, win, R0, c0, D, seeds[o], sigma, dk, nullptr, nullptr, 1, 1);
      const C* x = xo + (int64_t)o * ostride;
      for (int e = tid; e < KCH * NV; e += NT) {
        const int64_t c = c0 + e / NV;
        xs[e] = c < cend ? x[c * NV + e % NV] : zc<T>();
      }
      __syncthreads();
#pragma unroll 4
      for (int k = 0; k < KCH; ++k) {
        C h[TR], xv[TV];
#pragma unroll
        for (int i = 0; i < TR; ++i) h[i] = hs[(r0 + i) * LD + k];
#pragma unroll
        for (int j = 0; j < TV; ++j) xv[j] = xs[k * NV + tv + j * (NV / TV)];
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
          for (int j = 0; j < TV; ++j) {
            acc[i][j].x = fma(h[i].x, xv[j].x, acc[i][j].x);
            acc[i][j].x = fma(-h[i].y, xv[j].y, acc[i][j].x);
            acc[i][j].y = fma(h[i].x, xv[j].y, acc[i][j].y);
            acc[i][j].y = fma(h[i].y, xv[j].x, acc[i][j].y);
          }
      }
      __syncthreads();
    }
  }
  C* out = part + ((int64_t)blockIdx.y * dpad + R0) * NV;
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int j = 0; j < TV; ++j) out[(r0 + i) * NV + tv + j * (NV / TV)] = acc[i][j];
}

template <typename T, int NV, int TR, int TV, int NT>
static cudaError_t launch_sb_t(const Plan& p, const void* xo, int64_t ostride, void* part) {
  using C = typename cplx<T>::t;
  const size_t sm = rows_smem_bytes<T, NV>();
  auto k = sb_rows<T, NV, TR, TV, NT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)p.ntile, (unsigned)p.rows_nsplit);
  const T sigma = sizeof(T) == 4 ? (T)p.sigma32 : (T)p.sigma64;
  k<<<grid, NT, sm, p.stream>>>(p.D, p.ntile * (int64_t)kTile, p.rows_split_cols, p.sb_nop, p.d_sb_seeds, sigma,
                                (const C*)xo, ostride, (C*)part);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_sb_g(const Plan& p, const void* xo, int64_t ostride, void* part, int64_t nb) {
  switch (nb) {
    case 2: return launch_sb_t<T, 2, 1, 1, 256>(p, xo, ostride, part);
    case 4: return launch_sb_t<T, 4, 1, 2, 256>(p, xo, ostride, part);
    case 6: return launch_sb_t<T, 6, 1, 3, 256>(p, xo, ostride, part);
    case 8: return launch_sb_t<T, 8, 2, 2, 256>(p, xo, ostride, part);
    case 12: return launch_sb_t<T, 12, 2, 3, 256>(p, xo, ostride, part);
    case 16: return launch_sb_t<T, 16, 2, 4, 256>(p, xo, ostride, part);
    case 32: return launch_sb_t<T, 32, 4, 4, 256>(p, xo, ostride, part);
    case 64:
      if constexpr (sizeof(T) == 4) return launch_sb_t<T, 64, 4, 8, 256>(p, xo, ostride, part);
      else return launch_sb_t<T, 64, 2, 8, 512>(p, xo, ostride, part);
  }
  return cudaErrorNotSupported;
}

cudaError_t launch_sb_rows(const Plan& p, const void* xo, int64_t ostride, void* part, int64_t nb) {
  return p.prec == MF_PREC_FP64 ? launch_sb_g<double>(p, xo, ostride, part, nb)
                                : launch_sb_g<float>(p, xo, ostride, part, nb);
}

}  // namespace mf
