// k_rows.cu -- multi-vector generate-and-apply, row-owner form (SIMT).
//
// The product Y = H X (Sec. IV.A, Eq. generic_multivector) for the cases the
// Hermitian-reuse and DVR window kernels do not take (more than 16 vectors,
// hermitian_reuse = 0, stored DVR blocks, the FP64 DVR form, row slices) is
// computed by CTAs that own a 128-row output tile and sweep a column range
// in chunks of 32 columns (Eq. blockmatvec: phi^[n] = sum_m H^[n,m] psi^[m],
// scheduled by output block rows as in Sec. III.B).  Each chunk H[128 x 32]
// is generated into shared memory -- canonical entries from the Philox
// ensemble, entries below the diagonal as conjugates of their canonical
// partners (so H stays exactly Hermitian), DVR entries from a window table --
// or copied from the HBM block cache, then contracted with the chunk's rows of
// X on the FMA pipe with register-blocked TR x TV output sub-tiles.  The
// column range of a CTA is a split-K slot; a fixed-order FP64 reduction sums
// the slots.
#include <cuda_runtime.h>

#include "rows_body.cuh"

namespace mf {

// Split-K launcher: CTA (row tile, column range) -> part[slot][row][v].
template <typename T, int GEN, int NV, int TR, int TV, int NT>
__global__ void __launch_bounds__(NT, NT <= 256 ? 2 : 1) rows_simt(int64_t D, int64_t dpad, int64_t ksplit_cols, uint64_t seed,
                                                T sigma, dvr_consts dk, const typename cplx<T>::t* __restrict__ xc,
                                                typename cplx<T>::t* __restrict__ part,
                                                const typename cplx<T>::t* __restrict__ cache,
                                                const int64_t* __restrict__ slot_of_pair, int64_t b, int64_t nblk,
                                                const typename cplx<T>::t* __restrict__ hcache, int64_t tile0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // tile0: first row tile of a row-distributed plan (0 otherwise); the
  // partial slots hold the plan's rows only
  const int64_t R0 = (tile0 + (int64_t)blockIdx.x) * RT;
  const int64_t cbeg = (int64_t)blockIdx.y * ksplit_cols;
  const int64_t cend = cbeg + ksplit_cols < D ? cbeg + ksplit_cols : D;
  row_tile<T, GEN, NV, TR, TV, NT>(smem_raw, R0, cbeg, cend, D, seed, sigma, dk, xc,
                                   part + ((int64_t)blockIdx.y * dpad + R0 - tile0 * RT) * NV, cache, slot_of_pair, b,
                                   nblk, hcache);
}

template <typename T, int GEN, int NV, int TR, int TV, int NT>
static cudaError_t launch_rows_t(const Plan& p, const void* xc, void* part) {
  using C = typename cplx<T>::t;
  const size_t sm = rows_smem_bytes<T, NV>();
  auto k = rows_simt<T, GEN, NV, TR, TV, NT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = p.sliced ? p.slice_nt : p.ntile;
  dim3 grid((unsigned)ntiles, (unsigned)p.rows_nsplit);
  const T sigma = sizeof(T) == 4 ? (T)p.sigma32 : (T)p.sigma64;
  k<<<grid, NT, sm, p.stream>>>(p.D, ntiles * (int64_t)kTile, p.rows_split_cols, p.seed, sigma, p.dvr,
                                (const C*)xc, (C*)part, (const C*)p.d_cache, p.d_pair_slot, p.b, p.nblk,
                                (const C*)p.d_hblocks, p.sliced ? p.slice_t0 : 0);
  return cudaGetLastError();
}

// FP32 form with 32 or 64 vectors (blocks in HBM or generated): the ring
// tile of the batched kernel -- two staged 32-column chunks copied by
// cp.async while the previous one is contracted, two columns per 16-byte
// shared load, the complex product in packed FP32 pairs (A += (h_r, h_r) x,
// B += (h_i, h_i) x, Y = A + iB) -- on 4 x 4 complex register tiles.
template <int GEN, int NV, int NT>
__global__ void __launch_bounds__(NT, NT <= 256 ? 2 : 1) rows_simt_f32(int64_t D, int64_t dpad, int64_t ksplit_cols,
                                                               uint64_t seed, float sigma, dvr_consts dk,
                                                               const float2* __restrict__ xc,
                                                               float2* __restrict__ part,
                                                               const float2* __restrict__ cache,
                                                               const int64_t* __restrict__ slot_of_pair, int64_t b,
                                                               int64_t nblk, int64_t tile0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t R0 = (tile0 + (int64_t)blockIdx.x) * RT;
  const int64_t cbeg = (int64_t)blockIdx.y * ksplit_cols;
  const int64_t cend = cbeg + ksplit_cols < D ? cbeg + ksplit_cols : D;
  row_tile_async_f32<GEN, NV, 4, 4, NT, 1>(smem_raw, R0, cbeg, cend, seed, sigma, dk, xc,
                                           part + ((int64_t)blockIdx.y * dpad + R0 - tile0 * RT) * NV, cache,
                                           slot_of_pair, b, nblk);
}

template <int GEN, int NV, int NT>
static cudaError_t launch_rows_f32(const Plan& p, const void* xc, void* part) {
  static_assert((RT / 4) * (NV / 4) == NT, "4 x 4 tiles cover the row tile");
  const size_t sm = rows_smem_bytes_f32<NV>();
  auto k = rows_simt_f32<GEN, NV, NT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = p.sliced ? p.slice_nt : p.ntile;
  dim3 grid((unsigned)ntiles, (unsigned)p.rows_nsplit);
  k<<<grid, NT, sm, p.stream>>>(p.D, ntiles * (int64_t)kTile, p.rows_split_cols, p.seed, p.sigma32, p.dvr,
                                (const float2*)xc, (float2*)part, (const float2*)p.d_cache, p.d_pair_slot, p.b,
                                p.nblk, p.sliced ? p.slice_t0 : 0);
  return cudaGetLastError();
}

template <typename T, int GEN>
static cudaError_t launch_rows_g(const Plan& p, const void* xc, void* part, int64_t nvec) {
  if constexpr (sizeof(T) == 4) {
    // host-resident blocks take the synchronous tile (it reads them in place)
    if (!p.d_hblocks && nvec == 32) return launch_rows_f32<GEN, 32, 256>(p, xc, part);
    if (!p.d_hblocks && nvec == 64) return launch_rows_f32<GEN, 64, 512>(p, xc, part);
  }
  // (RT/TR) * (NV/TV) threads
  switch (nvec) {
    case 2: return launch_rows_t<T, GEN, 2, 1, 1, 256>(p, xc, part);
    case 4: return launch_rows_t<T, GEN, 4, 1, 2, 256>(p, xc, part);
    case 6: return launch_rows_t<T, GEN, 6, 1, 3, 256>(p, xc, part);
    case 8: return launch_rows_t<T, GEN, 8, 2, 2, 256>(p, xc, part);
    case 12: return launch_rows_t<T, GEN, 12, 2, 3, 256>(p, xc, part);
    case 16: return launch_rows_t<T, GEN, 16, 2, 4, 256>(p, xc, part);
    case 32: return launch_rows_t<T, GEN, 32, 4, 4, 256>(p, xc, part);
    case 64:
      if constexpr (sizeof(T) == 4) return launch_rows_t<T, GEN, 64, 4, 8, 256>(p, xc, part);
      else return launch_rows_t<T, GEN, 64, 2, 8, 512>(p, xc, part);
  }
  return cudaErrorNotSupported;
}

// Vector counts the row kernels are compiled for (2, 4, 6, 8, 12, 16, 32,
// 64); other counts are padded up by the caller to the next one.
int64_t rows_nvec_bucket(int64_t nvec) {
  static const int64_t kB[] = {2, 4, 6, 8, 12, 16, 32, 64};
  for (int64_t b : kB)
    if (nvec <= b) return b;
  return 64;
}

cudaError_t launch_rows_apply(const Plan& p, const void* xc, void* part, int64_t nvec_bucket) {
  if (p.prec == MF_PREC_FP64)
    return p.gen != MF_GEN_SINC_DVR_HO ? launch_rows_g<double, MF_GEN_PHILOX_GUE>(p, xc, part, nvec_bucket)
                                       : launch_rows_g<double, MF_GEN_SINC_DVR_HO>(p, xc, part, nvec_bucket);
  return p.gen != MF_GEN_SINC_DVR_HO ? launch_rows_g<float, MF_GEN_PHILOX_GUE>(p, xc, part, nvec_bucket)
                                     : launch_rows_g<float, MF_GEN_SINC_DVR_HO>(p, xc, part, nvec_bucket);
}

}  // namespace mf
