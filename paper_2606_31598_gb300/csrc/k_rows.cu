// k_rows.cu -- multi-vector generate-and-apply, row-owner form (SIMT).
//
// For nvec >= 2 the product Y = H X (Sec. IV.A, Eq. generic_multivector) is
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

#include "mf_internal.h"

namespace mf {

namespace {

constexpr int RT = 128;   // rows per CTA
constexpr int KCH = 32;   // columns per chunk
constexpr int HPAD = 1;   // pad of the chunk rows (complex elements)

template <typename T> __device__ __forceinline__ typename cplx<T>::t zc() {
  typename cplx<T>::t z;
  z.x = T(0);
  z.y = T(0);
  return z;
}

}  // namespace

// Generate (or load) H[R0 : R0+RT, c0 : c0+KCH] into hs[RT][KCH+HPAD].
template <typename T, int GEN, int NT>
__device__ __forceinline__ void fill_chunk(typename cplx<T>::t* hs, T* win, int64_t R0, int64_t c0, int64_t D,
                                           uint64_t seed, T sigma, const dvr_consts& dk,
                                           const typename cplx<T>::t* __restrict__ cache,
                                           const int64_t* __restrict__ slot_of_pair, int64_t b, int64_t nblk) {
  using C = typename cplx<T>::t;
  const int tid = threadIdx.x;
  constexpr int LD = KCH + HPAD;
  // cached block pair?  (the chunk lies inside one block pair since b is a
  // multiple of 128 and chunks are 32-aligned)
  int64_t slot = -1;
  bool transposed = false;
  int64_t n = R0 / b, m = c0 / b;
  if (cache) {
    if (n <= m) {
      slot = slot_of_pair[n * nblk + m];
    } else {
      slot = slot_of_pair[m * nblk + n];
      transposed = true;
    }
  }
  if (slot >= 0) {
    const int64_t bb = b * b;
    for (int e = tid; e < RT * KCH; e += NT) {
      const int r = e / KCH, c = e % KCH;
      C h;
      if (!transposed) {
        h = cache[slot * bb + (R0 + r - n * b) * b + (c0 + c - m * b)];
      } else {
        h = cache[slot * bb + (c0 + c - m * b) * b + (R0 + r - n * b)];
        h.y = -h.y;
      }
      hs[r * LD + c] = h;
    }
    return;
  }
  if (GEN == MF_GEN_SINC_DVR_HO) {
    // window table: T(k) for k = r - c in (R0 - c0 - KCH, R0 - c0 + RT)
    const long long kmin = (long long)(R0 - c0) - (KCH - 1);
    for (int j = tid; j < RT + KCH - 1; j += NT) win[j] = dvr_T(dk, kmin + j, T());
    __syncthreads();
    for (int e = tid; e < RT * KCH; e += NT) {
      const int r = e / KCH, c = e % KCH;
      C h;
      h.x = win[r - c + KCH - 1];
      h.y = T(0);
      hs[r * LD + c] = h;
    }
    return;
  }
  if (c0 >= R0 + RT) {
    // strictly above the diagonal: canonical pairs along rows
    for (int e = tid; e < RT * (KCH / 2); e += NT) {
      const int r = e / (KCH / 2), pc = e % (KCH / 2);
      C h0, h1;
      gue_pair<T>(seed, sigma, (uint32_t)(R0 + r), (uint32_t)((c0 >> 1) + pc), h0, h1);
      hs[r * LD + 2 * pc] = h0;
      hs[r * LD + 2 * pc + 1] = h1;
    }
  } else if (c0 + KCH <= R0) {
    // strictly below: H[r][c] = conj(H[c][r]); canonical row c holds the
    // pair of columns (rows here) r = 2p, 2p + 1
    for (int e = tid; e < KCH * (RT / 2); e += NT) {
      const int c = e / (RT / 2), pr = e % (RT / 2);
      C h0, h1;
      gue_pair<T>(seed, sigma, (uint32_t)(c0 + c), (uint32_t)((R0 >> 1) + pr), h0, h1);
      h0.y = -h0.y;
      h1.y = -h1.y;
      hs[(2 * pr) * LD + c] = h0;
      hs[(2 * pr + 1) * LD + c] = h1;
    }
  } else {
    for (int e = tid; e < RT * KCH; e += NT) {
      const int r = e / KCH, c = e % KCH;
      hs[r * LD + c] = gue_entry<T>(seed, sigma, R0 + r, c0 + c);
    }
  }
}

// Y[R0 : R0+RT, :] over columns [cbeg, cend) -> part[slot][row][v].
template <typename T, int GEN, int NV, int TR, int TV, int NT>
__global__ void __launch_bounds__(NT) rows_simt(int64_t D, int64_t dpad, int64_t ksplit_cols, uint64_t seed,
                                                T sigma, dvr_consts dk, const typename cplx<T>::t* __restrict__ xc,
                                                typename cplx<T>::t* __restrict__ part,
                                                const typename cplx<T>::t* __restrict__ cache,
                                                const int64_t* __restrict__ slot_of_pair, int64_t b, int64_t nblk) {
  using C = typename cplx<T>::t;
  static_assert((RT / TR) * (NV / TV) == NT, "thread blocking must cover the tile");
  constexpr int LD = KCH + HPAD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* hs = reinterpret_cast<C*>(smem_raw);      // [RT][LD]
  C* xs = hs + RT * LD;                         // [KCH][NV]
  T* win = reinterpret_cast<T*>(xs + KCH * NV);  // [RT + KCH]

  const int tid = threadIdx.x;
  const int64_t R0 = (int64_t)blockIdx.x * RT;
  const int64_t cbeg = (int64_t)blockIdx.y * ksplit_cols;
  const int64_t cend = cbeg + ksplit_cols < D ? cbeg + ksplit_cols : D;
  const int tv = tid % (NV / TV), tr = tid / (NV / TV);
  const int r0 = tr * TR;  // thread rows r0..r0+TR-1, vectors tv + j*(NV/TV)

  C acc[TR][TV];
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int j = 0; j < TV; ++j) acc[i][j] = zc<T>();

  for (int64_t c0 = cbeg; c0 < cend; c0 += KCH) {
    fill_chunk<T, GEN, NT>(hs, win, R0, c0, D, seed, sigma, dk, cache, slot_of_pair, b, nblk);
    for (int e = tid; e < KCH * NV; e += NT) {
      const int64_t c = c0 + e / NV;
      xs[e] = c < cend ? xc[c * NV + e % NV] : zc<T>();
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < KCH; ++k) {
      C h[TR], x[TV];
#pragma unroll
      for (int i = 0; i < TR; ++i) h[i] = hs[(r0 + i) * LD + k];
#pragma unroll
      for (int j = 0; j < TV; ++j) x[j] = xs[k * NV + tv + j * (NV / TV)];
#pragma unroll
      for (int i = 0; i < TR; ++i)
#pragma unroll
        for (int j = 0; j < TV; ++j) {
          acc[i][j].x = fma(h[i].x, x[j].x, acc[i][j].x);
          acc[i][j].x = fma(-h[i].y, x[j].y, acc[i][j].x);
          acc[i][j].y = fma(h[i].x, x[j].y, acc[i][j].y);
          acc[i][j].y = fma(h[i].y, x[j].x, acc[i][j].y);
        }
    }
    __syncthreads();
  }
  C* out = part + ((int64_t)blockIdx.y * dpad + R0) * NV;
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int j = 0; j < TV; ++j) out[(r0 + i) * NV + tv + j * (NV / TV)] = acc[i][j];
}

template <typename T, int NV>
static size_t rows_smem_bytes() {
  using C = typename cplx<T>::t;
  return sizeof(C) * ((size_t)RT * (KCH + HPAD) + (size_t)KCH * NV) + sizeof(T) * (RT + KCH);
}

template <typename T, int GEN, int NV, int TR, int TV, int NT>
static cudaError_t launch_rows_t(const Plan& p, const void* xc, void* part) {
  using C = typename cplx<T>::t;
  const size_t sm = rows_smem_bytes<T, NV>();
  auto k = rows_simt<T, GEN, NV, TR, TV, NT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)p.ntile, (unsigned)p.rows_nsplit);
  const T sigma = sizeof(T) == 4 ? (T)p.sigma32 : (T)p.sigma64;
  k<<<grid, NT, sm, p.stream>>>(p.D, p.ntile * (int64_t)kTile, p.rows_split_cols, p.seed, sigma, p.dvr,
                                (const C*)xc, (C*)part, (const C*)p.d_cache, p.d_pair_slot, p.b, p.nblk);
  return cudaGetLastError();
}

template <typename T, int GEN>
static cudaError_t launch_rows_g(const Plan& p, const void* xc, void* part, int64_t nvec) {
  // (RT/TR) * (NV/TV) threads
  switch (nvec) {
    case 2: return launch_rows_t<T, GEN, 2, 1, 1, 256>(p, xc, part);
    case 4: return launch_rows_t<T, GEN, 4, 1, 2, 256>(p, xc, part);
    case 8: return launch_rows_t<T, GEN, 8, 2, 2, 256>(p, xc, part);
    case 16: return launch_rows_t<T, GEN, 16, 2, 4, 256>(p, xc, part);
    case 32: return launch_rows_t<T, GEN, 32, 4, 4, 256>(p, xc, part);
    case 64:
      if (sizeof(T) == 4) return launch_rows_t<T, GEN, 64, 4, 8, 256>(p, xc, part);
      return launch_rows_t<T, GEN, 64, 2, 8, 512>(p, xc, part);
  }
  return cudaErrorNotSupported;
}

// Vector counts the row kernels are compiled for; other counts are padded up
// by the caller to the next one.
int64_t rows_nvec_bucket(int64_t nvec) {
  int64_t b = 2;
  while (b < nvec) b *= 2;
  return b;
}

cudaError_t launch_rows_apply(const Plan& p, const void* xc, void* part, int64_t nvec_bucket) {
  if (p.prec == MF_PREC_FP64)
    return p.gen == MF_GEN_PHILOX_GUE ? launch_rows_g<double, MF_GEN_PHILOX_GUE>(p, xc, part, nvec_bucket)
                                      : launch_rows_g<double, MF_GEN_SINC_DVR_HO>(p, xc, part, nvec_bucket);
  return p.gen == MF_GEN_PHILOX_GUE ? launch_rows_g<float, MF_GEN_PHILOX_GUE>(p, xc, part, nvec_bucket)
                                    : launch_rows_g<float, MF_GEN_SINC_DVR_HO>(p, xc, part, nvec_bucket);
}

}  // namespace mf
