// k_rows_herm.cu -- multi-vector generate-and-apply with Hermitian reuse.
//
// Y = H X for 2..16 vectors (compiled for 2, 4, 6, 8, 12, 16; Sec. IV.A,
// Eq. generic_multivector), each
// canonical entry generated (or read from the block cache) once and applied
// twice, as H^[n,m] and as H^[m,n] = (H^[n,m])^dagger (Sec. III.A).  A CTA
// owns a 128-row tile ti and a range of columns c >= 128 ti (the upper part
// and the diagonal tile, items balanced across the grid).  For each 32-column
// chunk it stages H[rows, chunk] in shared memory, adds H X[chunk] to its
// rows (register tiles, as the row-owner kernel) and, for chunks strictly
// above the diagonal tile, adds H^dagger X[rows] to the chunk's 32 rows.
// Partial sums go to fixed slots -- item slot s for the owner rows, slot
// NS + ti for the transposed rows -- that the fixed-order FP64 reduction
// adds up; unwritten slots are zeroed before the launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "rows_body.cuh"

namespace mf {
namespace {

// Transposed product of one staged chunk: y[c][v] += sum_r conj(hs[r][c])
// xr[r][v] for the chunk's 32 columns.  Thread (part p, slot q) owns CT
// columns x VT vectors over the rows of part p (register tile: each staged
// value read once per CT or VT products); the P parts are combined later.
template <typename T, int NV> struct Dag {
  static constexpr int VT = NV % 3 == 0 ? 3 : (NV < 4 ? NV : 4);     // vectors per thread
  static constexpr int CT = (NV == 16 && sizeof(T) == 4) ? 4 : 2;    // columns per thread
  static constexpr int TPP = (KCH / CT) * (NV / VT);                 // threads per part
};

template <typename T, int NV, int NT>
__device__ __forceinline__ void chunk_dagger(const typename cplx<T>::t* hs, const typename cplx<T>::t* xr,
                                             typename cplx<T>::t (&yt)[Dag<T, NV>::CT][Dag<T, NV>::VT]) {
  using C = typename cplx<T>::t;
  constexpr int LD = KCH + HPAD;
  constexpr int VT = Dag<T, NV>::VT, CT = Dag<T, NV>::CT, TPP = Dag<T, NV>::TPP;
  constexpr int P = NT / TPP, RP = RT / P;
  const int tid = threadIdx.x, p = tid / TPP, q = tid % TPP;
  const int cg = q / (NV / VT), vg = q % (NV / VT);
  for (int r = p * RP; r < (p + 1) * RP; ++r) {
    C h[CT], x[VT];
#pragma unroll
    for (int j = 0; j < CT; ++j) h[j] = hs[r * LD + cg + j * (KCH / CT)];
#pragma unroll
    for (int i = 0; i < VT; ++i) x[i] = xr[r * NV + vg + i * (NV / VT)];
#pragma unroll
    for (int j = 0; j < CT; ++j)
#pragma unroll
      for (int i = 0; i < VT; ++i) {
        // yt += conj(h) x
        yt[j][i].x = fma(h[j].x, x[i].x, yt[j][i].x);
        yt[j][i].x = fma(h[j].y, x[i].y, yt[j][i].x);
        yt[j][i].y = fma(h[j].x, x[i].y, yt[j][i].y);
        yt[j][i].y = fma(-h[j].y, x[i].x, yt[j][i].y);
      }
  }
}

template <typename T, int GEN, int NV, int TR, int TV, int NT>
__global__ void __launch_bounds__(NT, NT <= 256 ? 2 : 1)
    rows_herm(const HermItem* __restrict__ items, int64_t D, int64_t dpad, int64_t ns, int nop,
              const uint64_t* __restrict__ seeds, uint64_t seed, T sigma, dvr_consts dk,
              const typename cplx<T>::t* __restrict__ xc, int64_t xstride, typename cplx<T>::t* __restrict__ part,
              const typename cplx<T>::t* __restrict__ cache, const int64_t* __restrict__ slot_of_pair, int64_t b,
              int64_t nblk, const typename cplx<T>::t* __restrict__ hcache) {
  using C = typename cplx<T>::t;
  static_assert((RT / TR) * (NV / TV) == NT, "thread blocking must cover the tile");
  constexpr int LD = KCH + HPAD;
  constexpr int O = KCH * NV;
  constexpr int VT = Dag<T, NV>::VT, CT = Dag<T, NV>::CT, TPP = Dag<T, NV>::TPP;
  constexpr int P = NT / TPP;
  static_assert(NT % TPP == 0 && RT % P == 0, "transposed tile must cover the chunk");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* hs = reinterpret_cast<C*>(smem_raw);     // [RT][LD]
  C* xs = hs + RT * LD;                        // [KCH][NV]
  C* xr = xs + KCH * NV;                       // [RT][NV]
  C* red = xr + RT * NV;                       // [P][O]
  T* win = reinterpret_cast<T*>(red + P * O);  // [RT + KCH]

  const HermItem it = items[blockIdx.x];
  const int64_t R0 = (int64_t)it.ti * RT;
  const int64_t cend = it.c_end < D ? it.c_end : D;
  const int tid = threadIdx.x;
  const int tv = tid % (NV / TV), tr = tid / (NV / TV);
  const int r0 = tr * TR;
  C acc[TR][TV];
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int j = 0; j < TV; ++j) acc[i][j] = zc<T>();

  for (int64_t c0 = it.c_beg; c0 < cend; c0 += KCH) {
    const bool upper = c0 >= R0 + RT;
    C yt[CT][VT];
#pragma unroll
    for (int j = 0; j < CT; ++j)
#pragma unroll
      for (int i = 0; i < VT; ++i) yt[j][i] = zc<T>();
    for (int o = 0; o < nop; ++o) {
      const C* x = xc + (int64_t)o * xstride;
      const uint64_t sd = seeds ? seeds[o] : seed;
      fill_chunk<T, GEN, NT>(hs, win, R0, c0, D, sd, sigma, dk, cache, slot_of_pair, b, nblk, hcache);
      for (int e = tid; e < KCH * NV; e += NT) {
        const int64_t c = c0 + e / NV;
        xs[e] = c < cend ? x[c * NV + e % NV] : zc<T>();
      }
      if (upper)
        for (int e = tid; e < RT * NV; e += NT) {
          const int64_t r = R0 + e / NV;
          xr[e] = r < D ? x[r * NV + e % NV] : zc<T>();
        }
      __syncthreads();
#pragma unroll 4
      for (int k = 0; k < KCH; ++k) {
        C h[TR], xv[TV];
#pragma unroll
        for (int i = 0; i < TR; ++i) h[i] = hs[(r0 + i) * LD + k];
#pragma unroll
        for (int j = 0; j < TV; ++j) xv[j] = xs[k * NV + tv + j * (NV / TV)];
        tile_cmac<T, TR, TV>(acc, h, xv);
      }
      if (upper) chunk_dagger<T, NV, NT>(hs, xr, yt);
      __syncthreads();
    }
    if (upper) {
      // combine the P parts over r in fixed order, then write the chunk's 32 rows
      {
        const int q = tid % TPP, pp = tid / TPP;
        const int cg = q / (NV / VT), vg = q % (NV / VT);
#pragma unroll
        for (int j = 0; j < CT; ++j)
#pragma unroll
          for (int i = 0; i < VT; ++i) red[pp * O + (cg + j * (KCH / CT)) * NV + vg + i * (NV / VT)] = yt[j][i];
      }
      __syncthreads();
      for (int o = tid; o < O; o += NT) {
        C sacc = red[o];
        for (int q2 = 1; q2 < P; ++q2) {
          sacc.x += red[q2 * O + o].x;
          sacc.y += red[q2 * O + o].y;
        }
        part[((ns + it.ti) * dpad + c0) * NV + o] = sacc;
      }
      __syncthreads();
    }
  }
  C* out = part + ((int64_t)it.slot * dpad + R0) * NV;
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int j = 0; j < TV; ++j) out[(r0 + i) * NV + tv + j * (NV / TV)] = acc[i][j];
}

template <typename T, int NV>
constexpr size_t herm_smem_bytes() {
  constexpr int O = KCH * NV;
  constexpr int NT = 256;
  constexpr int P = NT / Dag<T, NV>::TPP;
  return sizeof(typename cplx<T>::t) * ((size_t)RT * (KCH + HPAD) + (size_t)KCH * NV + (size_t)RT * NV + (size_t)P * O) +
         sizeof(T) * (RT + KCH);
}

template <typename T, int GEN, int NV, int TR, int TV, int NT>
cudaError_t launch_t(const Plan& p, const void* xc, int64_t xstride, void* part, int nop, const uint64_t* seeds) {
  using C = typename cplx<T>::t;
  const size_t sm = herm_smem_bytes<T, NV>();
  auto k = rows_herm<T, GEN, NV, TR, TV, NT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const T sigma = sizeof(T) == 4 ? (T)p.sigma32 : (T)p.sigma64;
  k<<<(unsigned)p.herm_nitems, NT, sm, p.stream>>>(p.d_herm_items, p.D, p.ntile * (int64_t)kTile, p.herm_ns, nop, seeds,
                                                   p.seed, sigma, p.dvr, (const C*)xc, xstride, (C*)part,
                                                   (const C*)p.d_cache, p.d_pair_slot, p.b, p.nblk,
                                                   (const C*)p.d_hblocks);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_g(const Plan& p, const void* xc, int64_t xstride, void* part, int64_t nb, int nop,
                     const uint64_t* seeds) {
  constexpr int G = MF_GEN_PHILOX_GUE;
  switch (nb) {
    case 2: return launch_t<T, G, 2, 1, 1, 256>(p, xc, xstride, part, nop, seeds);
    case 4: return launch_t<T, G, 4, 1, 2, 256>(p, xc, xstride, part, nop, seeds);
    case 6: return launch_t<T, G, 6, 1, 3, 256>(p, xc, xstride, part, nop, seeds);
    case 8: return launch_t<T, G, 8, 2, 2, 256>(p, xc, xstride, part, nop, seeds);
    case 12: return launch_t<T, G, 12, 2, 3, 256>(p, xc, xstride, part, nop, seeds);
    case 16: return launch_t<T, G, 16, 2, 4, 256>(p, xc, xstride, part, nop, seeds);
  }
  return cudaErrorNotSupported;
}

}  // namespace

// Column items of the Hermitian multi-vector kernel: for each row tile ti the
// columns [128 ti, D) in pieces of at most w columns (a multiple of 32), w
// chosen for about 12 items per SM (a short tail); longest items first.
std::vector<HermItem> rows_herm_items(int64_t D, int num_sms, int64_t* ns_out) {
  const int64_t ntile = (D + kTile - 1) / kTile;
  const double total = 0.5 * (double)ntile * (double)(D + kTile);
  int64_t w = (int64_t)std::ceil(total / (12.0 * num_sms));
  w = std::max<int64_t>(256, (w + 31) / 32 * 32);
  std::vector<HermItem> items;
  int64_t ns = 1;
  for (int64_t ti = 0; ti < ntile; ++ti) {
    int64_t s = 0;
    for (int64_t c = ti * kTile; c < D; c += w, ++s) items.push_back(HermItem{(int32_t)ti, (int32_t)s, c, std::min(c + w, D)});
    ns = std::max(ns, s);
  }
  std::stable_sort(items.begin(), items.end(),
                   [](const HermItem& a, const HermItem& b) { return a.c_end - a.c_beg > b.c_end - b.c_beg; });
  *ns_out = ns;
  return items;
}

cudaError_t launch_rows_herm(const Plan& p, const void* xc, int64_t xstride, void* part, int64_t nb, int nop,
                             const uint64_t* seeds) {
  return p.prec == MF_PREC_FP64 ? launch_g<double>(p, xc, xstride, part, nb, nop, seeds)
                                : launch_g<float>(p, xc, xstride, part, nb, nop, seeds);
}

}  // namespace mf
