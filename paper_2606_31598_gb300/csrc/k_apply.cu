// k_apply.cu -- Hermitian canonical-tile generate-and-apply kernel (SIMT,
// one vector, and two vectors in the FP32 form).
//
// Sec. III.A ("partial caching") and Eq. blockmatvec: each CTA owns one
// canonical kTile x kTile tile (ti <= tj).  Every canonical entry h_rc
// (r <= c) is generated in registers from the Philox ensemble -- or read from
// the HBM block cache when its block pair is cached -- exactly once, and
// applied twice: y_r += h_rc x_c (block H^[n,m]) and y_c += conj(h_rc) x_r
// (block H^[m,n] = (H^[n,m])^dagger).  Row and column sums of the tile go to
// partial-sum slots that a fixed-order FP64 reduction combines.
#include <cuda_runtime.h>

#include "mf_internal.h"

namespace mf {


template <typename T> __device__ __forceinline__ typename cplx<T>::t czero();
template <> __device__ __forceinline__ float2 czero<float>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 czero<double>() { return make_double2(0.0, 0.0); }

// acc += h * x
template <typename C> __device__ __forceinline__ void cmac(C& acc, const C& h, const C& x) {
  acc.x = fma(h.x, x.x, acc.x);
  acc.x = fma(-h.y, x.y, acc.x);
  acc.y = fma(h.x, x.y, acc.y);
  acc.y = fma(h.y, x.x, acc.y);
}
// acc += conj(h) * x
template <typename C> __device__ __forceinline__ void cmacc(C& acc, const C& h, const C& x) {
  acc.x = fma(h.x, x.x, acc.x);
  acc.x = fma(h.y, x.y, acc.x);
  acc.y = fma(h.x, x.y, acc.y);
  acc.y = fma(-h.y, x.x, acc.y);
}

// Procedural part of the Hermitian tile for NV vectors: thread rows
// r0 + [0, 8), columns c0 + [0, 8); DIAG selects the diagonal tile (entries
// below the diagonal skipped, the diagonal applied once), the off-diagonal
// tiles need no test.  x rows are staged [row][NV]; the row sums of vector v
// go to red[v][tx][row].
template <typename T, int GEN, bool DIAG, int NV>
__device__ __forceinline__ void proc_tile(typename cplx<T>::t (&yc)[8][NV], const typename cplx<T>::t (&xcv)[8][NV],
                                          const typename cplx<T>::t* xs_r,
                                          typename cplx<T>::t (*red)[16][kTile + 1], int64_t r0, int64_t c0, int ty,
                                          int tx, bool active, uint64_t seed, T sigma, const dvr_consts& dk) {
  using C = typename cplx<T>::t;
#pragma unroll 2
  for (int a = 0; a < 8; ++a) {
    C yra[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) yra[v] = czero<T>();
    const int64_t r = r0 + a;
    if (active) {
      C xa[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) xa[v] = xs_r[(ty * 8 + a) * NV + v];
#pragma unroll
      for (int pb = 0; pb < 4; ++pb) {
        const int64_t c = c0 + 2 * pb;
        if (DIAG && r > c + 1) continue;  // both entries below the diagonal
        C h0, h1;
        if (GEN == MF_GEN_PHILOX_GUE) {
          gue_pair<T>(seed, sigma, (uint32_t)r, (uint32_t)(c >> 1), h0, h1);
        } else {
          h0.x = dvr_T(dk, (long long)(r - c), T());
          h1.x = dvr_T(dk, (long long)(r - c - 1), T());
          h0.y = T(0);
          h1.y = T(0);
        }
        // entry (r, c), then entry (r, c + 1): applied as H (row sum) and,
        // strictly above the diagonal, as H^dagger (column sum)
        const bool up0 = !DIAG || r < c, on0 = DIAG && r == c;
        const bool up1 = !DIAG || r < c + 1, on1 = DIAG && r == c + 1;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if (up0 || on0) cmac(yra[v], h0, xcv[2 * pb][v]);
          if (up0) cmacc(yc[2 * pb][v], h0, xa[v]);
          if (up1 || on1) cmac(yra[v], h1, xcv[2 * pb + 1][v]);
          if (up1) cmacc(yc[2 * pb + 1][v], h1, xa[v]);
        }
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) red[v][tx][ty * 8 + a] = yra[v];
  }
}

// ---------------------------------------------------------------------------
// (1) Hermitian canonical-tile kernel, NV = 1 or 2 vectors.
// Thread (ty, tx) of the 16 x 16 grid owns rows ti*128 + ty*8 + [0,8) and
// columns tj*128 + tx*8 + [0,8): 32 Philox calls, 64 canonical entries,
// each applied to the NV vectors as H and as H^dagger.  part is
// [slot][dpad][NV] (one slot per tile row).
// ---------------------------------------------------------------------------
template <typename T, int GEN, int NV>
__device__ __forceinline__ void herm_tile_body(const WorkItem* __restrict__ work, int64_t D, int64_t dpad, uint64_t seed,
                                               T sigma, const dvr_consts& dk, const typename cplx<T>::t* __restrict__ xc,
                                               typename cplx<T>::t* __restrict__ part,
                                               const typename cplx<T>::t* __restrict__ cache, int64_t bstride,
                                               const typename cplx<T>::t* __restrict__ hcache) {
  using C = typename cplx<T>::t;
  __shared__ C xs_r[kTile * NV], xs_c[kTile * NV];
  __shared__ C red[NV][16][kTile + 1];

  const WorkItem it = work[blockIdx.x];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t rt0 = (int64_t)it.ti * kTile, ct0 = (int64_t)it.tj * kTile;
  for (int e = tid; e < 2 * kTile * NV; e += 256) {
    if (e < kTile * NV) {
      const int64_t r = rt0 + e / NV;
      xs_r[e] = r < D ? xc[r * NV + e % NV] : czero<T>();
    } else {
      const int f = e - kTile * NV;
      const int64_t c = ct0 + f / NV;
      xs_c[f] = c < D ? xc[c * NV + f % NV] : czero<T>();
    }
  }
  __syncthreads();

  // column accumulators and column-side x live in registers (indexed only by
  // unrolled loop counters); the row accumulators are NV values per row a,
  // parked in shared memory when the row is done
  C yc[8][NV], xcv[8][NV];
#pragma unroll
  for (int q = 0; q < 8; ++q)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      yc[q][v] = czero<T>();
      xcv[q][v] = xs_c[(tx * 8 + q) * NV + v];
    }
  const bool diag = it.ti == it.tj;
  const int64_t r0 = rt0 + ty * 8, c0 = ct0 + tx * 8;
  const bool active = !(diag && ty > tx);

  if (it.cache_off != -1) {
    // stored block pair: stream the canonical entries from the HBM cache
    // (offset >= 0) or from the external host array (offset -2 - e),
    // 16-byte loads, two rows of the thread's 8 x 8 sub-block in flight
    constexpr int PER16 = 16 / (int)sizeof(C);  // complex entries per 16-byte load
    const C* src = it.cache_off >= 0 ? cache + it.cache_off : hcache + (-2 - it.cache_off);
    const C* base = src + (int64_t)(ty * 8) * bstride + tx * 8;
#pragma unroll 1
    for (int a2 = 0; a2 < 8; a2 += 2) {
      C h[2][8];
      if (active) {
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int q = 0; q < 8; q += PER16) {
            const float4 v = *reinterpret_cast<const float4*>(base + (int64_t)(a2 + u) * bstride + q);
            const C* e = reinterpret_cast<const C*>(&v);
#pragma unroll
            for (int i = 0; i < PER16; ++i) h[u][q + i] = e[i];
          }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int a = a2 + u;
        C yra[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) yra[v] = czero<T>();
        if (active) {
          C xa[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) xa[v] = xs_r[(ty * 8 + a) * NV + v];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int dr = (ty * 8 + a) - (tx * 8 + q);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              if (!diag || dr < 0) {
                cmac(yra[v], h[u][q], xcv[q][v]);
                cmacc(yc[q][v], h[u][q], xa[v]);
              } else if (dr == 0) {
                cmac(yra[v], h[u][q], xcv[q][v]);
              }
            }
          }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) red[v][tx][ty * 8 + a] = yra[v];
      }
    }
  } else if (diag) {
    proc_tile<T, GEN, true, NV>(yc, xcv, xs_r, red, r0, c0, ty, tx, active, seed, sigma, dk);
  } else {
    proc_tile<T, GEN, false, NV>(yc, xcv, xs_r, red, r0, c0, ty, tx, active, seed, sigma, dk);
  }

  // row sums over the 16 column groups, then column sums over the 16 row
  // groups; thread tid < 128 NV sums row tid % 128 of vector tid / 128
  const int row = tid % kTile, vv = tid / kTile;
  const bool summer = tid < kTile * NV;
  __syncthreads();
  C rs = czero<T>();
  if (summer) {
#pragma unroll
    for (int g = 0; g < 16; ++g) {
      rs.x += red[vv][g][row].x;
      rs.y += red[vv][g][row].y;
    }
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int v = 0; v < NV; ++v) red[v][ty][tx * 8 + a] = yc[a][v];
  __syncthreads();
  if (summer) {
    C cs = czero<T>();
#pragma unroll
    for (int g = 0; g < 16; ++g) {
      cs.x += red[vv][g][row].x;
      cs.y += red[vv][g][row].y;
    }
    if (diag) {
      rs.x += cs.x;
      rs.y += cs.y;
      part[((int64_t)it.ti * dpad + rt0 + row) * NV + vv] = rs;
    } else {
      part[((int64_t)it.tj * dpad + rt0 + row) * NV + vv] = rs;  // rows of tile ti, slot tj
      part[((int64_t)it.ti * dpad + ct0 + row) * NV + vv] = cs;  // rows of tile tj, slot ti
    }
  }
}

template <typename T, int GEN>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) herm_tile_nv1(const WorkItem* __restrict__ work, int64_t D,
                                                     int64_t dpad, uint64_t seed, T sigma, dvr_consts dk,
                                                     const typename cplx<T>::t* __restrict__ xc,
                                                     typename cplx<T>::t* __restrict__ part,
                                                     const typename cplx<T>::t* __restrict__ cache,
                                                     int64_t bstride,
                                                     const typename cplx<T>::t* __restrict__ hcache) {
  herm_tile_body<T, GEN, 1>(work, D, dpad, seed, sigma, dk, xc, part, cache, bstride, hcache);
}

// Two vectors: the column sums and column x of both vectors in registers.
template <typename T, int GEN>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) herm_tile_nv2(const WorkItem* __restrict__ work, int64_t D,
                                                     int64_t dpad, uint64_t seed, T sigma, dvr_consts dk,
                                                     const typename cplx<T>::t* __restrict__ xc,
                                                     typename cplx<T>::t* __restrict__ part,
                                                     const typename cplx<T>::t* __restrict__ cache,
                                                     int64_t bstride,
                                                     const typename cplx<T>::t* __restrict__ hcache) {
  herm_tile_body<T, GEN, 2>(work, D, dpad, seed, sigma, dk, xc, part, cache, bstride, hcache);
}

cudaError_t launch_gue_apply(const Plan& p, const void* xc, void* part, int64_t nvec) {
  const int64_t dpad = p.dpad;
  const unsigned grid = (unsigned)p.nwork;
  if (nvec == 2 && p.prec == MF_PREC_FP32) {
    if (p.gen != MF_GEN_SINC_DVR_HO)
      herm_tile_nv2<float, MF_GEN_PHILOX_GUE><<<grid, 256, 0, p.stream>>>(
          p.d_work, p.D, dpad, p.seed, p.sigma32, p.dvr, (const float2*)xc, (float2*)part,
          (const float2*)p.d_cache, p.b, (const float2*)p.d_hblocks);
    else
      herm_tile_nv2<float, MF_GEN_SINC_DVR_HO><<<grid, 256, 0, p.stream>>>(
          p.d_work, p.D, dpad, p.seed, p.sigma32, p.dvr, (const float2*)xc, (float2*)part,
          (const float2*)p.d_cache, p.b, (const float2*)p.d_hblocks);
    return cudaGetLastError();
  }
  if (nvec != 1) return cudaErrorNotSupported;
  if (p.prec == MF_PREC_FP64) {
    if (p.gen != MF_GEN_SINC_DVR_HO)
      herm_tile_nv1<double, MF_GEN_PHILOX_GUE><<<grid, 256, 0, p.stream>>>(
          p.d_work, p.D, dpad, p.seed, p.sigma64, p.dvr, (const double2*)xc, (double2*)part,
          (const double2*)p.d_cache, p.b, (const double2*)p.d_hblocks);
    else
      herm_tile_nv1<double, MF_GEN_SINC_DVR_HO><<<grid, 256, 0, p.stream>>>(
          p.d_work, p.D, dpad, p.seed, p.sigma64, p.dvr, (const double2*)xc, (double2*)part,
          (const double2*)p.d_cache, p.b, (const double2*)p.d_hblocks);
  } else {
    if (p.gen != MF_GEN_SINC_DVR_HO)
      herm_tile_nv1<float, MF_GEN_PHILOX_GUE><<<grid, 256, 0, p.stream>>>(
          p.d_work, p.D, dpad, p.seed, p.sigma32, p.dvr, (const float2*)xc, (float2*)part,
          (const float2*)p.d_cache, p.b, (const float2*)p.d_hblocks);
    else
      herm_tile_nv1<float, MF_GEN_SINC_DVR_HO><<<grid, 256, 0, p.stream>>>(
          p.d_work, p.D, dpad, p.seed, p.sigma32, p.dvr, (const float2*)xc, (float2*)part,
          (const float2*)p.d_cache, p.b, (const float2*)p.d_hblocks);
  }
  return cudaGetLastError();
}

}  // namespace mf
