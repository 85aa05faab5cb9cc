// rows_body.cuh -- the row-owner generate-and-apply tile (device code) shared
// by the split-K launcher (k_rows.cu) and the batched persistent kernel
// (k_batch.cu), whose chunk generation, register-tile products and block
// lookup the Hermitian-reuse (k_rows_herm.cu), system-bath (k_sysbath.cu)
// and tcgen05 (k_tc.cu) kernels also use: CTAs own a 128-row output tile and
// sweep a column range in chunks of 32 columns; each chunk of H is generated
// (canonical entries, conjugates below the diagonal, DVR window table) or
// copied from the block cache into shared memory and contracted with the
// chunk's rows of X.
#pragma once
#include "mf_internal.h"

namespace mf {

namespace rows {

constexpr int RT = 128;   // rows per CTA
constexpr int KCH = 32;   // columns per chunk
constexpr int HPAD = 1;   // pad of the chunk rows (complex elements)

template <typename T> __device__ __forceinline__ typename cplx<T>::t zc() {
  typename cplx<T>::t z;
  z.x = T(0);
  z.y = T(0);
  return z;
}

}  // namespace rows
using namespace rows;

// Block index x / b of a row or column (x < 2^31, b a multiple of 128): a
// shift when b is a power of two (the planner's sizes), else a 32-bit
// division -- never the long 64-bit division sequence.
__device__ __forceinline__ int64_t blk_of(int64_t x, int64_t b) {
  if ((b & (b - 1)) == 0) return x >> (__ffsll((long long)b) - 1);
  return (int64_t)((uint32_t)x / (uint32_t)b);
}

// Stored block pair of chunk (R0, c0): the HBM cache slot (>= 0), the host
// array block -2 - slot (<= -2) or -1 (generated); transposed when the chunk
// lies below the diagonal and is read from the canonical pair (m, n).
__device__ __forceinline__ int64_t chunk_slot(int64_t R0, int64_t c0, const void* cache, const void* hcache,
                                              const int64_t* __restrict__ slot_of_pair, int64_t b, int64_t nblk,
                                              bool& transposed) {
  transposed = false;
  if (!cache && !hcache) return -1;
  const int64_t n = blk_of(R0, b), m = blk_of(c0, b);
  if (n <= m) return slot_of_pair[n * nblk + m];
  transposed = true;
  return slot_of_pair[m * nblk + n];
}

// Loads of a stored chunk into the thread's registers (element e = tid +
// i NT of the chunk); the transposed orientation walks the stored rows
// (r fastest) so a warp reads contiguous memory.
template <typename T, int NT, int PER>
__device__ __forceinline__ void chunk_load(typename cplx<T>::t (&h)[PER], int64_t slot, bool transposed,
                                           int64_t R0, int64_t c0, const typename cplx<T>::t* __restrict__ cache,
                                           const typename cplx<T>::t* __restrict__ hcache, int64_t b) {
  const int tid = threadIdx.x;
  const int64_t n = blk_of(R0, b), m = blk_of(c0, b);
  const typename cplx<T>::t* blk = slot >= 0 ? cache + slot * b * b : hcache + (-2 - slot) * b * b;
  static_assert(NT % KCH == 0 && NT % RT == 0, "element strides must be whole rows");
  // element e = tid + i NT: (row e / KCH, column e % KCH) advances by whole
  // rows, (row e % RT, column e / RT) by whole columns
  const typename cplx<T>::t* src =
      !transposed ? blk + (R0 + tid / KCH - n * b) * b + (c0 + tid % KCH - m * b)
                  : blk + (c0 + tid / RT - m * b) * b + (R0 + tid % RT - n * b);
  const int64_t step = (int64_t)(!transposed ? NT / KCH : NT / RT) * b;
#pragma unroll
  for (int i = 0; i < PER; ++i) h[i] = src[i * step];
}

template <typename T, int NT, int PER>
__device__ __forceinline__ void chunk_store(typename cplx<T>::t* hs, const typename cplx<T>::t (&h)[PER],
                                            bool transposed) {
  constexpr int LD = KCH + HPAD;
  const int tid = threadIdx.x;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = tid + i * NT;
    if (!transposed) {
      hs[(e / KCH) * LD + e % KCH] = h[i];
    } else {
      typename cplx<T>::t v = h[i];
      v.y = -v.y;
      hs[(e % RT) * LD + e / RT] = v;
    }
  }
}

// Generate H[R0 : R0+RT, c0 : c0+W] into hs[RT][LD] (W = KCH and LD =
// KCH+HPAD unless given): canonical entries from the Philox ensemble
// (conjugates below the diagonal) or DVR entries from a window table.
template <typename T, int GEN, int NT, int LD = KCH + HPAD, int W = KCH>
__device__ __forceinline__ void fill_chunk_gen(typename cplx<T>::t* hs, T* win, int64_t R0, int64_t c0,
                                               uint64_t seed, T sigma, const dvr_consts& dk) {
  using C = typename cplx<T>::t;
  const int tid = threadIdx.x;
  if (GEN == MF_GEN_SINC_DVR_HO) {
    // window table: T(k) for k = r - c in (R0 - c0 - W, R0 - c0 + RT)
    const long long kmin = (long long)(R0 - c0) - (W - 1);
    for (int j = tid; j < RT + W - 1; j += NT) win[j] = dvr_T(dk, kmin + j, T());
    __syncthreads();
    for (int e = tid; e < RT * W; e += NT) {
      const int r = e / W, c = e % W;
      C h;
      h.x = win[r - c + W - 1];
      h.y = T(0);
      hs[r * LD + c] = h;
    }
    return;
  }
  if (c0 >= R0 + RT) {
    // strictly above the diagonal: canonical pairs along rows
    for (int e = tid; e < RT * (W / 2); e += NT) {
      const int r = e / (W / 2), pc = e % (W / 2);
      C h0, h1;
      gue_pair<T>(seed, sigma, (uint32_t)(R0 + r), (uint32_t)((c0 >> 1) + pc), h0, h1);
      hs[r * LD + 2 * pc] = h0;
      hs[r * LD + 2 * pc + 1] = h1;
    }
  } else if (c0 + W <= R0) {
    // strictly below: H[r][c] = conj(H[c][r]); canonical row c holds the
    // pair of columns (rows here) r = 2p, 2p + 1
    for (int e = tid; e < W * (RT / 2); e += NT) {
      const int c = e / (RT / 2), pr = e % (RT / 2);
      C h0, h1;
      gue_pair<T>(seed, sigma, (uint32_t)(c0 + c), (uint32_t)((R0 >> 1) + pr), h0, h1);
      h0.y = -h0.y;
      h1.y = -h1.y;
      hs[(2 * pr) * LD + c] = h0;
      hs[(2 * pr + 1) * LD + c] = h1;
    }
  } else {
    for (int e = tid; e < RT * W; e += NT) {
      const int r = e / W, c = e % W;
      hs[r * LD + c] = gue_entry<T>(seed, sigma, R0 + r, c0 + c);
    }
  }
}

// Generate (or load) H[R0 : R0+RT, c0 : c0+KCH] into hs[RT][KCH+HPAD].
template <typename T, int GEN, int NT>
__device__ __forceinline__ void fill_chunk(typename cplx<T>::t* hs, T* win, int64_t R0, int64_t c0, int64_t D,
                                           uint64_t seed, T sigma, const dvr_consts& dk,
                                           const typename cplx<T>::t* __restrict__ cache,
                                           const int64_t* __restrict__ slot_of_pair, int64_t b, int64_t nblk,
                                           const typename cplx<T>::t* __restrict__ hcache = nullptr) {
  using C = typename cplx<T>::t;
  const int tid = threadIdx.x;
  constexpr int LD = KCH + HPAD;
  // cached block pair?  (the chunk lies inside one block pair since b is a
  // multiple of 128 and chunks are 32-aligned)
  int64_t slot = -1;
  bool transposed = false;
  int64_t n = blk_of(R0, b), m = blk_of(c0, b);
  if (cache || hcache) {
    if (n <= m) {
      slot = slot_of_pair[n * nblk + m];
    } else {
      slot = slot_of_pair[m * nblk + n];
      transposed = true;
    }
  }
  if (slot >= 0 || slot <= -2) {
    // every load of the thread first, then the shared-memory stores; the
    // transposed orientation walks the cached rows (r fastest) so a warp
    // reads contiguous memory
    constexpr int PER = RT * KCH / NT;
    constexpr int HALF = PER > 8 ? PER / 2 : PER;
    // HBM cache slot, or (slot <= -2) block -2 - slot of the host array
    const C* blk = slot >= 0 ? cache + slot * b * b : hcache + (-2 - slot) * b * b;
#pragma unroll
    for (int i0 = 0; i0 < PER; i0 += HALF) {
      C h[HALF];
      if (!transposed) {
#pragma unroll
        for (int i = 0; i < HALF; ++i) {
          const int e = tid + (i0 + i) * NT, r = e / KCH, c = e % KCH;
          h[i] = blk[(R0 + r - n * b) * b + (c0 + c - m * b)];
        }
#pragma unroll
        for (int i = 0; i < HALF; ++i) {
          const int e = tid + (i0 + i) * NT;
          hs[(e / KCH) * LD + e % KCH] = h[i];
        }
      } else {
#pragma unroll
        for (int i = 0; i < HALF; ++i) {
          const int e = tid + (i0 + i) * NT, r = e % RT, c = e / RT;
          h[i] = blk[(c0 + c - m * b) * b + (R0 + r - n * b)];
        }
#pragma unroll
        for (int i = 0; i < HALF; ++i) {
          const int e = tid + (i0 + i) * NT;
          C v = h[i];
          v.y = -v.y;
          hs[(e % RT) * LD + e / RT] = v;
        }
      }
    }
    return;
  }
  fill_chunk_gen<T, GEN, NT>(hs, win, R0, c0, seed, sigma, dk);
}

// acc[i][j] += h[i] x[j] (complex) for a TR x TV register tile.  (A packed
// FP32 form of these four fused operations measured slower here: its operand
// pairs cost more registers than the issue slots it saves.)
template <typename T, int TR, int TV>
__device__ __forceinline__ void tile_cmac(typename cplx<T>::t (&acc)[TR][TV], const typename cplx<T>::t (&h)[TR],
                                          const typename cplx<T>::t (&x)[TV]) {
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

// acc[i][j] += h[i] x[j] for real h (the sinc-DVR kinetic entries, whose
// imaginary parts are exactly zero whether generated or read from the cache):
// two fused operations per product instead of four.
template <typename T, int TR, int TV>
__device__ __forceinline__ void tile_rmac(typename cplx<T>::t (&acc)[TR][TV], const typename cplx<T>::t (&h)[TR],
                                          const typename cplx<T>::t (&x)[TV]) {
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int j = 0; j < TV; ++j) {
      acc[i][j].x = fma(h[i].x, x[j].x, acc[i][j].x);
      acc[i][j].y = fma(h[i].x, x[j].y, acc[i][j].y);
    }
}

// The product of one staged entry column with the thread's rows of X.
template <typename T, int GEN, int TR, int TV>
__device__ __forceinline__ void tile_mac(typename cplx<T>::t (&acc)[TR][TV], const typename cplx<T>::t (&h)[TR],
                                         const typename cplx<T>::t (&x)[TV]) {
  if constexpr (GEN == MF_GEN_SINC_DVR_HO)
    tile_rmac<T, TR, TV>(acc, h, x);
  else
    tile_cmac<T, TR, TV>(acc, h, x);
}

// Y[R0 : R0+RT, :] over columns [cbeg, cend) -> out[row][v] (row-major,
// NV vectors per row).  Called by all NT threads of the CTA; smem_raw holds
// rows_smem_bytes<T, NV>() bytes.
template <typename T, int GEN, int NV, int TR, int TV, int NT>
__device__ __forceinline__ void row_tile(unsigned char* smem_raw, int64_t R0, int64_t cbeg, int64_t cend, int64_t D,
                                         uint64_t seed, T sigma, const dvr_consts& dk,
                                         const typename cplx<T>::t* __restrict__ xc,
                                         typename cplx<T>::t* __restrict__ out,
                                         const typename cplx<T>::t* __restrict__ cache,
                                         const int64_t* __restrict__ slot_of_pair, int64_t b, int64_t nblk,
                                         const typename cplx<T>::t* __restrict__ hcache = nullptr) {
  using C = typename cplx<T>::t;
  static_assert((RT / TR) * (NV / TV) == NT, "thread blocking must cover the tile");
  constexpr int LD = KCH + HPAD;
  C* hs = reinterpret_cast<C*>(smem_raw);      // [RT][LD]
  C* xs = hs + RT * LD;                         // [KCH][NV]
  T* win = reinterpret_cast<T*>(xs + KCH * NV);  // [RT + KCH]

  const int tid = threadIdx.x;
  const int tv = tid % (NV / TV), tr = tid / (NV / TV);
  const int r0 = tr * TR;  // thread rows r0..r0+TR-1, vectors tv + j*(NV/TV)

  C acc[TR][TV];
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int j = 0; j < TV; ++j) acc[i][j] = zc<T>();

  // FP32 with up to 16 accumulators per thread: the next stored chunk's
  // loads are issued into registers before this chunk's products, so the
  // cache (or host) latency overlaps them
  constexpr bool kPipe = sizeof(T) == 4 && TR * TV <= 16;
  constexpr int PER = RT * KCH / NT;
  C hreg[kPipe ? PER : 1];
  bool ptrans = false;
  int64_t pslot = -1;
  if (kPipe && cbeg < cend) {
    pslot = chunk_slot(R0, cbeg, cache, hcache, slot_of_pair, b, nblk, ptrans);
    if (pslot != -1) chunk_load<T, NT, kPipe ? PER : 1>(hreg, pslot, ptrans, R0, cbeg, cache, hcache, b);
  }
  for (int64_t c0 = cbeg; c0 < cend; c0 += KCH) {
    if (kPipe && pslot != -1)
      chunk_store<T, NT, kPipe ? PER : 1>(hs, hreg, ptrans);
    else
      fill_chunk<T, GEN, NT>(hs, win, R0, c0, D, seed, sigma, dk, cache, slot_of_pair, b, nblk, hcache);
    for (int e = tid; e < KCH * NV; e += NT) {
      const int64_t c = c0 + e / NV;
      xs[e] = c < cend ? xc[c * NV + e % NV] : zc<T>();
    }
    __syncthreads();
    if (kPipe) {
      pslot = -1;
      if (c0 + KCH < cend) {
        pslot = chunk_slot(R0, c0 + KCH, cache, hcache, slot_of_pair, b, nblk, ptrans);
        if (pslot != -1) chunk_load<T, NT, kPipe ? PER : 1>(hreg, pslot, ptrans, R0, c0 + KCH, cache, hcache, b);
      }
    }
#pragma unroll 4
    for (int k = 0; k < KCH; ++k) {
      C h[TR], x[TV];
#pragma unroll
      for (int i = 0; i < TR; ++i) h[i] = hs[(r0 + i) * LD + k];
#pragma unroll
      for (int j = 0; j < TV; ++j) x[j] = xs[k * NV + tv + j * (NV / TV)];
      tile_mac<T, GEN, TR, TV>(acc, h, x);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int j = 0; j < TV; ++j) out[(r0 + i) * NV + tv + j * (NV / TV)] = acc[i][j];
}

// ---------------------------------------------------------------------------
// Asynchronous variant of row_tile for the persistent batched kernel: two
// chunk buffers and two buffers for the chunk's rows of X; a stored chunk and
// the next rows of X are copied into the free buffers with cp.async (no
// registers held) while the current chunk is contracted; a generated chunk is
// generated into its buffer after the contraction.  Chunks read transposed
// from the canonical pair are stored raw and conjugated as they are used.
// smem_raw holds rows_smem_bytes_async<T, NV>() bytes.
// ---------------------------------------------------------------------------
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* dst, const void* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename T, int NT, int LD = KCH + HPAD, int W = KCH>
__device__ __forceinline__ void chunk_copy_async(typename cplx<T>::t* hb, int64_t slot, bool transposed, int64_t R0,
                                                 int64_t c0, const typename cplx<T>::t* __restrict__ cache,
                                                 const typename cplx<T>::t* __restrict__ hcache, int64_t b) {
  using C = typename cplx<T>::t;
  const int tid = threadIdx.x;
  const int64_t n = blk_of(R0, b), m = blk_of(c0, b);
  const C* blk = slot >= 0 ? cache + slot * b * b : hcache + (-2 - slot) * b * b;
  static_assert(NT % W == 0 && NT % RT == 0, "element strides must be whole rows");
  constexpr int EPP = 16 / (int)sizeof(C);  // elements per 16-byte piece
  if (!transposed && EPP == 2 && LD % 2 == 0) {
    // 16-byte pieces: staged rows start on 16-byte boundaries (LD even) and
    // so do the stored ones (even columns of a block whose side is a
    // multiple of 128); piece p = tid + i NT: row p / (W / 2)
    constexpr int PPR = W / 2;
    const int r = tid / PPR, c = 2 * (tid % PPR);
    const C* src = blk + (R0 + r - n * b) * b + (c0 + c - m * b);
    C* dst = hb + r * LD + c;
    const int64_t sstep = (int64_t)(NT / PPR) * b;
#pragma unroll 4
    for (int i = 0; i < RT * PPR / NT; ++i) cp_async_elem<16>(dst + i * (NT / PPR) * LD, src + i * sstep);
  } else if (!transposed) {
    // element e = tid + i NT: row e / W advances by NT / W, column fixed
    const int r = tid / W, c = tid % W;
    const C* src = blk + (R0 + r - n * b) * b + (c0 + c - m * b);
    C* dst = hb + r * LD + c;
    const int64_t sstep = (int64_t)(NT / W) * b;
#pragma unroll 4
    for (int i = 0; i < RT * W / NT; ++i) cp_async_elem<(int)sizeof(C)>(dst + i * (NT / W) * LD, src + i * sstep);
  } else {
    // element e = tid + i NT: row e % RT fixed, column e / RT advances by NT / RT
    const int r = tid % RT, c = tid / RT;
    const C* src = blk + (c0 + c - m * b) * b + (R0 + r - n * b);
    C* dst = hb + r * LD + c;
    const int64_t sstep = (int64_t)(NT / RT) * b;
#pragma unroll 4
    for (int i = 0; i < RT * W / NT; ++i) cp_async_elem<(int)sizeof(C)>(dst + i * (NT / RT), src + i * sstep);
  }
  cp_async_commit();
}

// Rows c0 .. c0+W-1 of X (NV vectors each, contiguous and 16-byte aligned
// since c0 is a multiple of W and NV is even) into xs[W][NV] in 16-byte
// pieces; rows at or past cend are zero-filled by plain stores.
template <typename T, int NV, int NT, int W = KCH>
__device__ __forceinline__ void xchunk_copy_async(typename cplx<T>::t* xs, const typename cplx<T>::t* __restrict__ xc,
                                                  int64_t c0, int64_t cend) {
  using C = typename cplx<T>::t;
  static_assert(NV % 2 == 0, "a 16-byte piece must not straddle two rows");
  constexpr int EPP = 16 / (int)sizeof(C);  // elements per piece
  constexpr int NP = W * NV / EPP;
  const C* src = xc + c0 * NV;
  for (int pc = threadIdx.x; pc < NP; pc += NT) {
    const int e = pc * EPP;
    if (c0 + e / NV < cend) {
      const unsigned sa = (unsigned)__cvta_generic_to_shared(xs + e);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(src + e) : "memory");
    } else {
#pragma unroll
      for (int i = 0; i < EPP; ++i) xs[e + i] = zc<T>();
    }
  }
}

// KG k-groups: the threads form KG groups, each contracting its KCH / KG
// columns of every chunk with a TR x TV register tile (rows tr + i RT/TR, so
// consecutive lanes read consecutive rows); the groups' partial sums are
// added in group order at the end of the row tile.  Larger register tiles:
// fewer shared-memory loads per FMA.
template <typename T, int GEN, int NV, int TR, int TV, int NT, int KG = 1>
__device__ __forceinline__ void row_tile_async(unsigned char* smem_raw, int64_t R0, int64_t cbeg, int64_t cend,
                                               uint64_t seed, T sigma, const dvr_consts& dk,
                                               const typename cplx<T>::t* __restrict__ xc,
                                               typename cplx<T>::t* __restrict__ out,
                                               const typename cplx<T>::t* __restrict__ cache,
                                               const int64_t* __restrict__ slot_of_pair, int64_t b, int64_t nblk) {
  using C = typename cplx<T>::t;
  static_assert((RT / TR) * (NV / TV) * KG == NT, "thread blocking must cover the tile");
  static_assert(KCH % KG == 0 && (NT / KG) % 32 == 0, "a warp belongs to one k-group");
  static_assert((size_t)(KG - 1) * RT * NV <= (size_t)2 * RT * (KCH + HPAD), "k-group sums fit the chunk buffers");
  constexpr int LD = KCH + HPAD;
  constexpr int RS = RT / TR;       // row stride of a thread's rows
  constexpr int KPG = KCH / KG;     // columns of a chunk per k-group
  C* hs0 = reinterpret_cast<C*>(smem_raw);
  C* hs1 = hs0 + RT * LD;
  C* xs0 = hs1 + RT * LD;                         // [KCH][NV]
  C* xs1 = xs0 + KCH * NV;                        // [KCH][NV]
  T* win = reinterpret_cast<T*>(xs1 + KCH * NV);  // [RT + KCH]
  const int tid = threadIdx.x;
  const int kg = tid / (NT / KG), lt = tid % (NT / KG);
  const int tv = lt % (NV / TV), tr = lt / (NV / TV);
  C acc[TR][TV];
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int j = 0; j < TV; ++j) acc[i][j] = zc<T>();
  if (cbeg >= cend) return;
  // chunk 0 and its rows of X into buffers 0
  bool conj0 = false, conj1 = false;  // chunk in buffer 0 / 1 read transposed (conjugate on use)
  {
    bool t0 = false;
    const int64_t s0 = chunk_slot(R0, cbeg, cache, nullptr, slot_of_pair, b, nblk, t0);
    xchunk_copy_async<T, NV, NT>(xs0, xc, cbeg, cend);
    if (s0 != -1) {
      chunk_copy_async<T, NT>(hs0, s0, t0, R0, cbeg, cache, nullptr, b);
      conj0 = t0;
    } else {
      cp_async_commit();
      fill_chunk_gen<T, GEN, NT>(hs0, win, R0, cbeg, seed, sigma, dk);
    }
    cp_async_wait_all();
    __syncthreads();
  }
  int k = 0;
  for (int64_t c0 = cbeg; c0 < cend; c0 += KCH, ++k) {
    C* cur = (k & 1) ? hs1 : hs0;
    C* nxt = (k & 1) ? hs0 : hs1;
    const C* xcur = (k & 1) ? xs1 : xs0;
    C* xnxt = (k & 1) ? xs0 : xs1;
    const bool cj = (k & 1) ? conj1 : conj0;
    // the free buffers were last read before the previous barrier
    const int64_t c1 = c0 + KCH;
    bool t1 = false;
    int64_t s1 = -1;
    if (c1 < cend) {
      s1 = chunk_slot(R0, c1, cache, nullptr, slot_of_pair, b, nblk, t1);
      xchunk_copy_async<T, NV, NT>(xnxt, xc, c1, cend);
      if (s1 != -1)
        chunk_copy_async<T, NT>(nxt, s1, t1, R0, c1, cache, nullptr, b);
      else
        cp_async_commit();
    }
#pragma unroll 4
    for (int kk = kg * KPG; kk < kg * KPG + KPG; ++kk) {
      C h[TR], x[TV];
#pragma unroll
      for (int i = 0; i < TR; ++i) {
        h[i] = cur[(tr + i * RS) * LD + kk];
        if (cj) h[i].y = -h[i].y;
      }
#pragma unroll
      for (int j = 0; j < TV; ++j) x[j] = xcur[kk * NV + tv + j * (NV / TV)];
      tile_mac<T, GEN, TR, TV>(acc, h, x);
    }
    // (the window table was last read before the previous barrier)
    if (c1 < cend && s1 == -1) fill_chunk_gen<T, GEN, NT>(nxt, win, R0, c1, seed, sigma, dk);
    if (k & 1)
      conj0 = s1 != -1 && t1;
    else
      conj1 = s1 != -1 && t1;
    cp_async_wait_all();
    __syncthreads();
  }
  if constexpr (KG > 1) {
    // the chunk buffers are free after the last barrier: groups 1.. leave
    // their sums there, group 0 adds them in group order
    C* red = hs0;  // [KG - 1][RT][NV]
    if (kg > 0) {
#pragma unroll
      for (int i = 0; i < TR; ++i)
#pragma unroll
        for (int j = 0; j < TV; ++j) red[((kg - 1) * RT + tr + i * RS) * NV + tv + j * (NV / TV)] = acc[i][j];
    }
    __syncthreads();
    if (kg > 0) return;
#pragma unroll
    for (int g = 1; g < KG; ++g)
#pragma unroll
      for (int i = 0; i < TR; ++i)
#pragma unroll
        for (int j = 0; j < TV; ++j) {
          const C v = red[((g - 1) * RT + tr + i * RS) * NV + tv + j * (NV / TV)];
          acc[i][j].x += v.x;
          acc[i][j].y += v.y;
        }
  }
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int j = 0; j < TV; ++j) out[(tr + i * RS) * NV + tv + j * (NV / TV)] = acc[i][j];
}

// ---------------------------------------------------------------------------
// FP32 form of row_tile_async: a ring of S stages of W-column chunks, S - 1
// chunks (stored entries and rows of X) in flight while one is contracted
// (two stages of 32 columns: deeper rings of 16- or 32-column chunks timed
// 1-8 % slower, the contraction and not the copies' latency being what the
// ring waits for).  The staged
// rows have an even pitch (W + 2 complex, 16-byte aligned): a thread reads the
// entries of two consecutive columns in one 16-byte load and its TV
// contiguous vectors (tv TV .. tv TV + TV - 1) in 16-byte pieces; stored
// chunks are copied in 16-byte pieces, those read transposed kept in their
// stored orientation (two 8-byte loads per row and column pair).  The product
// is taken in packed FP32 pairs: A += (h_r, h_r) x and B += (h_i, h_i) x over
// the row tile, Y = A + i B at its end (the conjugate of a transposed chunk
// negates h_i, a compile-time branch of the contraction).
// ---------------------------------------------------------------------------
constexpr int F32_W = 32;  // columns per staged chunk
constexpr int F32_S = 2;   // stages of the ring

template <int W>
__host__ __device__ constexpr int f32_ld() { return W + 2; }

// A[i][j] += h_i x_j (real parts of h, or all of h for the real DVR entries)
// and B[i][j] += h_i^im x_j over the column pairs kk0 .. kk0 + KPG - 1 of the
// staged chunk (h_i^im negated when CJ).
template <int GEN, int NV, int TR, int TV, int KPG, int LD, bool CJ>
__device__ __forceinline__ void contract_f32(float2 (&A)[TR][TV], float2 (&B)[TR][TV], const float2* __restrict__ hst,
                                             int tr, const float2* __restrict__ xcol, int kk0) {
  constexpr int RS = RT / TR;
#pragma unroll (KPG <= 4 ? 2 : 1)
  for (int kk = kk0; kk < kk0 + KPG; kk += 2) {
    // h[i] = (H[r][kk], H[r][kk + 1]) of row r = tr + i RS: one 16-byte
    // load from a row-major chunk, two 8-byte loads from a transposed one
    float4 h[TR];
#pragma unroll
    for (int i = 0; i < TR; ++i) {
      if constexpr (CJ) {
        const float2 a = hst[kk * RT + tr + i * RS], c = hst[(kk + 1) * RT + tr + i * RS];
        h[i] = make_float4(a.x, a.y, c.x, c.y);
      } else {
        h[i] = *reinterpret_cast<const float4*>(hst + (tr + i * RS) * LD + kk);
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      float4 x[TV / 2];
#pragma unroll
      for (int m = 0; m < TV / 2; ++m) x[m] = *reinterpret_cast<const float4*>(xcol + (kk + q) * NV + 2 * m);
#pragma unroll
      for (int i = 0; i < TR; ++i) {
        const float hr = q ? h[i].z : h[i].x, hi = q ? h[i].w : h[i].y;
        const float2 hrr = make_float2(hr, hr);
        const float2 hii = CJ ? make_float2(-hi, -hi) : make_float2(hi, hi);
#pragma unroll
        for (int m = 0; m < TV / 2; ++m) {
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const float2 xv = u ? make_float2(x[m].z, x[m].w) : make_float2(x[m].x, x[m].y);
            A[i][2 * m + u] = __ffma2_rn(hrr, xv, A[i][2 * m + u]);
            if constexpr (GEN != MF_GEN_SINC_DVR_HO) B[i][2 * m + u] = __ffma2_rn(hii, xv, B[i][2 * m + u]);
          }
        }
      }
    }
  }
}

// A stored chunk read transposed (stored rows c0 .. c0 + W - 1 of the block
// pair hold H[c][r] for the tile's rows r) copied as it is stored, hb[c][r]
// with a pitch of RT, in 16-byte pieces (two rows r, r + 1 of one stored row;
// R0 + r is even and a stored block's side a multiple of 128).
template <int NT, int W>
__device__ __forceinline__ void chunk_copy_async_t(float2* hb, int64_t slot, int64_t R0, int64_t c0,
                                                   const float2* __restrict__ cache, int64_t b) {
  constexpr int PPR = RT / 2;  // pieces per stored row
  static_assert((PPR * W) % NT == 0 && NT % PPR == 0, "pieces in whole passes");
  const int tid = threadIdx.x;
  const int64_t n = blk_of(R0, b), m = blk_of(c0, b);
  const float2* blk = cache + slot * b * b;
  const int c = tid / PPR, pr = tid % PPR;
  const float2* src = blk + (c0 + c - m * b) * b + (R0 + 2 * pr - n * b);
  float2* dst = hb + c * RT + 2 * pr;
  const int64_t sstep = (int64_t)(NT / PPR) * b;
#pragma unroll 4
  for (int i = 0; i < PPR * W / NT; ++i) cp_async_elem<16>(dst + i * (NT / PPR) * RT, src + i * sstep);
  cp_async_commit();
}

// The generation of a chunk out of line: it is the rare path of the ring
// (stored chunks are the common one), and inlined it would hold registers
// across the whole contraction.
template <int GEN, int NT, int LD, int W>
__device__ __noinline__ void fill_chunk_gen_f32(float2* hs, float* win, int64_t R0, int64_t c0, uint64_t seed,
                                                float sigma, dvr_consts dk) {
  fill_chunk_gen<float, GEN, NT, LD, W>(hs, win, R0, c0, seed, sigma, dk);
}

template <int GEN, int NV, int TR, int TV, int NT, int KG = 1, int W = F32_W, int S = F32_S>
__device__ __forceinline__ void row_tile_async_f32(unsigned char* smem_raw, int64_t R0, int64_t cbeg, int64_t cend,
                                                   uint64_t seed, float sigma, const dvr_consts& dk,
                                                   const float2* __restrict__ xc, float2* __restrict__ out,
                                                   const float2* __restrict__ cache,
                                                   const int64_t* __restrict__ slot_of_pair, int64_t b, int64_t nblk) {
  using C = float2;
  constexpr int LD = f32_ld<W>();
  constexpr int RS = RT / TR;
  constexpr int KPG = W / KG;
  static_assert((RT / TR) * (NV / TV) * KG == NT, "thread blocking must cover the tile");
  static_assert(W % (2 * KG) == 0 && (NT / KG) % 32 == 0, "a warp belongs to one k-group, column pairs");
  static_assert(TV % 2 == 0 && NV % TV == 0, "vectors in 16-byte pieces");
  static_assert(S >= 2 && S <= 32 && 128 % W == 0, "a ring of whole chunks inside one stored block");
  static_assert((size_t)(KG - 1) * RT * NV <= (size_t)S * RT * LD, "k-group sums fit the chunk ring");
  C* hs = reinterpret_cast<C*>(smem_raw);                // [S][RT][LD]
  C* xs = hs + S * RT * LD;                              // [S][W][NV]
  float* win = reinterpret_cast<float*>(xs + S * W * NV);  // [RT + W]
  const int tid = threadIdx.x;
  const int kg = tid / (NT / KG), lt = tid % (NT / KG);
  const int tv = lt % (NV / TV), tr = lt / (NV / TV);
  C A[TR][TV], B[TR][TV];
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int j = 0; j < TV; ++j) A[i][j] = B[i][j] = zc<float>();
  if (cbeg >= cend) return;
  const int64_t nch = (cend - cbeg + W - 1) / W;
  uint32_t conj = 0;  // bit s: the chunk in stage s was read transposed (conjugate on use)
  // the stored block of the current column block: looked up once per block,
  // not per chunk (a dependent global load in front of every copy otherwise)
  int64_t blk_m = -1, sl = -1;
  bool t = false;
  // chunk q into stage q % S: one cp.async group per chunk (empty past the
  // end); a generated chunk is written by plain stores, visible after the
  // barrier that precedes its use
  auto issue = [&](int64_t q) {
    const int st = (int)(q % S);
    if (q >= nch) {
      cp_async_commit();
      return;
    }
    const int64_t c0 = cbeg + q * W;
    if (cache && blk_of(c0, b) != blk_m) {
      blk_m = blk_of(c0, b);
      sl = chunk_slot(R0, c0, cache, nullptr, slot_of_pair, b, nblk, t);
    }
    xchunk_copy_async<float, NV, NT, W>(xs + st * W * NV, xc, c0, cend);
    if (sl != -1 && t) {
      chunk_copy_async_t<NT, W>(hs + st * RT * LD, sl, R0, c0, cache, b);
      conj |= 1u << st;
    } else if (sl != -1) {
      chunk_copy_async<float, NT, LD, W>(hs + st * RT * LD, sl, false, R0, c0, cache, nullptr, b);
      conj &= ~(1u << st);
    } else {
      cp_async_commit();
      fill_chunk_gen_f32<GEN, NT, LD, W>(hs + st * RT * LD, win, R0, c0, seed, sigma, dk);
      conj &= ~(1u << st);
    }
  };
#pragma unroll 1
  for (int q = 0; q < S - 1; ++q) issue(q);
#pragma unroll 1
  for (int64_t k = 0; k < nch; ++k) {
    // chunk k has landed (for this thread's copies; the barrier for all
    // threads'), and the stage of chunk k - 1 is free for chunk k + S - 1
    asm volatile("cp.async.wait_group %0;" ::"n"(S - 2) : "memory");
    __syncthreads();
    issue(k + S - 1);
    const int st = (int)(k % S);
    const C* hst = hs + st * RT * LD;
    const C* xcol = xs + st * W * NV + tv * TV;
    if ((conj >> st) & 1u)
      contract_f32<GEN, NV, TR, TV, KPG, LD, true>(A, B, hst, tr, xcol, kg * KPG);
    else
      contract_f32<GEN, NV, TR, TV, KPG, LD, false>(A, B, hst, tr, xcol, kg * KPG);
  }
  cp_async_wait_all();
  __syncthreads();  // every thread is done with the ring
  if constexpr (GEN != MF_GEN_SINC_DVR_HO) {
#pragma unroll
    for (int i = 0; i < TR; ++i)
#pragma unroll
      for (int j = 0; j < TV; ++j) {
        A[i][j].x -= B[i][j].y;
        A[i][j].y += B[i][j].x;
      }
  }
  if constexpr (KG > 1) {
    C* red = hs;  // [KG - 1][RT][NV]
    if (kg > 0) {
#pragma unroll
      for (int i = 0; i < TR; ++i)
#pragma unroll
        for (int j = 0; j < TV; ++j) red[((kg - 1) * RT + tr + i * RS) * NV + tv * TV + j] = A[i][j];
    }
    __syncthreads();
    if (kg > 0) return;
#pragma unroll
    for (int g = 1; g < KG; ++g)
#pragma unroll
      for (int i = 0; i < TR; ++i)
#pragma unroll
        for (int j = 0; j < TV; ++j) {
          const C v = red[((g - 1) * RT + tr + i * RS) * NV + tv * TV + j];
          A[i][j].x += v.x;
          A[i][j].y += v.y;
        }
  }
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int j = 0; j < TV; ++j) out[(tr + i * RS) * NV + tv * TV + j] = A[i][j];
}

// ---------------------------------------------------------------------------
// Hermitian-reuse form of the FP32 ring tile (Sec. III.A canonical-pair
// reuse) for few vectors, where the stored bytes bound the product: row tile
// I sweeps only the upper band, columns [128 I, D), so every stored chunk is
// read once (always in its stored orientation) and applied twice -- as H to
// the tile's rows (register tiles, as row_tile_async_f32) and, for chunks
// strictly above the diagonal tile, as H^dagger to the chunk's W rows:
// Y[c][v] = sum_r conj(H[r][c]) X[r][v].  The H^dagger sum runs over the
// tile's rows in P parts of threads (CT = 1 column x NV vectors each, in
// packed FP32 pairs: A' += (h_r, h_r) x, B' += (h_i, h_i) x, conj(h) x =
// A' - i B'); the parts are added in fixed order after the next barrier and
// written to slot 1 + I of the chunk's rows: outd + (I * dpad + c) NV.  The
// owner rows go to out as in row_tile_async_f32.  Every slot that the
// reduction reads is written once per product.
// ---------------------------------------------------------------------------
template <int NV>
struct HermF32 {
  static constexpr int TPP = F32_W;      // threads per part: one column each, all NV vectors
  static constexpr int P = 256 / TPP;    // parts (256 threads)
  static constexpr int RP = RT / P;      // rows per part
  static constexpr int O = F32_W * NV;   // outputs per chunk
};

template <int NV, int W = F32_W, int S = F32_S>
__host__ __device__ constexpr size_t herm_smem_bytes_f32() {
  return sizeof(float2) * ((size_t)S * RT * f32_ld<W>() + (size_t)S * W * NV + (size_t)RT * NV +
                           2 * (size_t)HermF32<NV>::P * HermF32<NV>::O) +
         sizeof(float) * (RT + W);
}

template <int GEN, int NV, int TR, int TV, int NT, int KG>
__device__ __forceinline__ void row_tile_herm_f32(unsigned char* smem_raw, int64_t R0, int64_t D, uint64_t seed,
                                                  float sigma, const dvr_consts& dk, const float2* __restrict__ xc,
                                                  float2* __restrict__ out, float2* __restrict__ outd, int64_t dpad,
                                                  const float2* __restrict__ cache,
                                                  const int64_t* __restrict__ slot_of_pair, int64_t b, int64_t nblk) {
  using C = float2;
  constexpr int W = F32_W, S = F32_S;
  constexpr int LD = f32_ld<W>();
  constexpr int RS = RT / TR;
  constexpr int KPG = W / KG;
  using HP = HermF32<NV>;
  constexpr int P = HP::P, RP = HP::RP, O = HP::O;
  static_assert(NT == 256 && S == 2, "the part layout assumes 256 threads and two stages");
  static_assert((RT / TR) * (NV / TV) * KG == NT, "thread blocking must cover the tile");
  static_assert(W % (2 * KG) == 0 && (NT / KG) % 32 == 0, "a warp belongs to one k-group, column pairs");
  static_assert(TV % 2 == 0 && NV % TV == 0 && NV % 2 == 0, "vectors in 16-byte pieces");
  static_assert((size_t)(KG - 1) * RT * NV <= (size_t)S * RT * LD, "k-group sums fit the chunk ring");
  C* hs = reinterpret_cast<C*>(smem_raw);   // [S][RT][LD]
  C* xs = hs + S * RT * LD;                 // [S][W][NV]
  C* xr = xs + S * W * NV;                  // [RT][NV]: the tile's rows of X
  C* red = xr + RT * NV;                    // [2][P][O]: H^dagger parts
  float* win = reinterpret_cast<float*>(red + 2 * P * O);  // [RT + W]
  const int tid = threadIdx.x;
  const int kg = tid / (NT / KG), lt = tid % (NT / KG);
  const int tv = lt % (NV / TV), tr = lt / (NV / TV);
  const int dp = tid / HP::TPP, dc = tid % HP::TPP;  // H^dagger part and column
  C A[TR][TV], B[TR][TV];
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int j = 0; j < TV; ++j) A[i][j] = B[i][j] = zc<float>();
  const int64_t cbeg = R0;
  const int64_t nch = (D - cbeg + W - 1) / W;
  // the tile's rows of X (zero past D), in the first copy group
  for (int pc = tid; pc < RT * NV / 2; pc += NT) {
    const int e = 2 * pc;
    if (R0 + e / NV < D)
      cp_async_elem<16>(xr + e, xc + R0 * NV + e);
    else
      xr[e] = xr[e + 1] = zc<float>();
  }
  int64_t blk_m = -1, sl = -1;
  bool t = false;
  auto issue = [&](int64_t q) {
    const int st = (int)(q % S);
    if (q >= nch) {
      cp_async_commit();
      return;
    }
    const int64_t c0 = cbeg + q * W;
    if (cache && blk_of(c0, b) != blk_m) {
      blk_m = blk_of(c0, b);
      sl = chunk_slot(R0, c0, cache, nullptr, slot_of_pair, b, nblk, t);  // c0 >= R0: never transposed
    }
    xchunk_copy_async<float, NV, NT, W>(xs + st * W * NV, xc, c0, D);
    if (sl != -1) {
      chunk_copy_async<float, NT, LD, W>(hs + st * RT * LD, sl, false, R0, c0, cache, nullptr, b);
    } else {
      cp_async_commit();
      fill_chunk_gen_f32<GEN, NT, LD, W>(hs + st * RT * LD, win, R0, c0, seed, sigma, dk);
    }
  };
  // H^dagger parts of chunk q (in red[q % 2]) added in part order and stored
  auto drain = [&](int64_t q) {
    const C* rq = red + (q % 2) * P * O;
    const int64_t c0 = cbeg + q * W;
    for (int o = tid; o < O; o += NT) {
      C v = rq[o];
#pragma unroll
      for (int p2 = 1; p2 < P; ++p2) {
        v.x += rq[p2 * O + o].x;
        v.y += rq[p2 * O + o].y;
      }
      outd[(c0 + o / NV) * NV + o % NV] = v;
    }
  };
  issue(0);
  for (int64_t k = 0; k < nch; ++k) {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    const int64_t c0 = cbeg + k * W;
    if (k > 0 && c0 - W >= R0 + RT) drain(k - 1);
    issue(k + 1);
    const int st = (int)(k % S);
    const C* hst = hs + st * RT * LD;
    contract_f32<GEN, NV, TR, TV, KPG, LD, false>(A, B, hst, tr, xs + st * W * NV + tv * TV, kg * KPG);
    if (c0 >= R0 + RT) {
      // Y[c][v] over this part's rows: A' += h_r x, B' += h_i x
      C Ad[NV], Bd[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) Ad[v] = Bd[v] = zc<float>();
#pragma unroll 4
      for (int r = dp * RP; r < dp * RP + RP; ++r) {
        const C h = hst[r * LD + dc];
        const float2 hrr = make_float2(h.x, h.x), hii = make_float2(h.y, h.y);
#pragma unroll
        for (int m = 0; m < NV / 2; ++m) {
          const float4 x4 = *reinterpret_cast<const float4*>(xr + r * NV + 2 * m);
          const float2 x0 = make_float2(x4.x, x4.y), x1 = make_float2(x4.z, x4.w);
          Ad[2 * m] = __ffma2_rn(hrr, x0, Ad[2 * m]);
          Ad[2 * m + 1] = __ffma2_rn(hrr, x1, Ad[2 * m + 1]);
          if constexpr (GEN != MF_GEN_SINC_DVR_HO) {
            Bd[2 * m] = __ffma2_rn(hii, x0, Bd[2 * m]);
            Bd[2 * m + 1] = __ffma2_rn(hii, x1, Bd[2 * m + 1]);
          }
        }
      }
      C* rq = red + (k % 2) * P * O + dp * O + dc * NV;
#pragma unroll
      for (int v = 0; v < NV; ++v) rq[v] = make_float2(Ad[v].x + Bd[v].y, Ad[v].y - Bd[v].x);
    }
  }
  cp_async_wait_all();
  __syncthreads();  // every thread is done with the ring and the last parts
  if (nch > 0 && cbeg + (nch - 1) * W >= R0 + RT) drain(nch - 1);
  if constexpr (GEN != MF_GEN_SINC_DVR_HO) {
#pragma unroll
    for (int i = 0; i < TR; ++i)
#pragma unroll
      for (int j = 0; j < TV; ++j) {
        A[i][j].x -= B[i][j].y;
        A[i][j].y += B[i][j].x;
      }
  }
  if constexpr (KG > 1) {
    C* kred = hs;  // [KG - 1][RT][NV]
    if (kg > 0) {
#pragma unroll
      for (int i = 0; i < TR; ++i)
#pragma unroll
        for (int j = 0; j < TV; ++j) kred[((kg - 1) * RT + tr + i * RS) * NV + tv * TV + j] = A[i][j];
    }
    __syncthreads();
    if (kg > 0) return;
#pragma unroll
    for (int g = 1; g < KG; ++g)
#pragma unroll
      for (int i = 0; i < TR; ++i)
#pragma unroll
        for (int j = 0; j < TV; ++j) {
          const C v = kred[((g - 1) * RT + tr + i * RS) * NV + tv * TV + j];
          A[i][j].x += v.x;
          A[i][j].y += v.y;
        }
  }
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int j = 0; j < TV; ++j) out[(tr + i * RS) * NV + tv * TV + j] = A[i][j];
}

template <int NV, int W = F32_W, int S = F32_S>
__host__ __device__ constexpr size_t rows_smem_bytes_f32() {
  return sizeof(float2) * ((size_t)S * RT * f32_ld<W>() + (size_t)S * W * NV) + sizeof(float) * (RT + W);
}

template <typename T, int NV>
__host__ __device__ constexpr size_t rows_smem_bytes_async() {
  return sizeof(typename cplx<T>::t) * (2 * (size_t)RT * (KCH + HPAD) + 2 * (size_t)KCH * NV) + sizeof(T) * (RT + KCH);
}

template <typename T, int NV>
__host__ __device__ constexpr size_t rows_smem_bytes() {
  return sizeof(typename cplx<T>::t) * ((size_t)RT * (KCH + HPAD) + (size_t)KCH * NV) + sizeof(T) * (RT + KCH);
}

}  // namespace mf


