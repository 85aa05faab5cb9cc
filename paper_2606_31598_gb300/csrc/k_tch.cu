// k_tch.cu -- multi-vector generate-and-apply on the 5th-generation tensor
// cores with Hermitian reuse, BF16 hi+lo split form.
//
// Every canonical 128 x 128 tile H^[ti,tj] (ti <= tj; Sec. III.A caches and
// generates canonical pairs only) is generated once, or read once from the
// FP32 block cache, split into bf16 planes (re hi, re lo, im hi, im lo) in
// shared memory, and applied twice by tcgen05.mma:
//   H product   Y[ti] += H X[tj]:   A = the planes read K-major (rows x cols);
//   H^dag prod. Y[tj] += H^dag X[ti]: the same planes read MN-major (the
//               transpose), with the conjugate carried by the operand tiles:
//               H^dag X = Re(H)^T [Re X | Im X] + Im(H)^T [Im X | -Re X].
// X is pre-split per apply into operand tiles of 32 rows:
//   B1 = [Re X | Im X], B2 = [-Im X | Re X], B3 = -B2 (hi and lo each).
// The H product uses (A_re, B1) and (A_im, B2), the H^dag product
// (A_re^T, B1) and (A_im^T, B3); each real product is hi*hi + hi*lo + lo*hi.
//
// Work is cut into square units of s x s tiles of the upper triangle.  A
// persistent CTA (one per SM) takes units from an atomic counter; inside a
// unit it walks bands of W = 2 tile rows, and for each column tile tj of the
// unit (a "step") the band's tiles (a, tj).  The band's H products
// accumulate in W TMEM accumulators (one per band row) across the steps;
// the step's H^dag products accumulate in one of two further accumulators
// (alternating by step), drained into the unit's slot rows of tj while the
// next step runs.  The band
// accumulators are drained every SEG steps (the tensor core's FP32
// accumulation is not round-to-nearest over long chains) and at the end of
// the band.  Each unit owns its own slot rows (its row range and, off the
// diagonal, its column range), written first and then added to with
// round-to-nearest FP32 adds, so the result does not depend on which CTA
// ran which unit; tch_gather sums a row's unit partials in FP64 in a fixed
// order.
//
// Roles inside a CTA (640 threads): 18 generator warps fill the A tile
// region by region and drain the accumulators; one thread of the copy warp
// streams the operand tiles with bulk asynchronous copies into a ring of
// NBUF slots, running ahead of the MMAs as far as the ring allows; one
// thread of the MMA warp issues the MMAs (and copies cached tiles into A).  Tiles
// alternate their fill orientation (column chunks, then row chunks): the
// product that runs along the fill overlaps it, the other one releases the
// A regions the next tile fills first, so generation never waits for a
// whole tile's MMAs.  Every wait
// is bounded: on time-out the thread records a code in the error word (in
// 130..139), the CTA stops, waits (with a fixed long bound) for the copies
// and MMAs it issued, frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "rows_body.cuh"
#include "tc_ptx.cuh"

namespace mf {
namespace tch {

using namespace ptx;

constexpr int RT = 128;                    // tile edge
constexpr int KC = 32;                     // K rows per operand copy / columns per chunk of the tile
constexpr int NGEN = 18;                   // generator warps
constexpr int GT = NGEN * 32;              // generator threads
// The MMA warp sits in SM sub-partition 3 and the operand-copy warp in
// sub-partition 2 (warp % 4), each beside 4 generator warps; sub-partitions
// 0 and 1 hold 5.  Generator warp w is generator number
// w - (w > LOAD_WARP) - (w > MMA_WARP).  20 warps leave the kernel 96
// registers per thread (24 warps: 80, with spills).
constexpr int LOAD_WARP = 2;               // operand-copy warp
constexpr int MMA_WARP = 3;                // MMA warp (also copies cached tiles into A)
constexpr int NTHREADS = (NGEN + 2) * 32;  // 640: 5 warps per SM sub-partition
constexpr int W = 2;                       // tile rows per band (band accumulators)
constexpr int SEG = 8;                     // steps between drains of the band accumulators
constexpr int PLANE = RT * RT * 2;         // one bf16 plane of the tile: 32 KB
constexpr int A_BYTES = 4 * PLANE;         // 128 KB
constexpr int PAIRS = RT * RT / 2;         // horizontal entry pairs of a tile
constexpr int CPAIRS = RT * KC / 2;        // pairs of a 32-column chunk
constexpr int MAXPR = (CPAIRS + GT - 1) / GT;  // pairs of a region per generator thread (at most)
constexpr int kMaxSmem = 229376;           // dynamic shared memory this kernel may take
constexpr uint32_t kDrainSpin = kDefaultSpin;

template <int NV>
struct Cfg {
  static constexpr int N = 2 * NV;                 // MMA N: [Re | Im] of NV vectors
  static constexpr int BT = N * KC * 2;            // bytes of one operand tile (N x 32 bf16)
  static constexpr int BSLOT = 4 * BT;             // one copy: four operand tiles
  static constexpr int NBUF = (A_BYTES + 3 * BSLOT <= kMaxSmem) ? 3 : 2;
  static constexpr int QC = N / 4;                 // TMEM columns per thread in a drain
  // accumulators: W band rows (H products), two for the steps' H^dag partials
  static constexpr uint32_t TMEM_COLS = (uint32_t)((W + 2) * N) < 32u ? 32u : (uint32_t)((W + 2) * N);
  static constexpr size_t SMEM = (size_t)A_BYTES + (size_t)NBUF * BSLOT;
};

// Byte offset of element (r, c) in one plane of the A tile: canonical
// no-swizzle core matrices (8 rows x 16 bytes), column groups fastest.
// Read K-major (the H product): LBO = 128 B (next 8 columns), SBO = 2048 B
// (next 8 rows).  Read MN-major (the transpose): LBO = 2048 B (next 8 rows,
// now the K direction), SBO = 128 B (next 8 columns, now M).  The block
// cache of these plans stores every tile in this layout too (four planes
// back to back), so a cached tile is copied as it is.
__host__ __device__ __forceinline__ uint32_t aoff(int r, int c) {
  return (uint32_t)((r >> 3) * 2048 + (c >> 3) * 128 + (r & 7) * 16 + (c & 7) * 2);
}
// Operand tile (N x 32, K-major): LBO = 128 B, SBO = 512 B.
__host__ __device__ __forceinline__ uint32_t boff(int n, int k) {
  return (uint32_t)((n >> 3) * 512 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2);
}

// Pair p (0 .. CPAIRS-1) of region q of a tile -> its row and even column.
// Orientation 0: region q is column chunk q (32 columns, all rows): 16 row
// groups x 4 column groups of core matrices.  Orientation 1: region q is row
// chunk q (32 rows, all columns): 4 row groups x 16 column groups.  The 32
// pairs of a warp's store (p = 32 k .. 32 k + 31) fill one 128-byte core
// matrix: rows 8 rg + lane / 4, columns 8 cg + 2 (lane % 4), +1.
__device__ __forceinline__ void region_rc(int o, int q, int p, int& r, int& c) {
  const int cb = p >> 5, l = p & 31;
  if (o == 0) {
    r = 8 * (cb >> 2) + (l >> 2);
    c = 32 * q + 8 * (cb & 3) + 2 * (l & 3);
  } else {
    r = 32 * q + 8 * (cb >> 4) + (l >> 2);
    c = 8 * (cb & 15) + 2 * (l & 3);
  }
}

// The bf16 plane words of entries (r, c), (r, c + 1) of the tile at (R0, C0):
// the FP32-form entries of the Philox ensemble (conjugates below the
// diagonal of a diagonal tile), split hi + lo.
__device__ __forceinline__ void gen_words(uint64_t seed, float sigma, int64_t R0, int64_t C0, bool diag_tile, int r,
                                          int c, uint32_t* w) {
  float2 h0, h1;
  if (!diag_tile) {
    gue_pair<float>(seed, sigma, (uint32_t)(R0 + r), (uint32_t)((C0 + c) >> 1), h0, h1);
  } else {
    h0 = gue_entry<float>(seed, sigma, R0 + r, C0 + c);
    h1 = gue_entry<float>(seed, sigma, R0 + r, C0 + c + 1);
  }
  split_pair(h0, h1, w);
}

__device__ __forceinline__ void put_words(unsigned char* A, int r, int c, const uint32_t* w) {
  const uint32_t off = aoff(r, c);
#pragma unroll
  for (int pl = 0; pl < 4; ++pl) *reinterpret_cast<uint32_t*>(A + pl * PLANE + off) = w[pl];
}

// Tile traversal of one unit: bands of W rows, steps over the unit's column
// tiles, the band's tiles of each step.  The MMA thread and the generator
// warps walk the same sequence.
struct Walk {
  int r0, r1, c0, c1;  // tile rows [r0, r1), tile columns [c0, c1)
  bool diag;
  int br, bw, tj, a, sib;  // band start and height, step column, tile row, step index in the band
  __device__ void start(int ur, int uc, int s, int T) {
    r0 = ur * s;
    r1 = min(T, r0 + s);
    c0 = uc * s;
    c1 = min(T, c0 + s);
    diag = ur == uc;
    br = r0;
    bw = min(W, r1 - br);
    tj = diag ? br : c0;
    a = br;
    sib = 0;
  }
  __device__ int a_end() const { return min(br + bw, tj + 1); }
  __device__ bool step_end() const { return a + 1 == a_end(); }
  __device__ bool step_has_herm() const { return br < tj; }  // the band's first row is the smallest
  __device__ bool d1_drain() const { return tj + 1 == c1 || (sib + 1) % SEG == 0; }
  __device__ bool drain() const { return step_has_herm() || d1_drain(); }
  // advance to the next tile; false at the end of the unit
  __device__ bool next() {
    if (++a < a_end()) return true;
    if (++tj < c1) {
      a = br;
      ++sib;
      return true;
    }
    br += W;
    if (br >= r1) return false;
    bw = min(W, r1 - br);
    tj = diag ? br : c0;
    a = br;
    sib = 0;
    return true;
  }
};

// The jobs of the MMA thread, in issue order.  A job is the H product of
// column chunk c (operand rows 32 c.. of X[tj]) or the H^dag product of row
// chunk r (operand rows 32 r.. of X[a]).  Tiles alternate their fill
// orientation with the CTA's running tile count: an even tile is filled by
// column chunks, so its H product follows the fill and its H^dag product
// comes after, releasing row chunks; an odd tile is filled by row chunks,
// the H^dag product follows the fill and the H product comes after,
// releasing column chunks.  Diagonal tiles have only the H product.
struct JobWalk {
  Walk w;
  int k;
  uint32_t tile;  // the CTA's running tile count of w's tile
  bool live;
  __device__ bool herm() const { return w.a < w.tj; }
  __device__ int njobs() const { return herm() ? 8 : 4; }
  __device__ int orient() const { return (int)(tile & 1u); }
  // true: H product of column chunk idx(); false: H^dag product of row chunk idx()
  __device__ bool is_h() const { return !herm() || (orient() == 0 ? k < 4 : k >= 4); }
  __device__ int idx() const { return k & 3; }
  __device__ void start(int ur, int uc, int s, int T, uint32_t tile0) {
    w.start(ur, uc, s, T);
    k = 0;
    tile = tile0;
    live = true;
  }
  __device__ void next() {
    if (++k < njobs()) return;
    k = 0;
    ++tile;
    live = w.next();
  }
};

// Cache slot of tile (a, tj) (a <= tj: canonical orientation), -1 when generated.
__device__ __forceinline__ int64_t tile_slot(int a, int tj, const unsigned char* ccache,
                                             const int64_t* __restrict__ slot_of_pair, int64_t b, int64_t nblk) {
  if (!ccache) return -1;
  return slot_of_pair[blk_of((int64_t)a * RT, b) * nblk + blk_of((int64_t)tj * RT, b)];
}
// Byte offset of tile (a, tj) in the consumer-format cache: its block's
// slot, then the tile's place in the block (row-major over the (b/128)^2
// tiles), 128 KB per tile.
__device__ __forceinline__ int64_t tile_cache_off(int a, int tj, int64_t slot, int64_t b) {
  const int64_t tpb = b / RT;
  const int64_t tl = ((int64_t)a * RT - blk_of((int64_t)a * RT, b) * b) / RT;
  const int64_t cl = ((int64_t)tj * RT - blk_of((int64_t)tj * RT, b) * b) / RT;
  return (slot * tpb * tpb + tl * tpb + cl) * (int64_t)A_BYTES;
}

// The drain duty of generator warp w: its TMEM lane quadrant w % 4 (a warp
// may only read the lanes of its SM sub-partition) and its column quarter
// 0..3 among the generator warps of that quadrant, or -1 (no drain duty).
__device__ __forceinline__ int drain_quarter(int warp) {
  const int h = (warp >> 2) - ((warp & 3) >= 2 ? 1 : 0);
  return h >= 0 && h < 4 ? h : -1;
}

// Drain one TMEM accumulator (columns col0 .. col0 + N - 1) into the slot
// rows starting at row `srow` (N floats per row, D's column order
// [Re v0.. | Im v0..]): store when first, else add.  Warp w reads TMEM
// lanes 32 (w % 4) .. +31 and columns h QC .. +QC, h = drain_quarter(w).
// The adds are reductions performed at L2 (float4 atomic adds, each
// component rounded to nearest): the draining warp does not wait for the
// slot's old value.  A slot element is always drained by the same thread
// (the mapping above does not change), so its store and adds happen in
// program order and the sum is the same on every run.
template <int NV>
__device__ __forceinline__ void drain_acc(uint32_t tmem, uint32_t col0, float* __restrict__ slots, int64_t srow,
                                          bool first) {
  constexpr int N = Cfg<NV>::N, QC = Cfg<NV>::QC;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, h = drain_quarter(warp);
  constexpr int PIECE = QC < 16 ? QC : 16;  // TMEM columns loaded at a time
  float4* dst = reinterpret_cast<float4*>(slots + (srow + q * 32 + lane) * N + h * QC);
#pragma unroll
  for (int pc = 0; pc < QC / PIECE; ++pc) {
    float v[PIECE];
    tmem_load<PIECE>(tmem + ((uint32_t)(q * 32) << 16) + col0 + (uint32_t)(h * QC + pc * PIECE), v);
#pragma unroll
    for (int i = 0; i < PIECE / 4; ++i) {
      float4 o = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
      float4* d4 = dst + pc * (PIECE / 4) + i;
      if (first) *d4 = o;
      else atomicAdd(d4, o);
    }
  }
}

__device__ __forceinline__ void arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Generator warp: wait (lane 0 polls, the warp follows) with error code on time-out.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, uint32_t spin, int* err, int code,
                                          volatile int* abort_flag) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, spin);
  ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
  if (!ok && (threadIdx.x & 31) == 0) {
    atomicCAS(err, 0, code);
    *abort_flag = 1;
  }
  return ok;
}

template <int NV>
__global__ void __launch_bounds__(NTHREADS, 1)
    tch_apply(int32_t T, int32_t s, int32_t U, int32_t nunits, const int2* __restrict__ units,
              const int64_t* __restrict__ off2d, int* __restrict__ counter, float* __restrict__ slots,
              const unsigned char* __restrict__ gB, uint64_t seed, float sigma,
              const unsigned char* __restrict__ ccache, const int64_t* __restrict__ slot_of_pair, int64_t b,
              int64_t nblk, int* __restrict__ err, uint32_t spin) {
  using C = Cfg<NV>;
  constexpr int N = C::N, BT = C::BT, BSLOT = C::BSLOT, NBUF = C::NBUF;
  constexpr uint32_t ID_K = idesc_bf16_m128(N, 0), ID_T = idesc_bf16_m128(N, 1);
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* A = smem;
  unsigned char* Bring = smem + A_BYTES;
  // a_full[q]: region q of a tile written (or, for a cached tile, released
  // by the previous one); rel[q]: region q (in
  // the next tile's orientation) no longer read by this tile's MMAs
  // d1_full / d1_free: band accumulators complete / drained; d2_full[b] /
  // d2_free[b]: the H^dag accumulator b of a step complete / drained
  __shared__ uint64_t a_full[4], rel[4], a_copy, b_full[NBUF], b_free[NBUF], d1_full, d1_free, d2_full[2],
      d2_free[2];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  __shared__ int cur_unit;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int c = 0; c < 4; ++c) {
      mbar_init(&a_full[c], NGEN);
      mbar_init(&rel[c], 1);
    }
    mbar_init(&a_copy, 1);
    for (int i = 0; i < NBUF; ++i) {
      mbar_init(&b_full[i], 1);
      mbar_init(&b_free[i], 1);
    }
    mbar_init(&d1_full, 1);
    mbar_init(&d1_free, NGEN);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&d2_full[i], 1);
      mbar_init(&d2_free[i], NGEN);
    }
    abort_flag = 0;
    fence_async_smem();
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  // counters that run across units (barrier phases): every tile (a_full,
  // rel), cached tiles (a_copy), band-accumulator drains (d1_*), steps with
  // H^dag products (d2_*: accumulator hs & 1)
  uint32_t tiles = 0, ctiles = 0, d1c = 0, hs = 0;
  // MMA thread: band accumulators to overwrite on their next MMA, the next
  // H^dag accumulator starts a step, a band drain is pending
  uint32_t fresh = (1u << W) - 1;
  bool fresh2 = true, need_d1 = false;
  uint32_t loads = 0;                      // copy thread: operand copies issued
  uint32_t bslot = 0, bpar = 0;            // MMA thread: ring slot of the next job and its phase parity
  uint64_t* last_bar = nullptr;            // MMA thread: barrier and phase of the last commit
  uint32_t last_par = 0;
  bool tile_copy = false;                  // MMA thread: a copy of cached tile planes is in flight

  for (;;) {
    __syncthreads();
    if (tid == 0) cur_unit = abort_flag ? nunits : atomicAdd(counter, 1);
    __syncthreads();
    const int u = cur_unit;
    if (u >= nunits) break;
    const int ur = units[u].x, uc = units[u].y;
    const int64_t rowR = off2d[(int64_t)ur * U + uc];                        // slot row of region R
    const int64_t rowC = rowR + (int64_t)min(s, T - ur * s) * RT;            // region C (off the diagonal)

    if (warp == LOAD_WARP) {
      if (lane == 0) {
        // operand copies of the unit's jobs, in job order, each into the next
        // ring slot once the MMAs of the job that used it before are done
        JobWalk lw;
        lw.start(ur, uc, s, T, tiles);
        bool ok = true;
        for (; lw.live && !abort_flag; lw.next()) {
          const int slot = (int)(loads % NBUF);
          if (loads >= (uint32_t)NBUF && !mbar_wait(&b_free[slot], (loads / NBUF - 1) & 1u, spin)) {
            atomicCAS(err, 0, 130);
            ok = false;
            break;
          }
          const bool h = lw.is_h();
          const int64_t xt = h ? lw.w.tj : lw.w.a;  // operand rows: X[tj] (H) or X[a] (H^dag)
          const unsigned char* src = gB + ((int64_t)xt * 4 + lw.idx()) * (6 * (int64_t)BT) + (h ? 0 : 2 * BT);
          mbar_expect_tx(&b_full[slot], (uint32_t)BSLOT);
          bulk_g2s(Bring + slot * BSLOT, src, (uint32_t)BSLOT, &b_full[slot]);
          ++loads;
          // the tile count of the walk runs with the MMA thread's
        }
        tiles = lw.tile;
        if (!ok || lw.live) {
          abort_flag = 1;
          // the CTA stops: wait for this thread's copies still in flight
          for (uint32_t i = loads > (uint32_t)NBUF ? loads - NBUF : 0; i < loads; ++i)
            mbar_wait(&b_full[i % NBUF], (i / NBUF) & 1u, kDrainSpin);
        }
      }
      __syncwarp();
    } else if (warp == MMA_WARP) {
      if (lane == 0) {
        // The MMA thread shares its SM sub-partition with busy generator
        // warps, so its work per job is kept to a few instructions: the
        // descriptors are bases plus offsets in 16-byte units (shared-memory
        // addresses stay below 256 KB, so the 14-bit address field never
        // carries), and the tile decode happens once per tile.
        const uint64_t dK = smem_desc_nosw(smem_u32(A), 128, 2048);   // A, K-major
        const uint64_t dT = smem_desc_nosw(smem_u32(A), 2048, 128);   // A^T, MN-major
        const uint64_t dB = smem_desc_nosw(smem_u32(Bring), 128, 512);
        constexpr uint32_t PL16 = PLANE >> 4, BT16 = BT >> 4, BS16 = BSLOT >> 4;
        auto commit = [&](uint64_t* bar, uint32_t par) {
          mma_commit(bar);
          last_bar = bar;
          last_par = par;
        };
        Walk w;
        w.start(ur, uc, s, T);
        bool ok = true, more = true;
        for (; more && ok && !abort_flag; more = w.next()) {
          const bool herm = w.a < w.tj;
          const int o = (int)(tiles & 1u), nj = herm ? 8 : 4, j = w.a - w.br;
          const uint32_t ph = tiles & 1u;
          const int64_t cs = tile_slot(w.a, w.tj, ccache, slot_of_pair, b, nblk);
          const bool cached = cs >= 0;
          if (cached) {
            // the generator warps pass through every tile: their arrivals
            // say the previous tile has released all of A (and keep the
            // two roles within one tile of each other)
            bool fr = true;
            for (int q = 0; q < 4 && fr; ++q) fr = mbar_wait(&a_full[q], ph, spin);
            if (!fr) {
              atomicCAS(err, 0, 137);
              ok = false;
              break;
            }
            const unsigned char* src = ccache + tile_cache_off(w.a, w.tj, cs, b);
            mbar_expect_tx(&a_copy, (uint32_t)A_BYTES);
            for (int pl = 0; pl < 4; ++pl) bulk_g2s(A + pl * PLANE, src + pl * PLANE, (uint32_t)PLANE, &a_copy);
            tile_copy = true;
            if (!mbar_wait(&a_copy, ctiles & 1u, kDrainSpin)) {  // the copy this thread issued
              atomicCAS(err, 0, 138);
              ok = false;
              break;
            }
            tile_copy = false;
          }
          const uint32_t dD1 = tmem + (uint32_t)(j * N);
          const uint32_t dD2 = tmem + (uint32_t)((W + (int)(hs & 1u)) * N);
          for (int kj = 0; kj < nj; ++kj) {
            const bool h = !herm || (o == 0 ? kj < 4 : kj >= 4);
            const int ci = kj & 3;
            if (!mbar_wait(&b_full[bslot], bpar, spin)) {
              atomicCAS(err, 0, 131);
              ok = false;
              break;
            }
            if (!cached) {
              // the regions of the fill this job reads: the job's own region
              // while the fill is in progress, all four for the product after it
              bool fine = true;
              if ((o == 0) == h) fine = mbar_wait(&a_full[ci], ph, spin);
              else if (o == 1 && !herm && ci == 0)
                for (int q = 0; q < 4 && fine; ++q) fine = mbar_wait(&a_full[q], ph, spin);
              if (!fine) {
                atomicCAS(err, 0, 132);
                ok = false;
                break;
              }
            }
            if (h && need_d1) {  // the band accumulators are being drained
              if (!mbar_wait(&d1_free, d1c & 1u, spin)) {
                atomicCAS(err, 0, 133);
                ok = false;
                break;
              }
              ++d1c;
              need_d1 = false;
            }
            if (!h && fresh2 && hs >= 2 && !mbar_wait(&d2_free[hs & 1u], ((hs >> 1) - 1) & 1u, spin)) {
              // the drain of the step before the last, which used this accumulator
              atomicCAS(err, 0, 134);
              ok = false;
              break;
            }
            tc_fence_after();
            const uint64_t bb = dB + (uint64_t)(bslot * BS16);
            if (h) {
              // H product: D1[j] += A[:, 32ci .. 32ci+31] B(X[tj]); slot = [B2h B2l B1h B1l]
              const uint64_t a = dK + (uint64_t)(ci * 32);
              const uint32_t acc0 = ((fresh >> j) & 1u) ? 0u : 1u;
#pragma unroll
              for (int ks = 0; ks < 2; ++ks) {
                const uint64_t ak = a + (uint64_t)(ks * 16), bk = bb + (uint64_t)(ks * 16);
                // re hi (B1 hi + B1 lo) + re lo B1 hi, im hi (B2 hi + B2 lo) + im lo B2 hi
                mma_bf16_x6(dD1, ak, ak + PL16, ak + 2 * PL16, ak + 3 * PL16, bk + 2 * BT16, bk + 3 * BT16, bk,
                            bk + BT16, ID_K, ks == 0 ? acc0 : 1u);
              }
              fresh &= ~(1u << j);
            } else {
              // H^dag product: D2 += A^T[:, rows 32ci ..] B(X[a]); slot = [B1h B1l B3h B3l]
              const uint64_t a = dT + (uint64_t)(ci * 512);
              const uint32_t acc0 = fresh2 ? 0u : 1u;
#pragma unroll
              for (int ks = 0; ks < 2; ++ks) {
                const uint64_t ak = a + (uint64_t)(ks * 256), bk = bb + (uint64_t)(ks * 16);
                // re^T hi (B1 hi + B1 lo) + re^T lo B1 hi, im^T hi (B3 hi + B3 lo) + im^T lo B3 hi
                mma_bf16_x6(dD2, ak, ak + PL16, ak + 2 * PL16, ak + 3 * PL16, bk, bk + BT16, bk + 2 * BT16,
                            bk + 3 * BT16, ID_T, ks == 0 ? acc0 : 1u);
              }
              fresh2 = false;
            }
            commit(&b_free[bslot], bpar);
            if (++bslot == NBUF) {
              bslot = 0;
              bpar ^= 1u;
            }
            // releases for the next tile (the other orientation): an even tile
            // frees row chunk ci after its H^dag product of ci (all four after
            // its last H product when it has none); an odd tile frees column
            // chunk ci after its H product of ci
            if (o == 0 && !h) commit(&rel[ci], ph);
            else if (o == 0 && !herm && ci == 3)
              for (int q = 0; q < 4; ++q) commit(&rel[q], ph);
            else if (o == 1 && h) commit(&rel[ci], ph);
          }
          if (!ok) break;
          if (w.step_end() && w.step_has_herm()) {
            commit(&d2_full[hs & 1u], (hs >> 1) & 1u);
            ++hs;
            fresh2 = true;
          }
          if (w.step_end() && w.d1_drain()) {
            commit(&d1_full, d1c & 1u);
            need_d1 = true;
            fresh = (1u << W) - 1;
          }
          ++tiles;
          if (cached) ++ctiles;
        }
        if (!ok || more) {
          abort_flag = 1;
          // the CTA stops: wait for the copies and MMAs this thread issued
          if (tile_copy) mbar_wait(&a_copy, ctiles & 1u, kDrainSpin);
          if (last_bar) mbar_wait(last_bar, last_par, kDrainSpin);
        }
      }
      __syncwarp();
    } else {
      // generator warps: a generated tile is filled region by region in its
      // orientation; before writing region q the warps wait until the
      // previous tile has released it.  Thread gt fills pairs gt, gt + GT,
      // gt + 2 GT, ... (< CPAIRS) of each region: npr of them.
      const int gt = (warp - (warp > MMA_WARP ? 1 : 0) - (warp > LOAD_WARP ? 1 : 0)) * 32 + lane;
      const int npr = (CPAIRS - gt + GT - 1) / GT;
      const bool drainer = drain_quarter(warp) >= 0;
      Walk w;
      w.start(ur, uc, s, T);
      uint64_t touchR = 0, touchC = 0;  // row tiles of the unit's slot regions written so far
      bool pend = false;                // an H^dag partial waits to be drained
      uint32_t pend_b = 0, pend_par = 0;
      int pend_rt = 0;
      // drain H^dag accumulator bb (phase parity par of d2_full[bb]) into row
      // tile rt of the unit's column region (its row region on the diagonal)
      auto drain_d2 = [&](uint32_t bb, uint32_t par, int rt) -> bool {
        if (!warp_wait(&d2_full[bb], par, spin, err, 138, &abort_flag)) return false;
        tc_fence_after();
        uint64_t& mask = w.diag ? touchR : touchC;
        if (drainer)
          drain_acc<NV>(tmem, (uint32_t)((W + (int)bb) * N), slots, (w.diag ? rowR : rowC) + (int64_t)rt * RT,
                        !((mask >> rt) & 1ull));
        mask |= 1ull << rt;
        tc_fence_before();
        __syncwarp();
        if (lane == 0) arrive(&d2_free[bb]);
        return true;
      };
      for (bool more = true; more; more = w.next()) {
        if (abort_flag) break;
        if (tile_slot(w.a, w.tj, ccache, slot_of_pair, b, nblk) >= 0) {
          // a cached tile (copied into A by the MMA thread): pass through its
          // regions like a generated tile, without writing, so that the MMA
          // thread copies only once the previous tile has released all of A
          bool ok = true;
          for (int q = 0; q < 4; ++q) {
            if (tiles > 0 && !(ok = warp_wait(&rel[q], (tiles - 1) & 1u, spin, err, 139, &abort_flag))) break;
            __syncwarp();
            if (lane == 0) arrive(&a_full[q]);
          }
          if (!ok) break;
        } else {
          const int64_t R0 = (int64_t)w.a * RT, C0 = (int64_t)w.tj * RT;
          const bool dt = w.a == w.tj;
          const int o = (int)(tiles & 1u);
          bool ok = true;
#pragma unroll 1
          for (int q = 0; q < 4; ++q) {
            if (tiles > 0 && !(ok = warp_wait(&rel[q], (tiles - 1) & 1u, spin, err, 135, &abort_flag))) break;
#pragma unroll
            for (int i = 0; i < MAXPR; ++i)
              if (i < npr) {
                int r, c;
                region_rc(o, q, gt + GT * i, r, c);
                uint32_t wd[4];
                gen_words(seed, sigma, R0, C0, dt, r, c, wd);
                put_words(A, r, c, wd);
              }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) arrive(&a_full[q]);
          }
          if (!ok) break;
        }
        ++tiles;
        // the H^dag partial of the step before this tile's fill, drained now
        // so that the fill never waits for it
        if (pend && !drain_d2(pend_b, pend_par, pend_rt)) break;
        pend = false;
        if (w.step_end() && w.step_has_herm()) {
          pend = true;
          pend_b = hs & 1u;
          pend_par = (hs >> 1) & 1u;
          pend_rt = w.tj - (w.diag ? w.r0 : w.c0);
          ++hs;
        }
        if (w.step_end() && w.d1_drain()) {
          if (!warp_wait(&d1_full, d1c & 1u, spin, err, 136, &abort_flag)) break;
          tc_fence_after();
          for (int j = 0; j < w.bw; ++j) {
            if (w.br + j > w.tj) continue;  // that band row has no tile yet
            const int rt = w.br + j - w.r0;
            if (drainer)
              drain_acc<NV>(tmem, (uint32_t)(j * N), slots, rowR + (int64_t)rt * RT, !((touchR >> rt) & 1ull));
            touchR |= 1ull << rt;
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) arrive(&d1_free);
          ++d1c;
        }
      }
      if (pend && !abort_flag) drain_d2(pend_b, pend_par, pend_rt);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS)
                 : "memory");
}

// Consumer-format block cache of the Hermitian tensor-core plans: every
// 128 x 128 tile of each cached canonical block pair (upper tiles of the
// diagonal blocks) as the four bf16 planes of the A layout, the same words
// the generator warps write, so cached and generated tiles are identical.
__global__ void tch_cache_fill(const int2* __restrict__ pairs, int64_t b, uint64_t seed, float sigma,
                               unsigned char* __restrict__ cache) {
  const int64_t slot = blockIdx.x;
  const int64_t tpb = b / RT, t = blockIdx.y;
  const int64_t tl = t / tpb, cl = t % tpb;
  const int2 nm = pairs[slot];
  if (nm.x == nm.y && tl > cl) return;
  const int64_t R0 = (int64_t)nm.x * b + tl * RT, C0 = (int64_t)nm.y * b + cl * RT;
  unsigned char* dst = cache + (slot * tpb * tpb + t) * (int64_t)A_BYTES;
  for (int p = threadIdx.x; p < PAIRS; p += blockDim.x) {
    int r, c;
    region_rc(0, p / CPAIRS, p % CPAIRS, r, c);
    uint32_t w[4];
    gen_words(seed, sigma, R0, C0, R0 == C0, r, c, w);
    put_words(dst, r, c, w);
  }
}

// Operand tiles of X for every 32-row chunk q, six tiles of N x 32 bf16
// (K-major, boff layout) back to back: B2 hi, B2 lo, B1 hi, B1 lo, B3 hi,
// B3 lo, with B1 = [Re X | Im X], B2 = [-Im X | Re X], B3 = -B2.  The H
// product copies the first four, the H^dag product the last four.  Rows of
// X past D are zero.
template <int NV>
__global__ void tch_split_x(const float2* __restrict__ xc, int64_t D, int64_t nchunk, unsigned char* __restrict__ gB) {
  constexpr int N = 2 * NV, BT = N * KC * 2;
  const int64_t total = nchunk * KC * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / (KC * N);
    const int rem = (int)(e % (KC * N));
    const int n = rem / KC, k = rem % KC;
    const int64_t c = q * KC + k;
    float2 xv = make_float2(0.f, 0.f);
    const int vec = n < NV ? n : n - NV;
    if (c < D) xv = xc[c * NV + vec];
    const float v1 = n < NV ? xv.x : xv.y;
    const float v2 = n < NV ? -xv.y : xv.x;
    unsigned char* base = gB + q * 6 * BT;
    const uint32_t off = boff(n, k);
    const __nv_bfloat16 h1 = __float2bfloat16_rn(v1), h2 = __float2bfloat16_rn(v2);
    const __nv_bfloat16 l1 = __float2bfloat16_rn(v1 - __bfloat162float(h1));
    const __nv_bfloat16 l2 = __float2bfloat16_rn(v2 - __bfloat162float(h2));
    *reinterpret_cast<__nv_bfloat16*>(base + 0 * BT + off) = h2;
    *reinterpret_cast<__nv_bfloat16*>(base + 1 * BT + off) = l2;
    *reinterpret_cast<__nv_bfloat16*>(base + 2 * BT + off) = h1;
    *reinterpret_cast<__nv_bfloat16*>(base + 3 * BT + off) = l1;
    *reinterpret_cast<__nv_bfloat16*>(base + 4 * BT + off) = __hneg(h2);
    *reinterpret_cast<__nv_bfloat16*>(base + 5 * BT + off) = __hneg(l2);
  }
}

// y-partials of the unit walk: for row `row` of tile t, the row-region
// partials of the units (t/s, uc >= t/s) and the column-region partials of
// the units (ur < t/s, t/s), summed in FP64 in that fixed order, handed on
// as two FP32 slots (hi = float(sum), lo = float(sum - hi)) of the slot
// layout the reduction and the Chebyshev update read ([2][dpad][NV]).
template <int NV>
__global__ void tch_gather(const float* __restrict__ slots, const int64_t* __restrict__ off2d, int32_t T, int32_t s,
                           int32_t U, int64_t D, int64_t dpad, float2* __restrict__ part) {
  constexpr int N = 2 * NV;
  const int64_t n = D * NV;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / NV;
    const int v = (int)(e % NV);
    const int t = (int)(row >> 7);
    const int ut = t / s;
    const int64_t rin = (int64_t)(t - ut * s) * RT + (row & 127);
    double sr = 0.0, si = 0.0;
    for (int uc = ut; uc < U; ++uc) {
      const float* p = slots + (off2d[(int64_t)ut * U + uc] + rin) * N;
      sr += (double)p[v];
      si += (double)p[NV + v];
    }
    for (int ur = 0; ur < ut; ++ur) {
      const int64_t base = off2d[(int64_t)ur * U + ut] + (int64_t)min(s, T - ur * s) * RT;
      const float* p = slots + (base + rin) * N;
      sr += (double)p[v];
      si += (double)p[NV + v];
    }
    const float hr = (float)sr, hi = (float)si;
    part[e] = make_float2(hr, hi);
    part[dpad * NV + e] = make_float2((float)(sr - (double)hr), (float)(si - (double)hi));
  }
}

static inline unsigned grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 1 << 20));
}

template <int NV>
cudaError_t launch_t(const Plan& p, const void* xc, void* part, void* gB) {
  using C = Cfg<NV>;
  const int64_t nchunk = p.ntile * 4;
  tch_split_x<NV><<<grid_for(nchunk * KC * C::N), 256, 0, p.stream>>>((const float2*)xc, p.D, nchunk,
                                                                     (unsigned char*)gB);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(p.d_tch_counter, 0, sizeof(int), p.stream)) != cudaSuccess) return e;
  auto k = tch_apply<NV>;
  if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM)) != cudaSuccess)
    return e;
  const int grid = std::min<int>(p.num_sms, (int)p.tch_nunits);
  k<<<grid, NTHREADS, C::SMEM, p.stream>>>((int32_t)p.ntile, p.tch_s, p.tch_U, (int32_t)p.tch_nunits, p.d_tch_units,
                                           p.d_tch_off, p.d_tch_counter, (float*)p.d_tch_slots,
                                           (const unsigned char*)gB, p.seed, p.sigma32,
                                           p.pairs_cached > 0 ? (const unsigned char*)p.d_cache : nullptr,
                                           p.d_pair_slot, p.b, p.nblk, p.d_err, p.spin);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  tch_gather<NV><<<grid_for(p.D * NV), 256, 0, p.stream>>>((const float*)p.d_tch_slots, p.d_tch_off,
                                                           (int32_t)p.ntile, p.tch_s, p.tch_U, p.D,
                                                           p.ntile * (int64_t)RT, (float2*)part);
  return cudaGetLastError();
}

}  // namespace tch

// Unit size s (tiles) of the Hermitian tensor-core walk for T tile rows: the
// largest power of two <= 32 that still gives at least 4 units per SM, so
// the dynamic unit queue balances the SMs; the units in the order the CTAs
// take them (unit columns from the right, rows from the top: the CTAs
// running at one time share the operand rows of one unit column in L2); and
// the slot row offsets of each unit (row region, then column region off the
// diagonal).  Returns the total slot rows.
int64_t tch_layout(int64_t T, int num_sms, int32_t* s_out, int32_t* U_out, std::vector<int2>& units,
                   std::vector<int64_t>& off2d) {
  int32_t s = 32;
  auto nunits = [&](int32_t sv) {
    const int64_t U = (T + sv - 1) / sv;
    return U * (U + 1) / 2;
  };
  while (s > 1 && nunits(s) < 4 * (int64_t)num_sms) s /= 2;
  const int32_t U = (int32_t)((T + s - 1) / s);
  units.clear();
  for (int32_t uc = U - 1; uc >= 0; --uc)
    for (int32_t ur = 0; ur <= uc; ++ur) units.push_back(make_int2(ur, uc));
  off2d.assign((size_t)U * U, -1);
  int64_t rows = 0;
  for (int32_t ur = 0; ur < U; ++ur)
    for (int32_t uc = ur; uc < U; ++uc) {
      off2d[(size_t)ur * U + uc] = rows;
      const int64_t rr = std::min<int64_t>(s, T - (int64_t)ur * s) * tch::RT;
      const int64_t rc = std::min<int64_t>(s, T - (int64_t)uc * s) * tch::RT;
      rows += ur == uc ? rr : rr + rc;
    }
  *s_out = s;
  *U_out = U;
  return rows;
}

size_t tch_operand_bytes(int64_t D, int64_t nv_bucket) {
  const int64_t nchunk = (D + tch::RT - 1) / tch::RT * 4;
  return (size_t)nchunk * 6 * (size_t)(2 * nv_bucket) * tch::KC * 2;
}

cudaError_t launch_tch_cache_fill(const Plan& p, const int2* d_pairs, int64_t npairs) {
  if (npairs == 0) return cudaSuccess;
  const int64_t tpb = p.b / tch::RT;
  if (npairs > 0x7fffffff || tpb * tpb > 65535) return cudaErrorInvalidValue;
  tch::tch_cache_fill<<<dim3((unsigned)npairs, (unsigned)(tpb * tpb)), 256, 0, p.stream>>>(d_pairs, p.b, p.seed,
                                                                                          p.sigma32,
                                                                                          (unsigned char*)p.d_cache);
  return cudaGetLastError();
}

cudaError_t launch_tch_apply(const Plan& p, const void* xc, void* part, void* gB, int64_t nv_bucket) {
  switch (nv_bucket) {
    case 8: return tch::launch_t<8>(p, xc, part, gB);
    case 16: return tch::launch_t<16>(p, xc, part, gB);
    case 32: return tch::launch_t<32>(p, xc, part, gB);
    case 64: return tch::launch_t<64>(p, xc, part, gB);
  }
  return cudaErrorNotSupported;
}

}  // namespace mf
