// k_tc.cu -- multi-vector generate-and-apply on the 5th-generation tensor
// cores (tcgen05, TMEM accumulators), BF16 hi+lo split form.
//
// Row-owner form of Y = H X (Sec. IV.A, Eq. generic_multivector; output
// block rows as in Sec. III.B): a CTA owns 128 output rows and sweeps its
// column range in chunks of 32 columns with 16 generator warps and one
// copy/MMA warp.  For every chunk
//   * the generator warps generate H[128 x 32] (Philox canonical entries,
//     conjugates below the diagonal, DVR window table) or read it from the
//     FP32 block cache, split each real part into bf16 hi + lo and store the
//     four planes (re hi, re lo, im hi, im lo) straight into shared memory in
//     the canonical no-swizzle K-major layout the tensor core reads;
//   * one thread of the copy/MMA warp streams the chunk's operand tiles of X
//     (pre-split per apply into the same layout: B1 = [Re X | Im X],
//     B2 = [-Im X | Re X], hi and lo) with bulk asynchronous copies
//     completing on an mbarrier;
//   * the same thread issues twelve tcgen05.mma (two K steps of 16, six split
//     products each: A_re_hi B1_hi, A_re_hi B1_lo, A_re_lo B1_hi and the same
//     for A_im with B2) accumulating D[128 x 2 NV] = [Re Y | Im Y] in TMEM;
//     tcgen05.commit arrives on the stage's mbarrier when they finish.
// Two shared-memory stages let the generation of chunk k+1 run on the SIMT
// pipes while the tensor core works on chunk k.  Every 32 chunks the TMEM
// accumulator is drained (tcgen05.ld) into an FP32 accumulator in shared
// memory with round-to-nearest adds; the epilogue writes that accumulator to
// the split-K partial slot.  Every wait is bounded; on time-out the kernel
// records the stage in the plan's error word, drains its own outstanding work
// (again bounded), frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "rows_body.cuh"
#include "tc_ptx.cuh"

namespace mf {
namespace tc {

using namespace ptx;

constexpr int RT = 128;          // rows per CTA (MMA M)
constexpr int KC = 32;           // columns per chunk
constexpr int NGEN = 16;                     // generator warps (fill the A planes)
constexpr int MMA_WARP = NGEN;               // the copy/MMA-issuing warp
constexpr int NTHREADS = (NGEN + 1) * 32;
constexpr int A_PLANE = RT * KC * 2;  // bytes of one bf16 plane of the chunk (8 KB)
// Waits for work this CTA issued itself (its bulk copies, its committed
// MMAs) always complete; they keep this bound whatever the plan's spin limit,
// so that a CTA never leaves with a copy or an MMA in flight.
constexpr uint32_t kDrainSpin = kDefaultSpin;
// The tensor core's FP32 accumulation is not round-to-nearest over long
// chains, so TMEM accumulates SEG chunks (SEG * 12 MMAs) at a time and is
// then drained into an FP32 accumulator in shared memory with ordinary
// round-to-nearest adds.
constexpr int SEG = 32;

// byte offset of element (row, k) in a canonical no-swizzle K-major tile
// whose core matrices (8 rows x 16 bytes) are laid out K-core-fastest:
// LBO (next K core) = 128 B, SBO (next 8-row group) = 4 * 128 B.
__device__ __forceinline__ uint32_t kmajor_off(int row, int k) {
  return (uint32_t)((row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  const uint64_t lbo = 128 >> 4, sbo = 512 >> 4;
  return (uint64_t)((saddr >> 4) & 0x3FFF) | (lbo << 16) | (sbo << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: D f32, A and B bf16, both K-major,
// N = n, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// entries (r, k) and (r, k + 1), k even: one 32-bit store per plane
__device__ __forceinline__ void put_hpair(unsigned char* A, int r, int k, float2 h0, float2 h1) {
  uint32_t w[4];
  split_pair(h0, h1, w);
  const uint32_t off = kmajor_off(r, k);
#pragma unroll
  for (int pl = 0; pl < 4; ++pl) *reinterpret_cast<uint32_t*>(A + pl * A_PLANE + off) = w[pl];
}

// entries (r, k) and (r + 1, k), r even: two 16-bit stores per plane
__device__ __forceinline__ void put_vpair(unsigned char* A, int r, int k, float2 h0, float2 h1) {
  uint32_t w[4];
  split_pair(h0, h1, w);
  const uint32_t off = kmajor_off(r, k);
#pragma unroll
  for (int pl = 0; pl < 4; ++pl) {
    *reinterpret_cast<uint16_t*>(A + pl * A_PLANE + off) = (uint16_t)(w[pl] & 0xFFFFu);
    *reinterpret_cast<uint16_t*>(A + pl * A_PLANE + off + 16) = (uint16_t)(w[pl] >> 16);
  }
}

// Fill the four A planes of chunk [R0, R0+128) x [c0, c0+32) (called by the
// NGEN generator warps only; no block-wide synchronisation).  Warp w covers
// the 8-row group w (16 groups) and, per K core kc (4 cores of 8 columns),
// one 8 x 8 core matrix: horizontal pairs with lane -> (row lane/4, columns
// 2 (lane%4), +1), vertical pairs with lane -> (rows 2 (lane%4), +1, column
// lane/4); both keep a warp's stores inside one 128-byte core matrix.
template <int GEN>
__device__ __forceinline__ void fill_a(unsigned char* A, int64_t R0, int64_t c0, uint64_t seed,
                                       float sigma, const dvr_consts& dk, const float2* __restrict__ cache,
                                       const int64_t* __restrict__ slot_of_pair, int64_t b, int64_t nblk,
                                       const float2* __restrict__ hcache) {
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int hr = 8 * g + (lane >> 2), hk = 2 * (lane & 3);   // horizontal pair origin within a K core
  const int vr = 8 * g + 2 * (lane & 3), vk = lane >> 2;     // vertical pair origin within a K core
  int64_t slot = -1;
  bool transposed = false;
  const int64_t n = blk_of(R0, b), m = blk_of(c0, b);
  if (cache || hcache) {
    if (n <= m) slot = slot_of_pair[n * nblk + m];
    else {
      slot = slot_of_pair[m * nblk + n];
      transposed = true;
    }
  }
  if (slot >= 0 || slot <= -2) {
    // HBM cache slot, or (slot <= -2) block -2 - slot of the host array
    const float2* blk = slot >= 0 ? cache + slot * b * b : hcache + (-2 - slot) * b * b;
    float4 q[4];
    if (!transposed) {
      // H[r][k], H[r][k+1] adjacent in the cached row: one 16-byte load
#pragma unroll
      for (int kc = 0; kc < 4; ++kc)
        q[kc] = *reinterpret_cast<const float4*>(blk + (R0 + hr - n * b) * b + (c0 + 8 * kc + hk - m * b));
#pragma unroll
      for (int kc = 0; kc < 4; ++kc)
        put_hpair(A, hr, 8 * kc + hk, make_float2(q[kc].x, q[kc].y), make_float2(q[kc].z, q[kc].w));
    } else {
      // H[r][k] = conj(C[k][r]): rows r, r+1 adjacent in the cached row k
#pragma unroll
      for (int kc = 0; kc < 4; ++kc)
        q[kc] = *reinterpret_cast<const float4*>(blk + (c0 + 8 * kc + vk - m * b) * b + (R0 + vr - n * b));
#pragma unroll
      for (int kc = 0; kc < 4; ++kc)
        put_vpair(A, vr, 8 * kc + vk, make_float2(q[kc].x, -q[kc].y), make_float2(q[kc].z, -q[kc].w));
    }
    return;
  }
  if (GEN == MF_GEN_SINC_DVR_HO) {
    const long long d0 = (long long)(R0 - c0) + hr;
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      const int k = 8 * kc + hk;
      put_hpair(A, hr, k, make_float2(dvr_T_f32(dk, d0 - k), 0.f), make_float2(dvr_T_f32(dk, d0 - k - 1), 0.f));
    }
    return;
  }
  if (c0 >= R0 + RT) {
    // above the diagonal: canonical pairs along rows
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      const int k = 8 * kc + hk;
      float2 h0, h1;
      gue_pair<float>(seed, sigma, (uint32_t)(R0 + hr), (uint32_t)((c0 + k) >> 1), h0, h1);
      put_hpair(A, hr, k, h0, h1);
    }
  } else if (c0 + KC <= R0) {
    // below: the canonical row c0 + k holds the pair of columns R0 + r, +1
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      const int k = 8 * kc + vk;
      float2 h0, h1;
      gue_pair<float>(seed, sigma, (uint32_t)(c0 + k), (uint32_t)((R0 + vr) >> 1), h0, h1);
      h0.y = -h0.y;
      h1.y = -h1.y;
      put_vpair(A, vr, k, h0, h1);
    }
  } else {
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      const int k = 8 * kc + hk;
      put_hpair(A, hr, k, gue_entry<float>(seed, sigma, R0 + hr, c0 + k),
                gue_entry<float>(seed, sigma, R0 + hr, c0 + k + 1));
    }
  }
}

// Y[R0:R0+128, :] over columns [cbeg, cend) into part[slot][row][NV].
// Warps 0..NGEN-1 generate the A planes of each chunk and arrive on the
// stage's a_full barrier; warp MMA_WARP streams the X tiles (b_full) and,
// once both are complete, issues the chunk's MMAs and commits them to the
// stage's mma barrier, which frees the stage for the chunk two ahead.  The
// only block-wide barriers are at the SEG-chunk drains.
template <int GEN, int NV>
__global__ void __launch_bounds__(NTHREADS, 1)
    tc_rows(int64_t D, int64_t dpad, int64_t split_cols, uint64_t seed, float sigma, dvr_consts dk,
            const unsigned char* __restrict__ gB, float2* __restrict__ part, const float2* __restrict__ cache,
            const int64_t* __restrict__ slot_of_pair, int64_t b, int64_t nblk, int* __restrict__ err,
            const float2* __restrict__ hcache, uint32_t spin) {
  constexpr int N = 2 * NV;             // MMA N: [Re | Im] of NV vectors
  constexpr int B_TILE = N * KC * 2;    // bytes of one bf16 B tile
  constexpr int B_CHUNK = 4 * B_TILE;   // B1 hi, B1 lo, B2 hi, B2 lo
  constexpr int STAGE = 4 * A_PLANE + B_CHUNK;
  constexpr int QC = N / 4;             // TMEM columns per thread in the drains
  constexpr uint32_t TMEM_COLS = N < 32 ? 32 : N;
  constexpr uint32_t IDESC = idesc_bf16(N);
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t a_full[2], b_full[2], mma_bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // drain mapping (generator warps): warp w reads TMEM lanes 32 (w % 4) ..
  // +31 (rows) and columns (w / 4) * QC .. +QC of D = [Re Y | Im Y]
  const int lane_grp = warp & 3, quarter = warp >> 2;
  const int drow = lane_grp * 32 + lane;
  float* accs = reinterpret_cast<float*>(smem + 2 * STAGE);  // [N][RT], column-major
  for (int e = tid; e < N * RT; e += NTHREADS) accs[e] = 0.f;
  const int64_t R0 = (int64_t)blockIdx.x * RT;
  const int64_t cbeg = (int64_t)blockIdx.y * split_cols;
  const int64_t cend = cbeg + split_cols < D ? cbeg + split_cols : D;
  const int nchunk = (int)((cend - cbeg + KC - 1) / KC);

  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&a_full[s], NGEN);
      mbar_init(&b_full[s], 1);
      mbar_init(&mma_bar[s], 1);
    }
    abort_flag = 0;
    fence_async_smem();
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  bool done_all = false;
  for (int k0 = 0; k0 < nchunk; k0 += SEG) {
    const int k1 = k0 + SEG < nchunk ? k0 + SEG : nchunk;
    if (warp == MMA_WARP) {
      if (lane == 0) {
        int last = -1;
        for (int kc = k0; kc < k1 && !abort_flag; ++kc) {
          const int s = kc & 1;
          unsigned char* A = smem + s * STAGE;
          unsigned char* B = A + 4 * A_PLANE;
          // the stage's previous MMAs (chunk kc - 2) must be done before its X tiles are replaced
          if (kc >= 2 && !mbar_wait(&mma_bar[s], (uint32_t)(((kc - 2) >> 1) & 1), spin)) {
            atomicCAS(err, 0, 100 + s);
            abort_flag = 1;
            break;
          }
          mbar_expect_tx(&b_full[s], (uint32_t)B_CHUNK);
          bulk_g2s(B, gB + ((cbeg + (int64_t)kc * KC) / KC) * (int64_t)B_CHUNK, (uint32_t)B_CHUNK, &b_full[s]);
          const bool a_ok = mbar_wait(&a_full[s], (uint32_t)((kc >> 1) & 1), spin);
          // the copy just issued: wait for it in any case
          const bool b_ok = mbar_wait(&b_full[s], (uint32_t)((kc >> 1) & 1), kDrainSpin);
          if (!a_ok || !b_ok) {
            atomicCAS(err, 0, a_ok ? 111 : 110);
            abort_flag = 1;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
#pragma unroll
          for (int ks = 0; ks < KC / 16; ++ks) {
            const uint32_t ko = (uint32_t)ks * 256;  // two 8-element K cores of 128 B
            const uint64_t are_h = smem_desc(a0 + 0 * A_PLANE + ko), are_l = smem_desc(a0 + 1 * A_PLANE + ko);
            const uint64_t aim_h = smem_desc(a0 + 2 * A_PLANE + ko), aim_l = smem_desc(a0 + 3 * A_PLANE + ko);
            const uint64_t b1_h = smem_desc(b0 + 0 * B_TILE + ko), b1_l = smem_desc(b0 + 1 * B_TILE + ko);
            const uint64_t b2_h = smem_desc(b0 + 2 * B_TILE + ko), b2_l = smem_desc(b0 + 3 * B_TILE + ko);
            const uint32_t acc0 = (kc != k0 || ks > 0) ? 1u : 0u;
            mma_bf16(tmem, are_h, b1_h, IDESC, acc0);
            mma_bf16(tmem, are_h, b1_l, IDESC, 1u);
            mma_bf16(tmem, are_l, b1_h, IDESC, 1u);
            mma_bf16(tmem, aim_h, b2_h, IDESC, 1u);
            mma_bf16(tmem, aim_h, b2_l, IDESC, 1u);
            mma_bf16(tmem, aim_l, b2_h, IDESC, 1u);
          }
          mma_commit(&mma_bar[s]);
          last = kc;
        }
        // the segment's MMAs complete in issue order: wait for the last one
        if (last >= 0 && !mbar_wait(&mma_bar[last & 1], (uint32_t)((last >> 1) & 1), kDrainSpin)) {
          atomicCAS(err, 0, 120);
          abort_flag = 1;
        }
        if (last != k1 - 1) abort_flag = 1;
      }
      __syncwarp();
    } else {
      for (int kc = k0; kc < k1; ++kc) {
        const int s = kc & 1;
        if (kc >= 2) {
          bool ok = true;
          if (lane == 0) ok = mbar_wait(&mma_bar[s], (uint32_t)(((kc - 2) >> 1) & 1), spin);
          ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
          if (!ok) {
            if (lane == 0) {
              atomicCAS(err, 0, 102 + s);
              abort_flag = 1;
            }
            break;
          }
        }
        if (abort_flag) break;
        fill_a<GEN>(smem + s * STAGE, R0, cbeg + (int64_t)kc * KC, seed, sigma, dk, cache, slot_of_pair, b, nblk,
                    hcache);
        fence_async_smem();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&a_full[s])) : "memory");
      }
    }
    __syncthreads();
    if (abort_flag) break;
    tc_fence_after();
    if (warp < NGEN) {
      float v[QC];
      tmem_load<QC>(tmem + ((uint32_t)(lane_grp * 32) << 16) + (uint32_t)(quarter * QC), v);
#pragma unroll
      for (int i = 0; i < QC; ++i) accs[(quarter * QC + i) * RT + drow] += v[i];
    }
    tc_fence_before();
    __syncthreads();
    done_all = k1 == nchunk;
  }
  if (!abort_flag && done_all && warp < NGEN) {
    float* out = reinterpret_cast<float*>(part + ((int64_t)blockIdx.y * dpad + R0 + drow) * NV);
#pragma unroll
    for (int i = 0; i < QC; ++i) {
      const int col = quarter * QC + i;
      const int vec = col < NV ? col : col - NV;
      out[2 * vec + (col < NV ? 0 : 1)] = accs[col * RT + drow];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// Operand tiles of X for every 32-row chunk: B1 = [Re X | Im X],
// B2 = [-Im X | Re X] (N = 2 NV columns, row = vector part), split into
// bf16 hi and lo, K-major canonical layout; rows of X beyond D are zero.
template <int NV>
__global__ void tc_split_x(const float2* __restrict__ xc, int64_t D, int64_t nchunk, unsigned char* __restrict__ gB) {
  constexpr int N = 2 * NV;
  constexpr int B_TILE = N * KC * 2;
  const int64_t total = nchunk * KC * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / (KC * N);
    const int rem = (int)(e % (KC * N));
    const int n = rem / KC, k = rem % KC;
    const int64_t c = q * KC + k;
    float2 xv = make_float2(0.f, 0.f);
    const int vec = n < NV ? n : n - NV;
    if (c < D) xv = xc[c * NV + vec];
    const float v1 = n < NV ? xv.x : xv.y;   // B1: [Re | Im]
    const float v2 = n < NV ? -xv.y : xv.x;  // B2: [-Im | Re]
    unsigned char* base = gB + q * 4 * B_TILE;
    const uint32_t off = kmajor_off(n, k);
    const __nv_bfloat16 h1 = __float2bfloat16_rn(v1), h2 = __float2bfloat16_rn(v2);
    *reinterpret_cast<__nv_bfloat16*>(base + 0 * B_TILE + off) = h1;
    *reinterpret_cast<__nv_bfloat16*>(base + 1 * B_TILE + off) = __float2bfloat16_rn(v1 - __bfloat162float(h1));
    *reinterpret_cast<__nv_bfloat16*>(base + 2 * B_TILE + off) = h2;
    *reinterpret_cast<__nv_bfloat16*>(base + 3 * B_TILE + off) = __float2bfloat16_rn(v2 - __bfloat162float(h2));
  }
}

template <int GEN, int NV>
cudaError_t launch_tc_t(const Plan& p, const void* xc, void* part, void* gB, int* err) {
  constexpr int N = 2 * NV;
  constexpr size_t STAGE = 4 * (size_t)A_PLANE + 4 * (size_t)N * KC * 2;
  const size_t smem = 2 * STAGE + (size_t)N * RT * sizeof(float);
  const int64_t nchunk = (p.D + KC - 1) / KC;
  tc_split_x<NV><<<(unsigned)std::min<int64_t>((nchunk * KC * N + 255) / 256, 65535), 256, 0, p.stream>>>(
      (const float2*)xc, p.D, nchunk, (unsigned char*)gB);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  auto k = tc_rows<GEN, NV>;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)p.ntile, (unsigned)p.rows_nsplit);
  k<<<grid, NTHREADS, smem, p.stream>>>(p.D, p.ntile * (int64_t)kTile, p.rows_split_cols, p.seed, p.sigma32, p.dvr,
                                        (const unsigned char*)gB, (float2*)part,
                                        p.pairs_cached > 0 ? (const float2*)p.d_cache : nullptr, p.d_pair_slot, p.b,
                                        p.nblk, err, (const float2*)p.d_hblocks, p.spin);
  return cudaGetLastError();
}

}  // namespace tc

size_t tc_operand_bytes(int64_t D, int64_t nv_bucket) {
  const int64_t nchunk = (D + tc::KC - 1) / tc::KC;
  return (size_t)nchunk * 4 * (size_t)(2 * nv_bucket) * tc::KC * 2;
}

int64_t tc_nvec_bucket(int64_t nvec) {
  int64_t b = 8;
  while (b < nvec) b *= 2;
  return b;
}

cudaError_t launch_tc_apply(const Plan& p, const void* xc, void* part, void* gB, int64_t nv_bucket) {
  if (p.rows_split_cols % tc::KC != 0) return cudaErrorInvalidValue;
  const bool dvr = p.gen == MF_GEN_SINC_DVR_HO;
  switch (nv_bucket) {
    case 8: return dvr ? tc::launch_tc_t<MF_GEN_SINC_DVR_HO, 8>(p, xc, part, gB, p.d_err)
                       : tc::launch_tc_t<MF_GEN_PHILOX_GUE, 8>(p, xc, part, gB, p.d_err);
    case 16: return dvr ? tc::launch_tc_t<MF_GEN_SINC_DVR_HO, 16>(p, xc, part, gB, p.d_err)
                        : tc::launch_tc_t<MF_GEN_PHILOX_GUE, 16>(p, xc, part, gB, p.d_err);
    case 32: return dvr ? tc::launch_tc_t<MF_GEN_SINC_DVR_HO, 32>(p, xc, part, gB, p.d_err)
                        : tc::launch_tc_t<MF_GEN_PHILOX_GUE, 32>(p, xc, part, gB, p.d_err);
    case 64: return dvr ? tc::launch_tc_t<MF_GEN_SINC_DVR_HO, 64>(p, xc, part, gB, p.d_err)
                        : tc::launch_tc_t<MF_GEN_PHILOX_GUE, 64>(p, xc, part, gB, p.d_err);
  }
  return cudaErrorNotSupported;
}

}  // namespace mf
