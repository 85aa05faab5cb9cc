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

#include <algorithm>

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

// ---------------------------------------------------------------------------
// FP32 form: persistent row-split kernel.
//
// Row tiles of kDvrRB = 4096 rows; warp w of a CTA owns rows 512 w + [0, 512)
// of the tile, lane L the 16 rows 16 L + [0, 16), so every row's sum stays in
// one thread's registers: no cross-warp reduction.  The work (row tile,
// 16-column block) pairs are numbered row tile by row tile and split into
// gridDim.x contiguous, equal ranges, so the load is balanced to one block.
// A CTA stages each 2048-column chunk it touches (x chunk and the RB + KC - 1
// window entries T(r - c), generated once per chunk) in shared memory and
// keeps its accumulators in registers across the chunks of a row tile.
//
// Per 16 x 16 block a lane reads its 31 window entries (32 with one spare)
// with eight 16-byte loads (the table is padded by 4 floats per 16 entries,
// so the lanes' 80-byte strided loads are free of bank conflicts) and the 16
// x entries with eight 16-byte broadcast loads, then issues 256 packed FMAs
// (__ffma2_rn: per lane and component the rounding of __fmaf_rn) updating
// the real and imaginary parts of a row together.
//
// Each CTA writes one partial per row tile it touched into slot
// (its index - index of the first CTA of that row tile); the CTA holding the
// row tile's last block also zero-fills the slots above its own, so every
// slot row the reduction reads is written.
// ---------------------------------------------------------------------------
constexpr int kDvrP = 16, kDvrU = 16, kDvrWarps = 8;
constexpr int kDvrRB = kDvrWarps * 32 * kDvrP;  // 4096 rows per row tile
constexpr int kDvrKC = 4096;                    // staged columns per chunk
constexpr int kDvrNTB = kDvrRB + kDvrKC - 1;    // window entries per chunk
constexpr int kDvrTbFloats = ((kDvrNTB + 1 + 15) / 16) * 20;
constexpr size_t kDvrSmem = (size_t)kDvrTbFloats * sizeof(float) + (size_t)kDvrKC * sizeof(float2);

__host__ __device__ __forceinline__ int64_t split_lo(int64_t b, int64_t n, int64_t g) { return b * n / g; }
// CTA whose range [split_lo(b), split_lo(b + 1)) holds item i
__host__ __device__ __forceinline__ int64_t split_owner(int64_t i, int64_t n, int64_t g) {
  int64_t b = i * g / n;
  while (split_lo(b + 1, n, g) <= i) ++b;
  while (split_lo(b, n, g) > i) --b;
  return b;
}
__device__ __forceinline__ int dvr_wpad(int j) { return j + (j >> 4) * 4; }

__global__ void __launch_bounds__(256, 2) dvr_rows_f32(int64_t D, int64_t dpad, int64_t nslot, int64_t nbc,
                                                       int64_t nblocks, dvr_consts dk, const float2* __restrict__ xc,
                                                       float2* __restrict__ part) {
  constexpr int P = kDvrP, U = kDvrU, KC = kDvrKC, BPC = KC / U;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* tb = reinterpret_cast<float*>(smem_raw);
  float2* xs = reinterpret_cast<float2*>(tb + kDvrTbFloats);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t G = gridDim.x, b = blockIdx.x;
  const int64_t lo = split_lo(b, nblocks, G), hi = split_lo(b + 1, nblocks, G);
  const int jb0 = 512 * w + P * lane + KC - U;  // window start of the chunk's first block
  float2 acc[P];
  for (int64_t cur = lo; cur < hi;) {
    const int64_t rt = cur / nbc, cb = cur - rt * nbc;
    const int64_t chunk = cb / BPC;
    const int64_t seg_end = min(hi, rt * nbc + min((chunk + 1) * BPC, nbc));
    if (cur == lo || cb == 0) {
#pragma unroll
      for (int a = 0; a < P; ++a) acc[a] = make_float2(0.f, 0.f);
    }
    const int64_t R0 = rt * kDvrRB, C0 = chunk * KC;
    __syncthreads();  // the previous segment is done with the staged chunk
    for (int c = tid; c < KC; c += 256) {
      const int64_t g = C0 + c;
      xs[c] = g < D ? xc[g] : make_float2(0.f, 0.f);
    }
    const long long kmin = (long long)(R0 - C0) - KC + 1;
    for (int j = tid; j <= kDvrNTB; j += 256) tb[dvr_wpad(j)] = j < kDvrNTB ? dvr_T_f32(dk, kmin + j) : 0.f;
    __syncthreads();
    const int cc_beg = (int)(cb - chunk * BPC) * U, cc_end = cc_beg + (int)(seg_end - cur) * U;
#pragma unroll 1
    for (int cc = cc_beg; cc < cc_end; cc += U) {
      const int jb = jb0 - cc;  // a multiple of 16
      float win[32];
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const float4* q = reinterpret_cast<const float4*>(tb + dvr_wpad(jb + 16 * g));
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float4 v = q[i];
          win[16 * g + 4 * i] = v.x;
          win[16 * g + 4 * i + 1] = v.y;
          win[16 * g + 4 * i + 2] = v.z;
          win[16 * g + 4 * i + 3] = v.w;
        }
      }
      float2 xv[U];
      const float4* xq = reinterpret_cast<const float4*>(xs + cc);
#pragma unroll
      for (int i = 0; i < U / 2; ++i) {
        const float4 v = xq[i];
        xv[2 * i] = make_float2(v.x, v.y);
        xv[2 * i + 1] = make_float2(v.z, v.w);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int a = 0; a < P; ++a) {
          const float t = win[a - u + U - 1];
          acc[a] = __ffma2_rn(make_float2(t, t), xv[u], acc[a]);
        }
    }
    cur = seg_end;
    const int64_t rt_end = (rt + 1) * nbc;
    if (cur == hi || cur == rt_end) {
      const int64_t slot = b - split_owner(rt * nbc, nblocks, G);
      const int64_t row = R0 + 512 * w + P * lane;
#pragma unroll
      for (int a = 0; a < P; ++a) part[slot * dpad + row + a] = acc[a];
      if (cur == rt_end)
        for (int64_t s = slot + 1; s < nslot; ++s)
#pragma unroll
          for (int a = 0; a < P; ++a) part[s * dpad + row + a] = make_float2(0.f, 0.f);
    }
  }
}

// ---------------------------------------------------------------------------
// FP32 form, NV = 2, 4, 8 or 16 vectors: the same persistent row split with
// a lane owning 16 rows of ONE vector.  The 32 lanes of a warp are 32 / NV
// row groups x NV vectors (lane L: group L / NV, vector L % NV), so a row
// tile has RB = 8 * 16 * 32 / NV rows and every lane keeps 16 accumulators,
// whatever NV.  Lanes of one row group read the same window entries
// (broadcast); the chunk's x is staged vector-major, xs[v][KC + 2], so a lane
// reads its 16 columns with eight 16-byte loads (the pad of 2 elements per
// vector row spreads the NV rows over the banks).  KC = 8192 / NV columns
// per chunk keeps the staged x at 64 KB.  Per 16 x 16 block a lane issues
// 256 packed FMAs against 16 shared-memory loads, as in the one-vector kernel.
// part[slot][row][v] as the row-owner kernels lay it out.
// ---------------------------------------------------------------------------
template <int NV>
struct DvrMv {
  static constexpr int GPW = 32 / NV;                  // row groups per warp
  static constexpr int RB = kDvrWarps * kDvrP * GPW;   // rows per row tile
  static constexpr int KC = 8192 / NV;                 // staged columns per chunk
  static constexpr int XLD = KC + 2;                   // staged row length (elements)
  static constexpr int NTB = RB + KC - 1;              // window entries per chunk
  static constexpr int TB_FLOATS = ((NTB + 1 + 15) / 16) * 20;
  static constexpr size_t SMEM = (size_t)TB_FLOATS * sizeof(float) + (size_t)NV * XLD * sizeof(float2);
};

template <int NV>
__global__ void __launch_bounds__(256, 2) dvr_rows_mv_f32(int64_t D, int64_t dpad, int64_t nslot, int64_t nbc,
                                                          int64_t nblocks, dvr_consts dk,
                                                          const float2* __restrict__ xc, float2* __restrict__ part) {
  using S = DvrMv<NV>;
  constexpr int P = kDvrP, U = kDvrU, KC = S::KC, BPC = KC / U;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* tb = reinterpret_cast<float*>(smem_raw);
  float2* xs = reinterpret_cast<float2*>(tb + S::TB_FLOATS);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int grp = lane / NV, v = lane % NV;
  const int64_t G = gridDim.x, b = blockIdx.x;
  const int64_t lo = split_lo(b, nblocks, G), hi = split_lo(b + 1, nblocks, G);
  const int rl0 = P * (S::GPW * w + grp);  // first tile row of the lane
  const int jb0 = rl0 + KC - U;            // window start of the chunk's first block
  const float2* xv_base = xs + v * S::XLD;
  float2 acc[P];
  for (int64_t cur = lo; cur < hi;) {
    const int64_t rt = cur / nbc, cb = cur - rt * nbc;
    const int64_t chunk = cb / BPC;
    const int64_t seg_end = min(hi, rt * nbc + min((chunk + 1) * BPC, nbc));
    if (cur == lo || cb == 0) {
#pragma unroll
      for (int a = 0; a < P; ++a) acc[a] = make_float2(0.f, 0.f);
    }
    const int64_t R0 = rt * S::RB, C0 = chunk * KC;
    __syncthreads();  // the previous segment is done with the staged chunk
    for (int e = tid; e < KC * NV; e += 256) {
      const int c = e / NV, vv = e % NV;
      const int64_t g = C0 + c;
      xs[vv * S::XLD + c] = g < D ? xc[g * NV + vv] : make_float2(0.f, 0.f);
    }
    const long long kmin = (long long)(R0 - C0) - KC + 1;
    for (int j = tid; j <= S::NTB; j += 256) tb[dvr_wpad(j)] = j < S::NTB ? dvr_T_f32(dk, kmin + j) : 0.f;
    __syncthreads();
    const int cc_beg = (int)(cb - chunk * BPC) * U, cc_end = cc_beg + (int)(seg_end - cur) * U;
#pragma unroll 1
    for (int cc = cc_beg; cc < cc_end; cc += U) {
      const int jb = jb0 - cc;  // a multiple of 16
      float win[32];
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const float4* q = reinterpret_cast<const float4*>(tb + dvr_wpad(jb + 16 * g));
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float4 t4 = q[i];
          win[16 * g + 4 * i] = t4.x;
          win[16 * g + 4 * i + 1] = t4.y;
          win[16 * g + 4 * i + 2] = t4.z;
          win[16 * g + 4 * i + 3] = t4.w;
        }
      }
      float2 xv[U];
      const float4* xq = reinterpret_cast<const float4*>(xv_base + cc);
#pragma unroll
      for (int i = 0; i < U / 2; ++i) {
        const float4 t4 = xq[i];
        xv[2 * i] = make_float2(t4.x, t4.y);
        xv[2 * i + 1] = make_float2(t4.z, t4.w);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int a = 0; a < P; ++a) {
          const float t = win[a - u + U - 1];
          acc[a] = __ffma2_rn(make_float2(t, t), xv[u], acc[a]);
        }
    }
    cur = seg_end;
    const int64_t rt_end = (rt + 1) * nbc;
    if (cur == hi || cur == rt_end) {
      const int64_t slot = b - split_owner(rt * nbc, nblocks, G);
      const int64_t row = R0 + rl0;
#pragma unroll
      for (int a = 0; a < P; ++a) part[(slot * dpad + row + a) * NV + v] = acc[a];
      if (cur == rt_end)
        for (int64_t s = slot + 1; s < nslot; ++s)
#pragma unroll
          for (int a = 0; a < P; ++a) part[(s * dpad + row + a) * NV + v] = make_float2(0.f, 0.f);
    }
  }
}

static DvrRowsShape rows_split_shape(int64_t D, int64_t rb, int64_t kc, int num_sms) {
  DvrRowsShape s{};
  s.rows = rb;
  s.cols = kc;
  s.rtiles = (D + rb - 1) / rb;
  s.nbc = (D + kDvrU - 1) / kDvrU;
  s.nblocks = s.rtiles * s.nbc;
  s.grid = std::min<int64_t>(2 * (int64_t)num_sms, s.nblocks);
  s.dpad = s.rtiles * rb;
  s.nslot = 1;
  for (int64_t rt = 0; rt < s.rtiles; ++rt) {
    const int64_t f = split_owner(rt * s.nbc, s.nblocks, s.grid);
    const int64_t l = split_owner(rt * s.nbc + s.nbc - 1, s.nblocks, s.grid);
    s.nslot = std::max(s.nslot, l - f + 1);
  }
  return s;
}

int64_t dvr_mv_bucket(int64_t nvec) { return nvec <= 2 ? 2 : nvec <= 4 ? 4 : nvec <= 8 ? 8 : 16; }

DvrRowsShape dvr_mv_shape(int64_t D, int64_t nb, int num_sms) {
  switch (nb) {
    case 2: return rows_split_shape(D, DvrMv<2>::RB, DvrMv<2>::KC, num_sms);
    case 4: return rows_split_shape(D, DvrMv<4>::RB, DvrMv<4>::KC, num_sms);
    case 8: return rows_split_shape(D, DvrMv<8>::RB, DvrMv<8>::KC, num_sms);
    default: return rows_split_shape(D, DvrMv<16>::RB, DvrMv<16>::KC, num_sms);
  }
}

template <int NV>
static cudaError_t launch_mv_t(const Plan& p, const void* xc, void* part) {
  const DvrRowsShape s = dvr_mv_shape(p.D, NV, p.num_sms);
  auto k = dvr_rows_mv_f32<NV>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DvrMv<NV>::SMEM);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)s.grid, 256, DvrMv<NV>::SMEM, p.stream>>>(p.D, s.dpad, s.nslot, s.nbc, s.nblocks, p.dvr,
                                                          (const float2*)xc, (float2*)part);
  return cudaGetLastError();
}

cudaError_t launch_dvr_mv(const Plan& p, const void* xc, void* part, int64_t nb) {
  if (p.prec != MF_PREC_FP32) return cudaErrorNotSupported;
  switch (nb) {
    case 2: return launch_mv_t<2>(p, xc, part);
    case 4: return launch_mv_t<4>(p, xc, part);
    case 8: return launch_mv_t<8>(p, xc, part);
    case 16: return launch_mv_t<16>(p, xc, part);
  }
  return cudaErrorNotSupported;
}

DvrRowsShape dvr_rows_shape(int64_t D, int num_sms) { return rows_split_shape(D, kDvrRB, kDvrKC, num_sms); }

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
  if (p.prec == MF_PREC_FP64) {
    constexpr int P = 8;
    const int kc = p.dvr_cols;
    const int64_t nslot = (p.D + kc - 1) / kc;
    const size_t sm = dvr_smem_bytes<double, P>(kc);
    auto k = dvr_window<double, P>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 grid((unsigned)((p.D + 32 * P - 1) / (32 * P)), (unsigned)nslot);
    k<<<grid, 256, sm, p.stream>>>(p.D, p.dpad, kc, p.dvr, (const double2*)xc, (double2*)part);
  } else {
    const DvrRowsShape s = dvr_rows_shape(p.D, p.num_sms);
    cudaFuncSetAttribute(dvr_rows_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDvrSmem);
    dvr_rows_f32<<<(unsigned)s.grid, 256, kDvrSmem, p.stream>>>(p.D, s.dpad, s.nslot, s.nbc, s.nblocks, p.dvr,
                                                                (const float2*)xc, (float2*)part);
  }
  return cudaGetLastError();
}

}  // namespace mf
