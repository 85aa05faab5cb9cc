// k_batch.cu -- many independent Hermitian problems in one persistent launch.
//
// Parameter-parallel execution (Sec. IV.H, "Adaptive parallelization"):
// independent problems need no communication, so on one GPU they share the
// SMs.  Every problem is a plan of its own (block size and cache chosen by
// its planner, bounds by Lanczos, Chebyshev coefficients for its own R*dt);
// each Chebyshev term forks one persistent kernel per work list (vector
// bucket and form: row-owner, or Hermitian-reuse for the FP32 problems of
// 1-6 vectors) onto side streams, each draining its (problem, 128-row tile)
// items through an atomic counter, so problems of uneven D and vector count
// balance across the SMs; the whole propagation -- every step and term --
// is captured once in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "rows_body.cuh"

namespace mf {

struct BatchProb {
  int64_t D, ntile, b, nblk, nv, nb;
  int64_t herm;  // Hermitian-reuse form: part holds 1 + ntile slots of dpad rows
  int64_t dpad;
  uint64_t seed;
  float sigma32;
  double sigma64;
  dvr_consts dk;
  void* xc;
  void* part;
  const void* cache;
  const int64_t* slot;
  double2* q[2];
  double2* acc;
  double2* psi;
  const double* J;
  double c, rinv, ph_r, ph_i;  // centre, 1 / half-width, e^{-i c dt}
};

struct BatchItem {
  int32_t prob, tile;
};

namespace {

// The work lists of the batched kernel: the row-owner form per vector bucket
// (batch_nvec_bucket of max(2, nvec)) and the Hermitian-reuse form (FP32, few
// vectors, where the stored bytes bound the product) for buckets 2, 4 and 6
// (at 8 vectors the row-owner form is faster: 16.7 vs 17.6 ms for 38
// problems of D = 16384).
// The batch pads a problem's vectors to the next of 2, 4, ..., 16 (10 and 14
// too: 9-10 vectors on the 10-wide tile take 17.8 ms where the 12-wide one
// takes 20.8, 13-14 on the 14-wide 24.9 where the 16-wide takes 27.2, for 38
// problems of D = 16384); the plan's workspace, sized for its row-kernel
// bucket (at least as many vectors), holds the batch's layout.
constexpr int kOwnerBuckets = 8;
constexpr int kBuckets = 11;
constexpr int kBucketNV[kBuckets] = {2, 4, 6, 8, 10, 12, 14, 16, 2, 4, 6};
constexpr bool kBucketHerm[kBuckets] = {false, false, false, false, false, false, false, false, true, true, true};

int64_t batch_nvec_bucket(int64_t nvec) {
  for (int k = 0; k < kOwnerBuckets; ++k)
    if (nvec <= kBucketNV[k]) return kBucketNV[k];
  return kBucketNV[kOwnerBuckets - 1];
}

// One row tile of a problem of bucket NB.  Register tiles (rows x vectors)
// and k-groups per bucket: the FP32 form takes 2 x 2 to 4 x 6 complex tiles
// in packed FP32 pairs over 2 to 8 k-groups (chosen by timing each bucket
// over a full cache); the FP64 form keeps one k-group (its registers are the
// limit).
template <typename T, int GEN, int NB>
__device__ __forceinline__ void batch_tile(unsigned char* smem_raw, const BatchProb& P, int64_t R0) {
  using C = typename cplx<T>::t;
  const C* xc = (const C*)P.xc;
  const C* cache = (const C*)P.cache;
  C* out = (C*)P.part + R0 * P.nb;
  if constexpr (sizeof(T) == 4) {
    constexpr int TR = NB == 2 ? 2 : NB == 4 ? 4 : NB == 6 ? 2 : NB == 8 ? 4 : NB == 10 ? 2 : NB == 12 ? 2 : NB == 14 ? 1 : 4;
    constexpr int TV = NB == 2 ? 2 : NB == 4 ? 4 : NB == 6 ? 6 : NB == 8 ? 4 : NB == 10 ? 10 : NB == 12 ? 6 : NB == 14 ? 14 : 4;
    constexpr int KG = NB == 2 ? 4 : NB == 4 ? 8 : NB == 6 ? 4 : NB == 8 ? 4 : NB == 10 ? 4 : 2;
    row_tile_async_f32<GEN, NB, TR, TV, 256, KG>(smem_raw, R0, 0, P.D, P.seed, P.sigma32, P.dk, (const float2*)xc,
                                                 (float2*)out, (const float2*)cache, P.slot, P.b, P.nblk);
  } else {
    constexpr int TR = NB <= 6 || NB == 10 || NB == 14 ? 1 : 2;
    constexpr int TV = NB == 2 ? 1 : NB == 4 ? 2 : NB == 6 ? 3 : NB == 8 ? 2 : NB == 10 ? 5 : NB == 12 ? 3 : NB == 14 ? 7 : 4;
    row_tile_async<T, GEN, NB, TR, TV, 256>(smem_raw, R0, 0, P.D, P.seed, (T)P.sigma64, P.dk, xc, out, cache, P.slot,
                                            P.b, P.nblk);
  }
}

// Persistent kernel of one bucket: drains its (problem, row tile) items,
// most expensive first, through an atomic counter.  One kernel per bucket
// (launched side by side) keeps each bucket's register allocation its own.
template <typename T, int GEN, int NB>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_batch_apply(const BatchItem* __restrict__ items, int n_items,
                                                     const BatchProb* __restrict__ probs, int* __restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= n_items) break;
    const BatchItem w = items[it];
    batch_tile<T, GEN, NB>(smem_raw, probs[w.prob], (int64_t)w.tile * rows::RT);
  }
}

// Hermitian-reuse form (FP32): row tile I sweeps the upper band, owner rows
// to slot 0, the chunks' H^dagger rows to slot 1 + I.
template <int GEN, int NB>
__device__ __forceinline__ void batch_tile_herm(unsigned char* smem_raw, const BatchProb& P, int64_t ti) {
  constexpr int TR = NB == 4 ? 4 : 2;
  constexpr int TV = NB;
  constexpr int KG = NB == 4 ? 8 : 4;
  const int64_t R0 = ti * rows::RT;
  float2* part = (float2*)P.part;
  row_tile_herm_f32<GEN, NB, TR, TV, 256, KG>(smem_raw, R0, P.D, P.seed, P.sigma32, P.dk, (const float2*)P.xc,
                                              part + R0 * NB, part + (1 + ti) * P.dpad * NB, P.dpad,
                                              (const float2*)P.cache, P.slot, P.b, P.nblk);
}

template <typename T, int GEN, int NB>
__global__ void __launch_bounds__(256, 2) k_batch_herm(const BatchItem* __restrict__ items, int n_items,
                                                       const BatchProb* __restrict__ probs, int* __restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= n_items) break;
    const BatchItem w = items[it];
    if constexpr (sizeof(T) == 4) batch_tile_herm<GEN, NB>(smem_raw, probs[w.prob], (int64_t)w.tile);
  }
}

template <typename T, int GEN>
using BatchKernel = void (*)(const BatchItem*, int, const BatchProb*, int*);

template <typename T, int GEN>
BatchKernel<T, GEN> batch_kernel(int k) {
  switch (k) {
    case 0: return k_batch_apply<T, GEN, 2>;
    case 1: return k_batch_apply<T, GEN, 4>;
    case 2: return k_batch_apply<T, GEN, 6>;
    case 3: return k_batch_apply<T, GEN, 8>;
    case 4: return k_batch_apply<T, GEN, 10>;
    case 5: return k_batch_apply<T, GEN, 12>;
    case 6: return k_batch_apply<T, GEN, 14>;
    case 7: return k_batch_apply<T, GEN, 16>;
    case 8: return k_batch_herm<T, GEN, 2>;
    case 9: return k_batch_herm<T, GEN, 4>;
    default: return k_batch_herm<T, GEN, 6>;
  }
}

template <typename T>
size_t batch_smem(int k) {
  if constexpr (sizeof(T) == 4) {
    switch (k) {
      case 0: return rows_smem_bytes_f32<2>();
      case 1: return rows_smem_bytes_f32<4>();
      case 2: return rows_smem_bytes_f32<6>();
      case 3: return rows_smem_bytes_f32<8>();
      case 4: return rows_smem_bytes_f32<10>();
      case 5: return rows_smem_bytes_f32<12>();
      case 6: return rows_smem_bytes_f32<14>();
      case 7: return rows_smem_bytes_f32<16>();
      case 8: return herm_smem_bytes_f32<2>();
      case 9: return herm_smem_bytes_f32<4>();
      default: return herm_smem_bytes_f32<6>();
    }
  } else {
    switch (k) {
      case 0: return rows_smem_bytes_async<double, 2>();
      case 1: return rows_smem_bytes_async<double, 4>();
      case 2: return rows_smem_bytes_async<double, 6>();
      case 3: return rows_smem_bytes_async<double, 8>();
      case 4: return rows_smem_bytes_async<double, 10>();
      case 5: return rows_smem_bytes_async<double, 12>();
      case 6: return rows_smem_bytes_async<double, 14>();
      default: return rows_smem_bytes_async<double, 16>();
    }
  }
}

int bucket_index(int64_t nb, bool herm) {
  for (int k = 0; k < kBuckets; ++k)
    if (kBucketNV[k] == nb && kBucketHerm[k] == herm) return k;
  return kOwnerBuckets - 1;
}

// q_cur = psi, acc = J0 psi, xc = compute copy (padding zero); grid.y = problem
template <typename C>
__global__ void k_batch_init(const BatchProb* __restrict__ probs, int parity) {
  const BatchProb& P = probs[blockIdx.y];
  const int64_t n = P.D * P.nb;
  const double a0 = P.J[0];
  double2* q = P.q[parity];
  C* xc = (C*)P.xc;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / P.nb, v = e % P.nb;
    C o;
    o.x = 0;
    o.y = 0;
    if (v < P.nv) {
      const int64_t i = row * P.nv + v;
      const double2 a = P.psi[i];
      q[i] = a;
      P.acc[i] = make_double2(a0 * a.x, a0 * a.y);
      o.x = (decltype(o.x))a.x;
      o.y = (decltype(o.y))a.y;
    }
    xc[e] = o;
  }
}

// y = part + V q; t = (y - c q)/R (as a product with 1/R, like the one-plan
// update); q_next = t or 2t - q_prev; acc += a_j q_next
template <typename C>
__global__ void k_batch_update(const BatchProb* __restrict__ probs, int parity, int32_t j, int gen_dvr) {
  const BatchProb& P = probs[blockIdx.y];
  const int64_t n = P.D * P.nv;
  const double2* qc = P.q[parity];
  double2* qp = P.q[1 - parity];
  const C* part = (const C*)P.part;
  C* xc = (C*)P.xc;
  const double aj = 2.0 * P.J[j], c = P.c, rinv = P.rinv;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / P.nv, v = e % P.nv, ci = row * P.nb + v;
    const C pv = part[ci];
    double yr = (double)pv.x, yi = (double)pv.y;
    if (P.herm) {
      // the H^dagger rows from the row tiles above this row's, in tile order
      const int64_t tile = row / rows::RT;
      for (int64_t s2 = 1; s2 <= tile; ++s2) {
        const C ps = part[s2 * P.dpad * P.nb + ci];
        yr += (double)ps.x;
        yi += (double)ps.y;
      }
    }
    const double2 q = qc[e];
    if (gen_dvr) {
      const double V = dvr_V(P.dk, row);
      yr = fma(V, q.x, yr);
      yi = fma(V, q.y, yi);
    }
    double tr = (yr - c * q.x) * rinv, ti = (yi - c * q.y) * rinv;
    if (j > 1) {
      const double2 o = qp[e];
      tr = 2.0 * tr - o.x;
      ti = 2.0 * ti - o.y;
    }
    qp[e] = make_double2(tr, ti);
    double rr, ri;
    switch (j & 3) {
      case 0: rr = tr; ri = ti; break;
      case 1: rr = ti; ri = -tr; break;
      case 2: rr = -tr; ri = -ti; break;
      default: rr = -ti; ri = tr; break;
    }
    double2 a = P.acc[e];
    a.x = fma(aj, rr, a.x);
    a.y = fma(aj, ri, a.y);
    P.acc[e] = a;
    C o;
    o.x = (decltype(o.x))tr;
    o.y = (decltype(o.y))ti;
    xc[ci] = o;
  }
}

__global__ void k_batch_final(const BatchProb* __restrict__ probs) {
  const BatchProb& P = probs[blockIdx.y];
  const int64_t n = P.D * P.nv;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = P.acc[e];
    P.psi[e] = make_double2(P.ph_r * a.x - P.ph_i * a.y, P.ph_r * a.y + P.ph_i * a.x);
  }
}

}  // namespace
}  // namespace mf

using namespace mf;

struct mf_batch {
  std::vector<mf_plan_t> plans;
  std::vector<int64_t> offsets;  // element offsets of each problem in the packed vector
  int32_t gen = 0, prec = MF_PREC_FP32;
  int num_sms = 0, persist_grid = 0;
  cudaStream_t user = nullptr, own = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  BatchProb* d_probs = nullptr;
  BatchItem* d_items = nullptr;
  int n_items = 0;
  int* d_counter = nullptr;  // one per bucket
  // per bucket: its items d_items[begin[k] .. begin[k + 1]), dynamic shared
  // memory, persistent grid, and a side stream (the buckets' kernels run side
  // by side: fork from own, join back)
  int begin[kBuckets + 1] = {};
  size_t smem[kBuckets] = {};
  int grid[kBuckets] = {};
  cudaStream_t side[kBuckets] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kBuckets] = {};
  int64_t max_elems = 0;
  // Hermitian-reuse problems: their 1 + ntile slots of dpad rows (owned)
  std::vector<void*> hbuf;
  // captured propagation and the arguments it was captured for
  cudaGraphExec_t graph = nullptr;
  double g_dt = 0.0;
  int32_t g_steps = 0, g_order = -1;
  void* g_psi = nullptr;
  int32_t g_terms = 0;
};

namespace {

void batch_release(mf_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (auto p : b->plans) mf_plan_destroy(p);
  for (void* h : b->hbuf)
    if (h) cudaFree(h);
  if (b->d_probs) cudaFree(b->d_probs);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_counter) cudaFree(b->d_counter);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  for (int k = 0; k < kBuckets; ++k) {
    if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
    if (b->side[k]) cudaStreamDestroy(b->side[k]);
  }
  if (b->own) cudaStreamDestroy(b->own);
  delete b;
}

unsigned grid_x(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096)); }

template <typename T>
cudaError_t launch_batch_apply(mf_batch* b, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, kBuckets * sizeof(int), s);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_fork, s);
  for (int k = 0; k < kBuckets && e == cudaSuccess; ++k) {
    const int n = b->begin[k + 1] - b->begin[k];
    if (n == 0) continue;
    e = cudaStreamWaitEvent(b->side[k], b->ev_fork, 0);
    if (e != cudaSuccess) break;
    auto kern = b->gen == MF_GEN_PHILOX_GUE ? batch_kernel<T, MF_GEN_PHILOX_GUE>(k)
                                            : batch_kernel<T, MF_GEN_SINC_DVR_HO>(k);
    kern<<<b->grid[k], 256, b->smem[k], b->side[k]>>>(b->d_items + b->begin[k], n, b->d_probs, b->d_counter + k);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_join[k], b->side[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev_join[k], 0);
  }
  return e;
}

// Enqueue nsteps Chebyshev steps of nterms terms on stream s.
template <typename T>
cudaError_t enqueue_propagation(mf_batch* b, int32_t nsteps, int32_t nterms, cudaStream_t s) {
  using C = typename cplx<T>::t;
  const unsigned gx = grid_x(b->max_elems);
  const unsigned np = (unsigned)b->plans.size();
  const int dvr = b->gen == MF_GEN_SINC_DVR_HO;
  for (int32_t step = 0; step < nsteps; ++step) {
    int parity = 0;
    k_batch_init<C><<<dim3(gx, np), 256, 0, s>>>(b->d_probs, parity);
    for (int32_t j = 1; j < nterms; ++j) {
      cudaError_t e = launch_batch_apply<T>(b, s);
      if (e != cudaSuccess) return e;
      k_batch_update<C><<<dim3(gx, np), 256, 0, s>>>(b->d_probs, parity, j, dvr);
      parity ^= 1;
    }
    k_batch_final<<<dim3(gx, np), 256, 0, s>>>(b->d_probs);
  }
  return cudaGetLastError();
}

}  // namespace

extern "C" {

mf_status mf_batch_create(mf_batch_t* out, int32_t nprob, const int64_t* D, const int32_t* nvec,
                          const uint64_t* seeds, int32_t generator, size_t cache_budget_bytes,
                          const mf_options* opt) {
  return guard([&]() -> mf_status {
    if (!out || nprob < 1 || !D || !nvec || !seeds) return MF_ERR_INVALID;
    *out = nullptr;
    mf_options o;
    if (opt) o = *opt; else mf_options_default(&o);
    if (o.precision == MF_PREC_BF16X2) return MF_ERR_UNSUPPORTED;
    for (int32_t i = 0; i < nprob; ++i)
      if (D[i] < 2 || nvec[i] < 1 || nvec[i] > 16) return MF_ERR_INVALID;
    mf_batch* b = new (std::nothrow) mf_batch();
    if (!b) return MF_ERR_OOM;
    b->gen = generator;
    b->prec = o.precision;
    b->user = (cudaStream_t)o.stream;
    if (cudaSetDevice(o.device) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, o.device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
      batch_release(b);
      return MF_ERR_CUDA;
    }
    for (int k = 0; k < kBuckets; ++k)
      if (cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming) != cudaSuccess) {
        batch_release(b);
        return MF_ERR_CUDA;
      }
    // cache budget shared in proportion to each problem's full canonical cache
    const double eb = o.precision == MF_PREC_FP64 ? 16.0 : 8.0;
    double total_full = 0.0;
    for (int32_t i = 0; i < nprob; ++i) total_full += eb * (double)D[i] * (double)D[i] / 2.0;
    b->offsets.push_back(0);
    for (int32_t i = 0; i < nprob; ++i) {
      mf_options oi = o;
      oi.nvec_hint = nvec[i];
      oi.stream = b->own;
      oi.hermitian_reuse = 0;  // the batched kernel writes one row-owner slot per row
      oi.row_begin = oi.row_end = 0;
      const double share = cache_budget_bytes == 0 ? 0.0
                           : std::min((double)cache_budget_bytes, 1e18) * (eb * (double)D[i] * D[i] / 2.0) / total_full;
      mf_plan_t p = nullptr;
      mf_status st = mf_plan_create(&p, D[i], D[i], generator, seeds[i], 0, (size_t)share, &oi);
      if (st != MF_OK && st != MF_WARN_DENSE_WORK) {
        batch_release(b);
        return st;
      }
      b->plans.push_back(p);
      if ((st = plan_workspace(p->p, std::max<int64_t>(2, nvec[i]))) != MF_OK || (st = plan_bounds(p->p)) != MF_OK) {
        batch_release(b);
        return st;
      }
      b->offsets.push_back(b->offsets.back() + D[i] * nvec[i]);
      b->max_elems = std::max<int64_t>(b->max_elems, D[i] * rows_nvec_bucket(std::max<int32_t>(2, nvec[i])));
    }
    // Hermitian-reuse form for the FP32 problems of buckets 2, 4 and 6 (their
    // products are bound by the stored bytes, which it halves) while the
    // slots of 1 + ntile partial rows fit, all together, in a tenth of the
    // memory free after the plans (they grow as D^2 / 128 per vector); the
    // row-owner form otherwise
    b->hbuf.assign(nprob, nullptr);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      free_b = 0;
    }
    size_t slot_room = free_b / 10;
    for (int32_t i = 0; i < nprob && o.precision == MF_PREC_FP32; ++i) {
      const Plan& P = b->plans[i]->p;
      const int64_t nb = batch_nvec_bucket(std::max<int32_t>(2, nvec[i]));
      if (nb > 6) continue;
      const size_t bytes = (size_t)(1 + P.ntile) * (size_t)(P.ntile * rows::RT) * (size_t)nb * sizeof(float2);
      if (bytes > slot_room) continue;
      slot_room -= bytes;
      if (dev_malloc(&b->hbuf[i], bytes) != cudaSuccess) {
        cudaGetLastError();
        b->hbuf[i] = nullptr;
      }
    }
    // work lists: every (problem, row tile), by vector bucket and form, each
    // list's most expensive first
    std::vector<BatchItem> items;
    std::vector<double> cost;
    std::vector<int> bucket;
    for (int32_t i = 0; i < nprob; ++i) {
      const Plan& P = b->plans[i]->p;
      const int64_t nb = batch_nvec_bucket(std::max<int32_t>(2, nvec[i]));
      const bool herm = b->hbuf[i] != nullptr;
      for (int64_t t = 0; t < P.ntile; ++t) {
        items.push_back(BatchItem{i, (int32_t)t});
        cost.push_back((double)(herm ? P.D - t * rows::RT : P.D) * (double)nb);
        bucket.push_back(bucket_index(nb, herm));
      }
    }
    std::vector<size_t> idx(items.size());
    for (size_t k = 0; k < idx.size(); ++k) idx[k] = k;
    std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t c) {
      return bucket[a] != bucket[c] ? bucket[a] < bucket[c] : cost[a] > cost[c];
    });
    std::vector<BatchItem> sorted;
    for (size_t k : idx) sorted.push_back(items[k]);
    for (int k = 0; k <= kBuckets; ++k) b->begin[k] = 0;
    for (int bk : bucket) ++b->begin[bk + 1];
    for (int k = 0; k < kBuckets; ++k) b->begin[k + 1] += b->begin[k];
    b->n_items = (int)sorted.size();
    cudaError_t e = dev_malloc((void**)&b->d_items, sorted.size() * sizeof(BatchItem));
    if (e == cudaSuccess)
      e = cudaMemcpy(b->d_items, sorted.data(), sorted.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = dev_malloc((void**)&b->d_counter, kBuckets * sizeof(int));
    if (e == cudaSuccess) e = dev_malloc((void**)&b->d_probs, (size_t)nprob * sizeof(BatchProb));
    // persistent grid per bucket: resident CTAs per SM x SMs, at most its items
    for (int k = 0; k < kBuckets && e == cudaSuccess; ++k) {
      const bool f64 = o.precision == MF_PREC_FP64;
      b->smem[k] = f64 ? batch_smem<double>(k) : batch_smem<float>(k);
      const void* kern =
          f64 ? (generator == MF_GEN_PHILOX_GUE ? (const void*)batch_kernel<double, MF_GEN_PHILOX_GUE>(k)
                                                : (const void*)batch_kernel<double, MF_GEN_SINC_DVR_HO>(k))
              : (generator == MF_GEN_PHILOX_GUE ? (const void*)batch_kernel<float, MF_GEN_PHILOX_GUE>(k)
                                                : (const void*)batch_kernel<float, MF_GEN_SINC_DVR_HO>(k));
      int per_sm = 0;
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem[k]);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, b->smem[k]);
      const int n = b->begin[k + 1] - b->begin[k];
      b->grid[k] = std::max(1, std::min(std::max(1, per_sm) * b->num_sms, n));
      b->persist_grid = std::max(b->persist_grid, b->grid[k]);
    }
    if (e != cudaSuccess) {
      batch_release(b);
      return e == cudaErrorMemoryAllocation ? MF_ERR_OOM : MF_ERR_CUDA;
    }
    *out = b;
    return MF_OK;
  });
}

mf_status mf_batch_destroy(mf_batch_t b) {
  if (!b) return MF_OK;
  cudaStreamSynchronize(b->own);
  batch_release(b);
  return MF_OK;
}

mf_status mf_batch_offsets(mf_batch_t b, int64_t* offsets) {
  if (!b || !offsets) return MF_ERR_INVALID;
  std::memcpy(offsets, b->offsets.data(), b->offsets.size() * sizeof(int64_t));
  return MF_OK;
}

mf_status mf_batch_propagate(mf_batch_t b, void* psi, double dt, int32_t nsteps, int32_t order, int32_t* nterms_out) {
  return guard([&]() -> mf_status {
    if (!b || !psi || !(dt > 0) || !std::isfinite(dt) || nsteps < 1 || order < 0) return MF_ERR_INVALID;
    const bool same = b->graph && b->g_dt == dt && b->g_steps == nsteps && b->g_order == order && b->g_psi == psi;
    if (!same) {
      // per-problem coefficients for its own R dt; a common term count (the
      // largest one needed, so every problem meets the tolerance)
      int32_t nt = order;
      std::vector<int32_t> need(b->plans.size());
      for (size_t i = 0; i < b->plans.size(); ++i) {
        Plan& P = b->plans[i]->p;
        const double R = 0.5 * (P.emax - P.emin);
        mf_status st = plan_coefficients(P, R * dt, order, &need[i]);
        if (st != MF_OK) return st;
        nt = std::max(nt, need[i]);
      }
      if (order == 0) {
        for (size_t i = 0; i < b->plans.size(); ++i) {
          Plan& P = b->plans[i]->p;
          const double R = 0.5 * (P.emax - P.emin);
          int32_t dummy = 0;
          mf_status st = plan_coefficients(P, R * dt, nt, &dummy);
          if (st != MF_OK) return st;
        }
      }
      std::vector<BatchProb> probs(b->plans.size());
      for (size_t i = 0; i < b->plans.size(); ++i) {
        Plan& P = b->plans[i]->p;
        BatchProb& q = probs[i];
        q.D = P.D;
        q.ntile = P.ntile;
        q.b = P.b;
        q.nblk = P.nblk;
        q.nv = b->offsets[i + 1] - b->offsets[i];
        q.nv /= P.D;
        q.nb = batch_nvec_bucket(std::max<int64_t>(2, q.nv));
        q.seed = P.seed;
        q.sigma32 = P.sigma32;
        q.sigma64 = P.sigma64;
        q.dk = P.dvr;
        q.xc = P.d_xc;
        q.herm = b->hbuf[i] != nullptr;
        q.dpad = P.ntile * rows::RT;
        q.part = q.herm ? b->hbuf[i] : P.d_part;
        q.cache = P.pairs_cached > 0 ? P.d_cache : nullptr;
        q.slot = P.d_pair_slot;
        q.q[0] = P.d_q[0];
        q.q[1] = P.d_q[1];
        q.acc = P.d_q[2];
        q.psi = (double2*)psi + b->offsets[i];
        q.J = P.d_J;
        q.c = 0.5 * (P.emax + P.emin);
        q.rinv = 1.0 / (0.5 * (P.emax - P.emin));
        q.ph_r = std::cos(q.c * dt);
        q.ph_i = -std::sin(q.c * dt);
      }
      if (cudaStreamSynchronize(b->own) != cudaSuccess) return MF_ERR_CUDA;
      if (cudaMemcpy(b->d_probs, probs.data(), probs.size() * sizeof(BatchProb), cudaMemcpyHostToDevice) != cudaSuccess)
        return MF_ERR_CUDA;
      // capture the whole propagation once
      if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
      }
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MF_ERR_CUDA;
      cudaError_t e = b->prec == MF_PREC_FP64 ? enqueue_propagation<double>(b, nsteps, nt, b->own)
                                              : enqueue_propagation<float>(b, nsteps, nt, b->own);
      cudaError_t e2 = cudaStreamEndCapture(b->own, &g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return MF_ERR_CUDA;
      }
      e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return MF_ERR_CUDA;
      b->g_dt = dt;
      b->g_steps = nsteps;
      b->g_order = order;
      b->g_psi = psi;
      b->g_terms = nt;
    }
    // order the graph after the caller's stream and the caller's stream after it
    if (cudaEventRecord(b->ev_in, b->user) != cudaSuccess || cudaStreamWaitEvent(b->own, b->ev_in, 0) != cudaSuccess ||
        cudaGraphLaunch(b->graph, b->own) != cudaSuccess || cudaEventRecord(b->ev_out, b->own) != cudaSuccess ||
        cudaStreamWaitEvent(b->user, b->ev_out, 0) != cudaSuccess)
      return MF_ERR_CUDA;
    if (nterms_out) *nterms_out = b->g_terms;
    return MF_OK;
  });
}

mf_status mf_batch_plan(mf_batch_t b, int32_t i, mf_plan_t* plan) {
  if (!b || !plan || i < 0 || i >= (int32_t)b->plans.size()) return MF_ERR_INVALID;
  *plan = b->plans[i];
  return MF_OK;
}

mf_status mf_batch_form(mf_batch_t b, int32_t i, int32_t* hermitian) {
  if (!b || !hermitian || i < 0 || i >= (int32_t)b->plans.size()) return MF_ERR_INVALID;
  *hermitian = b->hbuf[i] != nullptr;
  return MF_OK;
}

mf_status mf_batch_info(mf_batch_t b, int32_t* n_items, int32_t* persist_grid) {
  if (!b) return MF_ERR_INVALID;
  if (n_items) *n_items = b->n_items;
  if (persist_grid) *persist_grid = b->persist_grid;
  return MF_OK;
}

}  // extern "C"
