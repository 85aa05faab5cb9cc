// mf_api.cu -- host implementation of the C ABI declared in include/mf.h.
//
// Plan creation follows Sec. IV of the paper: a block partition (Sec. II),
// a storage mode and cache budget (Sec. III.A, Sec. IV.G, Eq.
// partial_cache_pairs), a memory-feasibility check (Eq.
// planner_memory_constraint), a dense-work safety estimate (Sec. IV.H) and a
// launch shape.  The apply follows Eq. blockmatvec; the propagator follows
// Sec. VII (centred Chebyshev with Lanczos bounds).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "mf_internal.h"

using namespace mf;

namespace mf {

namespace {
std::mutex g_fault_mu;
std::string g_fault_value;  // MF_FAULT as last seen
long long g_fault_count = 0;  // events of its site since it took that value
}  // namespace

bool fault_hit(const char* site) {
  const char* v = std::getenv("MF_FAULT");
  if (!v || !*v) return false;
  std::lock_guard<std::mutex> lock(g_fault_mu);
  if (g_fault_value != v) {
    g_fault_value = v;
    g_fault_count = 0;
  }
  const char* colon = std::strchr(v, ':');
  const size_t n = colon ? (size_t)(colon - v) : std::strlen(v);
  if (std::strlen(site) != n || std::strncmp(site, v, n) != 0) return false;
  const long long want = colon ? std::atoll(colon + 1) : 1;
  return ++g_fault_count == want;
}

cudaError_t dev_malloc(void** ptr, size_t bytes) {
  if (fault_hit("alloc")) {
    *ptr = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(ptr, bytes);
}

void dvr_setup(dvr_consts& k, int64_t D, double L) {
  k.L = L > 0 ? L : 0.9 * std::sqrt(2.0 * (double)D);
  k.dx = (2.0 * k.L) / (double)(D - 1);
  k.dx2 = k.dx * k.dx;
  const double PI2_6 = 0x1.a51a6625307d3p+0;  // pi^2 / 6 rounded to double
  k.t0_64 = PI2_6 / k.dx2;
  k.t0_32 = (float)k.t0_64;
  k.c32 = (float)(1.0 / k.dx2);
}

void dvr_fp32_window_shape(Plan& p) {
  const DvrRowsShape s = dvr_rows_shape(p.D, p.num_sms);
  p.dvr_rows = (int)s.rows;
  p.dvr_cols = (int)s.cols;
  p.nslot = s.nslot;
  p.dpad = s.dpad;
}

}  // namespace mf

namespace {

#define MF_CUDA(call)                                      \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) {                               \
      if (e_ == cudaErrorMemoryAllocation) return MF_ERR_OOM; \
      return MF_ERR_CUDA;                                  \
    }                                                      \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

template <typename T>
void free_dev(T*& ptr) {
  if (ptr) cudaFree((void*)ptr);
  ptr = nullptr;
}

// cudaMalloc through the fault-injection site, typed.
template <typename T>
cudaError_t dmalloc(T** ptr, size_t bytes) {
  void* v = nullptr;
  const cudaError_t e = dev_malloc(&v, bytes);
  *ptr = (T*)v;
  return e;
}

mf_status status_of_device_code(int code) {
  if (code == 0) return MF_OK;
  if (code >= kErrTimeoutFirst && code <= kErrTimeoutLast) return MF_ERR_TIMEOUT;
  return MF_ERR_CUDA;
}

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
}

// The device error word an earlier call left, read without blocking: only
// once the copy enqueued after that call has completed.  A nonzero word is
// cleared and reported; the calling entry point then enqueues nothing.
mf_status pending_device_error(Plan& p) {
  if (!p.err_pending || capturing(p.stream)) return MF_OK;
  const cudaError_t q = cudaEventQuery(p.err_ev);
  if (q == cudaErrorNotReady) return MF_OK;
  if (q != cudaSuccess) return MF_ERR_CUDA;
  p.err_pending = false;
  const int code = *(volatile int*)p.h_err;
  if (code == 0) return MF_OK;
  p.last_dev_err = code;
  if (cudaMemsetAsync(p.d_err, 0, sizeof(int), p.stream) != cudaSuccess) return MF_ERR_CUDA;
  return status_of_device_code(code);
}

// After a call whose kernels may set the word: enqueue its copy to the host.
mf_status post_device_error_copy(Plan& p) {
  if (!p.has_waits || capturing(p.stream)) return MF_OK;
  if (cudaMemcpyAsync(p.h_err, p.d_err, sizeof(int), cudaMemcpyDeviceToHost, p.stream) != cudaSuccess ||
      cudaEventRecord(p.err_ev, p.stream) != cudaSuccess)
    return MF_ERR_CUDA;
  p.err_pending = true;
  return MF_OK;
}

void release(Plan& p) {
  for (auto& e : p.ev) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  p.ev.clear();
  free_dev(p.d_cache);
  free_dev(p.d_work);
  free_dev(p.d_herm_items);
  free_dev(p.d_pair_slot);
  free_dev(p.d_part);
  free_dev(p.d_xc);
  free_dev(p.d_tcb);
  for (auto& q : p.d_q) free_dev(q);
  free_dev(p.d_J);
  free_dev(p.d_red);
  free_dev(p.d_err);
  if (p.h_err) cudaFreeHost(p.h_err);
  p.h_err = nullptr;
  if (p.err_ev) cudaEventDestroy(p.err_ev);
  p.err_ev = nullptr;
  p.err_pending = false;
  if (p.h_registered) cudaHostUnregister(const_cast<void*>(p.h_blocks));
  p.h_registered = false;
  free_dev(p.d_sb_seeds);
  free_dev(p.d_sb_M);
  free_dev(p.d_sb_HS);
  free_dev(p.d_sb_xo);
  free_dev(p.d_tch_units);
  free_dev(p.d_tch_off);
  free_dev(p.d_tch_counter);
  free_dev(p.d_tch_slots);
  p.tch_slots_cap = 0;
  p.part_cap = p.xc_cap = p.tcb_cap = p.sb_xo_cap = 0;
  for (auto& c : p.q_cap) c = 0;
}

// Vector shape of the path used for nvec vectors: the Hermitian or DVR
// window path for one vector; for several, the DVR window kernel (FP32
// procedural DVR, 2..16 vectors) or the row-owner path, padded to a
// compiled vector count.
// The Hermitian-reuse multi-vector path (each canonical entry applied as H
// and H^dagger) is used for the Philox ensemble and stored blocks with up to
// 16 vectors while its partial slots (one per owner item and per row tile)
// take at most min(16 GB, 10 % of the memory free at plan creation);
// otherwise the row-owner path.
bool use_rows_herm(const Plan& p, int64_t nb) {
  if (!p.d_herm_items || p.gen == MF_GEN_SINC_DVR_HO || p.prec == MF_PREC_BF16X2 || nb > 16) return false;
  if (p.opt.hermitian_reuse == 0) return false;
  const double bytes = (double)(p.herm_ns + p.ntile) * (double)(p.ntile * kTile) * (double)nb *
                       (double)compute_elem_bytes(p.prec);
  return bytes <= p.herm_limit;
}

// The Hermitian-reuse tensor-core walk: chosen at plan creation for BF16X2
// Philox plans over all rows (opt.hermitian_reuse != 0) whose unit slots
// for 64 vectors fit the plan's limit; such a plan keeps its cache in the
// walk's tile format, so every BF16X2 product of the plan takes the walk.
double tch_slot_bytes(const Plan& p, int64_t nb) { return (double)p.tch_rows * 2.0 * (double)nb * 4.0; }
bool use_tch(const Plan& p, int64_t) { return p.tch; }

// Two vectors in the FP32 form on the canonical-tile kernel (each generated
// or stored entry applied to both vectors as H and H^dagger from registers),
// for plans with the tile work list.
bool use_tile2(const Plan& p, int64_t nvec) {
  return nvec == 2 && p.prec == MF_PREC_FP32 && p.d_work && !p.use_dvr_window && !p.sliced && !p.sb_nop &&
         p.opt.hermitian_reuse != 0;
}

// The DVR window kernel for 2..16 vectors (FP32 form, procedural plans).
bool use_dvr_mv(const Plan& p, int64_t nvec) {
  return p.use_dvr_window && p.prec == MF_PREC_FP32 && !p.sb_nop && nvec >= 2 && nvec <= 16;
}

VecShape shape_for(const Plan& p, int64_t nvec) {
  if (p.prec == MF_PREC_BF16X2) {
    const int64_t nb = tc_nvec_bucket(nvec);
    // the unit walk hands its FP64 row sums on as two FP32 slots (hi, lo)
    return VecShape{nvec, nb, use_tch(p, nb) ? 2 : p.rows_nsplit, p.ntile * (int64_t)kTile};
  }
  if (p.sliced) return VecShape{nvec, rows_nvec_bucket(nvec), p.rows_nsplit, p.slice_nt * (int64_t)kTile};
  if (nvec == 1 && !p.sb_nop) return VecShape{1, 1, p.nslot, p.dpad};
  if (use_dvr_mv(p, nvec)) {
    const int64_t nb = dvr_mv_bucket(nvec);
    const DvrRowsShape s = dvr_mv_shape(p.D, nb, p.num_sms);
    return VecShape{nvec, nb, s.nslot, s.dpad};
  }
  if (use_tile2(p, nvec)) return VecShape{2, 2, p.nslot, p.dpad};
  const int64_t nb = rows_nvec_bucket(nvec);
  if (use_rows_herm(p, nb)) return VecShape{nvec, nb, p.herm_ns + p.ntile, p.ntile * (int64_t)kTile};
  return VecShape{nvec, nb, p.rows_nsplit, p.ntile * (int64_t)kTile};
}

// Workspace for nvec vectors: partial slots and compute copy (the larger of
// the one-vector and nvec shapes, each with its padded vector count), the
// tensor-core operand tiles, three FP64 vectors and the system-bath mixed
// inputs.  Each buffer grows when a call needs more than it holds; a smaller
// vector count can need more partial slots than a larger one, since it may
// take another kernel.
mf_status ensure_workspace(Plan& p, int64_t nvec) {
  const size_t eb = compute_elem_bytes(p.prec);
  const VecShape m = shape_for(p, nvec);
  size_t part_bytes = 0, xc_bytes = 0;
  for (const VecShape& s : {shape_for(p, 1), m}) {
    part_bytes = std::max(part_bytes, (size_t)s.nslot * (size_t)s.dpad * (size_t)s.nb * eb);
    xc_bytes = std::max(xc_bytes, (size_t)std::max<int64_t>(s.dpad, p.D) * (size_t)s.nb * eb);
  }
  const bool tch = p.prec == MF_PREC_BF16X2 && use_tch(p, m.nb);
  const size_t tcb_bytes =
      p.prec == MF_PREC_BF16X2 ? (tch ? tch_operand_bytes(p.D, m.nb) : tc_operand_bytes(p.D, m.nb)) : 0;
  const size_t tch_bytes = tch ? (size_t)tch_slot_bytes(p, m.nb) : 0;
  const size_t q_bytes = (size_t)p.D * (size_t)nvec * sizeof(double2);
  const int64_t sb_rows = std::max<int64_t>(m.dpad, p.D);
  const size_t xo_bytes = p.sb_nop ? (size_t)p.sb_nop * (size_t)sb_rows * (size_t)m.nb * eb : 0;
  auto grow = [](void** ptr, size_t& cap, size_t need, bool zero) -> mf_status {
    if (need <= cap) return MF_OK;
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    cap = 0;
    MF_CUDA(dev_malloc(ptr, need));
    if (zero) MF_CUDA(cudaMemset(*ptr, 0, need));
    cap = need;
    return MF_OK;
  };
  mf_status st = MF_OK;
  if ((st = grow(&p.d_part, p.part_cap, part_bytes, false)) != MF_OK) return st;
  if ((st = grow(&p.d_xc, p.xc_cap, xc_bytes, true)) != MF_OK) return st;
  if (tcb_bytes && (st = grow(&p.d_tcb, p.tcb_cap, tcb_bytes, false)) != MF_OK) return st;
  if (tch_bytes && (st = grow(&p.d_tch_slots, p.tch_slots_cap, tch_bytes, false)) != MF_OK) return st;
  for (int i = 0; i < 3; ++i)
    if ((st = grow((void**)&p.d_q[i], p.q_cap[i], q_bytes, false)) != MF_OK) return st;
  if (p.sb_nop) {
    if ((st = grow(&p.d_sb_xo, p.sb_xo_cap, xo_bytes, false)) != MF_OK) return st;
    p.sb_rows = sb_rows;
  }
  return MF_OK;
}

mf_status ensure_J(Plan& p, int32_t K) {
  if (K + 1 <= p.J_cap) return MF_OK;
  free_dev(p.d_J);
  const int32_t cap = std::max<int32_t>(K + 1, 256);
  MF_CUDA(dmalloc(&p.d_J, (size_t)cap * sizeof(double)));
  p.J_cap = cap;
  p.J_arg = -1.0;
  return MF_OK;
}

// The generate-and-apply kernel of the plan's path (xc -> partial slots),
// bracketed by CUDA events when profiling is on.
mf_status apply_kernel(Plan& p, int64_t nvec) {
  if (p.profiling) {
    if (p.ev_used == p.ev.size()) {
      std::pair<cudaEvent_t, cudaEvent_t> e;
      MF_CUDA(cudaEventCreate(&e.first));
      MF_CUDA(cudaEventCreate(&e.second));
      p.ev.push_back(e);
    }
    MF_CUDA(cudaEventRecord(p.ev[p.ev_used].first, p.stream));
  }
  if (fault_hit("launch")) return MF_ERR_CUDA;
  const int64_t nbr = rows_nvec_bucket(nvec);
  const bool tile2 = use_tile2(p, nvec);
  const bool herm =
      !tile2 && !p.sliced && (nvec > 1 || p.sb_nop) && p.prec != MF_PREC_BF16X2 && use_rows_herm(p, nbr);
  if (herm) {
    const VecShape sh = shape_for(p, nvec);
    MF_CUDA(cudaMemsetAsync(p.d_part, 0, (size_t)sh.nslot * sh.dpad * sh.nb * compute_elem_bytes(p.prec), p.stream));
  }
  if (p.sb_nop) {
    MF_CUDA(launch_sb_mix(p, p.d_xc, p.d_sb_xo, nbr, p.sb_rows));
    if (herm)
      MF_CUDA(launch_rows_herm(p, p.d_sb_xo, p.sb_rows * nbr, p.d_part, nbr, p.sb_nop, p.d_sb_seeds));
    else
      MF_CUDA(launch_sb_rows(p, p.d_sb_xo, p.sb_rows * nbr, p.d_part, nbr));
  } else if (p.prec == MF_PREC_BF16X2 && use_tch(p, tc_nvec_bucket(nvec)))
    MF_CUDA(launch_tch_apply(p, p.d_xc, p.d_part, p.d_tcb, tc_nvec_bucket(nvec)));
  else if (p.prec == MF_PREC_BF16X2)
    MF_CUDA(launch_tc_apply(p, p.d_xc, p.d_part, p.d_tcb, tc_nvec_bucket(nvec)));
  else if (tile2)
    MF_CUDA(launch_gue_apply(p, p.d_xc, p.d_part, 2));
  else if (nvec > 1 && herm)
    MF_CUDA(launch_rows_herm(p, p.d_xc, 0, p.d_part, nbr, 1, nullptr));
  else if (use_dvr_mv(p, nvec))
    MF_CUDA(launch_dvr_mv(p, p.d_xc, p.d_part, dvr_mv_bucket(nvec)));
  else if (nvec > 1 || p.sliced)
    MF_CUDA(launch_rows_apply(p, p.d_xc, p.d_part, nbr));
  else if (p.use_dvr_window)
    MF_CUDA(launch_dvr_apply(p, p.d_xc, p.d_part, 1));
  else
    MF_CUDA(launch_gue_apply(p, p.d_xc, p.d_part, 1));
  if (p.profiling) {
    MF_CUDA(cudaEventRecord(p.ev[p.ev_used].second, p.stream));
    ++p.ev_used;
  }
  return MF_OK;
}

// One product y = H x on device vectors; x FP64 [D][nvec].
mf_status apply_internal(Plan& p, double2* y, const double2* x, int64_t nvec) {
  mf_status st = ensure_workspace(p, nvec);
  if (st != MF_OK) return st;
  const VecShape sh = shape_for(p, nvec);
  MF_CUDA(launch_to_compute(p, x, p.d_xc, p.D, sh));
  if ((st = apply_kernel(p, nvec)) != MF_OK) return st;
  MF_CUDA(launch_reduce(p, p.d_part, x, y, sh));
  return MF_OK;
}

// Eigenvalue extremes of the symmetric tridiagonal (alpha, beta) by Sturm
// bisection (count of eigenvalues below s from the LDL^T pivots).
int sturm_count(const std::vector<double>& a, const std::vector<double>& b, double s) {
  int cnt = 0;
  double d = 1.0;
  for (size_t i = 0; i < a.size(); ++i) {
    const double bb = i ? b[i - 1] * b[i - 1] : 0.0;
    d = (a[i] - s) - (i ? bb / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0) ++cnt;
  }
  return cnt;
}

double tridiag_eig(const std::vector<double>& a, const std::vector<double>& b, int k) {
  double lo = 1e300, hi = -1e300;
  for (size_t i = 0; i < a.size(); ++i) {
    const double r = (i ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < a.size() ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count(a, b, mid) > k) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

mf_status compute_bounds(Plan& p) {
  if (p.have_bounds) return MF_OK;
  // a row slice cannot run Lanczos on its own: the caller sets the bounds
  if (p.sliced && p.gen != MF_GEN_SINC_DVR_HO) return MF_ERR_UNSUPPORTED;
  if (p.gen == MF_GEN_SINC_DVR_HO) {
    // symbol of the sinc-DVR kinetic operator is k^2/2 on |k| <= pi/dx, so
    // 0 <= T <= pi^2/(2 dx^2); 0 <= V <= L^2/2 on the grid.
    const double L = p.dvr.L;
    p.emin = 0.0;
    p.emax = M_PI * M_PI / (2.0 * p.dvr.dx2) + 0.5 * L * L;
    p.have_bounds = true;
    return MF_OK;
  }
  // one vector of the operator: [D] (plain) or [d_B][d_S] (system-bath)
  const int64_t nv = p.sb_nop ? p.sb_dS : 1;
  const int64_t n = p.D * nv;
  const int m = std::max(2, (int)std::min<int64_t>(p.opt.lanczos_m, n));
  mf_status st = ensure_workspace(p, nv);
  if (st != MF_OK) return st;
  double2 *v = p.d_q[0], *vp = p.d_q[1], *w = p.d_q[2];
  double* d_s = nullptr;
  MF_CUDA(dmalloc(&d_s, 2 * sizeof(double)));
  auto dot = [&](const double2* a, const double2* b, double* out) -> mf_status {
    MF_CUDA(launch_dot(p, a, b, n, d_s));
    MF_CUDA(cudaMemcpyAsync(out, d_s, sizeof(double), cudaMemcpyDeviceToHost, p.stream));
    MF_CUDA(cudaStreamSynchronize(p.stream));
    return MF_OK;
  };
  std::vector<double> al, be;
  double nrm2 = 0.0;
  MF_CUDA(launch_random_unit(p, v, n, p.seed ^ 0x5DEECE66Dull));
  st = dot(v, v, &nrm2);
  if (st == MF_OK) {
    MF_CUDA(launch_scale(p, v, v, 1.0 / std::sqrt(nrm2), n));
    double beta = 0.0;
    bool have_prev = false;
    for (int j = 0; j < m; ++j) {
      st = apply_internal(p, w, v, nv);
      if (st != MF_OK) break;
      double alpha = 0.0;
      if ((st = dot(v, w, &alpha)) != MF_OK) break;
      MF_CUDA(launch_axpby_lanczos(p, w, v, have_prev ? vp : nullptr, alpha, beta, n));
      double bn2 = 0.0;
      if ((st = dot(w, w, &bn2)) != MF_OK) break;
      al.push_back(alpha);
      const double bn = std::sqrt(bn2);
      if (j == m - 1 || bn < 1e-12) break;
      be.push_back(bn);
      std::swap(vp, v);  // vp <- v (old), v <- buffer to hold w/bn
      MF_CUDA(launch_scale(p, v, w, 1.0 / bn, n));
      beta = bn;
      have_prev = true;
    }
  }
  cudaFree(d_s);
  if (st != MF_OK) return st;
  if (be.size() + 1 > al.size()) be.resize(al.size() - 1);
  const double tmin = tridiag_eig(al, be, 0);
  const double tmax = tridiag_eig(al, be, (int)al.size() - 1);
  const double half = 0.5 * (tmax - tmin), pad = p.opt.bounds_pad * half;
  p.emin = tmin - pad;
  p.emax = tmax + pad;
  p.have_bounds = true;
  return MF_OK;
}

// Bessel coefficients J_k(z), k = 0..K on the device, cached per argument.
// With order == 0 the term count is the smallest n with |a_k| < tol for all
// k >= n (a_0 = J_0, a_k = 2 J_k), read back once per argument.
// kind 1 computes e^{-z} I_k(z) instead (imaginary-time filter), whose terms
// fall off past k ~ sqrt(z) rather than k ~ z: the same K bound covers them.
mf_status coefficients(Plan& p, double z, int32_t order, int32_t* nterms, int32_t kind = 0) {
  const int32_t Kmax = (int32_t)std::ceil(z) + 60 + (int32_t)(30.0 * std::cbrt(z + 1.0));
  const int32_t K = std::max(Kmax, order);
  if (p.J_arg != z || p.J_K < K || p.J_kind != kind) {
    mf_status st = ensure_J(p, K);
    if (st != MF_OK) return st;
    if (kind)
      MF_CUDA(launch_bessel_i(p, z, K, p.d_J));
    else
      MF_CUDA(launch_bessel(p, z, K, p.d_J));
    p.J_arg = z;
    p.J_K = K;
    p.J_kind = kind;
    p.J_terms = 0;
  }
  if (order > 0) {
    *nterms = order;
    return MF_OK;
  }
  if (p.J_terms == 0) {
    std::vector<double> J((size_t)p.J_K + 1);
    MF_CUDA(cudaMemcpyAsync(J.data(), p.d_J, J.size() * sizeof(double), cudaMemcpyDeviceToHost, p.stream));
    MF_CUDA(cudaStreamSynchronize(p.stream));
    int32_t last = 0;
    for (int32_t k = 0; k <= p.J_K; ++k) {
      const double a = k ? 2.0 * std::fabs(J[k]) : std::fabs(J[0]);
      if (a >= p.opt.cheb_tol) last = k;
    }
    p.J_terms = last + 1;
  }
  *nterms = p.J_terms;
  return MF_OK;
}

// Build a plan for one explicit candidate: block size b (> 0, multiple of the
// tile) and storage mode (procedural, partial or full; partial takes
// P_cache from the budget).  Arguments are validated by the caller.
// For MF_GEN_EXTERNAL, ext is the caller's host array of canonical blocks:
// the first P_cache pairs are copied into the HBM cache, the rest are read
// from the (registered) host array by the kernels.
mf_status create_fixed(mf_plan_t* out, int64_t D, int32_t generator, uint64_t seed, int64_t block,
                       size_t cache_budget_bytes, const mf_options& o, const void* ext = nullptr) {
  *out = nullptr;

  mf_plan* h = new (std::nothrow) mf_plan();
  if (!h) return MF_ERR_OOM;
  Plan& p = h->p;
  p.D = D;
  p.gen = generator;
  p.seed = seed;
  p.prec = o.precision;
  p.opt = o;
  p.stream = (cudaStream_t)o.stream;
  p.device = o.device;
  DeviceGuard guard(p.device);
  auto fail = [&](mf_status s) {
    release(p);
    delete h;
    return s;
  };
  if (cudaSetDevice(p.device) != cudaSuccess) return fail(MF_ERR_CUDA);
  if (cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, p.device) != cudaSuccess)
    return fail(MF_ERR_CUDA);
  size_t mfree = 0, mtotal = 0;
  if (cudaMemGetInfo(&mfree, &mtotal) != cudaSuccess) return fail(MF_ERR_CUDA);

  // generator constants
  p.sigma64 = std::sqrt(0.5 / (double)D);
  p.sigma32 = sqrtf(0.5f / (float)D);
  dvr_setup(p.dvr, D, o.dvr_L);
  // the tensor-core kernels are the ones with bounded waits
  p.has_waits = p.prec == MF_PREC_BF16X2;
  p.spin = o.spin_limit > 0 ? (uint32_t)o.spin_limit : kDefaultSpin;

  // partition (Sec. II / IV.F): b multiple of the tile, at most D rounded up
  const int64_t Dt = (D + kTile - 1) / kTile * kTile;
  p.b = std::min(block, Dt);
  p.nblk = (D + p.b - 1) / p.b;
  p.npair = p.nblk * (p.nblk + 1) / 2;
  p.ntile = (D + kTile - 1) / kTile;
  // row-distributed plan: the pairs its rows touch (block row n or block
  // column m among its blocks) are the ones it may cache
  p.sliced = o.row_end > 0;
  int64_t nb0 = 0, nb1 = p.nblk, npair_use = p.npair;
  if (p.sliced) {
    p.row0 = o.row_begin;
    p.row1 = o.row_end;
    p.slice_t0 = p.row0 / kTile;
    p.slice_nt = (p.row1 + kTile - 1) / kTile - p.slice_t0;
    nb0 = p.row0 / p.b;
    nb1 = (p.row1 + p.b - 1) / p.b;
    npair_use = 0;
    for (int64_t n = 0; n < p.nblk; ++n)
      for (int64_t m = n; m < p.nblk; ++m) npair_use += ((n >= nb0 && n < nb1) || (m >= nb0 && m < nb1)) ? 1 : 0;
  }

  // storage (Sec. III.A, IV.G): P_cache = min(N_pair, floor(M_cache / (B_c b^2)))
  const size_t eb = compute_elem_bytes(p.prec);
  size_t budget = cache_budget_bytes;
  if (budget == SIZE_MAX) budget = (size_t)(o.f_cache * (double)mfree);
  const double blk_bytes = (double)eb * (double)p.b * (double)p.b;
  int64_t pc = (int64_t)std::min<double>((double)npair_use, std::floor((double)budget / blk_bytes));
  int32_t storage = o.storage;
  if (storage == MF_STORE_PROCEDURAL && generator != MF_GEN_EXTERNAL) {
    pc = 0;
  } else if (storage == MF_STORE_FULL) {
    if (pc < npair_use) return fail(MF_ERR_OOM);
  }
  if (pc == npair_use) storage = MF_STORE_FULL;
  else if (generator == MF_GEN_EXTERNAL) storage = MF_STORE_PARTIAL;  // the rest stays in host memory
  else if (pc == 0) storage = MF_STORE_PROCEDURAL;
  p.storage = storage;
  p.pairs_cached = pc;
  p.cache_budget = budget;

  // memory feasibility (Eq. planner_memory_constraint): M_op + M_work <= alpha M_free
  const int64_t nv = std::max(1, o.nvec_hint);
  p.use_dvr_window = generator == MF_GEN_SINC_DVR_HO && pc == 0 && p.prec != MF_PREC_BF16X2 && !p.sliced;
  if (p.use_dvr_window && p.prec == MF_PREC_FP32) {
    dvr_fp32_window_shape(p);
  } else if (p.use_dvr_window) {
    const int P = 8;
    p.dvr_rows = 32 * P;
    const int64_t rtiles = (D + p.dvr_rows - 1) / p.dvr_rows;
    int kc = 4096;
    while (kc > 128 && rtiles * ((D + kc - 1) / kc) < 8 * (int64_t)p.num_sms) kc /= 2;
    p.dvr_cols = kc;
    p.nslot = (D + kc - 1) / kc;
    p.dpad = rtiles * p.dvr_rows;
  } else {
    p.nslot = p.ntile;
    p.dpad = p.ntile * kTile;
  }
  // multi-vector row-owner path: enough (row tile, column range) CTAs for
  // two waves, column ranges a multiple of the 32-column chunk and at most
  // kMaxSplitCols long, so that no FP32 partial sum runs over more terms
  // (the sums across ranges are FP64; at D = 262144 with 64 vectors one
  // FP32 chain over the whole row left 2.4e-5 of max|y| against the FP32
  // form's exact sums)
  {
    constexpr int64_t kMaxSplitCols = 16384;
    int64_t ns = std::max<int64_t>(1, std::min<int64_t>(64, (2 * (int64_t)p.num_sms + p.ntile - 1) / p.ntile));
    ns = std::max<int64_t>(ns, (D + kMaxSplitCols - 1) / kMaxSplitCols);
    int64_t cols = ((D + ns - 1) / ns + 31) / 32 * 32;
    p.rows_split_cols = cols;
    p.rows_nsplit = (D + cols - 1) / cols;
  }
  const int64_t nbk = p.prec == MF_PREC_BF16X2 ? tc_nvec_bucket(nv) : (nv > 1 ? rows_nvec_bucket(nv) : 1);
  // Hermitian tensor-core walk: Philox BF16X2 plans over all rows
  std::vector<int2> tch_units;
  std::vector<int64_t> tch_off;
  if (p.prec == MF_PREC_BF16X2 && generator == MF_GEN_PHILOX_GUE && !p.sliced && o.hermitian_reuse != 0) {
    p.tch_rows = tch_layout(p.ntile, p.num_sms, &p.tch_s, &p.tch_U, tch_units, tch_off);
    p.tch_nunits = (int64_t)tch_units.size();
    // the unit slots for the largest vector bucket must fit beside the cache
    const double room = std::max(0.0, (double)mfree - (double)pc * blk_bytes);
    p.tch_limit = std::min(24e9, 0.15 * room);
    p.tch = (double)p.tch_rows * 2.0 * 64.0 * 4.0 <= p.tch_limit;
  }
  const double part_b = (nv > 1 || p.prec == MF_PREC_BF16X2) ? std::max((double)p.nslot * p.dpad, (double)p.rows_nsplit * p.ntile * kTile * nbk)
                               : (double)p.nslot * p.dpad;
  const double m_tch = p.tch ? (double)p.tch_rows * 2.0 * (double)nbk * 4.0 + (double)tch_operand_bytes(D, nbk) : 0.0;
  const double m_work =
      part_b * eb + 3.0 * D * nv * 16.0 + (double)std::max(p.dpad, p.ntile * kTile) * nbk * eb + m_tch;
  p.m_work = m_work;
  const double m_op = (double)pc * blk_bytes;
  if (m_op + m_work > o.alpha_safety * (double)mfree) {
    if (o.storage == MF_STORE_FULL || (o.storage == MF_STORE_PARTIAL && generator != MF_GEN_EXTERNAL))
      return fail(MF_ERR_OOM);
    // shrink the cache until the plan fits
    const double room = o.alpha_safety * (double)mfree - m_work;
    pc = room > 0 ? (int64_t)std::floor(room / blk_bytes) : 0;
    pc = std::min(pc, npair_use);
    p.pairs_cached = pc;
    p.storage = pc == npair_use ? MF_STORE_FULL
                : (pc == 0 && generator != MF_GEN_EXTERNAL ? MF_STORE_PROCEDURAL : MF_STORE_PARTIAL);
    if (m_work > o.alpha_safety * (double)mfree) return fail(MF_ERR_OOM);
  }

  // dense-work safety estimate (Sec. IV.H): W_Hpsi ~ D^2 entries
  p.w_hpsi = (double)D * (double)D;
  p.dense_warn = p.w_hpsi > o.dense_work_limit;

  if (dmalloc(&p.d_err, sizeof(int)) != cudaSuccess) return fail(MF_ERR_OOM);
  if (cudaMemsetAsync(p.d_err, 0, sizeof(int), p.stream) != cudaSuccess) return fail(MF_ERR_CUDA);
  if (dmalloc(&p.d_red, kRedDoubles * sizeof(double)) != cudaSuccess) return fail(MF_ERR_OOM);
  if (p.has_waits) {
    if (cudaHostAlloc((void**)&p.h_err, sizeof(int), cudaHostAllocDefault) != cudaSuccess) return fail(MF_ERR_OOM);
    *p.h_err = 0;
    if (cudaEventCreateWithFlags(&p.err_ev, cudaEventDisableTiming) != cudaSuccess) return fail(MF_ERR_CUDA);
  }

  // cache: the first P_cache canonical pairs in row order
  p.pair_slot.assign((size_t)(p.nblk * p.nblk), -1);
  std::vector<int2> pairs;
  for (int64_t n = 0, s = 0; n < p.nblk && s < p.pairs_cached; ++n)
    for (int64_t m = n; m < p.nblk && s < p.pairs_cached; ++m) {
      if (!((n >= nb0 && n < nb1) || (m >= nb0 && m < nb1))) continue;
      p.pair_slot[(size_t)(n * p.nblk + m)] = s++;
      pairs.push_back(make_int2((int)n, (int)m));
    }
  if (generator == MF_GEN_EXTERNAL) {
    // pairs past P_cache stay in the caller's host array: slot -2 - k for
    // the k-th stored pair
    int64_t k = 0;
    for (int64_t n = 0; n < p.nblk; ++n)
      for (int64_t m = n; m < p.nblk; ++m, ++k)
        if (k >= p.pairs_cached) p.pair_slot[(size_t)(n * p.nblk + m)] = -2 - k;
    if (p.pairs_cached < p.npair) {
      const size_t bytes = (size_t)p.npair * (size_t)blk_bytes;
      void* hp = const_cast<void*>(ext);
      cudaError_t e = cudaHostRegister(hp, bytes, cudaHostRegisterMapped);
      if (e == cudaSuccess) {
        p.h_registered = true;
      } else if (e == cudaErrorHostMemoryAlreadyRegistered) {
        cudaGetLastError();
      } else {
        cudaGetLastError();
        return fail(MF_ERR_CUDA);
      }
      p.h_blocks = ext;
      void* dp = nullptr;
      if (cudaHostGetDevicePointer(&dp, hp, 0) != cudaSuccess) return fail(MF_ERR_CUDA);
      p.d_hblocks = dp;
    }
  }
  if (p.pairs_cached > 0) {
    p.cache_bytes = (size_t)p.pairs_cached * (size_t)blk_bytes;
    cudaError_t e = dev_malloc(&p.d_cache, p.cache_bytes);
    if (e != cudaSuccess) return fail(MF_ERR_OOM);
  }
  if (p.pairs_cached > 0 && generator == MF_GEN_EXTERNAL) {
    // the cached pairs are the first P_cache stored blocks: one copy
    if (cudaMemcpy(p.d_cache, ext, p.cache_bytes, cudaMemcpyHostToDevice) != cudaSuccess) return fail(MF_ERR_CUDA);
  } else if (p.pairs_cached > 0) {
    cudaError_t e;
    int2* d_pairs = nullptr;
    if (dmalloc(&d_pairs, pairs.size() * sizeof(int2)) != cudaSuccess) return fail(MF_ERR_OOM);
    cudaMemcpyAsync(d_pairs, pairs.data(), pairs.size() * sizeof(int2), cudaMemcpyHostToDevice, p.stream);
    e = p.tch ? launch_tch_cache_fill(p, d_pairs, (int64_t)pairs.size())
              : launch_cache_fill_pairs(p, d_pairs, (int64_t)pairs.size());
    cudaStreamSynchronize(p.stream);
    cudaFree(d_pairs);
    if (e != cudaSuccess) return fail(MF_ERR_CUDA);
  }

  // work list of canonical tiles, cached and procedural items interleaved so
  // HBM streaming and generation overlap on the SMs (Eq. runtime_overlap)
  if (!p.use_dvr_window && !p.sliced) {
    std::vector<WorkItem> cached, proc;
    const int64_t tpb = p.b / kTile;
    for (int64_t ti = 0; ti < p.ntile; ++ti)
      for (int64_t tj = ti; tj < p.ntile; ++tj) {
        const int64_t n = ti / tpb, m = tj / tpb;
        const int64_t slot = p.pair_slot[(size_t)(n * p.nblk + m)];
        WorkItem it{(int32_t)ti, (int32_t)tj, -1};
        const int64_t in_blk = (ti * kTile - n * p.b) * p.b + (tj * kTile - m * p.b);
        if (slot >= 0) {
          it.cache_off = slot * p.b * p.b + in_blk;
          cached.push_back(it);
        } else {
          // generated, or read from the external host array (block -2 - slot)
          if (slot <= -2) it.cache_off = -2 - ((-2 - slot) * p.b * p.b + in_blk);
          proc.push_back(it);
        }
      }
    std::vector<WorkItem> work;
    work.reserve(cached.size() + proc.size());
    size_t ic = 0, ip = 0;
    while (ic < cached.size() || ip < proc.size()) {
      // take from the list that is behind its share
      const bool take_c = ip >= proc.size() ||
                          (ic < cached.size() && (double)ic * proc.size() <= (double)ip * cached.size());
      work.push_back(take_c ? cached[ic++] : proc[ip++]);
    }
    p.nwork = (int64_t)work.size();
    if (dmalloc(&p.d_work, work.size() * sizeof(WorkItem)) != cudaSuccess) return fail(MF_ERR_OOM);
    if (cudaMemcpyAsync(p.d_work, work.data(), work.size() * sizeof(WorkItem), cudaMemcpyHostToDevice,
                        p.stream) != cudaSuccess)
      return fail(MF_ERR_CUDA);
  }
  if (!p.use_dvr_window && !p.sliced && generator != MF_GEN_SINC_DVR_HO && p.prec != MF_PREC_BF16X2) {
    // measured after the cache is allocated, so the slots never crowd it out
    size_t mfree_now = 0, mtotal_now = 0;
    if (cudaMemGetInfo(&mfree_now, &mtotal_now) != cudaSuccess) return fail(MF_ERR_CUDA);
    p.herm_limit = std::min(16e9, 0.1 * (double)mfree_now);
    const std::vector<HermItem> hi = rows_herm_items(D, p.num_sms, &p.herm_ns);
    p.herm_nitems = (int64_t)hi.size();
    if (dmalloc(&p.d_herm_items, hi.size() * sizeof(HermItem)) != cudaSuccess) return fail(MF_ERR_OOM);
    if (cudaMemcpyAsync(p.d_herm_items, hi.data(), hi.size() * sizeof(HermItem), cudaMemcpyHostToDevice,
                        p.stream) != cudaSuccess)
      return fail(MF_ERR_CUDA);
  }
  if (p.tch) {
    if (dmalloc(&p.d_tch_units, tch_units.size() * sizeof(int2)) != cudaSuccess ||
        dmalloc(&p.d_tch_off, tch_off.size() * sizeof(int64_t)) != cudaSuccess ||
        dmalloc(&p.d_tch_counter, sizeof(int)) != cudaSuccess)
      return fail(MF_ERR_OOM);
    if (cudaMemcpyAsync(p.d_tch_units, tch_units.data(), tch_units.size() * sizeof(int2), cudaMemcpyHostToDevice,
                        p.stream) != cudaSuccess ||
        cudaMemcpyAsync(p.d_tch_off, tch_off.data(), tch_off.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                        p.stream) != cudaSuccess)
      return fail(MF_ERR_CUDA);
  }
  if (p.pairs_cached > 0 || generator == MF_GEN_EXTERNAL) {
    const size_t nb = p.pair_slot.size() * sizeof(int64_t);
    if (dmalloc(&p.d_pair_slot, nb) != cudaSuccess) return fail(MF_ERR_OOM);
    if (cudaMemcpyAsync(p.d_pair_slot, p.pair_slot.data(), nb, cudaMemcpyHostToDevice, p.stream) != cudaSuccess)
      return fail(MF_ERR_CUDA);
  }
  mf_status st = ensure_workspace(p, nv);
  if (st != MF_OK) return fail(st);
  if (cudaStreamSynchronize(p.stream) != cudaSuccess) return fail(MF_ERR_CUDA);
  *out = h;
  return p.dense_warn ? MF_WARN_DENSE_WORK : MF_OK;
}


const char* gen_name(int g) {
  return g == MF_GEN_PHILOX_GUE ? "philox_gue" : (g == MF_GEN_SINC_DVR_HO ? "sinc_dvr_ho" : "external");
}
const char* prec_name(int g) { return g == MF_PREC_FP64 ? "fp64" : (g == MF_PREC_FP32 ? "fp32" : "bf16x2"); }
const char* store_name(int s) {
  return s == MF_STORE_FULL ? "full" : (s == MF_STORE_PARTIAL ? "partial" : "procedural");
}

}  // namespace

namespace mf {
mf_status plan_workspace(Plan& p, int64_t nvec) { return ensure_workspace(p, nvec); }
mf_status plan_bounds(Plan& p) { return compute_bounds(p); }
mf_status plan_coefficients(Plan& p, double z, int32_t order, int32_t* nterms, int32_t kind) {
  return coefficients(p, z, order, nterms, kind);
}
}  // namespace mf

namespace {

// Measured time of one application (Eq. measured_matvec_time): R_warm
// untimed applies, then the mean of R_bench applies each bracketed by CUDA
// events on the plan's stream (synchronised before and after).
mf_status measure_plan(Plan& p, int64_t nvec, int warm, int reps, double* t_mean) {
  double2 *x = nullptr, *y = nullptr;
  const size_t bytes = (size_t)p.D * (size_t)nvec * sizeof(double2);
  if (dmalloc(&x, bytes) != cudaSuccess) return MF_ERR_OOM;
  if (dmalloc(&y, bytes) != cudaSuccess) {
    cudaFree(x);
    return MF_ERR_OOM;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  mf_status st = MF_OK;
  double tot = 0.0;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) st = MF_ERR_CUDA;
  if (st == MF_OK && launch_random_unit(p, x, p.D * nvec, p.seed + 17) != cudaSuccess) st = MF_ERR_CUDA;
  for (int i = 0; st == MF_OK && i < warm; ++i) st = apply_internal(p, y, x, nvec);
  if (st == MF_OK && cudaStreamSynchronize(p.stream) != cudaSuccess) st = MF_ERR_CUDA;
  for (int i = 0; st == MF_OK && i < reps; ++i) {
    cudaEventRecord(a, p.stream);
    st = apply_internal(p, y, x, nvec);
    cudaEventRecord(b, p.stream);
    float ms = 0.f;
    if (st == MF_OK && (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess))
      st = MF_ERR_CUDA;
    tot += ms * 1e-3;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(x);
  cudaFree(y);
  if (st == MF_OK) *t_mean = tot / std::max(1, reps);
  return st;
}

// Device throughputs assumed by Algorithm 1 before any measurement: FMA
// pipe rate of the precision, measured-class HBM rate, and per-generator
// entry rates (the DVR window makes generation nearly free).
// Throughputs of the runtime model (Eq. runtime_overlap), measured on GB300:
// the FP32 pipe at 1.9 GHz, 6.7 TB/s of HBM streaming, the Philox
// one-vector canonical-entry rate of the FP32 generator (2.7e11/s; the
// BF16X2 form generates the same FP32 entries), the DVR window table (next
// to free), and for BF16X2 the BF16 tensor rate (1977 TFLOP/s, measured
// cuBLAS burst) over its three split products.  (An earlier model with
// 4e11/s Philox generation and the FP32 rate for BF16X2 picked plans up to
// 2x slower than the best for Philox with 16 and 64 vectors.)
mf_device_model device_model(int prec, int gen, int num_sms) {
  mf_device_model m{};
  const double clk = 1.9e9;
  m.flops_per_s = prec == MF_PREC_FP64 ? 1.2e12 : (double)num_sms * 128.0 * 2.0 * clk;
  if (prec == MF_PREC_BF16X2) m.flops_per_s = 1977e12 / 3.0;
  m.hbm_bytes_per_s = 6.7e12;
  if (gen == MF_GEN_SINC_DVR_HO) m.gen_entries_per_s = 1e15;
  else m.gen_entries_per_s = prec == MF_PREC_FP64 ? 1.5e10 : 2.7e11;
  return m;
}

std::string trial_json(const Plan& p, const mf_problem& pr, const mf_candidate& c, const mf_estimate& e,
                       double t_mv, double budget, double gpu_mem) {
  const char* sn = store_name(c.storage);
  const double lg = 1.0 / std::log(10.0);
  char buf[2048];
  std::snprintf(buf, sizeof(buf),
                "{\"generator\": \"%s\", \"precision\": \"%s\", \"D\": %lld, \"R\": %lld, \"block\": %lld, "
                "\"storage\": \"%s\", \"pairs_cached\": %lld, \"n_pair\": %lld, \"budget_bytes\": %.6g, "
                "\"t_mv\": %.9g, \"T_model\": %.9g, \"S_model\": %.9g, \"M_work\": %.6g, \"M_op\": %.6g, "
                "\"M_tot\": %.6g, \"M_free\": %.6g, \"F_mv\": %.6g, \"waves\": %lld, \"sms\": %d, "
                "\"features\": [%.6g, %.6g, %.6g, %.6g, %.6g, %.6g, %d, %lld, %d, %d, %d, 1, 0, 0, %.6g, %.6g, %.6g, "
                "%.6g, %.6g, %d]}",
                gen_name(p.gen), prec_name(p.prec), (long long)pr.D_in, (long long)pr.R, (long long)c.block, sn,
                (long long)e.pairs_cached, (long long)e.n_pair, budget, t_mv, e.T_model, e.S_model, e.M_work,
                e.M_op, e.M_tot, pr.M_free, e.F_mv, (long long)e.waves, p.num_sms, std::log((double)pr.D_in) * lg,
                std::log((double)pr.D_out) * lg, std::log((double)pr.R) * lg, std::log((double)e.n_blk) * lg,
                std::log((double)c.block) * lg, std::log((double)pr.N_task) * lg, c.p_row, (long long)e.waves,
                c.storage == MF_STORE_FULL, c.storage == MF_STORE_PARTIAL, c.storage == MF_STORE_PROCEDURAL,
                std::log(e.F_mv) * lg, e.M_op / pr.M_free, e.M_work / pr.M_free, e.M_tot / pr.M_free,
                gpu_mem / 1e9, p.num_sms);
  return std::string(buf);
}

}  // namespace

extern "C" {

mf_status mf_planner_device_model(int32_t precision, int32_t generator, int32_t num_sms, mf_device_model* out) {
  if (!out || num_sms < 1 || precision < MF_PREC_FP64 || precision > MF_PREC_BF16X2 ||
      generator < MF_GEN_PHILOX_GUE || generator > MF_GEN_SINC_DVR_HO)
    return MF_ERR_INVALID;
  *out = device_model(precision, generator, num_sms);
  return MF_OK;
}

void mf_options_default(mf_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = MF_PREC_FP32;
  o->storage = MF_STORE_AUTO;
  o->planner_mode = MF_PLANNER_ANALYTIC;
  o->nvec_hint = 1;
  o->cheb_tol = 1e-7;
  o->lanczos_m = 40;
  o->bounds_pad = 0.05;
  o->dvr_L = 0.0;
  o->stream = nullptr;
  o->alpha_safety = 0.9;
  o->f_cache = 0.8;
  o->autotune_k = 8;
  o->autotune_warmup = 1;
  o->autotune_repeats = 3;
  o->dense_work_limit = 1e13;
  o->device = 0;
  o->model = nullptr;
  o->hermitian_reuse = -1;
  o->row_begin = 0;
  o->row_end = 0;
  o->spin_limit = 0;
}

const char* mf_status_string(mf_status s) {
  switch (s) {
    case MF_OK: return "MF_OK";
    case MF_ERR_INVALID: return "MF_ERR_INVALID";
    case MF_ERR_OOM: return "MF_ERR_OOM";
    case MF_ERR_CUDA: return "MF_ERR_CUDA";
    case MF_ERR_UNSUPPORTED: return "MF_ERR_UNSUPPORTED";
    case MF_ERR_TIMEOUT: return "MF_ERR_TIMEOUT";
    case MF_WARN_DENSE_WORK: return "MF_WARN_DENSE_WORK";
  }
  return "MF_STATUS_UNKNOWN";
}

mf_status mf_plan_create(mf_plan_t* out, int64_t D, int64_t M, int32_t generator, uint64_t seed, int64_t block,
                         size_t cache_budget_bytes, const mf_options* opt) {
  return guard([&]() -> mf_status {
    if (!out) return MF_ERR_INVALID;
    *out = nullptr;
    mf_options o;
    if (opt) o = *opt; else mf_options_default(&o);
    if (D < 2 || M != D || D > (int64_t)1 << 31) return MF_ERR_INVALID;
    if (generator != MF_GEN_PHILOX_GUE && generator != MF_GEN_SINC_DVR_HO) return MF_ERR_INVALID;
    if (o.precision != MF_PREC_FP64 && o.precision != MF_PREC_FP32 && o.precision != MF_PREC_BF16X2)
      return MF_ERR_INVALID;
    if (block < 0 || (block > 0 && block % kTile != 0)) return MF_ERR_INVALID;
    // the FP32 steps of the DVR generator square an exact float(i - j)
    if (generator == MF_GEN_SINC_DVR_HO && o.precision != MF_PREC_FP64 && D > ((int64_t)1 << 24)) return MF_ERR_INVALID;
    if (o.storage < MF_STORE_AUTO || o.storage > MF_STORE_FULL) return MF_ERR_INVALID;
    if (o.planner_mode < MF_PLANNER_ANALYTIC || o.planner_mode > MF_PLANNER_HYBRID) return MF_ERR_INVALID;
    if (!(o.cheb_tol > 0) || o.lanczos_m < 2 || !(o.alpha_safety > 0 && o.alpha_safety <= 1)) return MF_ERR_INVALID;
    if (o.nvec_hint < 1 || o.nvec_hint > 64 || o.autotune_k < 1 || o.autotune_repeats < 1 || o.autotune_warmup < 0)
      return MF_ERR_INVALID;
    if (o.hermitian_reuse < -1 || o.hermitian_reuse > 1) return MF_ERR_INVALID;
    if (!(o.dvr_L >= 0.0) || !std::isfinite(o.dvr_L) || o.spin_limit < 0) return MF_ERR_INVALID;
    if ((o.planner_mode == MF_PLANNER_LEARNED || o.planner_mode == MF_PLANNER_HYBRID) && !o.model)
      return MF_ERR_INVALID;

    // row-distributed plan: one explicit candidate on the slice's rows
    if (o.row_begin != 0 || o.row_end != 0) {
      if (o.row_begin < 0 || o.row_end <= o.row_begin || o.row_end > D || o.row_begin % kTile != 0 ||
          (o.row_end % kTile != 0 && o.row_end != D))
        return MF_ERR_INVALID;
      if (o.precision == MF_PREC_BF16X2) return MF_ERR_UNSUPPORTED;
      const int64_t Dt = (D + kTile - 1) / kTile * kTile;
      const int64_t b = block > 0 ? block : std::min<int64_t>(2048, Dt);
      mf_options os = o;
      if (os.storage == MF_STORE_AUTO) os.storage = cache_budget_bytes > 0 ? MF_STORE_PARTIAL : MF_STORE_PROCEDURAL;
      os.planner_mode = MF_PLANNER_ANALYTIC;
      return create_fixed(out, D, generator, seed, b, cache_budget_bytes, os);
    }

    // one explicit candidate: no planning
    if (block > 0 && o.storage != MF_STORE_AUTO && o.planner_mode == MF_PLANNER_ANALYTIC)
      return create_fixed(out, D, generator, seed, block, cache_budget_bytes, o);

    DeviceGuard guard(o.device);
    if (cudaSetDevice(o.device) != cudaSuccess) return MF_ERR_CUDA;
    int num_sms = 0;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, o.device) != cudaSuccess) return MF_ERR_CUDA;
    size_t mfree = 0, mtotal = 0;
    if (cudaMemGetInfo(&mfree, &mtotal) != cudaSuccess) return MF_ERR_CUDA;
    const double budget = cache_budget_bytes == SIZE_MAX ? o.f_cache * (double)mfree : (double)cache_budget_bytes;
    const size_t eb = compute_elem_bytes(o.precision);

    // candidate block sizes (Sec. IV.F) and storage modes (Sec. IV.G)
    const int64_t Dt = (D + kTile - 1) / kTile * kTile;
    std::vector<int64_t> blocks;
    if (block > 0) blocks.push_back(std::min(block, Dt));
    else
      for (int64_t b = 256; b <= 4096; b *= 2)
        if (b <= Dt) blocks.push_back(b);
    if (blocks.empty()) blocks.push_back(Dt);
    std::vector<int32_t> stores;
    if (o.storage != MF_STORE_AUTO) stores.push_back(o.storage);
    else stores = {MF_STORE_PROCEDURAL, MF_STORE_PARTIAL, MF_STORE_FULL};

    mf_problem pr{D, D, o.nvec_hint, 1, 1, (double)eb, (double)mfree, 1};
    const mf_device_model dm = device_model(o.precision, generator, num_sms);
    struct Ranked {
      mf_candidate c;
      mf_estimate e;
    };
    std::vector<Ranked> ranked;
    for (int64_t b : blocks)
      for (int32_t st : stores) {
        mf_candidate c{b, st, -1, 1, 1, 4};
        mf_estimate e{};
        planner_estimate(pr, c, dm, o.alpha_safety, budget, e);
        if (st == MF_STORE_PARTIAL && (e.pairs_cached == 0 || e.pairs_cached == e.n_pair)) continue;
        if (st == MF_STORE_FULL && (double)e.n_pair * e.M_block > budget) continue;
        if (!e.feasible && st != MF_STORE_PROCEDURAL) continue;
        ranked.push_back({c, e});
      }
    if (ranked.empty()) return MF_ERR_OOM;
    // model score first; where the same term bounds two candidates (equal
    // scores), the one with less total work (fewer generated or streamed
    // entries competing with the contraction for the SMs)
    std::stable_sort(ranked.begin(), ranked.end(), [](const Ranked& a, const Ranked& b) {
      return a.e.S_model < b.e.S_model || (a.e.S_model == b.e.S_model && a.e.T_sum < b.e.T_sum);
    });

    auto budget_for = [&](const Ranked& r) -> size_t {
      if (r.c.storage == MF_STORE_PROCEDURAL) return 0;
      return (size_t)((double)r.e.pairs_cached * r.e.M_block);
    };
    auto build = [&](const Ranked& r, mf_plan_t* h) {
      if (fault_hit("plan")) return MF_ERR_OOM;  // injected: this candidate fails to build
      mf_options oc = o;
      oc.storage = r.c.storage;
      return create_fixed(h, D, generator, seed, r.c.block, budget_for(r), oc);
    };

    if (o.planner_mode == MF_PLANNER_ANALYTIC) {
      mf_status st = MF_ERR_OOM;
      for (const Ranked& r : ranked) {  // best feasible by the model
        st = build(r, out);
        if (st == MF_OK || st == MF_WARN_DENSE_WORK) {
          (*out)->p.s_model = r.e.S_model;
          (*out)->p.trials.push_back(trial_json((*out)->p, pr, r.c, r.e, -1.0, budget, (double)mtotal));
          return st;
        }
      }
      return st;
    }

    // Algorithm 2: measure the K_bench best candidates, keep the fastest job
    // score S_bench = W t_mv (Eq. bench_score, Eq. bench_argmin); Algorithm 3
    // (learned/hybrid) reorders the candidates by the surrogate first.
    if (o.planner_mode == MF_PLANNER_LEARNED || o.planner_mode == MF_PLANNER_HYBRID) {
      std::vector<double> pred(ranked.size(), 0.0);
      for (size_t i = 0; i < ranked.size(); ++i) {
        double t = 0.0;
        mf_status st = surrogate_predict(o.model, generator, o.precision, pr, ranked[i].c, ranked[i].e, budget,
                                         (double)mtotal, num_sms, &t);
        if (st != MF_OK) return st;
        pred[i] = t * (double)ranked[i].e.waves;
      }
      std::vector<size_t> idx(ranked.size());
      for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
      std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return pred[a] < pred[b]; });
      std::vector<Ranked> re;
      for (size_t i : idx) re.push_back(ranked[i]);
      ranked.swap(re);
      if (o.planner_mode == MF_PLANNER_LEARNED) {
        mf_status st = MF_ERR_OOM;
        for (const Ranked& r : ranked) {
          st = build(r, out);
          if (st == MF_OK || st == MF_WARN_DENSE_WORK) {
            (*out)->p.planner_used = MF_PLANNER_LEARNED;
            (*out)->p.s_model = r.e.S_model;
            return st;
          }
        }
        return st;
      }
    }
    const size_t K = std::min<size_t>((size_t)o.autotune_k, ranked.size());
    mf_plan_t best = nullptr;
    mf_status best_st = MF_ERR_OOM;
    double best_score = 1e300;
    std::vector<std::string> log;
    for (size_t i = 0; i < K; ++i) {
      mf_plan_t h = nullptr;
      mf_status st = build(ranked[i], &h);
      if (st != MF_OK && st != MF_WARN_DENSE_WORK) continue;
      double t = 0.0;
      mf_status ms = measure_plan(h->p, o.nvec_hint, o.autotune_warmup, o.autotune_repeats, &t);
      if (ms != MF_OK) {
        mf_plan_destroy(h);
        if (ms == MF_ERR_CUDA) return ms;
        continue;
      }
      log.push_back(trial_json(h->p, pr, ranked[i].c, ranked[i].e, t, budget, (double)mtotal));
      const double score = (double)ranked[i].e.waves * t;
      if (score < best_score) {
        if (best) mf_plan_destroy(best);
        best = h;
        best_st = st;
        best_score = score;
        best->p.s_model = ranked[i].e.S_model;
        best->p.t_measured = t;
      } else {
        mf_plan_destroy(h);
      }
    }
    if (!best) return MF_ERR_OOM;
    best->p.trials = log;
    best->p.planner_used = o.planner_mode;
    *out = best;
    return best_st;
  });
}

mf_status mf_plan_trials(mf_plan_t h, char* buf, size_t len, size_t* needed) {
  return guard([&]() -> mf_status {
    if (!h) return MF_ERR_INVALID;
    std::string all;
    for (const auto& t : h->p.trials) {
      all += t;
      all += "\n";
    }
    if (needed) *needed = all.size() + 1;
    if (!buf) return MF_OK;
    if (len == 0) return MF_ERR_INVALID;
    std::strncpy(buf, all.c_str(), len - 1);
    buf[len - 1] = '\0';
    return all.size() + 1 <= len ? MF_OK : MF_ERR_INVALID;
  });
}

mf_status mf_external_create(mf_plan_t* out, int64_t D, int64_t block, const void* blocks,
                             size_t cache_budget_bytes, const mf_options* opt) {
  return guard([&]() -> mf_status {
    if (!out) return MF_ERR_INVALID;
    *out = nullptr;
    mf_options o;
    if (opt) o = *opt; else mf_options_default(&o);
    if (D < 2 || D > (int64_t)1 << 31 || !blocks || block < kTile || block % kTile != 0) return MF_ERR_INVALID;
    if ((uintptr_t)blocks % 16 != 0) return MF_ERR_INVALID;  // the kernels read 16-byte words
    if (o.precision != MF_PREC_FP64 && o.precision != MF_PREC_FP32 && o.precision != MF_PREC_BF16X2)
      return MF_ERR_INVALID;
    if (!(o.cheb_tol > 0) || o.lanczos_m < 2 || !(o.alpha_safety > 0 && o.alpha_safety <= 1)) return MF_ERR_INVALID;
    if (o.nvec_hint < 1 || o.nvec_hint > 64 || o.spin_limit < 0) return MF_ERR_INVALID;
    if (o.hermitian_reuse < -1 || o.hermitian_reuse > 1) return MF_ERR_INVALID;
    // block larger than D rounded to the tile: the stored blocks would be
    // smaller than b x b
    if (block > (D + kTile - 1) / kTile * kTile) return MF_ERR_INVALID;
    // P_cache from the budget (Eq. partial_cache_pairs); STORE_FULL insists
    if (o.storage != MF_STORE_FULL) o.storage = MF_STORE_PARTIAL;
    o.row_begin = o.row_end = 0;
    o.planner_mode = MF_PLANNER_ANALYTIC;
    return create_fixed(out, D, MF_GEN_EXTERNAL, 0, block, cache_budget_bytes, o, blocks);
  });
}

mf_status mf_sysbath_create(mf_plan_t* out, int64_t d_S, int64_t d_B, int32_t n_int, const uint64_t* seeds,
                            const void* H_S, const void* A, double g, const mf_options* opt) {
  return guard([&]() -> mf_status {
    if (!out) return MF_ERR_INVALID;
    *out = nullptr;
    mf_options o;
    if (opt) o = *opt; else mf_options_default(&o);
    if (d_S < 1 || d_S > 64 || d_B < 2 || d_B > (int64_t)1 << 31 || n_int < 0 || n_int > 15 || !seeds || !H_S ||
        (n_int > 0 && !A) || !std::isfinite(g))
      return MF_ERR_INVALID;
    if (o.precision == MF_PREC_BF16X2) return MF_ERR_UNSUPPORTED;
    if (o.precision != MF_PREC_FP64 && o.precision != MF_PREC_FP32) return MF_ERR_INVALID;
    if (!(o.cheb_tol > 0) || o.lanczos_m < 2 || !(o.alpha_safety > 0 && o.alpha_safety <= 1)) return MF_ERR_INVALID;
    if (o.hermitian_reuse < -1 || o.hermitian_reuse > 1) return MF_ERR_INVALID;
    // the bath operators are generated on demand (procedural storage)
    o.storage = MF_STORE_PROCEDURAL;
    o.row_begin = o.row_end = 0;
    o.planner_mode = MF_PLANNER_ANALYTIC;
    o.nvec_hint = (int32_t)std::max<int64_t>(2, d_S);
    const int64_t Dt = (d_B + kTile - 1) / kTile * kTile;
    mf_status st = create_fixed(out, d_B, MF_GEN_PHILOX_GUE, seeds[0], std::min<int64_t>(1024, Dt), 0, o);
    if (st != MF_OK) return st;
    Plan& p = (*out)->p;
    DeviceGuard guard(p.device);
    const int nop = 1 + n_int;
    std::vector<double2> M((size_t)nop * d_S * d_S, make_double2(0.0, 0.0));
    for (int64_t v = 0; v < d_S; ++v) M[(size_t)(v * d_S + v)] = make_double2(1.0, 0.0);
    const double2* Ah = (const double2*)A;
    for (int a = 0; a < n_int; ++a)
      for (int64_t e = 0; e < d_S * d_S; ++e) {
        const double2 x = Ah[(size_t)a * d_S * d_S + e];
        M[(size_t)(a + 1) * d_S * d_S + e] = make_double2(g * x.x, g * x.y);
      }
    auto fail = [&](mf_status s) {
      mf_plan_destroy(*out);
      *out = nullptr;
      return s;
    };
    if (dmalloc(&p.d_sb_seeds, nop * sizeof(uint64_t)) != cudaSuccess ||
        dmalloc(&p.d_sb_M, M.size() * sizeof(double2)) != cudaSuccess ||
        dmalloc(&p.d_sb_HS, (size_t)d_S * d_S * sizeof(double2)) != cudaSuccess)
      return fail(MF_ERR_OOM);
    if (cudaMemcpy(p.d_sb_seeds, seeds, nop * sizeof(uint64_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p.d_sb_M, M.data(), M.size() * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p.d_sb_HS, H_S, (size_t)d_S * d_S * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(MF_ERR_CUDA);
    p.sb_nop = nop;
    p.sb_dS = (int32_t)d_S;
    p.have_bounds = false;
    // dense-work estimate of the composite: n_op bath operators per product
    p.w_hpsi = (double)nop * (double)d_B * (double)d_B;
    p.dense_warn = p.w_hpsi > o.dense_work_limit;
    return MF_OK;
  });
}

mf_status mf_plan_destroy(mf_plan_t h) {
  if (!h) return MF_OK;
  DeviceGuard guard(h->p.device);
  cudaStreamSynchronize(h->p.stream);
  release(h->p);
  delete h;
  return MF_OK;
}

mf_status mf_apply(mf_plan_t h, void* y, const void* x, int64_t nvec) {
  if (!h || !y || !x || nvec < 1 || nvec > 64) return MF_ERR_INVALID;
  Plan& p = h->p;
  if (p.sb_nop && nvec != p.sb_dS) return MF_ERR_INVALID;
  // x holds all rows; y the plan's rows (a slice for a row-distributed plan)
  const size_t xbytes = (size_t)p.D * (size_t)nvec * sizeof(double2);
  const size_t ybytes = (size_t)(p.sliced ? p.row1 - p.row0 : p.D) * (size_t)nvec * sizeof(double2);
  const char *yb = (const char*)y, *xb = (const char*)x;
  if (yb < xb + xbytes && xb < yb + ybytes) return MF_ERR_INVALID;
  DeviceGuard guard(p.device);
  mf_status st = pending_device_error(p);
  if (st != MF_OK) return st;
  if ((st = apply_internal(p, (double2*)y, (const double2*)x, nvec)) != MF_OK) return st;
  return post_device_error_copy(p);
}

mf_status mf_spectral_bounds(mf_plan_t h, double* emin, double* emax) {
  if (!h) return MF_ERR_INVALID;
  DeviceGuard guard(h->p.device);
  mf_status st = compute_bounds(h->p);
  if (st != MF_OK) return st;
  if (emin) *emin = h->p.emin;
  if (emax) *emax = h->p.emax;
  return MF_OK;
}

mf_status mf_plan_set_bounds(mf_plan_t h, double emin, double emax) {
  if (!h || !(emax > emin) || !std::isfinite(emin) || !std::isfinite(emax)) return MF_ERR_INVALID;
  h->p.emin = emin;
  h->p.emax = emax;
  h->p.have_bounds = true;
  h->p.J_arg = -1.0;
  return MF_OK;
}

mf_status mf_cheb_terms(mf_plan_t h, double dt, int32_t* nterms) {
  if (!h || !nterms || !(dt > 0) || !std::isfinite(dt)) return MF_ERR_INVALID;
  Plan& p = h->p;
  DeviceGuard guard(p.device);
  mf_status st = compute_bounds(p);
  if (st != MF_OK) return st;
  const double R = 0.5 * (p.emax - p.emin);
  return coefficients(p, R * dt, 0, nterms);
}

mf_status mf_cheb_propagate(mf_plan_t h, void* psi, int64_t nvec, double dt, int32_t order) {
  if (!h || !psi || nvec < 1 || nvec > 64 || !(dt > 0) || !std::isfinite(dt) || order < 0) return MF_ERR_INVALID;
  Plan& p = h->p;
  if (p.sb_nop && nvec != p.sb_dS) return MF_ERR_INVALID;
  if (p.sliced) return MF_ERR_UNSUPPORTED;  // row groups use mf_rows_cheb_*
  DeviceGuard guard(p.device);
  mf_status st = pending_device_error(p);
  if (st != MF_OK) return st;
  st = compute_bounds(p);
  if (st != MF_OK) return st;
  const double c = 0.5 * (p.emax + p.emin), R = 0.5 * (p.emax - p.emin);
  int32_t nt = 0;
  st = coefficients(p, R * dt, order, &nt);
  if (st != MF_OK) return st;
  st = ensure_workspace(p, nvec);
  if (st != MF_OK) return st;
  const VecShape sh = shape_for(p, nvec);
  double2* q_prev = p.d_q[0];
  double2* q_cur = p.d_q[1];
  double2* acc = p.d_q[2];
  MF_CUDA(launch_cheb_init(p, (const double2*)psi, q_cur, acc, p.d_xc, sh));
  for (int32_t j = 1; j < nt; ++j) {
    if ((st = apply_kernel(p, nvec)) != MF_OK) return st;
    MF_CUDA(launch_cheb_update(p, p.d_part, q_cur, q_prev, acc, p.d_xc, sh, j, c, R, 0));
    std::swap(q_cur, q_prev);
  }
  MF_CUDA(launch_cheb_final(p, acc, (double2*)psi, p.D * nvec, c, dt));
  return post_device_error_copy(p);
}

mf_status mf_rows_cheb_begin(mf_plan_t h, double dt, int32_t order, int32_t* nterms) {
  if (!h || !nterms || !(dt > 0) || !std::isfinite(dt) || order < 0) return MF_ERR_INVALID;
  Plan& p = h->p;
  if (!p.sliced) return MF_ERR_INVALID;
  DeviceGuard guard(p.device);
  mf_status st = compute_bounds(p);
  if (st != MF_OK) return st;
  const double R = 0.5 * (p.emax - p.emin);
  return coefficients(p, R * dt, order, nterms, 0);
}

mf_status mf_rows_cheb_init(mf_plan_t h, const void* psi_full, void* acc_slice, int64_t nvec) {
  if (!h || !psi_full || !acc_slice || nvec < 1 || nvec > 64) return MF_ERR_INVALID;
  Plan& p = h->p;
  if (!p.sliced || p.J_arg < 0) return MF_ERR_INVALID;
  DeviceGuard guard(p.device);
  MF_CUDA(launch_cheb_rows_init(p, (const double2*)psi_full, (double2*)acc_slice, nvec));
  return MF_OK;
}

mf_status mf_rows_cheb_term(mf_plan_t h, int32_t j, const void* q_full, void* q_prev_slice, void* q_next_slice,
                            void* acc_slice, int64_t nvec) {
  if (!h || !q_full || !q_prev_slice || !q_next_slice || !acc_slice || nvec < 1 || nvec > 64 || j < 1)
    return MF_ERR_INVALID;
  Plan& p = h->p;
  if (!p.sliced || p.J_arg < 0 || j > p.J_K) return MF_ERR_INVALID;
  DeviceGuard guard(p.device);
  mf_status st = pending_device_error(p);
  if (st != MF_OK) return st;
  if ((st = ensure_workspace(p, nvec)) != MF_OK) return st;
  // y = H q_j on the slice, into the plan's own vector workspace
  double2* y = p.d_q[2];
  if ((st = apply_internal(p, y, (const double2*)q_full, nvec)) != MF_OK) return st;
  const double c = 0.5 * (p.emax + p.emin), R = 0.5 * (p.emax - p.emin);
  MF_CUDA(launch_cheb_rows_term(p, y, (const double2*)q_full, (double2*)q_prev_slice, (double2*)q_next_slice,
                                (double2*)acc_slice, nvec, j, c, R));
  return post_device_error_copy(p);
}

mf_status mf_rows_cheb_final(mf_plan_t h, const void* acc_slice, void* psi_slice, int64_t nvec, double dt) {
  if (!h || !acc_slice || !psi_slice || nvec < 1 || nvec > 64 || !std::isfinite(dt)) return MF_ERR_INVALID;
  Plan& p = h->p;
  if (!p.sliced || !p.have_bounds) return MF_ERR_INVALID;
  DeviceGuard guard(p.device);
  const double c = 0.5 * (p.emax + p.emin);
  MF_CUDA(launch_cheb_final(p, (const double2*)acc_slice, (double2*)psi_slice, (p.row1 - p.row0) * nvec, c, dt));
  return MF_OK;
}

mf_status mf_cheb_filter_terms(mf_plan_t h, double tau, int32_t* nterms) {
  if (!h || !nterms || !(tau >= 0) || !std::isfinite(tau)) return MF_ERR_INVALID;
  Plan& p = h->p;
  DeviceGuard guard(p.device);
  mf_status st = compute_bounds(p);
  if (st != MF_OK) return st;
  const double R = 0.5 * (p.emax - p.emin);
  return coefficients(p, R * tau, 0, nterms, 1);
}

// Same recurrence as mf_cheb_propagate with the real coefficients of
// exp(-z x) = I_0(z) + 2 sum (-1)^k I_k(z) T_k(x), z = R tau, scaled by e^{-z}:
// the result is exp(-tau (H - E_min)) psi with E_min = c - R, so no factor
// e^{-tau E} can overflow or underflow.
mf_status mf_cheb_filter(mf_plan_t h, void* psi, int64_t nvec, double tau, int32_t order, int32_t normalize) {
  if (!h || !psi || nvec < 1 || nvec > 64 || !(tau >= 0) || !std::isfinite(tau) || order < 0) return MF_ERR_INVALID;
  Plan& p = h->p;
  if (p.sb_nop && nvec != p.sb_dS) return MF_ERR_INVALID;
  if (p.sliced) return MF_ERR_UNSUPPORTED;
  DeviceGuard guard(p.device);
  mf_status st = pending_device_error(p);
  if (st != MF_OK) return st;
  if ((st = compute_bounds(p)) != MF_OK) return st;
  const double c = 0.5 * (p.emax + p.emin), R = 0.5 * (p.emax - p.emin);
  int32_t nt = 0;
  st = coefficients(p, R * tau, order, &nt, 1);
  if (st != MF_OK) return st;
  st = ensure_workspace(p, nvec);
  if (st != MF_OK) return st;
  const VecShape sh = shape_for(p, nvec);
  double2* q_prev = p.d_q[0];
  double2* q_cur = p.d_q[1];
  double2* acc = p.d_q[2];
  MF_CUDA(launch_cheb_init(p, (const double2*)psi, q_cur, acc, p.d_xc, sh));
  for (int32_t j = 1; j < nt; ++j) {
    if ((st = apply_kernel(p, nvec)) != MF_OK) return st;
    MF_CUDA(launch_cheb_update(p, p.d_part, q_cur, q_prev, acc, p.d_xc, sh, j, c, R, 1));
    std::swap(q_cur, q_prev);
  }
  // a system-bath plan's [d_B][d_S] block is one composite vector
  if (p.sb_nop)
    MF_CUDA(launch_filter_final(p, acc, (double2*)psi, p.D * nvec, 1, normalize != 0));
  else
    MF_CUDA(launch_filter_final(p, acc, (double2*)psi, p.D, nvec, normalize != 0));
  return post_device_error_copy(p);
}

mf_status mf_plan_profile(mf_plan_t h, int32_t enable) {
  if (!h) return MF_ERR_INVALID;
  h->p.profiling = enable != 0;
  h->p.ev_used = 0;
  return MF_OK;
}

mf_status mf_plan_profile_read(mf_plan_t h, double* total_ms, int64_t* launches) {
  if (!h || !total_ms || !launches) return MF_ERR_INVALID;
  Plan& p = h->p;
  DeviceGuard guard(p.device);
  MF_CUDA(cudaStreamSynchronize(p.stream));
  double tot = 0.0;
  for (size_t i = 0; i < p.ev_used; ++i) {
    float ms = 0.f;
    MF_CUDA(cudaEventElapsedTime(&ms, p.ev[i].first, p.ev[i].second));
    tot += ms;
  }
  *total_ms = tot;
  *launches = (int64_t)p.ev_used;
  p.ev_used = 0;
  return MF_OK;
}

mf_status mf_sync(mf_plan_t h) {
  if (!h) return MF_ERR_INVALID;
  Plan& p = h->p;
  DeviceGuard guard(p.device);
  int err = 0;
  if (cudaMemcpyAsync(&err, p.d_err, sizeof(int), cudaMemcpyDeviceToHost, p.stream) != cudaSuccess)
    return MF_ERR_CUDA;
  if (cudaStreamSynchronize(p.stream) != cudaSuccess) return MF_ERR_CUDA;
  p.err_pending = false;
  if (err == 0) return MF_OK;
  p.last_dev_err = err;
  if (cudaMemsetAsync(p.d_err, 0, sizeof(int), p.stream) != cudaSuccess ||
      cudaStreamSynchronize(p.stream) != cudaSuccess)
    return MF_ERR_CUDA;
  return status_of_device_code(err);
}

// Plan record for continuation runs (the selected plan reused without
// planning, Sec. VII): a versioned text of "key=value" lines, integers in
// decimal and doubles as exact hexadecimal floats.
mf_status mf_plan_serialize(mf_plan_t h, char* buf, size_t len, size_t* needed) {
  return guard([&]() -> mf_status {
    if (!h) return MF_ERR_INVALID;
    const Plan& p = h->p;
    if (p.gen == MF_GEN_EXTERNAL || p.sb_nop) return MF_ERR_UNSUPPORTED;
    std::string t = "mf_plan v1\n";
    auto put_i = [&](const char* k, long long v) {
      char b[96];
      std::snprintf(b, sizeof(b), "%s=%lld\n", k, v);
      t += b;
    };
    auto put_d = [&](const char* k, double v) {
      char b[96];
      std::snprintf(b, sizeof(b), "%s=%a\n", k, v);
      t += b;
    };
    put_i("D", p.D);
    put_i("generator", p.gen);
    t += "seed=" + std::to_string((unsigned long long)p.seed) + "\n";
    put_i("precision", p.prec);
    put_i("block", p.b);
    put_i("storage", p.storage);
    put_i("pairs_cached", p.pairs_cached);
    put_d("dvr_L", p.dvr.L);
    put_i("nvec_hint", p.opt.nvec_hint);
    put_d("cheb_tol", p.opt.cheb_tol);
    put_i("lanczos_m", p.opt.lanczos_m);
    put_d("bounds_pad", p.opt.bounds_pad);
    put_d("alpha_safety", p.opt.alpha_safety);
    put_d("f_cache", p.opt.f_cache);
    put_d("dense_work_limit", p.opt.dense_work_limit);
    put_i("hermitian_reuse", p.opt.hermitian_reuse);
    put_i("row_begin", p.opt.row_begin);
    put_i("row_end", p.opt.row_end);
    put_i("spin_limit", p.opt.spin_limit);
    put_i("have_bounds", p.have_bounds ? 1 : 0);
    put_d("emin", p.emin);
    put_d("emax", p.emax);
    put_i("planner", p.planner_used);
    put_d("s_model", p.s_model);
    put_d("t_measured", p.t_measured);
    put_i("num_sms", p.num_sms);
    if (needed) *needed = t.size() + 1;
    if (!buf) return MF_OK;
    if (len == 0) return MF_ERR_INVALID;
    std::strncpy(buf, t.c_str(), len - 1);
    buf[len - 1] = '\0';
    return t.size() + 1 <= len ? MF_OK : MF_ERR_INVALID;
  });
}

mf_status mf_plan_deserialize(mf_plan_t* out, const char* rec, size_t len, const mf_options* opt) {
  return guard([&]() -> mf_status {
    if (!out || !rec) return MF_ERR_INVALID;
    *out = nullptr;
    const std::string text(rec, strnlen(rec, len));
    if (text.compare(0, 11, "mf_plan v1\n") != 0) return MF_ERR_INVALID;
    std::vector<std::pair<std::string, std::string>> kv;
    size_t pos = 11;
    while (pos < text.size()) {
      size_t eol = text.find('\n', pos);
      if (eol == std::string::npos) eol = text.size();
      const std::string line = text.substr(pos, eol - pos);
      pos = eol + 1;
      if (line.empty()) continue;
      const size_t eq = line.find('=');
      if (eq == std::string::npos || eq == 0) return MF_ERR_INVALID;
      kv.emplace_back(line.substr(0, eq), line.substr(eq + 1));
    }
    auto find = [&](const char* k) -> const std::string* {
      for (const auto& e : kv)
        if (e.first == k) return &e.second;
      return nullptr;
    };
    bool bad = false;
    auto get_i = [&](const char* k) -> long long {
      const std::string* v = find(k);
      if (!v || v->empty()) { bad = true; return 0; }
      char* end = nullptr;
      const long long r = std::strtoll(v->c_str(), &end, 10);
      if (*end) bad = true;
      return r;
    };
    auto get_u = [&](const char* k) -> unsigned long long {
      const std::string* v = find(k);
      if (!v || v->empty()) { bad = true; return 0; }
      char* end = nullptr;
      const unsigned long long r = std::strtoull(v->c_str(), &end, 10);
      if (*end) bad = true;
      return r;
    };
    auto get_d = [&](const char* k) -> double {
      const std::string* v = find(k);
      if (!v || v->empty()) { bad = true; return 0.0; }
      char* end = nullptr;
      const double r = std::strtod(v->c_str(), &end);
      if (*end) bad = true;
      return r;
    };
    mf_options o;
    if (opt) o = *opt; else mf_options_default(&o);
    const long long D = get_i("D");
    const int gen = (int)get_i("generator");
    const unsigned long long seed = get_u("seed");
    o.precision = (int32_t)get_i("precision");
    const long long block = get_i("block");
    o.storage = (int32_t)get_i("storage");
    const long long pc = get_i("pairs_cached");
    o.dvr_L = get_d("dvr_L");
    o.nvec_hint = (int32_t)get_i("nvec_hint");
    o.cheb_tol = get_d("cheb_tol");
    o.lanczos_m = (int32_t)get_i("lanczos_m");
    o.bounds_pad = get_d("bounds_pad");
    o.alpha_safety = get_d("alpha_safety");
    o.f_cache = get_d("f_cache");
    o.dense_work_limit = get_d("dense_work_limit");
    o.hermitian_reuse = (int32_t)get_i("hermitian_reuse");
    o.row_begin = get_i("row_begin");
    o.row_end = get_i("row_end");
    o.spin_limit = (int32_t)get_i("spin_limit");
    const bool hb = get_i("have_bounds") != 0;
    const double emin = get_d("emin"), emax = get_d("emax");
    const int planner = (int)get_i("planner");
    const double s_model = get_d("s_model"), t_meas = get_d("t_measured");
    o.planner_mode = MF_PLANNER_ANALYTIC;
    o.model = nullptr;
    if (bad) return MF_ERR_INVALID;
    if (D < 2 || D > (int64_t)1 << 31 || (gen != MF_GEN_PHILOX_GUE && gen != MF_GEN_SINC_DVR_HO)) return MF_ERR_INVALID;
    if (o.precision < MF_PREC_FP64 || o.precision > MF_PREC_BF16X2) return MF_ERR_INVALID;
    if (block < kTile || block % kTile != 0 || pc < 0) return MF_ERR_INVALID;
    if (o.storage < MF_STORE_PROCEDURAL || o.storage > MF_STORE_FULL) return MF_ERR_INVALID;
    if (!(o.dvr_L > 0) || !std::isfinite(o.dvr_L) || !(o.cheb_tol > 0) || o.lanczos_m < 2 ||
        !(o.alpha_safety > 0 && o.alpha_safety <= 1) || o.nvec_hint < 1 || o.nvec_hint > 64 ||
        o.hermitian_reuse < -1 || o.hermitian_reuse > 1 || o.spin_limit < 0)
      return MF_ERR_INVALID;
    if (o.row_begin != 0 || o.row_end != 0) {
      if (o.row_begin < 0 || o.row_end <= o.row_begin || o.row_end > D || o.row_begin % kTile != 0 ||
          (o.row_end % kTile != 0 && o.row_end != D))
        return MF_ERR_INVALID;
    }
    if (hb && !(emax > emin && std::isfinite(emin) && std::isfinite(emax))) return MF_ERR_INVALID;
    // the recorded block, storage and cache share: no planning, no measurement
    const double eb = (double)compute_elem_bytes(o.precision);
    const size_t budget = (size_t)((double)pc * eb * (double)block * (double)block);
    mf_status st = create_fixed(out, D, gen, seed, block, budget, o);
    if (st != MF_OK && st != MF_WARN_DENSE_WORK) return st;
    Plan& p = (*out)->p;
    if (hb) {  // the recorded bounds: the Chebyshev coefficients come out the same
      p.emin = emin;
      p.emax = emax;
      p.have_bounds = true;
    }
    p.planner_used = planner;
    p.s_model = s_model;
    p.t_measured = t_meas;
    p.deserialized = true;
    p.trials.push_back(std::string("{\"deserialized\": true, \"t_mv\": -1}"));
    return st;
  });
}

mf_status mf_plan_describe(mf_plan_t h, char* buf, size_t len) {
  if (!h || !buf || len == 0) return MF_ERR_INVALID;
  const Plan& p = h->p;
  char tmp[3072];
  const int n = std::snprintf(
      tmp, sizeof(tmp),
      "{\"D\": %lld, \"generator\": \"%s\", \"seed\": %llu, \"precision\": \"%s\", \"block\": %lld, "
      "\"n_blk\": %lld, \"n_pair\": %lld, \"storage\": \"%s\", \"cache_budget_bytes\": %zu, "
      "\"pairs_cached\": %lld, \"cache_bytes\": %zu, \"path\": \"%s\", \"tile\": %d, \"dvr_rows\": %d, "
      "\"dvr_cols\": %d, \"n_slot\": %lld, \"n_work\": %lld, \"w_hpsi\": %.6g, \"dense_warn\": %s, "
      "\"dvr_L\": %.17g, \"dvr_dx\": %.17g, \"have_bounds\": %s, \"emin\": %.17g, \"emax\": %.17g, "
      "\"num_sms\": %d, \"sb_nop\": %d, \"sb_dS\": %d, \"spin_limit\": %u, \"last_device_error\": %d, \"tc_walk\": \"%s\", "
      "\"tch_unit\": %d, \"tch_units\": %lld, \"cache_format\": \"%s\", "
      "\"planner\": %d, \"deserialized\": %s}",
      (long long)p.D, gen_name(p.gen), (unsigned long long)p.seed, prec_name(p.prec), (long long)p.b,
      (long long)p.nblk, (long long)p.npair, store_name(p.storage), p.cache_budget, (long long)p.pairs_cached,
      p.cache_bytes, p.sb_nop ? "sysbath_rows" : (p.use_dvr_window ? "dvr_window" : "herm_tile"), kTile, p.dvr_rows,
      p.dvr_cols,
      (long long)p.nslot, (long long)p.nwork, p.w_hpsi, p.dense_warn ? "true" : "false", p.dvr.L, p.dvr.dx,
      p.have_bounds ? "true" : "false", p.emin, p.emax, p.num_sms, p.sb_nop, p.sb_dS, p.spin, p.last_dev_err,
      p.prec != MF_PREC_BF16X2 ? "none" : (p.tch ? "hermitian" : "row_owner"), p.tch_s,
      (long long)p.tch_nunits, p.tch ? "bf16x2_tiles" : (p.prec == MF_PREC_FP64 ? "complex128" : "complex64"),
      p.planner_used, p.deserialized ? "true" : "false");
  if (n < 0) return MF_ERR_INVALID;
  std::strncpy(buf, tmp, len - 1);
  buf[len - 1] = '\0';
  return (size_t)n < len ? MF_OK : MF_ERR_INVALID;
}

mf_status mf_debug_entries(mf_plan_t h, int64_t r0, int64_t c0, int64_t rows, int64_t cols, void* out_host) {
  if (!h || !out_host || rows < 1 || cols < 1) return MF_ERR_INVALID;
  Plan& p = h->p;
  if (p.gen == MF_GEN_EXTERNAL) return MF_ERR_UNSUPPORTED;
  if (r0 < 0 || c0 < 0 || r0 + rows > p.D || c0 + cols > p.D) return MF_ERR_INVALID;
  DeviceGuard guard(p.device);
  const size_t bytes = (size_t)rows * (size_t)cols * compute_elem_bytes(p.prec);
  void* d = nullptr;
  MF_CUDA(dev_malloc(&d, bytes));
  cudaError_t e = launch_debug_entries(p, r0, c0, rows, cols, d);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, d, bytes, cudaMemcpyDeviceToHost, p.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p.stream);
  cudaFree(d);
  return e == cudaSuccess ? MF_OK : MF_ERR_CUDA;
}

}  // extern "C"
