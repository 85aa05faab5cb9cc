// mf_internal.h -- plan record and kernel launcher declarations shared by the
// translation units of libmf (host side).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/mf.h"
#include "gen.cuh"

namespace mf {

constexpr int kTile = 128;  // CTA tile edge of the Hermitian (canonical-pair) kernels

// Device error word codes: kernels set the word with atomicCAS(word, 0, code)
// when a bounded wait runs out; the code says which wait (100..199).
constexpr int kErrTimeoutFirst = 100, kErrTimeoutLast = 199;
// polls of a bounded wait: each poll suspends at most 5 us, so a wait that
// never completes ends within about 1.3 s
constexpr uint32_t kDefaultSpin = 1u << 18;

// Host-side fault injection (MF_FAULT="<site>:<n>", see include/mf.h): true
// when this event of the site is the n-th since the variable took its value.
bool fault_hit(const char* site);
// cudaMalloc through the "alloc" injection site.
cudaError_t dev_malloc(void** ptr, size_t bytes);

// One CTA work item of the Hermitian apply: canonical tile (ti <= tj) in units
// of kTile, and the byte offset of its block in the HBM cache (-1 when the
// block pair is generated procedurally).
struct WorkItem {
  int32_t ti, tj;
  // element offset of the tile in the HBM cache (>= 0), -1 when generated,
  // or -2 - (element offset in the external host array)
  int64_t cache_off;
};

// One CTA of the Hermitian multi-vector kernel (k_rows_herm.cu): row tile
// ti, its owner-row partial slot, and the columns [c_beg, c_end) it covers
// (c_beg >= 128 ti).
struct HermItem {
  int32_t ti, slot;
  int64_t c_beg, c_end;
};

struct Plan {
  // problem
  int64_t D = 0;
  int32_t gen = 0;
  uint64_t seed = 0;
  int32_t prec = MF_PREC_FP32;
  mf_options opt{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  // partition (Sec. II) and storage (Sec. III.A)
  int64_t b = 0, nblk = 0, npair = 0;
  int32_t storage = MF_STORE_PROCEDURAL;
  size_t cache_budget = 0, cache_bytes = 0;
  int64_t pairs_cached = 0;
  std::vector<int64_t> pair_slot;  // nblk*nblk (n<=m) -> cache slot or -1
  void* d_cache = nullptr;
  // externally stored blocks (MF_GEN_EXTERNAL): the caller's host array of
  // canonical blocks, registered and read by the kernels over the host link
  // for the pairs not copied into d_cache
  const void* h_blocks = nullptr;
  const void* d_hblocks = nullptr;  // device-visible address of h_blocks
  bool h_registered = false;
  // generator constants
  float sigma32 = 0.f;
  double sigma64 = 0.0;
  dvr_consts dvr{};
  // Hermitian (Philox) tiling
  int64_t ntile = 0;              // tile rows = ceil(D / kTile)
  WorkItem* d_work = nullptr;     // canonical tiles, cached/procedural interleaved
  int64_t nwork = 0;
  // multi-vector row-owner path: split-K over column ranges
  int64_t rows_nsplit = 1, rows_split_cols = 0;
  int64_t* d_pair_slot = nullptr;  // device copy of pair_slot
  // multi-vector Hermitian-reuse path: column items, owner slots per tile
  HermItem* d_herm_items = nullptr;
  int64_t herm_nitems = 0, herm_ns = 0;
  double herm_limit = 0.0;  // largest partial-slot buffer (bytes) the path may use
  // BF16X2 Hermitian tensor-core walk (k_tch.cu): units of tch_s x tch_s
  // tiles, their order and slot row offsets, the unit counter and the slots
  bool tch = false;                // the plan's BF16X2 apply uses it (its cache is then in the
                                   // walk's bf16 tile format, not FP32 complex)
  int32_t tch_s = 0, tch_U = 0;
  int64_t tch_nunits = 0, tch_rows = 0;
  int2* d_tch_units = nullptr;
  int64_t* d_tch_off = nullptr;
  int* d_tch_counter = nullptr;
  void* d_tch_slots = nullptr;     // [tch_rows][2 nb] FP32
  size_t tch_slots_cap = 0;
  double tch_limit = 0.0;          // largest slot buffer (bytes) the walk may use
  // row-distributed plan: output rows [row0, row1), row tiles slice_t0 ..
  // slice_t0 + slice_nt - 1 (row-owner kernels only)
  bool sliced = false;
  int64_t row0 = 0, row1 = 0, slice_t0 = 0, slice_nt = 0;
  // DVR launch shape
  int dvr_rows = 512, dvr_cols = 4096;
  // workspace buffers and the bytes each holds (grown on demand)
  size_t part_cap = 0, xc_cap = 0, tcb_cap = 0, sb_xo_cap = 0;
  size_t q_cap[3] = {0, 0, 0};
  int64_t nslot = 0;              // partial-sum slots per output row
  int64_t dpad = 0;               // rows per slot (D padded to the kernel's row tile)
  bool use_dvr_window = false;    // DVR procedural path (Toeplitz window kernel)
  void* d_part = nullptr;         // [nslot][D][nvec] complex (compute precision)
  void* d_xc = nullptr;           // compute-precision copy of the input
  void* d_tcb = nullptr;          // BF16X2: split operand tiles of X
  double2* d_q[3] = {nullptr, nullptr, nullptr};  // Chebyshev q_prev, q_cur, acc
  double* d_J = nullptr;          // Bessel J_k(R dt), or scaled I_k(R tau) for the filter
  int32_t J_cap = 0;
  double* d_red = nullptr;        // small reduction scratch (dots/norms)
  int* d_err = nullptr;           // device error word
  int* h_err = nullptr;           // pinned host copy of the word, read without blocking
  cudaEvent_t err_ev = nullptr;   // recorded after the copy into h_err
  bool err_pending = false;       // a copy into h_err was enqueued and not yet read
  bool has_waits = false;         // the plan's kernels have bounded waits (tensor-core form)
  uint32_t spin = kDefaultSpin;   // polls of one bounded wait (mf_options.spin_limit)
  int last_dev_err = 0;           // last device error code reported
  // spectral bounds
  bool have_bounds = false;
  double emin = 0.0, emax = 0.0;
  // Chebyshev coefficient cache
  double J_arg = -1.0;
  int32_t J_kind = 0;             // 0: J_k (real time), 1: e^{-z} I_k (imaginary time)
  int32_t J_K = 0;
  int32_t J_terms = 0;
  // per-launch timing of the apply kernel (CUDA events on the plan's stream)
  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  size_t ev_used = 0;
  // planner record: Algorithm 1 score, measured time, trial log (JSON lines)
  double m_work = 0.0;
  double s_model = 0.0;
  double t_measured = -1.0;
  int32_t planner_used = MF_PLANNER_ANALYTIC;
  bool deserialized = false;      // created by mf_plan_deserialize (no planning)
  std::vector<std::string> trials;
  // safety estimate (Sec. IV.H)
  double w_hpsi = 0.0;
  bool dense_warn = false;
  // system-bath composite (Sec. VII, k_sysbath.cu): D is the bath dimension
  // d_B, vectors are [d_B][d_S] with nvec == d_S; sb_nop = 1 + n_int bath
  // operators (0: a plain plan)
  int32_t sb_nop = 0, sb_dS = 0;
  uint64_t* d_sb_seeds = nullptr;  // [nop] Philox seeds of H_B, B_1..B_n
  double2* d_sb_M = nullptr;       // [nop][dS][dS]: M_0 = I, M_a = g A_a
  double2* d_sb_HS = nullptr;      // [dS][dS] system Hamiltonian
  void* d_sb_xo = nullptr;         // [nop][rows][nb] mixed inputs X M_o^T (compute precision)
  int64_t sb_rows = 0;             // rows of each mixed input
};

// Generator constants of the sinc-DVR operator on D points of [-L, L]
// (L <= 0 selects 0.9 sqrt(2D)), and the launch shape of the FP32 Toeplitz
// window kernel for one vector (dvr_rows, dvr_cols, nslot, dpad).  Shared by
// plan creation and the allocation-free entry point.
void dvr_setup(dvr_consts& k, int64_t D, double L);
void dvr_fp32_window_shape(Plan& p);

// Plan services shared with the batched path (mf_api.cu).
mf_status plan_workspace(Plan& p, int64_t nvec);
mf_status plan_bounds(Plan& p);
mf_status plan_coefficients(Plan& p, double z, int32_t order, int32_t* nterms, int32_t kind = 0);

// ---- launchers (return cudaError_t of the launch) ----
// Hermitian canonical-tile apply, nvec == 1 register kernel.
cudaError_t launch_gue_apply(const Plan& p, const void* xc, void* part, int64_t nvec);
// DVR Toeplitz-window apply (FP64 form: rows x column chunk per CTA; FP32
// form: persistent row-split kernel with the shape below).
cudaError_t launch_dvr_apply(const Plan& p, const void* xc, void* part, int64_t nvec);
// Launch shape of the FP32 persistent DVR kernel: row tile and staged chunk
// sizes, 16-column blocks per row tile, work items, grid, partial slots and
// padded rows per slot.
struct DvrRowsShape {
  int64_t rows, cols, rtiles, nbc, nblocks, grid, nslot, dpad;
};
DvrRowsShape dvr_rows_shape(int64_t D, int num_sms);
// Multi-vector DVR window kernel (FP32 form): vector buckets 2, 4, 8, 16,
// its row split for nb vectors and the launch (xc [rows][nb] -> part).
int64_t dvr_mv_bucket(int64_t nvec);
DvrRowsShape dvr_mv_shape(int64_t D, int64_t nb, int num_sms);
cudaError_t launch_dvr_mv(const Plan& p, const void* xc, void* part, int64_t nb);
// Fill the cache blocks listed in d_pairs (block pair (n, m) per cache slot).
cudaError_t launch_cache_fill_pairs(const Plan& p, const int2* d_pairs, int64_t npairs);
// Multi-vector row-owner apply (nvec bucket 2..64).
cudaError_t launch_rows_apply(const Plan& p, const void* xc, void* part, int64_t nvec_bucket);
// Hermitian-reuse multi-vector apply (k_rows_herm.cu): nop operators (seeds
// per operator, or the plan's seed when seeds == nullptr) on inputs xc + o
// xstride; part must be zero-filled ([herm_ns + ntile][ntile 128][nb]).
std::vector<HermItem> rows_herm_items(int64_t D, int num_sms, int64_t* ns_out);
cudaError_t launch_rows_herm(const Plan& p, const void* xc, int64_t xstride, void* part, int64_t nb, int nop,
                             const uint64_t* seeds);
int64_t rows_nvec_bucket(int64_t nvec);
// Tensor-core BF16X2 apply (k_tc.cu): vector buckets 8..64, operand tiles of
// X in gB (tc_operand_bytes bytes).
cudaError_t launch_tc_apply(const Plan& p, const void* xc, void* part, void* gB, int64_t nv_bucket);
size_t tc_operand_bytes(int64_t D, int64_t nv_bucket);
int64_t tc_nvec_bucket(int64_t nvec);
// Hermitian-reuse tensor-core apply (k_tch.cu): unit layout for T tile rows
// (returns the slot rows), operand bytes, and the launch (operand split,
// persistent unit walk, gather into two slots of part).
int64_t tch_layout(int64_t T, int num_sms, int32_t* s_out, int32_t* U_out, std::vector<int2>& units,
                   std::vector<int64_t>& off2d);
size_t tch_operand_bytes(int64_t D, int64_t nv_bucket);
cudaError_t launch_tch_apply(const Plan& p, const void* xc, void* part, void* gB, int64_t nv_bucket);
// Fill the cache of a Hermitian tensor-core plan in its consumer format
// (every tile of the listed block pairs as the kernel's four bf16 planes).
cudaError_t launch_tch_cache_fill(const Plan& p, const int2* d_pairs, int64_t npairs);

// Vector layouts: the FP64 master x/y is [D][nv]; the compute copy xc and the
// partial slots use a padded vector stride nb >= nv ([D][nb], [slot][dpad][nb])
// with zeros in the padding.  nslot/dpad describe the path in use.
// C++ exceptions must not cross the C boundary: entry points that build host
// containers (pair lists, work items, candidate lists, JSON records) run
// their body through guard(), which maps a host allocation failure to
// MF_ERR_OOM and anything else thrown to MF_ERR_INVALID.
template <typename F>
mf_status guard(F&& body) {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return MF_ERR_OOM;
  } catch (...) {
    return MF_ERR_INVALID;
  }
}

struct VecShape {
  int64_t nv, nb, nslot, dpad;
};
// FP64 master -> compute-precision copy (padding written as zeros).
cudaError_t launch_to_compute(const Plan& p, const double2* x, void* xc, int64_t D, VecShape s);
// y = sum of partial slots (+ V x for the DVR), FP64.
cudaError_t launch_reduce(const Plan& p, const void* part, const double2* x, double2* y, VecShape s);
// Chebyshev pieces.
cudaError_t launch_cheb_init(const Plan& p, const double2* psi, double2* q, double2* acc, void* xc, VecShape s);
cudaError_t launch_cheb_update(const Plan& p, const void* part, const double2* qcur, double2* qprev,
                               double2* acc, void* xc, VecShape s, int32_t k_next, double c, double R,
                               int imag_time);
cudaError_t launch_cheb_final(const Plan& p, const double2* acc, double2* psi, int64_t n, double c, double dt);
cudaError_t launch_bessel(const Plan& p, double z, int32_t K, double* J);
// Row-distributed Chebyshev pieces (slice of the plan's rows, see k_vec.cu).
cudaError_t launch_cheb_rows_init(const Plan& p, const double2* psi, double2* acc, int64_t nvec);
cudaError_t launch_cheb_rows_term(const Plan& p, const double2* y, const double2* qfull, double2* qprev,
                                  double2* qnext, double2* acc, int64_t nvec, int32_t j, double c, double R);
// Imaginary-time filter pieces: scaled I_k(z) and the final copy with optional
// per-column renormalisation (reduction scratch in d_red: 64*64 + 64 doubles).
cudaError_t launch_bessel_i(const Plan& p, double z, int32_t K, double* I);
// rows x nv columns, each column normalised on its own when normalize != 0.
cudaError_t launch_filter_final(const Plan& p, const double2* acc, double2* psi, int64_t rows, int64_t nv,
                                int normalize);
constexpr int64_t kRedDoubles = 64 * 64 + 64 + 512;
// Lanczos helpers: out[0] = Re<a,b>, FP64 reduction into d_red slot.
cudaError_t launch_dot(const Plan& p, const double2* a, const double2* b, int64_t n, double* out);
cudaError_t launch_axpby_lanczos(const Plan& p, double2* w, const double2* v, const double2* vprev,
                                 double alpha, double beta, int64_t n);
cudaError_t launch_scale(const Plan& p, double2* dst, const double2* src, double s, int64_t n);
cudaError_t launch_random_unit(const Plan& p, double2* v, int64_t n, uint64_t seed);
// Entry dump of the generator (plan precision form) into a device buffer.
cudaError_t launch_debug_entries(const Plan& p, int64_t r0, int64_t c0, int64_t rows, int64_t cols,
                                 void* out);

size_t compute_elem_bytes(int prec);  // bytes of one complex compute-format element

// System-bath composite (k_sysbath.cu): mixed inputs xo[o] = xc M_o^T and
// the fused multi-operator row kernel (vector bucket nb).
cudaError_t launch_sb_mix(const Plan& p, const void* xc, void* xo, int64_t nb, int64_t rows);
cudaError_t launch_sb_rows(const Plan& p, const void* xo, int64_t ostride, void* part, int64_t nb);

// Surrogate prediction of one candidate's time (k_mlp.cu); model is an mf_mlp.
mf_status surrogate_predict(void* model, int32_t generator, int32_t precision, const mf_problem& pr,
                            const mf_candidate& c, const mf_estimate& e, double budget, double gpu_mem, int sms,
                            double* t);
void mlp_features(int32_t generator, int32_t precision, const mf_problem& pr, const mf_candidate& c,
                  const mf_estimate& e, double budget, float* x);

// Algorithm 1 estimate of one candidate (planner.cu).
void planner_estimate(const mf_problem& pr, const mf_candidate& c, const mf_device_model& dm, double alpha,
                      double cache_budget, mf_estimate& e);

}  // namespace mf

// The opaque handle of the C ABI.
struct mf_plan {
  mf::Plan p;
};
