/*
 * mf.h -- C ABI of the GB300 matrix-free block-procedural operator library.
 *
 * The library applies a dense Hermitian operator H (D x D, complex) to one or
 * more vectors without materialising H: every block H^[n,m] is generated on
 * demand inside the apply kernel, or read from an HBM block cache that holds
 * none, some or all canonical block pairs (n <= m) under a memory budget.
 * A centred Chebyshev expansion of exp(-i dt H) is built on the product.
 *
 * Paper: U. Shafir, R. Kosloff, "Memory-Scalable and Hardware-Adaptive
 * Matrix-Free Quantum Simulation".  Section/equation numbers below refer to it.
 *
 * Conventions shared by every call
 *  - Vectors are complex128 (interleaved re, im doubles), row-major [D][nvec]
 *    with the vector index fastest (the Y = A X layout of Sec. IV.A,
 *    Eq. generic_multivector).  Pointers passed to mf_apply/mf_cheb_propagate
 *    are DEVICE pointers owned by the caller; the library never frees them.
 *  - The plan owns its cache, workspace and CUDA resources; mf_plan_destroy
 *    releases them.  Work is enqueued on the plan's stream (mf_options.stream,
 *    NULL = the legacy default stream) and is asynchronous unless stated.
 *  - Every call returns an mf_status.  Argument errors are detected on the host
 *    before anything is enqueued and leave the plan unchanged.  CUDA launch
 *    errors are returned as MF_ERR_CUDA by the call that hit them.  Kernel-side
 *    failures (the plan's device error word: a bounded wait that ran out) are
 *    returned by mf_sync, or by the next mf_apply / mf_cheb_propagate /
 *    mf_cheb_filter / mf_rows_cheb_term on the plan once the earlier work has
 *    finished (read without blocking); that call then enqueues nothing.  The
 *    word is cleared when it is reported, so the plan stays usable.
 *  - Fault injection for tests of these paths (host side only, no GPU fault is
 *    ever caused): the environment variable MF_FAULT="<site>:<n>" makes the
 *    n-th event of <site>, counted from the moment the variable took that
 *    value, fail: "alloc" (a device allocation of the library reports out of
 *    memory), "launch" (an apply kernel launch reports a launch failure,
 *    nothing is launched), "plan" (a candidate plan the planner builds fails,
 *    so the planner moves on to the next one).
 *  - Hermitian generators require M == D.  y must not alias x.
 *  - A plan (or batch) is used by one host thread at a time: its calls share
 *    the plan's workspace, partial slots and events.  Distinct plans are
 *    independent and may be driven from different threads and streams.
 */
#ifndef MF_H
#define MF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mf_plan* mf_plan_t;
typedef struct mf_mlp* mf_mlp_t;
typedef struct mf_batch* mf_batch_t;

typedef enum {
  MF_OK = 0,
  MF_ERR_INVALID = 1,      /* bad argument; nothing enqueued */
  MF_ERR_OOM = 2,          /* device allocation failed or plan exceeds memory */
  MF_ERR_CUDA = 3,         /* a CUDA runtime call or launch failed */
  MF_ERR_UNSUPPORTED = 4,  /* valid request this build does not implement */
  MF_ERR_TIMEOUT = 5,      /* a bounded device wait ran out */
  MF_WARN_DENSE_WORK = 6   /* plan created, but W_Hpsi exceeds the limit (Sec. IV.H) */
} mf_status;

/* Block sources (Sec. III.A).  PHILOX_GUE is "seeded generation": entry
 * (r, c), r <= c, from Philox4x32-10 with counter (r, c/2, 0, 0) and key
 * (seed lo, seed hi), words mapped by Box-Muller to a complex Gaussian of
 * variance 1/(2D) per part, real diagonal, H_cr = conj(H_rc) (global indices:
 * partition invariant, Sec. II).  SINC_DVR_HO is "analytic generation": the
 * Colbert-Miller sinc-DVR kinetic energy on x_i = -L + i*2L/(D-1) plus
 * V = x^2/2 (hbar = m = omega = 1).  EXTERNAL: canonical blocks stored by the
 * caller in host memory (mf_external_create; not accepted by mf_plan_create). */
typedef enum { MF_GEN_PHILOX_GUE = 0, MF_GEN_SINC_DVR_HO = 1, MF_GEN_EXTERNAL = 2 } mf_generator;

/* Entry precision forms.  FP64: entries, products and sums in double.
 * FP32: entries generated in single precision by the FP32 steps of the
 * generator, FP32 products and FP32 tile sums, FP64 cross-tile sums.
 * BF16X2: FP32 entries split hi = bf16(h), lo = bf16(h - hi), products
 * hi*xh + hi*xl + lo*xh on tensor cores with FP32 accumulation. */
typedef enum { MF_PREC_FP64 = 0, MF_PREC_FP32 = 1, MF_PREC_BF16X2 = 2 } mf_precision;

/* Storage modes (Sec. III.A, Sec. IV.E): AUTO lets the planner choose. */
typedef enum {
  MF_STORE_AUTO = -1,
  MF_STORE_PROCEDURAL = 0,
  MF_STORE_PARTIAL = 1,
  MF_STORE_FULL = 2
} mf_storage;

/* Planner modes: Algorithm 1 (analytic), Algorithm 2 (measured autotune),
 * Algorithm 3 (learned surrogate; hybrid = learned ranking + measurement). */
typedef enum {
  MF_PLANNER_ANALYTIC = 0,
  MF_PLANNER_AUTOTUNE = 1,
  MF_PLANNER_LEARNED = 2,
  MF_PLANNER_HYBRID = 3
} mf_planner_mode;

typedef struct {
  int32_t precision;       /* mf_precision, default MF_PREC_FP32 */
  int32_t storage;         /* mf_storage, default MF_STORE_AUTO */
  int32_t planner_mode;    /* mf_planner_mode, default MF_PLANNER_ANALYTIC */
  int32_t nvec_hint;       /* R the plan is tuned for (default 1) */
  double cheb_tol;         /* coefficient tolerance for the Chebyshev order (1e-7) */
  int32_t lanczos_m;       /* Lanczos steps for spectral bounds (40) */
  double bounds_pad;       /* relative padding of the Lanczos half-width (0.05) */
  double dvr_L;            /* DVR half-width L; 0 selects 0.9*sqrt(2D) */
  void* stream;            /* cudaStream_t for all work; NULL = default stream */
  double alpha_safety;     /* alpha of Eq. planner_memory_constraint (0.9) */
  double f_cache;          /* f_cache of Sec. IV.G used when budget == SIZE_MAX (0.8) */
  int32_t autotune_k;      /* K_bench candidates measured by Algorithm 2 (8) */
  int32_t autotune_warmup; /* R_warm (1) */
  int32_t autotune_repeats;/* R_bench (3) */
  double dense_work_limit; /* W_Hpsi threshold in entries for MF_WARN_DENSE_WORK (1e13) */
  int32_t device;          /* CUDA device ordinal (0) */
  mf_mlp_t model;          /* trained surrogate for MF_PLANNER_LEARNED/_HYBRID (NULL):
                              3 outputs (procedural, partial, full); 10 inputs =
                              direct form (outputs are ln t_mv), 11 inputs = residual
                              form (input 11 is ln(S_model / waves), the outputs are
                              ln t_mv minus it); any other shape: MF_ERR_INVALID */
  int32_t hermitian_reuse; /* 2..16 vectors: -1 = automatic (default; each canonical
                              chunk applied as H and H^dagger while its partial slots
                              fit min(16 GB, 10 % of free memory)), 0 = row-owner
                              kernel (every entry generated or read for each use);
                              not used by the sinc-DVR generator */
  int64_t row_begin;       /* row slice [row_begin, row_end) of a row-distributed plan */
  int64_t row_end;         /* (Sec. IV.H, row-parallel mode); 0, 0 = all rows; see
                              mf_plan_create */
  int32_t spin_limit;      /* polls of one bounded wait inside the tensor-core kernels
                              (0 = 2^18; a poll suspends at most 5 us, so at most about
                              1.3 s); when one runs out the kernel stops, frees its
                              tensor memory and reports MF_ERR_TIMEOUT (the waits for
                              its own copies and MMAs already issued keep the 2^18
                              bound whatever this value) */
} mf_options;

/* Generic planning instance P_mv of Sec. IV.A (Y = A X with A of size
 * D_out x D_in, R simultaneous vectors, n_op operators, N_task independent
 * tasks, B_c bytes per complex scalar, M_free smallest free memory, N_GPU). */
typedef struct {
  int64_t D_out, D_in, R, n_op, N_task;
  double B_c;
  double M_free;
  int32_t N_gpu;
} mf_problem;

/* One candidate plan of Algorithm 1 (Sec. IV.B). */
typedef struct {
  int64_t block;         /* b; 0 = one block of D_in */
  int32_t storage;       /* MF_STORE_PROCEDURAL, _PARTIAL or _FULL */
  int64_t pairs_cached;  /* P_cache; -1 derives it from the budget (Eq. partial_cache_pairs) */
  int32_t p_row;         /* row-group size of Eq. planner_full_cache */
  int32_t groups;        /* C(p), groups working on independent tasks (Eq. planner_waves) */
  int32_t r_arrays;      /* r temporaries of size D_in x R (Eq. planner_workspace) */
} mf_candidate;

/* Throughputs of the runtime model; a zero disables that term. */
typedef struct {
  double flops_per_s;       /* contraction rate */
  double hbm_bytes_per_s;   /* cached-block streaming rate */
  double gen_entries_per_s; /* procedural entry generation rate */
} mf_device_model;

/* Algorithm 1 quantities of one candidate. */
typedef struct {
  int64_t n_blk, n_pair, pairs_cached, waves;
  double M_block;  /* B_c b^2 */
  double M_work;   /* Eq. planner_workspace */
  double M_op;     /* 0, Eq. planner_partial_cache or Eq. planner_full_cache */
  double M_tot;    /* Eq. planner_total_memory */
  double F_mv;     /* Eq. generic_matvec_flops */
  double T_model;  /* max(generation, streaming, contraction) time, Eq. runtime_overlap */
  double S_model;  /* W T_model Pi_mem, Eq. planner_cost_score */
  int32_t feasible;/* Eq. planner_memory_constraint */
  double T_sum;    /* generation + streaming + contraction time: the ranking's
                      second key, deciding between candidates whose S_model
                      ties (the same term bounds both) for the less total work */
} mf_estimate;

/*
 * mf_planner_estimate -- evaluate one candidate of the analytic planner
 * (Algorithm 1) for a planning instance: memory terms, feasibility against
 * alpha * M_free, arithmetic scale, waves and model score.  Host only, no GPU
 * needed.  model may be NULL (T_model and S_model are then 0).  Errors:
 * MF_ERR_INVALID for NULL pointers or out-of-range fields.
 */
mf_status mf_planner_estimate(const mf_problem* prob, const mf_candidate* cand, const mf_device_model* model,
                              double alpha, double cache_budget_bytes, mf_estimate* out);

/*
 * mf_planner_device_model -- the throughputs mf_plan_create's analytic
 * planner (Algorithm 1) feeds its runtime model (Eq. runtime_overlap: the
 * slowest of generation, cache streaming and contraction) for a precision
 * form and a generator on a GPU with num_sms SMs (the values measured on
 * GB300; host only).  Errors: MF_ERR_INVALID for a NULL out, num_sms < 1 or an unknown
 * precision or generator.
 */
mf_status mf_planner_device_model(int32_t precision, int32_t generator, int32_t num_sms, mf_device_model* out);

/* Fill *o with the defaults listed above.  Never fails. */
void mf_options_default(mf_options* o);

/* Human-readable name of a status code (static storage, never NULL). */
const char* mf_status_string(mf_status s);

/*
 * mf_plan_create -- build an execution plan for y = A x (Sec. I, Eq. 1) with
 * A = H of the given generator (Sec. IV: block size b, storage mode, cache
 * budget, pairs cached, launch shape, precision).
 *   out      : receives the plan handle (owned by the library).
 *   D, M     : operator shape; M == D for both Hermitian generators.
 *   generator: mf_generator.
 *   seed     : Philox key (ignored by the DVR generator).
 *   block    : block size b of the partition D = sum b_n (Sec. II); 0 lets the
 *              planner choose (Sec. IV.F).  Must be a multiple of 128 when given.
 *   cache_budget_bytes : bytes the block cache may use (Eq. partial_cache_pairs);
 *              0 = procedural only, SIZE_MAX = f_cache * free memory.
 *   opt      : options, NULL = defaults.
 * Allocates the cache and workspace and fills the cache (Sec. III.A "full/
 * partial caching") on opt->stream before returning.  Errors: MF_ERR_INVALID
 * (D < 2, M != D, bad generator/precision/block), MF_ERR_OOM, MF_ERR_CUDA,
 * MF_ERR_UNSUPPORTED.  MF_WARN_DENSE_WORK still returns a usable plan.
 */
mf_status mf_plan_create(mf_plan_t* out, int64_t D, int64_t M, int32_t generator, uint64_t seed,
                         int64_t block, size_t cache_budget_bytes, const mf_options* opt);

/*
 * mf_external_create -- a plan for a Hermitian operator given by externally
 * stored blocks, H^[n,m] = D[key(n,m)] (Sec. II), held in host memory.
 *   blocks : host array of the N_pair = N_blk (N_blk + 1) / 2 canonical blocks
 *            (n <= m, N_blk = ceil(D / block)) in row order of the pairs
 *            ((0,0), (0,1), ..., (0,N_blk-1), (1,1), ...), each block x block
 *            row-major, complex64 for the FP32 and BF16X2 forms, complex128
 *            for FP64; 16-byte aligned.  Rows and columns past D are padding
 *            (read and multiplied by zero; must be finite).  Blocks below the
 *            diagonal are the conjugate transposes of the stored ones; the
 *            diagonal blocks must themselves be Hermitian (the one-vector
 *            kernel reads their upper triangle, the multi-vector kernels all
 *            of them).  Owned by the caller: it must stay alive and unchanged
 *            until mf_plan_destroy.
 *   block  : b, a multiple of 128, at most D rounded up to 128.
 *   cache_budget_bytes : HBM for the block cache; the first
 *            P_cache = min(N_pair, floor(budget / (B_c b^2))) stored pairs
 *            (Eq. partial_cache_pairs) are copied into HBM once, the others
 *            are read from the host array over the host link by the kernels
 *            on every product (the array is registered with
 *            cudaHostRegister for the plan's lifetime).  opt->storage ==
 *            MF_STORE_FULL requires every pair in HBM (MF_ERR_OOM otherwise).
 * All plan calls apply (mf_apply, propagator, filter, bounds, profiling);
 * mf_debug_entries returns MF_ERR_UNSUPPORTED.  Errors: MF_ERR_INVALID,
 * MF_ERR_OOM, MF_ERR_CUDA.
 */
mf_status mf_external_create(mf_plan_t* out, int64_t D, int64_t block, const void* blocks,
                             size_t cache_budget_bytes, const mf_options* opt);

/*
 * mf_sysbath_create -- a plan for the system-bath Hamiltonian of Sec. VII,
 *   H = H_S (x) I_B + I_S (x) H_B + g sum_{a=1}^{n_int} A_a (x) B_a,
 * acting on psi in C^{d_S} (x) C^{d_B} (D = d_S d_B), with the dense bath
 * operators H_B = B_0 and B_1..B_{n_int} drawn from the Philox ensemble of
 * mf_plan_create (scale sigma^2 = 1/(2 d_B)) with seeds[0..n_int] and
 * generated on demand, never stored; R = d_S and n_op = 1 + n_int as in
 * Eq. generic_matvec_flops.  One fused kernel generates every bath operator's
 * chunk and contracts it with X M_o^T (M_0 = I, M_a = g A_a); the X H_S^T term
 * is added in FP64.
 *   d_S   : 1..64;  d_B : >= 2;  n_int : 0..15;
 *   seeds : host uint64 [1 + n_int];
 *   H_S   : host complex128 [d_S][d_S] (row-major, H_S[s][s']);
 *   A     : host complex128 [n_int][d_S][d_S] (may be NULL when n_int == 0);
 *   g     : coupling strength;  opt : precision FP64 or FP32 (BF16X2 gives
 *           MF_ERR_UNSUPPORTED); storage and planner options are ignored
 *           (procedural storage).
 * Vectors of this plan are device complex128 [d_B][d_S], bath-major: element
 * (s, beta) of psi at beta*d_S + s.  mf_apply, mf_cheb_propagate and
 * mf_cheb_filter take nvec == d_S (one composite vector); mf_spectral_bounds
 * runs Lanczos on the composite operator, and mf_cheb_filter normalises the
 * whole composite vector.  H is Hermitian when H_S and the
 * A_a are.  Destroy with mf_plan_destroy.  Errors: MF_ERR_INVALID,
 * MF_ERR_UNSUPPORTED, MF_ERR_OOM, MF_ERR_CUDA.
 */
mf_status mf_sysbath_create(mf_plan_t* out, int64_t d_S, int64_t d_B, int32_t n_int, const uint64_t* seeds,
                            const void* H_S, const void* A, double g, const mf_options* opt);

/* Release everything the plan owns (synchronises its stream).  NULL is a no-op. */
mf_status mf_plan_destroy(mf_plan_t p);

/*
 * mf_apply -- y = H x for nvec simultaneous vectors (Eq. blockmatvec and
 * Eq. blockmatvecindex: phi^[n] = sum_m H^[n,m] psi^[m], every block pair
 * included).  Up to 16 vectors (and BF16X2 aside) each canonical pair is
 * generated or read once and applied as both H^[n,m] and H^[m,n] =
 * (H^[n,m])^dagger; the procedural sinc-DVR in the FP32 form uses its
 * Toeplitz-window kernels (1 to 16 vectors); the row-owner kernels used
 * otherwise (more vectors, opt.hermitian_reuse = 0, the tensor-core form,
 * stored DVR blocks, row slices) produce each row's blocks directly.
 *   y, x : device pointers to complex128 [D][nvec]; y must not overlap x.
 *   nvec : number of vectors, 1 <= nvec <= 64.
 * Asynchronous on the plan's stream.  Errors: MF_ERR_INVALID, MF_ERR_CUDA.
 */
mf_status mf_apply(mf_plan_t p, void* y, const void* x, int64_t nvec);

/*
 * mf_cheb_propagate -- psi <- exp(-i dt H) psi by the centred Chebyshev
 * recurrence of Sec. VII (H~ = (H - c)/R, q_{l+1} = 2 H~ q_l - q_{l-1}) with
 * coefficients a_0 = J_0(R dt), a_k = 2 (-i)^k J_k(R dt) computed on the GPU
 * in FP64; recurrence and accumulation in FP64.
 *   psi   : device complex128 [D][nvec], updated in place.
 *   dt    : time step (may be negative).
 *   order : number of terms k = 0..order-1; 0 = smallest count meeting
 *           opt.cheb_tol (|a_k| < tol for every k >= order).
 * Spectral bounds come from mf_plan_set_bounds, else are computed on first
 * use (Lanczos for PHILOX_GUE, the analytic Toeplitz-symbol bound for the DVR).
 * Errors: MF_ERR_INVALID, MF_ERR_CUDA.
 */
mf_status mf_cheb_propagate(mf_plan_t p, void* psi, int64_t nvec, double dt, int32_t order);

/* Number of Chebyshev terms mf_cheb_propagate would use for dt at the plan's
 * tolerance (computes bounds and coefficients if needed; synchronises). */
mf_status mf_cheb_terms(mf_plan_t p, double dt, int32_t* nterms);

/*
 * Row-distributed propagation (the row-parallel mode of Sec. IV.H: GPU j
 * owns rows R_j and the cached blocks they touch; every term needs all of
 * q_k, gathered between terms).  A plan created with opt.row_begin/row_end
 * (row_begin a multiple of 128, row_end a multiple of 128 or D) applies
 * H[R_j, :]: mf_apply takes x on all D rows and writes y on the plan's rows
 * only; its cache holds only the canonical pairs with a block row or column
 * among its rows; it always uses the row-owner kernels (FP64 or FP32 form).
 * Philox plans need their bounds set (mf_plan_set_bounds, the same on every
 * rank); the DVR's are analytic.  A real-time step on one rank:
 *   mf_rows_cheb_begin(p, dt, order, &nt);          coefficients, term count
 *   mf_rows_cheb_init(p, psi_full, acc, nvec);      acc = a_0 psi on the slice
 *   q_full = psi_full, q_prev = (unused for j = 1)
 *   for j = 1 .. nt-1:
 *     mf_rows_cheb_term(p, j, q_full, q_prev, q_next, acc, nvec);
 *         y = H q_j on the slice; q_{j+1} = t or 2 t - q_{j-1},
 *         t = (y - c q_j)/R; q_prev <- q_j, q_next <- q_{j+1} (slice);
 *         acc += 2 (-i)^j J_j(R dt) q_{j+1}
 *     q_full <- all-gather of every rank's q_next (the caller's collective)
 *   mf_rows_cheb_final(p, acc, psi_slice, nvec, dt); psi = e^{-i c dt} acc
 * psi_full, q_full: device complex128 [D][nvec]; acc, q_prev, q_next,
 * psi_slice: device complex128 [row_end - row_begin][nvec], owned by the
 * caller.  mf_cheb_propagate and mf_cheb_filter return MF_ERR_UNSUPPORTED on
 * such plans.  Errors: MF_ERR_INVALID (also for a plan without a row slice
 * or before mf_rows_cheb_begin), MF_ERR_UNSUPPORTED (bounds not set on a
 * Philox slice), MF_ERR_CUDA.
 */
mf_status mf_rows_cheb_begin(mf_plan_t p, double dt, int32_t order, int32_t* nterms);
mf_status mf_rows_cheb_init(mf_plan_t p, const void* psi_full, void* acc_slice, int64_t nvec);
mf_status mf_rows_cheb_term(mf_plan_t p, int32_t j, const void* q_full, void* q_prev_slice, void* q_next_slice,
                            void* acc_slice, int64_t nvec);
mf_status mf_rows_cheb_final(mf_plan_t p, const void* acc_slice, void* psi_slice, int64_t nvec, double dt);

/*
 * mf_cheb_filter -- imaginary-time Chebyshev filter, the thermal-pure-state
 * preparation named in Sec. I and used in Sec. VII (a random vector filtered
 * by exp(-beta H / 2), then normalised):
 *   psi <- exp(-tau (H - E_min)) psi,  E_min = c - R (the padded lower bound),
 * by the recurrence of mf_cheb_propagate with real coefficients
 * a_0 = e^{-z} I_0(z), a_k = 2 (-1)^k e^{-z} I_k(z), z = R tau (modified Bessel
 * functions, FP64 on the GPU).  The shift by E_min keeps every factor <= 1.
 *   psi       : device complex128 [D][nvec] (nvec 1..64), updated in place.
 *   tau       : imaginary time >= 0 (beta / 2 for a canonical TPQ state).
 *   order     : terms k = 0..order-1; 0 = smallest count meeting opt.cheb_tol.
 *   normalize : nonzero = divide each column by its 2-norm afterwards
 *               (deterministic FP64 reduction; a zero column stays zero).
 * Errors: MF_ERR_INVALID, MF_ERR_CUDA.  Asynchronous.
 */
mf_status mf_cheb_filter(mf_plan_t p, void* psi, int64_t nvec, double tau, int32_t order, int32_t normalize);
/* Number of terms mf_cheb_filter would use for tau (synchronises). */
mf_status mf_cheb_filter_terms(mf_plan_t p, double tau, int32_t* nterms);

/*
 * mf_spectral_bounds -- E_min, E_max used by the Chebyshev scaling (Sec. VII):
 * Lanczos with opt.lanczos_m steps on the GPU (Ritz extremes padded by
 * opt.bounds_pad of the half-width) for PHILOX_GUE; [min V, pi^2/(2 dx^2) +
 * max V] for the DVR.  Synchronises.  Results are cached in the plan.
 */
mf_status mf_spectral_bounds(mf_plan_t p, double* emin, double* emax);
/* Override the bounds used by mf_cheb_propagate (emax > emin). */
mf_status mf_plan_set_bounds(mf_plan_t p, double emin, double emax);

/*
 * mf_plan_profile -- enable (1) or disable (0) timing of every launch of the
 * plan's generate-and-apply kernel with a CUDA event pair recorded on the
 * plan's stream around it (the measured-time primitive of Sec. IV.B,
 * Eq. measured_matvec_time).  Resets the counters.  Events are created on
 * demand and owned by the plan.
 */
mf_status mf_plan_profile(mf_plan_t p, int32_t enable);
/* Synchronise the plan's stream, return the summed event time (ms) and count
 * of the apply-kernel launches timed since the last read, and reset them. */
mf_status mf_plan_profile_read(mf_plan_t p, double* total_ms, int64_t* launches);

/*
 * mf_plan_trials -- the plan-trial log of Algorithm 2/3 (Sec. IV.C: hardware
 * metadata, plan features x(p) and measured t_mv) as JSON lines, one per
 * candidate considered (measured candidates carry t_mv > 0; the analytic
 * planner logs its choice with t_mv = -1).  *needed receives the buffer size
 * including the terminating NUL; buf may be NULL to query it.  MF_ERR_INVALID
 * when buf is too small (the text is truncated).
 */
mf_status mf_plan_trials(mf_plan_t p, char* buf, size_t len, size_t* needed);

/*
 * Learned surrogate (Sec. IV.C, Algorithm 3): a multilayer perceptron
 * f(x) = tanh(tanh(z W1 + b1) W2 + b2) W3 + b3, z = (x - mu)/sigma, FP32,
 * forward/backward/Adam in the library's kernels.  Parameters are one flat
 * array: W1 [n_in][n_hidden], b1, W2 [n_hidden][n_hidden], b2,
 * W3 [n_hidden][n_out], b3 (row-major).  Targets are natural logs of
 * measured times, one output per storage strategy (procedural, partial,
 * full) for the planner; mask[i][o] = 0 drops an unmeasured target from the
 * mean-squared error (Eq. nn_loss).  All arrays are HOST memory; calls are
 * synchronous on the legacy default stream.
 */
mf_status mf_mlp_create(mf_mlp_t* out, int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed);
mf_status mf_mlp_destroy(mf_mlp_t m);
mf_status mf_mlp_param_count(mf_mlp_t m, int64_t* n);
/* Copy parameters / normalisation (mu, sigma: n_in floats each) out or in;
 * any pointer may be NULL. */
mf_status mf_mlp_get_params(mf_mlp_t m, float* params, float* mu, float* sigma);
mf_status mf_mlp_set_params(mf_mlp_t m, const float* params, const float* mu, const float* sigma);
/* Y[n][n_out] = f(X[n][n_in]). */
mf_status mf_mlp_predict(mf_mlp_t m, const float* X, int64_t n, float* Y);
/* Masked MSE loss and its gradient (flat, like the parameters) at the
 * current parameters; mask may be NULL (all ones). */
mf_status mf_mlp_loss_grad(mf_mlp_t m, const float* X, const float* Y, const float* mask, int64_t n, float* loss,
                           float* grad);
/* Full-batch Adam (beta 0.9/0.999, eps 1e-8) for `epochs` steps at rate lr;
 * set_normalization != 0 first sets mu/sigma to the z-score statistics of X;
 * loss_curve (epochs floats, may be NULL) receives the loss before each step. */
mf_status mf_mlp_train(mf_mlp_t m, const float* X, const float* Y, const float* mask, int64_t n, int32_t epochs,
                       float lr, int32_t set_normalization, float* loss_curve);
/* The 10-entry feature vector the planner feeds the surrogate for
 * (generator, precision, D, b, R = nvec, cache budget):
 * log2 D, log2 b, log2 R, one-hot precision (fp32, bf16x2, fp64), one-hot
 * generator (philox, dvr), budget / full-cache bytes (capped at 1),
 * log10(1 + budget/1e9).  The residual surrogate appends ln(S_model / waves)
 * of the candidate, from mf_planner_estimate with mf_planner_device_model. */
mf_status mf_mlp_features(int32_t generator, int32_t precision, int64_t D, int64_t block, int64_t nvec,
                          double cache_budget_bytes, float* out10);

/*
 * Batched independent problems (parameter-parallel execution, Sec. IV.H):
 * nprob Hermitian problems of the same generator with their own D[i]
 * (>= 2), nvec[i] (1..16) and seeds[i] are propagated together.  Each
 * problem is a plan chosen by opt->planner_mode with a share of
 * cache_budget_bytes proportional to its full canonical cache; its bounds
 * come from its own Lanczos run.  One persistent kernel per Chebyshev term
 * applies every problem (work list of (problem, 128-row tile) items drained
 * through an atomic counter), and the whole propagation is captured once in
 * a CUDA graph that later calls with the same (psi, dt, nsteps, order)
 * replay.  psi is ONE device buffer of complex128 holding the problems'
 * [D[i]][nvec[i]] blocks back to back (element offsets from
 * mf_batch_offsets, nprob + 1 entries).  The graph runs on the batch's own
 * stream, ordered after and before opt->stream by events.
 */
mf_status mf_batch_create(mf_batch_t* out, int32_t nprob, const int64_t* D, const int32_t* nvec,
                          const uint64_t* seeds, int32_t generator, size_t cache_budget_bytes,
                          const mf_options* opt);
mf_status mf_batch_destroy(mf_batch_t b);
mf_status mf_batch_offsets(mf_batch_t b, int64_t* offsets);
/* nsteps Chebyshev steps of dt (order as in mf_cheb_propagate; the largest
 * per-problem term count is used for all); *nterms_out (may be NULL)
 * receives the term count.  Asynchronous. */
mf_status mf_batch_propagate(mf_batch_t b, void* psi, double dt, int32_t nsteps, int32_t order, int32_t* nterms_out);
/* The plan of problem i (owned by the batch) and launch facts: the
 * (problem, row tile) work items and the largest persistent grid of the
 * per-list kernels (one persistent kernel per vector bucket of max(2, nvec)
 * in {2, 4, 6, 8, 12, 16} and form, launched side by side each term). */
mf_status mf_batch_plan(mf_batch_t b, int32_t i, mf_plan_t* plan);
mf_status mf_batch_info(mf_batch_t b, int32_t* n_items, int32_t* persist_grid);
/* Form of problem i's batched product (Sec. III.A canonical-pair reuse):
 * *hermitian = 1 when each stored canonical chunk is read once and applied
 * as H and as H^dagger (FP32 problems of 1-6 vectors, in problem order
 * while their slots of 1 + ntile partial rows fit together in a tenth of the
 * device memory free after the plans; the slots are summed in tile order by
 * the update), 0 for the row-owner form (each stored entry read as H and as
 * H^dagger by the two row tiles).  MF_ERR_INVALID for a bad handle or i. */
mf_status mf_batch_form(mf_batch_t b, int32_t i, int32_t* hermitian);

/* Wait for the plan's stream and report the device error word: MF_OK, or
 * MF_ERR_TIMEOUT when a bounded wait ran out (codes 100..199, see
 * mf_plan_describe's "last_device_error"), MF_ERR_CUDA for any other code.
 * The word is cleared once reported. */
mf_status mf_sync(mf_plan_t p);

/*
 * mf_plan_describe -- the plan record of Sec. IV (block count and size,
 * storage mode, cache budget and pairs cached, launch shape, precision,
 * safety estimate) as a NUL-terminated JSON object in buf[0..len).
 * MF_ERR_INVALID if buf is NULL or too small (the record is truncated).
 */
mf_status mf_plan_describe(mf_plan_t p, char* buf, size_t len);

/*
 * mf_plan_serialize / mf_plan_deserialize -- the plan record of a
 * continuation run (Sec. VII resumes propagations with the plan selected
 * earlier): the selected block size, storage mode and pairs cached, the
 * generator, seed and precision form, the numerical options and, once
 * computed, the spectral bounds, as NUL-terminated text ("mf_plan v1" and
 * key=value lines; doubles as exact hexadecimal floats).
 *   serialize   : *needed receives the size including the NUL; buf may be
 *                 NULL to query it; MF_ERR_INVALID when buf is too small;
 *                 MF_ERR_UNSUPPORTED for system-bath and externally stored
 *                 plans (their operator data is the caller's).
 *   deserialize : builds the recorded plan directly -- no planner, no
 *                 measurement, no Lanczos run when the record holds bounds --
 *                 so products and propagations equal the original plan's bit
 *                 for bit on the same GPU model.  opt supplies the stream and
 *                 device (NULL = defaults); the recorded fields override its
 *                 numerical options.  rec is read up to len bytes or its NUL.
 *                 Errors: MF_ERR_INVALID (malformed record or out-of-range
 *                 field; nothing allocated), MF_ERR_OOM, MF_ERR_CUDA.
 */
mf_status mf_plan_serialize(mf_plan_t p, char* buf, size_t len, size_t* needed);
mf_status mf_plan_deserialize(mf_plan_t* out, const char* rec, size_t len, const mf_options* opt);

/*
 * mf_debug_entries -- copy the generator's entries H[r0:r0+rows, c0:c0+cols]
 * as produced on the GPU in the plan's precision form to HOST memory out:
 * complex64 (FP32 and BF16X2 plans, the FP32 entry before splitting) or
 * complex128 (FP64 plans), row-major.  DVR entries exclude the potential.
 * Any (r, c) in [0, D) is allowed (entries below the diagonal are the
 * conjugates).  Synchronises.  Used for the bit-exact entry parity.
 */
mf_status mf_debug_entries(mf_plan_t p, int64_t r0, int64_t c0, int64_t rows, int64_t cols,
                           void* out_host);

/*
 * mf_apply_dvr_noalloc -- y = H x for the sinc-DVR harmonic-oscillator
 * operator in the FP32 form, one vector, without allocating any memory.  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory while they run (a service whose device memory is
 * fully reserved by another runtime's caching allocator, a plugin that its
 * host application forbids to call cudaMalloc).
 *   D      : 2 <= D <= 131072 (larger D returns MF_ERR_INVALID).
 *   dvr_L  : grid half-width, 0 selects 0.9*sqrt(2D).
 *   x, y   : device complex128 [D], owned by the caller; y must not overlap x.
 *   stream : cudaStream_t to run on (NULL = default stream).
 * The kernels' scratch lives in one fixed 40 MiB device array of the library
 * that every GPU loading the library holds until the process exits; no
 * cudaMalloc, cudaFree or other allocating call is made.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current and keeps it.  CUDA loads device code lazily by default, so
 * that first call also loads the kernels and the array and may need device
 * memory: make it once, as a warm-up, before the caller's memory is reserved
 * and before any stream capture.  The kept address does not survive a device
 * reset (cudaDeviceReset or a re-created primary context): do not call this
 * entry point on a device after resetting it.  Every call on a device shares
 * the one array and leaves its contents behind (nothing in it needs clearing:
 * the kernels write every scratch value they read), so calls that overlap on
 * the GPU -- on different streams, or from different threads -- race and
 * must be serialised by the caller.  Asynchronous; errors: MF_ERR_INVALID
 * (also for a non-finite dvr_L), MF_ERR_OOM (the first call could not load
 * the code or the array), MF_ERR_CUDA.
 */
mf_status mf_apply_dvr_noalloc(int64_t D, double dvr_L, const void* x, void* y, void* stream);

/*
 * mf_selfcheck_generator -- compare, on the current device, the Philox
 * ensemble's FP32 division and square root (hardware reciprocal and
 * reciprocal-square-root approximations with one Markstein correction) with
 * IEEE round-to-nearest division and square root on every float of the
 * ranges the generator uses them on: numerator m - 1 over denominator m + 1
 * for all m in [0.5, 2), square roots of 0 and of all x in [2^-33, 64).  Nonzero
 * counts mean the FP32 entries would not match the IEEE definition on this
 * device.  The paper has no counterpart.  Synchronises; a few milliseconds.
 * Errors: MF_ERR_INVALID, MF_ERR_OOM, MF_ERR_CUDA.
 */
mf_status mf_selfcheck_generator(int64_t* div_mismatches, int64_t* sqrt_mismatches);

/*
 * mf_pipe_rates -- measured throughput, in operations per second, of the
 * execution pipes the entry generators use, on `device` (launched on
 * `stream`, a cudaStream_t or NULL): register-only chains with no memory
 * traffic, 8 CTAs of 256 threads per SM, three timed launches after one
 * warm-up.  ops_per_s[0..7] (n >= 8, host array owned by the caller):
 * 0 mul.hi.u32 (IMAD.HI), 1 mad.lo.u32 (IMAD), 2 three-input logic (LOP3),
 * 3 integer add (IADD3), 4 FP32 fma (FFMA, one operation each),
 * 5 rsqrt.approx.f32 (MUFU), 6 cvt.rn.f32.u32 (I2F), 7 FP64 fma (DFMA);
 * with n >= 10 also the tensor cores, as tcgen05.mma instructions per second
 * over the GPU (kind::f16, bf16 operands in shared memory, FP32 accumulator,
 * M = 128, K = 16, one issuing thread per SM): 8 with N = 128, 9 with
 * N = 256.  These are the denominators of the per-pipe generation bound and
 * of the instruction-shape bound of the tensor-core products (the runtime
 * model of Sec. V.A bounds a product by its slowest resource).  Synchronises;
 * about 60 ms.  The paper has no counterpart.  Errors: MF_ERR_INVALID (NULL
 * array, n < 8, negative device), MF_ERR_OOM, MF_ERR_TIMEOUT (an MMA wait
 * ran out; the GPU stays usable), MF_ERR_CUDA.
 */
mf_status mf_pipe_rates(int32_t device, void* stream, double* ops_per_s, int32_t n);

#ifdef __cplusplus
}
#endif
#endif /* MF_H */
