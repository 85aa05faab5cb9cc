/*
 * mf_oracle.h -- plain CPU oracle for the block-procedural H*psi product.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this file; only the tests, the package smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code with the CUDA path.
 *
 * Every routine is a direct, unblocked, unfused statement of a definition
 * (see the comment above each one for the passage of the paper it follows).
 * Complex vectors are interleaved (re, im) doubles, row-major [D][nvec] with
 * the vector index fastest, matching the product ABI.
 */
#ifndef MF_ORACLE_H
#define MF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_GEN_PHILOX_GUE = 0, OR_GEN_SINC_DVR_HO = 1 };
/* Entry precision forms: FP64 is the reference operator; FP32 is the operator
 * whose entries are generated in single precision by the stated FP32 steps. */
enum { OR_FORM_FP64 = 0, OR_FORM_FP32 = 1 };

typedef struct {
  int32_t gen;     /* OR_GEN_* */
  int32_t form;    /* OR_FORM_* */
  uint64_t seed;   /* Philox key (lo word, hi word) */
  int64_t D;       /* dimension */
  double L;        /* DVR half-width of the grid [-L, L] */
} or_op;

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Project-defined elementary functions (polynomial, fixed operation order). */
double or_log(double u);
float or_logf(float u);
void or_sincos_2pi(double u, double* s, double* c);
void or_sincos_2pif(float u, float* s, float* c);

/* Single entries H_rc of the operator in the given form, as doubles. */
void or_entry(const or_op* op, int64_t r, int64_t c, double* re, double* im);
/* Form-native entries: the FP32 form returned without widening. */
void or_entry_f32(const or_op* op, int64_t r, int64_t c, float* re, float* im);
/* DVR: kinetic entry T(k), k = r - c, in the op's form (widened to double). */
double or_dvr_kinetic(const or_op* op, int64_t k);
/* DVR: the diagonal potential V_i = x_i^2/2 (always FP64). */
double or_dvr_potential(const or_op* op, int64_t i);

/* Dense window H[r0:r0+rows, c0:c0+cols] in complex128 (row-major). */
void or_window(const or_op* op, int64_t r0, int64_t c0, int64_t rows, int64_t cols, double* out);
/* Same window in the FP32 form's native precision: complex64 (row-major). */
void or_window_f32(const or_op* op, int64_t r0, int64_t c0, int64_t rows, int64_t cols, float* out);

/* y = H x, blockwise (block size b), FP64 accumulation. nthreads<=0: all. */
void or_apply(const or_op* op, int64_t b, int64_t nvec, const double* x, double* y, int nthreads);
/* Selected output rows only: y[k][:] = (H x)[rows[k]][:]. */
void or_apply_rows(const or_op* op, int64_t nvec, const double* x, int64_t nrows,
                   const int64_t* rows, double* y, int nthreads);

/* Bessel J_0..J_K(x) by Miller's backward recurrence. */
void or_bessel_j(double x, int32_t K, double* J);
/* Scaled modified Bessel functions exp(-x) I_k(x), k = 0..K (Miller). */
void or_bessel_i_scaled(double x, int32_t K, double* I);
/* Imaginary-time filter psi <- exp(-tau (H - Emin)) psi, Emin = c - R, with
 * nterms terms; columns renormalised to unit norm when normalize != 0. */
void or_cheb_imag_step(const or_op* op, int64_t b, int64_t nvec, double* psi, double tau, double c, double R,
                       int32_t nterms, int normalize, int nthreads);
/* Number of Chebyshev terms for argument z = R*dt at tolerance tol. */
int32_t or_cheb_terms(double z, double tol);
/* One Chebyshev step psi <- exp(-i dt H) psi with nterms terms (k = 0..nterms-1),
 * spectral centre c and half-width R; uses or_apply. */
void or_cheb_step(const or_op* op, int64_t b, int64_t nvec, double* psi, double dt,
                  double c, double R, int32_t nterms, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
