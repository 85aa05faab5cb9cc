/*
 * mf_oracle.c -- plain, slow, obviously correct CPU oracle (FP64 unless a form
 * says otherwise) for the block-procedural Hamiltonian-vector product of
 * "Memory-Scalable and Hardware-Adaptive Matrix-Free Quantum Simulation"
 * (Shafir & Kosloff).
 *
 * TEST INFRASTRUCTURE ONLY: only tests/, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA path; the two meet only through seeded inputs.
 *
 * Compile with -ffp-contract=off: every fused multiply-add below is an explicit
 * fma()/fmaf() call and every other operation rounds on its own, so the entry
 * generators follow one fixed sequence of IEEE operations.
 *
 * Parity status per function: all functions are pinned by tests (Philox
 * known-answer vectors, math-library comparisons, dense brute force,
 * closed-form spectra, scipy Bessel values, eigendecomposition).
 */
#include "mf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 -- Salmon et al., SC'11, Sec. 4: a 10-round Feistel-like     */
/* network on four 32-bit words; each round multiplies words 0 and 2 by the   */
/* constants M0, M1 (keeping both halves of the 64-bit product), XORs the     */
/* high halves with the other words and the round key, and permutes; the key  */
/* is bumped by the Weyl constants W0, W1 between rounds.                     */
/* ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------- */
/* Natural logarithm of a normal positive u (project definition).           */
/* u = m * 2^e with m in (sqrt(1/2), sqrt(2)]; ln m = 2 atanh(s),            */
/* s = (m-1)/(m+1), atanh(s)/s = sum_k z^k/(2k+1), z = s^2, evaluated by      */
/* Horner with fused multiply-adds; ln u = e*ln2 + ln m in one final fma.    */
/* ------------------------------------------------------------------------- */
static double u64_as_f64(uint64_t b) { double d; memcpy(&d, &b, 8); return d; }
static uint64_t f64_as_u64(double d) { uint64_t b; memcpy(&b, &d, 8); return b; }
static float u32_as_f32(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t f32_as_u32(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

double or_log(double u) {
  /* 1/(2k+1), k = 0..10, each the double nearest the rational */
  static const double A[11] = {
      0x1.0000000000000p+0, 0x1.5555555555555p-2, 0x1.999999999999ap-3,
      0x1.2492492492492p-3, 0x1.c71c71c71c71cp-4, 0x1.745d1745d1746p-4,
      0x1.3b13b13b13b14p-4, 0x1.1111111111111p-4, 0x1.e1e1e1e1e1e1ep-5,
      0x1.af286bca1af28p-5, 0x1.8618618618618p-5};
  const double LN2 = 0x1.62e42fefa39efp-1;
  const double SQRT2 = 0x1.6a09e667f3bcdp+0;
  uint64_t bits = f64_as_u64(u);
  int e = (int)((bits >> 52) & 0x7ff) - 1023;
  double m = u64_as_f64((bits & 0x000fffffffffffffull) | 0x3ff0000000000000ull);
  if (m > SQRT2) { m = m * 0.5; e = e + 1; }
  double s = (m - 1.0) / (m + 1.0);
  double z = s * s;
  double p = A[10];
  for (int k = 9; k >= 0; --k) p = fma(p, z, A[k]);
  double t = s * p;
  return fma((double)e, LN2, 2.0 * t);
}

float or_logf(float u) {
  static const float A[6] = {0x1.000000p+0f, 0x1.555556p-2f, 0x1.99999ap-3f,
                             0x1.24924ap-3f, 0x1.c71c72p-4f, 0x1.745d18p-4f};
  const float LN2 = 0x1.62e430p-1f;
  const float SQRT2 = 0x1.6a09e6p+0f;
  uint32_t bits = f32_as_u32(u);
  int e = (int)((bits >> 23) & 0xff) - 127;
  float m = u32_as_f32((bits & 0x007fffffu) | 0x3f800000u);
  if (m > SQRT2) { m = m * 0.5f; e = e + 1; }
  float s = (m - 1.0f) / (m + 1.0f);
  float z = s * s;
  float p = A[5];
  for (int k = 4; k >= 0; --k) p = fmaf(p, z, A[k]);
  float t = s * p;
  return fmaf((float)e, LN2, 2.0f * t);
}

/* ------------------------------------------------------------------------- */
/* sin(2 pi u), cos(2 pi u) for u in [0,1) (project definition).             */
/* v = 4u = q + f with q the quadrant (exact), f in [0,1) (exact); f is       */
/* reflected to 1-f when above 1/2 so that x = f*pi/2 lies in [0, pi/4];     */
/* Taylor series sin x = x * sum (-1)^k z^k/(2k+1)!, cos x = sum             */
/* (-1)^k z^k/(2k)!, z = x^2, by Horner with fmas; then the quadrant turn.    */
/* ------------------------------------------------------------------------- */
void or_sincos_2pi(double u, double* s_out, double* c_out) {
  static const double S[10] = {
      0x1.0000000000000p+0, -0x1.5555555555555p-3, 0x1.1111111111111p-7,
      -0x1.a01a01a01a01ap-13, 0x1.71de3a556c734p-19, -0x1.ae64567f544e4p-26,
      0x1.6124613a86d09p-33, -0x1.ae7f3e733b81fp-41, 0x1.952c77030ad4ap-49,
      -0x1.2f49b46814157p-57};
  static const double C[10] = {
      0x1.0000000000000p+0, -0x1.0000000000000p-1, 0x1.5555555555555p-5,
      -0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-16, -0x1.27e4fb7789f5cp-22,
      0x1.1eed8eff8d898p-29, -0x1.93974a8c07c9dp-37, 0x1.ae7f3e733b81fp-45,
      -0x1.6827863b97d97p-53};
  const double PIO2 = 0x1.921fb54442d18p+0;
  double v = 4.0 * u;
  int q = (int)v;
  double f = v - (double)q;
  int refl = f > 0.5;
  if (refl) f = 1.0 - f;
  double x = f * PIO2;
  double z = x * x;
  double ps = S[9];
  for (int k = 8; k >= 0; --k) ps = fma(ps, z, S[k]);
  double pc = C[9];
  for (int k = 8; k >= 0; --k) pc = fma(pc, z, C[k]);
  double sx = x * ps, cx = pc;
  double sb = refl ? cx : sx; /* sin(f0 pi/2) with f0 the unreflected f */
  double cb = refl ? sx : cx;
  switch (q & 3) {
    case 0: *s_out = sb; *c_out = cb; break;
    case 1: *s_out = cb; *c_out = -sb; break;
    case 2: *s_out = -sb; *c_out = -cb; break;
    default: *s_out = -cb; *c_out = sb; break;
  }
}

void or_sincos_2pif(float u, float* s_out, float* c_out) {
  static const float S[6] = {0x1.000000p+0f, -0x1.555556p-3f, 0x1.111112p-7f,
                             -0x1.a01a02p-13f, 0x1.71de3ap-19f, -0x1.ae6456p-26f};
  static const float C[7] = {0x1.000000p+0f, -0x1.000000p-1f, 0x1.555556p-5f,
                             -0x1.6c16c2p-10f, 0x1.a01a02p-16f, -0x1.27e4fcp-22f,
                             0x1.1eed8ep-29f};
  const float PIO2 = 0x1.921fb6p+0f;
  float v = 4.0f * u;
  int q = (int)v;
  float f = v - (float)q;
  int refl = f > 0.5f;
  if (refl) f = 1.0f - f;
  float x = f * PIO2;
  float z = x * x;
  float ps = S[5];
  for (int k = 4; k >= 0; --k) ps = fmaf(ps, z, S[k]);
  float pc = C[6];
  for (int k = 5; k >= 0; --k) pc = fmaf(pc, z, C[k]);
  float sx = x * ps, cx = pc;
  float sb = refl ? cx : sx;
  float cb = refl ? sx : cx;
  switch (q & 3) {
    case 0: *s_out = sb; *c_out = cb; break;
    case 1: *s_out = cb; *c_out = -sb; break;
    case 2: *s_out = -sb; *c_out = -cb; break;
    default: *s_out = -cb; *c_out = sb; break;
  }
}

/* ------------------------------------------------------------------------- */
/* Seeded generation (Sec. III.A "Seeded generation", Eq. for G_seed) made   */
/* partition invariant (Sec. II, on indexing the generator by global row and */
/* column).  For the canonical entry r <= c: Philox4x32-10 with counter       */
/* (r, floor(c/2), 0, 0) and key (seed lo, seed hi); words 0,1 feed column    */
/* 2*floor(c/2), words 2,3 column 2*floor(c/2)+1.  Box-Muller: u_a, u_b in    */
/* (0,1); rho = sqrt(-2 ln u_a), theta = 2 pi u_b; H_rc = sigma*rho*(cos,     */
/* sin), sigma^2 = 1/(2D); the diagonal keeps the real part; H_cr = conj.     */
/* FP64 form: u = (w + 1/2) 2^-32 (exact).  FP32 form: u = float nearest to */
/* (2w + 1) 2^-33 (one rounding of the same value), then the same steps in   */
/* single precision.                                                          */
/* ------------------------------------------------------------------------- */
static void gue_words(uint64_t seed, int64_t r, int64_t c, uint32_t* wa, uint32_t* wb) {
  uint32_t ctr[4] = {(uint32_t)r, (uint32_t)(c >> 1), 0u, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t w[4];
  or_philox4x32_10(ctr, key, w);
  if (c & 1) { *wa = w[2]; *wb = w[3]; } else { *wa = w[0]; *wb = w[1]; }
}

static void gue_entry64(uint64_t seed, int64_t D, int64_t r, int64_t c, double* re, double* im) {
  int conj = 0;
  if (r > c) { int64_t t = r; r = c; c = t; conj = 1; }
  uint32_t wa, wb;
  gue_words(seed, r, c, &wa, &wb);
  double ua = ((double)wa + 0.5) * 0x1p-32;
  double ub = ((double)wb + 0.5) * 0x1p-32;
  double rho = sqrt(-2.0 * or_log(ua));
  double sn, cs;
  or_sincos_2pi(ub, &sn, &cs);
  double sigma = sqrt(0.5 / (double)D);
  double a = sigma * rho;
  *re = a * cs;
  *im = (r == c) ? 0.0 : (conj ? -(a * sn) : a * sn);
}

static void gue_entry32(uint64_t seed, int64_t D, int64_t r, int64_t c, float* re, float* im) {
  int conj = 0;
  if (r > c) { int64_t t = r; r = c; c = t; conj = 1; }
  uint32_t wa, wb;
  gue_words(seed, r, c, &wa, &wb);
  float ua = (float)(2ull * (uint64_t)wa + 1ull) * 0x1p-33f;
  float ub = (float)(2ull * (uint64_t)wb + 1ull) * 0x1p-33f;
  float rho = sqrtf(-2.0f * or_logf(ua));
  float sn, cs;
  or_sincos_2pif(ub, &sn, &cs);
  float sigma = sqrtf(0.5f / (float)D);
  float a = sigma * rho;
  *re = a * cs;
  *im = (r == c) ? 0.0f : (conj ? -(a * sn) : a * sn);
}

/* ------------------------------------------------------------------------- */
/* Analytic generation (Sec. III.A "Analytic generation"): the Colbert-Miller */
/* sinc-DVR kinetic energy on the infinite interval (J. Chem. Phys. 96, 1982, */
/* 1992) with hbar = m = 1 on the grid x_i = -L + i dx, dx = 2L/(D-1):        */
/* T_ii = pi^2/(6 dx^2), T_ij = (-1)^(i-j) / (dx^2 (i-j)^2), plus the         */
/* harmonic potential V_i = x_i^2/2 on the diagonal.                          */
/* FP64 form: the formulas in double.  FP32 form of T: c32 = float(1/dx^2),   */
/* T32(0) = float(pi^2/(6 dx^2)), T32(k) = (-1)^k c32 / float(k^2); the       */
/* potential stays in FP64 in both forms.                                     */
/* ------------------------------------------------------------------------- */
static double dvr_dx(const or_op* op) { return (2.0 * op->L) / (double)(op->D - 1); }

static double dvr_T64(const or_op* op, int64_t k) {
  const double PI2_6 = 0x1.a51a6625307d3p+0; /* pi^2/6 */
  double dx = dvr_dx(op);
  double dx2 = dx * dx;
  if (k == 0) return PI2_6 / dx2;
  int64_t k2 = k * k;
  double t = 1.0 / (dx2 * (double)k2);
  return (k & 1) ? -t : t;
}

static float dvr_T32(const or_op* op, int64_t k) {
  const double PI2_6 = 0x1.a51a6625307d3p+0;
  double dx = dvr_dx(op);
  double dx2 = dx * dx;
  if (k == 0) return (float)(PI2_6 / dx2);
  float c32 = (float)(1.0 / dx2);
  int64_t k2 = k * k;
  float t = c32 / (float)k2;
  return (k & 1) ? -t : t;
}

double or_dvr_potential(const or_op* op, int64_t i) {
  double dx = dvr_dx(op);
  double x = -op->L + (double)i * dx;
  return 0.5 * (x * x);
}

double or_dvr_kinetic(const or_op* op, int64_t k) {
  return op->form == OR_FORM_FP64 ? dvr_T64(op, k) : (double)dvr_T32(op, k);
}

void or_entry_f32(const or_op* op, int64_t r, int64_t c, float* re, float* im) {
  if (op->gen == OR_GEN_PHILOX_GUE) {
    gue_entry32(op->seed, op->D, r, c, re, im);
  } else {
    *re = dvr_T32(op, r - c);
    *im = 0.0f;
  }
}

void or_entry(const or_op* op, int64_t r, int64_t c, double* re, double* im) {
  if (op->gen == OR_GEN_PHILOX_GUE) {
    if (op->form == OR_FORM_FP64) {
      gue_entry64(op->seed, op->D, r, c, re, im);
    } else {
      float a, b;
      gue_entry32(op->seed, op->D, r, c, &a, &b);
      *re = (double)a; *im = (double)b;
    }
  } else {
    double t = (op->form == OR_FORM_FP64) ? dvr_T64(op, r - c) : (double)dvr_T32(op, r - c);
    *re = (r == c) ? t + or_dvr_potential(op, r) : t;
    *im = 0.0;
  }
}

void or_window(const or_op* op, int64_t r0, int64_t c0, int64_t rows, int64_t cols, double* out) {
  for (int64_t a = 0; a < rows; ++a)
    for (int64_t b = 0; b < cols; ++b)
      or_entry(op, r0 + a, c0 + b, &out[2 * (a * cols + b)], &out[2 * (a * cols + b) + 1]);
}

void or_window_f32(const or_op* op, int64_t r0, int64_t c0, int64_t rows, int64_t cols, float* out) {
  for (int64_t a = 0; a < rows; ++a)
    for (int64_t b = 0; b < cols; ++b)
      or_entry_f32(op, r0 + a, c0 + b, &out[2 * (a * cols + b)], &out[2 * (a * cols + b) + 1]);
}

/* ------------------------------------------------------------------------- */
/* Block matvec, Eq. (blockmatvecindex): phi^[n]_alpha = sum_m sum_beta       */
/* H^[n,m]_{alpha beta} psi^[m]_beta, all blocks m included (dense, exact).   */
/* Output rows are independent, so threads split them.                        */
/* ------------------------------------------------------------------------- */
static void apply_row(const or_op* op, int64_t b, int64_t nvec, const double* x, int64_t i,
                      double* yrow) {
  const int64_t D = op->D;
  const int64_t nblk = (D + b - 1) / b;
  for (int64_t v = 0; v < nvec; ++v) { yrow[2 * v] = 0.0; yrow[2 * v + 1] = 0.0; }
  for (int64_t m = 0; m < nblk; ++m) {
    int64_t c_end = (m + 1) * b < D ? (m + 1) * b : D;
    for (int64_t j = m * b; j < c_end; ++j) {
      double hr, hi;
      or_entry(op, i, j, &hr, &hi);
      for (int64_t v = 0; v < nvec; ++v) {
        double xr = x[2 * (j * nvec + v)], xi = x[2 * (j * nvec + v) + 1];
        yrow[2 * v] += hr * xr - hi * xi;
        yrow[2 * v + 1] += hr * xi + hi * xr;
      }
    }
  }
}

void or_apply(const or_op* op, int64_t b, int64_t nvec, const double* x, double* y, int nthreads) {
  const int64_t D = op->D;
  if (b <= 0) b = D;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
#endif
  for (int64_t i = 0; i < D; ++i) apply_row(op, b, nvec, x, i, &y[2 * i * nvec]);
  (void)nthreads;
}

void or_apply_rows(const or_op* op, int64_t nvec, const double* x, int64_t nrows,
                   const int64_t* rows, double* y, int nthreads) {
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
  for (int64_t k = 0; k < nrows; ++k) apply_row(op, op->D, nvec, x, rows[k], &y[2 * k * nvec]);
  (void)nthreads;
}

/* ------------------------------------------------------------------------- */
/* Bessel functions J_k(x), k = 0..K, by Miller's backward recurrence          */
/* J_{k-1} = (2k/x) J_k - J_{k+1} started far above max(K, x), rescaled       */
/* against overflow, normalised by J_0 + 2 sum_{k>=1} J_{2k} = 1.  These are   */
/* the Chebyshev coefficients of exp(-i z x) (Tal-Ezer & Kosloff 1984, cited   */
/* in Sec. VII for the centred Chebyshev propagator).                         */
/* ------------------------------------------------------------------------- */
void or_bessel_j(double x, int32_t K, double* J) {
  if (x == 0.0) {
    J[0] = 1.0;
    for (int32_t k = 1; k <= K; ++k) J[k] = 0.0;
    return;
  }
  int64_t top = (int64_t)K > (int64_t)ceil(x) ? (int64_t)K : (int64_t)ceil(x);
  int64_t N = top + 30 + (int64_t)(20.0 * cbrt(x + 1.0));
  if (N & 1) N += 1;
  double jp1 = 0.0, j = 1.0, norm = 0.0;
  for (int32_t k = 0; k <= K; ++k) J[k] = 0.0;
  if (N <= K) J[N] = j;
  if ((N & 1) == 0) norm += 2.0 * j;
  for (int64_t k = N; k >= 1; --k) {
    double jm1 = (2.0 * (double)k / x) * j - jp1;
    jp1 = j;
    j = jm1;
    int64_t idx = k - 1;
    if (idx <= K) J[idx] = j;
    if (idx == 0) norm += j;
    else if ((idx & 1) == 0) norm += 2.0 * j;
    if (fabs(j) > 1e250) {
      const double s = 1e-250;
      j *= s; jp1 *= s; norm *= s;
      for (int64_t q = idx; q <= K; ++q) J[q] *= s;
    }
  }
  for (int32_t k = 0; k <= K; ++k) J[k] /= norm;
}

/* ------------------------------------------------------------------------- */
/* Scaled modified Bessel functions exp(-x) I_k(x), k = 0..K, by Miller's     */
/* backward recurrence I_{k-1} = (2k/x) I_k + I_{k+1} (all terms positive),   */
/* normalised with I_0 + 2 sum_{k>=1} I_k = exp(x), i.e. the scaled values    */
/* sum to one.  These are the Chebyshev coefficients of exp(-z x) on [-1, 1]:  */
/* exp(-z x) = I_0(z) + 2 sum (-1)^k I_k(z) T_k(x).                            */
/* ------------------------------------------------------------------------- */
void or_bessel_i_scaled(double x, int32_t K, double* I) {
  for (int32_t k = 0; k <= K; ++k) I[k] = 0.0;
  if (x == 0.0) {
    I[0] = 1.0;
    return;
  }
  int64_t top = (int64_t)K > (int64_t)ceil(x) ? (int64_t)K : (int64_t)ceil(x);
  int64_t N = top + 30 + (int64_t)(20.0 * cbrt(x + 1.0)) + (int64_t)(2.0 * sqrt(x));
  double ip1 = 0.0, i = 1.0, norm = 2.0;  /* I_N counted twice */
  if (N <= K) I[N] = i;
  for (int64_t k = N; k >= 1; --k) {
    double im1 = (2.0 * (double)k / x) * i + ip1;
    ip1 = i;
    i = im1;
    int64_t idx = k - 1;
    if (idx <= K) I[idx] = i;
    norm += (idx == 0) ? i : 2.0 * i;
    if (i > 1e250) {
      const double s = 1e-250;
      i *= s; ip1 *= s; norm *= s;
      for (int64_t q = idx; q <= K; ++q) I[q] *= s;
    }
  }
  for (int32_t k = 0; k <= K; ++k) I[k] /= norm;
}

/* Imaginary-time Chebyshev filter (the thermal-pure-state filter of the     */
/* paper's introduction and Sec. VII): exp(-tau H) = exp(-tau c) sum a_k      */
/* T_k(Ht), a_0 = I_0(z), a_k = 2 (-1)^k I_k(z), z = tau R; with the scaled   */
/* I_k the prefactor becomes exp(-tau (c - R)) = exp(-tau Emin), removed.     */
void or_cheb_imag_step(const or_op* op, int64_t b, int64_t nvec, double* psi, double tau, double c, double R,
                       int32_t nterms, int normalize, int nthreads) {
  const int64_t n = op->D * nvec;
  double* I = (double*)malloc(sizeof(double) * (size_t)(nterms + 1));
  or_bessel_i_scaled(tau * R, nterms, I);
  double* qm = (double*)malloc(sizeof(double) * 2 * (size_t)n);
  double* q = (double*)malloc(sizeof(double) * 2 * (size_t)n);
  double* y = (double*)malloc(sizeof(double) * 2 * (size_t)n);
  double* acc = (double*)malloc(sizeof(double) * 2 * (size_t)n);
  memcpy(q, psi, sizeof(double) * 2 * (size_t)n);
  for (int64_t e = 0; e < 2 * n; ++e) acc[e] = I[0] * q[e];
  for (int32_t k = 1; k < nterms; ++k) {
    or_apply(op, b, nvec, q, y, nthreads);
    for (int64_t e = 0; e < 2 * n; ++e) {
      double t = (y[e] - c * q[e]) / R;
      double qn = (k == 1) ? t : 2.0 * t - qm[e];
      qm[e] = q[e];
      q[e] = qn;
    }
    double ak = 2.0 * I[k] * ((k & 1) ? -1.0 : 1.0);
    for (int64_t e = 0; e < 2 * n; ++e) acc[e] += ak * q[e];
  }
  if (normalize) {
    for (int64_t v = 0; v < nvec; ++v) {
      double s = 0.0;
      for (int64_t r = 0; r < op->D; ++r) {
        double a = acc[2 * (r * nvec + v)], bb = acc[2 * (r * nvec + v) + 1];
        s += a * a + bb * bb;
      }
      s = sqrt(s);
      for (int64_t r = 0; r < op->D; ++r) {
        acc[2 * (r * nvec + v)] /= s;
        acc[2 * (r * nvec + v) + 1] /= s;
      }
    }
  }
  memcpy(psi, acc, sizeof(double) * 2 * (size_t)n);
  free(I); free(qm); free(q); free(y); free(acc);
}

/* Terms k = 0..n-1 such that |a_k| < tol for every k >= n, a_0 = J_0,        */
/* a_k = 2 J_k (the coefficient-tolerance reading of Sec. VII's --cheb-tol).   */
int32_t or_cheb_terms(double z, double tol) {
  int32_t M = (int32_t)ceil(z) + 60 + (int32_t)(30.0 * cbrt(z + 1.0));
  double* J = (double*)malloc(sizeof(double) * (size_t)(M + 1));
  or_bessel_j(z, M, J);
  int32_t last = 0;
  for (int32_t k = 0; k <= M; ++k) {
    double a = (k == 0) ? fabs(J[0]) : 2.0 * fabs(J[k]);
    if (a >= tol) last = k;
  }
  free(J);
  return last + 1;
}

/* ------------------------------------------------------------------------- */
/* Centred Chebyshev propagation, Sec. VII: Ht = (H - c)/R, q0 = psi,         */
/* q1 = Ht q0, q_{l+1} = 2 Ht q_l - q_{l-1};  exp(-i dt H) psi =              */
/* exp(-i c dt) sum_k a_k q_k with a_0 = J_0(R dt), a_k = 2 (-i)^k J_k(R dt). */
/* ------------------------------------------------------------------------- */
void or_cheb_step(const or_op* op, int64_t b, int64_t nvec, double* psi, double dt,
                  double c, double R, int32_t nterms, int nthreads) {
  const int64_t n = op->D * nvec; /* complex elements */
  double* J = (double*)malloc(sizeof(double) * (size_t)(nterms + 1));
  or_bessel_j(R * dt, nterms, J);
  double* qm = (double*)malloc(sizeof(double) * 2 * (size_t)n);
  double* q = (double*)malloc(sizeof(double) * 2 * (size_t)n);
  double* y = (double*)malloc(sizeof(double) * 2 * (size_t)n);
  double* acc = (double*)malloc(sizeof(double) * 2 * (size_t)n);
  memcpy(q, psi, sizeof(double) * 2 * (size_t)n);
  for (int64_t e = 0; e < 2 * n; ++e) acc[e] = J[0] * q[e];
  for (int32_t k = 1; k < nterms; ++k) {
    or_apply(op, b, nvec, q, y, nthreads);
    /* q_new = (y - c q)/R for k = 1, else 2 (y - c q)/R - q_prev */
    for (int64_t e = 0; e < 2 * n; ++e) {
      double t = (y[e] - c * q[e]) / R;
      double qn = (k == 1) ? t : 2.0 * t - qm[e];
      qm[e] = q[e];
      q[e] = qn;
    }
    /* a_k = 2 (-i)^k J_k: multiply q by (-i)^k then scale */
    double ak = 2.0 * J[k];
    for (int64_t e = 0; e < n; ++e) {
      double qr = q[2 * e], qi = q[2 * e + 1], tr, ti;
      switch (k & 3) {
        case 0: tr = qr; ti = qi; break;
        case 1: tr = qi; ti = -qr; break;
        case 2: tr = -qr; ti = -qi; break;
        default: tr = -qi; ti = qr; break;
      }
      acc[2 * e] += ak * tr;
      acc[2 * e + 1] += ak * ti;
    }
  }
  double ph_r = cos(c * dt), ph_i = -sin(c * dt);
  for (int64_t e = 0; e < n; ++e) {
    double ar = acc[2 * e], ai = acc[2 * e + 1];
    psi[2 * e] = ph_r * ar - ph_i * ai;
    psi[2 * e + 1] = ph_r * ai + ph_i * ar;
  }
  free(J); free(qm); free(q); free(y); free(acc);
}
