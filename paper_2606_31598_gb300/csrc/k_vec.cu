// k_vec.cu -- O(D * nvec) kernels around the apply: precision conversion,
// fixed-order partial-sum reduction, the Chebyshev recurrence epilogue and
// accumulation (FP64), Bessel coefficients (FP64), Lanczos vector kernels,
// the block-cache fill and the entry dump used for parity checks.
#include <cuda_runtime.h>

#include "mf_internal.h"

namespace mf {

static inline unsigned grid_for(int64_t n, int threads = 256) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 1 << 20) g = 1 << 20;
  if (g < 1) g = 1;
  return (unsigned)g;
}

size_t compute_elem_bytes(int prec) { return prec == MF_PREC_FP64 ? sizeof(double2) : sizeof(float2); }

// ------------------------------------------------------------- convert ----
// xc[row][v] = x[row][v] for v < nv, 0 for nv <= v < nb.
template <typename C>
__global__ void k_to_compute(const double2* __restrict__ x, C* __restrict__ xc, int64_t n, int64_t nv, int64_t nb) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / nb, v = e % nb;
    C o;
    if (v < nv) {
      const double2 a = x[row * nv + v];
      o.x = (decltype(o.x))a.x;
      o.y = (decltype(o.y))a.y;
    } else {
      o.x = 0;
      o.y = 0;
    }
    xc[e] = o;
  }
}

cudaError_t launch_to_compute(const Plan& p, const double2* x, void* xc, int64_t D, VecShape s) {
  const int64_t n = D * s.nb;
  if (p.prec == MF_PREC_FP64)
    k_to_compute<double2><<<grid_for(n), 256, 0, p.stream>>>(x, (double2*)xc, n, s.nv, s.nb);
  else
    k_to_compute<float2><<<grid_for(n), 256, 0, p.stream>>>(x, (float2*)xc, n, s.nv, s.nb);
  return cudaGetLastError();
}

// --------------------------------------------------- reduction + epilogue ----
// y[row][v] = sum_{s=0}^{nslot-1} part[s][row][v] in FP64 in slot order, plus
// V_row * x[row][v] for the DVR potential.
template <typename C>
__device__ __forceinline__ double2 slot_sum(const C* __restrict__ part, int64_t nslot, int64_t stride, int64_t idx) {
  double sr = 0.0, si = 0.0;
#pragma unroll 4
  for (int64_t s = 0; s < nslot; ++s) {
    const C v = part[s * stride + idx];
    sr += (double)v.x;
    si += (double)v.y;
  }
  return make_double2(sr, si);
}

// System term of the system-bath composite: (X H_S^T)[row][v] =
// sum_s x[row][s] H_S[v][s] (nv == dS), added to s in FP64.
__device__ __forceinline__ void add_system_term(double2& s, const double2* __restrict__ x, int64_t row, int64_t v,
                                                int64_t nv, const double2* __restrict__ hs) {
  const double2* xr = x + row * nv;
  const double2* h = hs + v * nv;
  for (int64_t k = 0; k < nv; ++k) {
    s.x += h[k].x * xr[k].x - h[k].y * xr[k].y;
    s.y += h[k].x * xr[k].y + h[k].y * xr[k].x;
  }
}

// row0: first output row of a row-distributed plan (0 otherwise); y and the
// slots hold the plan's rows, x all of them.
template <typename C>
__global__ void k_reduce(const C* __restrict__ part, VecShape sh, int64_t n, int dvr, dvr_consts dk,
                         const double2* __restrict__ x, double2* __restrict__ y, const double2* __restrict__ hs,
                         int64_t row0) {
  const int64_t stride = sh.dpad * sh.nb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / sh.nv, v = e % sh.nv;
    double2 s = slot_sum(part, sh.nslot, stride, row * sh.nb + v);
    if (dvr) {
      const double V = dvr_V(dk, row0 + row);
      const double2 xv = x[e + row0 * sh.nv];
      s.x = fma(V, xv.x, s.x);
      s.y = fma(V, xv.y, s.y);
    }
    if (hs) add_system_term(s, x, row, v, sh.nv, hs);
    y[e] = s;
  }
}

cudaError_t launch_reduce(const Plan& p, const void* part, const double2* x, double2* y, VecShape s) {
  const int64_t rows = p.sliced ? p.row1 - p.row0 : p.D, row0 = p.sliced ? p.row0 : 0;
  const int64_t n = rows * s.nv;
  const int dvr = p.gen == MF_GEN_SINC_DVR_HO;
  if (p.prec == MF_PREC_FP64)
    k_reduce<double2><<<grid_for(n), 256, 0, p.stream>>>((const double2*)part, s, n, dvr, p.dvr, x, y, p.d_sb_HS,
                                                         row0);
  else
    k_reduce<float2><<<grid_for(n), 256, 0, p.stream>>>((const float2*)part, s, n, dvr, p.dvr, x, y, p.d_sb_HS,
                                                        row0);
  return cudaGetLastError();
}

// Chebyshev (Sec. VII): q0 = psi, acc = a0 q0, compute-format copy of q0
// (padding of the copy written as zeros).
template <typename C>
__global__ void k_cheb_init(const double2* __restrict__ psi, double2* __restrict__ q, double2* __restrict__ acc,
                            C* __restrict__ xc, const double* __restrict__ J, int64_t nrow, int64_t nv, int64_t nb) {
  const double a0 = J[0];
  const int64_t n = nrow * nb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / nb, v = e % nb;
    C o;
    o.x = 0;
    o.y = 0;
    if (v < nv) {
      const int64_t i = row * nv + v;
      const double2 a = psi[i];
      q[i] = a;
      acc[i] = make_double2(a0 * a.x, a0 * a.y);
      o.x = (decltype(o.x))a.x;
      o.y = (decltype(o.y))a.y;
    }
    xc[e] = o;
  }
}

cudaError_t launch_cheb_init(const Plan& p, const double2* psi, double2* q, double2* acc, void* xc, VecShape s) {
  const int64_t n = p.D * s.nb;
  if (p.prec == MF_PREC_FP64)
    k_cheb_init<double2><<<grid_for(n), 256, 0, p.stream>>>(psi, q, acc, (double2*)xc, p.d_J, p.D, s.nv, s.nb);
  else
    k_cheb_init<float2><<<grid_for(n), 256, 0, p.stream>>>(psi, q, acc, (float2*)xc, p.d_J, p.D, s.nv, s.nb);
  return cudaGetLastError();
}

// y = H q_k (slot sum + potential); t = (y - c q_k)/R;
// q_{k+1} = t (k+1 == 1) or 2t - q_{k-1}; acc += a_{k+1} q_{k+1} with
// a_j = 2 (-i)^j J_j; q_{k+1} overwrites q_{k-1} and its compute copy xc.
// y = H q_k at element e (partial sums, potential and system term already
// added), q = q_k[e]: t = (y - c q) / R as (y - c q) * (1 / R);
// q_{k+1} = t (j == 1) or 2 t - q_{k-1}, written over q_{k-1}; acc += a_j
// (-i)^j q_{k+1} (real time) or a_j q_{k+1} (imaginary time); the
// compute-precision copy of q_{k+1} goes to xc[ci].
template <typename C>
__device__ __forceinline__ void cheb_term_finish(double2 y, double2 q, int64_t e, int64_t ci, int32_t j, double c,
                                                 double rinv, double aj, int imag_time, double2* __restrict__ qprev,
                                                 double2* __restrict__ acc, C* __restrict__ xc) {
  double tr = (y.x - c * q.x) * rinv, ti = (y.y - c * q.y) * rinv;
  if (j > 1) {
    const double2 qp = qprev[e];
    tr = 2.0 * tr - qp.x;
    ti = 2.0 * ti - qp.y;
  }
  qprev[e] = make_double2(tr, ti);
  double rr, ri;
  switch (imag_time ? 0 : (j & 3)) {
    case 0: rr = tr; ri = ti; break;
    case 1: rr = ti; ri = -tr; break;
    case 2: rr = -tr; ri = -ti; break;
    default: rr = -ti; ri = tr; break;
  }
  double2 a = acc[e];
  a.x = fma(aj, rr, a.x);
  a.y = fma(aj, ri, a.y);
  acc[e] = a;
  C o;
  o.x = (decltype(o.x))tr;
  o.y = (decltype(o.y))ti;
  xc[ci] = o;
}

template <typename C>
__global__ void k_cheb_update(const C* __restrict__ part, VecShape sh, int64_t n, int dvr, dvr_consts dk,
                              const double2* __restrict__ qcur, double2* __restrict__ qprev,
                              double2* __restrict__ acc, C* __restrict__ xc, const double* __restrict__ J,
                              int32_t j, double c, double rinv, int imag_time, const double2* __restrict__ hs) {
  // real time: a_j = 2 (-i)^j J_j; imaginary time: a_j = 2 (-1)^j e^{-z} I_j
  const double aj = (imag_time && (j & 1)) ? -2.0 * J[j] : 2.0 * J[j];
  const int64_t stride = sh.dpad * sh.nb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    // one vector needs no index division
    const int64_t row = sh.nv == 1 ? e : e / sh.nv, v = sh.nv == 1 ? 0 : e - row * sh.nv;
    const int64_t ci = row * sh.nb + v;
    double2 y = slot_sum(part, sh.nslot, stride, ci);
    const double2 q = qcur[e];
    if (dvr) {
      const double V = dvr_V(dk, row);
      y.x = fma(V, q.x, y.x);
      y.y = fma(V, q.y, y.y);
    }
    if (hs) add_system_term(y, qcur, row, v, sh.nv, hs);
    cheb_term_finish<C>(y, q, e, ci, j, c, rinv, aj, imag_time, qprev, acc, xc);
  }
}

cudaError_t launch_cheb_update(const Plan& p, const void* part, const double2* qcur, double2* qprev, double2* acc,
                               void* xc, VecShape s, int32_t k_next, double c, double R, int imag_time) {
  const int64_t n = p.D * s.nv;
  const int dvr = p.gen == MF_GEN_SINC_DVR_HO;
  const double rinv = 1.0 / R;  // once on the host: the FP64 pipe is GB300's slowest
  if (p.prec == MF_PREC_FP64)
    k_cheb_update<double2><<<grid_for(n), 256, 0, p.stream>>>((const double2*)part, s, n, dvr, p.dvr, qcur, qprev,
                                                              acc, (double2*)xc, p.d_J, k_next, c, rinv, imag_time,
                                                              p.d_sb_HS);
  else
    k_cheb_update<float2><<<grid_for(n), 256, 0, p.stream>>>((const float2*)part, s, n, dvr, p.dvr, qcur, qprev,
                                                             acc, (float2*)xc, p.d_J, k_next, c, rinv, imag_time,
                                                             p.d_sb_HS);
  return cudaGetLastError();
}

// Row-distributed Chebyshev term (row-parallel mode, Sec. IV.H): the plan's
// slice of one term.  y = H q_j on the plan's rows, q = q_j on all rows (the
// caller gathers it); t = (y - c q) / R; q_{j+1} = t (j == 1) or 2 t -
// q_{j-1}; q_prev <- q_j and q_next <- q_{j+1} on the slice (q_next is what
// the caller gathers for the next term); acc += a_j (-i)^j q_{j+1}.
__global__ void k_cheb_rows_init(const double2* __restrict__ psi, int64_t off, double2* __restrict__ acc, int64_t n,
                                 const double* __restrict__ J) {
  const double a0 = J[0];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = psi[off + e];
    acc[e] = make_double2(a0 * a.x, a0 * a.y);
  }
}

__global__ void k_cheb_rows_term(const double2* __restrict__ y, const double2* __restrict__ qfull, int64_t off,
                                 double2* __restrict__ qprev, double2* __restrict__ qnext, double2* __restrict__ acc,
                                 int64_t n, const double* __restrict__ J, int32_t j, double c, double rinv) {
  const double aj = 2.0 * J[j];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 yv = y[e], q = qfull[off + e];
    double tr = (yv.x - c * q.x) * rinv, ti = (yv.y - c * q.y) * rinv;
    if (j > 1) {
      const double2 qp = qprev[e];
      tr = 2.0 * tr - qp.x;
      ti = 2.0 * ti - qp.y;
    }
    qprev[e] = q;
    qnext[e] = make_double2(tr, ti);
    double rr, ri;
    switch (j & 3) {
      case 0: rr = tr; ri = ti; break;
      case 1: rr = ti; ri = -tr; break;
      case 2: rr = -tr; ri = -ti; break;
      default: rr = -ti; ri = tr; break;
    }
    double2 a = acc[e];
    a.x = fma(aj, rr, a.x);
    a.y = fma(aj, ri, a.y);
    acc[e] = a;
  }
}

cudaError_t launch_cheb_rows_init(const Plan& p, const double2* psi, double2* acc, int64_t nvec) {
  const int64_t n = (p.row1 - p.row0) * nvec;
  k_cheb_rows_init<<<grid_for(n), 256, 0, p.stream>>>(psi, p.row0 * nvec, acc, n, p.d_J);
  return cudaGetLastError();
}

cudaError_t launch_cheb_rows_term(const Plan& p, const double2* y, const double2* qfull, double2* qprev,
                                  double2* qnext, double2* acc, int64_t nvec, int32_t j, double c, double R) {
  const int64_t n = (p.row1 - p.row0) * nvec;
  k_cheb_rows_term<<<grid_for(n), 256, 0, p.stream>>>(y, qfull, p.row0 * nvec, qprev, qnext, acc, n, p.d_J, j, c,
                                                      1.0 / R);
  return cudaGetLastError();
}

// psi = exp(-i c dt) acc
__global__ void k_cheb_final(const double2* __restrict__ acc, double2* __restrict__ psi, int64_t n, double pr,
                             double pi) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = acc[e];
    psi[e] = make_double2(pr * a.x - pi * a.y, pr * a.y + pi * a.x);
  }
}

cudaError_t launch_cheb_final(const Plan& p, const double2* acc, double2* psi, int64_t n, double c, double dt) {
  double s, co;
  sincos(c * dt, &s, &co);
  k_cheb_final<<<grid_for(n), 256, 0, p.stream>>>(acc, psi, n, co, -s);
  return cudaGetLastError();
}

// Bessel J_0..J_K(z) by Miller's backward recurrence J_{k-1} = (2k/z) J_k -
// J_{k+1}, started well above max(K, z), rescaled against overflow and
// normalised with J_0 + 2 sum_{k>=1} J_{2k} = 1.  One thread: the recurrence
// is sequential and O(K + z) long.
__global__ void k_bessel(double z, int32_t K, double* __restrict__ J) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (z == 0.0) {
    J[0] = 1.0;
    for (int k = 1; k <= K; ++k) J[k] = 0.0;
    return;
  }
  const long long zc = (long long)ceil(z);
  long long start = (K > zc ? K : zc) + 30 + (long long)(20.0 * cbrt(z + 1.0));
  start += start & 1;
  for (int k = 0; k <= K; ++k) J[k] = 0.0;
  double hi = 0.0, cur = 1.0, sum = 2.0;  // J_start counts twice (start is even)
  if (start <= K) J[start] = cur;
  for (long long k = start; k >= 1; --k) {
    const double nxt = (2.0 * (double)k / z) * cur - hi;
    hi = cur;
    cur = nxt;
    const long long idx = k - 1;
    if (idx <= K) J[idx] = cur;
    sum += (idx == 0) ? cur : ((idx & 1) ? 0.0 : 2.0 * cur);
    if (fabs(cur) > 1e250) {
      cur *= 1e-250;
      hi *= 1e-250;
      sum *= 1e-250;
      for (long long q = idx; q <= K; ++q) J[q] *= 1e-250;
    }
  }
  const double inv = 1.0 / sum;
  for (int k = 0; k <= K; ++k) J[k] *= inv;
}

cudaError_t launch_bessel(const Plan& p, double z, int32_t K, double* J) {
  k_bessel<<<1, 32, 0, p.stream>>>(z, K, J);
  return cudaGetLastError();
}

// Scaled modified Bessel functions e^{-z} I_k(z), k = 0..K: Miller's backward
// recurrence I_{k-1} = (2k/z) I_k + I_{k+1} (every term positive, so no
// cancellation), normalised with I_0 + 2 sum_{k>=1} I_k = e^z.  These give the
// Chebyshev series of exp(-z x) on [-1, 1] with the factor e^{z} taken out.
__global__ void k_bessel_i(double z, int32_t K, double* __restrict__ I) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int k = 0; k <= K; ++k) I[k] = 0.0;
  if (z == 0.0) {
    I[0] = 1.0;
    return;
  }
  const long long zc = (long long)ceil(z);
  const long long start = (K > zc ? K : zc) + 30 + (long long)(20.0 * cbrt(z + 1.0)) + (long long)(2.0 * sqrt(z));
  double hi = 0.0, cur = 1.0, sum = 2.0;  // I_start counts twice
  if (start <= K) I[start] = cur;
  for (long long k = start; k >= 1; --k) {
    const double nxt = (2.0 * (double)k / z) * cur + hi;
    hi = cur;
    cur = nxt;
    const long long idx = k - 1;
    if (idx <= K) I[idx] = cur;
    sum += (idx == 0) ? cur : 2.0 * cur;
    if (cur > 1e250) {
      cur *= 1e-250;
      hi *= 1e-250;
      sum *= 1e-250;
      for (long long q = idx; q <= K; ++q) I[q] *= 1e-250;
    }
  }
  const double inv = 1.0 / sum;
  for (int k = 0; k <= K; ++k) I[k] *= inv;
}

cudaError_t launch_bessel_i(const Plan& p, double z, int32_t K, double* I) {
  k_bessel_i<<<1, 32, 0, p.stream>>>(z, K, I);
  return cudaGetLastError();
}

// Column norms of a [D][nv] complex128 block, deterministic: CTA (s, v) sums
// |a_{r,v}|^2 over rows r = s*256 + t (+ kColSplit*256 strides), then one
// thread per column adds the kColSplit partials in order and stores 1/norm
// (0 for a zero column, which is then left as zeros).
constexpr int kColSplit = 64;

__global__ void k_colnorm_partial(const double2* __restrict__ a, int64_t nrow, int64_t nv,
                                  double* __restrict__ partial) {
  __shared__ double sh[256];
  const int64_t v = blockIdx.y;
  double s = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * 256 + threadIdx.x; r < nrow; r += (int64_t)kColSplit * 256) {
    const double2 u = a[r * nv + v];
    s += u.x * u.x + u.y * u.y;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[v * kColSplit + blockIdx.x] = sh[0];
}

__global__ void k_colnorm_final(const double* __restrict__ partial, int64_t nv, double* __restrict__ inv) {
  const int64_t v = threadIdx.x;
  if (v >= nv) return;
  double s = 0.0;
  for (int q = 0; q < kColSplit; ++q) s += partial[v * kColSplit + q];
  inv[v] = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
}

// psi[r][v] = acc[r][v] * inv[v] (inv == nullptr: plain copy)
__global__ void k_scale_columns(const double2* __restrict__ acc, double2* __restrict__ psi, int64_t n, int64_t nv,
                                const double* __restrict__ inv) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double s = inv ? inv[e % nv] : 1.0;
    const double2 a = acc[e];
    psi[e] = make_double2(s * a.x, s * a.y);
  }
}

cudaError_t launch_filter_final(const Plan& p, const double2* acc, double2* psi, int64_t rows, int64_t nv,
                                int normalize) {
  const int64_t n = rows * nv;
  double* inv = nullptr;
  if (normalize) {
    double* partial = p.d_red;
    inv = p.d_red + kColSplit * 64;
    k_colnorm_partial<<<dim3(kColSplit, (unsigned)nv), 256, 0, p.stream>>>(acc, rows, nv, partial);
    k_colnorm_final<<<1, 64, 0, p.stream>>>(partial, nv, inv);
  }
  k_scale_columns<<<grid_for(n), 256, 0, p.stream>>>(acc, psi, n, nv, inv);
  return cudaGetLastError();
}

// ------------------------------------------------------------ Lanczos ----
// Deterministic two-stage FP64 reduction: 256 CTA partials, then one CTA sums
// them in index order.
__global__ void k_dot_partial(const double2* __restrict__ a, const double2* __restrict__ b, int64_t n,
                              double* __restrict__ partial) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 u = a[e], v = b[e];
    s += u.x * v.x + u.y * v.y;  // Re(conj(u) v)
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void k_sum_partials(const double* __restrict__ partial, int np, double* __restrict__ out) {
  __shared__ double sh[256];
  sh[threadIdx.x] = (int)threadIdx.x < np ? partial[threadIdx.x] : 0.0;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

cudaError_t launch_dot(const Plan& p, const double2* a, const double2* b, int64_t n, double* out) {
  k_dot_partial<<<256, 256, 0, p.stream>>>(a, b, n, p.d_red);
  k_sum_partials<<<1, 256, 0, p.stream>>>(p.d_red, 256, out);
  return cudaGetLastError();
}

// w = w - alpha v - beta vprev
__global__ void k_lanczos_axpby(double2* __restrict__ w, const double2* __restrict__ v,
                                const double2* __restrict__ vp, double alpha, double beta, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double2 a = w[e];
    const double2 b = v[e];
    a.x -= alpha * b.x;
    a.y -= alpha * b.y;
    if (vp) {
      const double2 c = vp[e];
      a.x -= beta * c.x;
      a.y -= beta * c.y;
    }
    w[e] = a;
  }
}

cudaError_t launch_axpby_lanczos(const Plan& p, double2* w, const double2* v, const double2* vprev, double alpha,
                                 double beta, int64_t n) {
  k_lanczos_axpby<<<grid_for(n), 256, 0, p.stream>>>(w, v, vprev, alpha, beta, n);
  return cudaGetLastError();
}

__global__ void k_scale(double2* __restrict__ dst, const double2* __restrict__ src, double s, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = src[e];
    dst[e] = make_double2(s * v.x, s * v.y);
  }
}

cudaError_t launch_scale(const Plan& p, double2* dst, const double2* src, double s, int64_t n) {
  k_scale<<<grid_for(n), 256, 0, p.stream>>>(dst, src, s, n);
  return cudaGetLastError();
}

// Lanczos start vector: uniform(-1/2, 1/2) parts from Philox words with a
// counter stream separate from the operator's (third counter word = 1).
__global__ void k_random(double2* __restrict__ v, int64_t n, uint64_t seed) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)e, (uint32_t)(e >> 32), 1u, 0u), (uint32_t)seed,
                                  (uint32_t)(seed >> 32));
    v[e] = make_double2(((double)w.x + 0.5) * 0x1p-32 - 0.5, ((double)w.y + 0.5) * 0x1p-32 - 0.5);
  }
}

cudaError_t launch_random_unit(const Plan& p, double2* v, int64_t n, uint64_t seed) {
  k_random<<<grid_for(n), 256, 0, p.stream>>>(v, n, seed);
  return cudaGetLastError();
}

// ------------------------------------------------------- cache fill -------
// One CTA per (cached slot, block row); block (n, m) of slot s holds
// H[n b + a][m b + c] for a, c in [0, b), zero outside [0, D).
template <typename T, int GEN>
__global__ void k_cache_fill(const int2* __restrict__ pairs, int64_t b, int64_t D, uint64_t seed, T sigma,
                             dvr_consts dk, typename cplx<T>::t* __restrict__ cache) {
  using C = typename cplx<T>::t;
  const int64_t slot = blockIdx.x;
  const int2 nm = pairs[slot];
  const int64_t a = blockIdx.y;
  const int64_t r = (int64_t)nm.x * b + a;
  C* row = cache + (slot * b + a) * b;
  for (int64_t cc = 2 * threadIdx.x; cc < b; cc += 2 * blockDim.x) {
    const int64_t c = (int64_t)nm.y * b + cc;
    C h0, h1;
    if (r >= D) {
      h0.x = h0.y = h1.x = h1.y = T(0);
    } else if (GEN == MF_GEN_PHILOX_GUE) {
      h0 = gue_entry<T>(seed, sigma, r, c);
      h1 = gue_entry<T>(seed, sigma, r, c + 1);
    } else {
      h0.x = dvr_T(dk, (long long)(r - c), T());
      h1.x = dvr_T(dk, (long long)(r - c - 1), T());
      h0.y = h1.y = T(0);
    }
    if (c >= D) h0.x = h0.y = T(0);
    if (c + 1 >= D) h1.x = h1.y = T(0);
    row[cc] = h0;
    if (cc + 1 < b) row[cc + 1] = h1;
  }
}

cudaError_t launch_cache_fill_pairs(const Plan& p, const int2* d_pairs, int64_t npairs) {
  if (npairs == 0) return cudaSuccess;
  if (p.b > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)npairs, (unsigned)p.b);
  if (p.prec == MF_PREC_FP64) {
    if (p.gen == MF_GEN_PHILOX_GUE)
      k_cache_fill<double, MF_GEN_PHILOX_GUE><<<grid, 256, 0, p.stream>>>(d_pairs, p.b, p.D, p.seed, p.sigma64,
                                                                           p.dvr, (double2*)p.d_cache);
    else
      k_cache_fill<double, MF_GEN_SINC_DVR_HO><<<grid, 256, 0, p.stream>>>(d_pairs, p.b, p.D, p.seed, p.sigma64,
                                                                            p.dvr, (double2*)p.d_cache);
  } else {
    if (p.gen == MF_GEN_PHILOX_GUE)
      k_cache_fill<float, MF_GEN_PHILOX_GUE><<<grid, 256, 0, p.stream>>>(d_pairs, p.b, p.D, p.seed, p.sigma32,
                                                                          p.dvr, (float2*)p.d_cache);
    else
      k_cache_fill<float, MF_GEN_SINC_DVR_HO><<<grid, 256, 0, p.stream>>>(d_pairs, p.b, p.D, p.seed, p.sigma32,
                                                                           p.dvr, (float2*)p.d_cache);
  }
  return cudaGetLastError();
}

// --------------------------------------------------------- entry dump ------
template <typename T, int GEN>
__global__ void k_debug_entries(int64_t r0, int64_t c0, int64_t rows, int64_t cols, uint64_t seed, T sigma,
                                dvr_consts dk, typename cplx<T>::t* __restrict__ out) {
  const int64_t n = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = r0 + e / cols, c = c0 + e % cols;
    typename cplx<T>::t h;
    if (GEN == MF_GEN_PHILOX_GUE) {
      h = gue_entry<T>(seed, sigma, r, c);
    } else {
      h.x = dvr_T(dk, (long long)(r - c), T());
      h.y = T(0);
    }
    out[e] = h;
  }
}

cudaError_t launch_debug_entries(const Plan& p, int64_t r0, int64_t c0, int64_t rows, int64_t cols, void* out) {
  const int64_t n = rows * cols;
  if (p.prec == MF_PREC_FP64) {
    if (p.gen == MF_GEN_PHILOX_GUE)
      k_debug_entries<double, MF_GEN_PHILOX_GUE><<<grid_for(n), 256, 0, p.stream>>>(r0, c0, rows, cols, p.seed,
                                                                                     p.sigma64, p.dvr, (double2*)out);
    else
      k_debug_entries<double, MF_GEN_SINC_DVR_HO><<<grid_for(n), 256, 0, p.stream>>>(r0, c0, rows, cols, p.seed,
                                                                                      p.sigma64, p.dvr, (double2*)out);
  } else {
    if (p.gen == MF_GEN_PHILOX_GUE)
      k_debug_entries<float, MF_GEN_PHILOX_GUE><<<grid_for(n), 256, 0, p.stream>>>(r0, c0, rows, cols, p.seed,
                                                                                    p.sigma32, p.dvr, (float2*)out);
    else
      k_debug_entries<float, MF_GEN_SINC_DVR_HO><<<grid_for(n), 256, 0, p.stream>>>(r0, c0, rows, cols, p.seed,
                                                                                     p.sigma32, p.dvr, (float2*)out);
  }
  return cudaGetLastError();
}

}  // namespace mf
