"""ctypes front-end of the CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this module.  It never imports the product package.

Every routine forwards to ``mf_oracle.c`` (plain FP64 C); the few numpy steps
here are library primitives (dense matrix products, FFTs) used as stated steps
of a definition, with no blocking or reordering beyond the definition.
"""
import ctypes
import os

import numpy as np

from . import build as _build

GEN_PHILOX_GUE = 0
GEN_SINC_DVR_HO = 1
FORM_FP64 = 0
FORM_FP32 = 1


class OrOp(ctypes.Structure):
    _fields_ = [
        ("gen", ctypes.c_int32),
        ("form", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("D", ctypes.c_int64),
        ("L", ctypes.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        d, i64, i32, u64 = ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
        vp = ctypes.c_void_p
        L.or_philox4x32_10.argtypes = [vp, vp, vp]
        L.or_log.argtypes = [d]; L.or_log.restype = d
        L.or_logf.argtypes = [ctypes.c_float]; L.or_logf.restype = ctypes.c_float
        L.or_sincos_2pi.argtypes = [d, P(d), P(d)]
        L.or_sincos_2pif.argtypes = [ctypes.c_float, P(ctypes.c_float), P(ctypes.c_float)]
        L.or_entry.argtypes = [P(OrOp), i64, i64, P(d), P(d)]
        L.or_dvr_potential.argtypes = [P(OrOp), i64]; L.or_dvr_potential.restype = d
        L.or_dvr_kinetic.argtypes = [P(OrOp), i64]; L.or_dvr_kinetic.restype = d
        L.or_window.argtypes = [P(OrOp), i64, i64, i64, i64, vp]
        L.or_window_f32.argtypes = [P(OrOp), i64, i64, i64, i64, vp]
        L.or_apply.argtypes = [P(OrOp), i64, i64, vp, vp, ctypes.c_int]
        L.or_apply_rows.argtypes = [P(OrOp), i64, vp, i64, vp, vp, ctypes.c_int]
        L.or_bessel_j.argtypes = [d, i32, vp]
        L.or_cheb_terms.argtypes = [d, d]; L.or_cheb_terms.restype = i32
        L.or_cheb_step.argtypes = [P(OrOp), i64, i64, vp, d, d, d, i32, ctypes.c_int]
        L.or_bessel_i_scaled.argtypes = [d, i32, vp]
        L.or_cheb_imag_step.argtypes = [P(OrOp), i64, i64, vp, d, d, d, i32, ctypes.c_int, ctypes.c_int]
        _lib = L
    return _lib


def dvr_default_L(D):
    """Grid half-width L = 0.9 sqrt(2D) of the DVR workload."""
    return 0.9 * np.sqrt(2.0 * float(D))


def make_op(gen, D, seed=1, form=FORM_FP64, L=None):
    if gen == GEN_SINC_DVR_HO and L is None:
        L = dvr_default_L(D)
    return OrOp(int(gen), int(form), int(seed) & 0xFFFFFFFFFFFFFFFF, int(D), float(L or 0.0))


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def log64(u):
    return lib().or_log(float(u))


def log32(u):
    return np.float32(lib().or_logf(ctypes.c_float(np.float32(u))))


def sincos64(u):
    s, c = ctypes.c_double(), ctypes.c_double()
    lib().or_sincos_2pi(float(u), ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def sincos32(u):
    s, c = ctypes.c_float(), ctypes.c_float()
    lib().or_sincos_2pif(ctypes.c_float(np.float32(u)), ctypes.byref(s), ctypes.byref(c))
    return np.float32(s.value), np.float32(c.value)


def entry(op, r, c):
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().or_entry(ctypes.byref(op), int(r), int(c), ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def kinetic(op, k):
    """DVR kinetic entry T(k), k = r - c, in op's form (as a double)."""
    return lib().or_dvr_kinetic(ctypes.byref(op), int(k))


def kinetic_window(op, r0, c0, rows, cols):
    ks = (r0 + np.arange(rows))[:, None] - (c0 + np.arange(cols))[None, :]
    table = {int(k): kinetic(op, int(k)) for k in np.unique(ks)}
    return np.vectorize(lambda k: table[int(k)])(ks).astype(np.float64)


def potential(op, i):
    return lib().or_dvr_potential(ctypes.byref(op), int(i))


def window(op, r0, c0, rows, cols):
    """H[r0:r0+rows, c0:c0+cols] as complex128 (entries of op's form)."""
    out = np.zeros((rows, cols), dtype=np.complex128)
    lib().or_window(ctypes.byref(op), int(r0), int(c0), int(rows), int(cols), out.ctypes.data)
    return out


def window_native(op, r0, c0, rows, cols):
    """FP32-form window in its native complex64 (potential not included)."""
    out = np.zeros((rows, cols), dtype=np.complex64)
    lib().or_window_f32(ctypes.byref(op), int(r0), int(c0), int(rows), int(cols), out.ctypes.data)
    return out


def dense(op):
    return window(op, 0, 0, op.D, op.D)


def apply(op, x, block=0, nthreads=0):
    """y = H x (x: [D] or [D, nvec] complex), blockwise FP64 sum."""
    x = np.asarray(x, dtype=np.complex128)
    squeeze = x.ndim == 1
    X = np.ascontiguousarray(x.reshape(op.D, -1))
    Y = np.zeros_like(X)
    lib().or_apply(ctypes.byref(op), int(block), int(X.shape[1]), X.ctypes.data, Y.ctypes.data,
                   int(nthreads))
    return Y.reshape(-1) if squeeze else Y


def apply_rows(op, x, rows, nthreads=0):
    x = np.asarray(x, dtype=np.complex128)
    X = np.ascontiguousarray(x.reshape(op.D, -1))
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    Y = np.zeros((rows.size, X.shape[1]), dtype=np.complex128)
    lib().or_apply_rows(ctypes.byref(op), int(X.shape[1]), X.ctypes.data, int(rows.size),
                        rows.ctypes.data, Y.ctypes.data, int(nthreads))
    return Y


def bessel_j(x, K):
    J = np.zeros(K + 1, dtype=np.float64)
    lib().or_bessel_j(float(x), int(K), J.ctypes.data)
    return J


def bessel_i_scaled(x, K):
    I = np.zeros(K + 1, dtype=np.float64)
    lib().or_bessel_i_scaled(float(x), int(K), I.ctypes.data)
    return I


def cheb_imag_terms(z, tol):
    """Smallest n with |a_k| < tol for every k >= n, a_0 = e^-z I_0(z),
    a_k = 2 e^-z I_k(z) (the coefficients decrease monotonically in k)."""
    K = int(np.ceil(z)) + 60 + int(30.0 * np.cbrt(z + 1.0))
    I = bessel_i_scaled(z, K)
    a = np.concatenate([[I[0]], 2.0 * I[1:]])
    big = np.nonzero(a >= tol)[0]
    return int(big[-1]) + 1 if big.size else 1


def cheb_imag_step(op, psi, tau, c, R, nterms, normalize=True, block=0, nthreads=0):
    """psi <- exp(-tau (H - Emin)) psi (Emin = c - R), optionally renormalised."""
    psi = np.asarray(psi, dtype=np.complex128)
    shape = psi.shape
    P = np.ascontiguousarray(psi.reshape(op.D, -1)).copy()
    lib().or_cheb_imag_step(ctypes.byref(op), int(block), int(P.shape[1]), P.ctypes.data, float(tau), float(c),
                            float(R), int(nterms), int(bool(normalize)), int(nthreads))
    return P.reshape(shape)


def cheb_terms(z, tol):
    return int(lib().or_cheb_terms(float(z), float(tol)))


def cheb_coeffs(z, nterms):
    """a_k = J_0 (k=0), 2 (-i)^k J_k(z) (k>=1), k = 0..nterms-1."""
    J = bessel_j(z, nterms)
    a = 2.0 * J[:nterms] * ((-1j) ** np.arange(nterms))
    a[0] = J[0]
    return a


def cheb_step(op, psi, dt, c, R, nterms, block=0, nthreads=0):
    """One Chebyshev step of exp(-i dt H) on psi ([D] or [D, nvec])."""
    psi = np.asarray(psi, dtype=np.complex128)
    shape = psi.shape
    P = np.ascontiguousarray(psi.reshape(op.D, -1)).copy()
    lib().or_cheb_step(ctypes.byref(op), int(block), int(P.shape[1]), P.ctypes.data, float(dt),
                       float(c), float(R), int(nterms), int(nthreads))
    return P.reshape(shape)


def cheb_step_fn(apply_fn, psi, dt, c, R, nterms):
    """The Chebyshev step with the product y = apply_fn(q) of any operator
    form: q_{k+1} = 2 (H q_k - c q_k)/R - q_{k-1}, acc += a_k q_k, final
    phase e^{-i c dt}."""
    a = cheb_coeffs(R * dt, nterms)
    q_prev = None
    q = np.array(psi, dtype=np.complex128)
    acc = a[0] * q
    for k in range(1, nterms):
        t = (apply_fn(q) - c * q) / R
        qn = t if k == 1 else 2.0 * t - q_prev
        q_prev, q = q, qn
        acc = acc + a[k] * q
    return np.exp(-1j * c * dt) * acc


def cheb_step_dense(H, psi, dt, c, R, nterms):
    """The same recurrence with a materialised H (small D), matrix products
    by numpy."""
    return cheb_step_fn(lambda q: H @ q, psi, dt, c, R, nterms)


# ------------------------------------------------------------- BF16X2 form --
def bf16_rn(a):
    """Round float32 values to the nearest bfloat16 (ties to even), returned
    as float32 (the bfloat16 value widened)."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def split_bf16(a):
    """hi = bf16(a), lo = bf16(a - hi), a in float32."""
    a = np.asarray(a, dtype=np.float32)
    hi = bf16_rn(a)
    lo = bf16_rn((a - hi).astype(np.float32))
    return hi, lo


def apply_bf16x2(op, x, H32=None):
    """y = H x in the BF16X2 form: FP32-form entries and the FP32 copy of x
    are split into bf16 hi + lo; each real product a*b is taken as
    a_hi b_hi + a_hi b_lo + a_lo b_hi (the lo*lo term dropped), summed exactly
    in FP64; the DVR potential is applied in FP64 to the FP64 x.  H32: the
    FP32-form window of the whole operator (complex64), computed if None."""
    x = np.asarray(x, dtype=np.complex128)
    X = x.reshape(op.D, -1)
    if H32 is None:
        H32 = window_native(make_op(op.gen, op.D, seed=op.seed, form=FORM_FP32, L=op.L or None), 0, 0, op.D, op.D)
    Ar_h, Ar_l = split_bf16(H32.real)
    Ai_h, Ai_l = split_bf16(H32.imag)
    X32 = X.astype(np.complex64)
    Xr_h, Xr_l = split_bf16(X32.real)
    Xi_h, Xi_l = split_bf16(X32.imag)
    f = lambda a: a.astype(np.float64)
    def prod(ah, al, bh, bl):
        return f(ah) @ f(bh) + f(ah) @ f(bl) + f(al) @ f(bh)
    yr = prod(Ar_h, Ar_l, Xr_h, Xr_l) - prod(Ai_h, Ai_l, Xi_h, Xi_l)
    yi = prod(Ar_h, Ar_l, Xi_h, Xi_l) + prod(Ai_h, Ai_l, Xr_h, Xr_l)
    Y = yr + 1j * yi
    if op.gen == GEN_SINC_DVR_HO:
        V = np.array([potential(op, i) for i in range(op.D)])
        Y = Y + V[:, None] * X
    return Y.reshape(x.shape)


def apply_rows_bf16x2(op, x, rows):
    """Rows of y = H x in the BF16X2 form (as apply_bf16x2 states it) for any
    D: each sampled row of the FP32-form operator is generated on its own
    (a 1 x D window), split hi/lo, and multiplied with the split FP32 copy of
    x, the three kept partial products summed exactly in FP64; the DVR
    potential is added in FP64 to the FP64 x.  For full-size checks where
    the dense operator cannot be formed."""
    x = np.asarray(x, dtype=np.complex128)
    X = x.reshape(op.D, -1)
    op32 = make_op(op.gen, op.D, seed=op.seed, form=FORM_FP32, L=op.L or None)
    X32 = X.astype(np.complex64)
    Xr_h, Xr_l = split_bf16(X32.real)
    Xi_h, Xi_l = split_bf16(X32.imag)
    f = lambda a: a.astype(np.float64)
    out = np.zeros((len(rows), X.shape[1]), dtype=np.complex128)
    for i, r in enumerate(rows):
        h = window_native(op32, int(r), 0, 1, op.D)
        Ar_h, Ar_l = split_bf16(h.real)
        Ai_h, Ai_l = split_bf16(h.imag)

        def prod(ah, al, bh, bl):
            return f(ah) @ f(bh) + f(ah) @ f(bl) + f(al) @ f(bh)

        yr = prod(Ar_h, Ar_l, Xr_h, Xr_l) - prod(Ai_h, Ai_l, Xi_h, Xi_l)
        yi = prod(Ar_h, Ar_l, Xi_h, Xi_l) + prod(Ai_h, Ai_l, Xr_h, Xr_l)
        out[i] = (yr + 1j * yi)[0]
        if op.gen == GEN_SINC_DVR_HO:
            out[i] += potential(op, int(r)) * X[int(r)]
    return out


class DvrToeplitz:
    """The sinc-DVR operator at any D (the benchmark's D = 131072 included)
    as Toeplitz products by the FFT.  T is symmetric Toeplitz in k = r - c,
    so T x is the first D entries of the circular convolution of the 2D
    embedding [t(0..D-1), 0, t(D-1..1)] with [x, 0] (a library FFT as one
    step).  apply64: the FP64 form.  apply_bf16x2: the BF16X2 form as
    apply_bf16x2 states it -- FP32-form entries split hi/lo, x rounded to
    complex64 and its parts split hi/lo, the three kept partial products
    (the split of T(k) depends on k only, so each is a Toeplitz product).
    apply32: the FP32 form's entries and the complex64 copy of x with exact
    sums (the form's own rounding, without the FP32 tile sums).  All add
    V_i x_i in FP64 with the FP64 x."""

    def __init__(self, D, L=None):
        self.D = D
        op64 = make_op(GEN_SINC_DVR_HO, D, L=L)
        op32 = make_op(GEN_SINC_DVR_HO, D, form=FORM_FP32, L=L)
        t64 = kinetic_window(op64, 0, 0, D, 1)[:, 0]
        t32 = kinetic_window(op32, 0, 0, D, 1)[:, 0].astype(np.float32)
        th, tl = split_bf16(t32)
        self.V = np.array([potential(op64, i) for i in range(D)])

        def embed(t):
            return np.fft.fft(np.concatenate([t, [0.0], t[:0:-1]]))

        self.f64 = embed(t64)
        self.f32 = embed(t32.astype(np.float64))
        self.fhi = embed(th.astype(np.float64))
        self.flo = embed(tl.astype(np.float64))

    def _toeplitz(self, ft, v):
        vp = np.concatenate([v, np.zeros(self.D, dtype=np.complex128)])
        return np.fft.ifft(ft * np.fft.fft(vp))[:self.D]

    def apply64(self, x):
        x = np.asarray(x, dtype=np.complex128).reshape(self.D)
        return self._toeplitz(self.f64, x) + self.V * x

    def apply32(self, x):
        x = np.asarray(x, dtype=np.complex128).reshape(self.D)
        x32 = x.astype(np.complex64).astype(np.complex128)
        return self._toeplitz(self.f32, x32) + self.V * x

    def apply_bf16x2(self, x):
        x = np.asarray(x, dtype=np.complex128).reshape(self.D)
        x32 = x.astype(np.complex64)
        rh, rl = split_bf16(x32.real)
        ih, il = split_bf16(x32.imag)
        xh = rh.astype(np.float64) + 1j * ih.astype(np.float64)
        xl = rl.astype(np.float64) + 1j * il.astype(np.float64)
        return (self._toeplitz(self.fhi, xh) + self._toeplitz(self.fhi, xl) + self._toeplitz(self.flo, xh)
                + self.V * x)


# ------------------------------------------------------- system-bath form ---
# H = H_S (x) I_B + I_S (x) H_B + g sum_a A_a (x) B_a (Sec. VII), with the bath
# operators H_B = B_0 and B_1..B_n Philox ensembles of their own seeds and the
# small system matrices given.  Two independent statements of the operator:
# the dense Kronecker form in system-major order (index s*d_B + beta), and the
# matrix-free form on the bath-major layout X[beta][s] = psi[s*d_B + beta]:
#   Phi = H_B X + X H_S^T + g sum_a B_a X A_a^T.

def sysbath_dense(d_S, d_B, seeds, H_S, A, g, form=FORM_FP64):
    """Dense D x D composite operator, D = d_S d_B, system-major order."""
    H_S = np.asarray(H_S, dtype=np.complex128).reshape(d_S, d_S)
    A = np.asarray(A, dtype=np.complex128).reshape(-1, d_S, d_S)
    HB = dense(make_op(GEN_PHILOX_GUE, d_B, seed=seeds[0], form=form))
    H = np.kron(H_S, np.eye(d_B)) + np.kron(np.eye(d_S), HB)
    for a in range(A.shape[0]):
        Ba = dense(make_op(GEN_PHILOX_GUE, d_B, seed=seeds[1 + a], form=form))
        H = H + g * np.kron(A[a], Ba)
    return H


def sysbath_apply(d_S, d_B, seeds, H_S, A, g, X, form=FORM_FP64):
    """Phi = H_B X + X H_S^T + g sum_a B_a X A_a^T for X [d_B][d_S] (bath-major)."""
    H_S = np.asarray(H_S, dtype=np.complex128).reshape(d_S, d_S)
    A = np.asarray(A, dtype=np.complex128).reshape(-1, d_S, d_S)
    X = np.asarray(X, dtype=np.complex128).reshape(d_B, d_S)
    Phi = apply(make_op(GEN_PHILOX_GUE, d_B, seed=seeds[0], form=form), X).reshape(d_B, d_S) + X @ H_S.T
    for a in range(A.shape[0]):
        BX = apply(make_op(GEN_PHILOX_GUE, d_B, seed=seeds[1 + a], form=form), X).reshape(d_B, d_S)
        Phi = Phi + g * (BX @ A[a].T)
    return Phi


def bath_major(psi, d_S, d_B):
    """System-major psi[s*d_B + beta] -> bath-major X[beta][s]."""
    return np.ascontiguousarray(np.asarray(psi).reshape(d_S, d_B).T)


# ------------------------------------------------ externally stored blocks ---
# H^[n,m] = D[key(n,m)] (Sec. II): a Hermitian operator given by its canonical
# blocks n <= m, stored in row order of the pairs, each b x b (rows/columns
# past D are padding).  Off-diagonal blocks below the diagonal are the
# conjugate transposes; inside a diagonal block only the upper triangle
# (diagonal included) is read and the lower triangle is its conjugate.

def external_pairs(D, b):
    """The canonical pairs (n, m), n <= m, in storage order."""
    nblk = -(-D // b)
    return [(n, m) for n in range(nblk) for m in range(n, nblk)]


def external_dense(D, b, blocks):
    """Dense D x D operator assembled from the stored canonical blocks."""
    blocks = np.asarray(blocks, dtype=np.complex128)
    pairs = external_pairs(D, b)
    blocks = blocks.reshape(len(pairs), b, b)
    nblk = -(-D // b)
    P = nblk * b
    H = np.zeros((P, P), dtype=np.complex128)
    for k, (n, m) in enumerate(pairs):
        B = blocks[k]
        if n == m:
            U = np.triu(B)
            H[n * b:(n + 1) * b, n * b:(n + 1) * b] = U + np.triu(U, 1).conj().T
        else:
            H[n * b:(n + 1) * b, m * b:(m + 1) * b] = B
            H[m * b:(m + 1) * b, n * b:(n + 1) * b] = B.conj().T
    return H[:D, :D]


def dvr_apply_fft(op, x):
    """DVR product y = (T + V) x for any D by the FFT: T is the symmetric
    Toeplitz matrix of T(k), so T x is the first D entries of the circular
    convolution of the length-2D embedding [T(0..D-1), 0, T(D-1..1)] with
    [x, 0] (a library FFT as one step), plus V_i x_i."""
    D = op.D
    x = np.asarray(x, dtype=np.complex128).reshape(D)
    t = kinetic_window(op, 0, 0, D, 1)[:, 0]
    c = np.concatenate([t, [0.0], t[:0:-1]])
    xp = np.concatenate([x, np.zeros(D, dtype=np.complex128)])
    y = np.fft.ifft(np.fft.fft(c) * np.fft.fft(xp))[:D]
    V = np.array([potential(op, i) for i in range(D)])
    return y + V * x
