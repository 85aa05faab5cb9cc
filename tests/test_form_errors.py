"""Errors of the precision forms against the FP64 form on the DVR workload
(D = 131072, a 64-term Chebyshev step of the coherent state), computed by the
oracle in exact form arithmetic, and the oracle pieces they rest on pinned
against the dense and blockwise statements.  The GPU's own FP32-form error is
measured by bench.py; the kernels' agreement with each form is the subject
of the GPU parity tests."""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O


@pytest.mark.parametrize("D", [700, 1024])
def test_fft_forms_match_the_dense_statements(D):
    """DvrToeplitz (FFT, any D) against the dense BF16X2 statement and the
    blockwise FP64 product at sizes both can run."""
    T = O.DvrToeplitz(D)
    rng = np.random.default_rng(D)
    x = rng.standard_normal(D) + 1j * rng.standard_normal(D)
    op = O.make_op(O.GEN_SINC_DVR_HO, D)
    ref_bf = O.apply_bf16x2(op, x)
    ref64 = O.apply(op, x)
    assert np.max(np.abs(T.apply_bf16x2(x) - ref_bf)) < 1e-12 * np.max(np.abs(ref_bf))
    assert np.max(np.abs(T.apply64(x) - ref64)) < 1e-12 * np.max(np.abs(ref64))
    # FP32 form with exact sums: the C oracle's FP32-form product of the
    # complex64-rounded x (its potential term takes the rounded x too)
    x32 = x.astype(np.complex64).astype(np.complex128)
    V = np.array([O.potential(op, i) for i in range(D)])
    ref32 = O.apply(O.make_op(O.GEN_SINC_DVR_HO, D, form=O.FORM_FP32), x32) - V * x32 + V * x
    assert np.max(np.abs(T.apply32(x) - ref32)) < 1e-12 * np.max(np.abs(ref32))


def test_python_recurrence_matches_the_c_oracle():
    """cheb_step_fn with the FFT product against the C oracle's step."""
    D, dt = 1000, 2e-3
    op = O.make_op(O.GEN_SINC_DVR_HO, D)
    L = O.dvr_default_L(D)
    dx = 2.0 * L / (D - 1)
    emax = np.pi ** 2 / (2.0 * dx * dx) + 0.5 * L * L
    c, R = 0.5 * emax, 0.5 * emax
    nt = O.cheb_terms(R * dt, 1e-12)
    psi = W.wavepacket(D)
    got = O.cheb_step_fn(O.DvrToeplitz(D).apply64, psi, dt, c, R, nt)
    assert np.max(np.abs(got - O.cheb_step(op, psi, dt, c, R, nt))) < 1e-12


def test_bf16x2_form_error_on_the_dvr_workload():
    """One 64-term step (tau = 4e-4, R tau = 41.2) of the D = 131072 coherent
    state: the BF16X2 form's state differs from the FP64 form's by 1.74e-5
    in the 2-norm (FP32 form on the GPU: 5.3e-7); a single product on a
    random vector by 1.7e-6 of max|y|.  (On the smooth coherent state a
    single product loses far more, 0.12 of max|y|: T psi cancels terms of
    size T(0) ~ 6.6e4, which magnifies the 2^-17 split rounding; the
    Chebyshev step does not inherit it.)"""
    D, tau = 131072, 4.0e-4
    T = O.DvrToeplitz(D)
    L = O.dvr_default_L(D)
    dx = 2.0 * L / (D - 1)
    emax = np.pi ** 2 / (2.0 * dx * dx) + 0.5 * L * L
    c, R = 0.5 * emax, 0.5 * emax
    psi = W.wavepacket(D)
    s64 = O.cheb_step_fn(T.apply64, psi, tau, c, R, 64)
    sbf = O.cheb_step_fn(T.apply_bf16x2, psi, tau, c, R, 64)
    err = np.linalg.norm(sbf - s64)
    assert 5e-6 < err < 5e-5, err
    # the FP32 form's own rounding (exact sums) accounts for nearly all of
    # the FP32 error measured on the GPU (5.3e-7 at tau = 4.14e-4)
    s32 = O.cheb_step_fn(T.apply32, psi, tau, c, R, 64)
    assert 3e-7 < np.linalg.norm(s32 - s64) < 8e-7
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(D) + 1j * rng.standard_normal(D)) / np.sqrt(2.0 * D)
    y64 = T.apply64(x)
    assert np.max(np.abs(T.apply_bf16x2(x) - y64)) < 5e-6 * np.max(np.abs(y64))


@pytest.mark.parametrize("gen", [O.GEN_PHILOX_GUE, O.GEN_SINC_DVR_HO])
def test_row_sampled_bf16x2_form_matches_the_dense_statement(gen):
    """apply_rows_bf16x2 (one generated row at a time, any D) against the
    dense BF16X2 statement at D = 700 with 5 vectors, rows at both ends,
    the diagonal blocks and a ragged tail."""
    D = 700
    op = O.make_op(gen, D, seed=3)
    X = W.random_state(D, 5, seed=4).reshape(D, 5)
    rows = [0, 1, 127, 128, 350, 698, 699]
    ref = O.apply_bf16x2(op, X)[rows]
    got = O.apply_rows_bf16x2(op, X, rows)
    assert np.max(np.abs(got - ref)) < 1e-13 * np.max(np.abs(ref))
