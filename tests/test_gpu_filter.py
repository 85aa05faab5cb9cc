"""GPU parity of the imaginary-time Chebyshev filter (thermal pure states,
Sec. I and Sec. VII) against the CPU oracle, through the C ABI.

Bars, relative to the largest input entry (the series adds terms of the
input's size into a smaller result): FP64 form 1e-13 (accumulation order
only), FP32 form 1e-5 (FP32 tile sums, as for the real-time propagator);
normalised outputs divide the bar by the filtered column norm.  The harmonic
oscillator's coherent-state closed form holds to 1e-8."""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mf():
    import paper_2606_31598_gb300 as mf
    mf.lib()
    return mf


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nvec", [1, 5])
@pytest.mark.parametrize("normalize", [False, True])
def test_filter_matches_oracle_gue(mf, prec, nvec, normalize):
    """D = 1000 (ragged against the 128-row tile) Philox ensemble (spectrum
    near [-2, 2]), tau = 3, bounds set explicitly so both sides use the same
    c and R.  The series sums terms of the input's size to a smaller result,
    so the bars are relative to the input (and, normalised, divided by the
    filtered column norm)."""
    D, tau = 1000, 3.0
    p = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=2, precision=prec)
    p.set_bounds(-2.2, 2.2)
    c, R = 0.0, 2.2
    nt = O.cheb_imag_terms(R * tau, 1e-15)
    op = O.make_op(O.GEN_PHILOX_GUE, D, seed=2, form=O.FORM_FP64 if prec == 0 else O.FORM_FP32)
    psi = W.random_state(D, nvec, seed=4)
    raw = O.cheb_imag_step(op, psi, tau, c, R, nt, normalize=False).reshape(D, nvec)
    ref = raw / np.linalg.norm(raw, axis=0) if normalize else raw
    d = _dev(psi)
    p.cheb_filter(d, nvec, tau, nt, normalize)
    torch.cuda.synchronize()
    out = d.cpu().numpy().reshape(D, nvec)
    tol = (1e-13 if prec == 0 else 1e-5) * np.max(np.abs(psi))
    if normalize:
        tol /= np.min(np.linalg.norm(raw, axis=0))
        assert np.max(np.abs(np.linalg.norm(out, axis=0) - 1)) < 1e-12
    assert np.max(np.abs(out - ref)) < tol


def test_filter_terms_rule(mf):
    p = mf.Plan(2048, mf.MF_GEN_PHILOX_GUE, seed=1, precision=0)
    emin, emax = p.bounds()
    R = 0.5 * (emax - emin)
    for tau in (0.0, 0.05, 0.5, 4.0):
        assert p.cheb_filter_terms(tau) == O.cheb_imag_terms(R * tau, 1e-7)


def test_filter_dvr_coherent_state_closed_form(mf):
    """exp(-tau H) moves the harmonic-oscillator coherent state from x0 to
    x0 e^{-tau}; with the analytic DVR bounds (E_min = 0) the unnormalised
    norm is e^{-tau/2} exp(-x0^2 (1 - e^{-2 tau}) / 4)."""
    D, tau, x0 = 512, 0.6, 2.0
    p = mf.Plan(D, mf.MF_GEN_SINC_DVR_HO, precision=0, cheb_tol=1e-15)
    emin, _ = p.bounds()
    assert emin == 0.0
    L = W.dvr_default_L(D)
    x = -L + 2 * L / (D - 1) * np.arange(D)
    g = lambda m: np.exp(-0.5 * (x - m) ** 2) / np.linalg.norm(np.exp(-0.5 * (x - m) ** 2))
    d = _dev(g(x0).astype(np.complex128))
    p.cheb_filter(d, 1, tau, 0, False)
    torch.cuda.synchronize()
    raw = d.cpu().numpy()
    assert abs(np.linalg.norm(raw) - np.exp(-tau / 2) * np.exp(-x0 ** 2 * (1 - np.exp(-2 * tau)) / 4)) < 1e-8
    d = _dev(g(x0).astype(np.complex128))
    p.cheb_filter(d, 1, tau, 0, True)
    torch.cuda.synchronize()
    assert np.max(np.abs(d.cpu().numpy() - g(x0 * np.exp(-tau)))) < 1e-8


def test_tpq_energy_decreases_with_beta(mf):
    """Canonical thermal pure states |beta> = exp(-beta H / 2) r / norm from
    one random vector: <H> falls monotonically with beta toward E_0, and is
    the infinite-temperature mean Tr H / D (about 0) at beta = 0.  The energy
    <beta|H|beta> is read through mf_apply."""
    D = 4096
    p = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=5, precision=0)
    r = W.random_state(D, 1, seed=7)
    E = []
    for beta in (0.0, 0.1, 0.4, 1.6):
        d = _dev(r)
        p.cheb_filter(d, 1, beta / 2, 0, True)
        y = torch.empty_like(d)
        p.apply(y, d, 1)
        torch.cuda.synchronize()
        E.append(float(torch.vdot(d, y).real))
    assert abs(E[0]) < 4.0   # Tr H / D ~ N(0, 1/D) per diagonal entry; r is random
    assert all(a > b for a, b in zip(E, E[1:]))
    emin, _ = p.bounds()
    assert E[-1] > emin


def test_filter_zero_tau_is_identity_and_bad_calls(mf):
    D = 700
    p = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=1, precision=1)
    psi = W.random_state(D, 2, seed=3)
    d = _dev(psi)
    p.cheb_filter(d, 2, 0.0, 0, False)
    torch.cuda.synchronize()
    assert np.max(np.abs(d.cpu().numpy() - psi)) < 1e-15
    with pytest.raises(mf.MFError):
        p.cheb_filter(d, 2, -0.1, 0, True)
    with pytest.raises(mf.MFError):
        p.cheb_filter(d, 65, 0.1, 0, True)
