"""GPU parity of the system-bath plan (Sec. VII: H_S (x) I + I (x) H_B +
g sum_a A_a (x) B_a with on-demand Philox bath operators) against the
oracle's matrix-free statement, and of its propagators against the dense
Kronecker form's eigendecomposition.

Bars: FP64 form 1e-12 of max|y| (accumulation order only); FP32 form 2e-5
(FP32 tile sums and FP32 mixed inputs, against the oracle on the same
FP32-form entries)."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mf():
    import paper_2606_31598_gb300 as mf
    mf.lib()
    return mf


def _herm(rng, n):
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return 0.5 * (M + M.conj().T)


def _model(d_S, n_int, seed=0):
    rng = np.random.default_rng(seed)
    H_S = _herm(rng, d_S)
    A = np.stack([_herm(rng, d_S) for _ in range(n_int)]) if n_int else np.zeros((0, d_S, d_S))
    seeds = [101 + 13 * k for k in range(n_int + 1)]
    return H_S, A, seeds


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("d_S,d_B,n_int", [(1, 1000, 1), (4, 1000, 1), (5, 700, 2), (16, 640, 3), (2, 300, 0)])
def test_sysbath_apply_matches_oracle(mf, prec, d_S, d_B, n_int):
    H_S, A, seeds = _model(d_S, n_int, seed=d_S)
    g = 0.45
    p = mf.Plan.sysbath(d_S, d_B, seeds, H_S, A, g, precision=prec)
    assert p.describe()["path"] == "sysbath_rows"
    rng = np.random.default_rng(7)
    X = rng.standard_normal((d_B, d_S)) + 1j * rng.standard_normal((d_B, d_S))
    ref = O.sysbath_apply(d_S, d_B, seeds, H_S, A, g, X, form=O.FORM_FP64 if prec == 0 else O.FORM_FP32)
    xd = _dev(X)
    yd = torch.empty_like(xd)
    p.apply(yd, xd, d_S)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    assert np.max(np.abs(y - ref)) < (1e-12 if prec == 0 else 2e-5) * np.max(np.abs(ref))
    p.close()


def test_sysbath_propagators_match_dense_kronecker_form(mf):
    """d_S = 4, d_B = 256 (D = 1024): exp(-i t H) psi and the normalised
    exp(-tau (H - E_min)) psi against eigh of the dense composite."""
    d_S, d_B, n_int, g = 4, 256, 2, 0.3
    H_S, A, seeds = _model(d_S, n_int, seed=11)
    H = O.sysbath_dense(d_S, d_B, seeds, H_S, A, g)
    w, V = np.linalg.eigh(H)
    p = mf.Plan.sysbath(d_S, d_B, seeds, H_S, A, g, precision=0, cheb_tol=1e-14)
    emin, emax = p.bounds()
    assert emin < w[0] and w[-1] < emax   # Lanczos on the composite encloses its spectrum
    rng = np.random.default_rng(5)
    psi = rng.standard_normal(d_S * d_B) + 1j * rng.standard_normal(d_S * d_B)
    psi /= np.linalg.norm(psi)
    d = _dev(O.bath_major(psi, d_S, d_B))
    p.cheb_propagate(d, d_S, 0.7, 0)
    torch.cuda.synchronize()
    exact = V @ (np.exp(-0.7j * w) * (V.conj().T @ psi))
    assert np.max(np.abs(d.cpu().numpy() - O.bath_major(exact, d_S, d_B))) < 1e-10
    tau = 0.8
    d = _dev(O.bath_major(psi, d_S, d_B))
    p.cheb_filter(d, d_S, tau, 0, True)
    torch.cuda.synchronize()
    f = V @ (np.exp(-tau * (w - emin)) * (V.conj().T @ psi))
    f /= np.linalg.norm(f)
    assert np.max(np.abs(d.cpu().numpy() - O.bath_major(f, d_S, d_B))) < 1e-10
    p.close()


def test_sysbath_hermitian_on_gpu(mf):
    d_S, d_B = 3, 900
    H_S, A, seeds = _model(d_S, 1, seed=4)
    p = mf.Plan.sysbath(d_S, d_B, seeds, H_S, A, 0.8, precision=0)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((d_B, d_S)) + 1j * rng.standard_normal((d_B, d_S))
    y = rng.standard_normal((d_B, d_S)) + 1j * rng.standard_normal((d_B, d_S))
    outs = []
    for v in (x, y):
        vd = _dev(v)
        od = torch.empty_like(vd)
        p.apply(od, vd, d_S)
        torch.cuda.synchronize()
        outs.append(od.cpu().numpy())
    lhs, rhs = np.vdot(x, outs[1]), np.vdot(outs[0], y)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    p.close()


def test_sysbath_bad_calls(mf):
    H_S, A, seeds = _model(4, 1)
    p = mf.Plan.sysbath(4, 500, seeds, H_S, A, 0.1, precision=1)
    x = _dev(np.zeros((500, 4), np.complex128))
    y = torch.empty_like(x)
    with pytest.raises(mf.MFError):
        p.apply(y, x, 2)             # nvec must be d_S
    with pytest.raises(mf.MFError):
        p.cheb_propagate(x, 3, 0.1, 4)
    p.close()
    with pytest.raises(mf.MFError):
        mf.Plan.sysbath(4, 500, seeds, H_S, A, 0.1, precision=mf.MF_PREC_BF16X2)
