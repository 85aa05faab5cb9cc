"""GPU parity of externally stored blocks (Sec. II: H^[n,m] = D[key(n,m)])
held in host memory: the first P_cache pairs copied into the HBM cache, the
rest read by the kernels over the host link, against the oracle's assembly
of the same blocks (dense product).

Bars: FP64 form 1e-12 of max|y|; FP32 form 2e-5 (FP32 tile sums, against the
FP64 product of the same complex64 blocks); BF16X2 form 1e-4 (bf16 hi + lo
split of the FP32 blocks)."""
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


def _hermitian(D, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
    return (M + M.conj().T) / np.sqrt(8.0 * D)


def _blocks(H, b, dtype):
    D = H.shape[0]
    nblk = -(-D // b)
    P = np.zeros((nblk * b, nblk * b), dtype=np.complex128)
    P[:D, :D] = H
    out = np.stack([P[n * b:(n + 1) * b, m * b:(m + 1) * b] for n, m in O.external_pairs(D, b)])
    return np.ascontiguousarray(out.astype(dtype))


def _apply(plan, X):
    xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    yd = torch.empty_like(xd)
    plan.apply(yd, xd, 1 if X.ndim == 1 else X.shape[1])
    torch.cuda.synchronize()
    return yd.cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("budget_pairs", [0, 3, 100])
@pytest.mark.parametrize("nvec", [1, 2, 3, 16])
def test_external_apply_matches_oracle(mf, prec, budget_pairs, nvec):
    D, b = 1000, 256   # 4 x 4 blocks, ragged last block; 10 stored pairs
    dt = np.complex128 if prec == 0 else np.complex64
    blocks = _blocks(_hermitian(D, 1), b, dt)
    eb = 16 if prec == 0 else 8
    plan = mf.Plan.external(D, b, blocks, cache_budget_bytes=budget_pairs * eb * b * b, precision=prec)
    d = plan.describe()
    assert d["generator"] == "external"
    assert d["pairs_cached"] == min(10, budget_pairs)
    H = O.external_dense(D, b, blocks)
    rng = np.random.default_rng(nvec)
    X = rng.standard_normal((D, nvec)) + 1j * rng.standard_normal((D, nvec))
    if nvec == 1:
        X = X[:, 0]
    ref = H @ X
    y = _apply(plan, X)
    assert np.max(np.abs(y - ref)) < (1e-12 if prec == 0 else 2e-5) * np.max(np.abs(ref))
    plan.close()


@pytest.mark.parametrize("budget_pairs", [0, 6])
def test_external_tensor_core_form(mf, budget_pairs):
    D, b = 1024, 256
    blocks = _blocks(_hermitian(D, 2), b, np.complex64)
    plan = mf.Plan.external(D, b, blocks, cache_budget_bytes=budget_pairs * 8 * b * b, precision=2)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((D, 16)) + 1j * rng.standard_normal((D, 16))
    ref = O.external_dense(D, b, blocks) @ X
    y = _apply(plan, X)
    assert np.max(np.abs(y - ref)) < 1e-4 * np.max(np.abs(ref))
    plan.close()


def test_external_propagator_matches_eigendecomposition(mf):
    D, b = 640, 128
    H = _hermitian(D, 5)
    blocks = _blocks(H, b, np.complex128)
    plan = mf.Plan.external(D, b, blocks, cache_budget_bytes=4 * 16 * b * b, precision=0, cheb_tol=1e-14)
    w, V = np.linalg.eigh(H)
    emin, emax = plan.bounds()
    assert emin < w[0] and w[-1] < emax
    rng = np.random.default_rng(2)
    psi = rng.standard_normal(D) + 1j * rng.standard_normal(D)
    psi /= np.linalg.norm(psi)
    d = torch.from_numpy(psi.copy()).cuda()
    plan.cheb_propagate(d, 1, 2.0, 0)
    torch.cuda.synchronize()
    exact = V @ (np.exp(-2.0j * w) * (V.conj().T @ psi))
    assert np.max(np.abs(d.cpu().numpy() - exact)) < 1e-11
    plan.close()


def test_external_blocks_of_the_philox_ensemble(mf):
    """The Philox operator's own entries stored as blocks give the Philox
    plan's product (FP32 form, different summation order)."""
    D, b = 768, 256
    gen = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=9, precision=1)
    full = gen.entries(0, 0, D, D).astype(np.complex128)
    blocks = _blocks(full, b, np.complex64)
    ext = mf.Plan.external(D, b, blocks, cache_budget_bytes=0, precision=1)
    rng = np.random.default_rng(4)
    x = rng.standard_normal(D) + 1j * rng.standard_normal(D)
    y1, y2 = _apply(gen, x), _apply(ext, x)
    assert np.max(np.abs(y1 - y2)) < 2e-5 * np.max(np.abs(y1))
    gen.close()
    ext.close()


def test_external_bad_calls(mf):
    blocks = _blocks(_hermitian(300, 1), 128, np.complex64)
    with pytest.raises(mf.MFError):
        mf.Plan.external(300, 128, blocks.astype(np.complex128), precision=1)   # wrong element type
    with pytest.raises(mf.MFError):
        mf.Plan.external(300, 100, blocks, precision=1)                        # b not a multiple of 128
    plan = mf.Plan.external(300, 128, blocks, precision=1)
    with pytest.raises(mf.MFError):
        plan.entries(0, 0, 4, 4)                                               # no generator to dump
    plan.close()
