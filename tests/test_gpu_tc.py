"""Tensor-core (tcgen05) BF16 hi+lo split form against the oracle's BF16X2
product: FP32-form entries and the FP32 copy of X split into bf16 hi + lo,
three products per real product, exact sums.  The GPU accumulates in FP32,
so the bar is 2e-5 of max|y| (FP32 sums of up to 6 D exact products)."""
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


def _apply(mf, plan, X):
    x = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    y = torch.empty_like(x)
    plan.apply(y, x, 1 if X.ndim == 1 else X.shape[1])
    torch.cuda.synchronize()
    plan.sync()
    return y.cpu().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("gen", [0, 1])
@pytest.mark.parametrize("nvec", [1, 8, 13, 16, 24, 40, 64])
def test_bf16x2_apply_matches_oracle(mf, gen, nvec):
    D = 1000
    p = mf.Plan(D, gen, seed=3, block=256, precision=mf.MF_PREC_BF16X2)
    X = W.random_state(D, nvec, seed=5)
    Y = _apply(mf, p, X)
    op = O.make_op(gen, D, seed=3)
    H32 = O.window_native(O.make_op(gen, D, seed=3, form=O.FORM_FP32), 0, 0, D, D)
    ref = O.apply_bf16x2(op, X, H32)
    assert _rel(Y, ref) < 2e-5
    if gen == 0:
        # stated error of the split form against the FP64 operator
        assert _rel(Y, O.apply(op, X)) < 1e-4


def test_bf16x2_split_k_and_ragged_tail(mf):
    """D = 4100: several column splits and a ragged last row tile and chunk."""
    D, nvec = 4100, 16
    p = mf.Plan(D, 0, seed=8, block=512, precision=mf.MF_PREC_BF16X2, nvec_hint=nvec)
    X = W.random_state(D, nvec, seed=9)
    Y = _apply(mf, p, X)
    rows = np.array([0, 1, 127, 128, 2047, 4095, 4096, 4099])
    op = O.make_op(O.GEN_PHILOX_GUE, D, seed=8)
    H32 = O.window_native(O.make_op(O.GEN_PHILOX_GUE, D, seed=8, form=O.FORM_FP32), 0, 0, D, D)
    Hr = H32[rows]
    # oracle rows of the split product
    Ar_h, Ar_l = O.split_bf16(Hr.real)
    Ai_h, Ai_l = O.split_bf16(Hr.imag)
    X32 = X.astype(np.complex64)
    Xr_h, Xr_l = O.split_bf16(X32.real)
    Xi_h, Xi_l = O.split_bf16(X32.imag)
    f = lambda a: a.astype(np.float64)
    pr = lambda ah, al, bh, bl: f(ah) @ f(bh) + f(ah) @ f(bl) + f(al) @ f(bh)
    ref = (pr(Ar_h, Ar_l, Xr_h, Xr_l) - pr(Ai_h, Ai_l, Xi_h, Xi_l)) + 1j * (
        pr(Ar_h, Ar_l, Xi_h, Xi_l) + pr(Ai_h, Ai_l, Xr_h, Xr_l))
    assert np.max(np.abs(Y[rows] - ref)) / np.max(np.abs(ref)) < 2e-5
    assert _rel(Y[rows], O.apply_rows(op, X, rows)) < 1e-4


@pytest.mark.parametrize("gen", [0, 1])
def test_bf16x2_cache_modes_bit_identical(mf, gen):
    D, b, nvec = 1000, 256, 16
    X = W.random_state(D, nvec, seed=4)
    ys = []
    for storage, budget in [(mf.MF_STORE_PROCEDURAL, 0), (mf.MF_STORE_PARTIAL, 4 * b * b * 8),
                            (mf.MF_STORE_FULL, 10 * b * b * 8)]:
        p = mf.Plan(D, gen, seed=2, block=b, cache_budget_bytes=budget, precision=mf.MF_PREC_BF16X2, storage=storage)
        ys.append(_apply(mf, p, X))
    assert np.array_equal(ys[0], ys[1]) and np.array_equal(ys[0], ys[2])


def test_bf16x2_chebyshev_multivector(mf):
    D, nvec = 1024, 16
    p = mf.Plan(D, 0, seed=4, block=512, precision=mf.MF_PREC_BF16X2)
    emin, emax = p.bounds()
    X = W.random_state(D, nvec, seed=12)
    d = torch.from_numpy(X.copy()).cuda()
    p.cheb_propagate(d, nvec, 0.5, 20)
    torch.cuda.synchronize()
    p.sync()
    out = d.cpu().numpy()
    H = O.dense(O.make_op(O.GEN_PHILOX_GUE, D, seed=4))
    c, R = 0.5 * (emax + emin), 0.5 * (emax - emin)
    ref = O.cheb_step_dense(H, X, 0.5, c, R, 20)
    assert np.max(np.abs(out - ref)) < 3e-4
    assert np.max(np.abs(np.linalg.norm(out, axis=0) - 1)) < 1e-4


def test_hermitian_walk_is_deterministic_across_runs(mf):
    """The Hermitian tensor-core walk hands units to CTAs through an atomic
    counter, so which SM runs which unit changes from run to run; every unit
    owns its slot rows, each slot element is drained by one thread in a
    fixed order and the gather sums in FP64 in a fixed order, so repeated
    products are bitwise equal (and agree with the row-owner kernel within
    the form's tolerance)."""
    D, nvec = 8192 + 96, 64
    X = W.random_state(D, nvec, seed=21).reshape(D, nvec)
    p = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=3, block=1024, precision=mf.MF_PREC_BF16X2, nvec_hint=nvec,
                cache_budget_bytes=6 * 1024 * 1024 * 8, storage=mf.MF_STORE_PARTIAL)
    assert p.describe()["tc_walk"] == "hermitian"
    ys = [_apply(mf, p, X) for _ in range(3)]
    assert np.array_equal(ys[0], ys[1]) and np.array_equal(ys[0], ys[2])
    q = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=3, block=1024, precision=mf.MF_PREC_BF16X2, nvec_hint=nvec,
                hermitian_reuse=0)
    assert q.describe()["tc_walk"] != "hermitian"
    assert _rel(ys[0], _apply(mf, q, X)) < 2e-5
    p.close()
    q.close()
