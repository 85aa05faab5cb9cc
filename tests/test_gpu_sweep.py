"""Seeded sweep over shapes and plan options through the C ABI.

Each case draws a generator, a precision form, a storage mode, a block size,
a dimension D (every size next to a tile, chunk or block edge first, then
random sizes up to 1500) and a vector count (1..20, so every compiled
vector bucket and its padding is reached), applies the plan, then applies it
again with another vector count (the workspace is re-sized or reused), and
compares both products with the oracle within the bar of the form:

* FP64 form: 1e-12 of max|y| (summation order only);
* FP32 form: 2e-5 of max|y| against the oracle product of the FP32-form
  entries (FP32 tile sums);
* BF16X2 form: 2e-5 of max|y| against the oracle's split product.

Fixed-size tests pin each kernel; this sweep is there for index and
workspace mistakes at sizes nobody picked by hand.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

EDGE_D = [2, 3, 15, 16, 17, 31, 33, 127, 128, 129, 255, 256, 257, 383, 511, 513, 1023, 1025]
NVECS = [1, 1, 2, 3, 4, 5, 6, 7, 8, 9, 11, 12, 13, 16, 17, 20]


def _cases(n=54, seed=2024):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        D = EDGE_D[i] if i < len(EDGE_D) else int(rng.integers(2, 1501))
        gen = int(rng.integers(0, 2))
        prec = int(rng.integers(0, 3))
        storage = int(rng.integers(0, 3))
        nvec = int(rng.choice(NVECS))
        nvec2 = int(rng.choice(NVECS))
        out.append((i, gen, prec, storage, D, nvec, nvec2))
    return out


@pytest.fixture(scope="module")
def mf():
    import paper_2606_31598_gb300 as mf
    mf.lib()
    return mf


def _make_plan(mf, gen, prec, storage, D, nvec):
    """Storage modes with an explicit 128 block so a partial cache exists
    whenever D spans two blocks; full caches get room for every pair."""
    eb = 16 if prec == 0 else 8
    nblk = (D + 127) // 128
    npair = nblk * (nblk + 1) // 2
    if storage == 1 and npair < 2:
        storage = 2
    if storage == 0:
        return mf.Plan(D, gen, seed=11, block=0, precision=prec, storage=mf.MF_STORE_PROCEDURAL, nvec_hint=nvec)
    budget = eb * 128 * 128 * (npair if storage == 2 else max(1, npair // 3))
    st = mf.MF_STORE_FULL if storage == 2 else mf.MF_STORE_PARTIAL
    return mf.Plan(D, gen, seed=11, block=128, cache_budget_bytes=budget, precision=prec, storage=st, nvec_hint=nvec)


def _reference(gen, prec, D, X):
    op = O.make_op(gen, D, seed=11, form=O.FORM_FP64 if prec == 0 else O.FORM_FP32)
    if prec == 2:
        H32 = O.window_native(O.make_op(gen, D, seed=11, form=O.FORM_FP32), 0, 0, D, D)
        return O.apply_bf16x2(O.make_op(gen, D, seed=11), X, H32)
    return O.apply(op, X)


@pytest.mark.parametrize("case", _cases(), ids=lambda c: "c%d-g%d-p%d-s%d-D%d-v%d-v%d" % c)
def test_sweep_apply_matches_oracle(mf, case):
    _, gen, prec, storage, D, nvec, nvec2 = case
    p = _make_plan(mf, gen, prec, storage, D, nvec)
    bar = 1e-12 if prec == 0 else 2e-5
    for k, nv in enumerate((nvec, nvec2)):
        X = W.random_state(D, nv, seed=100 + k)
        X = X.reshape(D, nv)
        x = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        y = torch.empty_like(x)
        p.apply(y, x, nv)
        torch.cuda.synchronize()
        p.sync()
        Y = y.cpu().numpy()
        ref = _reference(gen, prec, D, X)
        err = float(np.max(np.abs(Y - ref)) / np.max(np.abs(ref)))
        assert err < bar, (nv, err)
    p.close()


def _cheb_cases(n=16, seed=77):
    rng = np.random.default_rng(seed)
    out = []
    edges = [2, 129, 513]
    for i in range(n):
        D = edges[i] if i < len(edges) else int(rng.integers(2, 901))
        out.append((i, int(rng.integers(0, 2)), int(rng.integers(0, 2)), int(rng.integers(0, 3)), D,
                    int(rng.choice(NVECS)), float(rng.uniform(0.2, 1.0))))
    return out


@pytest.mark.parametrize("case", _cheb_cases(), ids=lambda c: "c%d-g%d-p%d-s%d-D%d-v%d-t%.2f" % c)
def test_sweep_chebyshev_matches_oracle(mf, case):
    """One Chebyshev step of exp(-i dt H) (Sec. VII) at drawn shapes; dt is
    capped so R dt <= 8 (a few tens of terms) and the oracle runs the same
    recurrence on the same form's entries with the plan's bounds."""
    _, gen, prec, storage, D, nvec, dt = case
    p = _make_plan(mf, gen, prec, storage, D, nvec)
    emin, emax = p.bounds()
    c, R = 0.5 * (emax + emin), 0.5 * (emax - emin)
    dt = min(dt, 8.0 / R)
    nt = p.cheb_terms(dt)
    X = W.random_state(D, nvec, seed=5).reshape(D, nvec)
    d = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    p.cheb_propagate(d, nvec, dt, nt)
    torch.cuda.synchronize()
    got = d.cpu().numpy()
    op = O.make_op(gen, D, seed=11, form=O.FORM_FP64 if prec == 0 else O.FORM_FP32)
    ref = O.cheb_step(op, X, dt, c, R, nt)
    err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    assert err < (1e-11 if prec == 0 else 2e-5), err
    p.close()


def _slice_cases(n=12, seed=99):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        D = int(rng.integers(129, 1501))
        ntile = -(-D // 128)
        world = int(rng.integers(2, min(4, ntile) + 1))
        out.append((i, int(rng.integers(0, 2)), int(rng.integers(0, 2)), D, world, int(rng.choice(NVECS))))
    return out


@pytest.mark.parametrize("case", _slice_cases(), ids=lambda c: "c%d-g%d-p%d-D%d-w%d-v%d" % c)
def test_sweep_row_slices_reassemble_the_product(mf, case):
    """Row-slice plans (row-parallel mode of Sec. IV.H) at drawn sizes and
    rank counts, every other slice with a partial cache of its block pairs:
    the slices' products stacked are the oracle's product."""
    from paper_2606_31598_gb300 import rowgroup
    _, gen, prec, D, world, nvec = case
    eb = 16 if prec == 0 else 8
    X = W.random_state(D, nvec, seed=6).reshape(D, nvec)
    xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    parts = []
    for k, (r0, r1) in enumerate(rowgroup.slices(D, world)):
        budget = eb * 128 * 128 * 2 if k % 2 else 0
        p = mf.Plan(D, gen, seed=11, block=128, precision=prec, cache_budget_bytes=budget,
                    storage=mf.MF_STORE_PARTIAL if budget else mf.MF_STORE_PROCEDURAL, row_begin=r0, row_end=r1)
        y = torch.empty((r1 - r0, nvec), dtype=torch.complex128, device="cuda")
        p.apply(y, xd, nvec)
        torch.cuda.synchronize()
        parts.append(y.cpu().numpy())
        p.close()
    got = np.concatenate(parts)
    ref = O.apply(O.make_op(gen, D, seed=11, form=O.FORM_FP64 if prec == 0 else O.FORM_FP32), X)
    err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    assert err < (1e-12 if prec == 0 else 2e-5), err
