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
