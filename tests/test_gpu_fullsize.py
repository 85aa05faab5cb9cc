"""The 64-vector workload at its full size, in the launch shape the benchmark
times: Philox ensemble D = 262144 (seed 1), block 2048 (128 block rows,
8256 canonical pairs), 120 GB partial cache (the first 3576 pairs: block
rows 0..30 and pairs (31, 31..103)), 64 unit vectors (seed 2), in the BF16X2
and FP32 forms.  Sampled output rows are computed by the oracle one by one
and compared element by element at 2e-5 of max|y|: rows at row-tile (128),
block (2048) and cache boundaries and the last row.  The dense operator
(1.1 TB in complex128) is never formed."""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

D, R, B = 262144, 64, 2048
BUDGET = int(120e9)
ROWS = np.array([0, 127, 128, 2047, 2048, 63488, 63615, 65535, 65536, 131071, 212991, 212992, 262143])


@pytest.fixture(scope="module")
def mf():
    import paper_2606_31598_gb300 as mf
    mf.lib()
    return mf


@pytest.fixture(scope="module")
def X():
    return W.random_state(D, R, seed=2).reshape(D, R)


def _product_rows(mf, X, prec):
    plan = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=1, block=B, cache_budget_bytes=BUDGET, precision=prec,
                   storage=mf.MF_STORE_PARTIAL, nvec_hint=R)
    desc = plan.describe()
    assert desc["pairs_cached"] == 3576 and desc["n_pair"] == 8256
    x = torch.from_numpy(X).cuda()
    y = torch.empty_like(x)
    plan.apply(y, x, R)
    torch.cuda.synchronize()
    plan.sync()
    rows = y[torch.from_numpy(ROWS).cuda()].cpu().numpy()
    plan.close()
    del x, y
    torch.cuda.empty_cache()
    return rows


def test_full_size_bf16x2_sampled_rows(mf, X):
    got = _product_rows(mf, X, mf.MF_PREC_BF16X2)
    ref = O.apply_rows_bf16x2(O.make_op(O.GEN_PHILOX_GUE, D, seed=1), X, ROWS)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) / scale < 2e-5
    # stated error of the split form against the FP64 operator on these rows
    ref64 = O.apply_rows(O.make_op(O.GEN_PHILOX_GUE, D, seed=1), X, ROWS)
    assert np.max(np.abs(got - ref64)) / np.max(np.abs(ref64)) < 1e-4


def test_full_size_fp32_sampled_rows(mf, X):
    got = _product_rows(mf, X, mf.MF_PREC_FP32)
    ref = O.apply_rows(O.make_op(O.GEN_PHILOX_GUE, D, seed=1, form=O.FORM_FP32), X, ROWS)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 2e-5
