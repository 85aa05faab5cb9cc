"""Plan records for continuation runs: a plan rebuilt by mf_plan_deserialize
from mf_plan_serialize's record takes the recorded block size, storage mode
and cache share without planning (no candidates measured) and the recorded
spectral bounds without a Lanczos run, and gives the original plan's
products and Chebyshev steps bit for bit (and the oracle's within the form's
tolerance)."""
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


def _same_plan(mf, p, q):
    a, b = p.describe(), q.describe()
    for k in ("D", "generator", "seed", "precision", "block", "n_blk", "storage", "pairs_cached", "path",
              "dvr_rows", "dvr_cols", "n_slot", "tc_walk", "tch_unit", "cache_format"):
        assert a[k] == b[k], k
    assert b["deserialized"] and not a["deserialized"]


def _apply(plan, X, nvec):
    x = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    y = torch.empty((plan._rows(), nvec) if nvec > 1 else (plan._rows(),), dtype=torch.complex128, device="cuda")
    plan.apply(y, x, nvec)
    torch.cuda.synchronize()
    plan.sync()
    return y.cpu().numpy()


def _step(plan, X, nvec, dt):
    d = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    plan.cheb_propagate(d, nvec, dt, 0)
    torch.cuda.synchronize()
    plan.sync()
    return d.cpu().numpy()


def test_autotuned_plan_round_trip(mf):
    D, nv = 4096, 4
    p = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=5, precision=mf.MF_PREC_FP32, nvec_hint=nv,
                cache_budget_bytes=1 << 30, planner_mode=mf.MF_PLANNER_AUTOTUNE, autotune_k=3, autotune_repeats=1)
    assert len(p.trials()) >= 2  # the autotuner measured candidates
    emin, emax = p.bounds()
    rec = p.serialize()
    q = mf.Plan.deserialize(rec)
    _same_plan(mf, p, q)
    assert q.bounds() == (emin, emax)  # recorded, not recomputed
    assert len(q.trials()) == 1 and q.trials()[0]["deserialized"]
    X = W.random_state(D, nv, seed=7).reshape(D, nv)
    ya, yb = _apply(p, X, nv), _apply(q, X, nv)
    assert np.array_equal(ya, yb)
    ref = O.apply(O.make_op(O.GEN_PHILOX_GUE, D, seed=5, form=O.FORM_FP32), X)
    assert np.max(np.abs(yb - ref)) / np.max(np.abs(ref)) < 2e-5
    assert np.array_equal(_step(p, X, nv, 0.7), _step(q, X, nv, 0.7))
    assert q.serialize() == rec
    p.close()
    q.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_dvr_plan_round_trip(mf, prec):
    D = 10000
    p = mf.Plan(D, mf.MF_GEN_SINC_DVR_HO, precision=prec)
    p.bounds()
    q = mf.Plan.deserialize(p.serialize())
    _same_plan(mf, p, q)
    x = W.random_state(D, 1, seed=3)
    assert np.array_equal(_apply(p, x, 1), _apply(q, x, 1))
    assert np.array_equal(_step(p, x, 1, 2e-4), _step(q, x, 1, 2e-4))
    p.close()
    q.close()


def test_tensor_core_plan_with_cache_round_trip(mf):
    D, nv, b = 4100, 16, 512
    p = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=8, block=b, precision=mf.MF_PREC_BF16X2, nvec_hint=nv,
                cache_budget_bytes=12 * b * b * 8, storage=mf.MF_STORE_PARTIAL)
    q = mf.Plan.deserialize(p.serialize())
    _same_plan(mf, p, q)
    assert q.describe()["pairs_cached"] == 12
    X = W.random_state(D, nv, seed=9).reshape(D, nv)
    assert np.array_equal(_apply(p, X, nv), _apply(q, X, nv))
    p.close()
    q.close()


def test_row_slice_plan_round_trip(mf):
    D, nv = 1000, 2
    p = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=6, block=256, precision=mf.MF_PREC_FP64, row_begin=256, row_end=768,
                cache_budget_bytes=2 * 16 * 256 * 256)
    q = mf.Plan.deserialize(p.serialize())
    _same_plan(mf, p, q)
    assert (q.row_begin, q.row_end) == (256, 768)
    X = W.random_state(D, nv, seed=2).reshape(D, nv)
    ya, yb = _apply(p, X, nv), _apply(q, X, nv)
    assert np.array_equal(ya, yb)
    ref = O.apply(O.make_op(O.GEN_PHILOX_GUE, D, seed=6), X)[256:768]
    assert np.max(np.abs(yb - ref)) / np.max(np.abs(ref)) < 1e-12
    p.close()
    q.close()


def test_system_bath_plans_are_not_serialised(mf):
    H = np.eye(2, dtype=np.complex128)
    p = mf.Plan.sysbath(2, 256, [1], H, None, 0.0, precision=mf.MF_PREC_FP64)
    with pytest.raises(mf.MFError) as e:
        p.serialize()
    assert e.value.status == mf.MF_ERR_UNSUPPORTED
    p.close()
