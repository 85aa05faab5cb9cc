"""Failure detection without a GPU fault.

* A bounded device wait made to run out: a tensor-core (BF16X2) plan whose
  spin limit is one poll.  The kernel must stop on its own, free its tensor
  memory and report MF_ERR_TIMEOUT through mf_sync or through the next call;
  the report clears the word, and the context stays usable (a fresh plan then
  computes the right product).
* Host-side injection (MF_FAULT, include/mf.h): a failing device allocation at
  every allocation site of plan creation returns MF_ERR_OOM and leaks no
  device memory; a failing launch returns MF_ERR_CUDA and the plan works on
  the next call; a candidate that fails to build makes the planner take the
  next one.
"""
import os

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


@pytest.fixture
def fault():
    """Set MF_FAULT for one test and always clear it afterwards."""
    def set_(v):
        os.environ["MF_FAULT"] = v
    yield set_
    os.environ.pop("MF_FAULT", None)


def _bf16x2_ref(D, X):
    return O.apply_bf16x2(O.make_op(O.GEN_PHILOX_GUE, D, seed=1), X)


def test_bounded_wait_times_out_and_reports(mf):
    D, nv = 1024, 8
    X = W.random_state(D, nv, seed=2).reshape(D, nv)
    xd = torch.from_numpy(X).cuda()
    yd = torch.empty_like(xd)
    p = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=1, precision=mf.MF_PREC_BF16X2, nvec_hint=nv, spin_limit=1)
    assert p.describe()["spin_limit"] == 1
    p.apply(yd, xd, nv)
    with pytest.raises(mf.MFError) as e:
        p.sync()
    assert e.value.status == mf.MF_ERR_TIMEOUT
    code = p.describe()["last_device_error"]
    assert 100 <= code <= 199
    p.sync()  # the report cleared the word
    # the next call reports a time-out of the call before it, without blocking
    p.apply(yd, xd, nv)
    torch.cuda.synchronize()
    with pytest.raises(mf.MFError) as e:
        p.apply(yd, xd, nv)
    assert e.value.status == mf.MF_ERR_TIMEOUT
    p.close()
    # the context is intact: a plan with the default limit computes the product
    q = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=1, precision=mf.MF_PREC_BF16X2, nvec_hint=nv)
    q.apply(yd, xd, nv)
    q.sync()
    ref = _bf16x2_ref(D, X)
    got = yd.cpu().numpy()
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 2e-5
    q.close()


def _create_cached_plan(mf):
    # partial cache, so creation allocates the cache, pair lists, work list,
    # Hermitian items and the workspace
    return mf.Plan(4096, mf.MF_GEN_PHILOX_GUE, seed=3, block=512, cache_budget_bytes=20 * 512 * 512 * 8,
                   precision=mf.MF_PREC_FP32, storage=mf.MF_STORE_PARTIAL, nvec_hint=4)


def test_injected_allocation_failures_leak_nothing(mf, fault):
    p = _create_cached_plan(mf)  # warm-up: loads the code, sizes any driver pools
    p.close()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    n_fail = 0
    for n in range(1, 64):
        fault("alloc:%d" % n)
        try:
            p = _create_cached_plan(mf)
        except mf.MFError as e:
            assert e.status == mf.MF_ERR_OOM
            n_fail += 1
            continue
        p.close()
        break
    else:
        pytest.fail("plan creation never got past the injected failures")
    assert n_fail >= 6  # every allocation site of this plan was hit once
    os.environ.pop("MF_FAULT", None)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) <= 4 << 20
    # and a plan created afterwards works
    p = _create_cached_plan(mf)
    X = W.random_state(4096, 4, seed=5).reshape(4096, 4)
    xd = torch.from_numpy(X).cuda()
    yd = torch.empty_like(xd)
    p.apply(yd, xd, 4)
    torch.cuda.synchronize()
    ref = O.apply(O.make_op(O.GEN_PHILOX_GUE, 4096, seed=3, form=O.FORM_FP32), X)
    assert np.max(np.abs(yd.cpu().numpy() - ref)) / np.max(np.abs(ref)) < 2e-5
    p.close()


def test_injected_launch_failure_then_recovery(mf, fault):
    D = 2048
    x = W.random_state(D, 1, seed=6)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    p = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=2, precision=mf.MF_PREC_FP64)
    fault("launch:1")
    with pytest.raises(mf.MFError) as e:
        p.apply(yd, xd, 1)
    assert e.value.status == mf.MF_ERR_CUDA
    p.apply(yd, xd, 1)  # the second launch is not injected
    torch.cuda.synchronize()
    ref = O.apply(O.make_op(O.GEN_PHILOX_GUE, D, seed=2), x)
    assert np.max(np.abs(yd.cpu().numpy() - ref)) / np.max(np.abs(ref)) < 1e-12
    p.close()


def test_planner_moves_past_a_candidate_that_fails(mf, fault):
    D = 4096
    base = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=1, precision=mf.MF_PREC_FP32, cache_budget_bytes=1 << 30)
    first = base.describe()
    base.close()
    fault("plan:1")
    p = mf.Plan(D, mf.MF_GEN_PHILOX_GUE, seed=1, precision=mf.MF_PREC_FP32, cache_budget_bytes=1 << 30)
    second = p.describe()
    assert (second["block"], second["storage"]) != (first["block"], first["storage"])
    x = W.random_state(D, 1, seed=7)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    p.apply(yd, xd, 1)
    torch.cuda.synchronize()
    ref = O.apply(O.make_op(O.GEN_PHILOX_GUE, D, seed=1, form=O.FORM_FP32), x)
    assert np.max(np.abs(yd.cpu().numpy() - ref)) / np.max(np.abs(ref)) < 2e-5
    p.close()
