"""The allocation-free entry point mf_apply_dvr_noalloc.

Callers that cannot allocate device memory while they run use this call; it
must give the same product as the plan-based mf_apply (same kernels, same
launch shape) and stay correct when called repeatedly, since every call
reuses the library's one fixed scratch array.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("D", [131072, 1000])
def test_noalloc_matches_plan_apply_twice(D):
    import paper_2606_31598_gb300 as mf
    L = mf.lib()
    stream = torch.cuda.current_stream().cuda_stream
    plan = mf.Plan(D, mf.MF_GEN_SINC_DVR_HO, precision=mf.MF_PREC_FP32, stream=stream)
    for seed in (1, 2):  # two calls in a row, different inputs
        x = torch.from_numpy(W.random_state(D, 1, seed=seed)).cuda()
        y_plan = torch.empty_like(x)
        plan.apply(y_plan, x, 1)
        y = torch.full_like(x, float("nan"))
        st = L.mf_apply_dvr_noalloc(ctypes.c_int64(D), ctypes.c_double(0.0), ctypes.c_void_p(x.data_ptr()),
                                    ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(stream))
        assert st == mf.MF_OK
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), y_plan.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.max(np.abs(a - b)) / np.max(np.abs(b)) < 2e-5
    plan.close()


def test_noalloc_rejects_sizes_beyond_limit():
    import paper_2606_31598_gb300 as mf
    L = mf.lib()
    x = torch.zeros(4, dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    st = L.mf_apply_dvr_noalloc(ctypes.c_int64(131073), ctypes.c_double(0.0), ctypes.c_void_p(x.data_ptr()),
                                ctypes.c_void_p(y.data_ptr()), None)
    assert st == mf.MF_ERR_INVALID
    st = L.mf_apply_dvr_noalloc(ctypes.c_int64(4), ctypes.c_double(0.0), ctypes.c_void_p(x.data_ptr()),
                                ctypes.c_void_p(x.data_ptr()), None)
    assert st == mf.MF_ERR_INVALID
