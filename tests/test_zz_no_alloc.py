"""The allocation-free entry point mf_apply_dvr_noalloc.

Some callers cannot allocate device memory while they run -- a service whose
device memory is already reserved by another runtime's caching allocator, or
a plugin whose host application forbids cudaMalloc -- so this call keeps its
scratch in one fixed array of the library.  It runs the same kernels in the
same launch shape as the plan path, so its product must equal mf_apply's bit
for bit, and it must stay so when calls of different sizes follow each other
on the shared array (the large case first leaves its data behind for the
small one).  The product is also checked against the oracle, and the device's
free memory must not change across a warmed-up call.  This file is collected
last.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _noalloc(L, D, x, y, stream):
    return L.mf_apply_dvr_noalloc(ctypes.c_int64(D), ctypes.c_double(0.0), ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(stream))


@pytest.mark.parametrize("D", [131072, 1000])
def test_noalloc_matches_plan_apply_and_oracle_twice(D):
    import paper_2606_31598_gb300 as mf
    L = mf.lib()
    stream = torch.cuda.current_stream().cuda_stream
    plan = mf.Plan(D, mf.MF_GEN_SINC_DVR_HO, precision=mf.MF_PREC_FP32, stream=stream)
    op32 = O.make_op(O.GEN_SINC_DVR_HO, D, form=O.FORM_FP32)
    for seed in (1, 2):  # two calls in a row, different inputs
        xh = W.random_state(D, 1, seed=seed)
        x = torch.from_numpy(xh).cuda()
        y_plan = torch.empty_like(x)
        plan.apply(y_plan, x, 1)
        y = torch.full_like(x, float("nan"))
        assert _noalloc(L, D, x, y, stream) == mf.MF_OK
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), y_plan.cpu().numpy()
        assert np.array_equal(a, b)
        ref = O.dvr_apply_fft(op32, xh)
        # a random x has no cancellation: the FP32 tile sums hold 2e-5 of max|y|
        assert np.max(np.abs(a - ref)) / np.max(np.abs(ref)) < 2e-5
    plan.close()


def test_noalloc_call_allocates_nothing():
    import paper_2606_31598_gb300 as mf
    L = mf.lib()
    D = 131072
    stream = torch.cuda.current_stream().cuda_stream
    x = torch.from_numpy(W.random_state(D, 1, seed=3)).cuda()
    y = torch.empty_like(x)
    assert _noalloc(L, D, x, y, stream) == mf.MF_OK  # warm-up: loads the code and the array
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _noalloc(L, D, x, y, stream) == mf.MF_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_bad_arguments():
    import paper_2606_31598_gb300 as mf
    L = mf.lib()
    x = torch.zeros(4, dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    args = lambda D, Lh, xp, yp: (ctypes.c_int64(D), ctypes.c_double(Lh), ctypes.c_void_p(xp), ctypes.c_void_p(yp),
                                  None)
    assert L.mf_apply_dvr_noalloc(*args(131073, 0.0, x.data_ptr(), y.data_ptr())) == mf.MF_ERR_INVALID
    assert L.mf_apply_dvr_noalloc(*args(4, 0.0, x.data_ptr(), x.data_ptr())) == mf.MF_ERR_INVALID
    assert L.mf_apply_dvr_noalloc(*args(4, float("inf"), x.data_ptr(), y.data_ptr())) == mf.MF_ERR_INVALID
    assert L.mf_apply_dvr_noalloc(*args(4, float("nan"), x.data_ptr(), y.data_ptr())) == mf.MF_ERR_INVALID
