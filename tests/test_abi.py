"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point declared in include/mf.h, and rejects bad arguments before
touching CUDA."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def _declared():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(mf_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def mf():
    import paper_2606_31598_gb300 as mf
    from paper_2606_31598_gb300 import _build
    _build.build()
    return mf


def test_header_declares_core_calls():
    names = _declared()
    for n in ("mf_plan_create", "mf_apply", "mf_cheb_propagate", "mf_plan_destroy", "mf_debug_entries"):
        assert n in names


def test_library_exports_every_declared_symbol(mf):
    lib = mf.lib()
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_options_default_and_status_strings(mf):
    o = mf.mf_options_default()
    assert o.precision == mf.MF_PREC_FP32 and o.lanczos_m == 40 and abs(o.cheb_tol - 1e-7) < 1e-20
    assert o.storage == mf.MF_STORE_AUTO and o.alpha_safety == pytest.approx(0.9)
    for s, name in [(0, "MF_OK"), (1, "MF_ERR_INVALID"), (5, "MF_ERR_TIMEOUT"), (6, "MF_WARN_DENSE_WORK")]:
        assert mf.status_string(s) == name


@pytest.mark.parametrize(
    "D,M,gen,block,prec",
    [(1, 1, 0, 0, 1), (100, 99, 0, 0, 1), (100, 100, 7, 0, 1), (1000, 1000, 0, 100, 1), (1000, 1000, 0, -128, 1),
     (1000, 1000, 1, 0, 9)],
)
def test_plan_create_rejects_bad_arguments_without_gpu(mf, D, M, gen, block, prec):
    h = ctypes.c_void_p()
    o = mf.mf_options_default(precision=prec)
    st = mf.lib().mf_plan_create(ctypes.byref(h), D, M, gen, 1, block, 0, ctypes.byref(o))
    assert st == mf.MF_ERR_INVALID
    assert not h.value


def test_null_handles_are_invalid(mf):
    L = mf.lib()
    assert L.mf_apply(None, None, None, 1) == mf.MF_ERR_INVALID
    assert L.mf_cheb_propagate(None, None, 1, 0.1, 0) == mf.MF_ERR_INVALID
    assert L.mf_plan_destroy(None) == mf.MF_OK
    assert L.mf_sync(None) == mf.MF_ERR_INVALID


def test_vector_arguments_are_checked_before_the_library(mf):
    """The binding hands the kernels bare device addresses, so it refuses
    what would make them read or write the wrong memory: host tensors, other
    element types, strided views and tensors too small for rows x nvec."""
    torch = pytest.importorskip("torch")
    from paper_2606_31598_gb300 import _vec
    assert _vec(1234, 10, "raw address") == 1234
    bad = [torch.zeros(8, dtype=torch.complex128),               # host memory
           torch.zeros(8, dtype=torch.complex64),                # element type
           torch.zeros((4, 4), dtype=torch.complex128).t(),      # strided view
           "not a tensor"]
    for t in bad:
        with pytest.raises(mf.MFError) as e:
            _vec(t, 4, "x")
        assert e.value.status == mf.MF_ERR_INVALID


def test_every_entry_point_rejects_null_handles_and_bad_arguments(mf):
    """Each call checks its arguments on the host before any CUDA call, so
    on a machine without a GPU every one of these returns MF_ERR_INVALID."""
    L = mf.lib()
    INV = mf.MF_ERR_INVALID
    d = ctypes.c_double()
    i32 = ctypes.c_int32()
    i64 = ctypes.c_int64()
    vp = ctypes.c_void_p()
    checks = {
        "mf_cheb_filter": L.mf_cheb_filter(None, None, 1, 0.1, 0, 1),
        "mf_cheb_terms": L.mf_cheb_terms(None, 0.1, ctypes.byref(i32)),
        "mf_cheb_filter_terms": L.mf_cheb_filter_terms(None, 0.1, ctypes.byref(i32)),
        "mf_spectral_bounds": L.mf_spectral_bounds(None, ctypes.byref(d), ctypes.byref(d)),
        "mf_plan_set_bounds": L.mf_plan_set_bounds(None, 0.0, 1.0),
        "mf_plan_describe": L.mf_plan_describe(None, None, 0),
        "mf_debug_entries": L.mf_debug_entries(None, 0, 0, 1, 1, None),
        "mf_plan_profile": L.mf_plan_profile(None, 1),
        "mf_plan_profile_read": L.mf_plan_profile_read(None, ctypes.byref(d), ctypes.byref(i64)),
        "mf_plan_trials": L.mf_plan_trials(None, None, 0, None),
        "mf_rows_cheb_begin": L.mf_rows_cheb_begin(None, 0.1, 0, ctypes.byref(i32)),
        "mf_rows_cheb_init": L.mf_rows_cheb_init(None, None, None, 1),
        "mf_rows_cheb_term": L.mf_rows_cheb_term(None, 1, None, None, None, None, 1),
        "mf_rows_cheb_final": L.mf_rows_cheb_final(None, None, None, 1, 0.1),
        "mf_batch_propagate": L.mf_batch_propagate(None, None, 0.1, 1, 0, None),
        "mf_batch_offsets": L.mf_batch_offsets(None, None),
        "mf_batch_plan": L.mf_batch_plan(None, 0, ctypes.byref(vp)),
        "mf_batch_info": L.mf_batch_info(None, None, None),
        "mf_batch_form": L.mf_batch_form(None, 0, ctypes.byref(i32)),
        "mf_batch_create (no problems)": L.mf_batch_create(ctypes.byref(vp), 0, None, None, None, 0, 0, None),
        "mf_mlp_param_count": L.mf_mlp_param_count(None, ctypes.byref(i64)),
        "mf_mlp_predict": L.mf_mlp_predict(None, None, 1, None),
        "mf_external_create (block 100)": L.mf_external_create(ctypes.byref(vp), 300, 100, None, 0, None),
        "mf_sysbath_create (d_S 0)": L.mf_sysbath_create(ctypes.byref(vp), 0, 100, 0, None, None, None, 0.1, None),
        "mf_apply_dvr_noalloc (D 1)": L.mf_apply_dvr_noalloc(1, 0.0, None, None, None),
        "mf_pipe_rates (NULL)": L.mf_pipe_rates(0, None, None, 8),
        "mf_pipe_rates (n 7)": L.mf_pipe_rates(0, None, (ctypes.c_double * 8)(), 7),
        "mf_pipe_rates (device -1)": L.mf_pipe_rates(-1, None, (ctypes.c_double * 8)(), 8),
    }
    bad = {k: v for k, v in checks.items() if v != INV}
    assert not bad, bad
    assert L.mf_batch_destroy(None) == mf.MF_OK


def test_plan_deserialize_rejects_malformed_records_without_gpu(mf):
    """A malformed or out-of-range plan record is refused before anything is
    allocated (no GPU needed)."""
    import ctypes
    L = mf.lib()
    good = (b"mf_plan v1\nD=4096\ngenerator=0\nseed=1\nprecision=1\nblock=512\nstorage=0\npairs_cached=0\n"
            b"dvr_L=0x1.4p+6\nnvec_hint=1\ncheb_tol=0x1.ad7f29abcaf48p-24\nlanczos_m=40\nbounds_pad=0x1.999999999999ap-5\n"
            b"alpha_safety=0x1.ccccccccccccdp-1\nf_cache=0x1.999999999999ap-1\ndense_work_limit=0x1.2309ce54p+43\n"
            b"hermitian_reuse=-1\nrow_begin=0\nrow_end=0\nspin_limit=0\nhave_bounds=0\nemin=0x0p+0\nemax=0x0p+0\n"
            b"planner=0\ns_model=0x0p+0\nt_measured=-0x1p+0\nnum_sms=152\n")
    bad = [b"", b"garbage", b"mf_plan v2\n" + good[11:], good.replace(b"D=4096", b"D=1"),
           good.replace(b"block=512", b"block=500"), good.replace(b"precision=1", b"precision=7"),
           good.replace(b"seed=1\n", b""), good.replace(b"cheb_tol=0x1.ad7f29abcaf48p-24", b"cheb_tol=x"),
           good.replace(b"storage=0", b"storage=5"), good.replace(b"row_end=0", b"row_end=100")]
    for rec in bad:
        h = ctypes.c_void_p()
        st = L.mf_plan_deserialize(ctypes.byref(h), rec, len(rec), None)
        assert st == mf.MF_ERR_INVALID, rec[:40]
        assert not h.value
    assert L.mf_plan_deserialize(None, good, len(good), None) == mf.MF_ERR_INVALID
    assert L.mf_plan_serialize(None, None, 0, None) == mf.MF_ERR_INVALID
