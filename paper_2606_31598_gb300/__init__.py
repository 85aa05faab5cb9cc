"""Python binding of libmf, the GB300 matrix-free block-procedural operator library.

Argument marshalling only: every function forwards to the C ABI of
``include/mf.h`` under the same name; every step of the computation runs in
the library's CUDA kernels.  Tensors are passed by device pointer; PyTorch is
used only for device memory and streams.  There is no fallback: if
``libmf.so`` has not been built (``python -c "import __graft_entry__ as g;
g.build()"``) every call raises.
"""
import ctypes
import json
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmf.so")

MF_OK = 0
MF_ERR_INVALID = 1
MF_ERR_OOM = 2
MF_ERR_CUDA = 3
MF_ERR_UNSUPPORTED = 4
MF_ERR_TIMEOUT = 5
MF_WARN_DENSE_WORK = 6

MF_GEN_PHILOX_GUE = 0
MF_GEN_SINC_DVR_HO = 1
MF_PREC_FP64 = 0
MF_PREC_FP32 = 1
MF_PREC_BF16X2 = 2
MF_STORE_AUTO = -1
MF_STORE_PROCEDURAL = 0
MF_STORE_PARTIAL = 1
MF_STORE_FULL = 2
MF_PLANNER_ANALYTIC = 0
MF_PLANNER_AUTOTUNE = 1
MF_PLANNER_LEARNED = 2
MF_PLANNER_HYBRID = 3
SIZE_MAX = (1 << 64) - 1


class MFError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__("%s%s" % (status_string(status), (": " + what) if what else ""))


class mf_options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("storage", ctypes.c_int32),
        ("planner_mode", ctypes.c_int32),
        ("nvec_hint", ctypes.c_int32),
        ("cheb_tol", ctypes.c_double),
        ("lanczos_m", ctypes.c_int32),
        ("bounds_pad", ctypes.c_double),
        ("dvr_L", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("alpha_safety", ctypes.c_double),
        ("f_cache", ctypes.c_double),
        ("autotune_k", ctypes.c_int32),
        ("autotune_warmup", ctypes.c_int32),
        ("autotune_repeats", ctypes.c_int32),
        ("dense_work_limit", ctypes.c_double),
        ("device", ctypes.c_int32),
        ("model", ctypes.c_void_p),
        ("hermitian_reuse", ctypes.c_int32),
        ("row_begin", ctypes.c_int64),
        ("row_end", ctypes.c_int64),
        ("spin_limit", ctypes.c_int32),
    ]


class mf_problem(ctypes.Structure):
    _fields_ = [("D_out", ctypes.c_int64), ("D_in", ctypes.c_int64), ("R", ctypes.c_int64),
                ("n_op", ctypes.c_int64), ("N_task", ctypes.c_int64), ("B_c", ctypes.c_double),
                ("M_free", ctypes.c_double), ("N_gpu", ctypes.c_int32)]


class mf_candidate(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int64), ("storage", ctypes.c_int32), ("pairs_cached", ctypes.c_int64),
                ("p_row", ctypes.c_int32), ("groups", ctypes.c_int32), ("r_arrays", ctypes.c_int32)]


class mf_device_model(ctypes.Structure):
    _fields_ = [("flops_per_s", ctypes.c_double), ("hbm_bytes_per_s", ctypes.c_double),
                ("gen_entries_per_s", ctypes.c_double)]


class mf_estimate(ctypes.Structure):
    _fields_ = [("n_blk", ctypes.c_int64), ("n_pair", ctypes.c_int64), ("pairs_cached", ctypes.c_int64),
                ("waves", ctypes.c_int64), ("M_block", ctypes.c_double), ("M_work", ctypes.c_double),
                ("M_op", ctypes.c_double), ("M_tot", ctypes.c_double), ("F_mv", ctypes.c_double),
                ("T_model", ctypes.c_double), ("S_model", ctypes.c_double), ("feasible", ctypes.c_int32),
                ("T_sum", ctypes.c_double)]


_lib = None


def lib():
    """Load libmf.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmf.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        P = ctypes.POINTER
        L.mf_options_default.argtypes = [P(mf_options)]
        L.mf_options_default.restype = None
        L.mf_status_string.argtypes = [ctypes.c_int]
        L.mf_status_string.restype = ctypes.c_char_p
        L.mf_plan_create.argtypes = [P(vp), i64, i64, i32, u64, i64, ctypes.c_size_t, P(mf_options)]
        L.mf_sysbath_create.argtypes = [P(vp), i64, i64, i32, vp, vp, vp, d, P(mf_options)]
        L.mf_external_create.argtypes = [P(vp), i64, i64, vp, ctypes.c_size_t, P(mf_options)]
        L.mf_selfcheck_generator.argtypes = [P(i64), P(i64)]
        L.mf_rows_cheb_begin.argtypes = [vp, d, i32, P(i32)]
        L.mf_rows_cheb_init.argtypes = [vp, vp, vp, i64]
        L.mf_rows_cheb_term.argtypes = [vp, i32, vp, vp, vp, vp, i64]
        L.mf_rows_cheb_final.argtypes = [vp, vp, vp, i64, d]
        for name in ("mf_rows_cheb_begin", "mf_rows_cheb_init", "mf_rows_cheb_term", "mf_rows_cheb_final"):
            getattr(L, name).restype = ctypes.c_int
        L.mf_selfcheck_generator.restype = ctypes.c_int
        L.mf_pipe_rates.argtypes = [i32, vp, P(d), i32]
        L.mf_pipe_rates.restype = ctypes.c_int
        L.mf_plan_destroy.argtypes = [vp]
        L.mf_apply.argtypes = [vp, vp, vp, i64]
        L.mf_cheb_propagate.argtypes = [vp, vp, i64, d, i32]
        L.mf_cheb_terms.argtypes = [vp, d, P(i32)]
        L.mf_cheb_filter.argtypes = [vp, vp, i64, d, i32, i32]
        L.mf_cheb_filter_terms.argtypes = [vp, d, P(i32)]
        L.mf_spectral_bounds.argtypes = [vp, P(d), P(d)]
        L.mf_plan_set_bounds.argtypes = [vp, d, d]
        L.mf_sync.argtypes = [vp]
        L.mf_plan_describe.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
        L.mf_debug_entries.argtypes = [vp, i64, i64, i64, i64, vp]
        L.mf_apply_dvr_noalloc.argtypes = [i64, d, vp, vp, vp]
        L.mf_plan_profile.argtypes = [vp, i32]
        L.mf_planner_estimate.argtypes = [P(mf_problem), P(mf_candidate), P(mf_device_model), d, d, P(mf_estimate)]
        L.mf_planner_device_model.argtypes = [i32, i32, i32, P(mf_device_model)]
        L.mf_planner_device_model.restype = ctypes.c_int
        L.mf_plan_trials.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t, P(ctypes.c_size_t)]
        L.mf_plan_serialize.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t, P(ctypes.c_size_t)]
        L.mf_plan_deserialize.argtypes = [P(vp), ctypes.c_char_p, ctypes.c_size_t, P(mf_options)]
        L.mf_plan_serialize.restype = ctypes.c_int
        L.mf_plan_deserialize.restype = ctypes.c_int
        fp = P(ctypes.c_float)
        L.mf_mlp_create.argtypes = [P(vp), i32, i32, i32, u64]
        L.mf_mlp_destroy.argtypes = [vp]
        L.mf_mlp_param_count.argtypes = [vp, P(i64)]
        L.mf_mlp_get_params.argtypes = [vp, vp, vp, vp]
        L.mf_mlp_set_params.argtypes = [vp, vp, vp, vp]
        L.mf_mlp_predict.argtypes = [vp, vp, i64, vp]
        L.mf_mlp_loss_grad.argtypes = [vp, vp, vp, vp, i64, vp, vp]
        L.mf_mlp_train.argtypes = [vp, vp, vp, vp, i64, i32, ctypes.c_float, i32, vp]
        L.mf_mlp_features.argtypes = [i32, i32, i64, i64, i64, d, vp]
        L.mf_batch_create.argtypes = [P(vp), i32, vp, vp, vp, i32, ctypes.c_size_t, P(mf_options)]
        L.mf_batch_destroy.argtypes = [vp]
        L.mf_batch_offsets.argtypes = [vp, vp]
        L.mf_batch_propagate.argtypes = [vp, vp, d, i32, i32, P(i32)]
        L.mf_batch_plan.argtypes = [vp, i32, P(vp)]
        L.mf_batch_info.argtypes = [vp, P(i32), P(i32)]
        L.mf_batch_form.argtypes = [vp, i32, P(i32)]
        for name in ("mf_batch_create", "mf_batch_destroy", "mf_batch_offsets", "mf_batch_propagate",
                     "mf_batch_plan", "mf_batch_info", "mf_batch_form"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("mf_planner_estimate", "mf_plan_trials", "mf_mlp_create", "mf_mlp_destroy", "mf_mlp_param_count",
                     "mf_mlp_get_params", "mf_mlp_set_params", "mf_mlp_predict", "mf_mlp_loss_grad", "mf_mlp_train",
                     "mf_mlp_features"):
            getattr(L, name).restype = ctypes.c_int
        L.mf_plan_profile_read.argtypes = [vp, P(d), P(i64)]
        for name in ("mf_plan_create", "mf_sysbath_create", "mf_external_create", "mf_plan_destroy", "mf_apply",
                     "mf_cheb_propagate",
                     "mf_cheb_terms",
                     "mf_cheb_filter", "mf_cheb_filter_terms", "mf_spectral_bounds", "mf_plan_set_bounds", "mf_sync", "mf_plan_describe",
                     "mf_debug_entries", "mf_plan_profile", "mf_plan_profile_read", "mf_apply_dvr_noalloc"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def status_string(s):
    try:
        return lib().mf_status_string(int(s)).decode()
    except Exception:  # library missing: still format the code
        return "mf_status(%d)" % int(s)


def _check(st, what=""):
    if st not in (MF_OK, MF_WARN_DENSE_WORK):
        raise MFError(st, what)
    return st


def _vec(t, n, what):
    """Device address of a vector argument: a contiguous complex128 CUDA
    tensor holding at least n elements (n = 0: size not checked).  An int is
    taken as a raw device address, unchecked.  Anything else raises
    MF_ERR_INVALID before the library sees it: the kernels read and write
    rows x nvec complex128 elements from the address they are given."""
    if isinstance(t, int):
        return t
    import torch
    ok = (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous()
          and t.numel() >= n)
    if not ok:
        got = ("%s %s on %s, %d elements" % (tuple(t.shape), t.dtype, t.device, t.numel())
               if isinstance(t, torch.Tensor) else type(t).__name__)
        raise MFError(MF_ERR_INVALID, "%s: expected a contiguous complex128 CUDA tensor of at least %d elements, "
                      "got %s" % (what, n, got))
    return t.data_ptr()


def mf_options_default(**overrides):
    o = mf_options()
    lib().mf_options_default(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def current_stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def mf_plan_create(D, M, generator, seed, block=0, cache_budget_bytes=0, options=None):
    h = ctypes.c_void_p()
    opt = options if options is not None else mf_options_default(stream=current_stream())
    st = lib().mf_plan_create(ctypes.byref(h), int(D), int(M), int(generator), int(seed) & (2 ** 64 - 1),
                              int(block), int(cache_budget_bytes), ctypes.byref(opt))
    _check(st, "mf_plan_create")
    return h


def mf_plan_destroy(plan):
    return _check(lib().mf_plan_destroy(plan), "mf_plan_destroy")


def mf_sysbath_create(d_S, d_B, seeds, H_S, A, g, options=None):
    import numpy as np
    seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
    H_S = np.ascontiguousarray(np.asarray(H_S, dtype=np.complex128).reshape(d_S, d_S))
    n_int = len(seeds) - 1
    A = np.ascontiguousarray(np.asarray(A, dtype=np.complex128).reshape(n_int, d_S, d_S)) if n_int else None
    h = ctypes.c_void_p()
    opt = options if options is not None else mf_options_default(stream=current_stream())
    st = lib().mf_sysbath_create(ctypes.byref(h), int(d_S), int(d_B), int(n_int), seeds.ctypes.data,
                                 H_S.ctypes.data, None if A is None else A.ctypes.data, float(g), ctypes.byref(opt))
    _check(st, "mf_sysbath_create")
    return h


def mf_external_create(D, block, blocks, cache_budget_bytes=0, options=None):
    """blocks: a numpy array of the canonical blocks (kept referenced by the
    returned Plan; it must not change while the plan exists)."""
    h = ctypes.c_void_p()
    opt = options if options is not None else mf_options_default(stream=current_stream())
    st = lib().mf_external_create(ctypes.byref(h), int(D), int(block), ctypes.c_void_p(blocks.ctypes.data),
                                  int(cache_budget_bytes), ctypes.byref(opt))
    _check(st, "mf_external_create")
    return h


def mf_selfcheck_generator():
    """(division mismatches, square-root mismatches) of the generator's FP32
    arithmetic against IEEE on the current device (both 0 when exact)."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().mf_selfcheck_generator(ctypes.byref(a), ctypes.byref(b)), "mf_selfcheck_generator")
    return a.value, b.value


PIPES = ("imad_hi", "imad", "lop3", "iadd3", "ffma", "mufu", "i2f", "dfma", "mma128", "mma256")


def mf_pipe_rates(device=0, stream=None):
    """Measured operations per second of each generator pipe on `device`,
    and tcgen05 MMA instructions per second (M = 128, K = 16; N = 128 and
    N = 256) over the GPU (dict keyed by PIPES)."""
    out = (ctypes.c_double * len(PIPES))()
    st = stream if stream is not None else current_stream()
    _check(lib().mf_pipe_rates(int(device), ctypes.c_void_p(st), out, len(PIPES)), "mf_pipe_rates")
    return dict(zip(PIPES, list(out)))


def mf_apply(plan, y, x, nvec=1):
    return _check(lib().mf_apply(plan, _vec(y, 0, "mf_apply y"), _vec(x, 0, "mf_apply x"), int(nvec)), "mf_apply")


def mf_cheb_propagate(plan, psi, nvec, dt, order=0):
    return _check(lib().mf_cheb_propagate(plan, _vec(psi, 0, "mf_cheb_propagate psi"), int(nvec), float(dt),
                                          int(order)),
                  "mf_cheb_propagate")


def mf_cheb_terms(plan, dt):
    n = ctypes.c_int32()
    _check(lib().mf_cheb_terms(plan, float(dt), ctypes.byref(n)), "mf_cheb_terms")
    return n.value


def mf_cheb_filter(plan, psi, nvec, tau, order=0, normalize=True):
    return _check(lib().mf_cheb_filter(plan, _vec(psi, 0, "mf_cheb_filter psi"), int(nvec), float(tau), int(order),
                                       int(bool(normalize))),
                  "mf_cheb_filter")


def mf_cheb_filter_terms(plan, tau):
    n = ctypes.c_int32()
    _check(lib().mf_cheb_filter_terms(plan, float(tau), ctypes.byref(n)), "mf_cheb_filter_terms")
    return n.value


def mf_spectral_bounds(plan):
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(lib().mf_spectral_bounds(plan, ctypes.byref(lo), ctypes.byref(hi)), "mf_spectral_bounds")
    return lo.value, hi.value


def mf_plan_set_bounds(plan, emin, emax):
    return _check(lib().mf_plan_set_bounds(plan, float(emin), float(emax)), "mf_plan_set_bounds")


def mf_sync(plan):
    return _check(lib().mf_sync(plan), "mf_sync")


def mf_plan_describe(plan):
    buf = ctypes.create_string_buffer(4096)
    _check(lib().mf_plan_describe(plan, buf, len(buf)), "mf_plan_describe")
    return json.loads(buf.value.decode())


def mf_debug_entries(plan, r0, c0, rows, cols, out_host):
    """out_host: a contiguous numpy array (complex64 or complex128 per plan)."""
    return _check(lib().mf_debug_entries(plan, int(r0), int(c0), int(rows), int(cols),
                                         out_host.ctypes.data), "mf_debug_entries")


def mf_apply_dvr_noalloc(D, dvr_L, x, y, stream=None):
    """Allocation-free DVR apply (FP32 form, one vector); see include/mf.h."""
    return _check(lib().mf_apply_dvr_noalloc(int(D), float(dvr_L), _vec(x, int(D), "mf_apply_dvr_noalloc x"),
                                             _vec(y, int(D), "mf_apply_dvr_noalloc y"), stream),
                  "mf_apply_dvr_noalloc")


def mf_planner_estimate(problem, candidate, model=None, alpha=0.9, cache_budget_bytes=0.0):
    """Algorithm 1 quantities of one candidate (host only)."""
    out = mf_estimate()
    _check(lib().mf_planner_estimate(ctypes.byref(problem), ctypes.byref(candidate),
                                     ctypes.byref(model) if model is not None else None, float(alpha),
                                     float(cache_budget_bytes), ctypes.byref(out)), "mf_planner_estimate")
    return out


def mf_planner_device_model(precision, generator, num_sms=152):
    """The runtime-model throughputs the analytic planner uses (host only)."""
    out = mf_device_model()
    _check(lib().mf_planner_device_model(int(precision), int(generator), int(num_sms), ctypes.byref(out)),
           "mf_planner_device_model")
    return out


def mf_plan_trials(plan):
    """The plan-trial log as a list of dicts (one per candidate)."""
    need = ctypes.c_size_t()
    _check(lib().mf_plan_trials(plan, None, 0, ctypes.byref(need)), "mf_plan_trials")
    buf = ctypes.create_string_buffer(max(1, need.value))
    _check(lib().mf_plan_trials(plan, buf, len(buf), None), "mf_plan_trials")
    return [json.loads(l) for l in buf.value.decode().splitlines() if l.strip()]


def mf_plan_serialize(plan):
    """The plan record (bytes, without the NUL) for a later mf_plan_deserialize."""
    need = ctypes.c_size_t()
    _check(lib().mf_plan_serialize(plan, None, 0, ctypes.byref(need)), "mf_plan_serialize")
    buf = ctypes.create_string_buffer(max(1, need.value))
    _check(lib().mf_plan_serialize(plan, buf, len(buf), None), "mf_plan_serialize")
    return buf.value


def mf_plan_deserialize(record, options=None):
    h = ctypes.c_void_p()
    opt = options if options is not None else mf_options_default(stream=current_stream())
    rec = bytes(record)
    _check(lib().mf_plan_deserialize(ctypes.byref(h), rec, len(rec), ctypes.byref(opt)), "mf_plan_deserialize")
    return h


def _fptr(a):
    return None if a is None else a.ctypes.data


class MLP:
    """The learned planner's surrogate network (host arrays in, host arrays out)."""

    def __init__(self, n_in=10, n_hidden=64, n_out=3, seed=0):
        import numpy as np
        self._np = np
        self.handle = ctypes.c_void_p()
        _check(lib().mf_mlp_create(ctypes.byref(self.handle), n_in, n_hidden, n_out, seed), "mf_mlp_create")
        self.n_in, self.n_hidden, self.n_out = n_in, n_hidden, n_out
        n = ctypes.c_int64()
        _check(lib().mf_mlp_param_count(self.handle, ctypes.byref(n)), "mf_mlp_param_count")
        self.n_params = n.value

    def _f32(self, a, shape=None):
        a = self._np.ascontiguousarray(a, dtype=self._np.float32)
        return a if shape is None else a.reshape(shape)

    def params(self):
        np = self._np
        p = np.zeros(self.n_params, np.float32)
        mu = np.zeros(self.n_in, np.float32)
        sd = np.zeros(self.n_in, np.float32)
        _check(lib().mf_mlp_get_params(self.handle, p.ctypes.data, mu.ctypes.data, sd.ctypes.data), "get_params")
        return p, mu, sd

    def set_params(self, params=None, mu=None, sd=None):
        a = [None if v is None else self._f32(v) for v in (params, mu, sd)]
        _check(lib().mf_mlp_set_params(self.handle, *[_fptr(v) for v in a]), "set_params")

    def predict(self, X):
        X = self._f32(X, (-1, self.n_in))
        Y = self._np.zeros((X.shape[0], self.n_out), self._np.float32)
        _check(lib().mf_mlp_predict(self.handle, X.ctypes.data, X.shape[0], Y.ctypes.data), "predict")
        return Y

    def loss_grad(self, X, Y, mask=None):
        X = self._f32(X, (-1, self.n_in))
        Y = self._f32(Y, (-1, self.n_out))
        M = None if mask is None else self._f32(mask, (-1, self.n_out))
        loss = self._np.zeros(1, self._np.float32)
        g = self._np.zeros(self.n_params, self._np.float32)
        _check(lib().mf_mlp_loss_grad(self.handle, X.ctypes.data, Y.ctypes.data, _fptr(M), X.shape[0],
                                      loss.ctypes.data, g.ctypes.data), "loss_grad")
        return float(loss[0]), g

    def train(self, X, Y, mask=None, epochs=1000, lr=1e-3, set_normalization=True):
        X = self._f32(X, (-1, self.n_in))
        Y = self._f32(Y, (-1, self.n_out))
        M = None if mask is None else self._f32(mask, (-1, self.n_out))
        curve = self._np.zeros(max(1, epochs), self._np.float32)
        _check(lib().mf_mlp_train(self.handle, X.ctypes.data, Y.ctypes.data, _fptr(M), X.shape[0], int(epochs),
                                  float(lr), int(bool(set_normalization)), curve.ctypes.data), "train")
        return curve[:epochs]

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().mf_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mf_mlp_features(generator, precision, D, block, nvec, cache_budget_bytes):
    import numpy as np
    out = np.zeros(10, np.float32)
    _check(lib().mf_mlp_features(int(generator), int(precision), int(D), int(block), int(nvec),
                                 float(cache_budget_bytes), out.ctypes.data), "mf_mlp_features")
    return out


class Batch:
    """Batched independent problems sharing one persistent launch per term."""

    def __init__(self, Ds, nvecs, seeds, generator, cache_budget_bytes=0, **opts):
        import numpy as np
        self._np = np
        o = mf_options_default()
        if "stream" not in opts:
            opts["stream"] = current_stream()
        for k, v in opts.items():
            setattr(o, k, v)
        self.options = o
        self.Ds = np.ascontiguousarray(Ds, dtype=np.int64)
        self.nvecs = np.ascontiguousarray(nvecs, dtype=np.int32)
        sd = np.ascontiguousarray(seeds, dtype=np.uint64)
        self.handle = ctypes.c_void_p()
        _check(lib().mf_batch_create(ctypes.byref(self.handle), len(self.Ds), self.Ds.ctypes.data,
                                     self.nvecs.ctypes.data, sd.ctypes.data, int(generator), int(cache_budget_bytes),
                                     ctypes.byref(o)), "mf_batch_create")
        self.offsets = np.zeros(len(self.Ds) + 1, dtype=np.int64)
        _check(lib().mf_batch_offsets(self.handle, self.offsets.ctypes.data), "mf_batch_offsets")

    def propagate(self, psi, dt, nsteps=1, order=0):
        nt = ctypes.c_int32()
        psi_p = _vec(psi, int(self.offsets[-1]), "Batch.propagate psi")
        _check(lib().mf_batch_propagate(self.handle, psi_p, float(dt), int(nsteps), int(order), ctypes.byref(nt)),
               "mf_batch_propagate")
        return nt.value

    def plan(self, i):
        h = ctypes.c_void_p()
        _check(lib().mf_batch_plan(self.handle, int(i), ctypes.byref(h)), "mf_batch_plan")
        return h

    def hermitian(self, i):
        """True when problem i takes the Hermitian-reuse form of the batched product."""
        h = ctypes.c_int32()
        _check(lib().mf_batch_form(self.handle, int(i), ctypes.byref(h)), "mf_batch_form")
        return bool(h.value)

    def info(self):
        a, b = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().mf_batch_info(self.handle, ctypes.byref(a), ctypes.byref(b)), "mf_batch_info")
        return a.value, b.value

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().mf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mf_plan_profile(plan, enable):
    return _check(lib().mf_plan_profile(plan, int(enable)), "mf_plan_profile")


def mf_plan_profile_read(plan):
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(lib().mf_plan_profile_read(plan, ctypes.byref(ms), ctypes.byref(n)), "mf_plan_profile_read")
    return ms.value, n.value


class Plan:
    """Owning handle with the calls as methods (destroyed on close/GC)."""

    def __init__(self, D, generator, seed=1, block=0, cache_budget_bytes=0, M=None, **opts):
        o = mf_options_default()
        if "stream" not in opts:
            opts["stream"] = current_stream()
        for k, v in opts.items():
            if k == "model" and hasattr(v, "handle"):
                v = v.handle.value
            setattr(o, k, v)
        self.options = o
        self.D = int(D)
        self.row_begin = int(o.row_begin)
        self.row_end = int(o.row_end) if o.row_end else int(D)
        self.handle = mf_plan_create(D, D if M is None else M, generator, seed, block, cache_budget_bytes, o)

    @classmethod
    def external(cls, D, block, blocks, cache_budget_bytes=0, **opts):
        """Externally stored canonical blocks (mf_external_create); blocks is a
        C-contiguous numpy array (complex64 for FP32/BF16X2, complex128 for
        FP64) that the plan keeps referenced."""
        import numpy as np
        self = cls.__new__(cls)
        o = mf_options_default()
        if "stream" not in opts:
            opts["stream"] = current_stream()
        for k, v in opts.items():
            setattr(o, k, v)
        want = np.complex128 if o.precision == MF_PREC_FP64 else np.complex64
        if blocks.dtype != want or not blocks.flags["C_CONTIGUOUS"]:
            raise MFError(MF_ERR_INVALID, "mf_external_create: blocks must be C-contiguous %s" % np.dtype(want).name)
        self.options = o
        self.D = int(D)
        self._blocks = blocks
        self.handle = mf_external_create(D, block, blocks, cache_budget_bytes, o)
        return self

    @classmethod
    def deserialize(cls, record, **opts):
        """A plan rebuilt from mf_plan_serialize's record (no planning);
        opts may set the stream and device."""
        self = cls.__new__(cls)
        o = mf_options_default()
        if "stream" not in opts:
            opts["stream"] = current_stream()
        for k, v in opts.items():
            setattr(o, k, v)
        self.handle = mf_plan_deserialize(record, o)
        d = mf_plan_describe(self.handle)
        self.options = o
        self.options.precision = {"fp64": MF_PREC_FP64, "fp32": MF_PREC_FP32, "bf16x2": MF_PREC_BF16X2}[d["precision"]]
        self.D = int(d["D"])
        fields = dict(l.split(b"=", 1) for l in bytes(record).splitlines()[1:] if b"=" in l)
        self.row_begin = int(fields.get(b"row_begin", b"0"))
        re_ = int(fields.get(b"row_end", b"0"))
        self.row_end = re_ if re_ else self.D
        return self

    def serialize(self):
        return mf_plan_serialize(self.handle)

    @classmethod
    def sysbath(cls, d_S, d_B, seeds, H_S, A, g, **opts):
        """System-bath plan (mf_sysbath_create): vectors [d_B][d_S], nvec = d_S."""
        self = cls.__new__(cls)
        o = mf_options_default()
        if "stream" not in opts:
            opts["stream"] = current_stream()
        for k, v in opts.items():
            setattr(o, k, v)
        self.options = o
        self.D = int(d_B)
        self.d_S = int(d_S)
        self.handle = mf_sysbath_create(d_S, d_B, seeds, H_S, A, g, o)
        return self

    def _rows(self):
        """Output rows of this plan: its row slice, else all D rows."""
        return getattr(self, "row_end", self.D) - getattr(self, "row_begin", 0)

    def apply(self, y, x, nvec=1):
        n = max(0, int(nvec))
        _vec(x, self.D * n, "Plan.apply x")
        _vec(y, self._rows() * n, "Plan.apply y")
        return mf_apply(self.handle, y, x, nvec)

    def cheb_propagate(self, psi, nvec, dt, order=0):
        _vec(psi, self.D * max(0, int(nvec)), "Plan.cheb_propagate psi")
        return mf_cheb_propagate(self.handle, psi, nvec, dt, order)

    def cheb_terms(self, dt):
        return mf_cheb_terms(self.handle, dt)

    # row-distributed propagation (plan created with row_begin / row_end)
    def rows_cheb_begin(self, dt, order=0):
        n = ctypes.c_int32()
        _check(lib().mf_rows_cheb_begin(self.handle, float(dt), int(order), ctypes.byref(n)), "mf_rows_cheb_begin")
        return n.value

    def rows_cheb_init(self, psi_full, acc, nvec):
        n = max(0, int(nvec))
        _check(lib().mf_rows_cheb_init(self.handle, _vec(psi_full, self.D * n, "rows_cheb_init psi_full"),
                                       _vec(acc, self._rows() * n, "rows_cheb_init acc"), int(nvec)),
               "mf_rows_cheb_init")

    def rows_cheb_term(self, j, q_full, q_prev, q_next, acc, nvec):
        n = max(0, int(nvec))
        rn = self._rows() * n
        _check(lib().mf_rows_cheb_term(self.handle, int(j), _vec(q_full, self.D * n, "rows_cheb_term q_full"),
                                       _vec(q_prev, rn, "rows_cheb_term q_prev"),
                                       _vec(q_next, rn, "rows_cheb_term q_next"), _vec(acc, rn, "rows_cheb_term acc"),
                                       int(nvec)), "mf_rows_cheb_term")

    def rows_cheb_final(self, acc, psi_slice, nvec, dt):
        rn = self._rows() * max(0, int(nvec))
        _check(lib().mf_rows_cheb_final(self.handle, _vec(acc, rn, "rows_cheb_final acc"),
                                        _vec(psi_slice, rn, "rows_cheb_final psi_slice"), int(nvec), float(dt)),
               "mf_rows_cheb_final")

    def cheb_filter(self, psi, nvec, tau, order=0, normalize=True):
        _vec(psi, self.D * max(0, int(nvec)), "Plan.cheb_filter psi")
        return mf_cheb_filter(self.handle, psi, nvec, tau, order, normalize)

    def cheb_filter_terms(self, tau):
        return mf_cheb_filter_terms(self.handle, tau)

    def bounds(self):
        return mf_spectral_bounds(self.handle)

    def set_bounds(self, emin, emax):
        return mf_plan_set_bounds(self.handle, emin, emax)

    def describe(self):
        return mf_plan_describe(self.handle)

    def trials(self):
        return mf_plan_trials(self.handle)

    def entries(self, r0, c0, rows, cols):
        import numpy as np
        dt = np.complex128 if self.options.precision == MF_PREC_FP64 else np.complex64
        out = np.zeros((rows, cols), dtype=dt)
        mf_debug_entries(self.handle, r0, c0, rows, cols, out)
        return out

    def sync(self):
        return mf_sync(self.handle)

    def profile(self, enable=True):
        return mf_plan_profile(self.handle, enable)

    def profile_read(self):
        return mf_plan_profile_read(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None:
            mf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
