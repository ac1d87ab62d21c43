"""Python binding of libcompar — argument marshalling only.

Every function named ``compar_*`` here has the C signature of the same name
in ``include/compar.h`` and forwards to it through ctypes; nothing of the
GEMM, the selection or the cost models runs in Python.  :class:`Context`
adds a convenience layer that takes PyTorch tensors (device memory and
streams come from PyTorch) and raises :class:`ComparError` on a negative
status.

The shared library is built in-tree by :func:`build` (nvcc, sm_103a).  There
is no fallback: importing this package without ``libcompar.so`` raises.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcompar.so")

# dtypes / statuses / variant ids (values of include/compar.h)
F32, BF16, F8E4M3 = 0, 1, 2
OK, ERR_INVALID, ERR_UNSUPPORTED, ERR_CUDA, ERR_TIMEOUT, ERR_IO, ERR_NO_VARIANT = 0, -1, -2, -3, -4, -5, -6
V_NAIVE, V_SIMT, V_TC_TF32, V_TC_BF16, V_TC_FP8, V_SPLIT3 = 0, 1, 2, 3, 4, 5
V_GROUPED = 6      # batched calls only
V_SPLIT6 = 7
V_SPLIT3_TF32 = 8
V_SPLIT3_FUSED = 9
NUM_VARIANTS = 10  # ids 0 .. 9 (id 6 never runs a single call)
MLP_OUTPUTS = 2 * NUM_VARIANTS   # log2 time and log10 error per variant
VARIANT_NAMES = ["naive-f32", "simt-f32", "tc-tf32", "tc-bf16", "tc-fp8", "split-3xbf16",
                 "grouped", "split-6xbf16", "split-3xtf32", "split-3xbf16-fused"]


S_NAIVE, S_TILED, S_TMA = 0, 1, 2
NUM_STENCIL_VARIANTS = 3
STENCIL_NAMES = ["stencil-naive", "stencil-tiled", "stencil-tma"]


class compar_stencil_params_t(ctypes.Structure):
    _fields_ = [("c", ctypes.c_float), ("gx", ctypes.c_float), ("gy", ctypes.c_float),
                ("gz", ctypes.c_float), ("amb", ctypes.c_float)]


class ComparError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {compar_status_string(status)} ({status}) {compar_last_error()}")


class compar_problem_t(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("lda", ctypes.c_int64), ("ldb", ctypes.c_int64), ("ldc", ctypes.c_int64),
                ("dtype", ctypes.c_int), ("A", ctypes.c_void_p), ("B", ctypes.c_void_p),
                ("C", ctypes.c_void_p), ("alpha", ctypes.c_float), ("beta", ctypes.c_float),
                ("scale_a", ctypes.c_float), ("scale_b", ctypes.c_float)]


class compar_record_t(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("dtype", ctypes.c_int32), ("variant", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("tol", ctypes.c_float), ("time_ms", ctypes.c_float), ("rel_err", ctypes.c_float)]


_i = ctypes.c_int
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_vp = ctypes.c_void_p
_d = ctypes.c_double
_f = ctypes.c_float
_fp = ctypes.POINTER(ctypes.c_float)

# name -> (restype, argtypes)
SIGNATURES = {
    "compar_init": (_i, [ctypes.POINTER(_vp), _i]),
    "compar_terminate": (_i, [_vp]),
    "compar_status_string": (ctypes.c_char_p, [_i]),
    "compar_last_error": (ctypes.c_char_p, []),
    "compar_gemm": (_i, [_vp, _i64, _i64, _i64, _i, _d, _vp, _vp, _vp, _vp]),
    "compar_gemm_host": (_i, [_vp, _i64, _i64, _i64, _i, _d, _vp, _vp, _vp, _vp]),
    "compar_stencil": (_i, [_vp, _i64, _i64, _i, ctypes.POINTER(compar_stencil_params_t),
                            _vp, _vp, _vp, _vp]),
    "compar_stencil_force_variant": (_i, [_vp, _i]),
    "compar_stencil_last_variant": (_i, [_vp]),
    "compar_stencil_variant_name": (ctypes.c_char_p, [_i]),
    "compar_stencil_supported": (_i, [_vp, _i, _i64, _i64]),
    "compar_stencil_select": (_i, [_vp, _i64, _i64, _i]),
    "compar_stencil_measure": (_i, [_vp, _i, _i64, _i64, _i,
                                    ctypes.POINTER(compar_stencil_params_t), _vp, _vp, _vp,
                                    _i, _i, _vp, ctypes.POINTER(ctypes.c_float)]),
    "compar_gemm_batched": (_i, [_vp, _i, ctypes.POINTER(compar_problem_t), _d, _vp]),
    "compar_force_variant": (_i, [_vp, _i]),
    "compar_set_scalars": (_i, [_vp, _f, _f]),
    "compar_set_fp8_scales": (_i, [_vp, _f, _f]),
    "compar_set_selector_mode": (_i, [_vp, _i]),
    "compar_last_variant": (_i, [_vp]),
    "compar_variant_count": (_i, []),
    "compar_variant_name": (ctypes.c_char_p, [_i]),
    "compar_variant_supported": (_i, [_vp, _i, _i64, _i64, _i64, _i]),
    "compar_clear_decisions": (_i, [_vp]),
    "compar_selector_load": (_i, [_vp, ctypes.c_char_p]),
    "compar_selector_save": (_i, [_vp, ctypes.c_char_p]),
    "compar_measure": (_i, [_vp, _i, _i64, _i64, _i64, _i, _d, _vp, _vp, _vp, _i, _i, _vp, _fp]),
    "compar_record_enable": (_i, [_vp, _i]),
    "compar_record_count": (_i64, [_vp]),
    "compar_record_get": (_i64, [_vp, ctypes.POINTER(compar_record_t), _i64]),
    "compar_record_add": (_i, [_vp, ctypes.POINTER(compar_record_t), _i64]),
    "compar_record_clear": (_i, [_vp]),
    "compar_check_device_error": (_i, [_vp, _vp]),
    "compar_set_wait_budget": (_i, [_vp, _u64]),
    "compar_selftest_timeout": (_i, [_vp, _vp]),
    "compar_gemm_simt_noalloc": (_i, [_i64, _i64, _i64, _f, _vp, _vp, _f, _vp, _vp]),
    "compar_autotune_batched": (_i, [_vp, _i, ctypes.POINTER(compar_problem_t), _d, _vp, _fp,
                                     ctypes.POINTER(_i)]),
    "compar_set_batched_config": (_i, [_vp, _i]),
    "compar_tc_plan": (_i, [_i, _i64, _i64, _i64, _i, ctypes.POINTER(_i64)]),
    "compar_tc_pair_plan": (_i, [_i, _i64, _i64, _i64, _i, ctypes.POINTER(_i64)]),
    "compar_set_tc_pairs": (_i, [_vp, _i]),
    "compar_simt_plan": (_i, [_i64, _i64, _i64, _i, _i64, _i, ctypes.POINTER(_i64)]),
    "compar_mlp_param_count": (_i, []),
    "compar_mlp_forward": (_i, [_vp, _fp, _i, _fp, _i, _fp]),
    "compar_mlp_train_steps": (_i, [_vp, _fp, _fp, _fp, _i, _fp, _fp, _fp, _i,
                                    ctypes.POINTER(ctypes.c_int32), _i, _i, _f, _i, _fp, _fp]),
    "compar_selector_train": (_i, [_vp, _i, _i, _f, _u64, _fp]),
    "compar_selector_finetune": (_i, [_vp, _i, _i, _f, _u64, _fp]),
    "compar_set_online": (_i, [_vp, _d, _i64, _i]),
    "compar_online_stats": (_i, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                 ctypes.POINTER(_i64)]),
    "compar_predict": (_i, [_vp, _i64, _i64, _i64, _i, _d, _i, _fp, _fp, _fp]),
    "compar_residual_check": (_i, [_vp, _i64, _i64, _i64, _i, _vp, _vp, _vp, _f, _i, _u64,
                                   ctypes.POINTER(_d), _vp]),
    "compar_init_host": (_i, [ctypes.POINTER(_vp), _i]),
    "compar_select": (_i, [_vp, _i64, _i64, _i64, _i, _d, _i]),
    "compar_error_model_set": (_i, [_vp, _i, _i, _d, _d, _d]),
    "compar_error_model_get": (_i, [_vp, _i, _i, ctypes.POINTER(_d), ctypes.POINTER(_d),
                                    ctypes.POINTER(_d)]),
    "compar_error_model_set_margin": (_i, [_vp, _d]),
    "compar_error_model_predict": (_d, [_vp, _i, _i, _i64]),
    "compar_profile_enable": (_i, [_vp, _i]),
    "compar_profile_read": (_i, [_vp, _i, ctypes.POINTER(_d), ctypes.POINTER(_i64)]),
    "compar_profile_reset": (_i, [_vp]),
    "compar_launch_count": (_i64, []),
    "compar_peak_ffma": (_i, [_vp, _fp, _vp]),
}

_lib = None


def build_library(force=False, verbose=False):
    """Compile libcompar.so in-tree (nvcc, sm_103a) and load it."""
    import importlib
    importlib.import_module(__name__ + ".build").build(force=force, verbose=verbose)
    return load(reload=True)


def _missing(name):
    def call(*args, **kwargs):
        raise ImportError(f"{name}: libcompar.so is not built ({LIB_PATH}); run "
                          "paper_2311_03543_b300.build_library() first")
    return call


def load(reload=False):
    """Load libcompar.so and bind every C-ABI function; raises if it is missing."""
    global _lib
    if _lib is not None and not reload:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libcompar.so is not built ({LIB_PATH}); run "
                          "paper_2311_03543_b300.build_library() first")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
        globals()[name] = fn
    _lib = lib
    return lib


def exported_symbols():
    return sorted(SIGNATURES)


# Bind at import when the library is present; otherwise every compar_* call
# raises ImportError (there is no fallback implementation).
for _name in SIGNATURES:
    globals()[_name] = _missing(_name)
if os.path.exists(LIB_PATH):
    try:
        load()
    except AttributeError:
        # a stale build without some symbol: calls raise until it is rebuilt
        _lib = None
        for _name in SIGNATURES:
            globals()[_name] = _missing(_name)


def _status(rc, what):
    if rc < 0:
        raise ComparError(rc, what)
    return rc


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _f32p(a):
    return a.ctypes.data_as(_fp)


def torch_dtype_code(t):
    import torch
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.bfloat16:
        return BF16
    if t.dtype in (torch.uint8, torch.float8_e4m3fn):
        return F8E4M3
    raise TypeError(f"unsupported dtype {t.dtype}")


# The trained selector shipped with the package (MLP, history table, error
# models, stencil models), written by train_selector.
DEFAULT_SELECTOR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_default.bin")


class Context:
    """A libcompar context bound to one CUDA device (tensor-level API).

    `selector`: the selector file loaded at creation — by default the
    shipped trained selector for a device context (unless COMPAR_SELECTOR_FILE
    names one, which compar_init has loaded) and none for a host-only one;
    None starts from the untrained models (roofline prior only), as a context
    that trains its own selector must."""

    def __init__(self, device=0, host_only=False, num_sms=148, selector="default"):
        load()
        h = ctypes.c_void_p()
        if host_only:
            _status(compar_init_host(ctypes.byref(h), num_sms), "compar_init_host")
        else:
            _status(compar_init(ctypes.byref(h), device), "compar_init")
        self.handle = h
        self.device = None if host_only else device
        if selector == "default":
            selector = None if (host_only or os.environ.get("COMPAR_SELECTOR_FILE")) \
                else DEFAULT_SELECTOR
        if selector is not None:
            try:
                self.selector_load(selector)
            except BaseException:
                self.close()
                raise

    @classmethod
    def host(cls, num_sms=148):
        """A host-only context (no GPU): selection, models, records, files."""
        return cls(host_only=True, num_sms=num_sms)

    def select(self, m, n, k, dtype=F32, tol=0.0, batch=1):
        return _status(compar_select(self.handle, m, n, k, dtype, float(tol), batch), "select")

    def error_model(self, variant, dtype):
        c = [ctypes.c_double() for _ in range(3)]
        _status(compar_error_model_get(self.handle, variant, dtype, *[ctypes.byref(x) for x in c]),
                "error_model_get")
        return tuple(x.value for x in c)

    def set_error_model(self, variant, dtype, c0, c1, c2):
        return _status(compar_error_model_set(self.handle, variant, dtype, c0, c1, c2),
                       "error_model_set")

    def set_error_margin(self, margin):
        return _status(compar_error_model_set_margin(self.handle, margin), "error_model_margin")

    def predict_error(self, variant, dtype, k):
        return compar_error_model_predict(self.handle, variant, dtype, k)

    def close(self):
        if self.handle:
            compar_terminate(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- compute -----------------------------------------------------------
    def gemm(self, A, B, C, tol=0.0, stream=None, dtype=None):
        """C = alpha*A@B + beta*C on the context's scalars; A, B, C CUDA tensors."""
        m, k = A.shape
        k2, n = B.shape
        if k != k2 or tuple(C.shape) != (m, n):
            raise ValueError("shape mismatch")
        for t in (A, B, C):
            if not t.is_contiguous():
                raise ValueError("tensors must be contiguous")
        dt = torch_dtype_code(A) if dtype is None else dtype
        rc = compar_gemm(self.handle, m, n, k, dt, float(tol), A.data_ptr(), B.data_ptr(),
                         C.data_ptr(), _stream_handle(stream))
        return _status(rc, "compar_gemm")

    def gemm_host(self, A, B, C, tol=0.0, stream=None, dtype=None):
        """The same on host matrices: A, B, C CPU torch tensors or NumPy
        arrays (C float32), row-major contiguous; pinned tensors transfer
        asynchronously.  C is ready once `stream` passes the call."""
        def ptr(x):
            if hasattr(x, "data_ptr"):
                if x.is_cuda or not x.is_contiguous():
                    raise ValueError("host tensors must be CPU and contiguous")
                return x.data_ptr()
            if not x.flags["C_CONTIGUOUS"]:
                raise ValueError("arrays must be C-contiguous")
            return x.ctypes.data
        m, k = A.shape
        k2, n = B.shape
        if k != k2 or tuple(C.shape) != (m, n):
            raise ValueError("shape mismatch")
        if dtype is None:
            if hasattr(A, "data_ptr"):
                dtype = torch_dtype_code(A)
            else:   # NumPy: float32, bf16 bit patterns (uint16) or E4M3 codes (uint8)
                dtype = {"float32": F32, "uint16": BF16, "uint8": F8E4M3}[str(A.dtype)]
        rc = compar_gemm_host(self.handle, m, n, k, dtype, float(tol), ptr(A), ptr(B), ptr(C),
                              _stream_handle(stream))
        return _status(rc, "compar_gemm_host")

    # -- thermal stencil (second component) ---------------------------------
    @staticmethod
    def stencil_params(c, gx, gy, gz, amb):
        return compar_stencil_params_t(c, gx, gy, gz, amb)

    def stencil(self, T_in, P, T_out, iters, params, stream=None):
        """T_out = `iters` explicit heat steps from T_in (CUDA float32 grids)."""
        rows, cols = T_in.shape
        if tuple(P.shape) != (rows, cols) or tuple(T_out.shape) != (rows, cols):
            raise ValueError("shape mismatch")
        for t in (T_in, P, T_out):
            if not t.is_contiguous():
                raise ValueError("grids must be contiguous")
        return _status(compar_stencil(self.handle, rows, cols, int(iters), ctypes.byref(params),
                                      T_in.data_ptr(), P.data_ptr(), T_out.data_ptr(),
                                      _stream_handle(stream)), "compar_stencil")

    def stencil_force_variant(self, v):
        return _status(compar_stencil_force_variant(self.handle, -1 if v is None else v),
                       "stencil_force_variant")

    def stencil_last_variant(self):
        return compar_stencil_last_variant(self.handle)

    def stencil_supported(self, v, rows, cols):
        return _status(compar_stencil_supported(self.handle, v, rows, cols),
                       "stencil_supported") == 1

    def stencil_select(self, rows, cols, iters):
        return _status(compar_stencil_select(self.handle, rows, cols, int(iters)),
                       "stencil_select")

    def stencil_measure(self, v, T_in, P, T_out, iters, params, warmup=1, reps=3, stream=None):
        rows, cols = T_in.shape
        out = ctypes.c_float()
        _status(compar_stencil_measure(self.handle, v, rows, cols, int(iters),
                                       ctypes.byref(params), T_in.data_ptr(), P.data_ptr(),
                                       T_out.data_ptr(), warmup, reps, _stream_handle(stream),
                                       ctypes.byref(out)), "compar_stencil_measure")
        return out.value

    def gemm_ptr(self, m, n, k, dtype, tol, a_ptr, b_ptr, c_ptr, stream_handle):
        return compar_gemm(self.handle, m, n, k, dtype, float(tol), a_ptr, b_ptr, c_ptr,
                           stream_handle)

    @staticmethod
    def problem_array(problems):
        """problems: list of dicts with keys m n k lda ldb ldc dtype A B C [alpha beta scale_a scale_b]."""
        arr = (compar_problem_t * len(problems))()
        for i, p in enumerate(problems):
            arr[i] = compar_problem_t(p["m"], p["n"], p["k"], p["lda"], p["ldb"], p["ldc"],
                                      p["dtype"], p["A"], p["B"], p["C"], p.get("alpha", 1.0),
                                      p.get("beta", 0.0), p.get("scale_a", 1.0),
                                      p.get("scale_b", 1.0))
        return arr

    def gemm_batched(self, problems, tol=0.0, stream=None):
        arr = problems if isinstance(problems, ctypes.Array) else self.problem_array(problems)
        return _status(compar_gemm_batched(self.handle, len(arr), arr, float(tol),
                                           _stream_handle(stream)), "compar_gemm_batched")

    @staticmethod
    def tc_plan(variant, m, n, k, num_sms=148, pairs=None):
        """Launch plan of a tensor-core variant (no device needed): dict of
        num_kb, tiles, splits, kb_per_split, sk_tile0, sk_cpt, sk_q, sk_ctas,
        sk_chunk_kb.  With `pairs` (a count of CTA pairs), the plan of the
        CTA-pair kernel: 256 x 256 tiles, "CTAs" counting pairs."""
        out = (_i64 * 9)()
        if pairs is not None:
            _status(compar_tc_pair_plan(int(variant), int(m), int(n), int(k), int(pairs), out),
                    "tc_pair_plan")
        else:
            _status(compar_tc_plan(int(variant), int(m), int(n), int(k), int(num_sms), out),
                    "tc_plan")
        keys = ("num_kb", "tiles", "splits", "kb_per_split", "sk_tile0", "sk_cpt", "sk_q",
                "sk_ctas", "sk_chunk_kb")
        return dict(zip(keys, (int(x) for x in out)))

    @staticmethod
    def simt_plan(m, n, k, dtype=0, ldb=None, num_sms=148):
        """Launch plan of the SIMT variant (no device needed): dict of
        skinny, rows, cols, splits, k_per, cluster."""
        out = (_i64 * 6)()
        _status(compar_simt_plan(int(m), int(n), int(k), int(dtype),
                                 int(n if ldb is None else ldb), int(num_sms), out), "simt_plan")
        keys = ("skinny", "rows", "cols", "splits", "k_per", "cluster")
        return dict(zip(keys, (int(x) for x in out)))

    def set_batched_config(self, config):
        """Force batched configuration 0..4 (None: autotuned / default)."""
        return _status(compar_set_batched_config(self.handle, -1 if config is None else
                                                 int(config)), "set_batched_config")

    def autotune_batched(self, problems, tol=0.0, stream=None):
        """Returns (best configuration, [median ms of configurations 0..4])."""
        arr = problems if isinstance(problems, ctypes.Array) else self.problem_array(problems)
        times = (ctypes.c_float * 5)()
        best = ctypes.c_int()
        _status(compar_autotune_batched(self.handle, len(arr), arr, float(tol),
                                        _stream_handle(stream), times, ctypes.byref(best)),
                "compar_autotune_batched")
        return best.value, list(times)

    def measure(self, variant, A, B, C, tol=0.0, warmup=3, reps=10, stream=None, dtype=None):
        """Median time (ms) of one variant on this call, CUDA events on `stream`."""
        m, k = A.shape
        n = B.shape[1]
        dt = torch_dtype_code(A) if dtype is None else dtype
        out = ctypes.c_float()
        _status(compar_measure(self.handle, variant, m, n, k, dt, float(tol), A.data_ptr(),
                               B.data_ptr(), C.data_ptr(), warmup, reps, _stream_handle(stream),
                               ctypes.byref(out)), "compar_measure")
        return out.value

    # -- control -----------------------------------------------------------
    def force_variant(self, v):
        return _status(compar_force_variant(self.handle, -1 if v is None else v), "force_variant")

    def set_scalars(self, alpha, beta):
        return _status(compar_set_scalars(self.handle, alpha, beta), "set_scalars")

    def set_fp8_scales(self, sa, sb):
        return _status(compar_set_fp8_scales(self.handle, sa, sb), "set_fp8_scales")

    def set_selector_mode(self, mode):
        return _status(compar_set_selector_mode(self.handle, mode), "set_selector_mode")

    def last_variant(self):
        return compar_last_variant(self.handle)

    def supported(self, v, m, n, k, dtype):
        return _status(compar_variant_supported(self.handle, v, m, n, k, dtype), "supported") == 1

    def clear_decisions(self):
        return _status(compar_clear_decisions(self.handle), "clear_decisions")

    def selector_load(self, path):
        return _status(compar_selector_load(self.handle, os.fsencode(path)), "selector_load")

    def selector_save(self, path):
        return _status(compar_selector_save(self.handle, os.fsencode(path)), "selector_save")

    # -- records / errors ----------------------------------------------------
    def record_enable(self, on=True):
        return _status(compar_record_enable(self.handle, 1 if on else 0), "record_enable")

    def records(self):
        n = _status(compar_record_count(self.handle), "record_count")
        buf = (compar_record_t * max(n, 1))()
        got = _status(compar_record_get(self.handle, buf, n), "record_get")
        return [buf[i] for i in range(got)]

    def record_add(self, recs):
        arr = (compar_record_t * len(recs))(*recs)
        return _status(compar_record_add(self.handle, arr, len(recs)), "record_add")

    def record_clear(self):
        return _status(compar_record_clear(self.handle), "record_clear")

    def check_device_error(self, stream=None):
        return compar_check_device_error(self.handle, _stream_handle(stream))

    def set_wait_budget(self, ns):
        return _status(compar_set_wait_budget(self.handle, int(ns)), "set_wait_budget")

    def set_tc_pairs(self, mode):
        """Tensor-core variants on CTA pairs: -1 automatic, 0 never, 1 always."""
        return _status(compar_set_tc_pairs(self.handle, int(mode)), "set_tc_pairs")

    # -- learned cost model ----------------------------------------------------
    def mlp_forward(self, params, X):
        """params: float32 (members, P); X: float32 (rows, 8) ->
        (members, rows, 2 * NUM_VARIANTS)."""
        import numpy as np
        params = np.ascontiguousarray(params, dtype=np.float32)
        X = np.ascontiguousarray(X, dtype=np.float32)
        if params.ndim != 2 or params.shape[1] != compar_mlp_param_count():
            raise ValueError(f"params must be (members, {compar_mlp_param_count()})")
        if X.ndim != 2 or X.shape[1] != 8:
            raise ValueError("X must be (rows, 8)")
        members, rows = params.shape[0], X.shape[0]
        Y = np.zeros((members, rows, MLP_OUTPUTS), dtype=np.float32)
        _status(compar_mlp_forward(self.handle, _f32p(params), members, _f32p(X), rows, _f32p(Y)),
                "mlp_forward")
        return Y

    def mlp_train_steps(self, params, X, T, mask, batch_idx, lr=1e-3, step0=1, m=None, v=None,
                        grads_only=False):
        """Runs Adam steps on the GPU; returns (params, m, v, loss) or (grads, loss)."""
        import numpy as np
        params = np.array(params, dtype=np.float32, order="C", copy=True)
        members = params.shape[0]
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        mask = np.ascontiguousarray(mask, dtype=np.float32)
        idx = np.ascontiguousarray(batch_idx, dtype=np.int32)   # (members, steps, batch)
        rows = X.shape[0]
        if params.ndim != 2 or params.shape[1] != compar_mlp_param_count():
            raise ValueError(f"params must be (members, {compar_mlp_param_count()})")
        if X.ndim != 2 or X.shape[1] != 8:
            raise ValueError("X must be (rows, 8)")
        if T.shape != (rows, MLP_OUTPUTS) or mask.shape != (rows, MLP_OUTPUTS):
            raise ValueError(f"T and mask must be (rows, {MLP_OUTPUTS})")
        if idx.ndim != 3 or idx.shape[0] != members or (idx.size and
                                                         (idx.min() < 0 or idx.max() >= rows)):
            raise ValueError("batch_idx must be (members, steps, batch) row indices")
        steps, batch = idx.shape[1], idx.shape[2]
        loss = np.zeros((members, steps), dtype=np.float32)
        ip = idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        if grads_only:
            g = np.zeros_like(params)
            _status(compar_mlp_train_steps(self.handle, _f32p(params), None, None, members,
                                           _f32p(X), _f32p(T), _f32p(mask), X.shape[0], ip,
                                           steps, batch, lr, step0, _f32p(g), _f32p(loss)),
                    "mlp_train_steps")
            return g, loss
        m = np.zeros_like(params) if m is None else np.array(m, dtype=np.float32, copy=True)
        v = np.zeros_like(params) if v is None else np.array(v, dtype=np.float32, copy=True)
        _status(compar_mlp_train_steps(self.handle, _f32p(params), _f32p(m), _f32p(v), members,
                                       _f32p(X), _f32p(T), _f32p(mask), X.shape[0], ip, steps,
                                       batch, lr, step0, None, _f32p(loss)), "mlp_train_steps")
        return params, m, v, loss

    def selector_train(self, steps=20000, batch=128, lr=1e-3, seed=1):
        vl = ctypes.c_float()
        _status(compar_selector_train(self.handle, steps, batch, lr, seed, ctypes.byref(vl)),
                "selector_train")
        return vl.value

    def selector_finetune(self, steps=500, batch=128, lr=5e-4, seed=1):
        vl = ctypes.c_float()
        _status(compar_selector_finetune(self.handle, steps, batch, lr, seed, ctypes.byref(vl)),
                "selector_finetune")
        return vl.value

    def set_online(self, epsilon=0.05, retrain_every=0, finetune_steps=0):
        return _status(compar_set_online(self.handle, float(epsilon), int(retrain_every),
                                         int(finetune_steps)), "set_online")

    def online_stats(self):
        """(explored picks, fine-tunes run, fine-tunes discarded)."""
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _status(compar_online_stats(self.handle, ctypes.byref(a), ctypes.byref(b),
                                    ctypes.byref(c)), "online_stats")
        return a.value, b.value, c.value

    def predict(self, m, n, k, dtype=F32, tol=0.0, batch=1):
        """MLP prediction: (time_ms, rel_err, spread), one entry per variant id."""
        t = (ctypes.c_float * NUM_VARIANTS)()
        e = (ctypes.c_float * NUM_VARIANTS)()
        s = (ctypes.c_float * NUM_VARIANTS)()
        _status(compar_predict(self.handle, m, n, k, dtype, float(tol), batch, t, e, s), "predict")
        return list(t), list(e), list(s)

    def residual_check(self, A, B, C, alpha=1.0, nrows=16, seed=1, stream=None, dtype=None):
        m, k = A.shape
        n = B.shape[1]
        dt = torch_dtype_code(A) if dtype is None else dtype
        out = ctypes.c_double()
        _status(compar_residual_check(self.handle, m, n, k, dt, A.data_ptr(), B.data_ptr(),
                                      C.data_ptr(), alpha, nrows, seed, ctypes.byref(out),
                                      _stream_handle(stream)), "residual_check")
        return out.value

    # -- kernel profiling ------------------------------------------------------
    def profile_enable(self, on=True):
        return _status(compar_profile_enable(self.handle, 1 if on else 0), "profile_enable")

    def profile_read(self, variant):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _status(compar_profile_read(self.handle, variant, ctypes.byref(ms), ctypes.byref(n)),
                "profile_read")
        return ms.value, n.value

    def profile_reset(self):
        return _status(compar_profile_reset(self.handle), "profile_reset")

    def peak_ffma(self, stream=None):
        out = ctypes.c_float()
        _status(compar_peak_ffma(self.handle, ctypes.byref(out), _stream_handle(stream)),
                "peak_ffma")
        return out.value

    def selftest_timeout(self, stream=None):
        return _status(compar_selftest_timeout(self.handle, _stream_handle(stream)),
                       "selftest_timeout")
