"""ctypes binding of libglm (include/glm.h).

Argument marshalling only: every step of SGD / CA-SGD runs in the CUDA
kernels of libglm.so.  Functions keep the C names (``glm_create``,
``glm_ca_sgd_run`` ...); ``Dataset`` is a thin convenience wrapper that owns a
handle and accepts torch tensors (device memory and streams come from
PyTorch) or numpy arrays (host memory).

Importing this module does not load the library; the first call does, and
raises ``ImportError`` if libglm.so has not been built -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
# GLM_LIBRARY names another build of the same ABI (the bounds-checked
# _build/libglm_checked.so); default: the package's libglm.so
LIB_PATH = os.environ.get("GLM_LIBRARY") or os.path.join(_PKG, "_build", "libglm.so")
CHECKED_LIB_PATH = os.path.join(_PKG, "_build", "libglm_checked.so")

# status codes
(GLM_OK, GLM_EINVAL, GLM_ENOMEM, GLM_ECUDA, GLM_ENONFINITE, GLM_ETIMEOUT, GLM_EUNSUPPORTED,
 GLM_EBOUNDS) = range(8)
STATUS_NAMES = {0: "GLM_OK", 1: "GLM_EINVAL", 2: "GLM_ENOMEM", 3: "GLM_ECUDA",
                4: "GLM_ENONFINITE", 5: "GLM_ETIMEOUT", 6: "GLM_EUNSUPPORTED",
                7: "GLM_EBOUNDS"}
# losses
GLM_LOGISTIC, GLM_LSQ, GLM_POISSON = 0, 1, 2
# element types
GLM_F32, GLM_BF16, GLM_F16, GLM_TF32, GLM_E4M3, GLM_F64 = range(6)
DTYPES = {"f32": GLM_F32, "bf16": GLM_BF16, "f16": GLM_F16, "tf32": GLM_TF32,
          "e4m3": GLM_E4M3, "f64": GLM_F64}

# every symbol include/glm.h declares (checked by the CPU test-suite)
EXPORTED = [
    "glm_last_error", "glm_version", "glm_checked_build", "glm_create_opts_default",
    "glm_create",
    "glm_create_ex", "glm_destroy", "glm_shape", "glm_stream", "glm_sync",
    "glm_ca_opts_default", "glm_sgd_run", "glm_sgd_run_ex", "glm_sgd_lowp_run", "glm_ca_sgd_run",
    "glm_ca_sgd_run_ex", "glm_ca_plan", "glm_kernel_times", "glm_loss",
    "glm_sample_indices", "glm_sample_indices_noalloc", "glm_gram_lower",
    "glm_storage_layout", "glm_storage_read", "glm_debug_fail_alloc",
    "glm_slab_reduce_floats", "glm_slab_partial", "glm_slab_finish", "glm_sum_buffers",
    "glm_batch_opts_default", "glm_batch_create", "glm_batch_run", "glm_batch_loss",
    "glm_batch_choice", "glm_batch_choice_kernel", "glm_tau_prior", "glm_batch_destroy",
]


class GlmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class glm_create_opts(ctypes.Structure):
    _fields_ = [("input_dtype", ctypes.c_int), ("input_on_host", ctypes.c_int),
                ("column_scales", ctypes.c_int), ("fp8_copy", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


class glm_ca_opts(ctypes.Structure):
    _fields_ = [("gram_dtype", ctypes.c_int), ("gemv_dtype", ctypes.c_int),
                ("recurrence_f64", ctypes.c_int), ("kahan", ctypes.c_int),
                ("first_iter", ctypes.c_int64), ("problem", ctypes.c_uint32),
                ("use_graph", ctypes.c_int), ("cluster", ctypes.c_int),
                ("chunk_outer", ctypes.c_int64), ("gram_impl", ctypes.c_int),
                ("timing", ctypes.c_int), ("accumulate", ctypes.c_int),
                ("state_dtype", ctypes.c_int), ("chain_impl", ctypes.c_int),
                ("wait_probe_cycles", ctypes.c_int64)]


class glm_run_plan(ctypes.Structure):
    _fields_ = [("chunk_outer", ctypes.c_int64), ("chunks", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("cluster", ctypes.c_int),
                ("gram_impl", ctypes.c_int), ("gram_dtype", ctypes.c_int),
                ("gemv_dtype", ctypes.c_int), ("recurrence_f64", ctypes.c_int),
                ("chain_impl", ctypes.c_int)]


class glm_problem_desc(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("loss", ctypes.c_int),
                ("lambda_", ctypes.c_float), ("eta", ctypes.c_float),
                ("iters", ctypes.c_int64), ("seed", ctypes.c_uint64), ("s", ctypes.c_int),
                ("b", ctypes.c_int64), ("gram_dtype", ctypes.c_int)]


class glm_batch_opts(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("input_dtype", ctypes.c_int),
                ("input_on_host", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("wait_probe_cycles", ctypes.c_int64), ("tau_bound", ctypes.c_double)]


_lib = None
_lock = threading.Lock()


def load():
    """Load libglm.so (ImportError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libglm.so not built ({LIB_PATH}); run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i64, u64, i32, f32 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64,
                                  ctypes.c_int, ctypes.c_float)
        sig = {
            "glm_last_error": ([], ctypes.c_char_p),
            "glm_version": ([], ctypes.c_char_p),
            "glm_checked_build": ([], i32),
            "glm_create_opts_default": ([ctypes.POINTER(glm_create_opts)], None),
            "glm_create": ([vp, vp, i64, i64, i32, i32, ctypes.POINTER(vp)], i32),
            "glm_create_ex": ([vp, vp, i64, i64, i32, i32, ctypes.POINTER(glm_create_opts),
                               ctypes.POINTER(vp)], i32),
            "glm_destroy": ([vp], i32),
            "glm_shape": ([vp, ctypes.POINTER(i64), ctypes.POINTER(i64)], i32),
            "glm_stream": ([vp], vp),
            "glm_sync": ([vp], i32),
            "glm_ca_opts_default": ([ctypes.POINTER(glm_ca_opts)], None),
            "glm_sgd_run": ([vp, i64, f32, f32, i64, u64, vp], i32),
            "glm_sgd_run_ex": ([vp, i64, f32, f32, i64, u64, vp,
                                ctypes.POINTER(glm_ca_opts)], i32),
            "glm_sgd_lowp_run": ([vp, i64, f32, f32, i64, u64, vp, i32, i64], i32),
            "glm_ca_sgd_run": ([vp, i32, i64, f32, f32, i64, u64, vp], i32),
            "glm_ca_sgd_run_ex": ([vp, i32, i64, f32, f32, i64, u64, vp,
                                   ctypes.POINTER(glm_ca_opts)], i32),
            "glm_ca_plan": ([vp, i32, i64, f32, f32, i64, ctypes.POINTER(glm_ca_opts),
                             ctypes.POINTER(glm_run_plan)], i32),
            "glm_kernel_times": ([vp, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(i64)], i32),
            "glm_loss": ([vp, vp, f32, ctypes.POINTER(ctypes.c_double)], i32),
            "glm_sample_indices": ([u64, ctypes.c_uint32, i64, i64, i64, vp], i32),
            "glm_sample_indices_noalloc": ([u64, ctypes.c_uint32, i64, i64, i64, vp], i32),
            "glm_gram_lower": ([vp, i32, i64, i32, i64, i64, i64, vp, vp, i32, vp], i32),
            "glm_storage_layout": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i64),
                                    ctypes.POINTER(i64)], i32),
            "glm_storage_read": ([vp, i64, i64, vp, vp, vp, vp], i32),
            "glm_debug_fail_alloc": ([i64], None),
            "glm_slab_reduce_floats": ([i32, i64, ctypes.POINTER(i64)], i32),
            "glm_slab_partial": ([vp, i32, i64, i32, u64, i64, vp, vp,
                                  ctypes.POINTER(glm_ca_opts)], i32),
            "glm_slab_finish": ([vp, i32, i64, i32, f32, f32, vp, vp,
                                 ctypes.POINTER(glm_ca_opts)], i32),
            "glm_sum_buffers": ([vp, ctypes.POINTER(vp), i32, i64, vp], i32),
            "glm_batch_opts_default": ([ctypes.POINTER(glm_batch_opts)], None),
            "glm_batch_create": ([i32, ctypes.POINTER(glm_problem_desc),
                                  ctypes.POINTER(glm_batch_opts), ctypes.POINTER(vp)], i32),
            "glm_batch_run": ([vp, ctypes.POINTER(vp), ctypes.POINTER(i32)], i32),
            "glm_batch_loss": ([vp, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_double)], i32),
            "glm_batch_choice": ([vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i64),
                                  ctypes.POINTER(i32)], i32),
            "glm_batch_choice_kernel": ([vp, i32, ctypes.POINTER(i32),
                                         ctypes.POINTER(ctypes.c_double)], i32),
            "glm_tau_prior": ([vp, i64, i32, i64, ctypes.c_double, i32, ctypes.c_double,
                               ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double)], i32),
            "glm_batch_destroy": ([vp], i32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def glm_last_error() -> str:
    return load().glm_last_error().decode()


def glm_version() -> str:
    return load().glm_version().decode()


def _check(rc: int):
    if rc != GLM_OK:
        raise GlmError(rc, glm_last_error())
    return rc


def _ptr(t) -> int:
    """Data pointer of a torch tensor or numpy array (None -> 0)."""
    if t is None:
        return 0
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


def default_create_opts() -> glm_create_opts:
    o = glm_create_opts()
    load().glm_create_opts_default(ctypes.byref(o))
    return o


def default_ca_opts(**kw) -> glm_ca_opts:
    o = glm_ca_opts()
    load().glm_ca_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k in ("gram_dtype", "gemv_dtype", "accumulate", "state_dtype") and isinstance(v, str):
            v = DTYPES[v]
        setattr(o, k, v)
    return o


# ---- thin same-name wrappers -------------------------------------------------
def glm_create_ex(A, y, m, n, loss, dtype, opts=None) -> int:
    h = ctypes.c_void_p()
    _check(load().glm_create_ex(_ptr(A), _ptr(y), m, n, loss, dtype,
                                ctypes.byref(opts) if opts is not None else None,
                                ctypes.byref(h)))
    return h.value


def glm_create(A, y, m, n, loss, dtype) -> int:
    h = ctypes.c_void_p()
    _check(load().glm_create(_ptr(A), _ptr(y), m, n, loss, dtype, ctypes.byref(h)))
    return h.value


def glm_destroy(h) -> None:
    _check(load().glm_destroy(h))


def glm_sync(h) -> int:
    return load().glm_sync(h)


def glm_sgd_run(h, b, eta, lam, iters, seed, x, opts=None) -> None:
    if opts is None:
        _check(load().glm_sgd_run(h, b, eta, lam, iters, seed, _ptr(x)))
    else:
        _check(load().glm_sgd_run_ex(h, b, eta, lam, iters, seed, _ptr(x), ctypes.byref(opts)))


def glm_sgd_lowp_run(h, b, eta, lam, iters, seed, x, accumulate="f32", first_iter=0) -> None:
    acc = DTYPES[accumulate] if isinstance(accumulate, str) else accumulate
    _check(load().glm_sgd_lowp_run(h, b, eta, lam, iters, seed, _ptr(x), acc, first_iter))


def glm_ca_sgd_run(h, s, b, eta, lam, iters, seed, x, opts=None) -> None:
    if opts is None:
        _check(load().glm_ca_sgd_run(h, s, b, eta, lam, iters, seed, _ptr(x)))
    else:
        _check(load().glm_ca_sgd_run_ex(h, s, b, eta, lam, iters, seed, _ptr(x),
                                        ctypes.byref(opts)))


def glm_loss(h, x, lam) -> float:
    out = ctypes.c_double()
    _check(load().glm_loss(h, _ptr(x), lam, ctypes.byref(out)))
    return out.value


def glm_sample_indices(seed, problem, first_draw, count, m, out) -> None:
    _check(load().glm_sample_indices(seed, problem, first_draw, count, m, _ptr(out)))


def glm_sample_indices_noalloc(seed, problem, first_draw, count, m, out) -> None:
    """Host-output index draw staged in a fixed device array (no allocation).

    out: host int32 buffer (numpy array) of at least `count` entries;
    count <= GLM_SAMPLE_NOALLOC_MAX.
    """
    if 0 < count <= GLM_SAMPLE_NOALLOC_MAX:   # larger counts: the C call rejects them
        import numpy as np
        if not isinstance(out, np.ndarray) or out.dtype != np.int32 or out.size < count \
                or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a contiguous host int32 numpy array of at least "
                             "count entries")
    _check(load().glm_sample_indices_noalloc(seed, problem, first_draw, count, m, _ptr(out)))


GLM_SAMPLE_NOALLOC_MAX = 1 << 20


def glm_gram_lower(Y, dtype, nouter, s, b, n, ld, row_scale, G, impl=0, stream=None) -> None:
    _check(load().glm_gram_lower(_ptr(Y), dtype, nouter, s, b, n, ld, _ptr(row_scale),
                                 _ptr(G), impl, stream))


def glm_storage_layout(h):
    """(dtype, lda, lda8) of what the handle stores."""
    dt, lda, lda8 = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().glm_storage_layout(h, ctypes.byref(dt), ctypes.byref(lda), ctypes.byref(lda8)))
    return dt.value, lda.value, lda8.value


def glm_storage_read(h, row0, rows, A_out=None, colscale_out=None, fp8_out=None,
                     rowscale_out=None) -> None:
    """Copy stored rows / scales into host numpy buffers (None: skipped); the
    buffers must hold rows * lda storage elements, n floats, rows * lda8
    bytes and rows floats."""
    _check(load().glm_storage_read(h, row0, rows, _ptr(A_out), _ptr(colscale_out),
                                   _ptr(fp8_out), _ptr(rowscale_out)))


def glm_debug_fail_alloc(after: int) -> None:
    """Failure-path test hook: the allocation after the next `after` ones
    fails with GLM_ENOMEM; a negative value disarms it."""
    load().glm_debug_fail_alloc(after)


def glm_slab_reduce_floats(s, b) -> int:
    c = ctypes.c_int64()
    _check(load().glm_slab_reduce_floats(s, b, ctypes.byref(c)))
    return c.value


def glm_slab_partial(h, s, b, sh, seed, first_iter, x, red, opts=None) -> None:
    _check(load().glm_slab_partial(h, s, b, sh, seed, first_iter, _ptr(x), _ptr(red),
                                   ctypes.byref(opts) if opts is not None else None))


def glm_slab_finish(h, s, b, sh, eta, lam, red, x, opts=None) -> None:
    _check(load().glm_slab_finish(h, s, b, sh, eta, lam, _ptr(red), _ptr(x),
                                  ctypes.byref(opts) if opts is not None else None))


def glm_sum_buffers(dst, srcs, count, stream=None) -> None:
    arr = (ctypes.c_void_p * len(srcs))(*[_ptr(t) for t in srcs])
    _check(load().glm_sum_buffers(_ptr(dst), arr, len(srcs), count, stream))


def glm_stream(h) -> int:
    return load().glm_stream(h)


def glm_ca_plan(h, s, b, eta, lam, iters, opts=None) -> glm_run_plan:
    out = glm_run_plan()
    _check(load().glm_ca_plan(h, s, b, eta, lam, iters,
                              ctypes.byref(opts) if opts is not None else None,
                              ctypes.byref(out)))
    return out


def glm_kernel_times(h):
    ms = (ctypes.c_double * 3)()
    n = (ctypes.c_int64 * 3)()
    _check(load().glm_kernel_times(h, ms, n))
    return list(ms), list(n)


# ---- convenience wrapper -------------------------------------------------------
class Dataset:
    """Owns a libglm dataset handle.

    A: (m, n) float32 (or BF16 bit patterns as int16/uint16 with
    ``input_dtype='bf16'``), torch tensor (host or device) or numpy array;
    y: (m,) float32.  ``dtype`` is the storage type ('f32', 'bf16', 'f16').
    ``stream``: a torch.cuda.Stream (default: the current stream)."""

    def __init__(self, A, y, loss, dtype="f32", *, fp8_copy=False, column_scales=True,
                 input_dtype="f32", stream=None):
        import torch
        m, n = int(A.shape[0]), int(A.shape[1])
        o = default_create_opts()
        o.input_dtype = DTYPES[input_dtype]
        on_host = not (hasattr(A, "is_cuda") and A.is_cuda)
        o.input_on_host = 1 if on_host else 0
        o.column_scales = 1 if column_scales else 0
        o.fp8_copy = 1 if fp8_copy else 0
        st = stream if stream is not None else torch.cuda.current_stream()
        # the legacy default stream has handle 0, which the C ABI reads as
        # "make a private stream"; pass cudaStreamLegacy (0x1) instead
        o.stream = st.cuda_stream or 1
        self.stream = st
        if hasattr(A, "contiguous"):
            A = A.contiguous()
        if hasattr(y, "contiguous"):
            y = y.contiguous()
        self._keep = (A, y)
        self.m, self.n, self.loss = m, n, loss
        self.h = glm_create_ex(A, y, m, n, loss, DTYPES[dtype] if isinstance(dtype, str)
                               else dtype, o)
        self._keep = None

    def close(self):
        if getattr(self, "h", None):
            glm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sgd(self, x, b, eta, lam, iters, seed, **opts):
        glm_sgd_run(self.h, b, eta, lam, iters, seed, x,
                    default_ca_opts(**opts) if opts else None)

    def sgd_lowp(self, x, b, eta, lam, iters, seed, accumulate="f32", first_iter=0):
        glm_sgd_lowp_run(self.h, b, eta, lam, iters, seed, x, accumulate, first_iter)

    def ca_sgd(self, x, s, b, eta, lam, iters, seed, **opts):
        glm_ca_sgd_run(self.h, s, b, eta, lam, iters, seed, x,
                       default_ca_opts(**opts) if opts else None)

    def loss_value(self, x, lam) -> float:
        return glm_loss(self.h, x, lam)

    def sync(self):
        _check(glm_sync(self.h))


# ---- batched fits -------------------------------------------------------------
def glm_batch_opts_default_struct() -> glm_batch_opts:
    o = glm_batch_opts()
    load().glm_batch_opts_default(ctypes.byref(o))
    return o


def glm_batch_create(P, descs, opts=None):
    arr = (glm_problem_desc * P)(*descs)
    out = ctypes.c_void_p()
    _check(load().glm_batch_create(P, arr, ctypes.byref(opts) if opts is not None else None,
                                   ctypes.byref(out)))
    return out.value


def glm_batch_run(bt, xs, status=None):
    """xs: sequence of device FP32 iterates (torch tensors); returns the
    per-problem status list (GLM_OK or GLM_ENONFINITE)."""
    P = len(xs)
    ptrs = (ctypes.c_void_p * P)(*[_ptr(x) for x in xs])
    st = (ctypes.c_int * P)()
    _check(load().glm_batch_run(bt, ptrs, st))
    return list(st)


def glm_batch_loss(bt, xs):
    P = len(xs)
    ptrs = (ctypes.c_void_p * P)(*[_ptr(x) for x in xs])
    out = (ctypes.c_double * P)()
    _check(load().glm_batch_loss(bt, ptrs, out))
    return list(out)


def glm_batch_choice(bt, p):
    s, b, g = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int()
    _check(load().glm_batch_choice(bt, p, ctypes.byref(s), ctypes.byref(b), ctypes.byref(g)))
    return s.value, b.value, g.value


def glm_batch_choice_kernel(bt, p):
    k, t = ctypes.c_int(), ctypes.c_double()
    _check(load().glm_batch_choice_kernel(bt, p, ctypes.byref(k), ctypes.byref(t)))
    return k.value, t.value


def glm_tau_prior(Y, s, b, alpha, loss, u_A, u_in):
    """(||H_L||_2 bound, tau_G) of the autotuner's prior for host rows Y."""
    import numpy as np
    Y = np.ascontiguousarray(Y, dtype=np.float32)
    hl, tau = ctypes.c_double(), ctypes.c_double()
    _check(load().glm_tau_prior(Y.ctypes.data, Y.shape[1], s, b, alpha, loss, u_A, u_in,
                                ctypes.byref(hl), ctypes.byref(tau)))
    return hl.value, tau.value


def glm_batch_destroy(bt):
    _check(load().glm_batch_destroy(bt))


class Batch:
    """Owns a batch of independent fits.  problems: list of dicts with keys
    A (host numpy (m, n) float32), y, loss, lam, eta, iters, seed, b and
    optionally s (0 = autotuned) and gram ('f32', 'tf32', 'bf16', 'f16')."""

    def __init__(self, problems, dtype="bf16", stream=None, wait_probe_cycles=0,
                 tau_bound=0.0):
        import numpy as np
        import torch
        self._keep = []
        descs = []
        for pr in problems:
            A = np.ascontiguousarray(pr["A"], dtype=np.float32)
            y = np.ascontiguousarray(pr["y"], dtype=np.float32)
            self._keep += [A, y]
            d = glm_problem_desc()
            d.A, d.y = A.ctypes.data, y.ctypes.data
            d.m, d.n = A.shape
            d.loss = pr["loss"]
            d.lambda_, d.eta = pr["lam"], pr["eta"]
            d.iters, d.seed = pr["iters"], pr["seed"]
            d.s, d.b = pr.get("s", 0), pr["b"]
            g = pr.get("gram")
            d.gram_dtype = -1 if g is None else DTYPES[g]
            descs.append(d)
        o = glm_batch_opts_default_struct()
        o.dtype = DTYPES[dtype]
        o.input_on_host = 1
        st = stream if stream is not None else torch.cuda.current_stream()
        o.stream = st.cuda_stream or 1
        o.wait_probe_cycles = wait_probe_cycles
        o.tau_bound = tau_bound
        self.stream = st
        self.P = len(descs)
        self.h = glm_batch_create(self.P, descs, o)
        self._keep = None

    def run(self, xs):
        return glm_batch_run(self.h, xs)

    def loss(self, xs):
        return glm_batch_loss(self.h, xs)

    def choice(self, p):
        return glm_batch_choice(self.h, p)

    def choice_kernel(self, p):
        return glm_batch_choice_kernel(self.h, p)

    def close(self):
        if getattr(self, "h", None):
            glm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
