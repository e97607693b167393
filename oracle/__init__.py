"""Plain FP64 CPU oracle for SGD and CA-SGD on GLMs.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only
callers.  The product path (``paper_2606_18463_gb300``) never imports this
package, and this package imports nothing from it.

The iterative algorithms live in ``glm_oracle.c`` (FP64, built with gcc).
This module adds ctypes wrappers and the numpy-level definitions used by the
kernel-level tests (roundings to the storage formats, the strictly
block-lower Gram, the closed-form ridge solution).  Sections cited are those
of the paper (Mixed-Precision Communication-Avoiding SGD for GLMs on GPUs).

Parity status per function (pins live in ``tests/test_oracle_*.py``):
  philox4x64_10 ... pinned (numpy.random.Philox, an independent library).
  sample_indices .. pinned (big-integer definition, chi-square uniformity).
  sgd ............. pinned (exact rational arithmetic on tiny LS inputs,
                    interpolation limit, finite-difference residuals).
  ca_sgd .......... pinned (exact-arithmetic identity with SGD, Assumption 6).
  loss ............ pinned (closed forms at x = 0, brute-force sums).
  ridge_closed_form pinned (stationarity of the independently coded gradient).
  gram_lower ...... pinned (element-wise brute force).
  round_* ......... pinned (numpy float16 cast, exhaustive bit-pattern checks).
  column_scales ... pinned (closed forms: RMS against mean |a|, rounding of the
                    log2 against flooring, the all-zero column).

``oracle.local_error`` (numpy) evaluates the first-order local error budget of
one outer step (Theorem 1, Sec. 5.2) and simulates that step with each
operation rounded at its own precision; its header lists its pins.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "glm_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

LOGISTIC, LSQ, POISSON = 0, 1, 2

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (portable flags only)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, u64, f64 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        vp = ctypes.c_void_p
        lib.orc_philox4x64_10.argtypes = [vp, vp, vp]
        lib.orc_philox4x64_10.restype = None
        lib.orc_draw_word.argtypes = [u64, u64, i64]
        lib.orc_draw_word.restype = u64
        lib.orc_sample_indices.argtypes = [u64, u64, i64, i64, i64, vp]
        lib.orc_sample_indices.restype = None
        lib.orc_dloss.argtypes = [ctypes.c_int, f64, f64]
        lib.orc_dloss.restype = f64
        lib.orc_loss_one.argtypes = [ctypes.c_int, f64, f64]
        lib.orc_loss_one.restype = f64
        lib.orc_loss.argtypes = [vp, vp, i64, i64, ctypes.c_int, f64, vp]
        lib.orc_loss.restype = f64
        lib.orc_sgd.argtypes = [vp, vp, i64, i64, ctypes.c_int, i64, f64, f64,
                                i64, u64, u64, i64, vp]
        lib.orc_sgd.restype = ctypes.c_int
        lib.orc_ca_sgd.argtypes = [vp, vp, i64, i64, ctypes.c_int, i64, i64,
                                   f64, f64, i64, u64, u64, i64, vp]
        lib.orc_ca_sgd.restype = ctypes.c_int
        _lib = lib
        return lib


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data


# --------------------------------------------------------------------------
# Random index stream (Algorithm 1, sampling step; generator: Philox4x64-10)
# --------------------------------------------------------------------------
def philox4x64_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    _load().orc_philox4x64_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def draw_word(seed: int, problem: int, q: int) -> int:
    return int(_load().orc_draw_word(seed, problem, q))


def sample_indices(seed: int, problem: int, first_draw: int, count: int,
                   m: int) -> np.ndarray:
    out = np.zeros(max(count, 0), dtype=np.int64)
    if count > 0:
        _load().orc_sample_indices(seed, problem, first_draw, count, m,
                                   out.ctypes.data)
    return out


# --------------------------------------------------------------------------
# Losses, residuals and the risk (Sec. 2.1, Sec. 3.1)
# --------------------------------------------------------------------------
def dloss(loss: int, r: float, y: float) -> float:
    return float(_load().orc_dloss(loss, r, y))


def loss_one(loss: int, r: float, y: float) -> float:
    return float(_load().orc_loss_one(loss, r, y))


def loss(A, y, loss_kind: int, lam: float, x) -> float:
    A, pa = _f32(A)
    y, py = _f32(y)
    x = np.ascontiguousarray(x, dtype=np.float64)
    m, n = A.shape
    return float(_load().orc_loss(pa, py, m, n, loss_kind, lam, x.ctypes.data))


# --------------------------------------------------------------------------
# SGD and CA-SGD (Sec. 2.1, Algorithm 1)
# --------------------------------------------------------------------------
def sgd(A, y, loss_kind: int, b: int, eta: float, lam: float, iters: int,
        seed: int, x0=None, problem: int = 0, first_iter: int = 0) -> np.ndarray:
    A, pa = _f32(A)
    y, py = _f32(y)
    m, n = A.shape
    x = (np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)).copy()
    rc = _load().orc_sgd(pa, py, m, n, loss_kind, b, eta, lam, iters, seed,
                         problem, first_iter, x.ctypes.data)
    if rc != 0:
        raise ValueError(f"orc_sgd failed with status {rc}")
    return x


def ca_sgd(A, y, loss_kind: int, s: int, b: int, eta: float, lam: float,
           iters: int, seed: int, x0=None, problem: int = 0,
           first_iter: int = 0) -> np.ndarray:
    A, pa = _f32(A)
    y, py = _f32(y)
    m, n = A.shape
    x = (np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)).copy()
    rc = _load().orc_ca_sgd(pa, py, m, n, loss_kind, s, b, eta, lam, iters,
                            seed, problem, first_iter, x.ctypes.data)
    if rc != 0:
        raise ValueError(f"orc_ca_sgd failed with status {rc}")
    return x


# --------------------------------------------------------------------------
# Kernel-level definitions (Algorithm 1 margin and Gram; Table 1 storage)
# --------------------------------------------------------------------------
def gram_lower(Y, s: int, b: int) -> np.ndarray:
    """Strictly block-lower part of G = Y Y^T (Algorithm 1 uses only G_{j,<j}),
    FP64, returned as a dense (s b) x (s b) matrix with zeros elsewhere."""
    Y = np.asarray(Y, dtype=np.float64)
    G = Y @ Y.T
    sb = s * b
    blk = np.arange(sb) // b
    mask = blk[:, None] > blk[None, :]
    return np.where(mask, G, 0.0)


def margin(Y, x) -> np.ndarray:
    """Base margin r = Y x (Algorithm 1) in FP64."""
    return np.asarray(Y, dtype=np.float64) @ np.asarray(x, dtype=np.float64)


def round_bf16(v) -> np.ndarray:
    """Round FP32 values to BF16 (IEEE round-to-nearest-even on the top 16
    bits), returned as FP32 values."""
    f = np.ascontiguousarray(v, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).copy()
    out[nan] = np.nan
    return out


def round_tf32(v) -> np.ndarray:
    """Round FP32 values to TF32 (10 explicit mantissa bits), round to
    nearest with ties away from zero, returned as FP32 values."""
    f = np.ascontiguousarray(v, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    sign = u & 0x80000000
    mag = u & 0x7FFFFFFF
    mag = ((mag + 0x1000) >> 13) << 13
    out = ((sign | mag) & 0xFFFFFFFF).astype(np.uint32).view(np.float32).copy()
    out[np.isnan(f)] = np.nan
    return out


def round_f16(v) -> np.ndarray:
    """Round FP32 values to IEEE binary16 (RNE), returned as FP32 values."""
    return np.asarray(v, dtype=np.float32).astype(np.float16).astype(np.float32)


E4M3_MAX = 448.0


def round_e4m3(v) -> np.ndarray:
    """Round to FP8 E4M3 (OCP 8-bit floating point: bias 7, 3 mantissa bits,
    max normal 448, subnormal step 2^-9), round-to-nearest-even with
    saturation to +-448, returned as FP64 values."""
    x = np.asarray(v, dtype=np.float64)
    a = np.abs(x)
    # exponent of the binade, clamped to the normal range [-6, 8]
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.clip(e, -6, 8)
    step = np.exp2(e - 3)  # spacing of representable values in the binade
    q = np.round(a / step) * step  # numpy rounds half to even
    q = np.minimum(q, E4M3_MAX)
    return np.sign(x) * q


def fp8_row_scales(A) -> np.ndarray:
    """Per-row scale rho_i = the smallest power of two with
    max|a_i| <= 448 rho_i (decided by exact comparisons), 1 for all-zero rows."""
    amax = np.max(np.abs(np.asarray(A, dtype=np.float64)), axis=1)
    out = np.ones_like(amax)
    for i, a in enumerate(amax):
        if a == 0.0:
            continue
        e = int(math.ceil(math.log2(a / E4M3_MAX)))
        while a > E4M3_MAX * math.ldexp(1.0, e):
            e += 1
        while a <= E4M3_MAX * math.ldexp(1.0, e - 1):
            e -= 1
        out[i] = math.ldexp(1.0, e)
    return out


def column_scales(A) -> np.ndarray:
    """Per-column power-of-two scale kappa_j nearest the column RMS (in log2),
    1 for all-zero columns."""
    A = np.asarray(A, dtype=np.float64)
    rms = np.sqrt(np.mean(A * A, axis=0))
    return np.where(rms > 0, np.exp2(np.round(np.log2(np.where(rms > 0, rms, 1.0)))), 1.0)


def ridge_closed_form(A, y, lam: float, chunk: int = 1 << 16) -> np.ndarray:
    """Least-squares ridge minimiser of F(x) = (1/2m)||Ax - y||^2 + (lam/2)||x||^2
    from the FP64 normal equations (A^T A / m + lam I) x = A^T y / m, solved by
    Cholesky.  A^T A is accumulated over row chunks (a library matmul)."""
    m, n = A.shape
    AtA = np.zeros((n, n))
    Aty = np.zeros(n)
    for i in range(0, m, chunk):
        blk = np.asarray(A[i:i + chunk], dtype=np.float64)
        AtA += blk.T @ blk
        Aty += blk.T @ np.asarray(y[i:i + chunk], dtype=np.float64)
    M = AtA / m + lam * np.eye(n)
    L = np.linalg.cholesky(M)
    w = np.linalg.solve(L, Aty / m)
    return np.linalg.solve(L.T, w)
