"""Host-side argument checks of the C ABI that run before any CUDA call, so
they are exercised here without a GPU: corrupted dataset arguments and
corrupted batch descriptors are rejected with GLM_EINVAL (or
GLM_EUNSUPPORTED) and a message, and nothing is created."""
import ctypes
import os

import numpy as np
import pytest

from paper_2606_18463_gb300 import glm

LIB = glm.LIB_PATH
pytestmark = pytest.mark.skipif(not os.path.exists(LIB), reason="libglm.so not built")


@pytest.fixture(scope="module")
def L():
    return glm.load()


def _create(L, A, y, m, n, loss, dtype):
    h = ctypes.c_void_p()
    rc = L.glm_create_ex(A, y, m, n, loss, dtype, None, ctypes.byref(h))
    return rc, h.value


def test_create_argument_errors(L):
    a = np.zeros((4, 3), dtype=np.float32)
    y = np.ones(4, dtype=np.float32)
    pa, py = a.ctypes.data, y.ctypes.data
    for args in [(0, py, 4, 3, 0, 0), (pa, 0, 4, 3, 0, 0), (pa, py, 0, 3, 0, 0),
                 (pa, py, 1 << 31, 3, 0, 0), (pa, py, 4, 0, 0, 0), (pa, py, 4, 70000, 0, 0),
                 (pa, py, 4, 3, 7, 0), (pa, py, 4, 3, 0, 9), (pa, py, 4, 3, 0, glm.GLM_E4M3)]:
        rc, h = _create(L, *args)
        assert rc == glm.GLM_EINVAL and h is None, args
        assert glm.glm_last_error()


def _desc(a_arr, y_arr, **kw):
    d = glm.glm_problem_desc()
    d.A, d.y = a_arr.ctypes.data, y_arr.ctypes.data
    d.m, d.n = a_arr.shape
    d.loss, d.lambda_, d.eta, d.iters, d.seed, d.s, d.b = 0, 1e-4, 0.1, 64, 1, 4, 16
    d.gram_dtype = -1
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("field,value,code", [
    ("A", 0, glm.GLM_EINVAL), ("y", 0, glm.GLM_EINVAL), ("m", 0, glm.GLM_EINVAL),
    ("n", 0, glm.GLM_EINVAL), ("n", 20000, glm.GLM_EINVAL), ("b", 0, glm.GLM_EINVAL),
    ("b", 2048, glm.GLM_EINVAL), ("s", -1, glm.GLM_EINVAL), ("s", 65, glm.GLM_EINVAL),
    ("iters", -5, glm.GLM_EINVAL), ("loss", 9, glm.GLM_EINVAL),
    ("eta", 0.0, glm.GLM_EINVAL), ("eta", float("nan"), glm.GLM_EINVAL),
    ("lambda_", -1.0, glm.GLM_EINVAL), ("lambda_", 20.0, glm.GLM_EINVAL),
    ("gram_dtype", glm.GLM_E4M3, glm.GLM_EINVAL),
    ("s", 64, glm.GLM_EINVAL),                      # s b = 1024 ok; with b = 256: too large
])
def test_corrupted_batch_descriptor_rejected(L, field, value, code):
    A = np.zeros((100, 8), dtype=np.float32)
    y = np.ones(100, dtype=np.float32)
    good = _desc(A, y)
    bad = _desc(A, y, **{field: value})
    if field == "s" and value == 64:
        bad.b = 256
    descs = (glm.glm_problem_desc * 3)(good, bad, good)
    out = ctypes.c_void_p()
    rc = L.glm_batch_create(3, descs, None, ctypes.byref(out))
    assert rc == code and out.value is None, (field, value, rc, glm.glm_last_error())
    assert glm.glm_last_error()


def test_mixed_gram_types_and_unsupported_decay(L):
    A = np.zeros((100, 8), dtype=np.float32)
    y = np.ones(100, dtype=np.float32)
    descs = (glm.glm_problem_desc * 2)(_desc(A, y, gram_dtype=glm.GLM_BF16),
                                       _desc(A, y, gram_dtype=glm.GLM_F32))
    out = ctypes.c_void_p()
    assert L.glm_batch_create(2, descs, None, ctypes.byref(out)) == glm.GLM_EINVAL
    assert "same gram_dtype" in glm.glm_last_error()
    # c^-(s-1) beyond 2^60: eta lambda = 0.5 at s = 64
    descs = (glm.glm_problem_desc * 1)(_desc(A, y, s=64, b=16, eta=0.5, lambda_=1.0))
    assert L.glm_batch_create(1, descs, None, ctypes.byref(out)) == glm.GLM_EUNSUPPORTED
    opts = glm.glm_batch_opts()
    L.glm_batch_opts_default(ctypes.byref(opts))
    opts.wait_probe_cycles = -1
    descs = (glm.glm_problem_desc * 1)(_desc(A, y))
    assert L.glm_batch_create(1, descs, ctypes.byref(opts), ctypes.byref(out)) == glm.GLM_EINVAL
