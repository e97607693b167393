"""CPU checks of the C ABI: the library builds, loads and exports every
function include/glm.h declares (no compute call is made without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "glm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(glm_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_expected_api():
    from paper_2606_18463_gb300 import glm
    assert sorted(glm.EXPORTED) == _header_functions()


def test_library_exports_every_symbol():
    from paper_2606_18463_gb300 import _build_lib, glm
    if not os.path.exists(glm.LIB_PATH):
        _build_lib.build()
    lib = glm.load()
    for name in _header_functions():
        assert hasattr(lib, name), name
    assert "sm_103a" in glm.glm_version()


def test_defaults_without_gpu():
    from paper_2606_18463_gb300 import glm
    o = glm.default_ca_opts()
    assert (o.gram_dtype, o.gemv_dtype, o.recurrence_f64, o.kahan, o.use_graph) == (-1, -1, -1, 1, 1)
    c = glm.default_create_opts()
    assert (c.input_dtype, c.column_scales, c.fp8_copy) == (glm.GLM_F32, 1, 0)


def test_no_cpu_fallback_in_product():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2606_18463_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_build_flags_target_sm103a():
    from paper_2606_18463_gb300 import _build_lib
    assert "arch=compute_103a,code=sm_103a" in _build_lib.ARCH


def test_checked_variant_exports_and_reports_itself():
    """The bounds-checked build (-DGLM_CHECKED) exports the same ABI and says
    so through glm_checked_build(); the product library says it is not."""
    import ctypes
    from paper_2606_18463_gb300 import _build_lib, glm
    if not os.path.exists(glm.CHECKED_LIB_PATH):
        _build_lib.build(checked=True)
    chk = ctypes.CDLL(glm.CHECKED_LIB_PATH)
    for name in _header_functions():
        assert hasattr(chk, name), name
    chk.glm_checked_build.restype = ctypes.c_int
    assert chk.glm_checked_build() == 1
    assert glm.load().glm_checked_build() == 0
