"""The bounds-checked build (libglm_checked.so, -DGLM_CHECKED) on the GPU
parity cases: every kernel tests its computed indices (drawn rows against m,
Gram output rows and G copies against the packed G of the launch) and an index
outside its buffer would surface as GLM_EBOUNDS at the next glm_sync or
glm_batch_run.  The small parity cases (every Gram kernel and operand type,
ragged shapes, both chains, the batched fits, the narrow recipes) run under it
in a child process and must pass unchanged."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASES = ["tests/test_gpu_parity.py", "tests/test_gpu_stream.py", "tests/test_gpu_batch.py",
         "tests/test_gpu_slab.py"]


def test_parity_cases_under_checked_build():
    from paper_2606_18463_gb300 import _build_lib, glm
    if not os.path.exists(glm.CHECKED_LIB_PATH):
        _build_lib.build(checked=True)
    env = dict(os.environ, GLM_LIBRARY=glm.CHECKED_LIB_PATH)
    probe = ("from paper_2606_18463_gb300 import glm; import sys; "
             "sys.exit(0 if glm.load().glm_checked_build() == 1 else 3)")
    assert subprocess.run([sys.executable, "-c", probe], env=env, cwd=ROOT).returncode == 0
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu",
                        "-k", "not large_lsq", *CASES],
                       env=env, cwd=ROOT, capture_output=True, text=True)
    print(r.stdout[-2000:])
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
