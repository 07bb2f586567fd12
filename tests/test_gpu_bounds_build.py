"""The bounds-checked debug build (compiled with MFD_BOUNDS_CHECK): every stencil
index is tested against the node set it points into before a kernel gathers
through it, and every stencil row when a simulation packs it; an index outside
its set is counted, replaced by 0 (no trap, no out-of-bounds read) and turns the
call into MFD_ERR_STATE. The small parity cases (collocated, staggered with
16-bit indices, 3D, batched, adjoint, checkpoint) run under that build in a
child process and pass, so no kernel met an index out of range.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_2508_18205_gb300")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_default_build_is_unchecked():
    assert M.lib().mfd_build_flags() == 0


def test_small_parity_cases_under_the_bounds_checked_build():
    from paper_2508_18205_gb300 import build as B
    path = B.build(bounds=True)
    env = dict(os.environ, MFD_LIB=path)
    flag = subprocess.run([sys.executable, "-c", "import paper_2508_18205_gb300 as M; print(M.lib().mfd_build_flags())"],
                          env=env, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert flag.returncode == 0 and flag.stdout.strip() == str(M.MFD_BUILD_BOUNDS_CHECK), flag.stderr[-2000:]
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider",
                        "tests/test_gpu_parity.py", "tests/test_gpu_batch.py", "tests/test_gpu_adjoint.py",
                        "tests/test_gpu_checkpoint.py", "-k", "not full_config"],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
