"""The bounds-checked library (-DCVWENO_CHECK, libcvweno_check.so).

Every kernel form of the path -- DG 1D (one-tile and tiled) and 2D at every degree, the
tensor-core and surrogate forms, the HWENO limiter, sensor, vertex data and features
modes, CG in 1D and 2D, Euler with the positivity limiter, the batched stages and the
allocation-free step -- runs through the checked library in a child process
(CVWENO_CHECKED=1), on meshes ragged against every tile, with 16-byte-aligned and
misaligned states:
  * no check fails (every status check is clean), and
  * every output equals the normal library's bit for bit: the checks guard accesses
    and change no arithmetic.
With a mesh's check extents narrowed by one float of the state or one cell, a step
reports CVWENO_ERR_CHECK (the access the check refused stays inside the real buffer, so
nothing faults), and the mesh runs clean again once the extents are restored.  The
normal library, which has no checks, answers CVWENO_ERR_UNSUPPORTED to the narrowing
call.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2601_16911_gb300 import build as B
from paper_2601_16911_gb300 import cvweno as cv
from paper_2601_16911_gb300 import inputs as I
from tests import checked_build_cases as C

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checked(tmp_path_factory):
    B.build(checked=True)
    out = tmp_path_factory.mktemp("checked") / "out.npz"
    env = dict(os.environ, CVWENO_CHECKED="1")
    r = subprocess.run([sys.executable, "-m", "tests.checked_build_cases", str(out)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-4000:])
    with np.load(out) as z:
        return {k: z[k] for k in z.files}


def test_the_child_ran_the_checked_library(checked):
    assert str(checked["library"][0]).endswith("libcvweno_check.so")
    assert not cv.checked() and cv.library_path().endswith("libcvweno.so")


def test_checked_outputs_equal_the_normal_library_bitwise(checked):
    normal = C.run_all()
    assert set(normal) == {k for k in checked if not k.startswith("narrowed/") and k != "library"}
    bad = [k for k in normal if not np.array_equal(normal[k], checked[k])]
    assert not bad, bad
    assert checked["step_static/status"][0] == 0


@pytest.mark.parametrize("case", ["dg2d-q2", "dg2d-q3", "cg2d-q2", "dg1d-p3", "euler-q2"])
def test_narrowed_extents_report_a_failed_check(checked, case):
    assert checked[f"narrowed/{case}/state"][0] == cv.ERR_CHECK
    assert checked[f"narrowed/{case}/cells"][0] == cv.ERR_CHECK
    assert checked[f"narrowed/{case}/restored"][0] == cv.OK


def test_normal_library_rejects_the_narrowing_call():
    d, ic = I.kpp(3, n=8, degree=2)
    m = cv.Mesh(d)
    with pytest.raises(cv.CvwenoError) as e:
        m.set_check_extents(10, 10)
    assert e.value.code == cv.ERR_UNSUPPORTED
    for bad in ((m.ncells * 9 + 1, 1), (1, m.ncells + 1), (-1, 3)):
        with pytest.raises(cv.CvwenoError) as e:
            m.set_check_extents(*bad)
        assert e.value.code == cv.ERR_ARG
    m.close()
    torch.cuda.synchronize()
