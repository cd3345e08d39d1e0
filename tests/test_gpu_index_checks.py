"""The bounds-checked build (compiled with FV_DEBUG, fv_index_checks() == 1).

Memory checkers cannot run here, so the library can be built with every
table-indexed gather tested against its array.  A child process loads that
build (FV_LIBRARY=debug), runs every kernel family on small meshes and steps
meshes whose device neighbour table was given one index outside its array.
The clean runs must give bitwise the results of the normal build (loaded by
this process), and every planted index must be reported as FV_EINDEX --
caught and skipped by the kernel, not read.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import index_check_runs as R
from paper_1408_5715_gb300 import binding as B
from paper_1408_5715_gb300 import build as BLD

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BLD.build()
    B.load()


@pytest.fixture(scope="module")
def child(tmp_path_factory):
    BLD.build(debug=True)
    out = tmp_path_factory.mktemp("idx") / "runs.npz"
    env = dict(os.environ, FV_LIBRARY="debug")
    res = subprocess.run([sys.executable, R.__file__, str(out)], env=env, capture_output=True,
                         text=True, timeout=900)
    assert res.returncode == 0, res.stdout[-3000:] + res.stderr[-3000:]
    return dict(np.load(out))


def test_normal_build_has_no_checks():
    lib = B.load()
    assert lib.fv_index_checks() == 0


def test_checked_build_gives_the_same_bits(child):
    ours = R.clean_runs()
    assert set(ours) <= set(child)
    for name, U in ours.items():
        assert np.array_equal(U, child[name]), name


def test_checked_build_reports_planted_indices(child):
    codes = {k[5:]: int(v) for k, v in child.items() if k.startswith("code_")}
    assert len(codes) == 5
    for name, code in codes.items():
        assert code == B.FV_EINDEX, (name, code)
