"""The allocation-free totals entry point (fv_conserved_totals_noalloc).

It serves callers that cannot allocate device memory (for example code inside
a framework that owns the device memory budget through its own caching
allocator).  Its partial sums live in a fixed array in the library's device
code instead of memory from cudaMalloc.  This file is collected last so that a
run stopping at the first failure has run every other test first; it passes
alone in a fresh process as well.
"""
import numpy as np
import pytest

from paper_1408_5715_gb300 import binding as B
from paper_1408_5715_gb300 import build as BLD
from paper_1408_5715_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BLD.build()
    B.load()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_noalloc_totals_match_allocating_entry_point_twice(prec):
    # 2*150*90 = 27,000 cells: six full tiles of 4096 cells and a ragged one
    mi = W.periodic_square(150, 90, seed=21)
    mesh = B.Mesh.from_input(mi, prec)
    mesh.renumber("hilbert")
    _, _, area = mesh.export()
    dt = torch.float64 if prec == "f64" else torch.float32
    U0 = W.isentropic_vortex(mi.centroids(), mach=0.5)
    U = torch.tensor(U0, dtype=dt, device="cuda")
    area_d = torch.tensor(area, dtype=torch.float64, device="cuda")
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    scale = np.abs(U0 * area[:, None]).sum(axis=0)
    for call in range(2):
        if call == 1:
            mesh.step(U, 7, 0.4)  # a different state for the second call
        want = mesh.totals(U)
        B.conserved_totals_noalloc(U, area_d, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert (np.abs(got - want) <= 1e-14 * scale).all(), (call, got, want)


def test_noalloc_rejects_sizes_beyond_scratch():
    lib = B.load()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = lib.fv_conserved_totals_noalloc(B._vp(out.data_ptr()), B._vp(out.data_ptr()),
                                         16_777_217, B.FV_F32, B._vp(out.data_ptr()), None)
    assert rc == B.FV_EINVAL
    assert "capacity" in lib.fv_last_error().decode()
    # zero cells is valid and gives zero totals
    rc = lib.fv_conserved_totals_noalloc(None, None, 0, B.FV_F64, B._vp(out.data_ptr()), None)
    torch.cuda.synchronize()
    assert rc == B.FV_OK and (out.cpu().numpy() == 0).all()
