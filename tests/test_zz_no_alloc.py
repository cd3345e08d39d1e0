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

CAPACITY = 4096 * 4096  # cells the fixed scratch array holds


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BLD.build()
    B.load()


def numpy_totals(U, area):
    """sum_T V_T U_T in float64 on the host: an independent check."""
    return (np.asarray(area, np.float64)[:, None] * np.asarray(U, np.float64)).sum(axis=0)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_noalloc_totals_match_allocating_entry_point_twice(prec):
    # 2*150*90 = 27,000 cells: six full tiles of 4096 cells and a ragged one
    mi = W.periodic_square(150, 90, seed=21)
    mesh = B.Mesh.from_input(mi, prec)
    perm = mesh.renumber("hilbert")
    _, _, area = mesh.export()
    dt = torch.float64 if prec == "f64" else torch.float32
    U0 = W.isentropic_vortex(mi.centroids(), mach=0.5)[perm]  # the mesh's cell order
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
        Uh = U.cpu().numpy()
        host = numpy_totals(Uh, area)
        # any summation order is within n * 2^-53 of the sum of magnitudes
        bound = Uh.shape[0] * 2.0 ** -53 * np.abs(area[:, None] * Uh).sum(axis=0)
        assert (np.abs(got - host) <= bound).all(), (call, got, host)


def test_noalloc_totals_at_full_capacity():
    # exactly 4096 full tiles: the last tile writes the last slots of the array
    rng = np.random.default_rng(5)
    U_h = rng.uniform(0.5, 2.0, size=(CAPACITY, 4)).astype(np.float32)
    area_h = rng.uniform(1e-8, 2e-8, size=CAPACITY)
    U = torch.from_numpy(U_h).cuda()
    area = torch.from_numpy(area_h).cuda()
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    host = numpy_totals(U_h, area_h)
    for _ in range(2):
        B.conserved_totals_noalloc(U, area, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert (np.abs(got - host) <= 1e-12 * np.abs(host)).all(), (got, host)
        U.mul_(0.5)
        host = host * 0.5


def test_noalloc_rejects_sizes_beyond_scratch():
    lib = B.load()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = lib.fv_conserved_totals_noalloc(B._vp(out.data_ptr()), B._vp(out.data_ptr()),
                                         CAPACITY + 1, B.FV_F32, B._vp(out.data_ptr()), None)
    assert rc == B.FV_EINVAL
    assert "capacity" in lib.fv_last_error().decode()
    # zero cells is valid and gives zero totals
    rc = lib.fv_conserved_totals_noalloc(None, None, 0, B.FV_F64, B._vp(out.data_ptr()), None)
    torch.cuda.synchronize()
    assert rc == B.FV_OK and (out.cpu().numpy() == 0).all()


def test_noalloc_rejects_misaligned_pointers():
    # the call returns before any device work: nothing misaligned is launched
    lib = B.load()
    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()  # 256-byte aligned
    cases = [(p + 8, p, B.FV_F32),    # FP32 records need 16 bytes
             (p + 16, p, B.FV_F64),   # FP64 records need 32 bytes
             (p, p + 4, B.FV_F32)]    # areas are doubles
    for u, a, prec in cases:
        rc = lib.fv_conserved_totals_noalloc(B._vp(u), B._vp(a), 8, prec, B._vp(p), None)
        assert rc == B.FV_EINVAL and "aligned" in lib.fv_last_error().decode()
    rc = lib.fv_conserved_totals_noalloc(B._vp(p), B._vp(p), 8, B.FV_F32, B._vp(p + 4), None)
    assert rc == B.FV_EINVAL and "aligned" in lib.fv_last_error().decode()
    torch.cuda.synchronize()
