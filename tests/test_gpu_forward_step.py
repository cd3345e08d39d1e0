"""The paper's own test case (Sec. 7.1): Mach 3 flow over a forward-facing
step, on a self-generated mesh refined toward the step corner, with a
supersonic far-field inflow, extrapolation outflow and slip walls."""
import numpy as np
import pytest

from conftest import rel_err_max
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


@pytest.fixture(scope="module")
def step_case():
    mi = W.forward_step(24, 84, 18, 72, seed=1)
    prim = W.mach3_inflow()
    return mi, prim, W.uniform_state(mi.n_tri, prim)


def mesh(mi, prim, prec):
    m = B.Mesh.from_input(mi, prec)
    m.set_freestream(*prim)
    return m


def test_fp64_matches_oracle_with_supersonic_boundaries(orc, step_case):
    mi, prim, U0 = step_case
    om = orc.Mesh(mi.xy, mi.tri, None, mi.bnd, 0, W.conserved(*prim))
    Uo, to, _, bad = om.run(U0, 150, 0.4)
    assert not bad
    g = mesh(mi, prim, "f64")
    U = torch.tensor(U0, device="cuda")
    assert g.step(U, 150, 0.4) == pytest.approx(to, rel=1e-13)
    assert rel_err_max(U.cpu().numpy(), Uo) <= 1e-12


def test_shock_forms_and_run_to_paper_end_time(step_case):
    mi, prim, U0 = step_case
    g32 = mesh(mi, prim, "f32")
    g32.renumber("rcm")
    perm = B.Mesh.from_input(mi, "f32").renumber("rcm")
    U = torch.tensor(U0[perm], dtype=torch.float32, device="cuda")
    t = 0.0
    while t < 4.0 - 1e-12:
        t += g32.step(U, 20000, 0.4, t_stop=4.0 - t)
    assert t == pytest.approx(4.0, rel=1e-12)
    Un = U.double().cpu().numpy()
    rho = Un[:, 0]
    assert np.isfinite(Un).all() and rho.min() > 0
    # the step compresses the flow: a detached shock raises the density well
    # above the inflow value, and the expansion round the corner lowers it
    assert rho.max() > 3.0 * prim[0] and rho.min() < 0.8 * prim[0]


def test_fp32_tracks_fp64_before_the_shock_interacts(step_case):
    mi, prim, U0 = step_case
    a = mesh(mi, prim, "f32")
    b = mesh(mi, prim, "f64")
    A = torch.tensor(U0, dtype=torch.float32, device="cuda")
    Bt = torch.tensor(U0, device="cuda")
    # each precision takes its own CFL steps (the bound is evaluated in the
    # state's precision); both stop at t = 0.2 exactly
    ta = a.step(A, 20000, 0.4, t_stop=0.2)
    tb = b.step(Bt, 20000, 0.4, t_stop=0.2)
    assert ta == pytest.approx(0.2, rel=1e-12) and tb == pytest.approx(0.2, rel=1e-12)
    x, y = A.double().cpu().numpy()[:, 0], Bt.cpu().numpy()[:, 0]
    assert np.linalg.norm(x - y) / np.linalg.norm(y) <= 1e-5


def test_paper_size_step_with_max_wave_speed_matches_oracle(orc):
    # the 410,400-cell mesh (the paper's largest size) with the one-sided
    # maximum wave speed, FP64, 30 steps from the Mach 3 start: the oracle
    # with the same reading, cell by cell
    mi = W.forward_step_394k()
    prim = W.mach3_inflow()
    U0 = W.uniform_state(mi.n_tri, prim)
    g = mesh(mi, prim, "f64")
    g.set_wave_speed("max")
    perm = g.renumber("hilbert")
    g.autotune(torch.tensor(U0[perm], device="cuda"))
    U = torch.tensor(U0[perm], device="cuda")
    t = g.step(U, 30, 0.4)
    orc.set_wave_speed("max")
    try:
        om = orc.Mesh(mi.xy, mi.tri, None, mi.bnd, 0, W.conserved(*prim))
        Uo, to, _, bad = om.run(U0, 30, 0.4)
    finally:
        orc.set_wave_speed("average")
    assert not bad and t == pytest.approx(to, rel=1e-13)
    out = np.empty_like(Uo)
    out[perm] = U.cpu().numpy()
    assert rel_err_max(out, Uo) <= 1e-12
