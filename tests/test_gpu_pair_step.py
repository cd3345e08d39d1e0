"""Two forward-Euler steps per launch (temporal blocking, the GPU form of the
paper's chained processors, Sec. 7) against single steps and the FP64 oracle.

With a fixed dt the two-step launch must be bitwise equal to two single
steps: every cell update does the single-step arithmetic.  With cfl > 0 both
steps of a pair use the CFL bound of the pair's first state, which the tests
rebuild from single steps with that fixed dt."""
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


def dev(U):
    return torch.tensor(np.ascontiguousarray(U), dtype=torch.float32, device="cuda")


def case(kind):
    if kind == "vortex":
        mi = W.periodic_square(72, 40, seed=3)  # 5,760 cells: 12 tiles of 512, ragged last
        U0 = W.isentropic_vortex(mi.centroids(), mach=0.5, beta=5.0)
        prim = (1.0, 0.5 * np.sqrt(1.4), 0.0, 1.0)
    elif kind == "channel":
        mi = W.channel_bump(90, 30, seed=4)  # walls and far field
        prim = W.freestream(0.5)
        U0 = W.random_smooth_state(mi.centroids(), seed=5)
    else:
        mi = W.forward_step(12, 42, 9, 36, seed=6)  # far-field inflow, extrapolation outflow
        prim = W.mach3_inflow()
        U0 = W.uniform_state(mi.n_tri, prim)
    return mi, prim, U0


def mesh(mi, prim, order="hilbert"):
    m = B.Mesh.from_input(mi, "f32")
    m.set_freestream(*prim)
    perm = m.renumber(order, seed=2)
    return m, perm


@pytest.mark.parametrize("kind", ["vortex", "channel", "step"])
@pytest.mark.parametrize("comp", [True, False])
@pytest.mark.parametrize("staged", [False, True])
def test_pairs_equal_single_steps_with_fixed_dt(kind, comp, staged):
    mi, prim, U0 = case(kind)
    a, perm = mesh(mi, prim)
    b, _ = mesh(mi, prim)
    for m in (a, b):
        m.set_compensation(comp)
    b.set_blocking(2, 512, staged)
    dt = 0.5 * a.compute_dt(dev(U0[perm]), 0.4)
    for nsteps in (1, 2, 7, 101, 200):  # odd tails, a graph of 96 steps plus a tail
        Ua, Ub = dev(U0[perm]), dev(U0[perm])
        ta = a.step(Ua, nsteps, -dt)
        tb = b.step(Ub, nsteps, -dt)
        assert ta == tb
        assert torch.equal(Ua, Ub), (kind, comp, nsteps)


@pytest.mark.parametrize("staged", [False, True])
def test_pairs_clamp_at_t_stop_like_single_steps(staged):
    mi, prim, U0 = case("vortex")
    a, perm = mesh(mi, prim)
    b, _ = mesh(mi, prim)
    b.set_blocking(2, 1024, staged)
    dt = a.compute_dt(dev(U0[perm]), 0.4)
    for t_stop in (0.5 * dt, 2.5 * dt, 3.0 * dt, 40.3 * dt):
        Ua, Ub = dev(U0[perm]), dev(U0[perm])
        ta = a.step(Ua, 60, -dt, t_stop=t_stop)
        tb = b.step(Ub, 60, -dt, t_stop=t_stop)
        assert ta == tb == pytest.approx(t_stop, rel=1e-14)
        assert torch.equal(Ua, Ub)


def test_tile_sizes_and_orders_agree():
    mi, prim, U0 = case("channel")
    ref = None
    for order in ("hilbert", "rcm"):
        for tile, staged in ((512, False), (1024, False), (2048, False), (512, True),
                             (1024, True)):
            m, perm = mesh(mi, prim, order)
            m.set_blocking(2, tile, staged)
            U = dev(U0[perm])
            m.step(U, 40, -2e-4)
            out = np.empty_like(U0, dtype=np.float32)
            out[perm] = U.cpu().numpy()
            if ref is None:
                ref = out
            np.testing.assert_array_equal(out, ref)


@pytest.mark.parametrize("comp", [True, False])
def test_cfl_mode_takes_one_dt_per_pair(comp):
    mi, prim, U0 = case("vortex")
    a, perm = mesh(mi, prim)
    b, _ = mesh(mi, prim)
    for m in (a, b):
        m.set_compensation(comp)
    b.set_blocking(2, 1024, True)
    Ua, Ub = dev(U0[perm]), dev(U0[perm])
    t_single = 0.0
    for _ in range(3):  # three pairs: dt from the state at the start of each
        dt = a.compute_dt(Ua, 0.4)
        t_single += a.step(Ua, 2, -dt)
    if comp:
        # each call starts from the caller's float state (no remainder), so
        # the pairs are taken in separate calls too
        tb = sum(b.step(Ub, 2, 0.4) for _ in range(3))
    else:
        tb = b.step(Ub, 6, 0.4)
    assert torch.equal(Ua, Ub)
    assert tb == pytest.approx(t_single, rel=1e-15)


def test_pairs_track_the_fp64_oracle(orc):
    mi, prim, U0 = case("vortex")
    uinf = W.conserved(*prim)
    om = orc.Mesh(mi.xy, mi.tri, mi.canon, mi.bnd, mi.default_bc, uinf)
    m, perm = mesh(mi, prim)
    m.set_blocking(2, 512)
    dt = m.compute_dt(dev(U0[perm]), 0.4)
    Uo, to, _, bad = om.run(U0, 120, -dt)
    assert not bad
    U = dev(U0[perm])
    assert m.step(U, 120, -dt) == pytest.approx(to, rel=1e-14)
    out = np.empty_like(Uo)
    out[perm] = U.double().cpu().numpy()
    rho, ref = out[:, 0], Uo[:, 0]
    assert np.linalg.norm(rho - ref) / np.linalg.norm(ref) <= 1e-5


def test_pairs_report_bad_states_and_refuse_other_schemes():
    mi, prim, U0 = case("vortex")
    m, perm = mesh(mi, prim)
    m.set_blocking(2)
    bad = U0[perm].copy()
    bad[len(bad) // 2, 3] = -1.0  # negative energy: negative pressure
    with pytest.raises(B.FVError) as e:
        m.step(dev(bad), 4, -1e-4)
    assert e.value.code == B.FV_ENONFINITE
    with pytest.raises(B.FVError, match="forward Euler"):
        m.step(dev(U0[perm]), 2, 0.4, scheme="rk2")
    m.set_blocking(1)
    m.step(dev(U0[perm]), 2, 0.4, scheme="rk2")


def test_pairs_on_tiny_and_empty_meshes():
    two = W.two_cells()
    m = B.Mesh.from_input(two, "f32")
    m.set_blocking(2, 512)
    U = dev(np.array([[1.0, 0.0, 0.0, 2.5], [0.125, 0.0, 0.0, 0.25]]))
    ref = B.Mesh.from_input(two, "f32")
    Ur = U.clone()
    assert m.step(U, 5, -1e-3) == ref.step(Ur, 5, -1e-3)
    assert torch.equal(U, Ur)
    e = B.Mesh(np.zeros((0, 2)), np.zeros((0, 3), np.int32))
    e.set_blocking(2)
    assert e.step(torch.zeros((0, 4), dtype=torch.float32, device="cuda"), 3, 0.4) == 0.0


def test_staged_pairs_bounded_wait_gives_timeout():
    # a wait limit of 0 makes every wait on a bulk copy give up at once: the
    # blocks drain their copies and return, the call reports FV_ETIMEOUT, and
    # the library stays usable
    mi, prim, U0 = case("vortex")
    m, perm = mesh(mi, prim)
    m.set_blocking(2, 512, True)
    m.set_wait_limit(0)
    with pytest.raises(B.FVError) as e:
        m.step(dev(U0[perm]), 4, -1e-4)
    assert e.value.code == B.FV_ETIMEOUT
    m.set_wait_limit(1 << 24)
    ref, _ = mesh(mi, prim)
    U, Ur = dev(U0[perm]), dev(U0[perm])
    m.step(U, 4, -1e-4)
    ref.step(Ur, 4, -1e-4)
    assert torch.equal(U, Ur)


def test_staged_pairs_on_a_large_mesh_match_single_steps():
    # many tiles per persistent block (both stages cycle many times), ragged end
    mi = W.periodic_square(400, 263, seed=9)  # 210,400 cells
    U0 = W.isentropic_vortex(mi.centroids(), mach=0.5, beta=5.0)
    prim = (1.0, 0.5 * np.sqrt(1.4), 0.0, 1.0)
    a, perm = mesh(mi, prim)
    b, _ = mesh(mi, prim)
    b.set_blocking(2, 1024, True)
    dt = a.compute_dt(dev(U0[perm]), 0.4)
    Ua, Ub = dev(U0[perm]), dev(U0[perm])
    a.step(Ua, 20, -dt)
    b.step(Ub, 20, -dt)
    assert torch.equal(Ua, Ub)


def test_pairs_on_the_16m_square_match_single_steps():
    # the benchmark's 16.8M-cell square in its launch configuration (tile 1024,
    # Hilbert): four steps with a fixed dt as two pairs, bitwise against four
    # single steps of the tiled one-step shape
    mi = W.vortex_square_16m()
    U0 = W.isentropic_vortex(mi.centroids(), mach=0.5)
    prim = (1.0, 0.5 * np.sqrt(1.4), 0.0, 1.0)
    a, perm = mesh(mi, prim)
    b, _ = mesh(mi, prim)
    a.set_variant(6)
    b.set_blocking(2, 1024)
    Ua = dev(U0[perm])
    dt = a.compute_dt(Ua, 0.4)
    Ub = Ua.clone()
    a.step(Ua, 4, -dt)
    b.step(Ub, 4, -dt)
    assert torch.equal(Ua, Ub)


def test_autotune_keeps_the_two_step_tile_size():
    # the autotuner times one-step shapes (and tile sizes that fill whole
    # waves); a mesh set to two steps per launch keeps its standard tile size
    mi, prim, U0 = case("channel")
    m, perm = mesh(mi, prim)
    m.set_blocking(2, 768)
    m.autotune(dev(U0[perm]))
    assert m.tiling()[1] == 768
    ref, _ = mesh(mi, prim)
    ref.set_blocking(2, 768)
    U, Ur = dev(U0[perm]), dev(U0[perm])
    m.step(U, 6, -1e-4)
    ref.step(Ur, 6, -1e-4)
    assert torch.equal(U, Ur)
