"""Normals from vertex coordinates (Sec. 7's alternative to stored normals)
against the stored geometry of the same snapped mesh and the FP64 oracle.

After fv_mesh_set_geometry(FV_GEOM_VERTEX) the nodes sit on a fixed-point
grid; the tile kernel forms each cell's normals from the grid coordinates
of its nodes and reads 1/V.  Those are bitwise the stored FP32 records of the
snapped mesh, so every step, residual and CFL bound must be bitwise equal to
the stored-record kernels, and within the FP32 tolerance of the oracle run on
the snapped node coordinates."""
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
        mi = W.periodic_square(72, 40, seed=3)  # 5,760 cells: ragged last tile at every size
        U0 = W.isentropic_vortex(mi.centroids(), mach=0.5, beta=5.0)
        prim = (1.0, 0.5 * np.sqrt(1.4), 0.0, 1.0)
    elif kind == "channel":
        mi = W.channel_bump(90, 30, seed=4)  # walls and far field
        prim = W.freestream(0.5)
        U0 = W.random_smooth_state(mi.centroids(), seed=5)
    else:
        mi = W.forward_step(12, 42, 9, 36, seed=6)  # supersonic inflow, extrapolation outflow
        prim = W.mach3_inflow()
        U0 = W.uniform_state(mi.n_tri, prim)
    return mi, prim, U0


def pair(mi, prim, order="hilbert"):
    """(vertex-form mesh, stored-record mesh of the same snapped nodes, perm)."""
    v = B.Mesh.from_input(mi, "f32")
    s = B.Mesh.from_input(mi, "f32")
    for m in (v, s):
        m.set_freestream(*prim)
    perm = v.renumber(order, seed=2)
    s.renumber(order, seed=2)
    v.set_geometry("vertex")
    s.set_geometry("vertex")
    s.set_geometry("stored")
    return v, s, perm


@pytest.mark.parametrize("kind", ["vortex", "channel", "step"])
@pytest.mark.parametrize("tile", [512, 768, 1024, 2048])
def test_vertex_form_equals_stored_records(kind, tile):
    mi, prim, U0 = case(kind)
    v, s, perm = pair(mi, prim)
    v.set_blocking(1, tile)
    s.set_variant(6)
    s.set_blocking(1, tile)
    for comp in (True, False):
        for m in (v, s):
            m.set_compensation(comp)
        for scheme in ("fe", "rk2"):
            Uv, Us = dev(U0[perm]), dev(U0[perm])
            tv = v.step(Uv, 23, 0.4, scheme=scheme)
            ts = s.step(Us, 23, 0.4, scheme=scheme)
            assert tv == ts
            assert torch.equal(Uv, Us), (kind, tile, comp, scheme)


@pytest.mark.parametrize("kind", ["vortex", "channel", "step"])
def test_vertex_form_equals_every_stored_shape(kind):
    mi, prim, U0 = case(kind)
    v, s, perm = pair(mi, prim)
    Uv = dev(U0[perm])
    tv = v.step(Uv, 17, 0.4)
    for shape in range(B.N_VARIANTS):
        s.set_variant(shape)
        Us = dev(U0[perm])
        assert s.step(Us, 17, 0.4) == tv
        assert torch.equal(Uv, Us), shape


def test_vertex_form_residual_and_max_wave_speed():
    mi, prim, U0 = case("step")
    v, s, perm = pair(mi, prim)
    s.set_variant(6)
    U = dev(U0[perm])
    U[:, 1] *= 0.7  # a non-uniform state: fluxes do not cancel
    np.testing.assert_array_equal(v.residual(U).cpu().numpy(), s.residual(U).cpu().numpy())
    for m in (v, s):
        m.set_wave_speed("max")
    Uv, Us = U.clone(), U.clone()
    assert v.step(Uv, 31, 0.4) == s.step(Us, 31, 0.4)
    assert torch.equal(Uv, Us)


@pytest.mark.parametrize("kind", ["vortex", "channel", "step"])
def test_vertex_form_tracks_the_fp64_oracle_on_the_snapped_nodes(orc, kind):
    mi, prim, U0 = case(kind)
    v, _, perm = pair(mi, prim)
    xy, _ = v.nodes()
    om = orc.Mesh(xy, mi.tri, mi.canon, mi.bnd, mi.default_bc, W.conserved(*prim))
    U = dev(U0[perm])
    dt = v.compute_dt(U, 0.4)
    Uo, to, _, bad = om.run(U0, 150, -dt)
    assert not bad
    assert v.step(U, 150, -dt) == pytest.approx(to, rel=1e-14)
    out = np.empty_like(Uo)
    out[perm] = U.double().cpu().numpy()
    for q in range(4):
        ref = Uo[:, q]
        scale = max(np.linalg.norm(ref), 1e-3 * np.sqrt(len(ref)) * np.abs(Uo).max())
        assert np.linalg.norm(out[:, q] - ref) / scale <= 1e-5, q


def test_vertex_form_conserves_and_keeps_a_free_stream():
    mi, prim, U0 = case("vortex")
    v, _, perm = pair(mi, prim)
    v.set_compensation(False)
    U = dev(U0[perm])
    T0 = v.totals(U)
    v.step(U, 200, 0.4)
    T1 = v.totals(U)
    # exact flux antisymmetry: the totals move only by the rounding of the
    # FP32 states
    area = v.export()[2]
    scale = np.abs(U0[perm] * area[:, None]).sum(axis=0)
    assert (np.abs(T1 - T0) <= 1e-5 * scale).all()
    uni = W.uniform_state(mi.n_tri, prim)
    Uf = dev(uni)
    v.step(Uf, 100, 0.4)
    assert np.abs(Uf.double().cpu().numpy() - uni).max() <= 1e-6


def test_vertex_form_autotunes_the_tile_shape_only():
    mi, prim, U0 = case("channel")
    v, s, perm = pair(mi, prim)
    best, us = v.autotune(dev(U0[perm]))
    assert best == 6
    assert all(not np.isfinite(t) for i, t in enumerate(us) if i != 6)
    assert np.isfinite(us[6])
    Uv, Us = dev(U0[perm]), dev(U0[perm])
    s.set_variant(1)
    assert v.step(Uv, 9, 0.4) == s.step(Us, 9, 0.4)
    assert torch.equal(Uv, Us)


def test_batches_of_snapped_meshes_match_their_vertex_runs():
    cases = [case("vortex"), case("channel"), case("step")]
    vs, states = [], []
    for mi, prim, U0 in cases:
        v, _, perm = pair(mi, prim)
        vs.append(v)
        states.append(U0[perm])
    b = B.Batch(vs)
    Ub = dev(b.pack(states))
    b.step(Ub, 12, 0.4)
    for m, U0, Ubi in zip(vs, states, b.unpack(Ub)):
        U = dev(U0)
        m.step(U, 12, 0.4)
        assert torch.equal(U, Ubi)


def test_vertex_form_with_two_steps_per_launch_uses_the_snapped_records():
    mi, prim, U0 = case("vortex")
    v, s, perm = pair(mi, prim)
    v.set_blocking(2, 1024)
    s.set_variant(6)
    dt = s.compute_dt(dev(U0[perm]), 0.4)
    Uv, Us = dev(U0[perm]), dev(U0[perm])
    v.step(Uv, 10, -dt)
    s.step(Us, 10, -dt)
    assert torch.equal(Uv, Us)


@pytest.mark.parametrize("workload", ["channel_1m", "square_16m"])
def test_vertex_form_at_full_size(workload):
    # the benchmark meshes in their launch configuration (Hilbert order,
    # autotuned tile size): a few steps bitwise against the stored records
    if workload == "channel_1m":
        mi = W.channel_bump_1m()
        prim = W.freestream(0.5)
        U0 = W.random_smooth_state(mi.centroids(), seed=5)
    else:
        mi = W.vortex_square_16m()
        prim = (1.0, 0.5 * np.sqrt(1.4), 0.0, 1.0)
        U0 = W.isentropic_vortex(mi.centroids(), mach=0.5)
    v, s, perm = pair(mi, prim)
    Uv = dev(U0[perm])
    v.autotune(Uv)
    s.set_variant(6)
    Us = Uv.clone()
    assert v.step(Uv, 4, 0.4) == s.step(Us, 4, 0.4)
    assert torch.equal(Uv, Us)


@pytest.mark.parametrize("geometry", ["stored", "vertex"])
def test_any_tile_size_gives_the_same_bits(geometry):
    # the one-step tile shape at sizes between the standard four (wave-fitted
    # sizes of the autotuner), ragged last tiles included
    mi, prim, U0 = case("channel")
    v, s, perm = pair(mi, prim)
    s.set_variant(1)
    Ur = dev(U0[perm])
    tr = s.step(Ur, 13, 0.4)
    m = v if geometry == "vertex" else s
    m.set_variant(6)
    if geometry == "stored":
        m.set_geometry("stored")
    for tile in (32, 96, 300, 672, 1000, 1344, 1700, 2048):
        m.set_blocking(1, tile)
        assert m.tiling() == (6, tile)
        U = dev(U0[perm])
        assert m.step(U, 13, 0.4) == tr
        assert torch.equal(U, Ur), tile


def test_snapping_then_renumbering_equals_renumbering_then_snapping():
    # the node grid does not depend on the cell order, and renumbering a
    # snapped mesh carries its node lists along
    mi, prim, U0 = case("channel")
    a = B.Mesh.from_input(mi, "f32")
    b = B.Mesh.from_input(mi, "f32")
    for m in (a, b):
        m.set_freestream(*prim)
    a.set_geometry("vertex")
    pa = a.renumber("rcm", seed=1)
    pb = b.renumber("rcm", seed=1)
    b.set_geometry("vertex")
    np.testing.assert_array_equal(pa, pb)
    np.testing.assert_array_equal(a.nodes()[0], b.nodes()[0])
    Ua, Ub = dev(U0[pa]), dev(U0[pb])
    assert a.step(Ua, 15, 0.4) == b.step(Ub, 15, 0.4)
    assert torch.equal(Ua, Ub)


def test_vertex_form_on_tiny_and_empty_meshes():
    two = W.two_cells()
    v = B.Mesh.from_input(two, "f32")
    s = B.Mesh.from_input(two, "f32")
    v.set_geometry("vertex")
    s.set_geometry("vertex")
    s.set_geometry("stored")
    U = dev(np.array([[1.0, 0.0, 0.0, 2.5], [0.125, 0.0, 0.0, 0.25]]))
    Us = U.clone()
    assert v.step(U, 5, -1e-3) == s.step(Us, 5, -1e-3)
    assert torch.equal(U, Us)
    e = B.Mesh(np.zeros((0, 2)), np.zeros((0, 3), np.int32))
    e.set_geometry("vertex")
    assert e.nodes()[1] is None
    assert e.step(torch.zeros((0, 4), dtype=torch.float32, device="cuda"), 3, 0.4) == 0.0
