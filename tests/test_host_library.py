"""Host-side logic of the CUDA library, checked without a GPU: exported
symbols, mesh building against the oracle, malformed meshes, renumbering
(bijection, neighbour remapping, locality) and the Sec. 4.1 diagnostics
against the oracle's by-definition implementations."""
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from paper_1408_5715_gb300 import binding as B
from paper_1408_5715_gb300 import build as BLD
from paper_1408_5715_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def built():
    BLD.build()


def header_functions():
    txt = open(os.path.join(ROOT, "include", "fv.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fv_\w+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = B.load()
    names = header_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    assert lib.fv_abi_version() == 1


def test_normal_build_refuses_the_debug_index_entry():
    # the test hook of the bounds-checked build answers FV_EINVAL in the
    # normal build, before any device work
    lib = B.load()
    assert lib.fv_index_checks() == 0
    m = B.Mesh.from_input(W.periodic_square(6, 4, seed=1), "f32")
    rc = lib.fv_mesh_debug_set_index(m._h, 0, 0, 0, 12345, None)
    assert rc == B.FV_EINVAL and "bounds-checked" in lib.fv_last_error().decode()


def test_oracle_is_not_linked_into_the_library():
    # the product library must not depend on the test oracle
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", B.library_path()], capture_output=True,
                         text=True).stdout
    assert "orc_" not in out


@pytest.mark.parametrize("kind", ["periodic", "channel", "strip", "two"])
def test_mesh_matches_oracle(orc, kind):
    mi = {"periodic": lambda: W.periodic_square(12, 10, seed=3),
          "channel": lambda: W.channel_bump(20, 9, seed=4),
          "strip": lambda: W.shock_tube_strip(15, 3, seed=5),
          "two": lambda: W.two_cells()}[kind]()
    m = B.Mesh.from_input(mi, "f64")
    nbr, nrm, area = m.export()
    om = orc.Mesh(mi.xy, mi.tri, mi.canon, mi.bnd, mi.default_bc)
    np.testing.assert_array_equal(nbr, om.nbr)
    np.testing.assert_array_equal(area, om.vol)
    # normals: identical except on periodic seams, where the library shares
    # one copy per face between both sides
    np.testing.assert_allclose(nrm, om.nrm, rtol=0, atol=1e-15)
    inner = nbr >= 0
    c, k = np.nonzero(inner)
    other = nbr[c, k]
    # each face's normal is exactly opposite to the one seen from across it
    back = np.array([np.nonzero(nbr[o] == cc)[0] for cc, o in zip(c, other)], dtype=object)
    for cc, kk, o, ks in zip(c, k, other, back):
        assert any((nrm[o, j] == -nrm[cc, kk]).all() for j in ks)


def test_malformed_meshes_are_rejected():
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0], [0.0, 1.0]])
    with pytest.raises(B.FVError, match="zero-area") as e:
        B.Mesh(xy, [[0, 1, 2]], default_bc=1)
    assert e.value.code == B.FV_EINVAL
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [0.0, -1.0], [1.0, 1.0]])
    with pytest.raises(B.FVError, match="more than two"):
        B.Mesh(xy, [[0, 1, 2], [0, 3, 1], [1, 0, 4]], default_bc=1)
    with pytest.raises(B.FVError, match="no boundary tag"):
        B.Mesh(xy[:3], [[0, 1, 2]], default_bc=0)
    with pytest.raises(B.FVError, match="out of range"):
        B.Mesh(xy[:3], [[0, 1, 7]], default_bc=1)
    with pytest.raises(B.FVError, match="collapsed"):
        B.Mesh(xy[:3], [[0, 1, 2]], canon=[0, 0, 2], default_bc=1)
    # clockwise input is reoriented
    m = B.Mesh(xy[:3], [[0, 2, 1]], default_bc=1)
    assert m.export()[2][0] == 0.5
    # empty mesh is valid
    e = B.Mesh(np.zeros((0, 2)), np.zeros((0, 3), np.int32))
    assert e.n == 0 and e.diagnostics() == (0, 0)


@pytest.mark.parametrize("order", ["identity", "shuffle", "rcm", "hilbert", "am1"])
def test_renumber_is_consistent_permutation(orc, order):
    mi = W.channel_bump(30, 12, seed=8)
    m = B.Mesh.from_input(mi, "f32")
    nbr0, nrm0, area0 = m.export()
    perm = m.renumber(order, seed=3)
    assert np.array_equal(np.sort(perm), np.arange(m.n))
    nbr1, nrm1, area1 = m.export()
    om = orc.Mesh.from_arrays(nbr0, nrm0, area0, np.zeros(4)).permuted(perm)
    np.testing.assert_array_equal(nbr1, om.nbr)
    np.testing.assert_array_equal(nrm1, om.nrm)
    np.testing.assert_array_equal(area1, om.vol)
    if order == "identity":
        assert np.array_equal(perm, np.arange(m.n))


def test_rcm_and_hilbert_improve_locality():
    mi = W.channel_bump(80, 30, seed=9)
    m = B.Mesh.from_input(mi, "f32")
    m.renumber("shuffle", seed=1)
    b_sh, s_sh = m.diagnostics()
    m.renumber("rcm")
    b_rcm, s_rcm = m.diagnostics()
    m.renumber("shuffle", seed=2)
    m.renumber("hilbert")
    b_h, s_h = m.diagnostics()
    assert b_rcm < b_sh / 20 and s_rcm < s_sh / 20
    # a structured 80x30 quad strip has a natural band of about 2*30 cells
    assert b_rcm <= 4 * 30
    # Hilbert order keeps consecutive cells close in space
    nbr, nrm, area = m.export()
    cen = None  # centroids are not exported; use the neighbour table instead
    inner = nbr >= 0
    gaps = np.abs(nbr - np.arange(m.n)[:, None])[inner]
    assert np.median(gaps) < 8


def test_rcm_on_a_path_has_bandwidth_one():
    # a strip of triangles one quad high and many long: its cell graph is a path
    nx = 50
    xy = np.array([[i, j] for j in range(2) for i in range(nx + 1)], np.float64)
    tri = []
    for i in range(nx):
        a, b, c, d = i, i + 1, nx + 2 + i, nx + 1 + i
        tri += [[a, b, c], [a, c, d]]
    m = B.Mesh(xy, tri, default_bc=1)
    m.renumber("shuffle", seed=4)
    m.renumber("rcm")
    assert m.diagnostics()[0] == 1


def test_diagnostics_match_definition(orc):
    rng = np.random.default_rng(5)
    for seed in range(6):
        mi = W.periodic_square(int(rng.integers(3, 9)), int(rng.integers(3, 6)), seed=seed)
        m = B.Mesh.from_input(mi, "f64")
        m.renumber(["shuffle", "rcm", "hilbert"][seed % 3], seed=seed)
        nbr, nrm, area = m.export()
        om = orc.Mesh.from_arrays(nbr, nrm, area, np.zeros(4))
        assert m.diagnostics() == (om.bandwidth(), om.serial_bandwidth())


def test_shuffle_is_seeded():
    mi = W.periodic_square(10, 10, seed=1)
    a = B.Mesh.from_input(mi).renumber("shuffle", seed=7)
    b = B.Mesh.from_input(mi).renumber("shuffle", seed=7)
    c = B.Mesh.from_input(mi).renumber("shuffle", seed=8)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_freestream_validation():
    m = B.Mesh.from_input(W.two_cells())
    with pytest.raises(B.FVError):
        m.set_freestream(-1.0, 0.0, 0.0, 1.0)
    m.set_freestream(1.0, 0.5, 0.0, 1.0)


def test_am1_matches_rcm_quality_on_degree_three_meshes():
    # Sec. 4.2: on the cell graphs of 2D triangulations (degree <= 3) AM1 gives
    # serial bandwidths close to GPS; here against RCM from the same kind of
    # pseudo-peripheral start
    for mi in (W.channel_bump(120, 40, seed=1), W.periodic_square(64, 40, seed=2)):
        m = B.Mesh.from_input(mi, "f32")
        m.renumber("shuffle", seed=3)
        b0, s0 = m.diagnostics()
        m.renumber("rcm")
        b_rcm, s_rcm = m.diagnostics()
        m.renumber("shuffle", seed=4)
        m.renumber("am1")
        b_am1, s_am1 = m.diagnostics()
        assert s_am1 < s0 / 10 and s_am1 <= 1.25 * s_rcm and b_am1 <= 1.25 * b_rcm


def test_am1_on_a_path_has_bandwidth_one():
    nx = 40
    xy = np.array([[i, j] for j in range(2) for i in range(nx + 1)], np.float64)
    tri = []
    for i in range(nx):
        a, b, c, d = i, i + 1, nx + 2 + i, nx + 1 + i
        tri += [[a, b, c], [a, c, d]]
    m = B.Mesh(xy, tri, default_bc=1)
    m.renumber("shuffle", seed=4)
    m.renumber("am1")
    assert m.diagnostics() == (1, 2)


@pytest.mark.parametrize("kind,order,tile", [("periodic", "hilbert", 512), ("channel", "hilbert", 1024),
                                             ("channel", "shuffle", 512), ("step", "rcm", 2048)])
def test_two_step_tile_halos_match_definition(kind, order, tile):
    # the halos of a tile: cells adjacent to the tile, then cells adjacent to
    # those (outside tile and first halo), by brute force over the neighbour table
    mi = {"periodic": lambda: W.periodic_square(60, 40, seed=2),
          "channel": lambda: W.channel_bump(60, 24, seed=3),
          "step": lambda: W.forward_step(10, 40, 8, 30, seed=4)}[kind]()
    m = B.Mesh.from_input(mi, "f32")
    m.renumber(order, seed=5)
    nbr, _, _ = m.export()
    n_tiles = (m.n + tile - 1) // tile
    for b in sorted({0, 1, n_tiles // 2, n_tiles - 1}):
        t0, t1 = b * tile, min((b + 1) * tile, m.n)
        inside = lambda x: (x >= t0) & (x < t1)  # noqa: E731
        nb = nbr[t0:t1].ravel()
        h1 = np.unique(nb[(nb >= 0) & ~inside(nb)])
        nb2 = nbr[h1].ravel()
        h2 = np.setdiff1d(np.unique(nb2[(nb2 >= 0) & ~inside(nb2)]), h1)
        g1, g2 = m.tile_halo(tile, b)
        np.testing.assert_array_equal(g1, h1)
        np.testing.assert_array_equal(g2, h2)
    with pytest.raises(B.FVError):
        m.tile_halo(tile, n_tiles)


def test_two_step_blocking_validation():
    m64 = B.Mesh.from_input(W.periodic_square(8, 8, seed=1), "f64")
    with pytest.raises(B.FVError, match="FV_F32"):
        m64.set_blocking(2)
    m64.set_blocking(1)
    m32 = B.Mesh.from_input(W.periodic_square(8, 8, seed=1), "f32")
    for bad in [(3, 0), (0, 0), (2, 100), (2, 4096), (2, 2048, True), (2, 768, True),
                (2, 672), (1, 16), (1, 4096)]:
        with pytest.raises(B.FVError):
            m32.set_blocking(*bad)
    m32.set_blocking(2, 512)
    m32.set_blocking(2, 1024, True)
    m32.set_blocking(2, 768)
    # one step per launch: the tile shape takes any size from 32 to 2048 cells
    m32.set_variant(6)
    for tile in (32, 672, 1344, 2048):
        m32.set_blocking(1, tile)
        assert m32.tiling() == (6, tile)
    m32.set_blocking(1, 0)
    assert m32.tiling() == (6, 1024)


def test_closure_engine_validation():
    # the engine is a host-side setting: both known engines are accepted on a
    # mesh that has never touched a device, anything else is FV_EINVAL
    m = B.Mesh.from_input(W.periodic_square(8, 8, seed=1), "f32")
    for engine in ("tcgen05", "mma.sync"):
        m.set_closure_engine(engine)
    for bad in (2, -1):
        rc = B.load().fv_mesh_set_closure_engine(m._h, bad)
        assert rc == B.FV_EINVAL and "engine" in B.load().fv_last_error().decode()


def test_tile_halo_limit_is_reported():
    # tile-local ids are 16 bits: a tile whose rings exceed 65533 cells (a
    # huge tile in a shuffled numbering) is refused, not wrapped
    mi = W.periodic_square(300, 200, seed=6)  # 120,000 cells
    m = B.Mesh.from_input(mi, "f32")
    m.renumber("shuffle", seed=2)
    with pytest.raises(B.FVError, match="65533") as e:
        m.tile_halo(40000, 0)
    assert e.value.code == B.FV_EINVAL
    m.renumber("hilbert")
    h1, h2 = m.tile_halo(40000, 0)  # a compact order keeps the same tile legal
    assert 0 < h1.size < 2000 and 0 < h2.size < 2000


# -- normals from vertex coordinates (fixed-point node grid) --------------------------------

def _vertex_case(kind):
    return {"periodic": lambda: W.periodic_square(12, 10, seed=3),
            "channel": lambda: W.channel_bump(20, 9, seed=4),
            "step": lambda: W.forward_step(4, 14, 3, 12, seed=6),
            "two": lambda: W.two_cells()}[kind]()


@pytest.mark.parametrize("kind", ["periodic", "channel", "step", "two"])
def test_vertex_grid_snaps_nodes_and_rebuilds_the_geometry(orc, kind):
    mi = _vertex_case(kind)
    m = B.Mesh.from_input(mi, "f32")
    xy0, e0 = m.nodes()
    assert e0 is None
    np.testing.assert_array_equal(xy0, mi.xy)
    m.set_geometry("vertex")
    xy, e = m.nodes()
    s = 2.0 ** e
    used = np.unique(mi.tri)
    q = xy[used] / s
    assert np.array_equal(q, np.round(q))  # grid points
    ext = max(np.ptp(mi.xy[used, 0]), np.ptp(mi.xy[used, 1]))
    assert ext / s <= 2**31 - 16 < 2 * ext / s  # the finest spacing that holds the extent
    assert np.abs(xy[used] - mi.xy[used]).max() <= s  # each node moves by at most one step
    # the library's geometry is now the snapped mesh's, as the oracle builds
    # it from the grid points by definition: normals exactly (integer edges
    # times a power of two), areas to the rounding of the cross product
    nbr, nrm, area = m.export()
    om = orc.Mesh(xy, mi.tri, mi.canon, mi.bnd, mi.default_bc)
    np.testing.assert_array_equal(nbr, om.nbr)
    np.testing.assert_array_equal(nrm, om.nrm)
    np.testing.assert_allclose(area, om.vol, rtol=2.0**-52, atol=0)
    # every interior face: the neighbour's face back has the exact opposite normal
    c, k = np.nonzero(nbr >= 0)
    d = nbr[c, k]
    back = np.zeros(c.size, bool)
    for k2 in range(3):
        back |= (nbr[d, k2] == c) & (nrm[d, k2] == -nrm[c, k]).all(-1)
    assert back.all()
    # a second call keeps the grid; going back to stored records keeps the nodes
    m.set_geometry("vertex")
    m.set_geometry("stored")
    xy2, e2 = m.nodes()
    assert e2 == e
    np.testing.assert_array_equal(xy2, xy)


def test_vertex_grid_keeps_periodic_offsets_after_renumbering(orc):
    mi = W.periodic_square(16, 12, seed=8)
    m = B.Mesh.from_input(mi, "f32")
    perm = m.renumber("hilbert")
    m.set_geometry("vertex")
    xy, e = m.nodes()
    # a copy sits a whole number of periods from its canonical node
    s = 2.0 ** e
    off = (xy - xy[mi.canon]) / s
    np.testing.assert_array_equal(off, np.round(off))
    nbr, nrm, area = m.export()
    om = orc.Mesh(xy, mi.tri, mi.canon, mi.bnd, mi.default_bc).permuted(perm)
    np.testing.assert_array_equal(nbr, om.nbr)
    np.testing.assert_array_equal(nrm, om.nrm)


def test_vertex_grid_refusals_leave_the_mesh_unchanged():
    with pytest.raises(B.FVError, match="FV_F32"):
        B.Mesh.from_input(W.two_cells(), "f64").set_geometry("vertex")
    # a sliver thinner than a grid step collapses on the grid
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, 1e-12], [0.5, -1.0]])
    tri = np.array([[0, 1, 2], [0, 3, 1]])
    m = B.Mesh(xy, tri, default_bc=B.FV_BC_WALL)
    before = m.export()
    with pytest.raises(B.FVError, match="collapses") as e:
        m.set_geometry("vertex")
    assert e.value.code == B.FV_EINVAL
    xy2, g = m.nodes()
    assert g is None
    np.testing.assert_array_equal(xy2, xy)
    for a, b in zip(m.export(), before):
        np.testing.assert_array_equal(a, b)
    # a periodic copy displaced across the seam by more than a grid step: the
    # stored records accept it (one normal per face), the grid cannot make
    # the two sides of its faces opposite
    mi = W.periodic_square(8, 6, seed=2)
    xy = mi.xy.copy()
    j = np.nonzero(mi.canon != np.arange(len(xy)))[0][3]
    xy[j, 1] += 1e-7
    m = B.Mesh(xy, mi.tri, mi.canon, mi.bnd, mi.default_bc)
    m.export()
    with pytest.raises(B.FVError, match="opposite"):
        m.set_geometry("vertex")
    assert m.nodes()[1] is None
    with pytest.raises(KeyError):
        m.set_geometry("faces")


@pytest.mark.parametrize("kind", ["periodic", "channel", "step"])
def test_vertex_tiles_stage_each_cells_nodes(kind):
    # the node lists the vertex-geometry tile kernel stages: every cell's
    # three counter-clockwise nodes sit at their grid points, each node once
    # per tile, every staged node used
    mi = _vertex_case(kind)
    m = B.Mesh.from_input(mi, "f32")
    with pytest.raises(B.FVError, match="vertex geometry"):
        m.tile_nodes(96, 0)
    perm = m.renumber("hilbert")
    m.set_geometry("vertex")
    xy, e = m.nodes()
    s = 2.0 ** e
    tri = mi.tri[perm].astype(np.int64)
    p0, p1, p2 = mi.xy[tri[:, 0]], mi.xy[tri[:, 1]], mi.xy[tri[:, 2]]
    cw = ((p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1])
          - (p2[:, 0] - p0[:, 0]) * (p1[:, 1] - p0[:, 1])) < 0
    tri[cw] = tri[cw][:, [0, 2, 1]]  # the library's counter-clockwise order
    n = m.n
    centre = None
    for tile_cells in (32, 96, 512):
        n_tiles = (n + tile_cells - 1) // tile_cells
        for t in sorted({0, n_tiles // 2, n_tiles - 1}):
            q, loc = m.tile_nodes(tile_cells, t)
            cells = tri[t * tile_cells:min((t + 1) * tile_cells, n)]
            assert loc.shape == cells.shape
            assert loc.max() < len(q) and set(np.unique(loc)) == set(range(len(q)))
            # one local id per node and one node per local id
            pairs = set(zip(cells.ravel().tolist(), loc.ravel().tolist()))
            assert len({a for a, _ in pairs}) == len(pairs) == len(q)
            c = xy[cells.ravel()] - q[loc.ravel()].astype(np.float64) * s
            if centre is None:
                centre = c[0]
                assert np.array_equal(centre / s, np.round(centre / s))
            np.testing.assert_array_equal(c, np.broadcast_to(centre, c.shape))
    with pytest.raises(B.FVError, match="out of range"):
        m.tile_nodes(512, (n + 511) // 512)
