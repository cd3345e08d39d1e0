"""GPU parity of the fused step kernels against the FP64 oracle, through the
C ABI.  Inputs are seeded and synthetic; the oracle builds its own mesh from
the same node/triangle arrays and never sees a value produced by the GPU.

Tolerances (written per test):
  FP64 path vs oracle: 1e-12 relative, max over cells and components, each
    component floored at 1e-3 of the largest magnitude of its quantity
    (density, momentum vector, energy) -- see conftest.rel_err_max;
  FP32 path: 1e-5 relative L2 error in density against the FP64 results.
"""
import math

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


def shuffled(mi, seed):
    """The same mesh with its triangle list shuffled (cell numbering by seed)."""
    p = np.random.default_rng(seed).permutation(mi.n_tri)
    return W.MeshInput(mi.xy, mi.tri[p], mi.canon, mi.bnd, mi.default_bc, dict(mi.info))


def pair(orc, mi, uinf_prim=(1.0, 0.0, 0.0, 1.0)):
    uinf = W.conserved(*uinf_prim)
    om = orc.Mesh(mi.xy, mi.tri, mi.canon, mi.bnd, mi.default_bc, uinf)
    g64 = B.Mesh.from_input(mi, "f64")
    g32 = B.Mesh.from_input(mi, "f32")
    for g in (g64, g32):
        g.set_freestream(*uinf_prim)
    return om, g64, g32


def dev(U, dtype):
    return torch.tensor(np.ascontiguousarray(U), dtype=dtype, device="cuda")


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def c1(orc):
    mi = shuffled(W.vortex_square_small(seed=1), seed=11)
    U0 = W.isentropic_vortex(mi.centroids(), mach=0.5, beta=5.0)
    return (mi, U0) + pair(orc, mi)


def test_c1_fp64_matches_oracle_100_steps(c1):
    mi, U0, om, g64, _ = c1
    Uo, to, steps, bad = om.run(U0, 100, 0.4)
    assert steps == 100 and not bad
    U = dev(U0, torch.float64)
    t = g64.step(U, 100, 0.4)
    assert t == pytest.approx(to, rel=1e-13)
    assert rel_err_max(U.cpu().numpy(), Uo) <= 1e-12


def test_c1_fp32_matches_fp64(c1):
    mi, U0, om, g64, g32 = c1
    U64 = dev(U0, torch.float64)
    U32 = dev(U0, torch.float32)
    g64.step(U64, 100, 0.4)
    g32.step(U32, 100, 0.4)
    a, b = U32.double().cpu().numpy(), U64.cpu().numpy()
    assert rel_l2(a[:, 0], b[:, 0]) <= 1e-5
    Uo, *_ = om.run(U0, 100, 0.4)
    assert rel_l2(a[:, 0], Uo[:, 0]) <= 1e-5


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_residual_dt_totals_match_oracle(orc, prec):
    mi = shuffled(W.channel_bump(37, 23, seed=5), seed=2)  # 1,702 cells: ragged last block
    uinf_prim = W.freestream(0.5)
    om, g64, g32 = pair(orc, mi, uinf_prim)
    g = g64 if prec == "f64" else g32
    dt_ = torch.float64 if prec == "f64" else torch.float32
    U0 = W.random_smooth_state(mi.centroids(), seed=4)
    U = dev(U0, dt_)
    R = g.residual(U).double().cpu().numpy()
    Ro = om.residual(U0 if prec == "f64" else U.double().cpu().numpy())
    tol = 1e-13 if prec == "f64" else 2e-5
    assert np.abs(R - Ro).max() <= tol * np.abs(Ro).max()
    dto = om.dt(U.double().cpu().numpy(), 0.4)
    assert g.compute_dt(U, 0.4) == pytest.approx(dto, rel=1e-14 if prec == "f64" else 1e-6)
    assert g.compute_dt(U, -2e-3) == 2e-3
    To = om.totals(U.double().cpu().numpy())
    scale = np.abs(U.double().cpu().numpy() * om.vol[:, None]).sum(axis=0)
    assert (np.abs(g.totals(U) - To) <= 1e-14 * scale).all()


def test_channel_walls_farfield_fp64_parity(orc):
    mi = shuffled(W.channel_bump(60, 25, seed=6), seed=3)
    uinf_prim = W.freestream(0.5)
    om, g64, g32 = pair(orc, mi, uinf_prim)
    U0 = W.uniform_state(mi.n_tri, uinf_prim)
    Uo, to, _, bad = om.run(U0, 150, 0.4)
    assert not bad
    U = dev(U0, torch.float64)
    t = g64.step(U, 150, 0.4)
    assert t == pytest.approx(to, rel=1e-13)
    assert rel_err_max(U.cpu().numpy(), Uo) <= 1e-12
    # the bump has disturbed the flow
    assert np.abs(Uo - U0).max() > 1e-3
    U32 = dev(U0, torch.float32)
    g32.step(U32, 150, 0.4)
    assert rel_l2(U32.double().cpu().numpy()[:, 0], Uo[:, 0]) <= 1e-5


def test_am1_ordered_channel_fp64_parity_on_every_shape(orc):
    # Amoeba1 (Sec. 4.2) renumbers the cells of a channel with walls and far
    # field; every kernel shape steps it and matches the oracle run on the
    # unpermuted mesh
    mi = shuffled(W.channel_bump(60, 25, seed=8), seed=5)
    uinf_prim = W.freestream(0.5)
    om, g64, _ = pair(orc, mi, uinf_prim)
    U0 = W.random_smooth_state(mi.centroids(), seed=3)
    Uo, to, _, bad = om.run(U0, 80, 0.4)
    assert not bad
    perm = g64.renumber("am1")
    assert sorted(perm) == list(range(mi.n_tri))
    bw, _ = g64.diagnostics()
    assert bw < mi.n_tri // 4  # a banded order, unlike the shuffled input
    for variant in range(8):
        g64.set_variant(variant)
        U = dev(U0[perm], torch.float64)
        t = g64.step(U, 80, 0.4)
        assert t == pytest.approx(to, rel=1e-13), variant
        assert rel_err_max(U.cpu().numpy(), Uo[perm]) <= 1e-12, variant


@pytest.mark.parametrize("scheme", ["fe", "rk2"])
def test_sod_strip_extrapolation_and_t_stop(orc, scheme):
    mi = shuffled(W.shock_tube_strip(120, 6, seed=7), seed=4)
    om, g64, _ = pair(orc, mi)
    U0 = W.sod_state(mi.centroids())
    Uo, to, steps, bad = om.run(U0, 10000, 0.4, t_stop=0.05, scheme=1 if scheme == "rk2" else 0)
    assert not bad and to == pytest.approx(0.05, rel=1e-14)
    U = dev(U0, torch.float64)
    t = g64.step(U, steps + 7, 0.4, t_stop=0.05, scheme=scheme)  # extra steps advance nothing
    assert t == pytest.approx(0.05, rel=1e-14)
    assert rel_err_max(U.cpu().numpy(), Uo) <= 1e-12


def test_rk2_fp64_matches_oracle(c1):
    mi, U0, om, g64, _ = c1
    Uo, to, _, _ = om.run(U0, 60, 0.4, scheme=1)
    U = dev(U0, torch.float64)
    t = g64.step(U, 60, 0.4, scheme="rk2")
    assert t == pytest.approx(to, rel=1e-13)
    assert rel_err_max(U.cpu().numpy(), Uo) <= 1e-12


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_split_calls_equal_one_call(c1, prec):
    # 197 steps in one call (two captured graphs + a remainder, odd count)
    # equal 96 + 1 + 100 steps in three calls, bit for bit; the compensated
    # FP32 update carries its remainder across the calls in a caller buffer
    mi, U0, om, g64, g32 = c1
    g = g64 if prec == "f64" else B.Mesh.from_input(mi, "f32")
    dt_ = torch.float64 if prec == "f64" else torch.float32
    A = dev(U0, dt_)
    Bt = dev(U0, dt_)
    ta = g.step(A, 197, 0.4)
    if prec == "f32":
        lo = torch.zeros((mi.n_tri, 4), dtype=torch.int16, device="cuda")
        g.set_remainder(lo)
    tb = g.step(Bt, 96, 0.4) + g.step(Bt, 1, 0.4) + g.step(Bt, 100, 0.4)
    assert torch.equal(A, Bt)
    assert ta == pytest.approx(tb, rel=1e-12)
    if prec == "f32":
        assert lo.abs().sum() > 0  # the remainder is carried, not zero
        # without the caller's remainder every call starts from zero again
        g.set_remainder(None)
        C = dev(U0, dt_)
        for k in (96, 1, 100):
            g.step(C, k, 0.4)
        assert not torch.equal(A, C)


def _resumed_mesh(mi, blocking):
    g = B.Mesh.from_input(mi, "f32")
    perm = g.renumber("hilbert")
    if blocking == 2:
        g.set_blocking(2, 512)
    return g, perm


@pytest.mark.parametrize("blocking,scheme", [(1, "fe"), (1, "rk2"), (2, "fe")])
def test_checkpoint_and_resume_is_bitwise(c1, tmp_path, blocking, scheme):
    # one call of 206 steps against three calls (103, 50, 53 steps), the
    # state and the compensated update's remainder saved to files after the
    # first and loaded into a new mesh and new buffers.  With two steps per
    # launch 103 and 50 end on an odd number of pair launches (the remainder
    # then sits in the second buffer) and 103 and 53 end with a single step.
    mi, U0, *_ = c1
    g, perm = _resumed_mesh(mi, blocking)
    A = dev(U0[perm], torch.float32)
    # two steps per launch take one CFL dt per pair, so calls of odd length
    # pair other steps than one call does; a fixed dt makes pairs bitwise
    # two single steps
    cfl = 0.4 if blocking == 1 else -0.5 * g.compute_dt(A, 0.4)
    ta = g.step(A, 206, cfl, scheme=scheme)
    g1, _ = _resumed_mesh(mi, blocking)
    Bt = dev(U0[perm], torch.float32)
    lo = torch.zeros((mi.n_tri, 4), dtype=torch.int16, device="cuda")
    g1.set_remainder(lo)
    tb = g1.step(Bt, 103, cfl, scheme=scheme)
    np.save(tmp_path / "U.npy", Bt.cpu().numpy())
    np.save(tmp_path / "lo.npy", lo.cpu().numpy())
    del g1, Bt, lo
    g2, _ = _resumed_mesh(mi, blocking)
    Bt = torch.tensor(np.load(tmp_path / "U.npy"), device="cuda")
    lo = torch.tensor(np.load(tmp_path / "lo.npy"), device="cuda")
    g2.set_remainder(lo)
    tb += g2.step(Bt, 50, cfl, scheme=scheme) + g2.step(Bt, 53, cfl, scheme=scheme)
    assert torch.equal(A, Bt)
    assert ta == pytest.approx(tb, rel=1e-12)


def test_remainder_refused_for_fp64(c1):
    mi, *_ = c1
    g = B.Mesh.from_input(mi, "f64")
    with pytest.raises(B.FVError):
        g.set_remainder(torch.zeros((mi.n_tri, 4), dtype=torch.int16, device="cuda"))
    g.set_remainder(None)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("order", ["rcm", "hilbert", "shuffle", "am1"])
def test_renumbering_leaves_results_unchanged(c1, prec, order):
    mi, U0, om, g64, g32 = c1
    dt_ = torch.float64 if prec == "f64" else torch.float32
    ref = B.Mesh.from_input(mi, prec)
    ren = B.Mesh.from_input(mi, prec)
    perm = ren.renumber(order, seed=9)
    A = dev(U0, dt_)
    Bt = dev(U0[perm], dt_)
    ta = ref.step(A, 120, 0.4)
    tb = ren.step(Bt, 120, 0.4)
    assert ta == tb
    assert torch.equal(Bt, A[torch.as_tensor(perm, device="cuda", dtype=torch.long)])


@pytest.mark.parametrize("scheme", ["fe", "rk2"])
def test_compensated_fp32_tracks_fp64_over_long_runs(scheme):
    # increments below half a float ulp of the state are lost by a plain float
    # update; the bfloat16 remainder keeps them
    mi = W.channel_bump(250, 80, seed=2)
    uinf_prim = W.freestream(0.5)
    U0 = W.uniform_state(mi.n_tri, uinf_prim)
    res = {}
    for prec, comp in (("f64", None), ("f32", True), ("f32", False)):
        g = B.Mesh.from_input(mi, prec)
        g.set_freestream(*uinf_prim)
        g.renumber("rcm")
        if comp is not None:
            g.set_compensation(comp)
        U = dev(U0, torch.float64 if prec == "f64" else torch.float32)
        g.step(U, 4000, 0.4, scheme=scheme)
        res[(prec, comp)] = U.double().cpu().numpy()[:, 0]
    ref = res[("f64", None)]
    e_comp = rel_l2(res[("f32", True)], ref)
    e_plain = rel_l2(res[("f32", False)], ref)
    assert e_comp <= 2e-7, e_comp
    assert e_plain > 10 * e_comp, (e_plain, e_comp)


@pytest.fixture(scope="module")
def big_square():
    # 240,000 cells: more than two sweeps of every persistent grid
    mi = W.periodic_square(400, 300, seed=31)
    return mi, W.isentropic_vortex(mi.centroids(), mach=0.6)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("scheme", ["fe", "rk2"])
def test_kernel_shapes_give_identical_results(big_square, prec, scheme):
    mi, U0 = big_square
    dt_ = torch.float64 if prec == "f64" else torch.float32
    outs, ts = [], []
    shapes = [(v, 1024) for v in range(B.N_VARIANTS)] + [(6, 512), (6, 2048), (7, 512)]
    for v, tile in shapes:
        g = B.Mesh.from_input(mi, prec)
        g.renumber("hilbert")
        g.set_variant(v)
        if v in (6, 7):
            g.set_blocking(1, tile)  # tile size of the shared-memory shapes
        U = dev(U0, dt_)
        ts.append(g.step(U, 30, 0.4, scheme=scheme))
        outs.append(U)
        g.close()
    for k in range(1, len(shapes)):
        assert ts[k] == ts[0]
        assert torch.equal(outs[k], outs[0]), shapes[k]


def test_autotune_picks_a_shape_and_leaves_state(big_square):
    mi, U0 = big_square
    g = B.Mesh.from_input(mi, "f32")
    U = dev(U0, torch.float32)
    before = U.clone()
    best, us = g.autotune(U)
    n = B.N_VARIANTS
    assert 0 <= best < n and len(us) == n and all(x > 0 for x in us)
    assert us[best] == min(us)
    assert torch.equal(U, before)
    with pytest.raises(B.FVError):
        g.set_variant(n)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_bounded_wait_gives_timeout_not_a_hang(big_square, prec):
    # the TMA-staged shape waits for its bulk copies on mbarriers with a poll
    # limit; a limit of 0 makes every wait give up at once: the kernel drains
    # its own copies, sets the timeout bit and returns, and the call reports
    # FV_ETIMEOUT
    mi, U0 = big_square
    dt_ = torch.float64 if prec == "f64" else torch.float32
    g = B.Mesh.from_input(mi, prec)
    g.set_variant(5)
    g.set_wait_limit(0)
    U = dev(U0, dt_)
    with pytest.raises(B.FVError) as e:
        g.step(U, 3, 0.4)
    assert e.value.code == B.FV_ETIMEOUT
    # the mesh and the device stay usable
    g.set_wait_limit(1 << 24)
    V = dev(U0, dt_)
    ref = B.Mesh.from_input(mi, prec)
    W_ = dev(U0, dt_)
    assert g.step(V, 5, 0.4) == ref.step(W_, 5, 0.4)
    assert torch.equal(V, W_)


def test_conservation_and_free_stream_on_gpu(c1):
    mi, U0, om, g64, g32 = c1
    U = dev(U0, torch.float64)
    T0 = g64.totals(U)
    g64.step(U, 300, 0.4)
    T1 = g64.totals(U)
    scale = np.abs(U0 * om.vol[:, None]).sum(axis=0)
    assert (np.abs(T1 - T0) <= 1e-12 * scale).all()
    prim0 = W.freestream(0.5, angle=0.3)
    Uf0 = W.uniform_state(mi.n_tri, prim0)
    Uf = dev(Uf0, torch.float64)
    g64.step(Uf, 300, 0.4)
    assert np.abs(Uf.cpu().numpy() - Uf0).max() <= 1e-13


def test_bad_state_is_reported(c1):
    mi, U0, om, g64, g32 = c1
    Ubad = U0.copy()
    Ubad[17, 3] = 0.1 * 0.5 * (Ubad[17, 1] ** 2 + Ubad[17, 2] ** 2) / Ubad[17, 0]  # p < 0
    for g, dt_ in ((g64, torch.float64), (g32, torch.float32)):
        U = dev(Ubad, dt_)
        with pytest.raises(B.FVError) as e:
            g.step(U, 3, 0.4)
        assert e.value.code == B.FV_ENONFINITE
        # the mesh stays usable afterwards
        V = dev(U0, dt_)
        assert g.step(V, 2, 0.4) > 0


def test_small_and_degenerate_sizes(orc):
    # one triangle with three wall faces stays at rest; empty mesh is a no-op
    mi = W.MeshInput(np.array([[0.0, 0.0], [1.0, 0.2], [0.3, 0.9]]), np.array([[0, 1, 2]], np.int32),
                     default_bc=W.TAG_WALL)
    om, g64, g32 = pair(orc, mi)
    U0 = W.uniform_state(1, (1.0, 0.0, 0.0, 1.0))
    for g, dt_ in ((g64, torch.float64), (g32, torch.float32)):
        U = dev(U0, dt_)
        g.step(U, 5, 0.4)
        # wall pressure forces cancel up to rounding of the three normals
        np.testing.assert_allclose(U.double().cpu().numpy(), U0, rtol=1e-6, atol=1e-12)
    e = B.Mesh(np.zeros((0, 2)), np.zeros((0, 3), np.int32), precision="f64")
    Z = torch.zeros((0, 4), dtype=torch.float64, device="cuda")
    assert e.step(Z, 10, 0.4) == 0.0
    assert (e.totals(Z) == 0).all()


def test_fixed_dt_mode(c1):
    mi, U0, om, g64, _ = c1
    Uo, to, _, _ = om.run(U0, 20, -1e-3)
    U = dev(U0, torch.float64)
    assert g64.step(U, 20, -1e-3) == pytest.approx(to, rel=1e-14)
    assert rel_err_max(U.cpu().numpy(), Uo) <= 1e-12


# ---------------------------------------------------------------------------
# full sizes, in the launch configuration of the benchmark (captured graphs)
# ---------------------------------------------------------------------------
def test_channel_1m_fp64_and_fp32_vs_oracle(orc):
    mi = shuffled(W.channel_bump_1m(), seed=12)
    uinf_prim = W.freestream(0.5)
    om, g64, g32 = pair(orc, mi, uinf_prim)
    g64.renumber("rcm")
    perm = g32.renumber("rcm")
    g64b = g64
    U0 = W.uniform_state(mi.n_tri, uinf_prim)
    Uo, to, _, bad = om.run(U0, 100, 0.4)
    assert not bad
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    U = dev(U0[perm], torch.float64)
    t = g64b.step(U, 100, 0.4)
    assert t == pytest.approx(to, rel=1e-13)
    assert rel_err_max(U.cpu().numpy()[inv], Uo) <= 1e-12
    U32 = dev(U0[perm], torch.float32)
    g32.step(U32, 100, 0.4)
    assert rel_l2(U32.double().cpu().numpy()[inv][:, 0], Uo[:, 0]) <= 1e-5


def test_square_16m_one_step_vs_oracle_and_invariants(orc):
    mi = W.vortex_square_16m()
    om = orc.Mesh(mi.xy, mi.tri, mi.canon, None, 0)
    U0 = W.isentropic_vortex(mi.centroids(), mach=0.5)
    Uo, to, _, _ = om.run(U0, 2, 0.4)
    for prec, dt_ in (("f64", torch.float64), ("f32", torch.float32)):
        g = B.Mesh.from_input(mi, prec)
        perm = g.renumber("hilbert")
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)
        U = dev(U0[perm], dt_)
        t = g.step(U, 2, 0.4)
        got = U.double().cpu().numpy()[inv]
        if prec == "f64":
            assert t == pytest.approx(to, rel=1e-13)
            assert rel_err_max(got, Uo) <= 1e-12
        else:
            assert rel_l2(got[:, 0], Uo[:, 0]) <= 1e-6
        # 192 more steps through the captured graphs: conservation holds
        T0 = g.totals(U)
        g.step(U, 192, 0.4)
        T1 = g.totals(U)
        scale = np.abs(U0 * om.vol[:, None]).sum(axis=0)
        tol = 1e-12 if prec == "f64" else 1e-5
        assert (np.abs(T1 - T0) <= tol * scale).all()
        del U
        g.close()


def test_tile_shape_residual_and_boundaries_match_oracle(orc):
    # the shared-memory shape on a mesh with walls and far field, FP64 against
    # the oracle, and its residual (through fv_residual, shape-independent)
    mi = W.channel_bump(60, 24, seed=12)
    prim = W.freestream(0.6)
    om = orc.Mesh(mi.xy, mi.tri, mi.canon, mi.bnd, mi.default_bc, W.conserved(*prim))
    U0 = W.random_smooth_state(mi.centroids(), seed=13)
    g = B.Mesh.from_input(mi, "f64")
    g.set_freestream(*prim)
    perm = g.renumber("hilbert")
    g.set_variant(6)
    g.set_blocking(1, 512)
    Uo, to, _, bad = om.run(U0, 60, 0.4)
    assert not bad
    U = dev(U0[perm], torch.float64)
    assert g.step(U, 60, 0.4) == pytest.approx(to, rel=1e-13)
    out = np.empty_like(Uo)
    out[perm] = U.cpu().numpy()
    assert rel_err_max(out, Uo) <= 1e-12


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_launch_chaining_leaves_results_unchanged(big_square, prec):
    # programmatic dependent launch only moves when the next step's blocks are
    # scheduled; they wait for the previous step in hardware before reading
    mi, U0 = big_square
    dt_ = torch.float64 if prec == "f64" else torch.float32
    for v in (0, 1, 3, 6):
        outs = []
        for chained in (True, False):
            g = B.Mesh.from_input(mi, prec)
            g.renumber("hilbert")
            g.set_variant(v)
            g.set_launch_chaining(chained)
            U = dev(U0, dt_)
            t = g.step(U, 101, 0.4)  # a graph of 96 steps and 5 direct launches
            outs.append((t, U))
            g.close()
        assert outs[0][0] == outs[1][0]
        assert torch.equal(outs[0][1], outs[1][1]), v



@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_max_wave_speed_matches_oracle_on_all_shapes(orc, prec):
    # the Rusanov wave speed on the Mach 3 step (far-field inflow,
    # extrapolation outflow, slip walls), 200 steps: FP64 against the oracle
    # with the same reading, every shape bitwise the same, FP32 close to FP64
    mi = W.forward_step(12, 42, 9, 36, seed=6)
    prim = W.mach3_inflow()
    U0 = W.uniform_state(mi.n_tri, prim)
    outs = []
    for v in (0, 1, 3, 6):
        g = B.Mesh.from_input(mi, prec)
        g.set_freestream(*prim)
        perm = g.renumber("hilbert")
        g.set_wave_speed("max")
        g.set_variant(v)
        U = dev(U0[perm], torch.float64 if prec == "f64" else torch.float32)
        t = g.step(U, 200, 0.4)
        out = np.empty_like(U0)
        out[perm] = U.double().cpu().numpy()
        outs.append((t, out))
        g.close()
    for t, out in outs[1:]:
        assert t == outs[0][0]
        assert np.array_equal(out, outs[0][1])
    orc.set_wave_speed("max")
    try:
        om = orc.Mesh(mi.xy, mi.tri, mi.canon, mi.bnd, mi.default_bc, W.conserved(*prim))
        Uo, to, _, bad = om.run(U0, 200, 0.4)
    finally:
        orc.set_wave_speed("average")
    assert not bad
    if prec == "f64":
        assert outs[0][0] == pytest.approx(to, rel=1e-13)
        assert rel_err_max(outs[0][1], Uo) <= 1e-12
    else:
        assert rel_l2(outs[0][1][:, 0], Uo[:, 0]) <= 1e-5


def test_max_wave_speed_refuses_closure_and_pairs():
    mi = W.periodic_square(16, 8, seed=2)
    g = B.Mesh.from_input(mi, "f32")
    g.set_wave_speed("max")
    U = dev(W.uniform_state(mi.n_tri, (1.0, 0.3, 0.0, 1.0)), torch.float32)
    g.set_blocking(2)
    with pytest.raises(B.FVError, match="wave"):
        g.step(U, 2, 0.4)
    g.set_blocking(1)
    g.step(U, 2, 0.4)
    with pytest.raises(B.FVError):
        B.Batch([g])
