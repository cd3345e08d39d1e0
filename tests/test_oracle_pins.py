"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a value
worked out by hand from Eq. 5 / Eq. 7, a closed form, an invariant of the
discrete scheme (conservation, free-stream preservation, antisymmetry,
rotation and permutation invariance), the exact Riemann solution, or brute
force on tiny inputs.  No GPU is needed.
"""
import math

import numpy as np
import pytest

from conftest import read_golden
from exact_riemann import sample, star_state
from paper_1408_5715_gb300 import workloads as W

G = 1.4


def prim(U):
    U = np.asarray(U, np.float64)
    rho = U[..., 0]
    u = U[..., 1] / rho
    v = U[..., 2] / rho
    p = (G - 1.0) * (U[..., 3] - 0.5 * rho * (u * u + v * v))
    return rho, u, v, p


def build(orc, mi, uinf=(1.0, 0.0, 0.0, 2.5)):
    return orc.Mesh(mi.xy, mi.tri, mi.canon, mi.bnd, mi.default_bc, uinf)


def random_state(rng, n=None):
    shape = () if n is None else (n,)
    rho = rng.uniform(0.3, 2.0, shape)
    u = rng.uniform(-1.0, 1.0, shape)
    v = rng.uniform(-1.0, 1.0, shape)
    p = rng.uniform(0.2, 2.0, shape)
    return W.conserved(rho, u, v, p)


# ---------------------------------------------------------------------------
# single-face flux
# ---------------------------------------------------------------------------
def test_two_cell_flux_matches_hand_computation(orc):
    g = read_golden("two_cell_flux.txt")
    mi = W.two_cells()
    mesh = build(orc, mi)
    # L is cell 0; its face 2 runs (1,1)->(0,0) and borders R
    assert mesh.nbr[0, 2] == 1 and mesh.nbr[1, 0] == 0
    np.testing.assert_array_equal(mesh.nrm[0, 2], [-1.0, 1.0])
    UL = np.array([1.0, 0.0, 0.0, 2.5])
    UR = np.array([0.125, 0.0, 0.0, 0.25])
    F = orc.face_flux(UL, UR, mesh.nrm[0, 2])
    want = [g["F_rho"], g["F_rhou"], g["F_rhov"], g["F_E"]]
    np.testing.assert_allclose(F, want, rtol=1e-14, atol=1e-15)
    # seen from R the same face carries exactly the opposite flux
    FR = orc.face_flux(UR, UL, mesh.nrm[1, 0])
    np.testing.assert_array_equal(mesh.nrm[1, 0], -mesh.nrm[0, 2])
    np.testing.assert_array_equal(FR, -F)
    # dt bound of L, reading R1
    assert orc.cell_dt_bound(UL, mesh.nrm[0], mesh.vol[0]) == pytest.approx(
        g["dt_over_cfl_L"], rel=1e-14)


def test_flux_antisymmetric_bitwise(orc):
    rng = np.random.default_rng(7)
    for _ in range(200):
        UL, UR = random_state(rng), random_state(rng)
        n = rng.normal(size=2)
        s = rng.uniform(0.2, 1.5)
        np.testing.assert_array_equal(orc.face_flux(UL, UR, n, s), -orc.face_flux(UR, UL, -n, s))


def test_flux_of_equal_states_is_physical_flux(orc):
    # U_L = U_R: the dissipation vanishes and F = |n| F(U).n-hat, written here in
    # x-y components without the face-frame rotation.
    rng = np.random.default_rng(8)
    for _ in range(100):
        U = random_state(rng)
        rho, u, v, p = prim(U)
        n = rng.normal(size=2)
        q = u * n[0] + v * n[1]
        want = [rho * q, rho * u * q + p * n[0], rho * v * q + p * n[1], (U[3] + p) * q]
        np.testing.assert_allclose(orc.face_flux(U, U, n), want, rtol=1e-13, atol=1e-13)


def test_flux_dissipation_is_linear_in_jump(orc):
    # F(s) = central part - s/2 |n| (|u-bar| + c-bar) (U_R - U_L)   (Eq. 5)
    rng = np.random.default_rng(9)
    for _ in range(50):
        UL, UR = random_state(rng), random_state(rng)
        n = rng.normal(size=2)
        _, uL, vL, pL = prim(UL)
        _, uR, vR, pR = prim(UR)
        ln = math.hypot(*n)
        nh = n / ln
        a = abs(0.5 * ((uL * nh[0] + vL * nh[1]) + (uR * nh[0] + vR * nh[1]))) + 0.5 * (
            math.sqrt(G * pL / UL[0]) + math.sqrt(G * pR / UR[0]))
        d = orc.face_flux(UL, UR, n, 1.0) - orc.face_flux(UL, UR, n, 0.0)
        np.testing.assert_allclose(d, -0.5 * ln * a * (UR - UL), rtol=1e-12, atol=1e-13)


def test_wall_ghost_closed_form(orc):
    # slip wall: no mass or energy crosses; momentum flux is normal,
    # |n| (rho u_n^2 + p + c rho u_n) n-hat
    rng = np.random.default_rng(10)
    for _ in range(50):
        U = random_state(rng)
        rho, u, v, p = prim(U)
        n = rng.normal(size=2)
        ln = math.hypot(*n)
        nh = n / ln
        UR = orc.ghost(orc.WALL, U, n, np.zeros(4))
        F = orc.face_flux(U, UR, n)
        un = u * nh[0] + v * nh[1]
        c = math.sqrt(G * p / rho)
        m = ln * (rho * un * un + p + c * rho * un)
        assert abs(F[0]) < 1e-14 * ln * rho and abs(F[3]) < 1e-13 * ln * U[3]
        np.testing.assert_allclose(F[1:3], m * nh, rtol=1e-12, atol=1e-13)
        # the ghost keeps density, energy and tangential momentum
        assert UR[0] == U[0] and UR[3] == U[3]
        assert UR[1] * -nh[1] + UR[2] * nh[0] == pytest.approx(U[1] * -nh[1] + U[2] * nh[0])
    uinf = np.array([1.0, 0.5, 0.1, 2.7])
    np.testing.assert_array_equal(orc.ghost(orc.FARFIELD, U, n, uinf), uinf)
    np.testing.assert_array_equal(orc.ghost(orc.EXTRAP, U, n, uinf), U)


# ---------------------------------------------------------------------------
# mesh geometry
# ---------------------------------------------------------------------------
def _brute_neighbours(mi):
    canon = mi.canon if mi.canon is not None else np.arange(mi.xy.shape[0])
    keys = {}
    for c, t in enumerate(mi.tri):
        for k in range(3):
            a, b = canon[t[k]], canon[t[(k + 1) % 3]]
            keys.setdefault(frozenset((a, b)), []).append(c)
    return keys, canon


@pytest.mark.parametrize("kind", ["periodic", "channel", "strip"])
def test_mesh_geometry_brute_force(orc, kind):
    mi = {"periodic": lambda: W.periodic_square(6, 4, seed=3),
          "channel": lambda: W.channel_bump(8, 5, seed=4),
          "strip": lambda: W.shock_tube_strip(7, 3, seed=5)}[kind]()
    mesh = build(orc, mi)
    keys, canon = _brute_neighbours(mi)
    tags = {}
    if mi.bnd is not None:
        for a, b, t in mi.bnd:
            tags[frozenset((canon[a], canon[b]))] = t
    for c in range(mi.n_tri):
        P = mi.xy[mi.tri[c]]
        area = 0.5 * abs((P[1, 0] - P[0, 0]) * (P[2, 1] - P[0, 1])
                         - (P[2, 0] - P[0, 0]) * (P[1, 1] - P[0, 1]))
        assert mesh.vol[c] == pytest.approx(area, rel=1e-14)
        cen = P.mean(axis=0)
        np.testing.assert_allclose(mesh.nrm[c].sum(axis=0), 0.0, atol=1e-15)
        edges = set()
        for k in range(3):
            n = mesh.nrm[c, k]
            # the face of n: the vertex pair whose edge is normal to n, of equal length
            found = None
            for i in range(3):
                a, b = i, (i + 1) % 3
                d = P[b] - P[a]
                if abs(d @ n) < 1e-12 and abs(math.hypot(*d) - math.hypot(*n)) < 1e-12:
                    mid = 0.5 * (P[a] + P[b])
                    if (mid - cen) @ n > 0:  # outward
                        found = frozenset((canon[mi.tri[c, a]], canon[mi.tri[c, b]]))
            assert found is not None
            edges.add(found)
            others = [x for x in keys[found] if x != c]
            if others:
                assert mesh.nbr[c, k] == others[0]
            else:
                assert mesh.nbr[c, k] == -tags[found]
        assert len(edges) == 3


def test_mesh_errors(orc):
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0], [0.0, 1.0]])
    with pytest.raises(ValueError, match="degenerate"):
        orc.Mesh(xy, np.array([[0, 1, 2]]), default_bc=1)
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [0.0, -1.0], [1.0, 1.0]])
    tri = np.array([[0, 1, 2], [0, 3, 1], [1, 0, 4]])
    with pytest.raises(ValueError, match="non-manifold"):
        orc.Mesh(xy, tri, default_bc=1)
    with pytest.raises(ValueError, match="open edge"):
        orc.Mesh(xy[:3], np.array([[0, 1, 2]]), default_bc=0)
    # a clockwise triangle is reoriented, not rejected
    m = orc.Mesh(xy[:3], np.array([[0, 2, 1]]), default_bc=1)
    assert m.vol[0] == 0.5


# ---------------------------------------------------------------------------
# whole-scheme invariants
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def c1(orc):
    mi = W.vortex_square_small(seed=1)
    return mi, build(orc, mi)


def test_free_stream_preserved_periodic(orc, c1):
    mi, mesh = c1
    prim0 = W.freestream(0.5, angle=0.3)
    U0 = W.uniform_state(mi.n_tri, prim0)
    U, t, steps, bad = mesh.run(U0, 100, 0.4)
    assert steps == 100 and not bad and t > 0
    assert np.abs(U - U0).max() <= 1e-13


def test_free_stream_preserved_farfield_box(orc):
    mi = W.periodic_square(16, 16, seed=5)
    prim0 = W.freestream(0.7, angle=-0.4)
    uinf = W.conserved(*prim0)
    # the same lattice with open sides: all boundary faces far field
    mesh = orc.Mesh(mi.xy, mi.tri, None, None, W.TAG_FARFIELD, uinf)
    assert (mesh.nbr == orc.FARFIELD).sum() == 2 * 16 * 2
    U0 = W.uniform_state(mi.n_tri, prim0)
    U, _, _, bad = mesh.run(U0, 100, 0.4)
    assert not bad and np.abs(U - U0).max() <= 1e-13


def _conservation_error(mesh, U0, U1):
    T0, T1 = mesh.totals(U0), mesh.totals(U1)
    scale = np.abs(U0 * mesh.vol[:, None]).sum(axis=0)
    return np.abs(T1 - T0) / scale


def test_conservation_periodic(orc, c1):
    mi, mesh = c1
    U0 = W.isentropic_vortex(mi.centroids(), mach=0.5)
    U, _, steps, bad = mesh.run(U0, 100, 0.4)
    assert steps == 100 and not bad
    assert _conservation_error(mesh, U0, U).max() <= 1e-12
    # the vortex has moved: the state did change
    assert np.abs(U - U0).max() > 1e-3


def test_permutation_invariance(orc, c1):
    mi, mesh = c1
    U0 = W.isentropic_vortex(mi.centroids(), mach=0.5)
    perm = np.random.default_rng(11).permutation(mi.n_tri)
    pm = mesh.permuted(perm)
    Ua, ta, _, _ = mesh.run(U0, 30, 0.4)
    Ub, tb, _, _ = pm.run(U0[perm], 30, 0.4)
    assert ta == tb
    np.testing.assert_array_equal(Ub, Ua[perm])
    # only the summation order of the totals differs
    scale = np.abs(Ua * mesh.vol[:, None]).sum(axis=0)
    assert (np.abs(pm.totals(Ub) - mesh.totals(Ua)) <= 1e-14 * scale).all()


def test_rotation_invariance(orc):
    # rotating the mesh and the flow by theta rotates the momentum residual and
    # leaves the density and energy residuals unchanged
    mi = W.channel_bump(24, 10, seed=6)
    th = 0.7
    Rm = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    U = W.random_smooth_state(mi.centroids(), seed=3)
    uinf = W.conserved(*W.freestream(0.5))
    m0 = build(orc, mi, uinf)
    uinf_r = uinf.copy()
    uinf_r[1:3] = Rm @ uinf[1:3]
    m1 = orc.Mesh(mi.xy @ Rm.T, mi.tri, None, mi.bnd, 0, uinf_r)
    Ur = U.copy()
    Ur[:, 1:3] = U[:, 1:3] @ Rm.T
    R0, R1 = m0.residual(U), m1.residual(Ur)
    scale = np.abs(R0).max(axis=0)
    np.testing.assert_allclose(R1[:, 0], R0[:, 0], atol=1e-12 * scale[0])
    np.testing.assert_allclose(R1[:, 3], R0[:, 3], atol=1e-12 * scale[3])
    np.testing.assert_allclose(R1[:, 1:3], R0[:, 1:3] @ Rm.T, atol=1e-12 * scale[1:3].max())


@pytest.fixture
def max_wave(orc):
    orc.set_wave_speed("max")
    try:
        yield orc
    finally:
        orc.set_wave_speed("average")


def test_max_wave_speed_two_cell_flux_by_hand(max_wave):
    # the two-cell case of the averaged pin with the one-sided maximum:
    # both cells are at rest, so the wave speed is max(c_L, c_R) = sqrt(1.4);
    # |n| = sqrt(2), jumps rho: -0.875, E: -2.25; pressure flux 1.1/2 n
    orc = max_wave
    UL = np.array([1.0, 0.0, 0.0, 2.5])
    UR = np.array([0.125, 0.0, 0.0, 0.25])
    F = orc.face_flux(UL, UR, np.array([-1.0, 1.0]))
    a_n = math.sqrt(1.4) * math.sqrt(2.0)
    expect = [0.5 * a_n * 0.875, -0.55, 0.55, 0.5 * a_n * 2.25]
    np.testing.assert_allclose(F, expect, rtol=1e-15, atol=1e-15)
    # swapped cells and normal: the exact negation
    G_ = orc.face_flux(UR, UL, np.array([1.0, -1.0]))
    assert np.array_equal(G_, -F)


def test_max_wave_speed_at_least_the_average(orc):
    # the dissipation coefficient of the maximum form is never below the
    # averaged one (|a + b| / 2 + (c + d) / 2 <= max(|a| + c, |b| + d))
    rng = np.random.default_rng(21)
    for _ in range(200):
        UL, UR = random_state(rng), random_state(rng)
        n = rng.normal(size=2)
        orc.set_wave_speed("average")
        Fa0 = orc.face_flux(UL, UR, n, scale=0.0)
        Fa1 = orc.face_flux(UL, UR, n)
        orc.set_wave_speed("max")
        try:
            Fm1 = orc.face_flux(UL, UR, n)
        finally:
            orc.set_wave_speed("average")
        jump = UR[0] - UL[0]
        if abs(jump) > 1e-3:
            da = (Fa1[0] - Fa0[0]) / -jump  # = |n| a_avg / 2
            dm = (Fm1[0] - Fa0[0]) / -jump  # = |n| a_max / 2
            assert dm >= da * (1 - 1e-12)


def test_double_rarefaction_positivity(orc):
    # two halves of a strip moving apart at twice the sound speed: the exact
    # solution keeps a positive pressure (no vacuum below 2 c / (gamma - 1)
    # = 5 c on each side).  With the paper's averaged wave speed the central
    # face sees u-bar_n = 0 and the update drives the pressure negative within
    # a few steps; the one-sided maximum keeps it positive.
    mi = W.shock_tube_strip(40, 2, seed=1)
    cen = mi.centroids()
    c = math.sqrt(G)
    u = np.where(cen[:, 0] < 0.5, -2.0 * c, 2.0 * c)
    U0 = W.conserved(np.ones(mi.n_tri), u, np.zeros(mi.n_tri), np.ones(mi.n_tri))
    results = {}
    for mode in ("average", "max"):
        orc.set_wave_speed(mode)
        try:
            om = build(orc, mi, W.conserved(1.0, 0.0, 0.0, 1.0))
            results[mode] = om.run(U0, 40, 0.4)
        finally:
            orc.set_wave_speed("average")
    assert results["average"][3]  # lost positivity
    Um, _, steps, bad = results["max"]
    assert not bad and steps == 40
    assert prim(Um)[3].min() > 0.0 and Um[:, 0].min() > 0.0


def test_vortex_is_advected_with_the_free_stream(orc):
    # an isentropic vortex in a uniform stream is a steady solution of the
    # Euler equations translated with velocity u_inf: after time t its centre
    # (the density minimum) sits at x0 + u_inf t (periodically).  The first-
    # order scheme damps the vortex but must carry it at the stream speed.
    mi = W.periodic_square(64, 32, seed=4)
    cen = mi.centroids()
    mach = 0.5
    u_inf = mach * math.sqrt(G)
    U0 = W.isentropic_vortex(cen, mach=mach, beta=5.0)
    mesh = build(orc, mi, W.conserved(1.0, u_inf, 0.0, 1.0))
    t_end = 0.5 / u_inf  # half a flow-through: the centre moves to x = 1.0 = 0.0
    U, t, _, bad = mesh.run(U0, 10 ** 6, 0.4, t_stop=t_end)
    assert not bad and t == pytest.approx(t_end, rel=1e-12)
    rho = U[:, 0]
    deficit = np.clip(rho.max() - rho, 0.0, None)
    # deficit-weighted centre, x taken on the circle (periodic)
    ang = 2.0 * math.pi * cen[:, 0]
    xc = (math.atan2((deficit * np.sin(ang)).sum(), (deficit * np.cos(ang)).sum())
          / (2.0 * math.pi)) % 1.0
    yc = (deficit * cen[:, 1]).sum() / deficit.sum()
    x_expect = (0.5 + u_inf * t_end) % 1.0
    dx, dy = 1.0 / 64, 1.0 / 32
    gap = min(abs(xc - x_expect), 1.0 - abs(xc - x_expect))
    assert gap <= 2 * dx and abs(yc - 0.5) <= 2 * dy
    # the minimum has not been smeared away: the vortex is still there
    assert rho.min() < 0.95 * rho.max()
    # a wrong stream speed (a dropped or doubled advection term) is caught
    assert min(abs(xc - 0.5), 1.0 - abs(xc - 0.5)) > 10 * dx


def test_dt_matches_brute_force(orc, c1):
    mi, mesh = c1
    U = W.isentropic_vortex(mi.centroids(), mach=0.5)
    rho, u, v, p = prim(U)
    P = mi.xy[mi.tri]
    perim = sum(np.hypot(*(P[:, (k + 1) % 3] - P[:, k]).T) for k in range(3))
    area = 0.5 * np.abs((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1])
                        - (P[:, 2, 0] - P[:, 0, 0]) * (P[:, 1, 1] - P[:, 0, 1]))
    lam = np.hypot(u, v) + np.sqrt(G * p / rho)
    want = 0.4 * np.min(2 * area / (perim * lam))
    assert mesh.dt(U, 0.4) == pytest.approx(want, rel=1e-13)
    assert mesh.dt(U, -1e-3) == 1e-3  # fixed-step mode


def test_t_stop_is_reached_exactly(orc, c1):
    mi, mesh = c1
    U0 = W.isentropic_vortex(mi.centroids(), mach=0.5)
    dt0 = mesh.dt(U0, 0.4)
    t_stop = 3.5 * dt0
    U, t, steps, bad = mesh.run(U0, 50, 0.4, t_stop=t_stop)
    assert t == pytest.approx(t_stop, rel=1e-15) and 4 <= steps <= 5 and not bad


def test_rk2_is_second_order_in_time(orc):
    # fixed mesh, fixed steps: the time error of Heun's scheme falls by ~4 per
    # halving of dt, that of forward Euler by ~2
    mi = W.periodic_square(16, 16, seed=2, jitter=0.1)
    mesh = build(orc, mi)
    U0 = W.isentropic_vortex(mi.centroids(), mach=0.5, radius=0.2)
    T = 0.02
    ref, *_ = mesh.run(U0, 1 << 20, -T / 512, t_stop=T, scheme=1)

    def err(scheme, n):
        U, t, _, _ = mesh.run(U0, n, -T / n, t_stop=T, scheme=scheme)
        assert t == pytest.approx(T)
        return np.abs(U - ref).max()

    rk = [err(1, n) for n in (8, 16, 32)]
    fe = [err(0, n) for n in (16, 32, 64)]
    assert 3.3 < rk[0] / rk[1] < 4.7 and 3.3 < rk[1] / rk[2] < 4.7
    assert 1.7 < fe[0] / fe[1] < 2.3 and 1.7 < fe[1] / fe[2] < 2.3


# ---------------------------------------------------------------------------
# the scheme against the exact Riemann solution
# ---------------------------------------------------------------------------
def test_exact_riemann_solver_matches_textbook():
    g = read_golden("sod_star_state.txt")
    p, u, rl, rr = star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert p == pytest.approx(g["p_star"], abs=1e-5)
    assert u == pytest.approx(g["u_star"], abs=1e-5)
    assert rl == pytest.approx(g["rho_star_L"], abs=1e-5)
    assert rr == pytest.approx(g["rho_star_R"], abs=1e-5)


def test_sod_converges_to_exact_solution(orc):
    errs, hs = [], []
    for nx in (40, 80, 160, 320):
        mi = W.shock_tube_strip(nx, max(nx // 20, 2), seed=nx)
        mesh = build(orc, mi)
        xc = mi.centroids()
        U0 = W.sod_state(xc)
        U, t, _, bad = mesh.run(U0, 100000, 0.4, t_stop=0.2)
        assert not bad and t == pytest.approx(0.2, rel=1e-14)
        ex = sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (xc[:, 0] - 0.5) / 0.2)
        errs.append(np.sum(mesh.vol * np.abs(U[:, 0] - ex[:, 0])) / mesh.vol.sum())
        hs.append(1.0 / nx)
        # the flow stays one-dimensional: transverse momentum is small
        assert np.abs(U[:, 2]).max() < 0.05 * np.abs(U[:, 1]).max()
    order = [math.log(errs[i] / errs[i + 1]) / math.log(2.0) for i in range(3)]
    assert all(e1 > e2 for e1, e2 in zip(errs, errs[1:])), errs
    assert order[-1] >= 0.5, (errs, order)
    assert errs[-1] < 0.03


# ---------------------------------------------------------------------------
# learned dissipation scale
# ---------------------------------------------------------------------------
def _random_theta(rng, scale=0.4):
    return rng.normal(scale=scale, size=orc_nparam())


def orc_nparam():
    import oracle
    return oracle.NPARAM


def test_closure_parameter_count(orc):
    assert orc._load().orc_closure_nparam() == orc.NPARAM == 8 * 32 + 32 + 32 * 32 + 32 + 32 + 1


def test_closure_scale_swap_invariant_and_bounded(orc):
    rng = np.random.default_rng(12)
    th = _random_theta(rng)
    for _ in range(100):
        UL, UR = random_state(rng), random_state(rng)
        n = rng.normal(size=2)
        fa = orc.closure_features(UL, UR, n)
        fb = orc.closure_features(UR, UL, -n)
        np.testing.assert_array_equal(fa, fb)
        s = orc.closure_scale(th, UL, UR, n)
        assert s == orc.closure_scale(th, UR, UL, -n)
        assert 0.2 <= s <= 1.5
        # features of a face between equal states
        f0 = orc.closure_features(UL, UL, n)
        assert f0[0] == f0[1] == f0[2] == f0[3] == f0[5] == 0.0 and f0[6] == f0[7] == 1.0


def test_closure_unit_scale_reproduces_plain_flux(orc, c1):
    mi, mesh = c1
    th = np.zeros(orc.NPARAM)
    th[-1] = math.log((0.8 / 1.3) / (1.0 - 0.8 / 1.3))  # s = 0.2 + 1.3 sigmoid(b3) = 1
    U = W.isentropic_vortex(mi.centroids(), mach=0.5)
    R_plain = mesh.residual(U)
    R_cl, sc = mesh.residual(U, theta=th, return_scales=True)
    np.testing.assert_allclose(sc, 1.0, rtol=1e-15)
    np.testing.assert_allclose(R_cl, R_plain, rtol=1e-13, atol=1e-13 * np.abs(R_plain).max())


def test_closure_keeps_conservation(orc, c1):
    mi, mesh = c1
    th = _random_theta(np.random.default_rng(13))
    U0 = W.isentropic_vortex(mi.centroids(), mach=0.5)
    U, _, steps, bad = mesh.run(U0, 30, 0.4, theta=th)
    assert steps == 30 and not bad
    assert _conservation_error(mesh, U0, U).max() <= 1e-12


@pytest.mark.parametrize("bf16", [False, True])
def test_closure_gradient_matches_finite_differences(orc, bf16):
    mi = W.channel_bump(10, 6, seed=7)
    uinf = W.conserved(*W.freestream(0.5))
    mesh = build(orc, mi, uinf)
    rng = np.random.default_rng(14)
    U0 = W.random_smooth_state(mi.centroids(), seed=5)
    Ut = U0 + 0.01 * rng.normal(size=U0.shape)
    th = _random_theta(rng, 0.5)
    w = np.array([1.0, 0.5, 0.5, 2.0])
    dt = 1e-3
    loss, g = mesh.closure_loss_grad(U0, Ut, dt, w, th, bf16_acts=bf16)
    assert np.isfinite(loss) and np.abs(g).max() > 0
    idx = rng.choice(orc.NPARAM, size=40, replace=False)
    idx = np.concatenate([idx, [orc.NPARAM - 1]])
    eps = 1e-6
    if bf16:
        # inputs of each layer are rounded to bfloat16; the derivative through
        # the rounding is taken as zero, so only the last layer can be checked
        # by differences that stay inside one rounding step
        idx = np.arange(orc.NPARAM - 33, orc.NPARAM)
    for i in idx:
        tp, tm = th.copy(), th.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (mesh.closure_loss_grad(U0, Ut, dt, w, tp, bf16, grad=False)
              - mesh.closure_loss_grad(U0, Ut, dt, w, tm, bf16, grad=False)) / (2 * eps)
        # central differences: rounding noise ~ eps_mach |loss| / eps
        noise = 100 * np.finfo(float).eps * abs(loss) / eps
        assert fd == pytest.approx(g[i], rel=1e-6, abs=noise), i


# ---------------------------------------------------------------------------
# renumbering diagnostics (Sec. 4.1)
# ---------------------------------------------------------------------------
def _graph_mesh(orc, adj):
    n = len(adj)
    nbr = np.full((n, 3), -1, np.int32)
    for i, a in enumerate(adj):
        nbr[i, :len(a)] = a
    return orc.Mesh.from_arrays(nbr, np.ones((n, 3, 2)), np.ones(n), np.zeros(4))


def test_bandwidth_and_serial_bandwidth_by_hand(orc):
    # path 0-1-2-3: B = 1; s = (1,0,1,2), e = (1,2,3,2); S = (0,0,1,2),
    # E = (1,2,3,3); S_BW = max(E - S) = 2
    path = _graph_mesh(orc, [[1], [0, 2], [1, 3], [2]])
    assert path.bandwidth() == 1 and path.serial_bandwidth() == 2
    # the same path labelled 0-2-1-3: edges (0,2), (2,1), (1,3): B = 2;
    # s = (2,2,0,1), e = (2,3,1,1); S = (0,0,0,1); E = (2,3,3,3); S_BW = 3
    lab = _graph_mesh(orc, [[2], [2, 3], [0, 1], [1]])
    assert lab.bandwidth() == 2 and lab.serial_bandwidth() == 3


def test_bandwidth_brute_force(orc, c1):
    mi, mesh = c1
    perm = np.random.default_rng(3).permutation(mi.n_tri)
    pm = mesh.permuted(perm)
    nb = pm.nbr
    i = np.repeat(np.arange(mi.n_tri), 3)
    j = nb.reshape(-1)
    ok = j >= 0
    assert pm.bandwidth() == np.abs(i[ok] - j[ok]).max()


# ---------------------------------------------------------------------------
# rounding ambiguity of the learned scale: error bounds and scale intervals
# ---------------------------------------------------------------------------
def _bf16(x):
    """bfloat16 round-to-nearest-even of float32 values, returned as float64."""
    f = np.asarray(x, np.float32).copy()
    b = f.view(np.uint32)
    b += np.uint32(0x7FFF) + ((b >> 16) & np.uint32(1))
    b &= np.uint32(0xFFFF0000)
    return f.astype(np.float64)


def _features_fp32(UL, UR, n):
    """The eight closure features evaluated in numpy float32 (every operation
    rounded to nearest), in an order of its own: velocities from the
    conserved state, face-normal components through the unit normal."""
    f32 = np.float32

    def prim(U):
        r, mx, my, E = (f32(x) for x in U)
        u, v = mx / r, my / r
        p = f32(0.4) * (E - f32(0.5) * (mx * u + my * v))
        return r, u, v, p, np.sqrt(f32(1.4) * p / r)

    nx, ny = f32(n[0]), f32(n[1])
    ln = np.sqrt(nx * nx + ny * ny)
    hx, hy = nx / ln, ny / ln
    rL, uL, vL, pL, cL = prim(UL)
    rR, uR, vR, pR, cR = prim(UR)
    unL, unR = uL * hx + vL * hy, uR * hx + vR * hy
    utL, utR = vL * hx - uL * hy, vR * hx - uR * hy
    cb = f32(0.5) * (cL + cR)
    return np.array([abs(rR - rL) / (f32(0.5) * (rL + rR)), abs(unR - unL) / cb,
                     abs(utR - utL) / cb, abs(pR - pL) / (f32(0.5) * (pL + pR)),
                     abs(f32(0.5) * (unL + unR)) / cb, abs(unR / cR - unL / cL),
                     min(cL, cR) / cb, max(cL, cR) / cb], np.float64)


def _mlp_fp32(th, x):
    """The MLP in float32 on bfloat16 inputs x: layer 1 accumulated term by
    term in float32 and rounded to bfloat16, layers 2 and 3 in float32."""
    f32 = np.float32
    W1 = th[:256].reshape(32, 8).astype(f32)
    b1, W2 = th[256:288].astype(f32), th[288:1312].reshape(32, 32).astype(f32)
    b2, w3, b3 = th[1312:1344].astype(f32), th[1344:1376].astype(f32), f32(th[1376])
    acc = np.zeros(32, f32)
    for j in range(8):
        acc = acc + W1[:, j] * f32(x[j])
    h1 = _bf16(np.maximum(acc + b1, f32(0))).astype(f32)
    acc = np.zeros(32, f32)
    for j in range(32):
        acc = acc + W2[:, j] * h1[j]
    h2 = np.maximum(acc + b2, f32(0))
    z = f32(0)
    for j in range(32):
        z = z + w3[j] * h2[j]
    z = z + b3
    return float(f32(0.2) + f32(1.3) / (f32(1) + np.exp(-z)))


def _bf16_theta(rng, scale=0.4):
    th = rng.normal(scale=scale, size=orc_nparam()).astype(np.float32).astype(np.float64)
    th[:256] = _bf16(th[:256])
    th[288:1312] = _bf16(th[288:1312])
    return th


def _face_pairs(rng, count):
    """Random faces: independent states, nearly equal states (small jumps,
    where the features cancel), and wall ghosts."""
    import oracle
    out = []
    for t in range(count):
        UL = random_state(rng).astype(np.float32).astype(np.float64)
        n = rng.normal(size=2) * 10.0 ** rng.uniform(-3, 0)
        kind = t % 3
        if kind == 0:
            UR = random_state(rng)
        elif kind == 1:
            UR = UL * (1.0 + 10.0 ** rng.uniform(-6, -2) * rng.normal(size=4))
        else:
            UR = oracle.ghost(oracle.WALL, UL, n, np.zeros(4))
        out.append((UL, UR.astype(np.float32).astype(np.float64), n))
    return out


def test_closure_feature_error_bounds_hold_for_an_fp32_evaluation(orc):
    # the bounds are first-order error propagation; an independent float32
    # evaluation must stay inside them (they are several times larger)
    rng = np.random.default_rng(21)
    worst = 0.0
    for UL, UR, n in _face_pairs(rng, 3000):
        f = orc.closure_features(UL, UR, n)
        e = orc.closure_feature_errors(UL, UR, n)
        g = _features_fp32(UL, UR, n)
        assert (e >= 0).all()
        assert (np.abs(g - f) <= e).all(), (UL, UR, n, g - f, e)
        worst = max(worst, float((np.abs(g - f) / np.maximum(e, 1e-300)).max()))
    assert worst > 1e-3  # the test really measures FP32 errors


def test_closure_scale_interval_contains_fp32_evaluations(orc):
    # a float32 evaluation of features and MLP lands inside the interval
    # (up to its own layer-2/3 rounding); a face whose roundings are all
    # determined has the oracle's bfloat16 scale as both ends
    rng = np.random.default_rng(22)
    th = _bf16_theta(rng)
    n_undet = 0
    pairs = _face_pairs(rng, 1500)
    for UL, UR, n in pairs:
        f = orc.closure_features(UL, UR, n)
        e = orc.closure_feature_errors(UL, UR, n)
        lo, hi, det = orc.closure_scale_interval(th, f, e)
        s32 = _mlp_fp32(th, _bf16(_features_fp32(UL, UR, n)))
        assert lo - 2e-6 <= s32 <= hi + 2e-6, (lo, hi, s32)
        s = orc.closure_scale(th, UL, UR, n, bf16_acts=True)
        assert lo <= s <= hi
        if det:
            assert lo == hi == s
        else:
            n_undet += 1
    assert 0 < n_undet < len(pairs)


def test_closure_scale_interval_covers_sampled_roundings(orc):
    # brute force: features and first-layer sums moved anywhere inside their
    # windows, then rounded, give scales inside the interval
    rng = np.random.default_rng(23)
    th = _bf16_theta(rng)
    W1, b1 = th[:256].reshape(32, 8), th[256:288]
    hit = 0
    for UL, UR, n in _face_pairs(rng, 300):
        f = orc.closure_features(UL, UR, n)
        e = orc.closure_feature_errors(UL, UR, n)
        lo, hi, det = orc.closure_scale_interval(th, f, e)
        for _ in range(20):
            x = _bf16(np.maximum(f + e * rng.uniform(-1, 1, 8), 0.0))
            a = b1 + W1 @ x
            mag = np.abs(b1) + np.abs(W1) @ x
            h1 = _bf16(np.maximum(a + 16.0 / 2 ** 23 * mag * rng.uniform(-1, 1, 32), 0.0))
            a2 = th[1312:1344] + th[288:1312].reshape(32, 32) @ h1
            z = th[1376] + th[1344:1376] @ np.maximum(a2, 0.0)
            s = 0.2 + 1.3 / (1.0 + math.exp(-z))
            assert lo - 1e-12 <= s <= hi + 1e-12
            hit += (not det) and s != lo
    assert hit > 0  # some samples really took another rounding
