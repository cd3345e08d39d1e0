"""The learned dissipation scale on the GPU (tensor-core MLP fused into the
flux) against the FP64 oracle's MLP with the same bfloat16 weights and the
same bfloat16 rounding of layer inputs.

The GPU evaluates the features in FP32 and accumulates layer 1 in FP32 before
rounding both to bfloat16, so a value within its FP32 evaluation error of a
bfloat16 rounding boundary may round either way.  The oracle bounds that error
for every rounded value and gives, per face, the interval of scales over all
admissible roundings and whether every rounding is determined
(orc_closure_scale_interval).  Every face is checked on its own: a face whose
roundings are determined must agree with the oracle's scale to 1e-5; every
other face must lie within its interval widened by 1e-5 (the FP32 rounding of
layers 2 and 3).  Gradients are compared on inputs drawn so that no face's
admissible roundings move its scale by more than 1e-6.
"""
import math

import numpy as np
import pytest

from paper_1408_5715_gb300 import binding as B
from paper_1408_5715_gb300 import build as BLD
from paper_1408_5715_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NP = B.CLOSURE_PARAMS
W1 = slice(0, 256)
W2 = slice(288, 288 + 1024)


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BLD.build()
    B.load()


def bf16(x):
    return torch.tensor(np.asarray(x, np.float32)).to(torch.bfloat16).float().numpy()


def make_theta(seed, scale=0.5):
    """FP32 parameters for the GPU and the FP64 values the GPU really uses
    (hidden-layer weights rounded to bfloat16) for the oracle."""
    rng = np.random.default_rng(seed)
    th = (rng.normal(size=NP) * scale).astype(np.float32)
    th[-1] = 0.3
    th64 = th.astype(np.float64)
    th64[W1] = bf16(th[W1])
    th64[W2] = bf16(th[W2])
    return th, th64


TOL_S = 1e-5  # FP32 rounding of layers 2 and 3 and of the sigmoid


def check_scales(s_gpu, s_orc, lo, hi, det):
    """Every entry: inside its admissible interval (widened by TOL_S); entries
    whose roundings are determined: within TOL_S of the oracle."""
    s_gpu, s_orc, lo, hi, det = (np.asarray(a).ravel() for a in (s_gpu, s_orc, lo, hi, det))
    out = (s_gpu < lo - TOL_S) | (s_gpu > hi + TOL_S)
    assert not out.any(), (np.nonzero(out)[0][:10], s_gpu[out][:5], lo[out][:5], hi[out][:5])
    d = np.abs(s_gpu - s_orc)[det]
    assert d.max() <= TOL_S, d.max()
    return det.mean()


def test_mlp_alone_matches_oracle(orc):
    th, th64 = make_theta(1)
    cl = B.Closure(th)
    rng = np.random.default_rng(2)
    rows = 5000
    f = np.abs(rng.normal(size=(rows, 8))) * np.array([0.3, 0.3, 0.3, 0.3, 0.5, 0.3, 1.0, 1.0])
    f = bf16(f).astype(np.float64)  # bfloat16-exact inputs: no rounding ambiguity at layer 1
    s_gpu = cl.eval(torch.tensor(f, dtype=torch.float32, device="cuda")).cpu().numpy()
    s_orc = np.array([orc.closure_mlp(th64, f[i], bf16_acts=True) for i in range(rows)])
    lo, hi, det = map(np.array, zip(*[orc.closure_scale_interval(th64, f[i]) for i in range(rows)]))
    assert (s_gpu >= 0.2).all() and (s_gpu <= 1.5).all()
    frac = check_scales(s_gpu, s_orc, lo, hi, det)
    assert frac > 0.5, frac
    # the scales really vary with the features
    assert s_gpu.std() > 0.05


@pytest.fixture(scope="module")
def vortex_case():
    mi = W.periodic_square(40, 24, seed=9)
    U0 = W.isentropic_vortex(mi.centroids(), mach=0.6, radius=0.15)
    U0 = U0.astype(np.float32).astype(np.float64)  # float-exact states
    return mi, U0


def test_face_scales_match_oracle_and_are_swap_invariant(orc, vortex_case):
    mi, U0 = vortex_case
    th, th64 = make_theta(3)
    cl = B.Closure(th)
    g = B.Mesh.from_input(mi, "f32")
    U = torch.tensor(U0, dtype=torch.float32, device="cuda")
    s = cl.scales(g, U).cpu().numpy()
    om = orc.Mesh(mi.xy, mi.tri, mi.canon, None, 0)
    _, so = om.residual(U0, theta=th64, bf16_acts=True, return_scales=True)
    lo, hi, det = om.closure_scale_intervals(U0, th64)
    check_scales(s, so, lo, hi, det)
    assert det.any() and (hi - lo).max() < 0.1
    # both cells of every face use the same scale, bit for bit
    nbr, nrm, _ = g.export()
    for c in range(mi.n_tri):
        for k in range(3):
            m = nbr[c, k]
            ks = [j for j in range(3) if nbr[m, j] == c and (nrm[m, j] == -nrm[c, k]).all()]
            assert ks and s[m, ks[0]] == s[c, k]


def test_closure_step_matches_oracle_and_conserves(orc, vortex_case):
    mi, U0 = vortex_case
    th, th64 = make_theta(4, scale=0.3)
    cl = B.Closure(th)
    g = B.Mesh.from_input(mi, "f32")
    U = torch.tensor(U0, dtype=torch.float32, device="cuda")
    T0 = g.totals(U)
    t = g.step(U, 120, 0.4, closure=cl)
    om = orc.Mesh(mi.xy, mi.tri, mi.canon, None, 0)
    Uo, to, _, bad = om.run(U0, 120, 0.4, theta=th64, bf16_acts=True)
    assert not bad and t == pytest.approx(to, rel=1e-5)
    got = U.double().cpu().numpy()
    assert np.linalg.norm(got[:, 0] - Uo[:, 0]) / np.linalg.norm(Uo[:, 0]) <= 1e-5
    # the closure changed the solution compared with the plain flux
    Up, *_ = om.run(U0, 120, 0.4)
    assert np.linalg.norm(Up[:, 0] - Uo[:, 0]) / np.linalg.norm(Uo[:, 0]) > 1e-4
    T1 = g.totals(U)
    scale = np.abs(U0 * om.vol[:, None]).sum(axis=0)
    assert (np.abs(T1 - T0) <= 1e-6 * scale).all()


@pytest.mark.parametrize("scheme", ["fe", "rk2"])
def test_unit_scale_reproduces_plain_flux(vortex_case, scheme):
    mi, U0 = vortex_case
    th = np.zeros(NP, np.float32)
    th[-1] = math.log((0.8 / 1.3) / (1.0 - 0.8 / 1.3))  # s = 0.2 + 1.3 sigmoid(b3) ~ 1
    cl = B.Closure(th)
    g = B.Mesh.from_input(mi, "f32")
    A = torch.tensor(U0, dtype=torch.float32, device="cuda")
    Bt = A.clone()
    g.step(A, 200, 0.4, scheme=scheme)
    g.step(Bt, 200, 0.4, scheme=scheme, closure=cl)
    a, b = A.double().cpu().numpy(), Bt.double().cpu().numpy()
    assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max()
    s = cl.scales(g, A).cpu().numpy()
    assert np.abs(s - 1.0).max() <= 2e-7


def test_closure_residual_and_errors(vortex_case):
    mi, U0 = vortex_case
    th, _ = make_theta(5)
    cl = B.Closure(th)
    g = B.Mesh.from_input(mi, "f32")
    U = torch.tensor(U0, dtype=torch.float32, device="cuda")
    R1 = g.residual(U, closure=cl)
    R0 = g.residual(U)
    assert torch.isfinite(R1).all() and not torch.equal(R0, R1)
    g64 = B.Mesh.from_input(mi, "f64")
    with pytest.raises(B.FVError):
        g64.step(torch.tensor(U0, device="cuda"), 1, 0.4, closure=cl)


SETTLED_WIDTH = 1e-6  # admissible roundings move a settled face's scale by at most this


def random_states(rng, k):
    """k cell states drawn independently (features O(1), no cancelling jumps)."""
    U = W.conserved(rng.uniform(0.5, 2.0, k), rng.uniform(-0.5, 0.5, k),
                    rng.uniform(-0.5, 0.5, k), rng.uniform(0.5, 2.0, k))
    return U.astype(np.float32).astype(np.float64)


def redraw_ambiguous_cells(om, U, theta, rng, max_iter=100):
    """Input generation for the gradient comparison: every cell with a face
    whose admissible bfloat16 roundings spread its scale by more than
    SETTLED_WIDTH gets a new random state, until no such face is left.  A
    face whose roundings are all determined has width 0; one whose only
    ambiguity is a feature at rounding noise next to zero (e.g. the
    tangential jump at a slip wall) has a width far below SETTLED_WIDTH."""
    U = U.copy()
    for _ in range(max_iter):
        lo, hi, _ = om.closure_scale_intervals(U, theta)
        bad = np.unique(np.nonzero(hi - lo > SETTLED_WIDTH)[0])
        if bad.size == 0:
            return U
        U[bad] = random_states(rng, bad.size)
    raise RuntimeError("ambiguous faces did not settle")


def test_closure_gradient_matches_oracle(orc):
    # channel with walls and far field: ghost faces take part too
    mi = W.channel_bump(36, 14, seed=12)
    prim = W.freestream(0.5)
    uinf = W.conserved(*prim)
    rng = np.random.default_rng(7)
    th, th64 = make_theta(8, scale=0.4)
    om = orc.Mesh(mi.xy, mi.tri, None, mi.bnd, 0, uinf)
    U0 = redraw_ambiguous_cells(om, random_states(rng, mi.n_tri), th64, rng)
    lo_s, hi_s, det = om.closure_scale_intervals(U0, th64)
    assert (hi_s - lo_s).max() <= SETTLED_WIDTH and det.mean() > 0.5
    Ut = (U0 + 0.02 * rng.normal(size=U0.shape)).astype(np.float32).astype(np.float64)
    dt, w = 2e-3, np.array([1.0, 0.5, 0.5, 2.0])
    g = B.Mesh.from_input(mi, "f32")
    g.set_freestream(*prim)
    cl = B.Closure(th)
    Ud = torch.tensor(U0, dtype=torch.float32, device="cuda")
    Utd = torch.tensor(Ut, dtype=torch.float32, device="cuda")
    loss, grad = cl.loss_grad(g, Ud, Utd, dt, w)
    grad = grad.cpu().numpy().astype(np.float64)
    lo, go = om.closure_loss_grad(U0, Ut, dt, w, th64, bf16_acts=True)
    assert loss == pytest.approx(lo, rel=1e-5)
    # each block of parameters on its own (W1, b1, W2, b2, w3, b3), and each
    # entry against its block's scale
    for sl in (slice(0, 256), slice(256, 288), slice(288, 1312), slice(1312, 1344),
               slice(1344, 1376), slice(1376, 1377)):
        ref = go[sl]
        assert np.linalg.norm(ref) > 0, sl
        e = np.linalg.norm(grad[sl] - ref) / np.linalg.norm(ref)
        assert e <= 1e-3, (sl, e)
        assert (np.abs(grad[sl] - ref) <= 1e-3 * np.abs(ref).max()).all(), sl
    # deterministic
    loss2, grad2 = cl.loss_grad(g, Ud, Utd, dt, w)
    assert loss2 == loss and np.array_equal(grad2.cpu().numpy().astype(np.float64), grad)


def test_adam_matches_reference_update():
    rng = np.random.default_rng(9)
    n = 1377
    th = rng.normal(size=n).astype(np.float32)
    m = np.zeros(n, np.float32)
    v = np.zeros(n, np.float32)
    t_th, t_m, t_v = (torch.tensor(x, device="cuda") for x in (th, m, v))
    for step in range(1, 4):
        gr = rng.normal(size=n).astype(np.float32)
        B.adam_step(t_th, torch.tensor(gr, device="cuda"), t_m, t_v, step, lr=1e-2)
        m = 0.9 * m + 0.1 * gr
        v = 0.999 * v + 0.001 * gr * gr
        th = th - 1e-2 * (m / (1 - 0.9 ** step)) / (np.sqrt(v / (1 - 0.999 ** step)) + 1e-8)
    np.testing.assert_allclose(t_th.cpu().numpy(), th, rtol=1e-5, atol=1e-6)


def test_training_lowers_one_step_loss(vortex_case):
    # target: one plain step with the dissipation halved everywhere (reachable
    # through b3 alone); a few Adam steps on the GPU must lower the loss
    mi, U0 = vortex_case
    g = B.Mesh.from_input(mi, "f32")
    U = torch.tensor(U0, dtype=torch.float32, device="cuda")
    th_t = np.zeros(NP, np.float32)
    th_t[-1] = math.log((0.3 / 1.3) / (1.0 - 0.3 / 1.3))  # s = 0.5
    target = B.Closure(th_t)
    dt = 0.4 * g.compute_dt(U, 1.0)
    Ut = U.clone()
    g.step(Ut, 1, -dt, closure=target)
    theta = torch.tensor(make_theta(10, scale=0.1)[0], device="cuda")
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    cl = B.Closure(theta.cpu().numpy())
    w = (1e-3, 1e-3, 1e-3, 1e-3)
    first = None
    for step in range(1, 61):
        loss, grad = cl.loss_grad(g, U, Ut, dt, w)
        first = loss if first is None else first
        B.adam_step(theta, grad, m, v, step, lr=3e-2)
        cl.set(theta)
    assert loss < 0.2 * first, (first, loss)


@pytest.mark.parametrize("scheme", ["fe", "rk2"])
def test_closure_step_is_bitwise_the_same_in_any_order(vortex_case, scheme):
    # a face shared by two cells of one warp is one MLP row, evaluated once; in
    # Hilbert order most warps share many faces, in a shuffled order almost
    # none.  The cell arithmetic is local, so the two runs agree bit for bit.
    mi, U0 = vortex_case
    th, _ = make_theta(7, scale=0.3)
    cl = B.Closure(th)
    outs = []
    for order in ("hilbert", "shuffle"):
        g = B.Mesh.from_input(mi, "f32")
        perm = g.renumber(order, seed=3)
        U = torch.tensor(U0[perm], dtype=torch.float32, device="cuda")
        t = g.step(U, 60, 0.4, scheme=scheme, closure=cl)
        out = np.empty_like(U0, dtype=np.float32)
        out[perm] = U.cpu().numpy()
        outs.append((t, out))
    assert outs[0][0] == outs[1][0]
    assert np.array_equal(outs[0][1], outs[1][1])


def test_captured_graphs_see_new_closure_parameters(vortex_case):
    # the output bias b3 is a kernel argument of a captured step graph: after
    # fv_closure_set the mesh recaptures, and a new closure in the old one's
    # place does not replay the old graph either
    mi, U0 = vortex_case
    th1, _ = make_theta(3, scale=0.3)
    th2, _ = make_theta(3, scale=0.3)
    th2[-1] = -1.5  # only the output bias differs
    g = B.Mesh.from_input(mi, "f32")
    cl = B.Closure(th1)
    U = torch.tensor(U0, dtype=torch.float32, device="cuda")
    g.step(U, 100, 0.4, closure=cl)  # 96 steps through a captured graph
    cl.set(th2)
    U = torch.tensor(U0, dtype=torch.float32, device="cuda")
    g.step(U, 100, 0.4, closure=cl)
    ref = B.Mesh.from_input(mi, "f32")
    Ur = torch.tensor(U0, dtype=torch.float32, device="cuda")
    ref.step(Ur, 100, 0.4, closure=B.Closure(th2))
    assert torch.equal(U, Ur)
    cl.close()
    cl = B.Closure(th1)
    U = torch.tensor(U0, dtype=torch.float32, device="cuda")
    g.step(U, 100, 0.4, closure=cl)
    Ur = torch.tensor(U0, dtype=torch.float32, device="cuda")
    ref.step(Ur, 100, 0.4, closure=B.Closure(th1))
    assert torch.equal(U, Ur)


@pytest.mark.parametrize("scheme", ["fe", "rk2"])
@pytest.mark.parametrize("tile", [256, 512, 1024])
def test_closure_on_tiles_gives_the_bits_of_the_two_passes(vortex_case, scheme, tile):
    # with shape 7 the learned step runs as one kernel on tiles (each face's
    # scale and flux formed once); the scale pass + scaled step gives the
    # same bits
    mi, U0 = vortex_case
    th, _ = make_theta(6, scale=0.3)
    cl = B.Closure(th)
    outs = []
    for variant in (1, 7):
        g = B.Mesh.from_input(mi, "f32")
        perm = g.renumber("hilbert")
        g.set_variant(variant)
        if variant == 7:
            g.set_blocking(1, tile)
        U = torch.tensor(U0[perm], dtype=torch.float32, device="cuda")
        t = g.step(U, 110, 0.4, scheme=scheme, closure=cl)  # a captured graph and a tail
        outs.append((t, U))
    assert outs[0][0] == outs[1][0]
    assert torch.equal(outs[0][1], outs[1][1])


def test_tcgen05_scales_match_oracle(orc, vortex_case):
    # the MLP on tcgen05 (128-row MMAs into tensor memory), per face against
    # the oracle as the mma.sync engine is checked above
    mi, U0 = vortex_case
    th, th64 = make_theta(3)
    cl = B.Closure(th)
    g = B.Mesh.from_input(mi, "f32")
    g.set_closure_engine("tcgen05")
    U = torch.tensor(U0, dtype=torch.float32, device="cuda")
    s = cl.scales(g, U).cpu().numpy()
    om = orc.Mesh(mi.xy, mi.tri, mi.canon, None, 0)
    _, so = om.residual(U0, theta=th64, bf16_acts=True, return_scales=True)
    lo, hi, det = om.closure_scale_intervals(U0, th64)
    check_scales(s, so, lo, hi, det)


@pytest.mark.parametrize("scheme", ["fe", "rk2"])
@pytest.mark.parametrize("variant,tile", [(1, None), (7, 256), (7, 832)])
def test_tcgen05_engine_gives_the_bits_of_mma_sync(vortex_case, scheme, variant, tile):
    # both tensor-core engines, in both forms of the learned step (scale pass +
    # scaled step; one kernel on shape 7's tiles), give the same bits
    mi, U0 = vortex_case
    th, _ = make_theta(6, scale=0.3)
    cl = B.Closure(th)
    outs = []
    for engine in ("mma.sync", "tcgen05"):
        g = B.Mesh.from_input(mi, "f32")
        perm = g.renumber("hilbert")
        g.set_variant(variant)
        if tile:
            g.set_blocking(1, tile)
        g.set_closure_engine(engine)
        U = torch.tensor(U0[perm], dtype=torch.float32, device="cuda")
        s = cl.scales(g, U)
        t = g.step(U, 110, 0.4, scheme=scheme, closure=cl)  # a captured graph and a tail
        outs.append((t, U, s))
    assert outs[0][0] == outs[1][0]
    assert torch.equal(outs[0][2], outs[1][2])
    assert torch.equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("variant", [1, 7])
def test_tcgen05_wait_timeout_is_reported(vortex_case, variant):
    # a wait limit of 0 polls makes every wait on the MMAs give up: the step
    # reports FV_ETIMEOUT after the block has drained its MMAs and freed its
    # tensor memory, and the mesh and device stay usable
    mi, U0 = vortex_case
    th, _ = make_theta(6, scale=0.3)
    cl = B.Closure(th)
    g = B.Mesh.from_input(mi, "f32")
    g.set_variant(variant)
    g.set_closure_engine("tcgen05")
    g.set_wait_limit(0)
    U = torch.tensor(U0, dtype=torch.float32, device="cuda")
    with pytest.raises(B.FVError) as e:
        g.step(U, 3, 0.4, closure=cl)
    assert e.value.code == B.FV_ETIMEOUT
    g.set_wait_limit(1 << 24)
    ref = B.Mesh.from_input(mi, "f32")
    ref.set_variant(variant)
    V, W_ = (torch.tensor(U0, dtype=torch.float32, device="cuda") for _ in range(2))
    assert g.step(V, 5, 0.4, closure=cl) == ref.step(W_, 5, 0.4, closure=cl)
    assert torch.equal(V, W_)
