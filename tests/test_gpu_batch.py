"""Batched many-mesh stepping on the GPU: every mesh of a batch advances bit
for bit as it does alone, with its own dt, time, free stream and totals."""
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


def make_set(seed, n_meshes=7):
    """Uneven meshes: periodic squares of several sizes and a channel with
    walls and far field, each with its own initial state and free stream."""
    rng = np.random.default_rng(seed)
    items = []
    for k in range(n_meshes):
        if k == 3:
            mi = W.channel_bump(40, 17, seed=k)
            prim = W.freestream(0.55)
            U0 = W.uniform_state(mi.n_tri, prim)
        else:
            ny = int(rng.integers(3, 40))
            mi = W.periodic_square(2 * ny + int(rng.integers(0, 3)), ny, seed=100 + k)
            mach = float(rng.uniform(0.3, 0.8))
            prim = W.freestream(mach)
            U0 = (W.isentropic_vortex(mi.centroids(), mach=mach) if rng.integers(0, 2)
                  else W.uniform_state(mi.n_tri, prim))
        items.append((mi, prim, U0))
    return items


def solo_and_batch(items, prec, nsteps, scheme, t_stop=0.0, comp=True, variant=5):
    dt_ = torch.float64 if prec == "f64" else torch.float32
    meshes, solo = [], []
    for mi, prim, U0 in items:
        m = B.Mesh.from_input(mi, prec)
        m.set_freestream(*prim)
        m.renumber("rcm")
        meshes.append(m)
    # states in each mesh's (renumbered) order: renumber is deterministic
    perms = []
    for (mi, prim, U0), m in zip(items, meshes):
        probe = B.Mesh.from_input(mi, prec)
        perms.append(probe.renumber("rcm"))
    for (mi, prim, U0), m, p in zip(items, meshes, perms):
        if prec == "f32":
            m.set_compensation(comp)
        U = torch.tensor(U0[p], dtype=dt_, device="cuda")
        t = m.step(U, nsteps, 0.4, t_stop=t_stop, scheme=scheme)
        solo.append((U.cpu().numpy(), t, m.totals(U)))
    batch = B.Batch(meshes)
    batch.set_variant(variant)
    if prec == "f32":
        batch.set_compensation(comp)
    flat = torch.tensor(batch.pack([U0[p] for (mi, prim, U0), p in zip(items, perms)]),
                        dtype=dt_, device="cuda")
    tb = batch.step(flat, nsteps, 0.4, t_stop=t_stop, scheme=scheme)
    return solo, batch, flat, tb


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("scheme", ["fe", "rk2"])
@pytest.mark.parametrize("variant", [5, 0, 6])
def test_batch_equals_solo_bitwise(prec, scheme, variant):
    items = make_set(5)
    solo, batch, flat, tb = solo_and_batch(items, prec, 131, scheme, variant=variant)
    got = batch.unpack(flat.cpu().numpy())
    tot = batch.totals(flat)
    for k, (Us, ts, Ts) in enumerate(solo):
        assert np.array_equal(got[k], Us), k
        assert tb[k] == ts, k
        scale = np.abs(Us).sum(axis=0) + 1e-300
        assert (np.abs(tot[k] - Ts) <= 1e-13 * np.abs(Ts).max() + 1e-300).all(), k
    # the meshes really have different time steps
    assert len(set(np.round(tb, 12))) > 1


def test_batch_t_stop_and_bad_state():
    items = make_set(6, n_meshes=4)
    solo, batch, flat, tb = solo_and_batch(items, "f64", 500, "fe", t_stop=0.01)
    assert np.allclose(tb, 0.01, rtol=1e-14)
    for k, (Us, ts, _) in enumerate(solo):
        assert np.array_equal(batch.unpack(flat.cpu().numpy())[k], Us)
    # a bad state in one mesh is reported for the batch
    bad = flat.clone()
    k = 2
    i = int(batch.offsets[k]) + 5
    bad[i, 3] = 0.01 * 0.5 * (bad[i, 1] ** 2 + bad[i, 2] ** 2) / bad[i, 0]
    with pytest.raises(B.FVError) as e:
        batch.step(bad, 3, 0.4)
    assert e.value.code == B.FV_ENONFINITE


@pytest.mark.parametrize("variant", [5, 0, 6])
def test_batch_split_calls_with_remainder_equal_one_call(variant):
    items = make_set(3, n_meshes=4)
    _, batch, flat, _ = solo_and_batch(items, "f32", 0, "fe", variant=variant)
    start = flat.clone()
    batch.step(flat, 151, 0.4)
    lo = torch.zeros((batch.n_padded, 4), dtype=torch.int16, device="cuda")
    batch.set_remainder(lo)
    split = start.clone()
    for k in (96, 1, 54):
        batch.step(split, k, 0.4)
    for k in range(len(items)):
        o0, o1 = batch.offsets[k], batch.offsets[k] + items[k][0].n_tri
        assert torch.equal(flat[o0:o1], split[o0:o1]), k


def test_batch_rejects_mixed_precision():
    a = B.Mesh.from_input(W.periodic_square(4, 4, seed=1), "f32")
    b = B.Mesh.from_input(W.periodic_square(4, 4, seed=1), "f64")
    with pytest.raises(B.FVError):
        B.Batch([a, b])


def test_full_size_batch_matches_solo_on_sampled_meshes(orc):
    # the benchmark's 256-mesh batch (13.1M cells, Hilbert order, the default
    # tiled shape): sampled meshes advance bit for bit as they do alone, and
    # the smallest sampled one matches the FP64 oracle's run in FP32 tolerance
    items = W.vortex_batch()
    meshes, states = [], []
    for mi, prim, U0 in items:
        m = B.Mesh.from_input(mi, "f32")
        m.set_freestream(*prim)
        perm = m.renumber("hilbert")
        meshes.append(m)
        states.append(U0[perm])
    batch = B.Batch(meshes)
    flat = torch.tensor(batch.pack(states), dtype=torch.float32, device="cuda")
    tb = batch.step(flat, 20, 0.4)
    got = batch.unpack(flat.cpu().numpy())
    rng = np.random.default_rng(11)
    sample = sorted(set(rng.choice(len(items), size=4, replace=False).tolist()) |
                    {int(np.argmin(batch.sizes))})
    for k in sample:
        U = torch.tensor(states[k], dtype=torch.float32, device="cuda")
        t = meshes[k].step(U, 20, 0.4)
        assert t == tb[k]
        assert np.array_equal(U.cpu().numpy(), got[k]), k
    k = int(np.argmin(batch.sizes))
    mi, prim, U0 = items[k]
    om = orc.Mesh(mi.xy, mi.tri, mi.canon, mi.bnd, mi.default_bc, W.conserved(*prim))
    Uo, to, _, bad = om.run(U0, 20, 0.4)
    assert not bad and tb[k] == pytest.approx(to, rel=1e-6)
    perm = B.Mesh.from_input(mi, "f32").renumber("hilbert")
    mine = np.empty_like(Uo)
    mine[perm] = got[k]
    assert np.linalg.norm(mine[:, 0] - Uo[:, 0]) / np.linalg.norm(Uo[:, 0]) <= 1e-5
    batch.close()
