"""The learned dissipation scale, trained on the GPU by the library's own
kernels from restricted fine-mesh FP64 runs, lowers the coarse-mesh error
against the restricted fine solution on held-out inflow Mach numbers."""
import numpy as np
import pytest

from paper_1408_5715_gb300 import binding as B
from paper_1408_5715_gb300 import build as BLD

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BLD.build()
    B.load()


@pytest.mark.parametrize("coarse", ["f32", "f64"])
def test_restriction_kernel_matches_host_area_weighted_mean(coarse):
    # fv_restrict_mean against a float64 NumPy mean of the 16 children, with
    # both meshes renumbered (children are scattered in the fine numbering)
    from paper_1408_5715_gb300 import workloads as W
    mc = W.channel_bump(30, 12, seed=4)
    mf, parent = W.refine_midpoint(mc, 2)
    gc, gf = B.Mesh.from_input(mc, "f32"), B.Mesh.from_input(mf, "f64")
    perm_c, perm_f = gc.renumber("hilbert"), gf.renumber("rcm")
    _, _, area_f = gf.export()
    inv_f = np.empty(mf.n_tri, np.int64)
    inv_f[perm_f] = np.arange(mf.n_tri)
    fine_of = inv_f[perm_c[:, None] * 16 + np.arange(16)[None, :]]
    assert (parent[perm_f[fine_of]] == perm_c[:, None]).all()
    Uf = W.random_smooth_state(mf.centroids(), seed=2)[perm_f]
    want = (area_f[fine_of][:, :, None] * Uf[fine_of]).sum(axis=1) / area_f[fine_of].sum(axis=1)[:, None]
    dt = torch.float32 if coarse == "f32" else torch.float64
    Uc = torch.full((mc.n_tri, 4), float("nan"), dtype=dt, device="cuda")
    B.restrict_mean(torch.tensor(Uf, device="cuda"), torch.tensor(area_f, device="cuda"),
                    torch.tensor(fine_of.astype(np.int32), device="cuda"), Uc)
    got = Uc.double().cpu().numpy()
    # summation order and the final rounding, against the mean magnitude
    mag = (area_f[fine_of][:, :, None] * np.abs(Uf[fine_of])).sum(axis=1) \
        / area_f[fine_of].sum(axis=1)[:, None]
    tol = 1e-14 if coarse == "f64" else 2.0 ** -24 + 1e-15
    assert (np.abs(got - want) <= tol * mag).all()
    # a uniform fine state restricts to itself (to the rounding of the mean)
    Uc.zero_()
    ones = np.tile(np.array([1.0, 0.5, -0.25, 3.0]), (mf.n_tri, 1))
    B.restrict_mean(torch.tensor(ones, device="cuda"), torch.tensor(area_f, device="cuda"),
                    torch.tensor(fine_of.astype(np.int32), device="cuda"), Uc)
    assert np.allclose(Uc.double().cpu().numpy(), ones[:mc.n_tri], rtol=1e-7, atol=0)


def test_trained_closure_beats_plain_lax_friedrichs_on_held_out_mach():
    from paper_1408_5715_gb300 import closure_training as CT
    cfg = CT.TrainConfig(coarse_nx=100, coarse_ny=32, n_train=4, n_test=2, horizon=0.3,
                         pairs_per_run=16, epochs=25, lr=3e-3, seed=11)
    report, cl, prob = CT.train_and_evaluate(cfg)
    assert report["loss_history"][-1] < report["loss_first"]
    for r in report["heldout"]:
        assert r["err_learned"] < r["err_plain"], r
    # the scales stay inside the closure's range
    assert 0.2 <= report["scale_stats"]["min"] and report["scale_stats"]["max"] <= 1.5
    # the fine reference differs from the coarse plain run by a resolvable amount
    assert min(r["err_plain"] for r in report["heldout"]) > 1e-4
