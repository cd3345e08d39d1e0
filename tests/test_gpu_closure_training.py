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
