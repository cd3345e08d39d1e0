"""Runs of every kernel family for the bounds-checked build test
(test_gpu_index_checks.py).  Imported by the test (normal library) and run as
a child process with FV_LIBRARY=debug (bounds-checked library), so that each
process loads exactly one library.

    python index_check_runs.py OUT.npz   # child: clean runs + planted indices
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1408_5715_gb300 import binding as B  # noqa: E402
from paper_1408_5715_gb300 import workloads as W  # noqa: E402


def _square():
    mi = W.periodic_square(40, 24, seed=9)
    return mi, W.isentropic_vortex(mi.centroids(), mach=0.6, radius=0.15)


def _channel():
    mi = W.channel_bump(40, 16, seed=3)
    return mi, W.uniform_state(mi.n_tri, W.freestream(0.5))


def clean_runs():
    """Every kernel family on small meshes; returns {name: final state}."""
    import torch
    out = {}
    mi, U0 = _square()
    for prec, dt in (("f32", torch.float32), ("f64", torch.float64)):
        for variant in range(8):
            m = B.Mesh.from_input(mi, prec)
            perm = m.renumber("hilbert")
            m.set_variant(variant)
            U = torch.tensor(U0[perm], dtype=dt, device="cuda")
            m.step(U, 30, 0.4)
            out[f"square_{prec}_v{variant}"] = U.cpu().numpy()
    mc, Uc = _channel()
    for variant in (1, 5, 6):
        m = B.Mesh.from_input(mc, "f32")
        m.set_freestream(*W.freestream(0.5))
        perm = m.renumber("hilbert")
        m.set_variant(variant)
        U = torch.tensor(Uc[perm], dtype=torch.float32, device="cuda")
        m.step(U, 30, 0.4, scheme="rk2")
        out[f"channel_rk2_v{variant}"] = U.cpu().numpy()
    for staged in (0, 1):
        m = B.Mesh.from_input(mi, "f32")
        perm = m.renumber("hilbert")
        m.set_blocking(2, 512, bool(staged))
        U = torch.tensor(U0[perm], dtype=torch.float32, device="cuda")
        m.step(U, 30, 0.4)
        out[f"pairs_staged{staged}"] = U.cpu().numpy()
    m = B.Mesh.from_input(mi, "f32")
    perm = m.renumber("hilbert")
    m.set_geometry("vertex")
    U = torch.tensor(U0[perm], dtype=torch.float32, device="cuda")
    m.step(U, 30, 0.4)
    out["vertex"] = U.cpu().numpy()
    rng = np.random.default_rng(3)
    cl = B.Closure((rng.normal(size=B.CLOSURE_PARAMS) * 0.3).astype(np.float32))
    for engine in ("mma.sync", "tcgen05"):
        for variant in (1, 7):  # scale pass + scaled step; one kernel on tiles
            m = B.Mesh.from_input(mi, "f32")
            perm = m.renumber("hilbert")
            m.set_variant(variant)
            m.set_closure_engine(engine)
            U = torch.tensor(U0[perm], dtype=torch.float32, device="cuda")
            m.step(U, 30, 0.4, closure=cl)
            out[f"closure_{engine}_v{variant}"] = U.cpu().numpy()
    meshes, states = [], []
    for k, (nx, ny) in enumerate(((20, 12), (44, 20), (30, 30))):
        mk = W.periodic_square(nx, ny, seed=40 + k)
        g = B.Mesh.from_input(mk, "f32")
        meshes.append(g)
        states.append(W.isentropic_vortex(mk.centroids(), mach=0.5)[g.renumber("hilbert")])
    batch = B.Batch(meshes)
    for variant in (0, 5, 6):
        batch.set_variant(variant)
        U = torch.tensor(batch.pack(states), dtype=torch.float32, device="cuda")
        batch.step(U, 20, 0.4)
        out[f"batch_v{variant}"] = np.concatenate(batch.unpack(U.cpu().numpy()))
    return out


def planted_runs():
    """Steps after one neighbour index was overwritten with an index outside
    its array; returns {name: status code of the step}."""
    import torch
    codes = {}
    mi, U0 = _square()
    n = mi.n_tri
    cases = [("global_f32_v1", "f32", 1, 0, 0, n + 7), ("global_f32_v0", "f32", 0, 0, 1, n + 7),
             ("global_f64_v0", "f64", 0, 0, 2, n + 7), ("local_f32_v6", "f32", 6, 1, 0, 0xF000),
             ("local_f32_pairs", "f32", None, 1, 1, 0xF000)]
    for name, prec, variant, table, slot, value in cases:
        m = B.Mesh.from_input(mi, prec)
        perm = m.renumber("hilbert")
        if variant is None:
            m.set_blocking(2, 512)
        else:
            m.set_variant(variant)
        dt = torch.float32 if prec == "f32" else torch.float64
        U = torch.tensor(U0[perm], dtype=dt, device="cuda")
        m.step(U, 2, 0.4)  # uploads the tables (and builds tiles)
        rc = B.load().fv_mesh_debug_set_index(m._h, table, n // 2, slot, value, None)
        assert rc == B.FV_OK, B.load().fv_last_error()
        try:
            m.step(U, 4, 0.4)
            codes[name] = B.FV_OK
        except B.FVError as e:
            codes[name] = e.code
        m.close()
    return codes


def main(path):
    lib = B.load()
    assert lib.fv_index_checks() == 1, "the child must load the bounds-checked library"
    runs = clean_runs()
    codes = planted_runs()
    np.savez(path, **runs, **{f"code_{k}": np.array(v) for k, v in codes.items()})


if __name__ == "__main__":
    main(sys.argv[1])
