"""Partitioned stepping on several processes (gloo, CPU).

The library's host partitioning (fv_partition_*) splits a renumbered mesh into
contiguous parts with halos.  Each rank advances its owned cells with the
FP64 oracle's residual (reading owned and halo states), the CFL minimum is
reduced over the ranks, and halo states are refreshed from their owners after
every step.  The gathered result equals the single-domain oracle run bit for
bit: the bookkeeping (global ids, local neighbour tables, halo owners) is
exactly right.
"""
import ctypes
import os
import socket

import numpy as np
import pytest

from paper_1408_5715_gb300 import binding as B
from paper_1408_5715_gb300 import build as BLD
from paper_1408_5715_gb300 import workloads as W

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(kind):
    if kind == "periodic":
        mi = W.vortex_square_small(seed=1)
        U0 = W.isentropic_vortex(mi.centroids(), mach=0.5)
        uinf = W.conserved(*W.freestream(0.5))
    else:
        mi = W.channel_bump(60, 20, seed=3)
        uinf = W.conserved(*W.freestream(0.6))
        U0 = W.uniform_state(mi.n_tri, W.freestream(0.6))
    return mi, U0, uinf


def _rank_main(rank, world, port, kind, order, nsteps, out_dir):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mi, U0, uinf = _case(kind)
    m = B.Mesh.from_input(mi, "f64")
    perm = m.renumber(order, seed=4)
    Ug = U0[perm]
    part = m.partition(world, rank)
    no = part["n_owned"]
    gid = part["global_ids"]
    U = np.ascontiguousarray(Ug[gid])  # owned then halo
    lib = oracle._load()
    nbr = np.ascontiguousarray(part["nbr"])
    nrm = np.ascontiguousarray(part["normals"])
    vol = np.ascontiguousarray(part["area"])
    uinf = np.ascontiguousarray(uinf)
    d = ctypes.POINTER(ctypes.c_double)
    i32 = ctypes.POINTER(ctypes.c_int32)
    starts = [m.n * p // world for p in range(world + 1)]
    for _ in range(nsteps):
        dt = lib.orc_dt(no, nrm.ctypes.data_as(d), vol.ctypes.data_as(d), U.ctypes.data_as(d), 0.4)
        t = torch.tensor([dt], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
        dt = float(t.item())
        R = np.empty((no, 4))
        lib.orc_residual(no, nbr.ctypes.data_as(i32), nrm.ctypes.data_as(d), vol.ctypes.data_as(d),
                         uinf.ctypes.data_as(d), U.ctypes.data_as(d), None, 0,
                         R.ctypes.data_as(d), None)
        U[:no] = U[:no] + dt * R
        # halo refresh: every rank's owned block to every rank
        blocks = [torch.zeros((starts[p + 1] - starts[p], 4), dtype=torch.float64)
                  for p in range(world)]
        dist.all_gather(blocks, torch.from_numpy(U[:no].copy()))
        full = torch.cat(blocks).numpy()
        U[no:] = full[gid[no:]]
        # every halo cell is owned by the part the library says
        own = np.searchsorted(starts, gid[no:], side="right") - 1
        assert np.array_equal(own, part["halo_owner"])
    blocks = [torch.zeros((starts[p + 1] - starts[p], 4), dtype=torch.float64)
              for p in range(world)]
    dist.all_gather(blocks, torch.from_numpy(U[:no].copy()))
    if rank == 0:
        np.save(os.path.join(out_dir, "result.npy"), torch.cat(blocks).numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,kind,order", [(2, "periodic", "rcm"), (4, "periodic", "hilbert"),
                                              (3, "channel", "rcm")])
def test_partitioned_run_equals_single_domain(tmp_path, world, kind, order):
    import torch.multiprocessing as mp
    import oracle
    BLD.build()
    oracle.build()
    nsteps = 25
    mp.spawn(_rank_main, args=(world, _free_port(), kind, order, nsteps, str(tmp_path)),
             nprocs=world, join=True)
    got = np.load(tmp_path / "result.npy")
    mi, U0, uinf = _case(kind)
    m = B.Mesh.from_input(mi, "f64")
    perm = m.renumber(order, seed=4)
    nbr, nrm, area = m.export()
    om = oracle.Mesh.from_arrays(nbr, nrm, area, uinf)
    want, *_ = om.run(U0[perm], nsteps, 0.4)
    np.testing.assert_array_equal(got, want)


def test_partition_covers_every_cell_once():
    mi, _, _ = _case("channel")
    m = B.Mesh.from_input(mi, "f32")
    m.renumber("rcm")
    nbr_g, _, _ = m.export()
    seen = []
    for p in range(5):
        part = m.partition(5, p)
        no, gid = part["n_owned"], part["global_ids"]
        seen.append(gid[:no])
        # local neighbour table maps back to the global one
        loc = part["nbr"]
        inner = loc >= 0
        back = np.where(inner, gid[np.maximum(loc, 0)], loc)
        np.testing.assert_array_equal(back, nbr_g[gid[:no]])
        # the halo is exactly the outside neighbours
        outside = nbr_g[gid[:no]]
        outside = outside[(outside >= 0) & ((outside < gid[0]) | (outside > gid[no - 1]))]
        np.testing.assert_array_equal(np.sort(np.unique(outside)), gid[no:])
    allc = np.concatenate(seen)
    np.testing.assert_array_equal(allc, np.arange(m.n))
    with pytest.raises(B.FVError):
        m.partition(3, 3)
