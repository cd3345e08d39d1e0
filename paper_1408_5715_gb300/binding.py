"""Thin ctypes binding of the C ABI in ``include/fv.h``.

Argument marshalling only: every step of the method runs in the CUDA library
``_lib/libfvgb300.so``.  Device state arrays are torch tensors (PyTorch is
used for device memory and streams); host arrays are numpy.  If the library
has not been built, loading it raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

FV_OK, FV_EINVAL, FV_ENOMEM, FV_ECUDA, FV_ENONFINITE, FV_ETIMEOUT, FV_ESTATE, FV_EINDEX = range(8)
N_VARIANTS = 8  # step-kernel shapes (fv_mesh_set_variant)
FV_F32, FV_F64 = 0, 1
FV_BC_NONE, FV_BC_WALL, FV_BC_FARFIELD, FV_BC_EXTRAP = 0, 1, 2, 3
ORDERS = {"identity": 0, "shuffle": 1, "rcm": 2, "hilbert": 3, "am1": 4}
SCHEMES = {"fe": 0, "rk2": 1}

_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_dbl = ctypes.c_double
_P = ctypes.POINTER


class FVError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[fv status {code}] {msg}")
        self.code = code


def library_path() -> str:
    """The library this process loads: the bounds-checked build when the
    environment sets FV_LIBRARY=debug, else the normal one."""
    return _build.LIB_DEBUG if os.environ.get("FV_LIBRARY") == "debug" else _build.LIB


def load():
    """Loads the built library (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        sig = {
            "fv_last_error": (ctypes.c_char_p, []),
            "fv_abi_version": (_i32, []),
            "fv_index_checks": (_i32, []),
            "fv_mesh_debug_set_index": (ctypes.c_int, [_vp, _i32, _i64, _i32, _i32, _vp]),
            "fv_mesh_create": (ctypes.c_int, [_vp, _i64, _vp, _i64, _vp, _vp, _i64, _i32, _i32,
                                              _P(_vp)]),
            "fv_mesh_destroy": (ctypes.c_int, [_vp]),
            "fv_mesh_info": (ctypes.c_int, [_vp, _P(_i64), _P(_i32)]),
            "fv_set_freestream": (ctypes.c_int, [_vp, _dbl, _dbl, _dbl, _dbl]),
            "fv_renumber": (ctypes.c_int, [_vp, _i32, ctypes.c_uint64, _vp]),
            "fv_mesh_diagnostics": (ctypes.c_int, [_vp, _P(_i64), _P(_i64)]),
            "fv_mesh_export": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
            "fv_mesh_upload": (ctypes.c_int, [_vp, _vp]),
            "fv_partition_sizes": (ctypes.c_int, [_vp, _i32, _i32, _P(_i64), _P(_i64)]),
            "fv_partition_local": (ctypes.c_int, [_vp, _i32, _i32, _vp, _vp, _vp, _vp, _vp]),
            "fv_mesh_set_compensation": (ctypes.c_int, [_vp, _i32]),
            "fv_mesh_set_remainder": (ctypes.c_int, [_vp, _vp]),
            "fv_mesh_set_variant": (ctypes.c_int, [_vp, _i32]),
            "fv_mesh_set_wait_limit": (ctypes.c_int, [_vp, ctypes.c_uint32]),
            "fv_mesh_set_blocking": (ctypes.c_int, [_vp, _i32, _i32, _i32]),
            "fv_mesh_set_launch_chaining": (ctypes.c_int, [_vp, _i32]),
            "fv_mesh_set_wave_speed": (ctypes.c_int, [_vp, _i32]),
            "fv_mesh_set_closure_engine": (ctypes.c_int, [_vp, _i32]),
            "fv_mesh_set_geometry": (ctypes.c_int, [_vp, _i32]),
            "fv_mesh_get_tiling": (ctypes.c_int, [_vp, _P(_i32), _P(_i32)]),
            "fv_mesh_tile_nodes": (ctypes.c_int, [_vp, _i32, _i64, _vp, _i64, _P(_i64), _vp]),
            "fv_mesh_nodes": (ctypes.c_int, [_vp, _P(_i64), _vp, _P(_i32)]),
            "fv_mesh_tile_halo": (ctypes.c_int, [_vp, _i32, _i64, _vp, _i64, _P(_i64), _P(_i64)]),
            "fv_mesh_autotune": (ctypes.c_int, [_vp, _vp, _i32, _vp, _P(_i32), _P(_dbl)]),
            "fv_step": (ctypes.c_int, [_vp, _vp, _i64, _dbl, _dbl, _i32, _vp, _vp, _P(_dbl)]),
            "fv_mesh_status": (ctypes.c_int, [_vp, _vp, _P(_dbl)]),
            "fv_residual": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
            "fv_compute_dt": (ctypes.c_int, [_vp, _vp, _dbl, _vp, _P(_dbl)]),
            "fv_conserved_totals": (ctypes.c_int, [_vp, _vp, _P(_dbl), _vp]),
            "fv_conserved_totals_noalloc": (ctypes.c_int, [_vp, _vp, _i64, _i32, _vp, _vp]),
            "fv_closure_create": (ctypes.c_int, [_vp, _P(_vp)]),
            "fv_closure_destroy": (ctypes.c_int, [_vp]),
            "fv_closure_set": (ctypes.c_int, [_vp, _vp, _i32, _vp]),
            "fv_closure_eval": (ctypes.c_int, [_vp, _vp, _vp, _i64, _vp]),
            "fv_closure_scales": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
            "fv_closure_loss_grad": (ctypes.c_int, [_vp, _vp, _vp, _dbl, _vp, _vp, _P(_dbl),
                                                    _vp, _vp]),
            "fv_restrict_mean": (ctypes.c_int, [_vp, _i32, _vp, _vp, _i64, _i32, _vp, _i32,
                                                _vp]),
            "fv_adam_step": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, _dbl, _dbl, _dbl, _dbl,
                                            _i64, _vp]),
            "fv_batch_create": (ctypes.c_int, [_vp, _i32, _P(_vp)]),
            "fv_batch_destroy": (ctypes.c_int, [_vp]),
            "fv_batch_info": (ctypes.c_int, [_vp, _P(_i64), _vp]),
            "fv_batch_set_compensation": (ctypes.c_int, [_vp, _i32]),
            "fv_batch_set_remainder": (ctypes.c_int, [_vp, _vp]),
            "fv_batch_set_variant": (ctypes.c_int, [_vp, _i32]),
            "fv_batch_get_variant": (ctypes.c_int, [_vp, _P(_i32)]),
            "fv_batch_step": (ctypes.c_int, [_vp, _vp, _i64, _dbl, _dbl, _i32, _vp, _vp]),
            "fv_batch_totals": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc):
    if rc != FV_OK:
        raise FVError(rc, load().fv_last_error().decode(errors="replace"))


def _remainder_ptr(lo, n):
    """Device pointer of a remainder tensor of 8 bytes per cell, or None."""
    if lo is None:
        return None
    if not lo.is_cuda or not lo.is_contiguous() or lo.numel() * lo.element_size() != 8 * n:
        raise ValueError(f"remainder must be a contiguous CUDA tensor of {8 * n} bytes")
    return _vp(lo.data_ptr())


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(_vp)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return _vp(stream.cuda_stream)


def _dev_ptr(t, dtype, n, what):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous() or t.numel() != 4 * n:
        raise ValueError(f"{what} must be contiguous with {4 * n} values (shape (n, 4))")
    return _vp(t.data_ptr())


class Mesh:
    """A triangle mesh owned by the library (fv_mesh)."""

    def __init__(self, xy, tri, canon=None, bnd=None, default_bc=FV_BC_NONE, precision="f32"):
        lib = load()
        xy = np.ascontiguousarray(xy, np.float64).reshape(-1, 2)
        tri = np.ascontiguousarray(tri, np.int32).reshape(-1, 3)
        canon = None if canon is None else np.ascontiguousarray(canon, np.int32)
        bnd = None if bnd is None else np.ascontiguousarray(bnd, np.int32).reshape(-1, 3)
        prec = {"f32": FV_F32, "f64": FV_F64}[precision]
        h = _vp()
        _check(lib.fv_mesh_create(_np_ptr(xy), xy.shape[0], _np_ptr(tri), tri.shape[0],
                                  _np_ptr(canon), _np_ptr(bnd), 0 if bnd is None else bnd.shape[0],
                                  int(default_bc), prec, ctypes.byref(h)))
        self._h = h
        self.precision = precision
        n = _i64()
        _check(lib.fv_mesh_info(h, ctypes.byref(n), None))
        self.n = int(n.value)

    @classmethod
    def from_input(cls, mi, precision="f32"):
        return cls(mi.xy, mi.tri, mi.canon, mi.bnd, mi.default_bc, precision)

    @property
    def torch_dtype(self):
        import torch
        return torch.float64 if self.precision == "f64" else torch.float32

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(load().fv_mesh_destroy(self._h))
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- host side -------------------------------------------------------------
    def set_freestream(self, rho, u, v, p):
        _check(load().fv_set_freestream(self._h, rho, u, v, p))

    def renumber(self, order="rcm", seed=0):
        perm = np.empty(self.n, np.int32)
        _check(load().fv_renumber(self._h, ORDERS[order], int(seed), _np_ptr(perm)))
        return perm

    def diagnostics(self):
        b, s = _i64(), _i64()
        _check(load().fv_mesh_diagnostics(self._h, ctypes.byref(b), ctypes.byref(s)))
        return int(b.value), int(s.value)

    def export(self):
        nbr = np.empty((self.n, 3), np.int32)
        nrm = np.empty((self.n, 3, 2), np.float64)
        area = np.empty(self.n, np.float64)
        _check(load().fv_mesh_export(self._h, _np_ptr(nbr), _np_ptr(nrm), _np_ptr(area)))
        return nbr, nrm, area

    def set_compensation(self, enable: bool):
        _check(load().fv_mesh_set_compensation(self._h, int(bool(enable))))

    def set_remainder(self, lo):
        """fv_mesh_set_remainder: ``lo`` is a caller-owned CUDA tensor of
        8 bytes per cell (e.g. int16 (n, 4) or uint8 (n, 8)) that carries the
        compensated update's remainder across fv_step calls; None returns to
        the remainder the library zeroes at every call.  The tensor must stay
        alive while it is set."""
        self._lo = lo
        _check(load().fv_mesh_set_remainder(self._h, _remainder_ptr(lo, self.n)))

    def partition(self, nparts, part):
        """Local view of one part: dict with global_ids, halo_owner, nbr,
        normals, area, n_owned (host numpy arrays)."""
        lib = load()
        no, nh = _i64(), _i64()
        _check(lib.fv_partition_sizes(self._h, nparts, part, ctypes.byref(no), ctypes.byref(nh)))
        no, nh = int(no.value), int(nh.value)
        gid = np.empty(no + nh, np.int64)
        owner = np.empty(nh, np.int32)
        nbr = np.empty((no, 3), np.int32)
        nrm = np.empty((no, 3, 2), np.float64)
        area = np.empty(no, np.float64)
        _check(lib.fv_partition_local(self._h, nparts, part, _np_ptr(gid), _np_ptr(owner),
                                      _np_ptr(nbr), _np_ptr(nrm), _np_ptr(area)))
        return dict(n_owned=no, global_ids=gid, halo_owner=owner, nbr=nbr, normals=nrm,
                    area=area)

    # -- device side -----------------------------------------------------------
    def upload(self, stream=None):
        _check(load().fv_mesh_upload(self._h, _stream_ptr(stream)))

    def step(self, U, nsteps, cfl, t_stop=0.0, scheme="fe", closure=None, stream=None, sync=True):
        """Advances U (CUDA tensor (n, 4)) in place; returns the time advanced
        when sync is True (and raises on a bad state), else None."""
        t = _dbl(0.0)
        _check(load().fv_step(self._h, _dev_ptr(U, self.torch_dtype, self.n, "U"), int(nsteps),
                              float(cfl), float(t_stop), SCHEMES[scheme],
                              None if closure is None else closure._h, _stream_ptr(stream),
                              ctypes.byref(t) if sync else None))
        return t.value if sync else None

    def set_variant(self, variant: int):
        _check(load().fv_mesh_set_variant(self._h, int(variant)))

    def set_wait_limit(self, polls: int):
        _check(load().fv_mesh_set_wait_limit(self._h, int(polls)))

    def set_wave_speed(self, mode: str):
        """'average' (the paper's interface averages, default) or 'max'
        (larger one-sided |u_n| + c, Rusanov)."""
        _check(load().fv_mesh_set_wave_speed(self._h, {"average": 0, "max": 1}[mode]))

    def set_closure_engine(self, engine="mma.sync"):
        """Tensor-core engine of the learned closure's MLP: "mma.sync" (warp
        MMAs, the default) or "tcgen05" (128-row MMAs into tensor memory);
        both give the same bits."""
        _check(load().fv_mesh_set_closure_engine(self._h, {"mma.sync": 0, "tcgen05": 1}[engine]))

    def set_geometry(self, form: str):
        """'stored' (precomputed normals and 1/V, default) or 'vertex'
        (normals formed from node coordinates on a fixed-point grid, 1/V read;
        FP32, tile shape).  The first 'vertex' snaps the nodes to the grid."""
        _check(load().fv_mesh_set_geometry(self._h, {"stored": 0, "vertex": 1}[form]))

    def nodes(self):
        """(node coordinates [n_nodes, 2] as the geometry uses them, grid
        exponent e of the spacing 2^e or None when not snapped)."""
        nn, e = _i64(), _i32()
        _check(load().fv_mesh_nodes(self._h, ctypes.byref(nn), None, None))
        xy = np.zeros((max(nn.value, 1), 2), np.float64)
        _check(load().fv_mesh_nodes(self._h, ctypes.byref(nn), _np_ptr(xy), ctypes.byref(e)))
        return xy[:nn.value].copy(), (None if e.value == -2**31 else int(e.value))

    def set_launch_chaining(self, enable: bool):
        """Programmatic dependent launch of the step kernels (default on)."""
        _check(load().fv_mesh_set_launch_chaining(self._h, int(bool(enable))))

    def set_blocking(self, steps_per_launch: int, tile_cells: int = 0, staged: bool = False):
        """1: one launch per step; 2: two forward-Euler steps per launch on
        shared-memory tiles of `tile_cells` cells (0 = 1024; with 1, the tile
        size of the one-step tile shape, 32..2048); staged: tile records by
        bulk copies into double-buffered shared memory."""
        _check(load().fv_mesh_set_blocking(self._h, int(steps_per_launch), int(tile_cells),
                                           int(bool(staged))))

    def tile_nodes(self, tile_cells: int, tile: int):
        """(grid coordinates [n, 2] of the nodes the vertex-geometry tile
        kernel stages for a tile, each cell's three tile-local node ids)."""
        nn = _i64()
        _check(load().fv_mesh_tile_nodes(self._h, int(tile_cells), int(tile), None, 0,
                                         ctypes.byref(nn), None))
        q = np.zeros((max(nn.value, 1), 2), np.int32)
        cells = max(0, min(int(tile_cells), self.n - int(tile) * int(tile_cells)))
        loc = np.zeros((max(cells, 1), 3), np.uint16)
        _check(load().fv_mesh_tile_nodes(self._h, int(tile_cells), int(tile), _np_ptr(q),
                                         nn.value, ctypes.byref(nn), _np_ptr(loc)))
        return q[:nn.value].copy(), loc[:cells].copy()

    def tiling(self):
        """(step-kernel shape, tile size in cells of the tiled shapes)."""
        v, t = _i32(), _i32()
        _check(load().fv_mesh_get_tiling(self._h, ctypes.byref(v), ctypes.byref(t)))
        return int(v.value), int(t.value)

    def tile_halo(self, tile_cells: int, tile: int):
        """(first halo, second halo) of a two-step tile, as global cell ids."""
        n1, n2 = _i64(), _i64()
        _check(load().fv_mesh_tile_halo(self._h, int(tile_cells), int(tile), None, 0,
                                        ctypes.byref(n1), ctypes.byref(n2)))
        ids = np.zeros(max(n1.value + n2.value, 1), np.int32)
        _check(load().fv_mesh_tile_halo(self._h, int(tile_cells), int(tile), _np_ptr(ids), ids.size,
                                        ctypes.byref(n1), ctypes.byref(n2)))
        return ids[:n1.value].copy(), ids[n1.value:n1.value + n2.value].copy()

    def autotune(self, U, scheme="fe", stream=None):
        """Picks the fastest step-kernel shape for this mesh; returns
        (best, microseconds per step of each shape)."""
        best = _i32()
        us = (_dbl * N_VARIANTS)()
        _check(load().fv_mesh_autotune(self._h, _dev_ptr(U, self.torch_dtype, self.n, "U"),
                                       SCHEMES[scheme], _stream_ptr(stream), ctypes.byref(best),
                                       us))
        return int(best.value), list(us)

    def status(self, stream=None):
        t = _dbl(0.0)
        _check(load().fv_mesh_status(self._h, _stream_ptr(stream), ctypes.byref(t)))
        return t.value

    def residual(self, U, closure=None, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(U)
        _check(load().fv_residual(self._h, _dev_ptr(U, self.torch_dtype, self.n, "U"),
                                  _dev_ptr(out, self.torch_dtype, self.n, "R"),
                                  None if closure is None else closure._h, _stream_ptr(stream)))
        return out

    def compute_dt(self, U, cfl, stream=None):
        dt = _dbl(0.0)
        _check(load().fv_compute_dt(self._h, _dev_ptr(U, self.torch_dtype, self.n, "U"),
                                    float(cfl), _stream_ptr(stream), ctypes.byref(dt)))
        return dt.value

    def totals(self, U, stream=None):
        out = (_dbl * 4)()
        _check(load().fv_conserved_totals(self._h, _dev_ptr(U, self.torch_dtype, self.n, "U"),
                                          out, _stream_ptr(stream)))
        return np.array(out[:], np.float64)


CLOSURE_PARAMS = 32 * 8 + 32 + 32 * 32 + 32 + 32 + 1


class Closure:
    """The learned dissipation scale (fv_closure); theta is the flat FP32
    parameter vector W1[32][8], b1, W2[32][32], b2, w3, b3."""

    def __init__(self, theta=None):
        lib = load()
        h = _vp()
        th = None if theta is None else np.ascontiguousarray(theta, np.float32)
        if th is not None and th.size != CLOSURE_PARAMS:
            raise ValueError(f"theta needs {CLOSURE_PARAMS} values")
        _check(lib.fv_closure_create(_np_ptr(th), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(load().fv_closure_destroy(self._h))
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set(self, theta, stream=None):
        """New parameters from a host array or a CUDA float32 tensor."""
        import torch
        if isinstance(theta, torch.Tensor):
            if not theta.is_cuda or theta.dtype != torch.float32 or theta.numel() != CLOSURE_PARAMS:
                raise ValueError("theta tensor must be CUDA float32 with 1377 values")
            _check(load().fv_closure_set(self._h, _vp(theta.data_ptr()), 1, _stream_ptr(stream)))
        else:
            th = np.ascontiguousarray(theta, np.float32)
            _check(load().fv_closure_set(self._h, _np_ptr(th), 0, _stream_ptr(stream)))

    def eval(self, features, out=None, stream=None):
        """Scales of the rows of a CUDA float32 (rows, 8) feature tensor."""
        import torch
        rows = features.shape[0]
        if out is None:
            out = torch.empty(rows, dtype=torch.float32, device=features.device)
        _check(load().fv_closure_eval(self._h, _vp(features.data_ptr()), _vp(out.data_ptr()),
                                      rows, _stream_ptr(stream)))
        return out

    def scales(self, mesh, U, out=None, stream=None):
        """Per-face scales (n, 3) the step would use for state U."""
        import torch
        if out is None:
            out = torch.empty((mesh.n, 3), dtype=torch.float32, device=U.device)
        _check(load().fv_closure_scales(mesh._h, _dev_ptr(U, mesh.torch_dtype, mesh.n, "U"),
                                        self._h, _vp(out.data_ptr()), _stream_ptr(stream)))
        return out

    def loss_grad(self, mesh, U0, Ut, dt, weights=(1.0, 1.0, 1.0, 1.0), grad=None, stream=None):
        """One-step training loss (host float) and its gradient (CUDA float32
        tensor of 1377 values)."""
        import torch
        if grad is None:
            grad = torch.empty(CLOSURE_PARAMS, dtype=torch.float32, device=U0.device)
        w = np.ascontiguousarray(weights, np.float64)
        loss = _dbl(0.0)
        _check(load().fv_closure_loss_grad(mesh._h, _dev_ptr(U0, mesh.torch_dtype, mesh.n, "U0"),
                                           _dev_ptr(Ut, mesh.torch_dtype, mesh.n, "Ut"),
                                           float(dt), _np_ptr(w), self._h, ctypes.byref(loss),
                                           _vp(grad.data_ptr()), _stream_ptr(stream)))
        return loss.value, grad


def adam_step(theta, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """In-place Adam update of CUDA float32 tensors (fv_adam_step)."""
    n = theta.numel()
    _check(load().fv_adam_step(_vp(theta.data_ptr()), _vp(grad.data_ptr()), _vp(m.data_ptr()),
                               _vp(v.data_ptr()), n, lr, beta1, beta2, eps, int(step),
                               _stream_ptr(stream)))


class Batch:
    """Many meshes advanced together (fv_batch).  ``offsets[k]`` is the first
    record of mesh k in the flattened state of ``n_padded`` records."""

    def __init__(self, meshes):
        lib = load()
        if not meshes:
            raise ValueError("need at least one mesh")
        arr = (_vp * len(meshes))(*[m._h for m in meshes])
        h = _vp()
        _check(lib.fv_batch_create(arr, len(meshes), ctypes.byref(h)))
        self._h = h
        self.precision = meshes[0].precision
        self.n_meshes = len(meshes)
        self.sizes = [m.n for m in meshes]
        n = _i64()
        off = np.empty(self.n_meshes + 1, np.int64)
        _check(lib.fv_batch_info(h, ctypes.byref(n), _np_ptr(off)))
        self.n_padded = int(n.value)
        self.offsets = off

    @property
    def torch_dtype(self):
        import torch
        return torch.float64 if self.precision == "f64" else torch.float32

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(load().fv_batch_destroy(self._h))
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pack(self, states):
        """Host: flattened (n_padded, 4) array from per-mesh (n_k, 4) arrays."""
        out = np.zeros((self.n_padded, 4), np.float64)
        for k, U in enumerate(states):
            out[self.offsets[k]:self.offsets[k] + self.sizes[k]] = U
        return out

    def unpack(self, flat):
        return [flat[self.offsets[k]:self.offsets[k] + self.sizes[k]] for k in range(self.n_meshes)]

    def set_compensation(self, enable: bool):
        _check(load().fv_batch_set_compensation(self._h, int(bool(enable))))

    def set_remainder(self, lo):
        """fv_batch_set_remainder: as Mesh.set_remainder, 8 bytes per cell of
        the padded batch (``n_padded`` cells)."""
        self._lo = lo
        _check(load().fv_batch_set_remainder(self._h, _remainder_ptr(lo, self.n_padded)))

    def set_variant(self, variant: int):
        _check(load().fv_batch_set_variant(self._h, int(variant)))

    def variant(self) -> int:
        """Kernel shape of the batch (-1 until the first device call)."""
        v = _i32()
        _check(load().fv_batch_get_variant(self._h, ctypes.byref(v)))
        return int(v.value)

    def step(self, U, nsteps, cfl, t_stop=0.0, scheme="fe", stream=None, sync=True):
        """Advances the flattened CUDA state U in place; returns each mesh's
        time advanced (numpy array) when sync is True."""
        t = np.zeros(self.n_meshes, np.float64) if sync else None
        _check(load().fv_batch_step(self._h, _dev_ptr(U, self.torch_dtype, self.n_padded, "U"),
                                    int(nsteps), float(cfl), float(t_stop), SCHEMES[scheme],
                                    _stream_ptr(stream), _np_ptr(t)))
        return t

    def totals(self, U, stream=None):
        out = np.empty((self.n_meshes, 4), np.float64)
        _check(load().fv_batch_totals(self._h, _dev_ptr(U, self.torch_dtype, self.n_padded, "U"),
                                      _np_ptr(out), _stream_ptr(stream)))
        return out


def restrict_mean(U_fine, area_fine, fine_of, U_coarse, stream=None):
    """fv_restrict_mean: coarse cell c of the CUDA tensor U_coarse ((n_c, 4),
    float32/float64) gets the area-weighted mean of the fine states
    U_fine[fine_of[c, :]] (CUDA int32 (n_c, children); areas: CUDA float64)."""
    import torch
    for t, what in ((U_fine, "U_fine"), (U_coarse, "U_coarse")):
        if t.dtype not in (torch.float32, torch.float64) or not t.is_cuda \
                or not t.is_contiguous() or t.dim() != 2 or t.shape[1] != 4:
            raise TypeError(f"{what} must be a contiguous CUDA (n, 4) float32/float64 tensor")
    if fine_of.dtype != torch.int32 or not fine_of.is_cuda or not fine_of.is_contiguous() \
            or fine_of.dim() != 2 or fine_of.shape[0] != U_coarse.shape[0]:
        raise TypeError("fine_of must be a contiguous CUDA int32 (n_coarse, children) tensor")
    if area_fine.dtype != torch.float64 or not area_fine.is_cuda \
            or area_fine.numel() != U_fine.shape[0]:
        raise TypeError("area_fine must be a CUDA float64 tensor of one area per fine cell")
    prec = {torch.float32: FV_F32, torch.float64: FV_F64}
    _check(load().fv_restrict_mean(_vp(U_fine.data_ptr()), prec[U_fine.dtype],
                                   _vp(area_fine.data_ptr()), _vp(fine_of.data_ptr()),
                                   int(U_coarse.shape[0]), int(fine_of.shape[1]),
                                   _vp(U_coarse.data_ptr()), prec[U_coarse.dtype],
                                   _stream_ptr(stream)))
    return U_coarse


def conserved_totals_noalloc(U, area, out, stream=None):
    """fv_conserved_totals_noalloc: totals of the CUDA state U ((n, 4), float32
    or float64) weighted by the CUDA cell areas ``area`` ((n,), float64), into
    the CUDA float64 tensor ``out`` (4 values).  Allocates no device memory
    and does not synchronise."""
    import torch
    if U.dtype not in (torch.float32, torch.float64) or not U.is_cuda or not U.is_contiguous():
        raise TypeError("U must be a contiguous CUDA float32/float64 tensor")
    n = U.numel() // 4
    if U.numel() != 4 * n:
        raise ValueError("U must have shape (n, 4)")
    for t, what, cnt in ((area, "area", n), (out, "out", 4)):
        if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != cnt:
            raise ValueError(f"{what} must be a contiguous CUDA float64 tensor of {cnt} values")
    prec = FV_F64 if U.dtype == torch.float64 else FV_F32
    _check(load().fv_conserved_totals_noalloc(_vp(U.data_ptr()), _vp(area.data_ptr()), n, prec,
                                              _vp(out.data_ptr()), _stream_ptr(stream)))
