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

FV_OK, FV_EINVAL, FV_ENOMEM, FV_ECUDA, FV_ENONFINITE, FV_ETIMEOUT = range(6)
FV_F32, FV_F64 = 0, 1
FV_BC_NONE, FV_BC_WALL, FV_BC_FARFIELD, FV_BC_EXTRAP = 0, 1, 2, 3
ORDERS = {"identity": 0, "shuffle": 1, "rcm": 2, "hilbert": 3}
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
    return _build.LIB


def load():
    """Loads the built library (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        sig = {
            "fv_last_error": (ctypes.c_char_p, []),
            "fv_abi_version": (_i32, []),
            "fv_mesh_create": (ctypes.c_int, [_vp, _i64, _vp, _i64, _vp, _vp, _i64, _i32, _i32,
                                              _P(_vp)]),
            "fv_mesh_destroy": (ctypes.c_int, [_vp]),
            "fv_mesh_info": (ctypes.c_int, [_vp, _P(_i64), _P(_i32)]),
            "fv_set_freestream": (ctypes.c_int, [_vp, _dbl, _dbl, _dbl, _dbl]),
            "fv_renumber": (ctypes.c_int, [_vp, _i32, ctypes.c_uint64, _vp]),
            "fv_mesh_diagnostics": (ctypes.c_int, [_vp, _P(_i64), _P(_i64)]),
            "fv_mesh_export": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
            "fv_mesh_upload": (ctypes.c_int, [_vp, _vp]),
            "fv_mesh_set_compensation": (ctypes.c_int, [_vp, _i32]),
            "fv_step": (ctypes.c_int, [_vp, _vp, _i64, _dbl, _dbl, _i32, _vp, _vp, _P(_dbl)]),
            "fv_mesh_status": (ctypes.c_int, [_vp, _vp, _P(_dbl)]),
            "fv_residual": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
            "fv_compute_dt": (ctypes.c_int, [_vp, _vp, _dbl, _vp, _P(_dbl)]),
            "fv_conserved_totals": (ctypes.c_int, [_vp, _vp, _P(_dbl), _vp]),
            "fv_conserved_totals_noalloc": (ctypes.c_int, [_vp, _vp, _i64, _i32, _vp, _vp]),
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
