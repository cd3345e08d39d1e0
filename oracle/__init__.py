"""FP64 CPU oracle of the cell-centred Lax-Friedrichs Euler step on triangles.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The library's product path never loads it, and the two share no
code: the arithmetic lives in ``fv_oracle.c`` (plain C, FP64, single thread,
``-ffp-contract=off``), written again from the paper (Nagy et al., Sec. 6:
Eq. 2, Eq. 4, Eq. 5, Eq. 7a-7d and the update equation), with the readings R0-R3
listed at the top of that file.  This module only compiles the C file with the
host compiler, loads it with ctypes and marshals numpy arrays.

Parity pins for every function here live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fv_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

WALL, FARFIELD, EXTRAP = -1, -2, -3
ERRORS = {
    -1: "degenerate triangle",
    -2: "non-manifold edge",
    -3: "open edge without boundary tag",
    -4: "edge collapsed by periodic identification",
    -5: "out of memory",
    -6: "bad input",
}

_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compiles fv_oracle.c into oracle/_build/liboracle.so (host compiler)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["cc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_build_mesh.restype = ctypes.c_int
            lib.orc_build_mesh.argtypes = [ctypes.c_int64, _d, ctypes.c_int64, _i32, _i32,
                                           ctypes.c_int64, _i32, ctypes.c_int32, _i32, _d, _d]
            lib.orc_set_wave_speed.restype = None
            lib.orc_set_wave_speed.argtypes = [ctypes.c_int32]
            lib.orc_face_flux.restype = None
            lib.orc_face_flux.argtypes = [_d, _d, _d, ctypes.c_double, _d]
            lib.orc_ghost.restype = None
            lib.orc_ghost.argtypes = [ctypes.c_int32, _d, _d, _d, _d]
            lib.orc_closure_nparam.restype = ctypes.c_int64
            lib.orc_closure_features.restype = None
            lib.orc_closure_features.argtypes = [_d, _d, _d, _d]
            lib.orc_closure_mlp.restype = ctypes.c_double
            lib.orc_closure_mlp.argtypes = [_d, ctypes.c_int32, _d]
            lib.orc_closure_scale.restype = ctypes.c_double
            lib.orc_closure_scale.argtypes = [_d, ctypes.c_int32, _d, _d, _d]
            lib.orc_residual.restype = ctypes.c_int
            lib.orc_residual.argtypes = [ctypes.c_int64, _i32, _d, _d, _d, _d, _d, ctypes.c_int32,
                                         _d, _d]
            lib.orc_cell_dt_bound.restype = ctypes.c_double
            lib.orc_cell_dt_bound.argtypes = [_d, _d, ctypes.c_double]
            lib.orc_dt.restype = ctypes.c_double
            lib.orc_dt.argtypes = [ctypes.c_int64, _d, _d, _d, ctypes.c_double]
            lib.orc_totals.restype = None
            lib.orc_totals.argtypes = [ctypes.c_int64, _d, _d, _d]
            lib.orc_run.restype = ctypes.c_int
            lib.orc_run.argtypes = [ctypes.c_int64, _i32, _d, _d, _d, _d, ctypes.c_int64,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_int32, _d,
                                    ctypes.c_int32, _d, _i64]
            lib.orc_closure_loss_grad.restype = ctypes.c_double
            lib.orc_closure_loss_grad.argtypes = [ctypes.c_int64, _i32, _d, _d, _d, _d, _d,
                                                  ctypes.c_double, _d, _d, ctypes.c_int32, _d]
            lib.orc_closure_feature_errors.restype = None
            lib.orc_closure_feature_errors.argtypes = [_d, _d, _d, _d]
            lib.orc_closure_scale_interval.restype = ctypes.c_int
            lib.orc_closure_scale_interval.argtypes = [_d, _d, _d, _d, _d]
            lib.orc_closure_face_intervals.restype = None
            lib.orc_closure_face_intervals.argtypes = [ctypes.c_int64, _i32, _d, _d, _d, _d,
                                                       _d, _d, _i32]
            lib.orc_bandwidth.restype = ctypes.c_int64
            lib.orc_bandwidth.argtypes = [ctypes.c_int64, _i32]
            lib.orc_serial_bandwidth.restype = ctypes.c_int64
            lib.orc_serial_bandwidth.argtypes = [ctypes.c_int64, _i32]
            _lib = lib
    return _lib


def _pd(a):
    return None if a is None else a.ctypes.data_as(_d)


def _pi(a):
    return None if a is None else a.ctypes.data_as(_i32)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def _i32a(a):
    return np.ascontiguousarray(a, dtype=np.int32)


NPARAM = 8 * 32 + 32 + 32 * 32 + 32 + 32 + 1


class Mesh:
    """Neighbour table, scaled outward normals and areas built by the oracle.

    ``nbr`` is (n, 3) int32 (negative = boundary kind), ``nrm`` (n, 3, 2) and
    ``vol`` (n,) float64; ``uinf`` the far-field conserved state.
    """

    def __init__(self, xy, tri, canon=None, bnd=None, default_bc=0, uinf=(1.0, 0.0, 0.0, 2.5)):
        lib = _load()
        xy = _f64(xy)
        tri = _i32a(tri)
        n = tri.shape[0]
        canon = None if canon is None else _i32a(canon)
        bnd = np.zeros((0, 3), np.int32) if bnd is None else _i32a(bnd).reshape(-1, 3)
        self.nbr = np.empty((n, 3), np.int32)
        self.nrm = np.empty((n, 3, 2), np.float64)
        self.vol = np.empty(n, np.float64)
        rc = lib.orc_build_mesh(xy.shape[0], _pd(xy), n, _pi(tri), _pi(canon), bnd.shape[0],
                                _pi(bnd), int(default_bc), _pi(self.nbr), _pd(self.nrm),
                                _pd(self.vol))
        if rc != 0:
            raise ValueError(f"oracle mesh build failed: {ERRORS.get(rc, rc)}")
        self.n = n
        self.uinf = _f64(uinf).copy()

    @classmethod
    def from_arrays(cls, nbr, nrm, vol, uinf):
        m = cls.__new__(cls)
        m.nbr = _i32a(nbr).reshape(-1, 3)
        m.nrm = _f64(nrm).reshape(-1, 3, 2)
        m.vol = _f64(vol).reshape(-1)
        m.n = m.nbr.shape[0]
        m.uinf = _f64(uinf).copy()
        return m

    def permuted(self, perm):
        """The same mesh with cells renumbered: new cell i is old cell perm[i]."""
        perm = np.asarray(perm, np.int64)
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)
        nbr = self.nbr[perm].copy()
        inner = nbr >= 0
        nbr[inner] = inv[nbr[inner]]
        return Mesh.from_arrays(nbr, self.nrm[perm], self.vol[perm], self.uinf)

    # -- method ------------------------------------------------------------
    def residual(self, U, theta=None, bf16_acts=False, return_scales=False):
        U = _f64(U, (self.n, 4))
        R = np.empty_like(U)
        sc = np.empty((self.n, 3), np.float64) if return_scales else None
        th = None if theta is None else _f64(theta)
        _load().orc_residual(self.n, _pi(self.nbr), _pd(self.nrm), _pd(self.vol), _pd(self.uinf),
                             _pd(U), _pd(th), int(bf16_acts), _pd(R), _pd(sc))
        return (R, sc) if return_scales else R

    def dt(self, U, cfl):
        U = _f64(U, (self.n, 4))
        return _load().orc_dt(self.n, _pd(self.nrm), _pd(self.vol), _pd(U), float(cfl))

    def totals(self, U):
        U = _f64(U, (self.n, 4))
        out = np.empty(4, np.float64)
        _load().orc_totals(self.n, _pd(self.vol), _pd(U), _pd(out))
        return out

    def run(self, U, nsteps, cfl, t_stop=0.0, scheme=0, theta=None, bf16_acts=False):
        """Advances a copy of U; returns (U, t_advanced, steps_done, bad_flag)."""
        U = _f64(U, (self.n, 4)).copy()
        t = ctypes.c_double(0.0)
        steps = ctypes.c_int64(0)
        th = None if theta is None else _f64(theta)
        bad = _load().orc_run(self.n, _pi(self.nbr), _pd(self.nrm), _pd(self.vol), _pd(self.uinf),
                              _pd(U), int(nsteps), float(cfl), float(t_stop), int(scheme), _pd(th),
                              int(bf16_acts), ctypes.byref(t), ctypes.byref(steps))
        if bad < 0:
            raise MemoryError("oracle run failed to allocate")
        return U, t.value, steps.value, bool(bad)

    def closure_loss_grad(self, U0, Ut, dt, w, theta, bf16_acts=False, grad=True):
        U0 = _f64(U0, (self.n, 4))
        Ut = _f64(Ut, (self.n, 4))
        w = _f64(w)
        th = _f64(theta)
        g = np.empty(NPARAM, np.float64) if grad else None
        loss = _load().orc_closure_loss_grad(self.n, _pi(self.nbr), _pd(self.nrm), _pd(self.vol),
                                             _pd(self.uinf), _pd(U0), _pd(Ut), float(dt), _pd(w),
                                             _pd(th), int(bf16_acts), _pd(g))
        return (loss, g) if grad else loss

    def closure_scale_intervals(self, U, theta):
        """Interval [lo, hi] of every face's scale over the admissible
        bfloat16 roundings of its features and first-layer activations
        (orc_closure_face_intervals), and whether every rounding of the face
        is determined.  Returns (lo, hi, determined), each (n, 3)."""
        U = _f64(U, (self.n, 4))
        th = _f64(theta)
        lo = np.empty((self.n, 3))
        hi = np.empty((self.n, 3))
        det = np.empty((self.n, 3), np.int32)
        _load().orc_closure_face_intervals(self.n, _pi(self.nbr), _pd(self.nrm), _pd(self.uinf),
                                           _pd(U), _pd(th), _pd(lo), _pd(hi), _pi(det))
        return lo, hi, det.astype(bool)

    def bandwidth(self):
        return _load().orc_bandwidth(self.n, _pi(self.nbr))

    def serial_bandwidth(self):
        return _load().orc_serial_bandwidth(self.n, _pi(self.nbr))


# -- single-face helpers -------------------------------------------------------
def set_wave_speed(mode: str):
    """Wave speed of the dissipation for every later oracle call: 'average'
    (the paper's interface averages, the default) or 'max' (larger one-sided
    |u_n| + c)."""
    _load().orc_set_wave_speed({"average": 0, "max": 1}[mode])


def face_flux(UL, UR, n, scale=1.0):
    UL, UR, n = _f64(UL), _f64(UR), _f64(n)
    F = np.empty(4, np.float64)
    _load().orc_face_flux(_pd(UL), _pd(UR), _pd(n), float(scale), _pd(F))
    return F


def ghost(code, UL, n, uinf):
    UL, n, uinf = _f64(UL), _f64(n), _f64(uinf)
    UR = np.empty(4, np.float64)
    _load().orc_ghost(int(code), _pd(UL), _pd(n), _pd(uinf), _pd(UR))
    return UR


def closure_features(UL, UR, n):
    UL, UR, n = _f64(UL), _f64(UR), _f64(n)
    f = np.empty(8, np.float64)
    _load().orc_closure_features(_pd(UL), _pd(UR), _pd(n), _pd(f))
    return f


def closure_scale(theta, UL, UR, n, bf16_acts=False):
    th, UL, UR, n = _f64(theta), _f64(UL), _f64(UR), _f64(n)
    return _load().orc_closure_scale(_pd(th), int(bf16_acts), _pd(UL), _pd(UR), _pd(n))


def closure_mlp(theta, feat, bf16_acts=False):
    th, f = _f64(theta), _f64(feat)
    return _load().orc_closure_mlp(_pd(th), int(bf16_acts), _pd(f))


def cell_dt_bound(U, nrm_cell, vol):
    U, nc = _f64(U), _f64(nrm_cell)
    return _load().orc_cell_dt_bound(_pd(U), _pd(nc), float(vol))


def closure_feature_errors(UL, UR, n):
    """Bounds on the FP32 evaluation error of the eight features of a face."""
    UL, UR, n = _f64(UL), _f64(UR), _f64(n)
    e = np.empty(8, np.float64)
    _load().orc_closure_feature_errors(_pd(UL), _pd(UR), _pd(n), _pd(e))
    return e


def closure_scale_interval(theta, feat, feat_err=None):
    """Interval of the MLP's scale for one feature vector over the admissible
    bfloat16 roundings (orc_closure_scale_interval); feat_err None takes the
    features as exact.  Returns (lo, hi, determined)."""
    th, f = _f64(theta), _f64(feat)
    e = None if feat_err is None else _f64(feat_err)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    det = _load().orc_closure_scale_interval(_pd(th), _pd(f), _pd(e), ctypes.byref(lo),
                                             ctypes.byref(hi))
    return lo.value, hi.value, bool(det)
