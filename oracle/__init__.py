"""CPU oracle of the Roe-AM finite-volume step (TEST INFRASTRUCTURE).

Only `tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` / reference leg of
`bench.py` may import this package. The product library (`paper_1711_09272_gb300`)
never imports it, and this package never imports the product library: the two
share only the seeded input generators of `workloads`.

The arithmetic lives in `roeam_oracle.c` (plain C, FP64; a second build in long
double bounds its rounding error). This module compiles it with gcc on first use
and marshals numpy arrays through ctypes. See the C file's header for the passages
of the paper each function follows and for the readings taken where the paper is
silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "roeam_oracle.c")
_SRC3 = os.path.join(_HERE, "roeam_oracle3.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS = {}


class OrcParams(C.Structure):
    _fields_ = [("gamma", C.c_double), ("m_ref", C.c_double), ("u_ref", C.c_double), ("eps2", C.c_double),
                ("eps1", C.c_int), ("use_s1", C.c_int), ("recon", C.c_int), ("xi_form", C.c_int),
                ("scheme", C.c_int), ("dup_mode", C.c_int), ("ufix", C.c_int), ("xi_roe", C.c_int),
                ("harten", C.c_double)]


class OrcGrid(C.Structure):
    _fields_ = [("ni", C.c_int), ("nj", C.c_int), ("bc", C.c_int * 4), ("inflow", C.c_double * 4),
                ("xv", C.POINTER(C.c_double)), ("yv", C.POINTER(C.c_double)),
                ("dx", C.c_double), ("dy", C.c_double), ("solid", C.POINTER(C.c_uint8)),
                ("prm", OrcParams)]


class Orc3Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("m_ref", C.c_double), ("u_ref", C.c_double), ("eps2", C.c_double),
                ("eps1", C.c_int), ("use_s1", C.c_int), ("xi_form", C.c_int), ("nscal", C.c_int)]


class Orc3Grid(C.Structure):
    _fields_ = [("ni", C.c_int), ("nj", C.c_int), ("nk", C.c_int), ("bc", C.c_int * 6), ("inflow", C.c_double * 8),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("prm", Orc3Params)]


def build(force: bool = False) -> Tuple[str, str]:
    """Compile the oracle (double and long double builds) into oracle/_build/."""
    os.makedirs(_BUILD, exist_ok=True)
    outs = []
    for tag, flags in (("", []), ("_ld", ["-DORC_LONG=1"])):
        out = os.path.join(_BUILD, f"liboracle{tag}.so")
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC3))
        if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
            tmp = out + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", *flags, "-o", tmp, _SRC, _SRC3,
                                   "-lm"])
            os.replace(tmp, out)
        outs.append(out)
    return outs[0], outs[1]


def _lib(long_double: bool = False):
    key = "ld" if long_double else "d"
    with _LOCK:
        if key not in _LIBS:
            d, ld = build()
            lib = C.CDLL(ld if long_double else d)
            sfx = "_ld" if long_double else ""
            dp = C.POINTER(C.c_double)
            getattr(lib, "orc_f" + sfx).restype = C.c_double
            getattr(lib, "orc_f" + sfx).argtypes = [C.c_double]
            getattr(lib, "orc_face_flux" + sfx).argtypes = [C.POINTER(OrcParams), C.c_int, dp, dp, dp, dp, dp]
            getattr(lib, "orc_roe_average" + sfx).argtypes = [C.c_int, dp, dp, C.c_double, dp]
            getattr(lib, "orc_residual" + sfx).argtypes = [C.POINTER(OrcGrid), dp, dp]
            getattr(lib, "orc_max_rate" + sfx).restype = C.c_double
            getattr(lib, "orc_max_rate" + sfx).argtypes = [C.POINTER(OrcGrid), dp]
            getattr(lib, "orc_rk_step" + sfx).restype = C.c_double
            getattr(lib, "orc_rk_step" + sfx).argtypes = [C.POINTER(OrcGrid), dp, C.c_double, C.c_double]
            getattr(lib, "orc_totals" + sfx).argtypes = [C.POINTER(OrcGrid), dp, dp]
            getattr(lib, "orc_detector" + sfx).argtypes = [C.POINTER(OrcGrid), dp, dp, dp]
            ip = C.POINTER(C.c_int)
            getattr(lib, "orc_face_states" + sfx).argtypes = [C.POINTER(OrcGrid), dp, C.c_int, ip, ip, dp, dp]
            getattr(lib, "orc3_face_flux" + sfx).argtypes = [C.POINTER(Orc3Params), C.c_int, dp, dp, dp, dp, dp]
            getattr(lib, "orc3_residual" + sfx).argtypes = [C.POINTER(Orc3Grid), dp, dp]
            getattr(lib, "orc3_max_rate" + sfx).restype = C.c_double
            getattr(lib, "orc3_max_rate" + sfx).argtypes = [C.POINTER(Orc3Grid), dp]
            getattr(lib, "orc3_rk_step" + sfx).restype = C.c_double
            getattr(lib, "orc3_rk_step" + sfx).argtypes = [C.POINTER(Orc3Grid), dp, C.c_double, C.c_double]
            getattr(lib, "orc3_totals" + sfx).argtypes = [C.POINTER(Orc3Grid), dp, dp]
            getattr(lib, "orc3_detector" + sfx).argtypes = [C.POINTER(Orc3Grid), dp, C.c_int, dp]
            _LIBS[key] = (lib, sfx)
        return _LIBS[key]


def _fn(name: str, long_double: bool = False):
    lib, sfx = _lib(long_double)
    return getattr(lib, name + sfx)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


_PARAM_NAMES = ("gamma", "m_ref", "u_ref", "eps2", "eps1", "use_s1", "recon", "xi_form", "scheme", "dup_mode",
                "ufix", "xi_roe", "harten")


def make_params(p=None, **over) -> OrcParams:
    """Oracle parameter block from a workloads.SchemeParams, with keyword overrides."""
    d = dict(gamma=1.4, m_ref=0.5, u_ref=1.0, eps2=0.05, eps1=0, use_s1=1, recon=0, xi_form=0, scheme=0,
             dup_mode=0, ufix=1, xi_roe=0, harten=0.0)
    if p is not None:
        d.update({k: getattr(p, k) for k in _PARAM_NAMES if hasattr(p, k)})
    unknown = set(over) - set(d)
    if unknown:
        raise TypeError(f"unknown scheme parameters {sorted(unknown)}")
    d.update(over)
    return OrcParams(*(float(d[k]) if k in ("gamma", "m_ref", "u_ref", "eps2", "harten") else int(d[k])
                       for k in _PARAM_NAMES))


class OracleGrid:
    """Holds a workloads.GridSpec in the oracle's C layout (keeps the arrays alive)."""

    def __init__(self, spec, params: Optional[OrcParams] = None, **variant):
        self.spec = spec
        self._xv = None if spec.xv is None else np.ascontiguousarray(spec.xv, dtype=np.float64)
        self._yv = None if spec.yv is None else np.ascontiguousarray(spec.yv, dtype=np.float64)
        self._solid = None if spec.solid is None else np.ascontiguousarray(spec.solid, dtype=np.uint8)
        g = OrcGrid()
        g.ni, g.nj = spec.ni, spec.nj
        g.bc[:] = list(spec.bc)
        g.inflow[:] = list(spec.inflow)
        g.xv = _dptr(self._xv) if self._xv is not None else C.POINTER(C.c_double)()
        g.yv = _dptr(self._yv) if self._yv is not None else C.POINTER(C.c_double)()
        g.dx, g.dy = spec.dx, spec.dy
        g.solid = (self._solid.ctypes.data_as(C.POINTER(C.c_uint8)) if self._solid is not None
                   else C.POINTER(C.c_uint8)())
        g.prm = params if params is not None else make_params(spec.params, **variant)
        self.g = g

    def _u(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        assert U.shape == (4, self.spec.nj, self.spec.ni), U.shape
        return U

    def residual(self, U, long_double: bool = False) -> np.ndarray:
        U = self._u(U)
        R = np.empty_like(U)
        _fn("orc_residual", long_double)(C.byref(self.g), _dptr(U), _dptr(R))
        return R

    def max_rate(self, U) -> float:
        U = self._u(U)
        return _fn("orc_max_rate")(C.byref(self.g), _dptr(U))

    def step(self, U, cfl: float = 0.5, dt_fixed: float = 0.0, nsteps: int = 1,
             long_double: bool = False) -> Tuple[np.ndarray, float]:
        """nsteps SSP-RK3 steps; returns (new state, last dt)."""
        U = self._u(U).copy()
        dt = 0.0
        for _ in range(nsteps):
            dt = _fn("orc_rk_step", long_double)(C.byref(self.g), _dptr(U), cfl, dt_fixed)
        return U, dt

    def totals(self, U) -> np.ndarray:
        U = self._u(U)
        out = np.zeros(4)
        _fn("orc_totals")(C.byref(self.g), _dptr(U), _dptr(out))
        return out

    def face_states(self, U, cells, dirs) -> Tuple[np.ndarray, np.ndarray]:
        """Reconstructed left / right primitives (rho, u, v, p) of the faces between cell
        cells[f] = (i, j) and its +i (dirs[f] = 0) or +j (dirs[f] = 1) neighbour: (n, 4) each."""
        U = self._u(U)
        ij = np.ascontiguousarray(np.asarray(cells, dtype=np.int32).reshape(-1, 2))
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(dirs, dtype=np.int32), (ij.shape[0],)))
        WL = np.zeros((ij.shape[0], 4))
        WR = np.zeros((ij.shape[0], 4))
        ip = C.POINTER(C.c_int)
        _fn("orc_face_states")(C.byref(self.g), _dptr(U), ij.shape[0], ij.ctypes.data_as(ip), d.ctypes.data_as(ip),
                               _dptr(WL), _dptr(WR))
        return WL, WR

    def detector(self, U) -> Tuple[np.ndarray, np.ndarray]:
        U = self._u(U)
        sx = np.empty((self.spec.nj, self.spec.ni + 1))
        sy = np.empty((self.spec.nj + 1, self.spec.ni))
        _fn("orc_detector")(C.byref(self.g), _dptr(U), _dptr(sx), _dptr(sy))
        return sx, sy


def f(phi: float, long_double: bool = False) -> float:
    """Eq. 98 Mach function."""
    return _fn("orc_f", long_double)(float(phi))


def face_flux(WL, WR, nrm, s1=None, params: Optional[OrcParams] = None, long_double: bool = False,
              **variant) -> np.ndarray:
    """Per-unit-length numerical flux for n faces. WL, WR: (n, 4) primitives (rho, u, v, p);
    nrm: (n, 2) unit normals from L to R; s1: (n,) detector values (default 1)."""
    WL = np.ascontiguousarray(np.atleast_2d(WL), dtype=np.float64)
    WR = np.ascontiguousarray(np.atleast_2d(WR), dtype=np.float64)
    nrm = np.ascontiguousarray(np.atleast_2d(nrm), dtype=np.float64)
    n = WL.shape[0]
    s = np.ones(n) if s1 is None else np.ascontiguousarray(np.broadcast_to(s1, (n,)), dtype=np.float64)
    P = params if params is not None else make_params(None, **variant)
    F = np.empty((n, 4))
    _fn("orc_face_flux", long_double)(C.byref(P), n, _dptr(WL), _dptr(WR), _dptr(nrm), _dptr(s), _dptr(F))
    return F


def roe_average(WL, WR, gamma: float = 1.4) -> np.ndarray:
    """(n, 5) array of Roe-averaged (rho, u, v, H, c)."""
    WL = np.ascontiguousarray(np.atleast_2d(WL), dtype=np.float64)
    WR = np.ascontiguousarray(np.atleast_2d(WR), dtype=np.float64)
    out = np.empty((WL.shape[0], 5))
    _fn("orc_roe_average")(WL.shape[0], _dptr(WL), _dptr(WR), gamma, _dptr(out))
    return out


def step_ref(spec, U, cfl=0.5, dt_fixed=0.0, nsteps=1, **variant):
    return OracleGrid(spec, **variant).step(U, cfl, dt_fixed, nsteps)


# ----------------------------------------------------------------------------- 3D with scalars
def make_params3(p=None, nscal: int = 0, **over) -> Orc3Params:
    """3D oracle parameters from a workloads.SchemeParams (gamma, m_ref, u_ref, eps2, eps1,
    use_s1, xi_form), with keyword overrides."""
    d = dict(gamma=1.4, m_ref=0.5, u_ref=1.0, eps2=0.05, eps1=0, use_s1=1, xi_form=0)
    if p is not None:
        d.update({k: getattr(p, k) for k in d if hasattr(p, k)})
    d.update(over)
    return Orc3Params(float(d["gamma"]), float(d["m_ref"]), float(d["u_ref"]), float(d["eps2"]), int(d["eps1"]),
                      int(d["use_s1"]), int(d["xi_form"]), int(nscal))


def face_flux3(WL, WR, nrm, s1=None, nscal: int = 0, long_double: bool = False, **params) -> np.ndarray:
    """Per-unit-area flux for n faces: W (n, 5 + nscal) = (rho, u, v, w, p, k..), unit normals
    (n, 3) from L to R."""
    nv = 5 + nscal
    WL = np.ascontiguousarray(np.atleast_2d(WL), dtype=np.float64)
    WR = np.ascontiguousarray(np.atleast_2d(WR), dtype=np.float64)
    nrm = np.ascontiguousarray(np.atleast_2d(nrm), dtype=np.float64)
    assert WL.shape[1] == nv and nrm.shape[1] == 3
    n = WL.shape[0]
    s = np.ones(n) if s1 is None else np.ascontiguousarray(np.broadcast_to(s1, (n,)), dtype=np.float64)
    P = make_params3(None, nscal, **params)
    F = np.empty((n, nv))
    _fn("orc3_face_flux", long_double)(C.byref(P), n, _dptr(WL), _dptr(WR), _dptr(nrm), _dptr(s), _dptr(F))
    return F


class OracleGrid3:
    """A workloads.GridSpec3 in the 3D oracle's layout."""

    def __init__(self, spec, **over):
        self.spec = spec
        g = Orc3Grid()
        g.ni, g.nj, g.nk = spec.ni, spec.nj, spec.nk
        g.bc[:] = list(spec.bc)
        inflow = list(spec.inflow) + [0.0] * (8 - len(spec.inflow))
        g.inflow[:] = inflow
        g.dx, g.dy, g.dz = spec.dx, spec.dy, spec.dz
        g.prm = make_params3(spec.params, spec.nscal, **over)
        self.g = g
        self.nv = 5 + spec.nscal

    def _u(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        assert U.shape == (self.nv, self.spec.nk, self.spec.nj, self.spec.ni), U.shape
        return U

    def residual(self, U, long_double: bool = False) -> np.ndarray:
        U = self._u(U)
        R = np.empty_like(U)
        _fn("orc3_residual", long_double)(C.byref(self.g), _dptr(U), _dptr(R))
        return R

    def max_rate(self, U) -> float:
        return _fn("orc3_max_rate")(C.byref(self.g), _dptr(self._u(U)))

    def step(self, U, cfl: float = 0.5, dt_fixed: float = 0.0, nsteps: int = 1, long_double: bool = False):
        U = self._u(U).copy()
        dt = 0.0
        for _ in range(nsteps):
            dt = _fn("orc3_rk_step", long_double)(C.byref(self.g), _dptr(U), cfl, dt_fixed)
        return U, dt

    def totals(self, U) -> np.ndarray:
        out = np.zeros(self.nv)
        _fn("orc3_totals")(C.byref(self.g), _dptr(self._u(U)), _dptr(out))
        return out

    def detector(self, U, axis: int) -> np.ndarray:
        U = self._u(U)
        out = np.empty((self.spec.nk, self.spec.nj, self.spec.ni))
        _fn("orc3_detector")(C.byref(self.g), _dptr(U), int(axis), _dptr(out))
        return out
