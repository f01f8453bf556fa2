"""ctypes binding of the libroeam C ABI (include/roeam.h).

Argument marshalling only: every step of the Roe-AM path runs in the library's CUDA
kernels. The module-level functions keep the C names; `Batch` is a small convenience
wrapper that owns a handle. There is no CPU fallback: if the compiled library is
missing or no GPU is present, the calls fail loudly.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libroeam.so")
DEBUG_LIB_PATH = os.path.join(HERE, "_build_debug", "libroeam.so")   # bounds-checked build (build(debug=True))

ROEAM_OK, ROEAM_E_ARG, ROEAM_E_CUDA, ROEAM_E_OOM, ROEAM_E_NONPOSITIVE, ROEAM_E_NONFINITE, ROEAM_E_TIMEOUT, \
    ROEAM_E_STATE, ROEAM_E_BOUNDS = range(9)
STATUS_NAMES = ["OK", "E_ARG", "E_CUDA", "E_OOM", "E_NONPOSITIVE", "E_NONFINITE", "E_TIMEOUT", "E_STATE",
                "E_BOUNDS"]
ROEAM_NORM_L2, ROEAM_NORM_LINF = 0, 1

# Entry points declared in include/roeam.h (checked by the tests).
EXPORTS = ["roeam_create_grid", "roeam_destroy_grid", "roeam_set_state", "roeam_get_state", "roeam_set_state_device",
           "roeam_get_state_device", "roeam_flux_residual",
           "roeam_rk_step", "roeam_residual_norm", "roeam_conserved_totals", "roeam_check", "roeam_launch_count",
           "roeam_cell_count", "roeam_last_error", "roeam_version", "roeam_tile_config_count",
           "roeam_tile_config_info", "roeam_set_tile_config", "roeam_autotune", "roeam_flux_residual_noalloc",
           "roeam_rk_stage", "roeam_rk_stage_part", "roeam_max_rate", "roeam_edge_rows", "roeam_set_halo",
           "roeam_set_halo_solid", "roeam_set_halo_vertices", "roeam_math_check", "roeam_step_host",
           "roeam_set_state_f32", "roeam_get_state_f32", "roeam_step_host_f32",
           "roeam3_create_grid", "roeam3_destroy_grid", "roeam3_set_state", "roeam3_get_state",
           "roeam3_flux_residual", "roeam3_rk_step", "roeam3_conserved_totals", "roeam3_check",
           "roeam3_launch_count"]


class RoeamError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"roeam {STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")


class roeam_params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("m_ref", C.c_double), ("u_ref", C.c_double), ("eps2", C.c_double),
                ("eps1", C.c_int), ("use_s1", C.c_int), ("recon", C.c_int), ("xi_form", C.c_int),
                ("precision", C.c_int), ("scheme", C.c_int), ("dup_mode", C.c_int), ("no_ufix", C.c_int),
                ("xi_roe", C.c_int), ("reserved_", C.c_int), ("harten", C.c_double)]


class roeam_grid_desc(C.Structure):
    _fields_ = [("ni", C.c_int), ("nj", C.c_int), ("bc", C.c_int * 4), ("inflow", C.c_double * 4),
                ("xv", C.POINTER(C.c_double)), ("yv", C.POINTER(C.c_double)), ("dx", C.c_double),
                ("dy", C.c_double), ("solid", C.POINTER(C.c_uint8)), ("p", roeam_params)]


class roeam3_grid_desc(C.Structure):
    _fields_ = [("ni", C.c_int), ("nj", C.c_int), ("nk", C.c_int), ("bc", C.c_int * 6), ("inflow", C.c_double * 8),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("nscal", C.c_int),
                ("reserved_", C.c_int), ("p", roeam_params)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libroeam.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libroeam.so not found at {path}; build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    vp, dp = C.c_void_p, C.POINTER(C.c_double)
    lib.roeam_create_grid.argtypes = [C.c_int, C.POINTER(roeam_grid_desc), C.c_int, vp, C.POINTER(vp)]
    lib.roeam_destroy_grid.argtypes = [vp]
    lib.roeam_destroy_grid.restype = None
    lib.roeam_set_state.argtypes = [vp, C.c_int, vp]
    lib.roeam_get_state.argtypes = [vp, C.c_int, vp]
    lib.roeam_set_state_device.argtypes = [vp, C.c_int, vp, vp]
    lib.roeam_get_state_device.argtypes = [vp, C.c_int, vp, vp]
    lib.roeam_flux_residual.argtypes = [vp, C.c_int, vp]
    lib.roeam_rk_step.argtypes = [vp, C.c_double, C.c_double, C.c_int, vp]
    lib.roeam_residual_norm.argtypes = [vp, C.c_int, C.c_int, dp]
    lib.roeam_conserved_totals.argtypes = [vp, C.c_int, dp]
    lib.roeam_check.argtypes = [vp]
    lib.roeam_launch_count.argtypes = [vp]
    lib.roeam_launch_count.restype = C.c_ulonglong
    lib.roeam_cell_count.argtypes = [vp, C.c_int]
    lib.roeam_cell_count.restype = C.c_longlong
    lib.roeam_last_error.restype = C.c_char_p
    lib.roeam_version.restype = C.c_int
    lib.roeam_tile_config_count.restype = C.c_int
    lib.roeam_tile_config_info.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.roeam_set_tile_config.argtypes = [vp, C.c_int]
    lib.roeam_autotune.argtypes = [vp, C.c_double, C.c_int, C.POINTER(C.c_int), dp]
    lib.roeam_flux_residual_noalloc.argtypes = [vp, C.c_int, vp]
    lib.roeam_rk_stage.argtypes = [vp, C.c_int, C.c_double]
    lib.roeam_rk_stage_part.argtypes = [vp, C.c_int, C.c_double, C.c_int]
    lib.roeam_set_halo_solid.argtypes = [vp, C.c_int, C.c_int, vp]
    lib.roeam_set_halo_vertices.argtypes = [vp, C.c_int, C.c_int, vp, vp]
    lib.roeam_math_check.argtypes = [C.c_int, C.c_int, dp, dp]
    lib.roeam_step_host.argtypes = [vp, C.c_double, C.c_double, C.c_int, vp, vp, vp]
    lib.roeam_step_host_f32.argtypes = [vp, C.c_double, C.c_double, C.c_int, vp, vp, vp]
    lib.roeam_set_state_f32.argtypes = [vp, C.c_int, vp]
    lib.roeam_get_state_f32.argtypes = [vp, C.c_int, vp]
    lib.roeam_max_rate.argtypes = [vp, dp]
    lib.roeam_edge_rows.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp]
    lib.roeam_set_halo.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp]
    lib.roeam3_create_grid.argtypes = [C.c_int, C.POINTER(roeam3_grid_desc), C.c_int, vp, C.POINTER(vp)]
    lib.roeam3_destroy_grid.argtypes = [vp]
    lib.roeam3_destroy_grid.restype = None
    lib.roeam3_set_state.argtypes = [vp, C.c_int, vp]
    lib.roeam3_get_state.argtypes = [vp, C.c_int, vp]
    lib.roeam3_flux_residual.argtypes = [vp, C.c_int, vp]
    lib.roeam3_rk_step.argtypes = [vp, C.c_double, C.c_double, C.c_int, vp]
    lib.roeam3_conserved_totals.argtypes = [vp, C.c_int, dp]
    lib.roeam3_check.argtypes = [vp]
    lib.roeam3_launch_count.argtypes = [vp]
    lib.roeam3_launch_count.restype = C.c_ulonglong
    for name in ("roeam_create_grid", "roeam_set_state", "roeam_get_state", "roeam_set_state_device",
                 "roeam_get_state_device", "roeam_flux_residual", "roeam_rk_step",
                 "roeam_residual_norm", "roeam_conserved_totals", "roeam_check", "roeam_tile_config_info",
                 "roeam_set_tile_config", "roeam_autotune", "roeam_flux_residual_noalloc", "roeam_rk_stage",
                 "roeam_max_rate", "roeam_edge_rows", "roeam_set_halo", "roeam_math_check", "roeam_step_host",
                 "roeam_rk_stage_part", "roeam_set_halo_solid", "roeam_set_halo_vertices", "roeam_step_host_f32",
                 "roeam_set_state_f32", "roeam_get_state_f32",
                 "roeam3_create_grid",
                 "roeam3_set_state", "roeam3_get_state", "roeam3_flux_residual", "roeam3_rk_step",
                 "roeam3_conserved_totals", "roeam3_check"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(st: int):
    if st != ROEAM_OK:
        raise RoeamError(st, _lib.roeam_last_error().decode())


def _ptr(a) -> int:
    """Address of a numpy array or a torch tensor (host, possibly pinned)."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


# ----------------------------------------------------------------------------- C names
def roeam_create_grid(descs: Sequence[roeam_grid_desc], device: int = 0, cuda_stream: int = 0) -> int:
    lib = load_library()
    arr = (roeam_grid_desc * len(descs))(*descs)
    h = C.c_void_p()
    _check(lib.roeam_create_grid(len(descs), arr, device, C.c_void_p(cuda_stream or None), C.byref(h)))
    return h.value


def roeam_destroy_grid(h: int) -> None:
    load_library().roeam_destroy_grid(C.c_void_p(h))


def roeam_set_state(h: int, grid_idx: int, cons) -> None:
    _check(load_library().roeam_set_state(C.c_void_p(h), grid_idx, C.c_void_p(_ptr(cons))))


def roeam_get_state(h: int, grid_idx: int, out) -> None:
    _check(load_library().roeam_get_state(C.c_void_p(h), grid_idx, C.c_void_p(_ptr(out))))


def roeam_set_state_device(h: int, grid_idx: int, cons_dev: int, cuda_stream: int = 0) -> None:
    """cons_dev: address of float64 device memory ([4][nj][ni] per grid); cuda_stream orders
    the call with the caller's work (include/roeam.h)."""
    _check(load_library().roeam_set_state_device(C.c_void_p(h), grid_idx, C.c_void_p(cons_dev),
                                                 C.c_void_p(cuda_stream or None)))


def roeam_get_state_device(h: int, grid_idx: int, cons_out_dev: int, cuda_stream: int = 0) -> None:
    _check(load_library().roeam_get_state_device(C.c_void_p(h), grid_idx, C.c_void_p(cons_out_dev),
                                                 C.c_void_p(cuda_stream or None)))


def roeam_flux_residual(h: int, grid_idx: int, out=None) -> None:
    _check(load_library().roeam_flux_residual(C.c_void_p(h), grid_idx, C.c_void_p(_ptr(out) if out is not None else None)))


def roeam_flux_residual_noalloc(h: int, grid_idx: int, out) -> None:
    """Residual of one grid into `out` without any device allocation by the library (its
    scratch is a fixed array in the library; see include/roeam.h)."""
    _check(load_library().roeam_flux_residual_noalloc(C.c_void_p(h), grid_idx, C.c_void_p(_ptr(out))))


def roeam_rk_step(h: int, cfl: float, dt_fixed: float, nsteps: int, dt_last=None) -> None:
    _check(load_library().roeam_rk_step(C.c_void_p(h), cfl, dt_fixed, nsteps,
                                        C.c_void_p(_ptr(dt_last) if dt_last is not None else None)))


def roeam_residual_norm(h: int, grid_idx: int, kind: int = ROEAM_NORM_L2) -> np.ndarray:
    out = np.zeros(4)
    _check(load_library().roeam_residual_norm(C.c_void_p(h), grid_idx, kind, out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def roeam_conserved_totals(h: int, grid_idx: int) -> np.ndarray:
    out = np.zeros(4)
    _check(load_library().roeam_conserved_totals(C.c_void_p(h), grid_idx, out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def roeam_check(h: int) -> None:
    _check(load_library().roeam_check(C.c_void_p(h)))


def roeam_launch_count(h: int) -> int:
    return int(load_library().roeam_launch_count(C.c_void_p(h)))


def roeam_cell_count(h: int, grid_idx: int = -1) -> int:
    return int(load_library().roeam_cell_count(C.c_void_p(h), grid_idx))


def roeam_version() -> int:
    return int(load_library().roeam_version())


def roeam_tile_config_count() -> int:
    return int(load_library().roeam_tile_config_count())


def roeam_tile_config_info(cfg: int):
    tx, ty, nt = C.c_int(), C.c_int(), C.c_int()
    _check(load_library().roeam_tile_config_info(cfg, C.byref(tx), C.byref(ty), C.byref(nt)))
    return tx.value, ty.value, nt.value


def roeam_set_tile_config(h: int, cfg: int) -> None:
    _check(load_library().roeam_set_tile_config(C.c_void_p(h), cfg))


def roeam_autotune(h: int, cfl: float = 0.5, steps: int = 3):
    """Returns (best tile config, ms per step of every config)."""
    n = roeam_tile_config_count()
    ms = np.zeros(n)
    best = C.c_int()
    _check(load_library().roeam_autotune(C.c_void_p(h), cfl, steps, C.byref(best),
                                         ms.ctypes.data_as(C.POINTER(C.c_double))))
    return best.value, ms


def roeam_step_host(h: int, cfl: float, dt_fixed: float, nsteps: int, cons_in, cons_out, dt_last=None) -> None:
    _check(load_library().roeam_step_host(C.c_void_p(h), cfl, dt_fixed, nsteps, C.c_void_p(_ptr(cons_in)),
                                          C.c_void_p(_ptr(cons_out)),
                                          C.c_void_p(_ptr(dt_last) if dt_last is not None else None)))


def roeam_step_host_f32(h: int, cfl: float, dt_fixed: float, nsteps: int, cons_in, cons_out, dt_last=None) -> None:
    """roeam_step_host with float32 host arrays (numpy float32 or torch float32, pinned or not)."""
    _check(load_library().roeam_step_host_f32(C.c_void_p(h), cfl, dt_fixed, nsteps, C.c_void_p(_ptr(cons_in)),
                                              C.c_void_p(_ptr(cons_out)),
                                              C.c_void_p(_ptr(dt_last) if dt_last is not None else None)))


def roeam_set_state_f32(h: int, grid_idx: int, cons) -> None:
    _check(load_library().roeam_set_state_f32(C.c_void_p(h), grid_idx, C.c_void_p(_ptr(cons))))


def roeam_get_state_f32(h: int, grid_idx: int, out) -> None:
    _check(load_library().roeam_get_state_f32(C.c_void_p(h), grid_idx, C.c_void_p(_ptr(out))))


def roeam_math_check(x, device: int = 0) -> np.ndarray:
    """(n, 6): the kernels' 1/x, 1/sqrt(x), sqrt(x) in FP64 and in FP32 (test hook)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros((x.size, 6))
    _check(load_library().roeam_math_check(device, x.size, x.ctypes.data_as(C.POINTER(C.c_double)),
                                           out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def roeam_rk_stage(h: int, stage: int, dt: float) -> None:
    _check(load_library().roeam_rk_stage(C.c_void_p(h), stage, dt))


ROEAM_PART_ALL, ROEAM_PART_INTERIOR, ROEAM_PART_EDGES = 0, 1, 2


def roeam_rk_stage_part(h: int, stage: int, dt: float, part: int) -> None:
    _check(load_library().roeam_rk_stage_part(C.c_void_p(h), stage, dt, part))


def roeam_set_halo_solid(h: int, grid_idx: int, side: int, rows) -> None:
    rows = np.ascontiguousarray(rows, dtype=np.uint8)
    _check(load_library().roeam_set_halo_solid(C.c_void_p(h), grid_idx, side, C.c_void_p(rows.ctypes.data)))


def roeam_set_halo_vertices(h: int, grid_idx: int, side: int, xv, yv) -> None:
    xv = np.ascontiguousarray(xv, dtype=np.float64)
    yv = np.ascontiguousarray(yv, dtype=np.float64)
    _check(load_library().roeam_set_halo_vertices(C.c_void_p(h), grid_idx, side, C.c_void_p(xv.ctypes.data),
                                                  C.c_void_p(yv.ctypes.data)))


def roeam_max_rate(h: int, count: int) -> np.ndarray:
    out = np.zeros(count)
    _check(load_library().roeam_max_rate(C.c_void_p(h), out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def roeam_edge_rows(h: int, grid_idx: int, side: int, stage: int, dst) -> None:
    _check(load_library().roeam_edge_rows(C.c_void_p(h), grid_idx, side, stage, C.c_void_p(_ptr(dst))))


def roeam_set_halo(h: int, grid_idx: int, side: int, stage: int, src) -> None:
    _check(load_library().roeam_set_halo(C.c_void_p(h), grid_idx, side, stage, C.c_void_p(_ptr(src))))


# ----------------------------------------------------------------------------- convenience
def make_desc(spec, precision: int = 64, keep: Optional[list] = None) -> roeam_grid_desc:
    """Descriptor from any object with the fields of workloads.GridSpec. Arrays it points
    to are appended to `keep` so they outlive the create call."""
    keep = keep if keep is not None else []
    d = roeam_grid_desc()
    d.ni, d.nj = int(spec.ni), int(spec.nj)
    d.bc[:] = [int(b) for b in spec.bc]
    d.inflow[:] = [float(x) for x in spec.inflow]
    if spec.xv is not None:
        xv = np.ascontiguousarray(spec.xv, dtype=np.float64)
        yv = np.ascontiguousarray(spec.yv, dtype=np.float64)
        keep += [xv, yv]
        d.xv = xv.ctypes.data_as(C.POINTER(C.c_double))
        d.yv = yv.ctypes.data_as(C.POINTER(C.c_double))
    d.dx, d.dy = float(spec.dx), float(spec.dy)
    if spec.solid is not None:
        s = np.ascontiguousarray(spec.solid, dtype=np.uint8)
        keep.append(s)
        d.solid = s.ctypes.data_as(C.POINTER(C.c_uint8))
    p = spec.params
    d.p = roeam_params(p.gamma, p.m_ref, p.u_ref, p.eps2, int(p.eps1), int(p.use_s1), int(p.recon),
                       int(p.xi_form), int(precision), int(getattr(p, "scheme", 0)), int(getattr(p, "dup_mode", 0)),
                       0 if int(getattr(p, "ufix", 1)) else 1, int(getattr(p, "xi_roe", 0)), 0,
                       float(getattr(p, "harten", 0.0)))
    return d


class Batch:
    """Owns a libroeam handle for a list of grid specs (workloads.GridSpec-like)."""

    def __init__(self, specs, precision: int = 64, device: int = 0, cuda_stream: int = 0):
        if not isinstance(specs, (list, tuple)):
            specs = [specs]
        self.specs = list(specs)
        keep: list = []
        descs = [make_desc(s, precision, keep) for s in self.specs]
        self.handle = roeam_create_grid(descs, device, cuda_stream)
        self.precision = precision
        self.sizes = [s.ni * s.nj for s in self.specs]
        self.offsets = np.concatenate([[0], np.cumsum([4 * n for n in self.sizes])]).astype(np.int64)

    def close(self):
        if self.handle:
            roeam_destroy_grid(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _shape(self, idx):
        s = self.specs[idx]
        return (4, s.nj, s.ni)

    def set_state(self, U, grid_idx: int = 0):
        if grid_idx < 0:
            roeam_set_state(self.handle, -1, U)
        else:
            U = np.ascontiguousarray(U, dtype=np.float64)
            assert U.shape == self._shape(grid_idx), (U.shape, self._shape(grid_idx))
            roeam_set_state(self.handle, grid_idx, U)

    def set_states(self, Us):
        packed = np.concatenate([np.ascontiguousarray(U, dtype=np.float64).ravel() for U in Us])
        roeam_set_state(self.handle, -1, packed)

    def set_state_device(self, U, grid_idx: int = 0, stream: int = 0):
        """U: a contiguous float64 CUDA tensor (or any object with data_ptr()) holding grid
        grid_idx's state (all grids, concatenated, with -1); stream: a cudaStream_t handle
        (e.g. torch.cuda.current_stream().cuda_stream) that the call is ordered with."""
        roeam_set_state_device(self.handle, grid_idx, U.data_ptr(), stream)

    def get_state_device(self, out, grid_idx: int = 0, stream: int = 0):
        """Writes the state into the float64 CUDA tensor `out` (ordered on `stream`)."""
        roeam_get_state_device(self.handle, grid_idx, out.data_ptr(), stream)
        return out

    def get_state(self, grid_idx: int = 0) -> np.ndarray:
        out = np.empty(self._shape(grid_idx))
        roeam_get_state(self.handle, grid_idx, out)
        return out

    def get_states(self):
        packed = np.empty(int(self.offsets[-1]))
        roeam_get_state(self.handle, -1, packed)
        return [packed[self.offsets[k]:self.offsets[k + 1]].reshape(self._shape(k)) for k in range(len(self.specs))]

    def residual(self, grid_idx: int = 0) -> np.ndarray:
        out = np.empty(self._shape(grid_idx))
        roeam_flux_residual(self.handle, grid_idx, out)
        return out

    def step(self, cfl: float = 0.5, dt_fixed: float = 0.0, nsteps: int = 1, want_dt: bool = False):
        dt = np.zeros(len(self.specs)) if want_dt else None
        roeam_rk_step(self.handle, cfl, dt_fixed, nsteps, dt)
        return dt

    def residual_norm(self, grid_idx: int = 0, kind: int = ROEAM_NORM_L2) -> np.ndarray:
        return roeam_residual_norm(self.handle, grid_idx, kind)

    def totals(self, grid_idx: int = 0) -> np.ndarray:
        return roeam_conserved_totals(self.handle, grid_idx)

    def check(self):
        roeam_check(self.handle)

    def set_tile_config(self, cfg: int):
        roeam_set_tile_config(self.handle, cfg)

    def autotune(self, cfl: float = 0.5, steps: int = 3):
        return roeam_autotune(self.handle, cfl, steps)

    # stage-by-stage stepping of row slabs (EXCHANGE sides; see include/roeam.h)
    def stage(self, stage: int, dt: float):
        roeam_rk_stage(self.handle, stage, dt)

    def stage_part(self, stage: int, dt: float, part: int):
        roeam_rk_stage_part(self.handle, stage, dt, part)

    def set_halo_solid(self, grid_idx: int, side: int, rows):
        """Solid-mask rows (2, ni) beyond EXCHANGE side `side` (static)."""
        roeam_set_halo_solid(self.handle, grid_idx, side, rows)

    def set_halo_vertices(self, grid_idx: int, side: int, xv, yv):
        """Vertex rows (2, ni + 1) beyond EXCHANGE side `side` (static, curvilinear grids)."""
        roeam_set_halo_vertices(self.handle, grid_idx, side, xv, yv)

    def max_rate(self) -> np.ndarray:
        return roeam_max_rate(self.handle, len(self.specs))

    def edge_rows(self, grid_idx: int, side: int, stage: int, out=None):
        """The two rows nearest `side` (2 = S, 3 = N) of the state stage `stage` reads, as
        (4, 2, ni) in the handle's precision; `out` may be a device tensor."""
        s = self.specs[grid_idx]
        if out is None:
            out = np.empty((4, 2, s.ni), dtype=np.float32 if self.precision == 32 else np.float64)
        roeam_edge_rows(self.handle, grid_idx, side, stage, out)
        return out

    def set_halo(self, grid_idx: int, side: int, stage: int, rows):
        """Ghost rows beyond EXCHANGE side `side` of the state stage `stage` reads."""
        if not hasattr(rows, "data_ptr"):
            rows = np.ascontiguousarray(rows, dtype=np.float32 if self.precision == 32 else np.float64)
        roeam_set_halo(self.handle, grid_idx, side, stage, rows)

    @property
    def launches(self) -> int:
        return roeam_launch_count(self.handle)


# ----------------------------------------------------------------------------- 3D (include/roeam3.h)
def roeam3_create_grid(descs: Sequence[roeam3_grid_desc], device: int = 0, cuda_stream: int = 0) -> int:
    lib = load_library()
    arr = (roeam3_grid_desc * len(descs))(*descs)
    h = C.c_void_p()
    _check(lib.roeam3_create_grid(len(descs), arr, device, C.c_void_p(cuda_stream or None), C.byref(h)))
    return h.value


def roeam3_destroy_grid(h: int) -> None:
    load_library().roeam3_destroy_grid(C.c_void_p(h))


def roeam3_set_state(h: int, grid_idx: int, cons) -> None:
    _check(load_library().roeam3_set_state(C.c_void_p(h), grid_idx, C.c_void_p(_ptr(cons))))


def roeam3_get_state(h: int, grid_idx: int, out) -> None:
    _check(load_library().roeam3_get_state(C.c_void_p(h), grid_idx, C.c_void_p(_ptr(out))))


def roeam3_flux_residual(h: int, grid_idx: int, out=None) -> None:
    _check(load_library().roeam3_flux_residual(C.c_void_p(h), grid_idx,
                                               C.c_void_p(_ptr(out) if out is not None else None)))


def roeam3_rk_step(h: int, cfl: float, dt_fixed: float, nsteps: int, dt_last=None) -> None:
    _check(load_library().roeam3_rk_step(C.c_void_p(h), cfl, dt_fixed, nsteps,
                                         C.c_void_p(_ptr(dt_last) if dt_last is not None else None)))


def roeam3_conserved_totals(h: int, grid_idx: int, nv: int) -> np.ndarray:
    out = np.zeros(nv)
    _check(load_library().roeam3_conserved_totals(C.c_void_p(h), grid_idx, out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def roeam3_check(h: int) -> None:
    _check(load_library().roeam3_check(C.c_void_p(h)))


def roeam3_launch_count(h: int) -> int:
    return int(load_library().roeam3_launch_count(C.c_void_p(h)))


def make_desc3(spec, precision: int = 64) -> roeam3_grid_desc:
    """Descriptor from any object with the fields of workloads.GridSpec3."""
    d = roeam3_grid_desc()
    d.ni, d.nj, d.nk = int(spec.ni), int(spec.nj), int(spec.nk)
    d.bc[:] = [int(b) for b in spec.bc]
    inflow = [float(x) for x in spec.inflow] + [0.0] * (8 - len(spec.inflow))
    d.inflow[:] = inflow[:8]
    d.dx, d.dy, d.dz = float(spec.dx), float(spec.dy), float(spec.dz)
    d.nscal = int(spec.nscal)
    p = spec.params
    d.p = roeam_params(p.gamma, p.m_ref, p.u_ref, p.eps2, int(p.eps1), int(p.use_s1), int(p.recon),
                       int(p.xi_form), int(precision), 0, 0, 0, 0, 0, 0.0)
    return d


class Batch3:
    """Owns a libroeam 3D handle for a list of workloads.GridSpec3-like specs."""

    def __init__(self, specs, precision: int = 64, device: int = 0, cuda_stream: int = 0):
        if not isinstance(specs, (list, tuple)):
            specs = [specs]
        self.specs = list(specs)
        self.handle = roeam3_create_grid([make_desc3(s, precision) for s in self.specs], device, cuda_stream)
        self.precision = precision
        self.nv = 5 + self.specs[0].nscal
        sizes = [self.nv * s.ni * s.nj * s.nk for s in self.specs]
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)

    def close(self):
        if self.handle:
            roeam3_destroy_grid(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _shape(self, idx):
        s = self.specs[idx]
        return (self.nv, s.nk, s.nj, s.ni)

    def set_state(self, U, grid_idx: int = 0):
        U = np.ascontiguousarray(U, dtype=np.float64)
        assert U.shape == self._shape(grid_idx), (U.shape, self._shape(grid_idx))
        roeam3_set_state(self.handle, grid_idx, U)

    def set_states(self, Us):
        packed = np.concatenate([np.ascontiguousarray(U, dtype=np.float64).ravel() for U in Us])
        roeam3_set_state(self.handle, -1, packed)

    def get_state(self, grid_idx: int = 0) -> np.ndarray:
        out = np.empty(self._shape(grid_idx))
        roeam3_get_state(self.handle, grid_idx, out)
        return out

    def get_states(self):
        packed = np.empty(int(self.offsets[-1]))
        roeam3_get_state(self.handle, -1, packed)
        return [packed[self.offsets[k]:self.offsets[k + 1]].reshape(self._shape(k)) for k in range(len(self.specs))]

    def residual(self, grid_idx: int = 0) -> np.ndarray:
        out = np.empty(self._shape(grid_idx))
        roeam3_flux_residual(self.handle, grid_idx, out)
        return out

    def step(self, cfl: float = 0.5, dt_fixed: float = 0.0, nsteps: int = 1, want_dt: bool = False):
        dt = np.zeros(len(self.specs)) if want_dt else None
        roeam3_rk_step(self.handle, cfl, dt_fixed, nsteps, dt)
        return dt

    def totals(self, grid_idx: int = 0) -> np.ndarray:
        return roeam3_conserved_totals(self.handle, grid_idx, self.nv)

    def check(self):
        roeam3_check(self.handle)

    @property
    def launches(self) -> int:
        return roeam3_launch_count(self.handle)
