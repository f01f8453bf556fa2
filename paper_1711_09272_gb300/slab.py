"""One 2D grid split into row slabs over several GPUs (one process per GPU).

Each slab is its own libroeam handle whose S/N sides between slabs are EXCHANGE sides
(include/roeam.h): their two ghost rows come from the neighbouring slab. An SSP-RK3 step is
run stage by stage with one global time step, CFL / (max over slabs of roeam_max_rate); before
each stage every slab sends its two edge rows of the state that stage reads (roeam_edge_rows)
to its neighbours, which store them as ghost rows (roeam_set_halo). This is the one exchange
the path has: per stage, 2 rows x 4 variables per side, plus a max-reduction of the rate per
step. With `overlap` (the default) a stage runs as two launches (roeam_rk_stage_part): the
slab's interior, whose stencils stay inside the slab, starts while the ghost rows are in
flight, and the rows next to the EXCHANGE sides follow once they have landed.

What does not change from step to step is set once: the solid-mask rows and (curvilinear
grids) the vertex rows beyond each EXCHANGE side (roeam_set_halo_solid / _vertices). A
curvilinear slab's coordinates are shifted by -j0 dy (j0 its first row), so that the library
stores small displacements from its reference grid, as it does for the whole grid.

The exchange is pluggable: `LocalExchange` for several slabs held by one process (tests, or a
GPU driving several handles), `DistExchange` for one slab per rank over torch.distributed
(NCCL between GPUs, with the rows in device memory; gloo on the CPU). The slab objects only
need the Batch methods set_state, get_state, max_rate, edge_rows, set_halo, stage, stage_part,
set_halo_solid and set_halo_vertices.
"""
from __future__ import annotations

from dataclasses import replace
from typing import Callable, Dict, List, Optional, Tuple

import numpy as np

EXCHANGE = 4
SIDE_S, SIDE_N = 2, 3
PERIODIC = 0
PART_ALL, PART_INTERIOR, PART_EDGES = 0, 1, 2


def slab_rows(nj: int, parts: int) -> List[Tuple[int, int]]:
    """Row ranges [j0, j1) of `parts` slabs of nearly equal height (each >= 4 rows)."""
    if parts < 1 or nj < 4 * parts:
        raise ValueError(f"{nj} rows cannot make {parts} slabs of at least 4 rows")
    base, rem = divmod(nj, parts)
    out, j = [], 0
    for r in range(parts):
        h = base + (1 if r < rem else 0)
        out.append((j, j + h))
        j += h
    return out


def _vertex_rows(spec, J0: int, count: int, shift: float) -> Tuple[np.ndarray, np.ndarray]:
    """Vertex rows J0 .. J0 + count - 1 of a curvilinear spec (rows outside 0..nj wrap through
    the periodic displacement from the reference grid), y shifted by `shift`."""
    nj, ni = spec.nj, spec.ni
    I = np.arange(ni + 1) * spec.dx
    xs, ys = [], []
    for J in range(J0, J0 + count):
        if 0 <= J <= nj:
            xs.append(spec.xv[J].astype(np.float64))
            ys.append(spec.yv[J].astype(np.float64) - shift)
        else:
            Jw = J % nj
            dX = spec.xv[Jw] - I
            dY = spec.yv[Jw] - Jw * spec.dy
            xs.append(I + dX)
            ys.append(J * spec.dy + dY - shift)
    return np.stack(xs), np.stack(ys)


def partition(spec, parts: int):
    """Slab specs of a workloads.GridSpec-like `spec`, each slab's (down, up) neighbour (None at
    a domain side that keeps its own boundary condition) and its static ghost rows: a dict with
    'solid' {side: (2, ni) uint8} and 'vertices' {side: (xv, yv) of shape (2, ni + 1)}."""
    rows = slab_rows(spec.nj, parts)
    periodic = spec.bc[2] == PERIODIC
    slabs = []
    for r, (j0, j1) in enumerate(rows):
        down = r - 1 if r > 0 else (parts - 1 if periodic and parts > 1 else None)
        up = r + 1 if r < parts - 1 else (0 if periodic and parts > 1 else None)
        bc = list(spec.bc)
        if down is not None:
            bc[2] = EXCHANGE
        if up is not None:
            bc[3] = EXCHANGE
        kw = dict(nj=j1 - j0, bc=tuple(bc))
        ghosts = {"solid": {}, "vertices": {}}
        shift = j0 * spec.dy
        if spec.xv is not None:
            kw.update(xv=np.ascontiguousarray(spec.xv[j0:j1 + 1], dtype=np.float64),
                      yv=np.ascontiguousarray(spec.yv[j0:j1 + 1], dtype=np.float64) - shift)
        if spec.solid is not None:
            kw.update(solid=np.ascontiguousarray(spec.solid[j0:j1], dtype=np.uint8))
        for side, is_ex, jrows, jverts in ((SIDE_S, down is not None, (j0 - 2, j0 - 1), j0 - 2),
                                           (SIDE_N, up is not None, (j1, j1 + 1), j1 + 1)):
            if not is_ex:
                continue
            if spec.solid is not None:
                ghosts["solid"][side] = np.stack([spec.solid[j % spec.nj] for j in jrows]).astype(np.uint8)
            if spec.xv is not None:
                ghosts["vertices"][side] = _vertex_rows(spec, jverts, 2, shift)
        slabs.append((replace(spec, **kw), (j0, j1), down, up, ghosts))
    return slabs


class LocalExchange:
    """All slabs in this process: messages are handed over directly."""

    def allreduce_max(self, x: float) -> float:
        return float(x)

    def buffer(self, like):
        return None   # the slab's own edge_rows allocates host rows

    def post(self, outgoing: Dict[Tuple[int, int], object], wanted: List[Tuple[int, int, int]]):
        return {(s, side): outgoing[(s, side)] for s, side, _ in wanted}

    def complete(self, pending):
        return pending


class DistExchange:
    """One slab per rank (slab index = rank) over torch.distributed. Messages carry the
    receiving side as tag, so a pair of ranks that are each other's up and down neighbour
    (two periodic slabs) keeps the two directions apart. With `device` (e.g. "cuda:0") the
    rows stay in device memory: roeam_edge_rows writes them into a device tensor, NCCL moves
    them, and roeam_set_halo reads them there; completion is a stream dependency, not a host
    wait, so the interior launch queued meanwhile overlaps the transfer."""

    def __init__(self, torch, device: Optional[str] = None, dtype=None):
        self.torch = torch
        self.dist = torch.distributed
        self.device = device
        self.dtype = dtype

    def _t(self, a):
        if hasattr(a, "data_ptr"):
            return a
        t = self.torch.from_numpy(np.ascontiguousarray(a))
        return t.to(self.device) if self.device else t

    def buffer(self, shape_dtype):
        """A device tensor for one message of (shape, numpy dtype), or None (host rows)."""
        if not self.device:
            return None
        shape, dt = shape_dtype
        tdt = self.torch.float32 if dt == np.float32 else self.torch.float64
        return self.torch.empty(shape, dtype=tdt, device=self.device)

    def allreduce_max(self, x: float) -> float:
        t = self._t(np.array([x], dtype=np.float64))
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.cpu().numpy()[0])

    def post(self, outgoing, wanted):
        reqs, inbox, keep = [], {}, []
        like = next(iter(outgoing.values()))
        for (dst, side), rows in outgoing.items():
            t = self._t(rows)
            keep.append(t)
            reqs.append(self.dist.isend(t, dst=dst, tag=side))
        for me, side, src in wanted:
            buf = self.torch.empty_like(self._t(like))
            inbox[(me, side)] = buf
            reqs.append(self.dist.irecv(buf, src=src, tag=side))
        return reqs, inbox, keep

    def complete(self, pending):
        reqs, inbox, _ = pending
        for q in reqs:
            q.wait()
        if self.device:
            return inbox
        return {k: v.numpy() for k, v in inbox.items()}


class SlabStepper:
    """Advances one grid split into `parts` row slabs; this process owns the slabs `mine`.

    make_slab(slab_spec) -> an object with the Batch methods (a one-grid libroeam Batch by
    default)."""

    def __init__(self, spec, parts: int, mine: List[int], exchange, make_slab: Optional[Callable] = None,
                 precision: int = 64, device: int = 0, overlap: bool = True):
        self.spec = spec
        self.slabs = partition(spec, parts)
        self.mine = list(mine)
        self.ex = exchange
        self.overlap = overlap
        self.precision = precision
        if make_slab is None:
            from .roeam import Batch

            def make_slab(s):
                return Batch([s], precision=precision, device=device)
        self.handles = {r: make_slab(self.slabs[r][0]) for r in self.mine}
        for r in self.mine:
            ghosts = self.slabs[r][4]
            for side, rows in ghosts["solid"].items():
                self.handles[r].set_halo_solid(0, side, rows)
            for side, (xv, yv) in ghosts["vertices"].items():
                self.handles[r].set_halo_vertices(0, side, xv, yv)

    def close(self):
        for h in self.handles.values():
            if hasattr(h, "close"):
                h.close()

    def set_state(self, U: np.ndarray):
        """U: the whole grid's state (4, nj, ni); each owned slab takes its rows."""
        for r in self.mine:
            j0, j1 = self.slabs[r][1]
            self.handles[r].set_state(np.ascontiguousarray(U[:, j0:j1]), 0)

    def get_state(self, U_out: np.ndarray) -> np.ndarray:
        """Writes the owned slabs' rows into U_out (4, nj, ni) and returns it."""
        for r in self.mine:
            j0, j1 = self.slabs[r][1]
            U_out[:, j0:j1] = self.handles[r].get_state(0)
        return U_out

    def _post_halos(self, stage: int):
        outgoing, wanted = {}, []
        dt = np.float32 if self.precision == 32 else np.float64
        for r in self.mine:
            _, _, down, up, _ = self.slabs[r]
            h = self.handles[r]
            shape = (4, 2, self.spec.ni)
            if down is not None:
                outgoing[(down, SIDE_N)] = h.edge_rows(0, SIDE_S, stage, self.ex.buffer((shape, dt)))
                wanted.append((r, SIDE_S, down))
            if up is not None:
                outgoing[(up, SIDE_S)] = h.edge_rows(0, SIDE_N, stage, self.ex.buffer((shape, dt)))
                wanted.append((r, SIDE_N, up))
        if not wanted:
            return None
        return self.ex.post(outgoing, wanted)

    def _land_halos(self, stage: int, pending):
        if pending is None:
            return
        for (r, side), rows in self.ex.complete(pending).items():
            self.handles[r].set_halo(0, side, stage, rows)

    def dt(self, cfl: float) -> float:
        local = max(float(self.handles[r].max_rate()[0]) for r in self.mine)
        return cfl / self.ex.allreduce_max(local)

    def step(self, cfl: float = 0.5, nsteps: int = 1, dt_fixed: float = 0.0) -> float:
        """nsteps SSP-RK3 steps; returns the last dt."""
        dt = dt_fixed
        for _ in range(nsteps):
            dt = dt_fixed if dt_fixed > 0 else self.dt(cfl)
            for s in range(3):
                pending = self._post_halos(s)
                if self.overlap:
                    for r in self.mine:
                        self.handles[r].stage_part(s, dt, PART_INTERIOR)
                    self._land_halos(s, pending)
                    for r in self.mine:
                        self.handles[r].stage_part(s, dt, PART_EDGES)
                else:
                    self._land_halos(s, pending)
                    for r in self.mine:
                        self.handles[r].stage(s, dt)
        return dt
