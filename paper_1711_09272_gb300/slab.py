"""One 2D grid split into row slabs over several GPUs (one process per GPU).

Each slab is its own libroeam handle whose S/N sides between slabs are EXCHANGE sides
(include/roeam.h): their two ghost rows come from the neighbouring slab. An SSP-RK3 step is
run stage by stage (roeam_rk_stage) with one global time step, CFL / (max over slabs of
roeam_max_rate), and before each stage every slab sends its two edge rows of the state that
stage reads (roeam_edge_rows) to its neighbours, which store them as ghost rows
(roeam_set_halo). This is the one exchange the path has: per stage, 2 rows x 4 variables per
side, plus a max-reduction of the rate per step.

The exchange is pluggable: `LocalExchange` for several slabs held by one process (tests, or a
GPU driving several handles), `DistExchange` for one slab per rank over torch.distributed
(NCCL between GPUs, gloo on the CPU). The slab objects only need the Batch methods set_state,
get_state, max_rate, edge_rows, set_halo and stage.
"""
from __future__ import annotations

from dataclasses import replace
from typing import Callable, Dict, List, Optional, Tuple

import numpy as np

EXCHANGE = 4
SIDE_S, SIDE_N = 2, 3
PERIODIC = 0


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


def partition(spec, parts: int):
    """Slab specs of a workloads.GridSpec-like `spec` and each slab's (down, up) neighbour
    (None at a domain side that keeps its own boundary condition)."""
    if spec.solid is not None and parts > 1:
        raise ValueError("grids with solid cells cannot be split into slabs")
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
        if spec.xv is not None:
            kw.update(xv=spec.xv[j0:j1 + 1], yv=spec.yv[j0:j1 + 1])
        slabs.append((replace(spec, **kw), (j0, j1), down, up))
    return slabs


class LocalExchange:
    """All slabs in this process: messages are handed over directly."""

    def allreduce_max(self, x: float) -> float:
        return float(x)

    def swap(self, outgoing: Dict[Tuple[int, int], np.ndarray], wanted: List[Tuple[int, int, int]]):
        return {(s, side): outgoing[(s, side)] for s, side, _ in wanted}


class DistExchange:
    """One slab per rank (slab index = rank) over torch.distributed. Messages carry the
    receiving side as tag, so a pair of ranks that are each other's up and down neighbour
    (two periodic slabs) keeps the two directions apart."""

    def __init__(self, torch, device: Optional[str] = None):
        self.torch = torch
        self.dist = torch.distributed
        self.device = device

    def _t(self, a):
        t = self.torch.from_numpy(np.ascontiguousarray(a))
        return t.to(self.device) if self.device else t

    def allreduce_max(self, x: float) -> float:
        t = self._t(np.array([x], dtype=np.float64))
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.cpu().numpy()[0])

    def swap(self, outgoing, wanted):
        reqs, inbox = [], {}
        for (dst, side), rows in outgoing.items():
            reqs.append(self.dist.isend(self._t(rows), dst=dst, tag=side))
        for me, side, src in wanted:
            buf = self._t(np.empty_like(next(iter(outgoing.values()))))
            inbox[(me, side)] = buf
            reqs.append(self.dist.irecv(buf, src=src, tag=side))
        for q in reqs:
            q.wait()
        return {k: v.cpu().numpy() for k, v in inbox.items()}


class SlabStepper:
    """Advances one grid split into `parts` row slabs; this process owns the slabs `mine`.

    make_slab(slab_spec) -> an object with the Batch methods (a one-grid libroeam Batch by
    default)."""

    def __init__(self, spec, parts: int, mine: List[int], exchange, make_slab: Optional[Callable] = None,
                 precision: int = 64, device: int = 0):
        self.spec = spec
        self.slabs = partition(spec, parts)
        self.mine = list(mine)
        self.ex = exchange
        if make_slab is None:
            from .roeam import Batch

            def make_slab(s):
                return Batch([s], precision=precision, device=device)
        self.handles = {r: make_slab(self.slabs[r][0]) for r in self.mine}

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

    def _refresh_halos(self, stage: int):
        outgoing, wanted = {}, []
        for r in self.mine:
            _, _, down, up = self.slabs[r]
            h = self.handles[r]
            if down is not None:
                outgoing[(down, SIDE_N)] = h.edge_rows(0, SIDE_S, stage)
                wanted.append((r, SIDE_S, down))
            if up is not None:
                outgoing[(up, SIDE_S)] = h.edge_rows(0, SIDE_N, stage)
                wanted.append((r, SIDE_N, up))
        if not wanted:
            return
        inbox = self.ex.swap(outgoing, wanted)
        for (r, side), rows in inbox.items():
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
                self._refresh_halos(s)
                for r in self.mine:
                    self.handles[r].stage(s, dt)
        return dt
