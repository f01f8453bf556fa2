"""A slab stand-in for the CPU tests of paper_1711_09272_gb300.slab: the Batch methods the
slab stepper uses, computed with the FP64 oracle on the slab extended by its ghost rows (the
oracle has no EXCHANGE sides; beyond two ghost rows nothing reaches the slab's cells). Solid
masks and curvilinear vertices of the ghost rows come from set_halo_solid / set_halo_vertices
as they do for the library; the interior part of a stage computes with whatever ghost rows it
holds and keeps only the rows whose stencils stay inside the slab, the edge part the rest."""
from dataclasses import replace

import numpy as np

import oracle
import workloads as W

EXCHANGE = 4
CA, CB = (0.0, 0.75, 1.0 / 3.0), (1.0, 0.25, 2.0 / 3.0)


class OracleSlab:
    def __init__(self, spec):
        self.spec = spec
        self.ex = [spec.bc[2] == EXCHANGE, spec.bc[3] == EXCHANGE]
        bc = tuple(W.OUTFLOW if b == EXCHANGE else b for b in spec.bc)
        self.plain = replace(spec, bc=bc)
        self.H = 2 if spec.params.recon else 1
        ni = spec.ni
        self.halo = {2: np.zeros((4, 2, ni)), 3: np.zeros((4, 2, ni))}
        self.halo_solid = {2: np.zeros((2, ni), np.uint8), 3: np.zeros((2, ni), np.uint8)}
        self.halo_vert = {}
        self.U = self.A = self.B = None
        self.pending = None

    def set_state(self, U, idx=0):
        self.U = np.array(U, dtype=np.float64)

    def get_state(self, idx=0):
        return self.U.copy()

    def max_rate(self):
        return np.array([oracle.OracleGrid(self.plain).max_rate(self.U)])

    def _source(self, stage):
        return (self.U, self.A, self.B)[stage]

    def edge_rows(self, idx, side, stage, out=None):
        S = self._source(stage)
        return (S[:, :2] if side == 2 else S[:, -2:]).copy()

    def set_halo(self, idx, side, stage, rows):
        self.halo[side] = np.array(rows, dtype=np.float64)

    def set_halo_solid(self, idx, side, rows):
        self.halo_solid[side] = np.array(rows, dtype=np.uint8)

    def set_halo_vertices(self, idx, side, xv, yv):
        self.halo_vert[side] = (np.array(xv, dtype=np.float64), np.array(yv, dtype=np.float64))

    def _residual(self, S):
        parts, lo = [], 0
        sol, xs, ys = [], [], []
        sp = self.plain
        if self.ex[0]:
            parts.append(self.halo[2])
            lo = 2
            sol.append(self.halo_solid[2])
            if sp.xv is not None:
                xs.append(self.halo_vert[2][0]); ys.append(self.halo_vert[2][1])
        parts.append(S)
        if sp.solid is not None:
            sol.append(sp.solid)
        if sp.xv is not None:
            xs.append(sp.xv); ys.append(sp.yv)
        if self.ex[1]:
            parts.append(self.halo[3])
            sol.append(self.halo_solid[3])
            if sp.xv is not None:
                # the slab's last vertex row is row nj; the ghost vertex rows are nj+1, nj+2
                xs.append(self.halo_vert[3][0]); ys.append(self.halo_vert[3][1])
        X = np.concatenate(parts, axis=1)
        kw = dict(nj=X.shape[1])
        if sp.solid is not None:
            kw["solid"] = np.ascontiguousarray(np.concatenate(sol, axis=0))
        if sp.xv is not None:
            kw["xv"] = np.ascontiguousarray(np.concatenate(xs, axis=0))
            kw["yv"] = np.ascontiguousarray(np.concatenate(ys, axis=0))
        ext = replace(sp, **kw)
        with np.errstate(all="ignore"):
            R = oracle.OracleGrid(ext).residual(X)
        return R[:, lo:lo + S.shape[1]]

    def _combine(self, stage, dt):
        S = self._source(stage)
        with np.errstate(all="ignore"):
            return CA[stage] * self.U + CB[stage] * (S + dt * self._residual(S))

    def _store(self, stage, out):
        if stage == 0:
            self.A = out
        elif stage == 1:
            self.B = out
        else:
            self.U = out

    def stage(self, stage, dt):
        self._store(stage, self._combine(stage, dt))

    def stage_part(self, stage, dt, part):
        if part == 0:
            return self.stage(stage, dt)
        nj = self.spec.nj
        lo = self.H if self.ex[0] else 0
        hi = nj - self.H if self.ex[1] else nj
        if hi <= lo:
            lo = hi = 0
        out = self._combine(stage, dt)
        if part == 1:
            self.pending = (stage, out[:, lo:hi].copy(), lo, hi)
            return
        st, interior, lo, hi = self.pending
        assert st == stage, "interior part of another stage"
        out[:, lo:hi] = interior
        self.pending = None
        self._store(stage, out)
