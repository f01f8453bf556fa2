"""A slab stand-in for the CPU tests of paper_1711_09272_gb300.slab: the Batch methods the
slab stepper uses, computed with the FP64 oracle on the slab extended by its ghost rows (the
oracle has no EXCHANGE sides; beyond two ghost rows nothing reaches the slab's cells)."""
from dataclasses import replace

import numpy as np

import oracle
import workloads as W

EXCHANGE = 4
CA, CB = (0.0, 0.75, 1.0 / 3.0), (1.0, 0.25, 2.0 / 3.0)


class OracleSlab:
    def __init__(self, spec):
        assert spec.xv is None, "Cartesian slabs only"
        self.spec = spec
        self.ex = [spec.bc[2] == EXCHANGE, spec.bc[3] == EXCHANGE]
        bc = tuple(W.OUTFLOW if b == EXCHANGE else b for b in spec.bc)
        self.plain = replace(spec, bc=bc)
        self.halo = {2: None, 3: None}
        self.U = self.A = self.B = None

    def set_state(self, U, idx=0):
        self.U = np.array(U, dtype=np.float64)

    def get_state(self, idx=0):
        return self.U.copy()

    def max_rate(self):
        return np.array([oracle.OracleGrid(self.plain).max_rate(self.U)])

    def _source(self, stage):
        return (self.U, self.A, self.B)[stage]

    def edge_rows(self, idx, side, stage):
        S = self._source(stage)
        return (S[:, :2] if side == 2 else S[:, -2:]).copy()

    def set_halo(self, idx, side, stage, rows):
        self.halo[side] = np.array(rows, dtype=np.float64)

    def _residual(self, S):
        parts, lo = [], 0
        if self.ex[0]:
            parts.append(self.halo[2])
            lo = 2
        parts.append(S)
        if self.ex[1]:
            parts.append(self.halo[3])
        X = np.concatenate(parts, axis=1)
        ext = replace(self.plain, nj=X.shape[1])
        R = oracle.OracleGrid(ext).residual(X)
        return R[:, lo:lo + S.shape[1]]

    def stage(self, stage, dt):
        S = self._source(stage)
        out = CA[stage] * self.U + CB[stage] * (S + dt * self._residual(S))
        if stage == 0:
            self.A = out
        elif stage == 1:
            self.B = out
        else:
            self.U = out
