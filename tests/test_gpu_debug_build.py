"""The bounds-checked debug build (ROEAM_DEBUG): every state, mask and vertex access of the 2D
stage kernels is checked against its buffer and a bad index is reported (ROEAM_E_BOUNDS)
instead of faulting. The tiny-grid and tile-edge parity cases, walls, MUSCL, curvilinear
grids, slabs with ghost rows and the allocation-free residual run once under it: no access
leaves its buffer and the results still match the oracle. (It runs in a child process: a
process loads one libroeam.)"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
import numpy as np
sys.path.insert(0, ROOT); sys.path.insert(0, ROOT + "/tests")
from paper_1711_09272_gb300 import build, roeam as R
R.load_library(build.build(debug=True))
import oracle
import workloads as W

def rel(Ug, Uo):
    m = np.sqrt(Uo[1] ** 2 + Uo[2] ** 2).max()
    sc = np.array([np.abs(Uo[0]).max(), m, m, np.abs(Uo[3]).max()])
    return float(np.max(np.abs(Ug - Uo).reshape(4, -1).max(axis=1) / sc))

checked = 0
for prec, tol in ((64, 1e-12), (32, 1e-5)):
    for ni, nj in ((4, 4), (5, 7), (31, 4), (33, 5), (4, 65), (61, 6), (29, 129)):
        for bc, recon in (((W.PERIODIC,) * 4, 0), ((W.INFLOW, W.OUTFLOW, W.WALL, W.WALL), 2)):
            spec = W.GridSpec(ni=ni, nj=nj, dx=0.1, dy=0.1, bc=bc, inflow=(1.1, 0.4, 0.0, 1.0),
                              params=W.SchemeParams(m_ref=0.4, recon=recon))
            U = W.random_rough_state(spec, seed=ni * 100 + nj, mach=0.8, jump=0.3)
            for cfg in (0, 5):
                with R.Batch([spec], precision=prec) as b:
                    b.set_tile_config(cfg)
                    b.set_state(U, 0)
                    U0 = b.get_state(0)
                    b.step(0.4, nsteps=1)
                    Ug = b.get_state(0)
                    b.check()
                Uo, _ = oracle.OracleGrid(spec).step(U0, cfl=0.4)
                assert rel(Ug, Uo) <= tol, (ni, nj, recon, prec, cfg)
                checked += 1
# the warped step (curvilinear, solid block, walls) and a first-order curvilinear grid
for spec, U in (W.warped_step(64, 48), (W.with_params(W.warped_periodic(24), recon=0), None)):
    if U is None:
        U = W.random_smooth_state(spec, seed=3, mach=0.6, amp=0.2)
    with R.Batch([spec], precision=32) as b:
        b.set_state(U, 0); U0 = b.get_state(0); b.step(0.5, nsteps=1); Ug = b.get_state(0); b.check()
        out = np.empty_like(U0)
        R.roeam_flux_residual_noalloc(b.handle, 0, out)
        b.check()
    Uo, _ = oracle.OracleGrid(spec).step(U0, cfl=0.5)
    assert rel(Ug, Uo) <= 1e-5
    checked += 1
# slabs: EXCHANGE ghost rows (state, mask, vertices) and the two-part stages
from paper_1711_09272_gb300.slab import LocalExchange, SlabStepper
spec, _ = W.warped_step(96, 60, with_state=False)
U = W.random_smooth_state(spec, seed=8, mach=2.0, amp=0.2)
st = SlabStepper(spec, 5, list(range(5)), LocalExchange(), precision=32)
st.set_state(U); st.step(0.5, nsteps=2)
for h in st.handles.values():
    h.check()
st.close()
print("debug build ok", checked)
'''


def test_debug_build_reports_no_bounds_violation():
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + SCRIPT], cwd=ROOT, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-3000:])
    assert "debug build ok" in r.stdout
