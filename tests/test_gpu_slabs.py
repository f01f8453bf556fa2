"""A grid split into row slabs (EXCHANGE sides, stage-by-stage stepping, ghost rows from the
neighbouring slab) on the GPU: the slabs reproduce the whole grid. Several slab handles are
driven from one process in lockstep (no kernel waits on another; the exchange is a host
copy between launches), which is what each GPU of a multi-GPU run does for its own slab."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def P():
    import paper_1711_09272_gb300 as pkg
    return pkg


def run_slabs(spec, U, parts, prec, nsteps=4, overlap=True):
    from paper_1711_09272_gb300.slab import LocalExchange, SlabStepper
    st = SlabStepper(spec, parts, list(range(parts)), LocalExchange(), precision=prec, overlap=overlap)
    try:
        st.set_state(U)
        dts = [st.step(0.5) for _ in range(nsteps)]
        return st.get_state(np.zeros_like(U)), dts
    finally:
        st.close()


CASES = {
    "periodic_first": lambda: W.GridSpec(ni=70, nj=41, dx=0.02, dy=0.025, params=W.SchemeParams(m_ref=0.4)),
    "periodic_vanleer": lambda: W.GridSpec(ni=64, nj=37, dx=0.02, dy=0.02, params=W.SchemeParams(m_ref=0.4, recon=2)),
    "wall_inflow_minmod": lambda: W.GridSpec(ni=50, nj=36, dx=0.03, dy=0.03, bc=(W.OUTFLOW, W.OUTFLOW, W.WALL, W.INFLOW),
                                             inflow=(1.2, 0.4, -0.1, 0.9), params=W.SchemeParams(m_ref=0.5, recon=1,
                                                                                                 eps1=1)),
}


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("case", sorted(CASES))
def test_slabs_reproduce_the_whole_grid(case, prec):
    """Cartesian slabs (2 and 3) against the whole grid stepped through the same stage calls:
    every cell sees the same neighbour values and the same dt, and every fused multiply-add
    of the kernels is explicit, so the slabs reproduce the whole grid bit for bit although a
    row sits at a different place within its work unit."""
    spec = CASES[case]()
    U = W.random_smooth_state(W.GridSpec(ni=spec.ni, nj=spec.nj, dx=spec.dx, dy=spec.dy, params=spec.params),
                              seed=9, mach=0.6, amp=0.3)
    U1, d1 = run_slabs(spec, U, 1, prec)
    for parts in (2, 3):
        Up, dp = run_slabs(spec, U, parts, prec)
        assert np.array_equal(dp, d1), parts
        assert np.array_equal(Up, U1), parts


@pytest.mark.parametrize("prec", [64, 32])
def test_stage_calls_match_rk_step_and_oracle(prec):
    """The stage-by-stage path of one grid matches roeam_rk_step (to rounding: the host-side
    dt and the kernels' work units) and the oracle."""
    spec = CASES["wall_inflow_minmod"]()
    U = W.random_smooth_state(W.GridSpec(ni=spec.ni, nj=spec.nj, dx=spec.dx, dy=spec.dy, params=spec.params),
                              seed=10, mach=0.6, amp=0.3)
    Us, dts = run_slabs(spec, U, 1, prec, nsteps=3)
    with P().Batch([spec], precision=prec) as b:
        b.set_state(U, 0)
        b.step(0.5, nsteps=3)
        Ur = b.get_state(0)
    scale = np.abs(Ur).reshape(4, -1).max(axis=1)[:, None, None]
    assert np.max(np.abs(Us - Ur) / scale) < (1e-14 if prec == 64 else 1e-5)
    g = oracle.OracleGrid(spec)
    Uo = U.copy()
    for dt in dts:
        Uo, _ = g.step(Uo, dt_fixed=dt)
    assert np.max(np.abs(Us - Uo) / scale) < (1e-11 if prec == 64 else 1e-4)


def test_curvilinear_slabs():
    """A warped periodic grid in 3 slabs (FP64): the slab vertex rows are stored relative to the
    slab's own reference rows, so the match is to rounding."""
    spec = W.with_params(W.warped_periodic(48, amp=0.15), recon=2, m_ref=0.4)
    U = W.random_smooth_state(spec, seed=12, mach=0.6, amp=0.3)
    U1, _ = run_slabs(spec, U, 1, 64)
    U3, _ = run_slabs(spec, U, 3, 64)
    scale = np.abs(U1).reshape(4, -1).max(axis=1)[:, None, None]
    assert np.max(np.abs(U3 - U1) / scale) < 1e-13


def test_exchange_api_errors():
    """Ghost rows only on EXCHANGE sides; stages in order; rk_step refuses an unfinished step."""
    spec = W.GridSpec(ni=32, nj=16, dx=0.05, dy=0.05, bc=(W.PERIODIC, W.PERIODIC, W.WALL, 4))
    U = W.free_stream(spec, 1.0, 0.2, 0.0, 1.0)
    with P().Batch([spec], precision=64) as b:
        b.set_state(U, 0)
        with pytest.raises(P().RoeamError):
            b.set_halo(0, 2, 0, np.ones((4, 2, 32)))       # S is a wall
        b.set_halo(0, 3, 0, b.edge_rows(0, 3, 0))
        with pytest.raises(P().RoeamError):
            b.stage(1, 1e-3)                                # stage 0 first
        b.stage(0, 1e-3)
        with pytest.raises(P().RoeamError) as e:
            b.step(0.5)
        assert e.value.status == 7
        b.set_halo(0, 3, 1, b.edge_rows(0, 3, 1))
        b.stage(1, 1e-3)
        b.set_halo(0, 3, 2, b.edge_rows(0, 3, 2))
        b.stage(2, 1e-3)
        b.step(0.5)                                         # a whole step works again
        assert np.all(np.isfinite(b.get_state(0)))
        # a stage in two parts: the interior first, then the edges, nothing in between
        with pytest.raises(P().RoeamError) as e:
            b.stage_part(0, 1e-3, 2)
        assert e.value.status == 7
        b.stage_part(0, 1e-3, 1)
        for bad in (lambda: b.stage_part(0, 1e-3, 1), lambda: b.stage(0, 1e-3), lambda: b.step(0.5)):
            with pytest.raises(P().RoeamError) as e:
                bad()
            assert e.value.status == 7
        b.stage_part(0, 1e-3, 2)
        b.stage_part(1, 1e-3, 0)
        b.stage(2, 1e-3)
        with pytest.raises(P().RoeamError):
            b.set_halo_solid(0, 3, np.zeros((2, 32), np.uint8))   # no solid mask in this grid
        with pytest.raises(P().RoeamError):
            b.set_halo_vertices(0, 3, np.zeros((2, 33)), np.zeros((2, 33)))   # Cartesian


@pytest.mark.parametrize("prec", [64, 32])
def test_warped_step_slabs_with_solid_block(prec):
    """The warped Mach-3 step (256 x 256: curvilinear, MUSCL van Leer, solid block, walls,
    inflow, outflow) in 2, 3 and 5 slabs against the whole grid stepped through the same stage
    calls. With 5 slabs the slab edge at row 52 lies one row above the block (rows 0-50), so a
    ghost row holds solid cells that reconstruction stencils mirror. The slabs store their
    vertices relative to their own first row, so the match is to the rounding of that storage."""
    spec, _ = W.warped_step(256, 256, with_state=False)
    U = W.random_smooth_state(spec, seed=21, mach=2.0, amp=0.2)
    U1, d1 = run_slabs(spec, U, 1, prec, nsteps=3)
    scale = np.abs(U1).reshape(4, -1).max(axis=1)[:, None, None]
    for parts in (2, 3, 5):
        Up, dp = run_slabs(spec, U, parts, prec, nsteps=3)
        assert np.allclose(dp, d1, rtol=1e-12 if prec == 64 else 1e-5, atol=0), parts
        assert np.max(np.abs(Up - U1) / scale) < (1e-12 if prec == 64 else 2e-5), parts


@pytest.mark.parametrize("prec", [64, 32])
def test_interior_and_edge_parts_equal_whole_stages(prec):
    """Each stage as two launches (the slab interior, then the rows next to the EXCHANGE sides
    once the ghost rows are set) gives the bits of whole-stage launches."""
    spec, _ = W.warped_step(160, 96, with_state=False)
    U = W.random_smooth_state(spec, seed=22, mach=2.0, amp=0.2)
    for parts in (2, 4):
        Ua, da = run_slabs(spec, U, parts, prec, nsteps=2, overlap=False)
        Ub, db = run_slabs(spec, U, parts, prec, nsteps=2, overlap=True)
        assert np.array_equal(Ua, Ub) and np.array_equal(da, db), parts
