"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (per-step state error, relative to the state's magnitude: max |rho|, max |rho q|
for both momentum components, max |rho E|): FP64 <= 1e-12, FP32 <= 1e-5. Momentum is
normalised by the momentum vector so that a component that is nearly zero everywhere (the
transverse momentum of a duct flow) does not turn rounding into a large "relative" error.
Residuals are compared against the flux scale sum_f |F||S| / V, which bounds the
rounding of their cancellation.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5}
# every work-unit shape the library is built with (roeam_tile_config_count() == 10); the
# autotuner may pick any of them for a run
TILE_CFGS = list(range(10))


def P():
    import paper_1711_09272_gb300 as pkg
    return pkg


def state_scale(U):
    m = np.sqrt(U[1] ** 2 + U[2] ** 2).max()
    return np.array([np.abs(U[0]).max(), m, m, np.abs(U[3]).max()])


def rel_state_err(Ug, Uo):
    return float(np.max(np.abs(Ug - Uo).reshape(4, -1).max(axis=1) / state_scale(Uo)))


def one_step_parity(spec, U, prec, cfl=0.5, dt_fixed=0.0, cfg=0, **variant):
    """Sets U on the GPU, reads back the (rounded) device state, advances one step on both
    sides from that same state and returns the relative state error. cfg selects the
    stage kernel's work-unit shape."""
    with P().Batch([spec], precision=prec) as b:
        assert P().roeam_tile_config_count() == len(TILE_CFGS)
        b.set_tile_config(cfg)
        b.set_state(U, 0)
        U0 = b.get_state(0)
        b.step(cfl=cfl, dt_fixed=dt_fixed, nsteps=1)
        Ug = b.get_state(0)
    Uo, _ = oracle.OracleGrid(spec, **variant).step(U0, cfl=cfl, dt_fixed=dt_fixed)
    return rel_state_err(Ug, Uo)


CASES = {
    "periodic_first": lambda: (W.GridSpec(ni=77, nj=45, dx=0.013, dy=0.021, params=W.SchemeParams(m_ref=0.3)), 1.2),
    "periodic_minmod": lambda: (W.GridSpec(ni=70, nj=37, dx=0.013, dy=0.021,
                                           params=W.SchemeParams(m_ref=0.3, recon=1)), 1.2),
    "periodic_vanleer_eps1": lambda: (W.GridSpec(ni=66, nj=41, dx=0.02, dy=0.02,
                                                 params=W.SchemeParams(m_ref=0.8, recon=2, eps1=1)), 2.5),
    "no_detector_xi_literal": lambda: (W.GridSpec(ni=40, nj=33, params=W.SchemeParams(use_s1=0, xi_form=1)), 1.5),
    "low_mach": lambda: (W.GridSpec(ni=48, nj=40, params=W.SchemeParams(m_ref=1e-3, recon=1)), 0.01),
    # ablation variants of Section 7
    "roe": lambda: (W.GridSpec(ni=45, nj=38, dx=0.013, dy=0.021, params=W.SchemeParams(scheme=1)), 1.2),
    "roe_harten_minmod": lambda: (W.GridSpec(ni=44, nj=35, params=W.SchemeParams(scheme=1, harten=0.2, recon=1)),
                                  1.5),
    "roe_harten_low_mach": lambda: (W.GridSpec(ni=40, nj=36, params=W.SchemeParams(scheme=1, harten=0.05,
                                                                                      m_ref=1e-2)), 0.01),
    "roeam_dup_zero": lambda: (W.GridSpec(ni=41, nj=37, params=W.SchemeParams(dup_mode=1, m_ref=0.05)), 0.05),
    "roeam_dup_roe_vanleer": lambda: (W.GridSpec(ni=43, nj=34, params=W.SchemeParams(dup_mode=2, recon=2,
                                                                                     m_ref=0.05)), 0.05),
    "roeam_no_ufix": lambda: (W.GridSpec(ni=42, nj=39, params=W.SchemeParams(ufix=0, m_ref=0.5)), 1.2),
    "roeam_roe_xi_and_dup_eps1": lambda: (W.GridSpec(ni=47, nj=33, params=W.SchemeParams(xi_roe=1, dup_mode=2,
                                                                                         eps1=1)), 1.5),
}


@pytest.mark.parametrize("cfg", TILE_CFGS)
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("case", sorted(CASES))
def test_step_parity_rough_states(case, prec, cfg):
    spec, mach = CASES[case]()
    U = W.random_rough_state(spec, seed=101, mach=mach, jump=0.4)
    err = one_step_parity(spec, U, prec, cfg=cfg)
    assert err <= TOL[prec], err


@pytest.mark.parametrize("prec", [64, 32])
def test_step_parity_walls_inflow_outflow(prec):
    spec, U = W.quirk(nx=90, ny=20, eps_y=0.1, x_shock=30.0, eps1=1, recon=2)
    U = U + 0.02 * W.random_smooth_state(spec, seed=5, mach=0.3, amp=0.3) * np.array([1, 0, 0, 1])[:, None, None]
    assert one_step_parity(spec, U, prec, cfl=0.4) <= TOL[prec]


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("recon", [0, 2])
def test_step_parity_warped_periodic(prec, recon):
    spec = W.with_params(W.warped_periodic(40, amp=0.2), recon=recon, m_ref=0.4)
    U = W.random_smooth_state(spec, seed=11, mach=0.7, amp=0.5)
    assert one_step_parity(spec, U, prec) <= TOL[prec]


@pytest.mark.parametrize("prec", [64, 32])
def test_step_parity_step_with_solid_block(prec):
    spec, U = W.warped_step(120, 40, recon=2)
    U = U * (1 + 0.05 * W.random_smooth_state(spec, seed=3, mach=0.3, amp=0.5)[0:1])
    assert one_step_parity(spec, U, prec, cfl=0.4) <= TOL[prec]


@pytest.mark.parametrize("prec", [64, 32])
def test_residual_parity(prec):
    spec = W.GridSpec(ni=53, nj=29, dx=0.05, dy=0.04, params=W.SchemeParams(m_ref=0.5, recon=2, eps1=1))
    U = W.random_rough_state(spec, seed=7, mach=1.5, jump=0.5)
    with P().Batch([spec], precision=prec) as b:
        b.set_state(U, 0)
        U0 = b.get_state(0)
        Rg = b.residual(0)
    g = oracle.OracleGrid(spec)
    Ro = g.residual(U0)
    rho, u, v, p = W.cons_to_prim(U0)
    fscale = np.max(rho * (np.abs(u) + np.abs(v)) ** 2 + p + (p * 3.5 + rho * (u * u + v * v)) * (np.abs(u) + np.abs(v) + 2))
    scale = fscale * 4 / min(spec.dx, spec.dy)
    err = np.max(np.abs(Rg - Ro)) / scale
    assert err <= (1e-13 if prec == 64 else 2e-6), err


def graded_state(spec, seed=11, drop=1e-8, mach=0.3):
    """Density and pressure fall by `drop` from column to column (levels 1, drop, drop^2,
    drop^3, repeating along i; factors 0.8-1.2), velocities at `mach` times the sound speed in
    random directions."""
    rng = np.random.default_rng(seed)
    lev = np.broadcast_to(np.arange(spec.ni)[None, :] % 4, (spec.nj, spec.ni))
    rho = drop ** lev * (0.8 + 0.4 * rng.random((spec.nj, spec.ni)))
    p = drop ** lev * (0.8 + 0.4 * rng.random((spec.nj, spec.ni)))
    c = np.sqrt(spec.params.gamma * p / rho)
    th = 2 * np.pi * rng.random((spec.nj, spec.ni))
    u, v = mach * c * np.cos(th), mach * c * np.sin(th)
    E = p / (spec.params.gamma - 1) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E])


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("recon", [1, 2])
def test_residual_across_eight_orders_of_magnitude(prec, recon):
    """A face whose upwind neighbour is 1e8 times heavier: van Leer's slope (up to twice the
    smaller difference) reconstructs the face's left state to about the lighter cell's level,
    which in FP32 lies within rounding of zero. The FP32 path must take the reconstruction (and
    its positivity decision) as the FP64 path does: a first-order fallback there would put the
    heavier cell's pressure on the face. Residuals are compared per cell against the flux scale
    of the cell and its four face neighbours, so that a face at the 1e-8 level is not hidden
    behind the heavy cells' fluxes."""
    spec = W.GridSpec(ni=40, nj=12, dx=0.02, dy=0.02, params=W.SchemeParams(m_ref=0.3, recon=recon))
    U = graded_state(spec)
    with P().Batch([spec], precision=prec) as b:
        b.set_state(U, 0)
        U0 = b.get_state(0)
        Rg = b.residual(0)
    Ro = oracle.OracleGrid(spec).residual(U0)
    rho, u, v, p = W.cons_to_prim(U0)
    a = np.abs(u) + np.abs(v)
    f = rho * a * a + p + (p * 3.5 + rho * (u * u + v * v)) * (a + 2)
    local = np.maximum.reduce([f, np.roll(f, 1, 0), np.roll(f, -1, 0), np.roll(f, 1, 1), np.roll(f, -1, 1)])
    scale = local * 4 / min(spec.dx, spec.dy)
    err = np.max(np.abs(Rg - Ro) / scale[None])
    assert np.all(np.isfinite(Rg))
    assert err <= (1e-12 if prec == 64 else 1e-5), err


@pytest.mark.parametrize("prec", [64, 32])
def test_free_stream_exact(prec):
    spec = W.GridSpec(ni=70, nj=19, dx=0.1, dy=0.1, params=W.SchemeParams(recon=2, m_ref=0.1))
    U = W.free_stream(spec, 1.3, 0.2, -0.1, 0.8)
    with P().Batch([spec], precision=prec) as b:
        b.set_state(U, 0)
        assert np.all(b.residual(0) == 0.0)
        U0 = b.get_state(0)
        b.step(0.5, nsteps=3)
        # the stage combinations 3/4 U + 1/4 U and 1/3 U + 2/3 U round to within a few ulp
        assert rel_state_err(b.get_state(0), U0) <= 8 * np.finfo(np.float32 if prec == 32 else np.float64).eps


def test_multi_step_vortex_trajectory_fp64():
    """Config-1 workload (64x64 periodic isentropic vortex, first order, CFL 0.5, 100 steps):
    the FP64 GPU trajectory stays with the oracle's."""
    spec, U = W.isentropic_vortex(64)
    with P().Batch([spec], precision=64) as b:
        b.set_state(U, 0)
        b.step(0.5, nsteps=100)
        Ug = b.get_state(0)
    Uo, _ = oracle.OracleGrid(spec).step(U, 0.5, nsteps=100)
    assert rel_state_err(Ug, Uo) <= 1e-11


def test_batch_ragged_grids_per_grid_dt():
    specs, states = W.batch(count=7, seed=77, ni_range=(4, 90), nj_range=(4, 70))
    with P().Batch(specs, precision=64) as b:
        b.set_states(states)
        dts = b.step(0.5, nsteps=1, want_dt=True)
        got = b.get_states()
    for k, (s, U) in enumerate(zip(specs, states)):
        Uo, dto = oracle.OracleGrid(s).step(U, 0.5)
        assert abs(dts[k] / dto - 1) < 1e-12
        assert rel_state_err(got[k], Uo) <= 1e-12, k


@pytest.mark.parametrize("prec", [64, 32])
def test_graph_replay_matches_direct_steps(prec):
    spec = W.GridSpec(ni=50, nj=30, params=W.SchemeParams(recon=1))
    U = W.random_smooth_state(spec, seed=2, mach=0.6, amp=0.3)
    with P().Batch([spec], precision=prec) as b1, P().Batch([spec], precision=prec) as b2:
        b1.set_state(U, 0)
        b2.set_state(U, 0)
        b1.step(0.5, nsteps=19)          # odd start, graph replays, direct tail
        for _ in range(19):
            b2.step(0.5, nsteps=1)
        assert np.array_equal(b1.get_state(0), b2.get_state(0))


@pytest.mark.parametrize("prec", [64, 32])
def test_totals_and_norms(prec):
    spec = W.with_params(W.warped_periodic(32), recon=2)
    U = W.random_smooth_state(spec, seed=4, mach=0.8, amp=0.4)
    g = oracle.OracleGrid(spec)
    with P().Batch([spec], precision=prec) as b:
        b.set_state(U, 0)
        U0 = b.get_state(0)
        T0 = b.totals(0)
        n2 = b.residual_norm(0, 0)
        ninf = b.residual_norm(0, 1)
        b.step(0.5, nsteps=10)
        T1 = b.totals(0)
    To = g.totals(U0)
    assert np.all(np.abs(T0 - To) <= (1e-13 if prec == 64 else 1e-6) * np.abs(To).max())
    assert np.all(np.abs(T1 - T0) <= (1e-13 if prec == 64 else 1e-5) * np.abs(T0).max())
    R = g.residual(U0)
    assert np.allclose(n2, np.sqrt(np.mean(R.reshape(4, -1) ** 2, axis=1)), rtol=1e-10 if prec == 64 else 1e-3,
                       atol=1e-12 * np.abs(R).max())
    assert np.allclose(ninf, np.abs(R).reshape(4, -1).max(axis=1), rtol=1e-10 if prec == 64 else 1e-3,
                       atol=1e-12 * np.abs(R).max())


def test_nonpositive_state_is_reported():
    """A host-made invalid state (negative pressure) is reported as a status, not a fault."""
    spec = W.GridSpec(ni=16, nj=16)
    U = W.free_stream(spec)
    U[3, 5, 5] = 0.01 * U[3, 5, 5] - 10.0
    import paper_1711_09272_gb300 as pkg
    with pkg.Batch([spec], precision=64) as b:
        b.set_state(U, 0)
        b.step(cfl=0.5, dt_fixed=1e-3, nsteps=1)
        with pytest.raises(pkg.RoeamError) as e:
            b.check()
        assert e.value.status in (4, 5)
        b.check()   # the status was cleared


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("variant", [dict(scheme=1, harten=0.05), dict(xi_roe=1, dup_mode=2)])
def test_step_parity_ablation_walls_and_curvilinear(prec, variant):
    """The ablation kernels on the duct (walls, inflow, outflow, MUSCL) and on a warped
    periodic grid."""
    spec, U = W.quirk(nx=60, ny=20, eps_y=0.1, x_shock=20.0, recon=2)
    spec = W.with_params(spec, **variant)
    assert one_step_parity(spec, U, prec, cfl=0.4) <= TOL[prec]
    spec = W.with_params(W.warped_periodic(36, amp=0.2), m_ref=0.4, **variant)
    U = W.random_smooth_state(spec, seed=12, mach=0.7, amp=0.5)
    assert one_step_parity(spec, U, prec) <= TOL[prec]


@pytest.mark.parametrize("prec", [64, 32])
def test_batch_mixing_schemes(prec):
    """One batch holding Roe-AM, classical Roe (with and without the entropy fix) and Roe-AM
    variants: each grid follows the oracle with its own scheme."""
    base = dict(ni=37, nj=29, dx=0.02, dy=0.03)
    plist = [W.SchemeParams(), W.SchemeParams(scheme=1), W.SchemeParams(scheme=1, harten=0.1),
             W.SchemeParams(dup_mode=1), W.SchemeParams(ufix=0, xi_roe=1)]
    specs = [W.GridSpec(params=p, **base) for p in plist]
    states = [W.random_rough_state(s, seed=300 + k, mach=0.9, jump=0.3) for k, s in enumerate(specs)]
    with P().Batch(specs, precision=prec) as b:
        b.set_states(states)
        U0 = b.get_states()
        dts = b.step(0.5, nsteps=1, want_dt=True)
        U1 = b.get_states()
    for k, s in enumerate(specs):
        Uo, dto = oracle.OracleGrid(s).step(U0[k], cfl=0.5)
        assert abs(dts[k] - dto) <= 1e-5 * dto
        assert rel_state_err(U1[k], Uo) <= TOL[prec], k


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("cfg", [0, 4, 8])
def test_step_host_matches_separate_calls(prec, cfg):
    """roeam_step_host (chunked, copies in, steps and copies out on three streams; each chunk's
    units cut from the tile shape so the chunk fills the resident warps) gives exactly the state
    and time steps of set_state + rk_step + get_state, for a batch spanning many chunks, with
    page-locked and with pageable host arrays, and with the tile shape changed between calls."""
    import torch
    specs, states = W.batch(40, seed=77)
    packed = np.concatenate([s.ravel() for s in states])
    h_in = torch.from_numpy(packed.copy()).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    dt_a = np.zeros(len(specs))
    with P().Batch(specs, precision=prec) as b:
        b.set_tile_config(cfg)
        P().roeam_step_host(b.handle, 0.5, 0.0, 1, h_in, h_out, dt_a)
        b.set_tile_config((cfg + 1) % len(TILE_CFGS))
        P().roeam_step_host(b.handle, 0.5, 0.0, 2, h_out, h_out, dt_a)
        got = h_out.numpy().copy()
        assert np.array_equal(np.concatenate([u.ravel() for u in b.get_states()]), got)
    with P().Batch(specs, precision=prec) as b:
        b.set_states(states)
        dt_b = b.step(0.5, nsteps=3, want_dt=True)
        ref = np.concatenate([u.ravel() for u in b.get_states()])
    assert np.array_equal(got, ref)
    assert np.array_equal(dt_a, dt_b)
    # pageable host arrays; in place (cons_out = cons_in) is allowed
    buf = packed.copy()
    with P().Batch(specs, precision=prec) as b:
        P().roeam_step_host(b.handle, 0.5, 0.0, 3, buf, buf)
    assert np.array_equal(buf, ref)


@pytest.mark.parametrize("count", [1, 2, 9, 10, 11, 25])
def test_step_host_chunking_over_grid_counts(count):
    """roeam_step_host_f32 cuts the batch into up to ten chunks of whole grids: with fewer grids
    than chunks, as many as chunks, and more, it gives the state and time steps of
    set_state + rk_step + get_state bit for bit (FP32 handle, float32 host arrays)."""
    import torch
    specs, states = W.batch(count, seed=400 + count, ni_range=(16, 120), nj_range=(8, 100))
    packed = np.concatenate([s.ravel() for s in states]).astype(np.float32)
    h_in = torch.from_numpy(packed.copy()).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    dt_a = np.zeros(count)
    with P().Batch(specs, precision=32) as b:
        P().roeam_step_host_f32(b.handle, 0.5, 0.0, 2, h_in, h_out, dt_a)
        got = h_out.numpy().copy()
    with P().Batch(specs, precision=32) as b:
        P().roeam_set_state_f32(b.handle, -1, packed)
        dt_b = b.step(0.5, nsteps=2, want_dt=True)
        ref = np.empty_like(packed)
        P().roeam_get_state_f32(b.handle, -1, ref)
    assert np.array_equal(got, ref)
    assert np.array_equal(dt_a, dt_b)


@pytest.mark.parametrize("cfg", TILE_CFGS)
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("shape", [(4, 4), (5, 7), (31, 4), (33, 5), (4, 65), (61, 6), (29, 129)])
def test_tiny_and_tile_edge_grids(shape, prec, cfg):
    """The smallest grids and sizes at the strip / segment edges (30 or 28 written columns per
    strip, segments of 16 to 128 rows, halved down to 2 rows for a single small grid):
    periodic and wall/inflow/outflow, first order and van Leer, every work-unit shape."""
    ni, nj = shape
    for bc, recon in (((W.PERIODIC,) * 4, 0), ((W.INFLOW, W.OUTFLOW, W.WALL, W.WALL), 2)):
        spec = W.GridSpec(ni=ni, nj=nj, dx=0.1, dy=0.1, bc=bc, inflow=(1.1, 0.4, 0.0, 1.0),
                          params=W.SchemeParams(m_ref=0.4, recon=recon))
        U = W.random_rough_state(spec, seed=ni * 100 + nj, mach=0.8, jump=0.3)
        assert one_step_parity(spec, U, prec, cfl=0.4, cfg=cfg) <= TOL[prec], (bc, recon)


def test_largest_batch_count():
    """A handle at its largest batch size, 65535 grids (4 to 7 cells a side, periodic or
    wall/inflow/outflow, van Leer, FP32): one step of the whole batch, with every 1000th grid
    and the last one recomputed by the oracle from the device's state."""
    rng = np.random.default_rng(65535)
    specs, states = [], []
    for k in range(65535):
        ni, nj = (int(x) for x in rng.integers(4, 8, size=2))
        walls = k % 2 == 1
        bc = (W.INFLOW, W.OUTFLOW, W.WALL, W.WALL) if walls else (W.PERIODIC,) * 4
        spec = W.GridSpec(ni=ni, nj=nj, dx=0.1, dy=0.1, bc=bc, inflow=(1.1, 0.4, 0.0, 1.0),
                          params=W.SchemeParams(m_ref=0.4, recon=2))
        specs.append(spec)
        states.append(W.random_rough_state(spec, seed=k, mach=0.8, jump=0.3))
    with P().Batch(specs, precision=32) as b:
        b.set_states(states)
        U0 = b.get_states()
        dts = b.step(0.4, nsteps=1, want_dt=True)
        U1 = b.get_states()
    for k in list(range(0, 65535, 1000)) + [65534]:
        Uo, _ = oracle.OracleGrid(specs[k]).step(U0[k], dt_fixed=float(dts[k]))
        assert rel_state_err(U1[k], Uo) <= TOL[32], k


@pytest.mark.parametrize("recon", [0, 2])
def test_tiny_magnitudes(recon):
    """The Euler equations are invariant under rho -> s rho, p -> s p at fixed velocity: a state
    scaled by s = 1e-24 (products of two conserved values then fall below the FP32 range) must
    step in FP32 without a positivity report and match the oracle."""
    spec = W.GridSpec(ni=40, nj=24, dx=0.02, dy=0.02, params=W.SchemeParams(m_ref=0.5, recon=recon))
    U = W.random_smooth_state(spec, seed=5, mach=0.5, amp=0.2) * 1e-24
    assert one_step_parity(spec, U, 32) <= TOL[32]


def _run_all_shapes(specs, states, prec, nsteps):
    outs, dts = [], []
    for cfg in TILE_CFGS:
        with P().Batch(specs, precision=prec) as b:
            b.set_tile_config(cfg)
            b.set_states(states)
            b.step(0.5, nsteps=nsteps - 1)
            dts.append(b.step(0.5, nsteps=1, want_dt=True))
            outs.append(b.get_states())
    return outs, dts


@pytest.mark.parametrize("kind", ["batch_first", "batch_vanleer_fp64", "walls_minmod", "warped_step", "ablation_mixed"])
def test_results_independent_of_tile_shape(kind):
    """The same state stepped with every work-unit shape (segments of 16, 32, 64 and 128 rows,
    so that a row sits at different places within its unit and is evaluated by different
    copies of the unrolled loop body) gives bit-identical states and time steps: the kernels'
    fused multiply-adds are all explicit, so the autotuner's choice cannot change a result."""
    if kind == "batch_first":
        specs, states = W.batch(512)
        prec, n = 32, 6
    elif kind == "batch_vanleer_fp64":
        specs, states = W.batch(160, seed=5)
        specs = [W.with_params(s, recon=2) for s in specs]
        prec, n = 64, 3
    elif kind == "walls_minmod":
        from dataclasses import replace
        specs, states = W.batch(256, seed=7)
        specs = [replace(W.with_params(s, recon=1), bc=(W.OUTFLOW, W.OUTFLOW, W.WALL, W.WALL)) if k % 3 == 0
                 else W.with_params(s, recon=1) for k, s in enumerate(specs)]
        prec, n = 32, 3
    elif kind == "warped_step":
        spec, U = W.warped_step(2048, 2048)
        specs, states, prec, n = [spec], [U], 32, 3
    else:
        specs, states = W.batch(256, seed=9)
        specs = [W.with_params(s, scheme=1, harten=0.1) if k % 2 else s for k, s in enumerate(specs)]
        prec, n = 32, 3
    outs, dts = _run_all_shapes(specs, states, prec, n)
    for cfg in TILE_CFGS[1:]:
        assert np.array_equal(dts[cfg], dts[0]), cfg
        for g in range(len(specs)):
            assert np.array_equal(outs[cfg][g], outs[0][g]), (cfg, g)


INCREMENT_CASES = ["low_mach", "periodic_first", "periodic_vanleer_eps1", "periodic_minmod"]


def increment_rel_err(U0, Ug, Uo):
    """Per variable: max |U_gpu - U_oracle| over the step / max |U_oracle^{n+1} - U^n| (the error
    relative to what the step changed rather than to the state)."""
    d = np.abs(Ug - Uo).reshape(4, -1).max(axis=1)
    inc = np.abs(Uo - U0).reshape(4, -1).max(axis=1)
    return d / inc


@pytest.mark.parametrize("prec", [64, 32])
def test_error_relative_to_the_increment(prec):
    """The per-step error measured against the step's increment instead of the state. At
    M_ref = 1e-3 (case low_mach: 48 x 40 cells, M ~ 0.01) the increment is about 1 % of the
    state, so this is the stricter measure there; FP32 stays within 1e-4 of the increment
    (measured 1.6e-5 there, about 1e-6 in the other cases), FP64 within 1e-12 (measured 4e-14).
    The measured values are reported in the test output."""
    import warnings
    worst = {}
    for case in INCREMENT_CASES:
        spec, mach = CASES[case]()
        U = W.random_rough_state(spec, seed=101, mach=mach, jump=0.4)
        with P().Batch([spec], precision=prec) as b:
            b.set_state(U, 0)
            U0 = b.get_state(0)
            b.step(cfl=0.5, nsteps=1)
            Ug = b.get_state(0)
        Uo, _ = oracle.OracleGrid(spec).step(U0, cfl=0.5)
        e = increment_rel_err(U0, Ug, Uo)
        worst[case] = float(e.max())
        assert e.max() <= (1e-4 if prec == 32 else 1e-12), (case, e)
    warnings.warn(f"FP{prec} error relative to the step increment: " +
                  ", ".join(f"{k} {v:.2e}" for k, v in worst.items()))


@pytest.mark.parametrize("prec", [64, 32])
def test_l2_error_after_n_steps(prec):
    """Independent trajectories: the GPU and the FP64 oracle each advance the isentropic vortex
    (64 x 64, FP64 config: first order, CFL 0.5) 100 steps from the same state; the L2 state
    difference relative to the oracle's state stays at rounding (FP64) or a few FP32 ulps per
    step accumulated (FP32), far below the discretisation error against the exact vortex."""
    import warnings
    spec, U = W.isentropic_vortex(64)
    with P().Batch([spec], precision=prec) as b:
        b.set_state(U, 0)
        U0 = b.get_state(0)
        b.step(cfl=0.5, nsteps=100)
        Ug = b.get_state(0)
    Uo, _ = oracle.OracleGrid(spec).step(U0, cfl=0.5, nsteps=100)
    l2 = np.sqrt(((Ug - Uo) ** 2).reshape(4, -1).sum(axis=1) / (Uo ** 2).reshape(4, -1).sum(axis=1))
    assert l2.max() <= (1e-13 if prec == 64 else 1e-5), l2   # (measured 2e-15 and 2.3e-6)
    warnings.warn(f"FP{prec} L2 state difference from the oracle after 100 steps: " +
                  " ".join(f"{x:.2e}" for x in l2))


@pytest.mark.parametrize("prec", [64, 32])
def test_injected_nan_and_bad_steps_are_reported(prec):
    """Host-side fault injection: a NaN in the state given to set_state is reported as
    ROEAM_E_NONFINITE after the next step (nothing traps, the context stays usable), and a
    non-positive fixed time step or CFL is refused before any work."""
    import paper_1711_09272_gb300 as pkg
    spec = W.GridSpec(ni=24, nj=20, dx=0.05, dy=0.05)
    U = W.free_stream(spec)
    U[1, 7, 9] = np.nan
    with pkg.Batch([spec], precision=prec) as b:
        b.set_state(U, 0)
        b.step(cfl=0.5, dt_fixed=1e-3, nsteps=1)
        with pytest.raises(pkg.RoeamError) as e:
            b.check()
        assert e.value.status == 5
        b.set_state(W.free_stream(spec), 0)      # the handle keeps working
        b.step(cfl=0.5, nsteps=2)
        b.check()
        for cfl, dt in ((0.0, 0.0), (-0.5, 0.0), (0.5, float("nan"))):
            with pytest.raises(pkg.RoeamError) as e:
                b.step(cfl=cfl, dt_fixed=dt, nsteps=1)
            assert e.value.status == 1


def test_autotuner_picks_a_shape_and_caches_it_per_workload():
    """roeam_autotune times the distinct layouts, keeps the fastest and restores the state; a
    second handle on the same workload gets the same choice and figures without timing, and a
    different workload is timed afresh."""
    import time
    specs, states = W.batch(96, seed=31)
    with P().Batch(specs, precision=32) as b:
        b.set_states(states)
        U0 = b.get_states()
        t0 = time.perf_counter()
        best, ms = b.autotune(0.5, 3)
        t_first = time.perf_counter() - t0
        assert 0 <= best < len(TILE_CFGS) and len(ms) == len(TILE_CFGS)
        assert ms[best] == min(ms) and all(m > 0 for m in ms)
        for k, u in enumerate(b.get_states()):
            assert np.array_equal(u, U0[k])          # the state is restored
        b.step(0.5, nsteps=2)
        Ua = b.get_states()
    with P().Batch(specs, precision=32) as b:
        b.set_states(states)
        t0 = time.perf_counter()
        best2, ms2 = b.autotune(0.5, 3)
        t_second = time.perf_counter() - t0
        assert best2 == best and list(ms2) == list(ms)
        b.step(0.5, nsteps=2)
        assert all(np.array_equal(x, y) for x, y in zip(b.get_states(), Ua))
    assert t_second < t_first
    other = [W.with_params(s, recon=2) for s in specs]
    with P().Batch(other, precision=32) as b:
        b.set_states(states)
        _, ms3 = b.autotune(0.5, 3)
        assert list(ms3) != list(ms)
