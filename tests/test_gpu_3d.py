"""GPU parity and physics of the 3D path (include/roeam3.h): Cartesian grids, first order, passive
scalars, against the 3D FP64 oracle. Tolerances as in 2D (per-step state error relative to the
state's magnitude: FP64 <= 1e-12, FP32 <= 1e-5; momentum normalised by the momentum vector,
scalars by max |rho k|)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5}


def P():
    import paper_1711_09272_gb300 as pkg
    return pkg


def scale3(U):
    m = np.sqrt(U[1] ** 2 + U[2] ** 2 + U[3] ** 2).max()
    return np.array([np.abs(U[0]).max(), m, m, m, np.abs(U[4]).max()] +
                    [np.abs(U[v]).max() for v in range(5, U.shape[0])])


def rel_err3(Ug, Uo):
    nv = Uo.shape[0]
    return float(np.max(np.abs(Ug - Uo).reshape(nv, -1).max(axis=1) / scale3(Uo)))


def one_step3(spec, U, prec, cfl=0.5, presteps=0):
    with P().Batch3([spec], precision=prec) as b:
        b.set_state(U, 0)
        if presteps:
            b.step(cfl, nsteps=presteps)
        U0 = b.get_state(0)
        b.step(cfl, nsteps=1)
        Ug = b.get_state(0)
    Uo, _ = oracle.OracleGrid3(spec).step(U0, cfl=cfl)
    return rel_err3(Ug, Uo)


CASES3 = {
    # ragged tiles in x and y (30 x 14 written per FP32 tile, 30 x 6 per FP64 one), several z segments
    "periodic_ns0": lambda: (W.GridSpec3(ni=37, nj=15, nk=11, dx=0.05, dy=0.06, dz=0.07,
                                         params=W.SchemeParams(m_ref=0.4)), 1.2),
    "periodic_ns0_tall": lambda: (W.GridSpec3(ni=34, nj=31, nk=6, dx=0.05, dy=0.045, dz=0.07,
                                              params=W.SchemeParams(m_ref=0.6)), 1.1),
    "periodic_ns1_eps1": lambda: (W.GridSpec3(ni=31, nj=13, nk=9, dx=0.05, dy=0.05, dz=0.05, nscal=1,
                                              params=W.SchemeParams(m_ref=0.8, eps1=1)), 1.5),
    "bcs_ns2": lambda: (W.GridSpec3(ni=33, nj=14, nk=10, dx=0.05, dy=0.04, dz=0.06, nscal=2,
                                    bc=(W.INFLOW, W.OUTFLOW, W.WALL, W.WALL, W.WALL, W.OUTFLOW),
                                    inflow=(1.3, 0.9, 0.1, -0.05, 1.1, 0.3, 0.8),
                                    params=W.SchemeParams(m_ref=0.5)), 1.0),
    "ns3_low_mach_no_detector": lambda: (W.GridSpec3(ni=20, nj=9, nk=7, dx=0.1, dy=0.1, dz=0.1, nscal=3,
                                                     params=W.SchemeParams(m_ref=0.02, use_s1=0, xi_form=1)),
                                         0.03),
}


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("case", sorted(CASES3))
def test_step_parity_3d(case, prec):
    spec, mach = CASES3[case]()
    U = W.random_rough_state3(spec, seed=17, mach=mach, jump=0.4)
    assert one_step3(spec, U, prec) <= TOL[prec]


@pytest.mark.parametrize("prec", [64, 32])
def test_residual_parity_3d(prec):
    spec = W.GridSpec3(ni=35, nj=13, nk=8, dx=0.05, dy=0.06, dz=0.04, nscal=1,
                       bc=(W.WALL, W.WALL, W.PERIODIC, W.PERIODIC, W.INFLOW, W.OUTFLOW),
                       inflow=(1.0, 0.2, 0.1, 0.7, 1.0, 0.5), params=W.SchemeParams(m_ref=0.6, eps1=1))
    U = W.random_rough_state3(spec, seed=23, mach=1.3, jump=0.5)
    with P().Batch3([spec], precision=prec) as b:
        b.set_state(U, 0)
        U0 = b.get_state(0)
        Rg = b.residual(0)
    Ro = oracle.OracleGrid3(spec).residual(U0)
    rho, u, v, w, p, k = W.cons_to_prim3(U0)
    fs = np.max(rho * (np.abs(u) + np.abs(v) + np.abs(w) + 3) ** 2 + 4 * p) * 6 / 0.04
    assert np.max(np.abs(Rg - Ro)) / fs <= (1e-13 if prec == 64 else 2e-6)


@pytest.mark.parametrize("prec", [64, 32])
def test_batch_of_3d_grids(prec):
    """A batch of uneven 3D grids with per-grid time steps: each follows the oracle."""
    specs = [W.GridSpec3(ni=n, nj=m, nk=l, dx=1 / n, dy=1 / n, dz=1 / n, nscal=1, params=W.SchemeParams(m_ref=0.3))
             for n, m, l in ((40, 12, 6), (17, 25, 9), (31, 7, 14))]
    states = [W.random_smooth_state3(s, seed=40 + k, mach=0.3 * (k + 1), amp=0.3) for k, s in enumerate(specs)]
    with P().Batch3(specs, precision=prec) as b:
        b.set_states(states)
        U0 = b.get_states()
        dts = b.step(0.5, nsteps=1, want_dt=True)
        U1 = b.get_states()
    for k, s in enumerate(specs):
        Uo, dto = oracle.OracleGrid3(s).step(U0[k], cfl=0.5)
        assert abs(dts[k] - dto) <= 1e-5 * dto
        assert rel_err3(U1[k], Uo) <= TOL[prec], k


@pytest.mark.parametrize("prec", [64, 32])
def test_taylor_green_conservation_and_trajectory(prec):
    """Taylor-Green vortex (24^3, M = 0.3, one scalar): 20 steps follow the oracle's trajectory
    (FP64 to 1e-10; FP32 to 1e-4), and the totals of every conserved variable stay put."""
    spec, U = W.taylor_green3(24, mach=0.3, nscal=1)
    with P().Batch3([spec], precision=prec) as b:
        b.set_state(U, 0)
        T0 = b.totals(0)
        dts = []
        for _ in range(20):
            dts.append(b.step(0.5, nsteps=1, want_dt=True)[0])
        Ug = b.get_state(0)
        T1 = b.totals(0)
    g = oracle.OracleGrid3(spec)
    Uo = U.copy()
    for dt in dts:
        Uo, _ = g.step(Uo, dt_fixed=dt)
    assert rel_err3(Ug, Uo) <= (1e-10 if prec == 64 else 1e-4)
    scale = np.array([abs(T0[0]), 1, 1, 1, abs(T0[4]), abs(T0[5])])
    assert np.max(np.abs(T1 - T0) / scale) <= (1e-13 if prec == 64 else 1e-5)


def test_one_cell_thick_3d_equals_2d_gpu():
    """A 3D grid one periodic cell thick in z reproduces the 2D kernels' steps (FP64, the same
    fixed dt: the 3D rate also counts the z direction)."""
    spec2 = W.GridSpec(ni=45, nj=19, dx=0.05, dy=0.07, bc=(W.WALL, W.OUTFLOW, W.PERIODIC, W.PERIODIC),
                       params=W.SchemeParams(m_ref=0.5, eps1=1))
    U2 = W.random_rough_state(spec2, seed=5, mach=1.1, jump=0.4)
    spec3 = W.GridSpec3(ni=45, nj=19, nk=1, dx=0.05, dy=0.07, dz=0.3,
                        bc=(W.WALL, W.OUTFLOW, W.PERIODIC, W.PERIODIC, W.PERIODIC, W.PERIODIC),
                        params=W.SchemeParams(m_ref=0.5, eps1=1))
    U3 = np.stack([U2[0], U2[1], U2[2], 0 * U2[0], U2[3]])[:, None]
    with P().Batch([spec2], precision=64) as b:
        b.set_state(U2, 0)
        b.step(0.0, dt_fixed=4e-3, nsteps=2)
        R2 = b.get_state(0)
    with P().Batch3([spec3], precision=64) as b:
        b.set_state(U3, 0)
        b.step(0.0, dt_fixed=4e-3, nsteps=2)
        R3 = b.get_state(0)[:, 0]
    assert np.max(np.abs(R3[3])) == 0.0
    got = np.stack([R3[0], R3[1], R3[2], R3[4]])
    assert np.max(np.abs(got - R2) / np.abs(R2).reshape(4, -1).max(axis=1)[:, None, None]) < 1e-12


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_shock_tube_along_each_axis(axis):
    """The Section 7.1.1 expansion tube along x, y and z (FP64, 100 cells, 2 x 2 periodic
    cross-section) gives the same solution on every axis, follows the oracle's trajectory, and
    the scalar marks the contact."""
    out = []
    for ax in (0, axis):
        spec, U = W.shock_tube3("expansion", n=100, axis=ax, nt=2, nscal=1)
        with P().Batch3([spec], precision=64) as b:
            b.set_state(U, 0)
            b.step(0.0, dt_fixed=0.2 / 80, nsteps=80)
            Ug = b.get_state(0)
        if ax == axis:
            Uo, _ = oracle.OracleGrid3(spec).step(U, dt_fixed=0.2 / 80, nsteps=80)
            assert rel_err3(Ug, Uo) < 1e-10
        line = [slice(0, 1)] * 3
        line[2 - ax] = slice(None)
        vel = Ug[1 + ax][tuple(line)].ravel()
        out.append((Ug[0][tuple(line)].ravel(), vel, Ug[5][tuple(line)].ravel()))
    for a, b_ in zip(out[0], out[1]):
        assert np.max(np.abs(a - b_)) <= 1e-12 * np.max(np.abs(a))
    rho, _, k = out[0]
    # the scalar's 1 -> 0 step rides on the contact, at x = 0.3 + u* t = 0.573 (u* = 1.364 from
    # the exact Riemann solution), smeared over a few cells at first order
    xk = (np.argmax(k < 0.5) + 0.5) / 100
    assert abs(xk - 0.573) < 0.06, xk


def test_full_size_sampled_parity_3d():
    """The 3D measurement workload (Taylor-Green vortex, 256^3 cells, one scalar, FP32) after 20
    steps: sampled cells of step 21 recomputed by the oracle on a 17^3 window around each (the
    window's cut faces lie 8 cells away, beyond the 3 stages x 2-cell reach of a step)."""
    n, R = 256, 8
    spec, U = W.taylor_green3(n, mach=0.1, nscal=1)
    with P().Batch3([spec], precision=32) as b:
        b.set_state(U, 0)
        b.step(0.5, nsteps=20)
        U0 = b.get_state(0)
        dt = b.step(0.5, nsteps=1, want_dt=True)[0]
        U1 = b.get_state(0)
    sc = scale3(U0)
    rng = W.SplitMix64(3)
    for _ in range(8):
        i, j, k = (int(rng.uniform() * n) for _ in range(3))
        idx = [np.arange(c - R, c + R + 1) % n for c in (k, j, i)]
        Uw = U0[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]]
        sub = W.GridSpec3(ni=2 * R + 1, nj=2 * R + 1, nk=2 * R + 1, dx=spec.dx, dy=spec.dy, dz=spec.dz,
                          bc=(W.OUTFLOW,) * 6, nscal=1, params=spec.params)
        Uo, _ = oracle.OracleGrid3(sub).step(Uw, dt_fixed=dt)
        err = np.max(np.abs(Uo[:, R, R, R] - U1[:, k, j, i]) / sc)
        assert err <= 1e-5, (i, j, k, err)


def test_tiny_magnitudes_3d():
    """rho -> s rho, p -> s p at fixed velocity leaves the Euler equations unchanged: the
    Taylor-Green state scaled by s = 1e-24 (products of two conserved values below the FP32
    range) steps in FP32 without a positivity report and matches the oracle."""
    spec, U = W.taylor_green3(16, mach=0.1, nscal=1)
    assert one_step3(spec, U * 1e-24, 32) <= 1e-5
