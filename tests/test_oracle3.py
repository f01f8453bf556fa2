"""Pins of the 3D oracle with passive scalars (Eq. 85's complete form, Eq. 96's 9-face detector)
against things other than itself: the independent 2D oracle, rotational invariance, the
scalar rows' structure, the physical flux, exact upwinding, conservation, symmetry and a
brute-force detector."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

G = 1.4


def states3(n, seed, mach=0.8, jump=0.5, nscal=0):
    r = W.SplitMix64(seed).uniforms(n * (5 + nscal)).reshape(n, 5 + nscal)
    rho = np.exp(jump * (2 * r[:, 0] - 1))
    p = np.exp(jump * (2 * r[:, 4] - 1))
    c = np.sqrt(G * p / rho)
    vel = [mach * c * (2 * r[:, k] - 1) for k in (1, 2, 3)]
    return np.column_stack([rho, *vel, p] + [r[:, 5 + s] for s in range(nscal)])


def unit_normals3(n, seed):
    v = W.SplitMix64(seed).uniforms(3 * n).reshape(n, 3) - 0.5
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def physical_flux3(W_, n):
    rho, u, v, w, p = W_[:5]
    U = n[0] * u + n[1] * v + n[2] * w
    H = G / (G - 1) * p / rho + 0.5 * (u * u + v * v + w * w)
    return np.array([rho * U, rho * u * U + p * n[0], rho * v * U + p * n[1], rho * w * U + p * n[2], rho * H * U] +
                    [rho * k * U for k in W_[5:]])


@pytest.mark.parametrize("kw", [dict(), dict(eps1=1), dict(m_ref=1e-2), dict(xi_form=1), dict(use_s1=0)])
def test_reduces_to_2d_oracle(kw):
    """w = 0, n_z = 0, no scalars: the 3D flux equals the independent 2D oracle's."""
    n = 300
    A3 = states3(n, 11)
    B3 = states3(n, 12)
    A3[:, 3] = 0.0
    B3[:, 3] = 0.0
    nr = unit_normals3(n, 13)
    nr[:, 2] = 0.0
    nr /= np.linalg.norm(nr, axis=1, keepdims=True)
    s1 = W.SplitMix64(14).uniforms(n)
    F3 = oracle.face_flux3(A3, B3, nr, s1, **kw)
    F2 = oracle.face_flux(A3[:, [0, 1, 2, 4]], B3[:, [0, 1, 2, 4]], nr[:, :2], s1, **kw)
    assert np.max(np.abs(F3[:, 3])) == 0.0
    scale = np.max(np.abs(F2), axis=1, keepdims=True)
    assert np.max(np.abs(F3[:, [0, 1, 2, 4]] - F2) / scale) < 1e-13


def rotation(seed):
    q = W.SplitMix64(seed).uniforms(4) - 0.5
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


@pytest.mark.parametrize("eps1", [0, 1])
def test_rotational_invariance(eps1):
    """Rotating both states' velocities and the normal rotates the momentum flux and leaves the
    other rows unchanged (covers the 3D reading of Eqs. 103-109 when eps1 = 1)."""
    n = 200
    A = states3(n, 21, nscal=2)
    B = states3(n, 22, nscal=2)
    nr = unit_normals3(n, 23)
    F = oracle.face_flux3(A, B, nr, nscal=2, eps1=eps1)
    for seed in (1, 2, 3):
        Q = rotation(seed)
        Ar, Br = A.copy(), B.copy()
        Ar[:, 1:4] = A[:, 1:4] @ Q.T
        Br[:, 1:4] = B[:, 1:4] @ Q.T
        Fr = oracle.face_flux3(Ar, Br, nr @ Q.T, nscal=2, eps1=eps1)
        ref = F.copy()
        ref[:, 1:4] = F[:, 1:4] @ Q.T
        scale = np.max(np.abs(F), axis=1, keepdims=True)
        assert np.max(np.abs(Fr - ref) / scale) < 1e-12


def test_scalar_rows():
    """Eq. 85's scalar rows: a uniform scalar k gives F_k = k F_rho exactly in structure (to
    rounding); the scalar rows are linear in the scalars and do not touch the other rows."""
    n = 200
    A = states3(n, 31, nscal=2)
    B = states3(n, 32, nscal=2)
    nr = unit_normals3(n, 33)
    A[:, 5] = B[:, 5] = 0.37
    F = oracle.face_flux3(A, B, nr, nscal=2)
    assert np.max(np.abs(F[:, 5] - 0.37 * F[:, 0]) / np.abs(F[:, 0]).max()) < 1e-14
    F0 = oracle.face_flux3(A[:, :5], B[:, :5], nr)
    assert np.array_equal(F[:, :5], F0)
    A2, B2 = A.copy(), B.copy()
    A2[:, 6] *= 3.0
    B2[:, 6] *= 3.0
    F2 = oracle.face_flux3(A2, B2, nr, nscal=2)
    assert np.max(np.abs(F2[:, 6] - 3.0 * F[:, 6])) < 1e-13 * np.abs(F[:, 6]).max()


def test_consistency_and_full_upwind():
    """F(W, W, n) is the physical flux; a face with both states supersonic along n takes the
    left state's physical flux (Eq. 44 with the Eq. 68 factor)."""
    n = 100
    A = states3(n, 41, nscal=1)
    nr = unit_normals3(n, 42)
    F = oracle.face_flux3(A, A, nr, nscal=1)
    for f in range(n):
        ref = physical_flux3(A[f], nr[f])
        assert np.max(np.abs(F[f] - ref)) <= 1e-14 * np.max(np.abs(ref))
    B = states3(n, 43, mach=0.2, nscal=1)
    for X in (A, B):
        c = np.sqrt(G * X[:, 4] / X[:, 0])
        X[:, 1:4] = 0.1 * X[:, 1:4] + (2.5 * c)[:, None] * nr
    F = oracle.face_flux3(A, B, nr, nscal=1)
    for f in range(n):
        ref = physical_flux3(A[f], nr[f])
        assert np.max(np.abs(F[f] - ref)) <= 1e-12 * np.max(np.abs(ref))


def grid2_of_3(spec3, U3, plane):
    """The 2D grid and state of a 3D grid that is one cell thick along the dropped axis."""
    keep = [a for a in range(3) if a != plane]
    h = (spec3.dx, spec3.dy, spec3.dz)
    n = (spec3.ni, spec3.nj, spec3.nk)
    bc = (spec3.bc[2 * keep[0]], spec3.bc[2 * keep[0] + 1], spec3.bc[2 * keep[1]], spec3.bc[2 * keep[1] + 1])
    spec2 = W.GridSpec(ni=n[keep[0]], nj=n[keep[1]], dx=h[keep[0]], dy=h[keep[1]], bc=bc, params=spec3.params)
    sq = U3.squeeze(axis=3 - plane)   # (5, a1, a0) with a0 = keep[0] fastest
    U2 = np.stack([sq[0], sq[1 + keep[0]], sq[1 + keep[1]], sq[4]])
    return spec2, U2


@pytest.mark.parametrize("plane", [2, 1, 0])
def test_one_cell_thick_grid_equals_2d(plane):
    """A 3D grid one (periodic) cell thick along an axis, with no velocity along it, has the 2D
    oracle's residual on the other two axes: the 3D face loops, ghost resolution and 9-face
    detector reduce to the 2D ones."""
    dims = [14, 11, 9]
    dims[plane] = 1
    bc = [W.PERIODIC, W.PERIODIC, W.WALL, W.OUTFLOW, W.PERIODIC, W.PERIODIC]
    if plane == 2:
        bc = [W.WALL, W.OUTFLOW, W.PERIODIC, W.PERIODIC, W.PERIODIC, W.PERIODIC]
    spec3 = W.GridSpec3(ni=dims[0], nj=dims[1], nk=dims[2], dx=0.1, dy=0.13, dz=0.07, bc=tuple(bc),
                        params=W.SchemeParams(m_ref=0.3))
    U3 = W.random_rough_state3(spec3, seed=51, mach=1.2, jump=0.4)
    rho, u, v, w, p = W.cons_to_prim3(U3)
    vel = [u, v, w]
    vel[plane] = 0.0 * u
    U3 = W.prim_to_cons3(rho, *vel, p)
    R3 = oracle.OracleGrid3(spec3).residual(U3)
    spec2, U2 = grid2_of_3(spec3, U3, plane)
    R2 = oracle.OracleGrid(spec2).residual(U2)
    keep = [a for a in range(3) if a != plane]
    R3s = R3.squeeze(axis=3 - plane)
    assert np.max(np.abs(R3s[1 + plane])) < 1e-12 * np.max(np.abs(R2))
    got = np.stack([R3s[0], R3s[1 + keep[0]], R3s[1 + keep[1]], R3s[4]])
    assert np.max(np.abs(got - R2)) <= 1e-12 * np.max(np.abs(R2))


def test_free_stream_and_rest_in_a_box():
    """A uniform flow on a periodic grid and a fluid at rest in a closed box (walls on all six
    sides) have zero residual."""
    spec = W.GridSpec3(ni=7, nj=6, nk=5, dx=0.2, dy=0.3, dz=0.25, nscal=1)
    U = W.prim_to_cons3(np.full((5, 6, 7), 1.3), 0.4, -0.2, 0.3, 0.9, [np.full((5, 6, 7), 0.6)])
    assert np.all(oracle.OracleGrid3(spec).residual(U) == 0.0)
    box = W.GridSpec3(ni=7, nj=6, nk=5, dx=0.2, dy=0.3, dz=0.25, bc=(W.WALL,) * 6, nscal=1)
    U = W.prim_to_cons3(np.full((5, 6, 7), 1.3), 0.0, 0.0, 0.0, 0.9, [np.full((5, 6, 7), 0.6)])
    assert np.max(np.abs(oracle.OracleGrid3(box).residual(U))) < 1e-13


def test_conservation_periodic():
    spec = W.GridSpec3(ni=10, nj=9, nk=8, dx=0.1, dy=0.1, dz=0.1, nscal=2, params=W.SchemeParams(eps1=1))
    U = W.random_rough_state3(spec, seed=61, mach=0.9, jump=0.3)
    g = oracle.OracleGrid3(spec)
    T0 = g.totals(U)
    U1, _ = g.step(U, 0.4, nsteps=3)
    T1 = g.totals(U1)
    scale = np.maximum(np.abs(T0), g.totals(np.abs(U)))
    assert np.max(np.abs(T1 - T0) / scale) < 1e-13


def test_axis_permutation_symmetry():
    """Relabelling the axes (x, y, z) -> (y, z, x) of the grid, the state and the velocity
    components relabels the residual."""
    spec = W.GridSpec3(ni=8, nj=7, nk=6, dx=0.1, dy=0.12, dz=0.09, nscal=1,
                       bc=(W.WALL, W.OUTFLOW, W.PERIODIC, W.PERIODIC, W.INFLOW, W.WALL),
                       inflow=(1.2, 0.3, -0.1, 0.5, 1.1, 0.25), params=W.SchemeParams(eps1=1))
    U = W.random_rough_state3(spec, seed=71, mach=1.1, jump=0.4)
    R = oracle.OracleGrid3(spec).residual(U)
    # new axes: x' = y, y' = z, z' = x  (array axes (k, j, i) -> (i, k, j))
    spec2 = W.GridSpec3(ni=7, nj=6, nk=8, dx=0.12, dy=0.09, dz=0.1, nscal=1,
                        bc=(W.PERIODIC, W.PERIODIC, W.INFLOW, W.WALL, W.WALL, W.OUTFLOW),
                        inflow=(1.2, -0.1, 0.5, 0.3, 1.1, 0.25), params=W.SchemeParams(eps1=1))
    perm = lambda A: np.transpose(A, (2, 0, 1))
    U2 = np.stack([perm(U[0]), perm(U[2]), perm(U[3]), perm(U[1]), perm(U[4]), perm(U[5])])
    R2 = oracle.OracleGrid3(spec2).residual(U2)
    ref = np.stack([perm(R[0]), perm(R[2]), perm(R[3]), perm(R[1]), perm(R[4]), perm(R[5])])
    assert np.max(np.abs(R2 - ref)) <= 1e-12 * np.max(np.abs(R))


def test_detector_brute_force():
    """s1 on every face of a periodic grid recomputed from Eqs. 95-97 directly (9 faces)."""
    spec = W.GridSpec3(ni=5, nj=4, nk=3)
    U = W.random_rough_state3(spec, seed=81, mach=0.5, jump=0.6)
    rho, _, _, _, p = W.cons_to_prim3(U)

    def Pf(a, b):
        return min(p[a] / p[b], p[b] / p[a], rho[a] / rho[b], rho[b] / rho[a])

    def wrap(k, j, i):
        return (k % 3, j % 4, i % 5)

    g = oracle.OracleGrid3(spec)
    for ax in range(3):
        s1 = g.detector(U, ax)
        d = [0, 0, 0]
        d[2 - ax] = 1           # array index order (k, j, i)
        for k in range(3):
            for j in range(4):
                for i in range(5):
                    c0 = (k, j, i)
                    c1 = wrap(k + d[0], j + d[1], i + d[2])
                    vals = [Pf(c0, c1)]
                    for t in range(3):
                        if t == 2 - ax:
                            continue
                        e = [0, 0, 0]
                        e[t] = 1
                        for c in (c0, c1):
                            lo = wrap(c[0] - e[0], c[1] - e[1], c[2] - e[2])
                            hi = wrap(c[0] + e[0], c[1] + e[1], c[2] + e[2])
                            vals += [Pf(lo, c), Pf(c, hi)]
                    a = min(vals)
                    ref = 1.0 if a >= 1 else oracle.f(a) ** 8
                    assert abs(s1[k, j, i] - ref) < 1e-15, (ax, k, j, i)


def test_long_double_bound():
    """The FP64 oracle's residual is within 1e-13 of the long-double build's (its own rounding)."""
    spec = W.GridSpec3(ni=6, nj=5, nk=4, dx=0.1, dy=0.1, dz=0.1, nscal=1, params=W.SchemeParams(eps1=1))
    U = W.random_rough_state3(spec, seed=91, mach=1.3, jump=0.5)
    g = oracle.OracleGrid3(spec)
    R = g.residual(U)
    Rl = g.residual(U, long_double=True)
    assert np.max(np.abs(R - Rl)) <= 1e-13 * np.max(np.abs(Rl))


@pytest.mark.parametrize("walls", [False, True])
def test_power_of_two_density_pressure_scaling_is_exact_3d(walls):
    """rho -> s rho, p -> s p (scalars k unchanged, so rho k -> s rho k) at fixed velocity
    leaves the equations unchanged; with s = 2^-60 the 3D oracle's step of the scaled state is
    the scaled step bit for bit, with the same dt (no additive floor or threshold on rho or p)."""
    s = 2.0 ** -60
    bc = (W.INFLOW, W.OUTFLOW, W.WALL, W.WALL, W.WALL, W.OUTFLOW) if walls else (W.PERIODIC,) * 6
    params = W.SchemeParams(m_ref=0.3, eps1=1)
    kw = dict(ni=9, nj=8, nk=7, dx=0.05, dy=0.04, dz=0.06, nscal=1, bc=bc, params=params)
    base = W.GridSpec3(inflow=(1.2, 0.6, 0.1, -0.05, 0.9, 0.3), **kw)
    scaled = W.GridSpec3(inflow=(1.2 * s, 0.6, 0.1, -0.05, 0.9 * s, 0.3), **kw)
    U = W.random_rough_state3(base, seed=19, mach=0.9)
    U1, dt1 = oracle.OracleGrid3(base).step(U, cfl=0.4, nsteps=2)
    U2, dt2 = oracle.OracleGrid3(scaled).step(U * s, cfl=0.4, nsteps=2)
    assert dt1 == dt2
    assert np.array_equal(U2, U1 * s)


def test_periodic_shift_invariance_is_exact_3d():
    """A fully periodic 3D grid: the step of a state shifted by (2, 3, 4) cells is the shifted
    step bit for bit, with the same dt."""
    spec = W.GridSpec3(ni=9, nj=8, nk=7, dx=0.05, dy=0.04, dz=0.06, nscal=1, params=W.SchemeParams(m_ref=0.3, eps1=1))
    U = W.random_rough_state3(spec, seed=29, mach=0.9)
    U1, dt1 = oracle.OracleGrid3(spec).step(U, cfl=0.4, nsteps=2)
    Us = np.roll(U, (4, 3, 2), axis=(1, 2, 3))
    U2, dt2 = oracle.OracleGrid3(spec).step(Us, cfl=0.4, nsteps=2)
    assert dt1 == dt2
    assert np.array_equal(U2, np.roll(U1, (4, 3, 2), axis=(1, 2, 3)))


@pytest.mark.parametrize("eps1", [0, 1])
def test_stationary_contact_and_shear_layer_are_exact_3d(eps1):
    """The 3D forms of two exact steady solutions: a stationary contact (rho and the scalar
    varying from cell to cell, zero velocity, p uniform) and a shear layer (w varying with x
    only, tangential to the x-faces across which it jumps; u = v = 0; rho, p, k uniform).
    Every dissipation term vanishes at zero normal velocity without normal-velocity or pressure
    jumps, and the rotated-Riemann estimate is |U^| = 0: the residual is exactly zero."""
    rng = W.SplitMix64(37)
    spec = W.GridSpec3(ni=9, nj=8, nk=7, dx=0.05, dy=0.04, dz=0.06, nscal=1, params=W.SchemeParams(m_ref=0.3, eps1=eps1))
    g = spec.params.gamma
    shape = (spec.nk, spec.nj, spec.ni)
    rho = 0.3 + 2.0 * rng.uniforms(int(np.prod(shape))).reshape(shape)
    k = rng.uniforms(int(np.prod(shape))).reshape(shape)
    zero = np.zeros(shape)
    contact = np.stack([rho, zero, zero, zero, np.full(shape, 1.0 / (g - 1)), rho * k])
    w = np.broadcast_to(rng.uniforms(spec.ni)[None, None, :] - 0.5, shape)
    shear = np.stack([np.ones(shape), zero, zero, w, 1.0 / (g - 1) + 0.5 * w * w, np.full(shape, 0.4)])
    for U in (contact, shear):
        assert np.all(oracle.OracleGrid3(spec).residual(U) == 0.0)


def test_ssp_rk3_is_third_order_in_time_3d():
    """The 3D step is third order in time: on a smooth flow supersonic along all three axes
    (every face fully upwind, a smooth semi-discrete operator) the error against a 2048-step
    solution falls 8-fold per halving of dt."""
    spec = W.GridSpec3(ni=10, nj=9, nk=8, dx=0.05, dy=0.05, dz=0.05, nscal=1, params=W.SchemeParams(m_ref=0.5))
    g = spec.params.gamma
    x, y, z = spec.cell_centres()
    L = (spec.ni * spec.dx, spec.nj * spec.dy, spec.nk * spec.dz)
    c = math.sqrt(g)
    rho = 1 + 0.05 * np.sin(2 * np.pi * x / L[0]) * np.cos(2 * np.pi * z / L[2])
    p = 1 + 0.05 * np.cos(2 * np.pi * y / L[1] + 1.0)
    u = 2.5 * c + 0.05 * np.sin(2 * np.pi * z / L[2])
    v = 2.3 * c + 0.05 * np.cos(2 * np.pi * x / L[0])
    w = 2.1 * c + 0.05 * np.sin(2 * np.pi * y / L[1])
    k = 0.5 + 0.2 * np.sin(2 * np.pi * (x / L[0] + y / L[1]))
    U = W.prim_to_cons3(rho, u, v, w, p, scalars=(k,), gamma=g)
    T = 0.05

    def run(n):
        return oracle.OracleGrid3(spec).step(U, dt_fixed=T / n, nsteps=n)[0]

    ref = run(2048)
    errs = [np.abs(run(n) - ref).max() for n in (8, 16, 32, 64)]
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(7.5 < r < 8.6 for r in ratios), ratios
