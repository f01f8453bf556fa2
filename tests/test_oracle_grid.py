"""Pins of the oracle's grid-level residual and time step against invariants, exact
solutions and the qualitative results the paper reports (Section 7)."""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W
from riemann_exact import sample, star_state

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_cases.txt")


def read_golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        k, v = [s.strip() for s in line.split("=", 1)]
        out[k] = [eval(t, {}) for t in v.split()]   # numbers and simple fractions only
    return out


# ----------------------------------------------------------------------------- inputs
def test_golden_matches_workloads():
    g = read_golden()
    for name in ("expansion", "near_vacuum", "strong"):
        l, r, x0, t = W.SHOCK_TUBES[name]
        assert list(l) == g[f"{name}.left"] and list(r) == g[f"{name}.right"]
        assert x0 == g[f"{name}.x0"][0] and t == g[f"{name}.t"][0]
    rho, p, u, v = g["quirk.left"]
    assert (rho, u, v, p) == W.QUIRK_POST
    rho, p, u, v = g["quirk.right"]
    assert (rho, u, v, p) == W.QUIRK_PRE


def test_quirk_states_are_mach6_rankine_hugoniot():
    """The Section 7.2 states are the post-shock state of a Mach-6 shock moving into
    (1.4, 0, 0, 1) at gamma = 1.4 (normal-shock relations in the shock frame)."""
    M, g = 6.0, 1.4
    rho1, u1, _, p1 = W.QUIRK_PRE
    c1 = math.sqrt(g * p1 / rho1)
    rho2 = rho1 * (g + 1) * M * M / ((g - 1) * M * M + 2)
    p2 = p1 * (1 + 2 * g / (g + 1) * (M * M - 1))
    u2 = M * c1 * (1 - rho1 / rho2)
    assert abs(rho2 - W.QUIRK_POST[0]) < 1e-12
    assert abs(p2 - W.QUIRK_POST[3]) < 1e-12
    assert abs(u2 - W.QUIRK_POST[1]) < 1e-12


@pytest.mark.parametrize("M,post,tol", [(5.09, "CORNER_POST", 2e-5), (10.0, "DMR_POST", 1e-12)])
def test_corner_and_dmr_states_are_rankine_hugoniot(M, post, tol):
    """The Section 7.3 state (printed to 6 digits) is the post-shock state of a Mach-5.09 shock
    into still air (1.4, 0, 0, 1); the Section 7.4 one that of the Mach-10 shock."""
    g, (rho1, _, _, p1) = 1.4, W.STILL_AIR
    rho2 = rho1 * (g + 1) * M * M / ((g - 1) * M * M + 2)
    p2 = p1 * (1 + 2 * g / (g + 1) * (M * M - 1))
    u2 = M * (1 - rho1 / rho2)
    ref = getattr(W, post)
    for a, b in ((rho2, ref[0]), (u2, ref[1]), (p2, ref[3])):
        assert abs(a - b) <= tol * abs(a), (a, b)


def test_wedge_grid_geometry():
    """The Section 7.4 wedge grid: flat wall up to the tip, then a 30-degree ramp; the cell areas
    add up to the area between the lid and the piecewise-linear wall."""
    spec, _ = W.wedge_dmr(80, 20, x_tip=0.5, ramp=3.0, height=2.8)
    yb = spec.yv[0]
    slope = np.diff(yb) / np.diff(spec.xv[0])
    assert np.allclose(slope[spec.xv[0][1:] > 0.5 + 1e-9][1:], math.tan(math.pi / 6))
    ones = W.prim_to_cons(np.ones((20, 80)), 0.0, 0.0, np.ones((20, 80)))
    area = oracle.OracleGrid(spec).totals(ones)[0]
    x = spec.xv[0]
    exact = float(np.sum(np.diff(x) * (2.8 - 0.5 * (yb[1:] + yb[:-1]))))   # trapezoids under the lid
    assert abs(area - exact) <= 1e-12 * exact


def test_exact_riemann_textbook_values():
    """The exact Riemann helper reproduces published star states (Toro 2009, Table 4.2:
    Sod's problem and the left half of the blast wave, which is the Section 7.1.3 case)."""
    ps, us = star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert abs(ps - 0.30313) < 1e-5 and abs(us - 0.92745) < 1e-5
    ps, us = star_state((1.0, 0.0, 1000.0), (1.0, 0.0, 0.01))
    assert abs(ps - 460.894) < 1e-3 and abs(us - 19.5975) < 1e-4


# ----------------------------------------------------------------------------- free stream
@pytest.mark.parametrize("recon", [0, 1, 2])
def test_free_stream_cartesian_exact(recon):
    spec = W.GridSpec(ni=12, nj=9, dx=0.3, dy=0.7, params=W.SchemeParams(recon=recon, m_ref=0.05))
    U = W.free_stream(spec, u=0.31, v=-0.17)
    assert np.all(oracle.OracleGrid(spec).residual(U) == 0.0)


@pytest.mark.parametrize("recon", [0, 2])
def test_free_stream_warped(recon):
    spec = W.with_params(W.warped_periodic(16), recon=recon, m_ref=0.3)
    U = W.free_stream(spec, u=0.31, v=-0.17)
    R = oracle.OracleGrid(spec).residual(U)
    # flux scale / cell volume * rounding
    assert np.max(np.abs(R)) < 1e-12 * 1.5 / (1 / 16) ** 2 * (1 / 16)


def test_wall_channel_free_stream():
    """Uniform flow parallel to the S/N walls, inflow W, outflow E: R = 0 (mirror states
    of a tangential flow reproduce it; the walls carry only pressure)."""
    spec = W.GridSpec(ni=10, nj=6, bc=(W.INFLOW, W.OUTFLOW, W.WALL, W.WALL), inflow=(1.2, 0.8, 0.0, 0.9),
                      params=W.SchemeParams(recon=2, m_ref=0.5))
    U = W.free_stream(spec, 1.2, 0.8, 0.0, 0.9)
    assert np.max(np.abs(oracle.OracleGrid(spec).residual(U))) < 1e-14


def test_rest_state_with_solid_block_on_warped_grid():
    spec, _ = W.warped_step(48, 16, recon=2)
    U = W.free_stream(spec, 1.4, 0.0, 0.0, 1.0)
    spec.bc = (W.WALL, W.WALL, W.WALL, W.WALL)
    R = oracle.OracleGrid(spec).residual(U)
    assert np.max(np.abs(R)) < 1e-11 * 1.0 / (3.0 / 48)


# ----------------------------------------------------------------------------- conservation
@pytest.mark.parametrize("case", ["cart1", "cart_muscl", "warped", "eps1"])
def test_conservation_periodic(case):
    if case == "warped":
        spec = W.with_params(W.warped_periodic(16), recon=2)
    else:
        spec = W.GridSpec(ni=14, nj=11, dx=1 / 14, dy=1 / 11,
                          params=W.SchemeParams(recon=0 if case == "cart1" else 1, eps1=int(case == "eps1")))
    U = W.random_smooth_state(spec, seed=3, mach=0.8, amp=0.4)
    g = oracle.OracleGrid(spec)
    T0 = g.totals(U)
    U1, _ = g.step(U, cfl=0.5, nsteps=5)
    T1 = g.totals(U1)
    assert np.all(np.abs(T1 - T0) <= 1e-14 * np.abs(T0).max() * 20)


# ----------------------------------------------------------------------------- symmetry
def _mirror_x(U):
    V = U[:, :, ::-1].copy()
    V[1] = -V[1]
    return V


@pytest.mark.parametrize("params", [dict(recon=0), dict(recon=1), dict(recon=2, eps1=1)])
def test_mirror_symmetry(params):
    spec = W.GridSpec(ni=12, nj=8, dx=0.1, dy=0.1, params=W.SchemeParams(m_ref=0.3, **params))
    U = W.random_rough_state(spec, seed=7, mach=1.5)
    Us = 0.5 * (U + _mirror_x(U))   # symmetric in x (u antisymmetric)
    R = oracle.OracleGrid(spec).residual(Us)
    assert np.max(np.abs(R - _mirror_x(R))) < 1e-12 * np.max(np.abs(R))


@pytest.mark.parametrize("params", [dict(recon=0), dict(recon=1), dict(recon=2, eps1=1)])
def test_transpose_symmetry(params):
    """Swapping x <-> y (and u <-> v) transposes the residual: pins the y-face indexing
    and the transposed detector stencil."""
    spec = W.GridSpec(ni=9, nj=7, dx=0.2, dy=0.3, params=W.SchemeParams(m_ref=0.3, **params))
    U = W.random_rough_state(spec, seed=9, mach=1.5)
    R = oracle.OracleGrid(spec).residual(U)
    specT = W.GridSpec(ni=7, nj=9, dx=0.3, dy=0.2, params=spec.params)
    UT = np.stack([U[0].T, U[2].T, U[1].T, U[3].T])
    RT = oracle.OracleGrid(specT).residual(UT)
    expect = np.stack([R[0].T, R[2].T, R[1].T, R[3].T])
    assert np.max(np.abs(RT - expect)) < 1e-12 * np.max(np.abs(R))


# ----------------------------------------------------------------------------- MUSCL limiters
# Reading A14 (the paper's tests are first order, Section 7): MUSCL on primitives,
# W_L = W_i + lim(W_i - W_{i-1}, W_{i+1} - W_i) / 2, W_R = W_{i+1} - lim(W_{i+1} - W_i,
# W_{i+2} - W_{i+1}) / 2, with minmod(a, b) = (sgn a + sgn b) min(|a|, |b|) / 2 and van Leer
# (a|b| + |a|b) / (|a| + |b|), 0 when ab <= 0.
#
# Four-cell stencils (cells i-1, i, i+1, i+2; face between i and i+1) with the face states
# worked out by hand from those definitions (slopes a = W_i - W_{i-1}, b = W_{i+1} - W_i on
# the left; a' = W_{i+1} - W_i, b' = W_{i+2} - W_{i+1} on the right):
#   (1, 2, 4, 5): left a = 1, b = 2; right a' = 2, b' = 1.
#       minmod: W_L = 2 + 1/2 = 2.5,  W_R = 4 - 1/2 = 3.5
#       van Leer: lim = 2 * 1 * 2 / 3 = 4/3 on both sides: W_L = 8/3, W_R = 10/3
#   (1, 3, 2, 2.5): left a = 2, b = -1 (opposite signs); right a' = -1, b' = 0.5 (opposite):
#       both limiters: W_L = 3, W_R = 2 (first order)
#   (3, 3, 5, 6): left a = 0 (flat); right a' = 2, b' = 1:
#       minmod: W_L = 3, W_R = 5 - 1/2 = 4.5;  van Leer: W_L = 3, W_R = 5 - 2/3 = 13/3
#   (6, 4, 3, 1): left a = -2, b = -1; right a' = -1, b' = -2 (both decreasing):
#       minmod: W_L = 4 - 1/2 = 3.5, W_R = 3 + 1/2 = 3.5
#       van Leer: lim = -4/3 on both sides: W_L = 4 - 2/3 = 10/3, W_R = 3 + 2/3 = 11/3
# A minmod taking the larger slope, or a van Leer without limiting (the central slope
# (a + b)/2), misses at least one of these values.
HAND_STENCILS = [
    ((1.0, 2.0, 4.0, 5.0), {1: (2.5, 3.5), 2: (8 / 3, 10 / 3)}),
    ((1.0, 3.0, 2.0, 2.5), {1: (3.0, 2.0), 2: (3.0, 2.0)}),
    ((3.0, 3.0, 5.0, 6.0), {1: (3.0, 4.5), 2: (3.0, 13 / 3)}),
    ((6.0, 4.0, 3.0, 1.0), {1: (3.5, 3.5), 2: (10 / 3, 11 / 3)}),
]


def _stencil_grid(vals, recon, axis):
    """A periodic 8 x 4 grid (4 x 8 for axis 1) whose primitives vary along `axis` only: the
    stencil occupies cells 2..5 and the face under test lies between cells 3 and 4. Each
    primitive is an affine image of the stencil values (the limiters commute with positive
    scaling and with negation, so the face states are the same images of the hand values)."""
    prof = np.array([vals[0], vals[0], vals[0], vals[1], vals[2], vals[3], vals[3], vals[3]])
    rho, u, v, p = 1.0 + prof, 0.1 * prof, -0.05 * prof, 2.0 * prof + 0.5
    if axis == 0:
        spec = W.GridSpec(ni=8, nj=4, dx=0.1, dy=0.1, params=W.SchemeParams(recon=recon))
        ext = lambda a: np.broadcast_to(a[None, :], (4, 8))
    else:
        spec = W.GridSpec(ni=4, nj=8, dx=0.1, dy=0.1, params=W.SchemeParams(recon=recon))
        ext = lambda a: np.broadcast_to(a[:, None], (8, 4))
    U = W.prim_to_cons(ext(rho), ext(u), ext(v), ext(p))
    return spec, U


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("recon", [1, 2])
def test_muscl_face_states_hand_values(recon, axis):
    for vals, expect in HAND_STENCILS:
        spec, U = _stencil_grid(vals, recon, axis)
        cells = [(3, 1)] if axis == 0 else [(1, 3)]
        WL, WR = oracle.OracleGrid(spec).face_states(U, cells, [axis])
        hl, hr = expect[recon]
        want_L = np.array([1.0 + hl, 0.1 * hl, -0.05 * hl, 2.0 * hl + 0.5])
        want_R = np.array([1.0 + hr, 0.1 * hr, -0.05 * hr, 2.0 * hr + 0.5])
        assert np.allclose(WL[0], want_L, rtol=1e-13, atol=1e-15), (vals, recon, WL[0], want_L)
        assert np.allclose(WR[0], want_R, rtol=1e-13, atol=1e-15), (vals, recon, WR[0], want_R)


@pytest.mark.parametrize("recon", [1, 2])
def test_muscl_face_states_stay_between_cells(recon):
    """Both limiters keep each reconstructed primitive between the face's two cell values
    (minmod: |lim| <= min(|a|, |b|); van Leer: the harmonic mean is at most twice the smaller
    slope), on every face of rough random states, Cartesian and warped."""
    for spec in (W.GridSpec(ni=11, nj=9, dx=0.1, dy=0.2, params=W.SchemeParams(recon=recon)),
                 W.with_params(W.warped_periodic(12), recon=recon)):
        for seed in (1, 2, 3):
            U = W.random_rough_state(spec, seed=seed, mach=1.5, jump=0.8)
            W0 = np.stack(W.cons_to_prim(U))
            ni, nj = spec.ni, spec.nj
            cells = [(i, j) for j in range(nj) for i in range(ni)]
            for axis in (0, 1):
                WL, WR = oracle.OracleGrid(spec).face_states(U, cells, [axis] * len(cells))
                for f, (i, j) in enumerate(cells):
                    A = W0[:, j, i]
                    B = W0[:, (j + axis) % nj, (i + 1 - axis) % ni]
                    lo, hi = np.minimum(A, B), np.maximum(A, B)
                    tol = 1e-14 * np.maximum(np.abs(A), np.abs(B))
                    assert np.all(WL[f] >= lo - tol) and np.all(WL[f] <= hi + tol), (recon, i, j, axis)
                    assert np.all(WR[f] >= lo - tol) and np.all(WR[f] <= hi + tol), (recon, i, j, axis)
            # and the limiter does limit: somewhere the face state differs from first order
            WL, _ = oracle.OracleGrid(spec).face_states(U, cells, [0] * len(cells))
            assert np.max(np.abs(WL - W0.reshape(4, -1).T)) > 1e-3


@pytest.mark.parametrize("recon", [1, 2])
def test_muscl_expansion_tube_creates_no_new_extrema(recon):
    """Section 7.1.1's expansion tube with MUSCL: over ten steps at CFL 0.4 no density or
    pressure leaves the range of the initial data (the limited reconstruction adds no
    extrema; an unlimited or wrongly limited slope overshoots at the contact and the
    shock)."""
    spec, U = W.shock_tube("expansion", 200, 2, recon=recon)
    g = oracle.OracleGrid(spec)
    r0, _, _, p0 = W.cons_to_prim(U)
    for _ in range(10):
        U, _ = g.step(U, cfl=0.4)
        r, _, _, p = W.cons_to_prim(U)
        assert r.max() <= r0.max() * (1 + 1e-13) and r.min() >= r0.min() * (1 - 1e-13)
        assert p.max() <= p0.max() * (1 + 1e-13) and p.min() >= p0.min() * (1 - 1e-13)


# ----------------------------------------------------------------------------- detector
def test_detector_brute_force():
    """Eqs. 95-97 on a tiny periodic grid, evaluated from the definition by brute force:
    a = min of P over the face and the four transverse faces of its two cells."""
    spec = W.GridSpec(ni=6, nj=5, params=W.SchemeParams())
    U = W.random_rough_state(spec, seed=17, jump=0.8)
    rho, _, _, p = W.cons_to_prim(U)
    ni, nj = 6, 5

    def P(a, b):
        (ia, ja), (ib, jb) = a, b
        ra, pa = rho[ja % nj, ia % ni], p[ja % nj, ia % ni]
        rb, pb = rho[jb % nj, ib % ni], p[jb % nj, ib % ni]
        return min(pa / pb, pb / pa, ra / rb, rb / ra)

    sx, sy = oracle.OracleGrid(spec).detector(U)
    for j in range(nj):
        for ic in range(ni + 1):
            i = ic - 1
            a = min(P((i, j), (i + 1, j)), P((i + 1, j), (i + 1, j - 1)), P((i + 1, j), (i + 1, j + 1)),
                    P((i, j), (i, j - 1)), P((i, j), (i, j + 1)))
            assert abs(sx[j, ic] - oracle.f(a) ** 8) < 1e-15
    for jc in range(nj + 1):
        for i in range(ni):
            j = jc - 1
            a = min(P((i, j), (i, j + 1)), P((i, j + 1), (i - 1, j + 1)), P((i, j + 1), (i + 1, j + 1)),
                    P((i, j), (i - 1, j)), P((i, j), (i + 1, j)))
            assert abs(sy[jc, i] - oracle.f(a) ** 8) < 1e-15


# ----------------------------------------------------------------------------- shock tubes
def run_tube(name, ni, cfl=0.5, ramp=False, **variant):
    spec, U = W.shock_tube(name, ni, 2)
    g = oracle.OracleGrid(spec, **variant)
    tend = W.SHOCK_TUBES[name][3]
    t, n = 0.0, 0
    while t < tend - 1e-14:
        c = min(cfl, 0.02 * 1.05 ** n) if ramp else cfl
        dt = min(c / g.max_rate(U), tend - t)
        U, _ = g.step(U, dt_fixed=dt)
        t += dt
        n += 1
        rho, _, _, p = W.cons_to_prim(U)
        if not (np.all(np.isfinite(p)) and p.min() > 0 and rho.min() > 0):
            return None, spec
    return U, spec


def l1_density_error(name, U, spec):
    l, r, x0, t = W.SHOCK_TUBES[name]
    xc, _ = spec.cell_centres()
    rho_ex, _, _ = sample(l, r, (xc[0] - x0) / t)
    return float(np.mean(np.abs(U[0, 0] - rho_ex)))


@pytest.mark.parametrize("name,ramp", [("expansion", False), ("near_vacuum", False), ("strong", True)])
def test_shock_tube_converges_to_exact(name, ramp):
    errs = []
    for ni in (100, 200, 400):
        U, spec = run_tube(name, ni, ramp=ramp, cfl=0.4 if ramp else 0.5)
        assert U is not None, (name, ni)
        errs.append(l1_density_error(name, U, spec))
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 0.7 * errs[0], errs


def test_expansion_shock_removed_by_eq92():
    """Section 7.1.1 / Fig. 3: classical Roe and Roe-AM without Eq. 92 keep an expansion
    shock at x = 0.3; the complete Roe-AM does not."""
    def max_jump(U):
        return float(np.max(np.abs(np.diff(U[0, 0]))[50:70]))   # cells around x = 0.3 (ni = 200)
    full, _ = run_tube("expansion", 200)
    nofix, _ = run_tube("expansion", 200, ufix=0)
    roe, _ = run_tube("expansion", 200, scheme=1)
    harten, _ = run_tube("expansion", 200, scheme=1, harten=0.2)
    assert max_jump(full) < 0.15
    assert max_jump(nofix) > 0.5 and max_jump(roe) > 0.5
    assert max_jump(harten) < 0.15   # the entropy fix of Eqs. 114-115 also removes it


def test_near_vacuum_positivity():
    """Section 7.1.2: Roe-AM keeps rho, p > 0 in the near-vacuum test; classical Roe fails
    (Section 4.3: the positivity conditions)."""
    U, _ = run_tube("near_vacuum", 200)
    assert U is not None
    U_roe, _ = run_tube("near_vacuum", 200, scheme=1)
    assert U_roe is None
    # the velocity-positivity form of xi (Eq. 86) is what keeps Roe-AM positive here: with
    # xi = |U| of Eq. 13 it fails like Roe; the Roe form of delta U_p does not matter
    U_xi, _ = run_tube("near_vacuum", 200, xi_roe=1)
    assert U_xi is None
    U_dup, _ = run_tube("near_vacuum", 200, dup_mode=2)
    assert U_dup is not None


# ----------------------------------------------------------------------------- low Mach
def test_low_mach_residual_scaling():
    """Section 3 asymptotics on the well-prepared Gresho vortex (p = p0 + M^2 p2): the
    Roe-AM momentum residual stays O(1) as M -> 0, the classical Roe residual grows as 1/M
    (the non-physical O(M) pressure mechanism that Eq. 88's f(M) removes)."""
    res = {}
    for scheme in (0, 1):
        v = []
        for M in (0.1, 0.01, 0.001):
            spec, U = W.gresho(32, mach=M, checker=0, recon=0)
            v.append(np.max(np.abs(oracle.OracleGrid(spec, scheme=scheme).residual(U)[1])))
        res[scheme] = (math.log10(v[0] / v[1]), math.log10(v[1] / v[2]))
    assert all(abs(s) < 0.05 for s in res[0]), res
    assert all(abs(s + 1) < 0.1 for s in res[1]), res


def test_checkerboard_mode():
    """Section 7.6: the pure pressure checkerboard at rest is invisible to the scheme with
    delta U_p = 0 (a stationary spurious mode); the Roe-AM delta U_p of Eq. 89 damps it
    (energy leaves the high-pressure cells)."""
    spec = W.GridSpec(ni=8, nj=8, dx=1 / 8, dy=1 / 8, params=W.SchemeParams(m_ref=0.01))
    jj, ii = np.meshgrid(np.arange(8), np.arange(8), indexing="ij")
    sign = np.where((ii + jj) % 2 == 0, 1.0, -1.0)
    p = 1 / 1.4 + 1e-6 * sign
    U = W.prim_to_cons(np.ones((8, 8)), 0.0, 0.0, p)
    R0 = oracle.OracleGrid(spec, dup_mode=1).residual(U)
    assert np.max(np.abs(R0)) < 1e-12
    R = oracle.OracleGrid(spec).residual(U)
    assert np.all(R[3] * sign < 0)


# ----------------------------------------------------------------------------- vortex
@pytest.mark.parametrize("recon,order", [(0, 0.7), (1, 1.4), (2, 1.4)])
def test_isentropic_vortex_convergence(recon, order):
    """Advected isentropic vortex: the error against the exact translated solution falls
    at the expected rate (about 1 at first order; 1.6-1.8 with minmod, which clips the
    slopes at the vortex's extrema, and about 2 with van Leer MUSCL)."""
    errs = []
    tend = 1.0
    for n in (32, 64, 128):
        spec, U = W.isentropic_vortex(n, recon=recon)
        g = oracle.OracleGrid(spec)
        t = 0.0
        while t < tend - 1e-14:
            dt = min(0.5 / g.max_rate(U), tend - t)
            U, _ = g.step(U, dt_fixed=dt)
            t += dt
        _, Ue = W.isentropic_vortex(n, t=tend, recon=recon)
        errs.append(float(np.sqrt(np.mean((U[0] - Ue[0]) ** 2))))
    rates = [math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])]
    assert min(rates) > order, (errs, rates)


def test_classical_roe_time_step_rule():
    """The classical Roe scheme takes theta = 1 in the time-step rule: on a Cartesian grid the
    rate is max_i (|u| + c) / dx + (|v| + c) / dy (closed form); Roe-AM at low M_ref is faster."""
    spec = W.GridSpec(ni=12, nj=9, dx=0.1, dy=0.07, params=W.SchemeParams(m_ref=0.05, scheme=1))
    U = W.random_smooth_state(spec, seed=4, mach=0.3, amp=0.3)
    rho, u, v, p = W.cons_to_prim(U)
    c = np.sqrt(1.4 * p / rho)
    ref = np.max((np.abs(u) + c) / spec.dx + (np.abs(v) + c) / spec.dy)
    rate = oracle.OracleGrid(spec).max_rate(U)
    assert abs(rate - ref) <= 1e-14 * ref
    assert oracle.OracleGrid(W.with_params(spec, scheme=0)).max_rate(U) > 2 * ref


# ----------------------------------------------------------------------------- cylinder grids
def test_ogrid_area_and_closure():
    """The O-grid of the Section 7.6 cylinder: total cell area equals the polygonal annulus
    (ni/2) sin(2 pi/ni) (r_far^2 - 1) (closed form), and a uniform flow has zero residual in
    every cell off the wall row (closed cells, bit-identical periodic seam, far field = free
    stream)."""
    spec, _ = W.cylinder_ogrid(ni=40, nj=24, mach=0.3, r_far=10.0)
    g = oracle.OracleGrid(spec)
    ones = W.prim_to_cons(np.ones((24, 40)), 0.0, 0.0, np.ones((24, 40)))
    area = g.totals(ones)[0]
    assert abs(area - 20 * math.sin(2 * math.pi / 40) * (100 - 1)) <= 1e-12 * area
    U = W.free_stream(spec, 1.0, 0.3, 0.0, 1 / 1.4)
    R = g.residual(U)
    xv, yv = spec.xv, spec.yv
    edge = lambda a, b: np.hypot(xv[a] - xv[b], yv[a] - yv[b])
    perim = (edge((slice(None, -1), slice(None, -1)), (slice(None, -1), slice(1, None))) +
             edge((slice(1, None), slice(None, -1)), (slice(1, None), slice(1, None))) +
             edge((slice(None, -1), slice(None, -1)), (slice(1, None), slice(None, -1))) +
             edge((slice(None, -1), slice(1, None)), (slice(1, None), slice(1, None))))
    Vc = 0.5 * ((xv[1:, 1:] - xv[:-1, :-1]) * (yv[1:, :-1] - yv[:-1, 1:]) -
                (yv[1:, 1:] - yv[:-1, :-1]) * (xv[1:, :-1] - xv[:-1, 1:]))
    scale = np.max((1 / 1.4 + 0.09) * perim / Vc)    # |F| |S| / V bound of the face fluxes
    assert np.max(np.abs(R[:, 1:])) <= 1e-13 * scale, np.max(np.abs(R[:, 1:])) / scale
    assert np.max(np.abs(R[:, 0])) > 1e-6   # the wall does act


@pytest.mark.parametrize("gen", ["ogrid", "blunt"])
def test_cylinder_mirror_symmetry(gen):
    """Both cylinder grids are symmetric about the x-axis with cell i mirrored to ni-1-i; the
    residual of a mirror-symmetric state is mirror-symmetric (rho v odd)."""
    if gen == "ogrid":
        spec, U = W.cylinder_ogrid(ni=40, nj=20, mach=0.2, r_far=8.0)
    else:
        spec, U = W.cylinder_blunt(ni=40, nj=10, mach=3.0)
        U = U * (1 + 0.1 * np.sin(np.linspace(0, 3, 10))[None, :, None] * np.array([1, 0, 0, 1])[:, None, None])
    R = oracle.OracleGrid(spec).residual(U)
    Rm = R[:, :, ::-1].copy()
    Rm[2] *= -1
    assert np.max(np.abs(R - Rm)) <= 1e-12 * np.max(np.abs(R))


@pytest.mark.parametrize("recon", [0, 1, 2])
@pytest.mark.parametrize("walls", [False, True])
def test_power_of_two_density_pressure_scaling_is_exact(recon, walls):
    """rho -> s rho, p -> s p at fixed velocity leaves the Euler equations unchanged. With
    s = 2^-60 every operation of a consistent scheme scales exactly in binary (square roots
    by 2^-30, quotients of like quantities not at all), so a step of the scaled state equals
    the scaled step bit for bit with the same dt: an additive floor or a threshold on rho or p
    anywhere in the flux, detector, reconstruction, boundary values or time step breaks it."""
    s = 2.0 ** -60
    bc = (W.INFLOW, W.OUTFLOW, W.WALL, W.WALL) if walls else (W.PERIODIC,) * 4
    params = W.SchemeParams(m_ref=0.3, recon=recon, eps1=1)
    base = W.GridSpec(ni=23, nj=17, dx=0.05, dy=0.04, bc=bc, inflow=(1.2, 0.6, 0.1, 0.9), params=params)
    scaled = W.GridSpec(ni=23, nj=17, dx=0.05, dy=0.04, bc=bc, inflow=(1.2 * s, 0.6, 0.1, 0.9 * s), params=params)
    U = W.random_rough_state(base, seed=17, mach=0.9, jump=0.5)
    U1, dt1 = oracle.OracleGrid(base).step(U, cfl=0.4, nsteps=2)
    U2, dt2 = oracle.OracleGrid(scaled).step(U * s, cfl=0.4, nsteps=2)
    assert dt1 == dt2
    assert np.array_equal(U2, U1 * s)


@pytest.mark.parametrize("recon", [0, 2])
def test_periodic_shift_invariance_is_exact(recon):
    """On a fully periodic grid no cell is special: stepping a state shifted by (3, 5) cells
    gives the shifted step, with the same dt, up to rounding (the oracle builds face vectors
    and volumes from vertex coordinates, whose differences round differently from cell to
    cell); a wrong index in the periodic wrap of the faces, the detector's transverse faces or
    the reconstruction stencil changes cells near the seam at first order."""
    spec = W.GridSpec(ni=19, nj=14, dx=0.05, dy=0.04, params=W.SchemeParams(m_ref=0.3, recon=recon, eps1=1))
    U = W.random_rough_state(spec, seed=23, mach=0.9, jump=0.5)
    U1, dt1 = oracle.OracleGrid(spec).step(U, cfl=0.4, nsteps=2)
    Us = np.roll(U, (5, 3), axis=(1, 2))
    U2, dt2 = oracle.OracleGrid(spec).step(Us, cfl=0.4, nsteps=2)
    assert abs(dt2 - dt1) <= 1e-13 * dt1
    err = np.abs(U2 - np.roll(U1, (5, 3), axis=(1, 2))).reshape(4, -1).max(axis=1)
    assert np.all(err <= 1e-13 * np.abs(U1).reshape(4, -1).max(axis=1)), err


@pytest.mark.parametrize("recon", [0, 1, 2])
@pytest.mark.parametrize("eps1", [0, 1])
def test_stationary_contact_and_shear_layer_are_exact(recon, eps1):
    """Two exact steady solutions that a Roe-type dissipation must leave alone: a stationary
    contact (rho varying from cell to cell, u = v = 0, p uniform) and a stationary shear layer
    (v varying with x only, u = 0, rho and p uniform). On every face the normal velocity and
    the jumps of normal velocity and pressure are zero, so each term of Eq. 85's dissipation
    vanishes (xi of Eq. 86 and its eps1 floor, dp_p, dp_u, dU_p, dU_u; for the shear layer the
    rotated-Riemann estimate of Eqs. 103-109 is |U^| = 0), and the central fluxes of a cell's
    opposite faces cancel: the residual is exactly zero."""
    rng = W.SplitMix64(31)
    spec = W.GridSpec(ni=16, nj=12, dx=0.05, dy=0.04, params=W.SchemeParams(m_ref=0.3, recon=recon, eps1=eps1))
    g = spec.params.gamma
    rho = 0.3 + 2.0 * rng.uniforms(spec.ni * spec.nj).reshape(spec.nj, spec.ni)
    zero = np.zeros_like(rho)
    contact = np.stack([rho, zero, zero, np.full_like(rho, 1.0 / (g - 1))])
    v = np.broadcast_to(rng.uniforms(spec.ni)[None, :] - 0.5, rho.shape)
    shear = np.stack([np.ones_like(rho), zero, v, 1.0 / (g - 1) + 0.5 * v * v])
    for U in (contact, shear):
        assert np.all(oracle.OracleGrid(spec).residual(U) == 0.0)


def test_ssp_rk3_is_third_order_in_time():
    """The stage combinations (1, 0), (3/4, 1/4), (1/3, 2/3) make the step third-order accurate
    in time: on a smooth flow that is supersonic in both directions (every face fully upwind by
    Eq. 44, so the semi-discrete operator is smooth) the error against a 4096-step solution
    falls 8-fold per halving of dt (a wrong combination gives first or second order)."""
    spec = W.GridSpec(ni=24, nj=20, dx=0.05, dy=0.05, params=W.SchemeParams(m_ref=0.5))
    g = spec.params.gamma
    x, y = spec.cell_centres()
    Lx, Ly = spec.ni * spec.dx, spec.nj * spec.dy
    c = math.sqrt(g)
    rho = 1 + 0.05 * np.sin(2 * np.pi * x / Lx) * np.cos(2 * np.pi * y / Ly)
    p = 1 + 0.05 * np.cos(2 * np.pi * x / Lx + 1.0)
    u = 2.5 * c + 0.05 * np.sin(2 * np.pi * y / Ly)
    v = 2.2 * c + 0.05 * np.cos(2 * np.pi * x / Lx)
    U = W.prim_to_cons(rho, u, v, p, gamma=g)
    T = 0.1

    def run(n):
        return oracle.OracleGrid(spec).step(U, dt_fixed=T / n, nsteps=n)[0]

    ref = run(4096)
    errs = [np.abs(run(n) - ref).max() for n in (16, 32, 64, 128)]
    ratios = [errs[k] / errs[k + 1] for k in range(3)]
    assert all(7.5 < r < 8.6 for r in ratios), ratios


@pytest.mark.parametrize("recon", [0, 1, 2])
@pytest.mark.parametrize("warped", [False, True])
def test_closed_box_conserves_mass_and_energy(recon, warped):
    """Walls on all four sides: a wall face's mirror state has the same rho, p and tangential
    velocity and the opposite normal velocity, so its Roe-average normal velocity is zero and
    every mass and energy term of the face flux vanishes (the central part cancels; xi acts on
    zero jumps; dU_u and the pressure-jump terms are zero). Total mass and energy of a rough
    state are then conserved to rounding, on a Cartesian and on a warped grid (a mirror of the
    wrong velocity component lets mass through the walls)."""
    params = W.SchemeParams(m_ref=0.4, recon=recon, eps1=1)
    if warped:
        spec = W.with_params(W.warped_periodic(20, amp=0.15), m_ref=0.4, recon=recon, eps1=1)
        spec.bc = (W.WALL,) * 4
    else:
        spec = W.GridSpec(ni=21, nj=17, dx=0.05, dy=0.04, bc=(W.WALL,) * 4, params=params)
    U = W.random_rough_state(spec, seed=41, mach=0.8, jump=0.4)
    g = oracle.OracleGrid(spec)
    T0 = g.totals(U)
    U1, _ = g.step(U, cfl=0.4, nsteps=3)
    T1 = g.totals(U1)
    for k in (0, 3):
        assert abs(T1[k] - T0[k]) <= 1e-13 * abs(T0[k]), (k, T0[k], T1[k])


def _residual_jacobian(spec, U, h=1e-7):
    """Central-difference Jacobian of the oracle residual (4 ni nj unknowns)."""
    g = oracle.OracleGrid(spec)
    n = U.size
    J = np.empty((n, n))
    for k in range(n):
        Up = U.copy().ravel()
        Um = U.copy().ravel()
        d = h * max(1.0, abs(Up[k]))
        Up[k] += d
        Um[k] -= d
        J[:, k] = (g.residual(Up.reshape(U.shape)) - g.residual(Um.reshape(U.shape))).ravel() / (2 * d)
    return J


@pytest.mark.parametrize("mach", [0.01, 0.05])
def test_time_step_rule_keeps_the_step_stable_at_low_mach(mach):
    """Reading R13 (the paper gives no time-step rule): the rate sum_dir (|U| + max(c, c~/theta))
    |S| / V bounds the scheme's fastest mode. Linearising the oracle residual on a smooth low-Mach
    state (8 x 8 periodic, M_ref = M) and applying SSP-RK3's amplification 1 + z + z^2/2 + z^3/6
    to its eigenvalues: with dt = 0.5 / rate no mode grows faster than the smooth flow itself
    (|g| <= 1 + 2e-3 per step), while the classical |U| + c rule at the same CFL lets the
    preconditioned delta U_p of Eq. 89 blow up (|g| > 100); the spectral radius stays within 2.5
    times the rate (SSP-RK3 is stable to -2.51 on the negative real axis)."""
    spec = W.GridSpec(ni=8, nj=8, dx=0.1, dy=0.1, params=W.SchemeParams(m_ref=mach))
    U = W.random_smooth_state(spec, seed=3, mach=mach, amp=0.02)
    lam = np.linalg.eigvals(_residual_jacobian(spec, U))
    rate = oracle.OracleGrid(spec).max_rate(U)
    rate_classical = oracle.OracleGrid(W.with_params(spec, scheme=1)).max_rate(U)

    def gmax(dt):
        z = dt * lam
        return float(np.max(np.abs(1 + z + z ** 2 / 2 + z ** 3 / 6)))

    assert gmax(0.5 / rate) <= 1 + 2e-3
    assert gmax(0.5 / rate_classical) > 100
    assert np.max(np.abs(lam)) <= 2.5 * rate
