"""GPU positive controls for the paper's Section 7 ablations: the variants the paper compares
Roe-AM with (classical Roe with and without the entropy fix of Eqs. 114-115; Roe-AM without
Eq. 92, with xi = |U| of Eq. 13, with delta U_p = 0 or the Roe form of Eq. 17) run on the GPU
and show the failures the paper reports, while Roe-AM does not.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from riemann_exact import sample

pytestmark = pytest.mark.gpu


def P():
    import paper_1711_09272_gb300 as pkg
    return pkg


def state_scale(U):
    m = np.sqrt(U[1] ** 2 + U[2] ** 2).max()
    return np.array([np.abs(U[0]).max(), m, m, np.abs(U[3]).max()])


def run_tube_gpu(name, prec=64, **variant):
    """Runs a Section 7.1 tube to its end time on the GPU; returns (state, dts)."""
    spec, U = W.shock_tube(name, 200, 4)
    spec = W.with_params(spec, **variant)
    tend = W.SHOCK_TUBES[name][3]
    ramp = name == "strong"
    dts = []
    with P().Batch([spec], precision=prec) as b:
        b.set_state(U, 0)
        Ug = U
        t, n = 0.0, 0
        while t < tend - 1e-14:
            cfl = min(0.4, 0.02 * 1.05 ** n) if ramp else 0.5
            dt = b.step(cfl, nsteps=1, want_dt=True)[0]
            if t + dt > tend:   # redo the last step with the remaining time
                b.set_state(Ug, 0)
                dt = tend - t
                b.step(0.5, dt_fixed=dt, nsteps=1)
            Ug = b.get_state(0)   # raises on a non-positive or non-finite state
            dts.append(dt)
            t += dt
            n += 1
    return spec, U, Ug, dts


def max_jump(U):
    return float(np.max(np.abs(np.diff(U[0, 0]))[50:70]))   # cells around x = 0.3


@pytest.mark.parametrize("variant,shock", [(dict(ufix=0), True), (dict(scheme=1), True),
                                           (dict(scheme=1, harten=0.2), False)])
def test_expansion_shock_variants(variant, shock):
    """Section 7.1.1 / Fig. 3: classical Roe and Roe-AM without Eq. 92 keep an expansion shock
    at x = 0.3 (the entropy fix removes it); the GPU trajectory follows the oracle's."""
    spec, U, Ug, dts = run_tube_gpu("expansion", **variant)
    g = oracle.OracleGrid(spec)
    Uo = U.copy()
    for dt in dts:
        Uo, _ = g.step(Uo, dt_fixed=dt)
    assert np.max(np.abs(Ug - Uo).reshape(4, -1).max(axis=1) / state_scale(Uo)) < 1e-9
    assert (max_jump(Ug) > 0.5) == shock, max_jump(Ug)


def test_strong_shock_roe_as_robust_as_roeam():
    """Section 7.1.3 / Fig. 5: classical Roe gets through the strong-shock tube like Roe-AM, with
    the same accuracy."""
    errs = {}
    for scheme in (0, 1):
        spec, U, Ug, _ = run_tube_gpu("strong", scheme=scheme)
        l, r, x0, t = W.SHOCK_TUBES["strong"]
        xc, _ = spec.cell_centres()
        rho_ex, _, _ = sample(l, r, (xc[0] - x0) / t)
        errs[scheme] = float(np.mean(np.abs(Ug[0, 0] - rho_ex)))
    assert abs(errs[1] - errs[0]) < 0.05 * errs[0], errs


@pytest.mark.parametrize("variant,fails", [(dict(), False), (dict(scheme=1), True), (dict(xi_roe=1), True),
                                           (dict(dup_mode=2), False)])
def test_near_vacuum_positivity_variants(variant, fails):
    """Section 7.1.2: classical Roe fails in the near-vacuum tube and so does Roe-AM with
    xi = |U| (without the velocity-positivity xi of Eq. 86); the device reports the failure as
    a status, the context stays usable."""
    if not fails:
        _, _, Ug, _ = run_tube_gpu("near_vacuum", **variant)
        assert np.all(W.cons_to_prim(Ug)[3] > 0)
        return
    with pytest.raises(P().RoeamError) as e:
        run_tube_gpu("near_vacuum", **variant)
    assert e.value.status in (4, 5)
    # the library keeps working after a reported failure
    _, _, Ug, _ = run_tube_gpu("near_vacuum")
    assert np.all(W.cons_to_prim(Ug)[0] > 0)


QUIRK_VARIANTS = {
    # name: (variant, min indicator, max indicator, min front spread, max front spread)
    "roe": (dict(scheme=1), 0.8, 9.0, 50, 800),                     # Fig. 6(a)
    "roe_harten_0.05": (dict(scheme=1, harten=0.05), 0.8, 9.0, 30, 800),   # Fig. 6(b)
    "roe_harten_0.2": (dict(scheme=1, harten=0.2), 0.3, 9.0, 0, 800),      # Fig. 6(c)
    "roeam_roe_xi_and_dup": (dict(xi_roe=1, dup_mode=2), 0.8, 9.0, 50, 800),  # Fig. 6(d)
    "roeam_pressure_positivity": (dict(xi_roe=1), 0.0, 0.8, 0, 8),          # Fig. 6(e)
    "roeam_velocity_positivity": (dict(dup_mode=2), 0.5, 9.0, 20, 800),     # Fig. 6(f)
    "roeam_eps1_0": (dict(), 0.0, 0.3, 0, 2),                               # Fig. 6(g)
    "roeam_eps1_1": (dict(eps1=1), 0.0, 0.05, 0, 1),                        # Fig. 6(i)
}


@pytest.mark.parametrize("name", list(QUIRK_VARIANTS))
def test_quirk_odd_even_fig6(name):
    """Section 7.2 / Fig. 6 at the paper's eps_y = 0.1 (800 x 20, FP32, CFL 0.25, t ~ 100):
    classical Roe destroys the Mach-6 shock, the entropy fix helps little, Roe-AM with the Roe
    xi and delta U_p behaves like Roe, the pressure-positivity delta U_p of Eq. 89 helps more
    than the velocity-positivity xi of Eq. 86, Roe-AM leaves a small oscillation that eps1 = 1
    removes. Indicator: max over columns of (max - min rho) / shock jump; front spread: range of
    the per-row shock position in cells."""
    variant, ind_lo, ind_hi, spread_lo, spread_hi = QUIRK_VARIANTS[name]
    spec, U = W.quirk(800, 20, eps_y=0.1)
    spec = W.with_params(spec, **variant)
    t = 0.0
    with P().Batch([spec], precision=32) as b:
        b.set_state(U, 0)
        while t < 100.0:
            dts = b.step(0.25, nsteps=50, want_dt=True)
            t += 50 * dts[0]   # dt changes slowly; t is approximate
        Ug = b.get_state(0)
    rho = Ug[0]
    ind = float(np.max(rho.max(axis=0) - rho.min(axis=0)) / (W.QUIRK_POST[0] - W.QUIRK_PRE[0]))
    mid = 0.5 * (W.QUIRK_POST[0] + W.QUIRK_PRE[0])
    front = [int(np.argmax(rho[j] < mid)) for j in range(rho.shape[0])]
    spread = max(front) - min(front)
    assert ind_lo <= ind <= ind_hi and spread_lo <= spread <= spread_hi, (ind, spread)


def checker_amplitude(U, n):
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    sign = np.where((ii + jj) % 2 == 0, 1.0, -1.0)
    _, _, _, p = W.cons_to_prim(U)
    return abs(np.mean((p - p.mean()) * sign))


def run_to_time(spec, U, tend, prec=32, cfl=0.5):
    """Steps to about tend (chunks sized from the current dt)."""
    with P().Batch([spec], precision=prec) as b:
        b.set_state(U, 0)
        t = 0.0
        while t < tend:
            dt = b.step(cfl, nsteps=1, want_dt=True)[0]
            t += dt
            k = int((tend - t) / dt * 0.9)
            if k > 1:
                t += k * b.step(cfl, nsteps=k, want_dt=True)[0]
        return b.get_state(0)


def test_checkerboard_delta_up_variants():
    """Section 7.6 / Fig. 11(b)-(d) on the Gresho vortex (64 x 64, first order, M = 0.01,
    seeded pressure checkerboard of 5% of the dynamic pressure, FP32): with delta U_p = 0 the
    checkerboard survives, the Roe delta U_p damps it weakly, the Roe-AM delta U_p of Eq. 89
    removes it."""
    amp = {}
    for dup in (0, 1, 2):
        spec, U = W.gresho(64, mach=0.01, checker=0.05, recon=0)
        spec = W.with_params(spec, dup_mode=dup)
        a0 = checker_amplitude(U, 64)
        amp[dup] = checker_amplitude(run_to_time(spec, U, 0.01), 64) / a0
    assert amp[1] > 0.4, amp
    assert 0.05 < amp[2] < 0.9 * amp[1], amp
    assert amp[0] < 0.01 * amp[2], amp


def kinetic_energy(U):
    return float(np.sum((U[1] ** 2 + U[2] ** 2) / U[0]))


def test_low_mach_dissipation_roe_vs_roeam():
    """Section 3 / Section 7.6 (the non-physical, Stokes-like solution of Roe at low Mach): on the
    Gresho vortex (64 x 64, first order, FP32) over a fixed time t = 0.05, Roe-AM keeps the
    same fraction of kinetic energy at M = 0.1 and M = 0.01 (its dissipation scales with the
    flow speed; measured loss ~5% at both), while classical Roe loses far more, and more as M
    falls (its dissipation scales with c; measured ~16% at M = 0.1, ~47% at M = 0.01).
    Pressure stays O(M^2): Ind(p) falls with slope >= 1.8 in log M for Roe-AM."""
    keep, ind = {}, {}
    for scheme in (0, 1):
        for M in (0.1, 0.01):
            spec, U = W.gresho(64, mach=M, checker=0, recon=0)
            spec = W.with_params(spec, scheme=scheme)
            Ug = run_to_time(spec, U, 0.05)
            keep[scheme, M] = kinetic_energy(Ug) / kinetic_energy(U)
            _, _, _, p = W.cons_to_prim(Ug)
            ind[scheme, M] = (p.max() - p.min()) / p.max()
    loss = {k: 1.0 - v for k, v in keep.items()}
    assert keep[0, 0.01] > 0.6 and abs(keep[0, 0.01] - keep[0, 0.1]) < 0.02, keep
    assert loss[1, 0.01] > 5 * loss[0, 0.01] and loss[1, 0.01] > 2 * loss[1, 0.1], keep
    assert math.log10(ind[0, 0.1] / ind[0, 0.01]) >= 1.8, (ind, keep)


def run_shock_case(spec, U, tend, prec=32, cfl=0.4, ramp=100):
    """Steps to tend (CFL ramped from 0.02 over the first `ramp` steps, then chunks of at most
    200 steps sized from the current dt; t is approximate to within one chunk's dt drift)."""
    with P().Batch([spec], precision=prec) as b:
        b.set_state(U, 0)
        t, n = 0.0, 0
        while t < tend:
            c = min(cfl, 0.02 * 1.05 ** n) if n < ramp else cfl
            dt = b.step(c, nsteps=1, want_dt=True)[0]
            t += dt
            n += 1
            if n >= ramp:
                k = min(int((tend - t) / dt * 0.95), 200)
                if k > 1:
                    t += k * b.step(c, nsteps=k, want_dt=True)[0]
                    n += k
        return b.get_state(0)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("case", ["corner", "dmr"])
def test_shock_case_parity(case, prec):
    """Full-grid one-step parity on the Section 7.3 corner (solid block, inflow, wall, outflow)
    and the Section 7.4 wedge (curvilinear, walls) once the shocks have formed."""
    spec, U = W.supersonic_corner(400) if case == "corner" else W.wedge_dmr(800, 200)
    with P().Batch([spec], precision=prec) as b:
        b.set_state(U, 0)
        for n in range(60):
            b.step(min(0.4, 0.02 * 1.05 ** n), nsteps=1)
        U0 = b.get_state(0)
        dt = b.step(0.4, nsteps=1, want_dt=True)[0]
        U1 = b.get_state(0)
    Uo, _ = oracle.OracleGrid(spec).step(U0, dt_fixed=dt)
    fluid = np.ones(U0.shape[1:], bool) if spec.solid is None else spec.solid == 0
    err = np.max(np.abs(U1 - Uo)[:, fluid].max(axis=1) / state_scale(Uo))
    assert err <= (1e-12 if prec == 64 else 1e-5), err


@pytest.mark.parametrize("variant,fails", [(dict(), False), (dict(eps1=1), False), (dict(scheme=1), True),
                                           (dict(scheme=1, harten=0.2), True), (dict(xi_roe=1), True)])
def test_supersonic_corner(variant, fails):
    """Section 7.3 / Fig. 8: the Mach-5.09 shock diffracting over the 90-degree corner (400 x 400,
    first order, FP32, t = 0.155). Roe-AM reaches the end with a positive state and the planar
    part of the shock where a Mach-5.09 shock should be (x = 0.05 + 5.09 t); classical Roe, with
    or without the entropy fix, and Roe-AM with xi = |U| (no velocity-positivity xi of Eq. 86) stop
    on a non-positive state in the near-vacuum expansion at the corner."""
    spec, U = W.supersonic_corner(400)
    spec = W.with_params(spec, **variant)
    if fails:
        with pytest.raises(P().RoeamError) as e:
            run_shock_case(spec, U, 0.155)
        assert e.value.status in (4, 5)
        return
    rho = run_shock_case(spec, U, 0.155)[0]
    fronts = [int(np.where(rho[j] > 2.0)[0].max()) for j in range(330, 400, 10)]
    x_front = (np.mean(fronts) + 0.5) / 400
    assert abs(x_front - (0.05 + 5.09 * 0.155)) < 0.02, fronts
    assert max(fronts) - min(fronts) <= 2, fronts   # the planar part stays planar


def test_double_mach_reflection_kinked_stem():
    """Section 7.4 / Fig. 9: the Mach-10 shock reflected from the 30-degree wedge (800 x 200,
    first order, FP32, t = 0.2). Classical Roe grows the kinked Mach stem: its foot runs ahead
    along the wall (~37 cells) and the stem leans forward (41 cells over its lowest 20 rows, vs 19
    for Roe-AM, close to a stem normal to the ramp); Roe-AM, with eps1 = 0 or 1, does not."""
    def stem(variant):
        spec, U = W.wedge_dmr(800, 200)
        rho = run_shock_case(W.with_params(spec, **variant), U, 0.2)[0]
        f = [int(np.where(rho[j] > 2.1)[0].max()) for j in (0, 20)]
        return f[0], f[0] - f[1]
    foot_roe, lean_roe = stem(dict(scheme=1))
    for v in (dict(), dict(eps1=1)):
        foot, lean = stem(v)
        assert lean <= 25 and foot_roe - foot >= 20 and lean_roe >= 32, (foot, lean, foot_roe, lean_roe)


def test_quirk_rotated_mach_number():
    """Section 7.2's printed number: with eps1 = 1, eps2 = 0.05 at eps_y = 0.1 and t ~ 100 the
    rotated Mach number f_rr / c on the faces parallel to x reaches about 1.73 on the perturbed
    centreline and near the shock and stays near zero in smooth flow. The time scheme and the
    paper's domain differ (RK4, unstated), so the range checked is loose: the maximum lies in
    1.5-2 (measured: 1.733, near the shock) and the median face is below 0.05. f_rr (Eqs.
    103-109) is evaluated here from the GPU state with the Roe averages, on the y-faces, with
    the normal of the unperturbed grid."""
    spec, U = W.quirk(800, 20, eps_y=0.1, eps1=1)
    t = 0.0
    with P().Batch([spec], precision=32) as b:
        b.set_state(U, 0)
        while t < 100.0:
            t += 50 * b.step(0.25, nsteps=50, want_dt=True)[0]
        Ug = b.get_state(0)
    rho, u, v, p = W.cons_to_prim(Ug)
    H = 3.5 * p / rho + 0.5 * (u * u + v * v)
    L, R = slice(0, -1), slice(1, None)           # y-faces between rows j and j+1
    sl, sr = np.sqrt(rho[L]), np.sqrt(rho[R])
    w = 1.0 / (sl + sr)
    uh = (sl * u[L] + sr * u[R]) * w
    vh = (sl * v[L] + sr * v[R]) * w
    Hh = (sl * H[L] + sr * H[R]) * w
    ch = np.sqrt(0.4 * (Hh - 0.5 * (uh * uh + vh * vh)))
    du, dv = u[R] - u[L], v[R] - v[L]
    dq = np.hypot(du, dv)
    big = dq >= 1e-5 * spec.params.u_ref
    n1x = np.where(big, du / np.where(big, dq, 1), 0.0)   # face normal n = (0, 1)
    n1y = np.where(big, dv / np.where(big, dq, 1), 1.0)
    U1 = n1x * uh + n1y * vh
    frr = np.abs(n1y * U1) + np.abs(vh - n1y * U1)        # |a1 U1| + |U - a1 U1| (Eq. 103)
    ratio = frr / ch
    assert 1.5 <= ratio.max() <= 2.0, ratio.max()
    assert np.median(ratio) < 0.05, np.median(ratio)
