"""Pins of the oracle's face flux against what the paper and the mathematics fix.

None of these retypes the oracle's formulas: each checks an identity, a limit, an
invariance or a textbook reduction that a dropped term, a wrong sign, a swapped
index or a missing factor would break.
"""
import math

import numpy as np
import pytest

import oracle
from workloads import SplitMix64

G = 1.4


def euler_flux(W, n, g=G):
    """Physical normal flux of the 2D Euler equations, Eqs. 3-4 (energy slot rho H U)."""
    W = np.atleast_2d(W)
    n = np.atleast_2d(n)
    r, u, v, p = W.T
    U = n[:, 0] * u + n[:, 1] * v
    H = g / (g - 1) * p / r + 0.5 * (u * u + v * v)
    return np.stack([r * U, r * u * U + p * n[:, 0], r * v * U + p * n[:, 1], r * H * U], axis=1)


def random_states(n, seed, mach=2.0, jump=1.0):
    rng = SplitMix64(seed)
    a = rng.uniforms(4 * n).reshape(n, 4)
    rho = np.exp(jump * (2 * a[:, 0] - 1))
    p = np.exp(jump * (2 * a[:, 3] - 1))
    c = np.sqrt(G * p / rho)
    u = mach * c * (2 * a[:, 1] - 1)
    v = mach * c * (2 * a[:, 2] - 1)
    return np.stack([rho, u, v, p], axis=1)


def random_normals(n, seed):
    rng = SplitMix64(seed)
    t = 2 * math.pi * rng.uniforms(n)
    return np.stack([np.cos(t), np.sin(t)], axis=1)


VARIANTS = [dict(), dict(eps1=1), dict(xi_form=1), dict(m_ref=1e-3), dict(m_ref=2.0), dict(scheme=1),
            dict(dup_mode=1), dict(dup_mode=2), dict(ufix=0), dict(xi_roe=1), dict(scheme=1, harten=0.2)]


# ----------------------------------------------------------------------------- Eq. 98
def test_f_closed_form_pins():
    # f(phi) = 1 exactly for phi >= 1: (1+phi^2)^2 - phi^2 (4 + (1-phi^2)^2) = -(phi^2-1)^3 <= 0.
    # (the FP64 evaluation just above phi = 1 may round to within a few ulp below 1)
    for phi in [1.0, 1.0000001, 1.5, 2.0, 7.0, 1e3]:
        assert abs(oracle.f(phi) - 1.0) <= 4 * np.finfo(float).eps
    assert oracle.f(0.0) == 0.0
    # small-phi asymptote f ~ sqrt(5) phi (from sqrt(4 + 1) at phi -> 0)
    for phi in [1e-4, 1e-6]:
        assert abs(oracle.f(phi) / (math.sqrt(5) * phi) - 1) < 1e-6
    # hand value: f(1/2) = (1/2) sqrt(4 + 9/16) / (5/4) = (2/5) sqrt(73/16) = sqrt(73)/10
    assert abs(oracle.f(0.5) - math.sqrt(73) / 10) < 1e-15
    # monotone on [0, 1]
    xs = np.linspace(0, 1, 201)
    fs = [oracle.f(x) for x in xs]
    assert all(b >= a for a, b in zip(fs, fs[1:]))


# ----------------------------------------------------------------------------- P1 consistency
@pytest.mark.parametrize("variant", VARIANTS)
def test_consistency(variant):
    """F(W, W, n) = physical flux: every difference term vanishes (Eq. 2 with Delta = 0)."""
    W = random_states(400, 11, mach=3.0)
    n = random_normals(400, 12)
    s1 = SplitMix64(13).uniforms(400)
    F = oracle.face_flux(W, W, n, s1, **variant)
    E = euler_flux(W, n)
    scale = np.abs(E).max(axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(F - E) / scale) < 1e-14


# ----------------------------------------------------------------------------- P2 full upwind
def supersonic_pairs(n, seed, sign=+1):
    rng = SplitMix64(seed)
    L, R, N = [], [], []
    while len(L) < n:
        a = rng.uniforms(10)
        t = 2 * math.pi * a[0]
        nx, ny = math.cos(t), math.sin(t)
        out = []
        for k in range(2):
            rho = math.exp(2 * a[1 + 4 * k] - 1)
            p = math.exp(2 * a[2 + 4 * k] - 1)
            c = math.sqrt(G * p / rho)
            Un = sign * c * (1.3 + 2.0 * a[3 + 4 * k])
            Ut = c * (2 * a[4 + 4 * k] - 1)
            out.append([rho, Un * nx - Ut * ny, Un * ny + Ut * nx, p])
        h = oracle.roe_average(out[0], out[1])[0]
        Uh = h[1] * nx + h[2] * ny
        if sign * Uh > h[4] * 1.05:
            L.append(out[0]); R.append(out[1]); N.append([nx, ny])
    return np.array(L), np.array(R), np.array(N)


@pytest.mark.parametrize("eps1", [0, 1])
def test_supersonic_full_upwind(eps1):
    """Eq. 44: for U >= c the flux must equal the upwind physical flux F_L (F_R for U <= -c)."""
    for sign in (+1, -1):
        L, R, n = supersonic_pairs(300, 21 + sign, sign)
        F = oracle.face_flux(L, R, n, SplitMix64(5).uniforms(len(L)), eps1=eps1)
        E = euler_flux(L if sign > 0 else R, n)
        scale = np.abs(E).max(axis=1, keepdims=True)
        assert np.max(np.abs(F - E) / scale) < 1e-13


def test_literal_eq86_breaks_full_upwind():
    """The literal Eq. 86 (no [1 - f^8(Mbar)] factor on dU/2) leaves an O(dU) rho_R term in
    the supersonic mass flux, contradicting Eq. 44; this is why xi_form = 0 is the reading."""
    L, R, n = supersonic_pairs(100, 31)
    F = oracle.face_flux(L, R, n, xi_form=1)
    E = euler_flux(L, n)
    dU = (R[:, 1] - L[:, 1]) * n[:, 0] + (R[:, 2] - L[:, 2]) * n[:, 1]
    # mass flux error is exactly -dU/4 (rho_R - rho_L) in exact arithmetic
    pred = -0.25 * dU * (R[:, 0] - L[:, 0])
    assert np.allclose(F[:, 0] - E[:, 0], pred, rtol=1e-9, atol=1e-12)


# ----------------------------------------------------------------------------- P3, invariances
@pytest.mark.parametrize("variant", VARIANTS)
def test_antisymmetry(variant):
    """Conservation of the face flux: F(W_L, W_R, n) = -F(W_R, W_L, -n)."""
    L = random_states(500, 41)
    R = random_states(500, 42)
    n = random_normals(500, 43)
    s1 = SplitMix64(44).uniforms(500)
    F1 = oracle.face_flux(L, R, n, s1, **variant)
    F2 = oracle.face_flux(R, L, -n, s1, **variant)
    scale = np.abs(F1).max(axis=1, keepdims=True) + np.abs(euler_flux(L, n)).max(axis=1, keepdims=True)
    assert np.max(np.abs(F1 + F2) / scale) < 1e-13


@pytest.mark.parametrize("variant", VARIANTS)
def test_rotation_invariance(variant):
    """Rotating both velocities and the normal rotates the momentum flux and leaves the
    mass and energy fluxes unchanged (catches x/y or u/v mix-ups)."""
    L = random_states(300, 51)
    R = random_states(300, 52)
    n = random_normals(300, 53)
    s1 = SplitMix64(54).uniforms(300)
    t = 0.7371
    c, s = math.cos(t), math.sin(t)

    def rot(W):
        W = W.copy()
        u, v = W[:, 1].copy(), W[:, 2].copy()
        W[:, 1] = c * u - s * v
        W[:, 2] = s * u + c * v
        return W

    nr = np.stack([c * n[:, 0] - s * n[:, 1], s * n[:, 0] + c * n[:, 1]], axis=1)
    F = oracle.face_flux(L, R, n, s1, **variant)
    Fr = oracle.face_flux(rot(L), rot(R), nr, s1, **variant)
    expect = F.copy()
    expect[:, 1] = c * F[:, 1] - s * F[:, 2]
    expect[:, 2] = s * F[:, 1] + c * F[:, 2]
    scale = np.abs(euler_flux(L, n)).max(axis=1, keepdims=True) + np.abs(F).max(axis=1, keepdims=True)
    assert np.max(np.abs(Fr - expect) / scale) < 1e-12


@pytest.mark.parametrize("variant", [dict(), dict(eps1=1), dict(m_ref=1e-2)])
def test_dimensional_scaling(variant):
    """Units: rho, p -> a rho, a p scales every flux by a; u -> b u, p -> b^2 p (c -> b c,
    u_ref -> b u_ref) scales mass, momentum, energy fluxes by b, b^2, b^3."""
    L = random_states(300, 61)
    R = random_states(300, 62)
    n = random_normals(300, 63)
    s1 = SplitMix64(64).uniforms(300)
    F = oracle.face_flux(L, R, n, s1, **variant)
    a = 3.7
    La, Ra = L.copy(), R.copy()
    for W in (La, Ra):
        W[:, 0] *= a
        W[:, 3] *= a
    Fa = oracle.face_flux(La, Ra, n, s1, **variant)
    scale = np.abs(euler_flux(L, n)).max(axis=1, keepdims=True) + np.abs(F).max(axis=1, keepdims=True)
    assert np.max(np.abs(Fa - a * F) / (a * scale)) < 1e-12
    b = 0.29
    Lb, Rb = L.copy(), R.copy()
    for W in (Lb, Rb):
        W[:, 1] *= b
        W[:, 2] *= b
        W[:, 3] *= b * b
    vb = dict(variant)
    vb["u_ref"] = b * 1.0
    Fb = oracle.face_flux(Lb, Rb, n, s1, **vb)
    for k, pw in enumerate([1, 2, 2, 3]):
        assert np.max(np.abs(Fb[:, k] - b ** pw * F[:, k]) / (b ** pw * scale[:, 0])) < 1e-12


# ----------------------------------------------------------------------------- P4 Roe
def jacobian_cs(Wh, n, g=G):
    """Jacobian d(F.n)/dQ of the physical flux at the state Wh by complex-step differentiation."""
    rho, u, v, H = Wh
    p = (g - 1) / g * rho * (H - 0.5 * (u * u + v * v))
    Q = np.array([rho, rho * u, rho * v, p / (g - 1) + 0.5 * rho * (u * u + v * v)], dtype=complex)

    def flux_q(Q):
        r = Q[0]
        uu = Q[1] / r
        vv = Q[2] / r
        pp = (g - 1) * (Q[3] - 0.5 * r * (uu * uu + vv * vv))
        Un = n[0] * uu + n[1] * vv
        return np.array([r * Un, Q[1] * Un + pp * n[0], Q[2] * Un + pp * n[1], (Q[3] + pp) * Un])

    J = np.empty((4, 4))
    h = 1e-30
    for k in range(4):
        Qk = Q.copy()
        Qk[k] += 1j * h
        J[:, k] = flux_q(Qk).imag / h
    return J


def cons(W, g=G):
    r, u, v, p = W
    return np.array([r, r * u, r * v, p / (g - 1) + 0.5 * r * (u * u + v * v)])


def test_roe_average_property():
    """Roe's defining property: A(w_hat)(Q_R - Q_L) = F(Q_R) - F(Q_L) for the averaged state."""
    L = random_states(60, 71)
    R = random_states(60, 72)
    n = random_normals(60, 73)
    h = oracle.roe_average(L, R)
    for k in range(60):
        A = jacobian_cs(h[k, :4], n[k])
        lhs = A @ (cons(R[k]) - cons(L[k]))
        rhs = euler_flux(R[k], n[k])[0] - euler_flux(L[k], n[k])[0]
        assert np.max(np.abs(lhs - rhs)) <= 1e-11 * np.max(np.abs(rhs))
        assert abs(h[k, 4] ** 2 - np.sort(np.abs(np.linalg.eigvals(A)))[-1] ** 2) >= 0  # sanity


def test_classical_roe_matrix_form():
    """The scale form (Eq. 7 with Eqs. 13-17) equals the matrix form of Eq. 5:
    F = (F_L + F_R)/2 - (1/2) R |Lambda| R^-1 dQ, with R, Lambda from numpy's eig."""
    L = random_states(80, 81)
    R = random_states(80, 82)
    n = random_normals(80, 83)
    F = oracle.face_flux(L, R, n, scheme=1)
    h = oracle.roe_average(L, R)
    for k in range(80):
        A = jacobian_cs(h[k, :4], n[k])
        lam, Rv = np.linalg.eig(A)
        absA = (Rv @ np.diag(np.abs(lam)) @ np.linalg.inv(Rv)).real
        ref = 0.5 * (euler_flux(L[k], n[k])[0] + euler_flux(R[k], n[k])[0]) - 0.5 * absA @ (cons(R[k]) - cons(L[k]))
        assert np.max(np.abs(F[k] - ref)) <= 1e-10 * np.max(np.abs(ref)), k


def test_harten_fix_matrix_form():
    """The entropy fix of Eqs. 114-115 in the scale form equals the matrix form with every
    eigenvalue magnitude below h = eps_lambda max|lambda| replaced by (lambda^2/h + h)/2, and
    vanishes as eps_lambda -> 0."""
    L = random_states(60, 181, mach=0.8)
    R = random_states(60, 182, mach=0.8)
    n = random_normals(60, 183)
    for eps in (0.05, 0.2, 0.6):
        F = oracle.face_flux(L, R, n, scheme=1, harten=eps)
        h = oracle.roe_average(L, R)
        for k in range(60):
            A = jacobian_cs(h[k, :4], n[k])
            lam, Rv = np.linalg.eig(A)
            a = np.abs(lam.real)
            hh = eps * a.max()
            a = np.where(a < hh, 0.5 * (a * a / hh + hh), a)
            absA = (Rv @ np.diag(a) @ np.linalg.inv(Rv)).real
            ref = 0.5 * (euler_flux(L[k], n[k])[0] + euler_flux(R[k], n[k])[0]) - 0.5 * absA @ (cons(R[k]) - cons(L[k]))
            assert np.max(np.abs(F[k] - ref)) <= 1e-10 * np.max(np.abs(ref)), (eps, k)
    F0 = oracle.face_flux(L, R, n, scheme=1)
    Ft = oracle.face_flux(L, R, n, scheme=1, harten=1e-300)
    assert np.array_equal(F0, Ft)


# ----------------------------------------------------------------------------- P5 positivity
def test_mass_flux_positivity_limit():
    """Eqs. 65-66: with U_hat = 0, M > 1 (delta U_p off) the Roe-AM mass flux is
    U_bar rho_L for U_bar > 0 and U_bar rho_R for U_bar < 0 (U_bar = (U_L + U_R)/2)."""
    # rho_L = 4, rho_R = 1 with U_L = -a, U_R = 2a gives a Roe-averaged normal velocity of 0.
    for a in (0.3, 1.0, 2.5):
        for sgn in (+1, -1):
            rl, rr = (4.0, 1.0) if sgn > 0 else (1.0, 4.0)
            ul, ur = (-a, 2 * a) if sgn > 0 else (-2 * a, a)
            # a large tangential speed makes the mean Mach number of Eq. 93 exceed 1
            L = np.array([[rl, ul, 5.0, 1.0]])
            R = np.array([[rr, ur, 5.0, 1.0]])
            h = oracle.roe_average(L, R)[0]
            assert abs(h[1]) < 1e-15
            F = oracle.face_flux(L, R, np.array([[1.0, 0.0]]))[0]
            ubar = 0.5 * (ul + ur)
            expect = ubar * (rl if ubar > 0 else rr)
            assert abs(F[0] - expect) < 1e-14 * max(1.0, abs(expect)), (a, sgn, F[0], expect)


# ----------------------------------------------------------------------------- low-Mach asymptotics
def test_low_mach_pressure_dissipation_scales_with_M():
    """Section 3.1 rule 1 (Eq. 22): the velocity-jump-driven pressure dissipation is
    O(rho u du) for Roe-AM, i.e. a factor f(M) ~ sqrt(5) M below classical Roe's O(rho c du)."""
    out = {}
    for scheme in (0, 1):
        vals = []
        for M in (1e-2, 1e-3):
            c = math.sqrt(G)
            L = np.array([[1.0, -0.5 * M * c, 0.3 * M * c, 1.0]])
            R = np.array([[1.0, 0.5 * M * c, 0.3 * M * c, 1.0]])
            F = oracle.face_flux(L, R, np.array([[1.0, 0.0]]), scheme=scheme, m_ref=M)[0]
            central = 0.5 * (euler_flux(L, [1.0, 0.0]) + euler_flux(R, [1.0, 0.0]))[0]
            vals.append(abs(F[1] - central[1]))
        out[scheme] = math.log10(vals[0] / vals[1])
    # du ~ M here, so Roe-AM's f(M) max(0, c - |U|') rho du ~ M^2 and classical Roe's ~ M.
    assert 1.9 < out[0] < 2.1, out
    assert 0.9 < out[1] < 1.1, out


def test_low_mach_pressure_driven_mass_flux():
    """Eq. 57: at U = 0, M -> 0 and theta = M_ref^2, the pressure-driven mass flux is
    -dp / (2 u_ref) with u_ref = c M_ref (the preconditioned delta U_p of Eqs. 89, 99-101)."""
    for mref in (1e-2, 1e-3):
        dp = 1e-9
        L = np.array([[1.0, 0.0, 0.0, 1.0 / G]])
        R = np.array([[1.0, 0.0, 0.0, 1.0 / G + dp]])
        F = oracle.face_flux(L, R, np.array([[1.0, 0.0]]), m_ref=mref)[0]
        c = 1.0
        assert abs(F[0] / (-dp / (2 * c * mref)) - 1) < 1e-6


# ----------------------------------------------------------------------------- P14 rounding
def test_double_within_long_double():
    """The FP64 oracle agrees with its long-double build on random faces from Mach 1e-3 to 20."""
    for mach, seed in ((1e-3, 91), (0.5, 92), (3.0, 93), (20.0, 94)):
        L = random_states(500, seed, mach=mach)
        R = random_states(500, seed + 100, mach=mach)
        n = random_normals(500, seed + 200)
        s1 = SplitMix64(seed + 300).uniforms(500)
        for variant in (dict(), dict(eps1=1), dict(m_ref=mach)):
            Fd = oracle.face_flux(L, R, n, s1, **variant)
            Fl = oracle.face_flux(L, R, n, s1, long_double=True, **variant)
            scale = np.abs(euler_flux(L, n)).max(axis=1) + np.abs(euler_flux(R, n)).max(axis=1)
            err = np.max(np.abs(Fd - Fl).max(axis=1) / scale)
            assert err < 1e-11 * max(1.0, mach * mach), (mach, variant, err)
