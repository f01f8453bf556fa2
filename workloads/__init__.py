"""Seeded synthetic workloads for the Roe-AM solver.

This module produces grids and initial states only. It holds none of the
scheme's arithmetic (no flux, no reconstruction, no time stepping), so both the
CPU oracle and the CUDA path can take their inputs from it without sharing any
of the method's code.

Every random draw comes from splitmix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), with uniform = (x >> 11) * 2**-53.

Conserved state layout everywhere: float64 array of shape (4, nj, ni), i fastest,
variables (rho, rho*u, rho*v, rho*E) — the 2D form of the conservative vector
Q of Eq. 1 (the w component dropped).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Tuple

import numpy as np

# Boundary-condition codes, shared by the oracle binding and the library binding.
PERIODIC, WALL, INFLOW, OUTFLOW = 0, 1, 2, 3
# Reconstruction codes.
RECON_FIRST, RECON_MINMOD, RECON_VANLEER = 0, 1, 2

GAMMA = 1.4
DEFAULT_SEED = 20171127


@dataclass
class SchemeParams:
    """Tunables of the Roe-AM scheme (Section 6.2, Eqs. 110-112) plus solver choices.

    m_ref: global reference Mach number of Eq. 101; u_ref: reference speed of Eq. 108.
    eps1: 0 or 1 (Eq. 111); eps2: entropy-fix constant (Eq. 112); use_s1: 1 evaluates
    the pressure-density detector of Eq. 95, 0 sets s1 = 1 (Eq. 110).
    recon: 0 first order, 1 MUSCL minmod, 2 MUSCL van Leer (primitive variables).
    xi_form: 0 keeps the [1 - f^8(Mbar)] factor of Eq. 68 on dU/2 in xi, 1 is Eq. 86 literally.

    Ablation variants of Section 7 (all defaults give Roe-AM as defined in Section 6.2):
    scheme: 0 Roe-AM, 1 classical Roe (Eq. 7 with Eqs. 8-12); harten: its entropy-fix
    constant eps_lambda of Eqs. 114-115 (0 = none); dup_mode: delta U_p of Roe-AM by Eq. 89 (0),
    zero (1), or the Roe form of Eq. 17 (2); ufix: 1 applies Eq. 92, 0 keeps |U|; xi_roe: 1
    takes xi = |U| (Eq. 13) in Roe-AM.
    """
    gamma: float = GAMMA
    m_ref: float = 0.5
    u_ref: float = 1.0
    eps2: float = 0.05
    eps1: int = 0
    use_s1: int = 1
    recon: int = RECON_FIRST
    xi_form: int = 0
    scheme: int = 0
    dup_mode: int = 0
    ufix: int = 1
    xi_roe: int = 0
    harten: float = 0.0


@dataclass
class GridSpec:
    """One structured 2D grid: ni x nj cells, boundary types (W, E, S, N).

    Cartesian when xv/yv are None (uniform spacing dx, dy). Curvilinear otherwise:
    xv, yv are float64 vertex coordinates of shape (nj+1, ni+1). solid is an
    optional uint8 mask of shape (nj, ni); solid cells are walls and are never updated.
    inflow is the (rho, u, v, p) state imposed on INFLOW sides.
    """
    ni: int
    nj: int
    dx: float = 1.0
    dy: float = 1.0
    bc: Tuple[int, int, int, int] = (PERIODIC, PERIODIC, PERIODIC, PERIODIC)
    inflow: Tuple[float, float, float, float] = (1.0, 0.0, 0.0, 1.0)
    xv: Optional[np.ndarray] = None
    yv: Optional[np.ndarray] = None
    solid: Optional[np.ndarray] = None
    params: SchemeParams = field(default_factory=SchemeParams)

    @property
    def ncells(self) -> int:
        return self.ni * self.nj

    def cell_centres(self) -> Tuple[np.ndarray, np.ndarray]:
        """Cell-centre coordinates (mean of the four vertices), shape (nj, ni)."""
        if self.xv is None:
            x = (np.arange(self.ni) + 0.5) * self.dx
            y = (np.arange(self.nj) + 0.5) * self.dy
            return np.meshgrid(x, y)
        xc = 0.25 * (self.xv[:-1, :-1] + self.xv[:-1, 1:] + self.xv[1:, :-1] + self.xv[1:, 1:])
        yc = 0.25 * (self.yv[:-1, :-1] + self.yv[:-1, 1:] + self.yv[1:, :-1] + self.yv[1:, 1:])
        return xc, yc


# ----------------------------------------------------------------------------- PRNG
class SplitMix64:
    """splitmix64 generator (Steele, Lea & Flood 2014)."""

    MASK = (1 << 64) - 1

    def __init__(self, seed: int = DEFAULT_SEED):
        self.state = seed & self.MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & self.MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniforms(self, n: int) -> np.ndarray:
        """The next n uniforms, vectorised: output m is the mix of state + (m+1) * golden."""
        if n <= 0:
            return np.zeros(0)
        with np.errstate(over="ignore"):
            z = (np.uint64(self.state) + np.arange(1, n + 1, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15))
            self.state = int(z[-1])
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# ----------------------------------------------------------------------------- helpers
def prim_to_cons(rho, u, v, p, gamma=GAMMA) -> np.ndarray:
    """(rho, u, v, p) -> (rho, rho u, rho v, rho E), E = p/((gamma-1) rho) + |q|^2/2."""
    rho = np.asarray(rho, dtype=np.float64)
    u = np.broadcast_to(np.asarray(u, dtype=np.float64), rho.shape)
    v = np.broadcast_to(np.asarray(v, dtype=np.float64), rho.shape)
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), rho.shape)
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def cons_to_prim(U: np.ndarray, gamma=GAMMA):
    rho = U[0]
    u = U[1] / rho
    v = U[2] / rho
    p = (gamma - 1.0) * (U[3] - 0.5 * rho * (u * u + v * v))
    return rho, u, v, p


# ----------------------------------------------------------------------------- workloads
def isentropic_vortex(n: int = 64, t: float = 0.0, beta: float = 5.0, mach: float = 0.5,
                      gamma: float = GAMMA, recon: int = RECON_FIRST) -> Tuple[GridSpec, np.ndarray]:
    """Isentropic vortex of strength beta on [0,10]^2, periodic, free stream at `mach`
    along (1,1)/sqrt(2) with rho_inf = p_inf = 1. With t > 0 returns the exact advected
    solution (point values at cell centres, periodic images of the vortex centre)."""
    L = 10.0
    spec = GridSpec(ni=n, nj=n, dx=L / n, dy=L / n,
                    params=SchemeParams(gamma=gamma, m_ref=mach, u_ref=mach * math.sqrt(gamma), recon=recon))
    x, y = spec.cell_centres()
    cinf = math.sqrt(gamma)
    uinf = mach * cinf / math.sqrt(2.0)
    x0 = (5.0 + uinf * t) % L
    y0 = (5.0 + uinf * t) % L
    dxp = (x - x0 + 0.5 * L) % L - 0.5 * L
    dyp = (y - y0 + 0.5 * L) % L - 0.5 * L
    r2 = dxp * dxp + dyp * dyp
    amp = beta / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    u = uinf - amp * dyp
    v = uinf + amp * dxp
    T = 1.0 - (gamma - 1.0) * beta * beta / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    return spec, prim_to_cons(rho, u, v, p, gamma)


def gresho(n: int = 256, mach: float = 0.01, checker: float = 1e-3, seed: int = DEFAULT_SEED,
           recon: int = RECON_MINMOD, gamma: float = GAMMA) -> Tuple[GridSpec, np.ndarray]:
    """Gresho vortex on [0,1]^2, periodic, rho = 1, peak swirl 1 at r = 0.2, background
    pressure p0 = 1/(gamma M^2). A seeded checkerboard of amplitude `checker` times the
    dynamic pressure, (-1)^(i+j) (0.5 + uniform), is added to p."""
    spec = GridSpec(ni=n, nj=n, dx=1.0 / n, dy=1.0 / n,
                    params=SchemeParams(gamma=gamma, m_ref=mach, u_ref=1.0, recon=recon))
    x, y = spec.cell_centres()
    dx = x - 0.5
    dy = y - 0.5
    r = np.sqrt(dx * dx + dy * dy)
    p0 = 1.0 / (gamma * mach * mach)
    uphi = np.where(r < 0.2, 5.0 * r, np.where(r < 0.4, 2.0 - 5.0 * r, 0.0))
    rs = np.maximum(r, 1e-300)
    p_in = p0 + 12.5 * r * r
    p_mid = p0 + 4.0 - 4.0 * math.log(0.2) + 12.5 * r * r - 20.0 * r + 4.0 * np.log(rs)
    p_out = p0 - 2.0 + 4.0 * math.log(2.0)
    p = np.where(r < 0.2, p_in, np.where(r < 0.4, p_mid, p_out))
    u = -uphi * dy / rs
    v = uphi * dx / rs
    if checker:
        rng = SplitMix64(seed)
        jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        sign = np.where((ii + jj) % 2 == 0, 1.0, -1.0)
        p = p + checker * sign * (0.5 + rng.uniforms(n * n).reshape(n, n))
    rho = np.ones_like(p)
    return spec, prim_to_cons(rho, u, v, p, gamma)


QUIRK_POST = (1512.0 / 205.0, 175.0 / 36.0, 0.0, 251.0 / 6.0)   # (rho, u, v, p) behind the Mach-6 shock
QUIRK_PRE = (1.4, 0.0, 0.0, 1.0)


def quirk(nx: int = 800, ny: int = 20, eps_y: float = 1e-6, x_shock: float = 10.0,
          eps1: int = 0, recon: int = RECON_FIRST) -> Tuple[GridSpec, np.ndarray]:
    """Quirk odd-even decoupling duct (Section 7.2): unit cells, centreline vertex row
    perturbed by +eps_y (even i) / -eps_y (odd i) as in Eq. 113, Mach-6 shock at x_shock.
    W: supersonic inflow of the post-shock state, E: zero-gradient outflow, S/N: walls."""
    X, Y = np.meshgrid(np.arange(nx + 1, dtype=np.float64), np.arange(ny + 1, dtype=np.float64))
    yv = Y.copy()
    jm = ny // 2
    i = np.arange(nx + 1)
    yv[jm, :] += np.where(i % 2 == 0, eps_y, -eps_y)
    spec = GridSpec(ni=nx, nj=ny, dx=1.0, dy=1.0, bc=(INFLOW, OUTFLOW, WALL, WALL), inflow=QUIRK_POST,
                    xv=X, yv=yv,
                    params=SchemeParams(m_ref=6.0, u_ref=QUIRK_POST[1], eps1=eps1, recon=recon))
    xc, _ = spec.cell_centres()
    left = xc < x_shock
    rho = np.where(left, QUIRK_POST[0], QUIRK_PRE[0])
    u = np.where(left, QUIRK_POST[1], QUIRK_PRE[1])
    p = np.where(left, QUIRK_POST[3], QUIRK_PRE[3])
    return spec, prim_to_cons(rho, u, 0.0 * rho, p)


SHOCK_TUBES = {
    # name: (left (rho,u,p), right (rho,u,p), x0, t_end) — Section 7.1
    "expansion": ((3.0, 0.9, 3.0), (1.0, 0.9, 1.0), 0.3, 0.2),
    "near_vacuum": ((1.0, -2.0, 0.4), (1.0, 2.0, 0.4), 0.5, 0.15),
    "strong": ((1.0, 0.0, 1000.0), (1.0, 0.0, 0.01), 0.5, 0.012),
}


def shock_tube(name: str, ni: int = 200, nj: int = 4, recon: int = RECON_FIRST) -> Tuple[GridSpec, np.ndarray]:
    """1D Riemann problem along x on [0,1] (ni x nj cells, y periodic, x zero-gradient)."""
    (rl, ul, pl), (rr, ur, pr), x0, _ = SHOCK_TUBES[name]
    spec = GridSpec(ni=ni, nj=nj, dx=1.0 / ni, dy=1.0 / ni, bc=(OUTFLOW, OUTFLOW, PERIODIC, PERIODIC),
                    params=SchemeParams(m_ref=1.0, u_ref=max(abs(ul), abs(ur), 1.0), recon=recon))
    xc, _ = spec.cell_centres()
    left = xc < x0
    return spec, prim_to_cons(np.where(left, rl, rr), np.where(left, ul, ur), 0.0 * xc, np.where(left, pl, pr))


def free_stream(spec: GridSpec, rho=1.0, u=0.3, v=-0.2, p=1.0) -> np.ndarray:
    z = np.zeros((spec.nj, spec.ni))
    return prim_to_cons(z + rho, z + u, z + v, z + p, spec.params.gamma)


def random_smooth_state(spec: GridSpec, seed: int = DEFAULT_SEED, mach: float = 0.5, amp: float = 0.2,
                        modes: int = 3) -> np.ndarray:
    """A seeded smooth periodic perturbation of a uniform state (rho, p > 0): a sum of
    `modes` random Fourier modes in each primitive variable."""
    rng = SplitMix64(seed)
    g = spec.params.gamma
    x, y = spec.cell_centres()
    Lx = spec.ni * spec.dx
    Ly = spec.nj * spec.dy
    out = []
    base = (1.0, mach * math.sqrt(g), -0.5 * mach * math.sqrt(g), 1.0)
    for k in range(4):
        f = np.full_like(x, base[k])
        for _ in range(modes):
            kx = 1 + int(rng.uniform() * 3)
            ky = 1 + int(rng.uniform() * 3)
            ph = 2 * math.pi * rng.uniform()
            a = amp * (rng.uniform() - 0.5) * (1.0 if k in (0, 3) else mach * math.sqrt(g))
            f = f + a * np.sin(2 * math.pi * (kx * x / Lx + ky * y / Ly) + ph)
        out.append(f)
    return prim_to_cons(*out, gamma=g)


def random_rough_state(spec: GridSpec, seed: int = DEFAULT_SEED, mach: float = 1.0,
                       jump: float = 0.5) -> np.ndarray:
    """Cell-by-cell seeded random state: rho, p log-uniform within a factor exp(+-jump),
    velocity components uniform in +-mach*c. Exercises every branch of the flux."""
    rng = SplitMix64(seed)
    n = spec.ni * spec.nj
    g = spec.params.gamma
    r = rng.uniforms(4 * n).reshape(4, spec.nj, spec.ni)
    rho = np.exp(jump * (2 * r[0] - 1))
    p = np.exp(jump * (2 * r[3] - 1))
    c = np.sqrt(g * p / rho)
    u = mach * c * (2 * r[1] - 1)
    v = mach * c * (2 * r[2] - 1)
    return prim_to_cons(rho, u, v, p, g)


def batch(count: int = 512, seed: int = DEFAULT_SEED, ni_range=(32, 512), nj_range=(32, 256),
          recon: int = RECON_FIRST, gamma: float = GAMMA) -> Tuple[List[GridSpec], List[np.ndarray]]:
    """Batch of independent periodic grids of uneven sizes. Sizes uniform in ni_range x
    nj_range, dx = dy = 1/ni, free stream rho = 1, p = 1/gamma (c = 1) at Mach
    10^U(-3, log10 20) in a uniform random direction, with Gaussian bumps of amplitude 0.1
    (sigma = 0.1, periodic minimum-image distance) on rho and on p at separate centres."""
    rng = SplitMix64(seed)
    specs, states = [], []
    lo, hi = -3.0, math.log10(20.0)
    for _ in range(count):
        ni = ni_range[0] + int(rng.uniform() * (ni_range[1] - ni_range[0] + 1))
        nj = nj_range[0] + int(rng.uniform() * (nj_range[1] - nj_range[0] + 1))
        mach = 10.0 ** (lo + (hi - lo) * rng.uniform())
        ang = 2.0 * math.pi * rng.uniform()
        cx = [rng.uniform(), rng.uniform()]
        cp = [rng.uniform(), rng.uniform()]
        d = 1.0 / ni
        spec = GridSpec(ni=ni, nj=nj, dx=d, dy=d,
                        params=SchemeParams(gamma=gamma, m_ref=max(mach, 1e-3), u_ref=mach, recon=recon))
        x, y = spec.cell_centres()
        Lx, Ly = 1.0, nj * d
        sig = 0.1 * Lx

        def bump(c):
            ddx = (x - c[0] * Lx + 0.5 * Lx) % Lx - 0.5 * Lx
            ddy = (y - c[1] * Ly + 0.5 * Ly) % Ly - 0.5 * Ly
            return 1.0 + 0.1 * np.exp(-(ddx * ddx + ddy * ddy) / (2 * sig * sig))

        rho = bump(cx)
        p = bump(cp) / gamma
        u = np.full_like(x, mach * math.cos(ang))
        v = np.full_like(x, mach * math.sin(ang))
        specs.append(spec)
        states.append(prim_to_cons(rho, u, v, p, gamma))
    return specs, states


def warped_step(n_i: int = 4096, n_j: int = 4096, amp: float = 0.1, recon: int = RECON_VANLEER,
                with_state: bool = True) -> Tuple[GridSpec, Optional[np.ndarray]]:
    """Mach-3 flow over a forward-facing step on [0,3]x[0,1] with n_i x n_j cells on a
    sinusoidally warped grid: x = X + amp*dx*s, y = Y + amp*dy*s, s = sin(16 pi X/3) sin(16 pi Y)
    (s = 0 on the outer boundary). Solid block: cells with centre x >= 0.6 and y < 0.2.
    W: supersonic inflow (rho, u, v, p) = (1.4, 3, 0, 1); E: outflow; S/N and block: walls."""
    dxb, dyb = 3.0 / n_i, 1.0 / n_j
    X, Y = np.meshgrid(np.arange(n_i + 1) * dxb, np.arange(n_j + 1) * dyb)
    s = np.sin(16.0 * math.pi * X / 3.0) * np.sin(16.0 * math.pi * Y)
    xv = X + amp * dxb * s
    yv = Y + amp * dyb * s
    ib = int(math.ceil(0.6 / dxb - 0.5 - 1e-9))
    jb = int(math.ceil(0.2 / dyb - 0.5 - 1e-9))
    solid = np.zeros((n_j, n_i), dtype=np.uint8)
    solid[:jb, ib:] = 1
    spec = GridSpec(ni=n_i, nj=n_j, dx=dxb, dy=dyb, bc=(INFLOW, OUTFLOW, WALL, WALL), inflow=(1.4, 3.0, 0.0, 1.0),
                    xv=xv, yv=yv, solid=solid, params=SchemeParams(m_ref=3.0, u_ref=3.0, recon=recon))
    if not with_state:
        return spec, None
    z = np.zeros((n_j, n_i))
    return spec, prim_to_cons(z + 1.4, z + 3.0, z, z + 1.0)


def warped_periodic(n: int = 32, amp: float = 0.1, seed: int = DEFAULT_SEED) -> GridSpec:
    """Periodic [0,1]^2 grid warped like warped_step (periodic warp, 2 wavelengths)."""
    d = 1.0 / n
    X, Y = np.meshgrid(np.arange(n + 1) * d, np.arange(n + 1) * d)
    s = np.sin(4.0 * math.pi * X) * np.sin(4.0 * math.pi * Y)
    return GridSpec(ni=n, nj=n, dx=d, dy=d, xv=X + amp * d * s, yv=Y + amp * d * s)


def cylinder_ogrid(ni: int = 100, nj: int = 72, mach: float = 0.01, r_far: float = 20.0,
                   recon: int = RECON_FIRST, gamma: float = GAMMA) -> Tuple[GridSpec, np.ndarray]:
    """Low-Mach inviscid flow past a unit cylinder (Section 7.6) on an O-grid of ni cells
    around the circumference and nj cells out to r_far, radii growing geometrically (first
    radial spacing about 2 pi / ni * 0.7). i runs clockwise from the upstream stagnation point
    (theta = pi - 2 pi i / ni; periodic W/E, the seam column repeats column 0 bit for bit), j
    outward: S is the cylinder wall, N the far field (the free stream imposed as INFLOW).
    Free stream rho = 1, p = 1/gamma (c = 1), u = mach along +x. Vertices are absolute
    coordinates (dx = dy = 0). Initial state: incompressible potential flow with Bernoulli
    pressure and isentropic density, evaluated at the cell centres."""
    q = r_far ** (1.0 / nj)
    r = q ** np.arange(nj + 1, dtype=np.float64)
    r[-1] = r_far
    th = np.pi - 2.0 * np.pi * np.arange(ni + 1, dtype=np.float64) / ni
    R, TH = np.meshgrid(r, th, indexing="ij")
    xv = R * np.cos(TH)
    yv = R * np.sin(TH)
    xv[:, ni] = xv[:, 0]
    yv[:, ni] = yv[:, 0]
    p_inf = 1.0 / gamma
    spec = GridSpec(ni=ni, nj=nj, dx=0.0, dy=0.0, bc=(PERIODIC, PERIODIC, WALL, INFLOW),
                    inflow=(1.0, mach, 0.0, p_inf), xv=xv, yv=yv,
                    params=SchemeParams(gamma=gamma, m_ref=mach, u_ref=mach, recon=recon))
    xc, yc = spec.cell_centres()
    rc2 = xc * xc + yc * yc
    c2t = (xc * xc - yc * yc) / rc2          # cos 2 theta
    s2t = 2.0 * xc * yc / rc2                # sin 2 theta
    u = mach * (1.0 - c2t / rc2)
    v = -mach * s2t / rc2
    p = p_inf + 0.5 * (mach * mach - (u * u + v * v))
    rho = (p / p_inf) ** (1.0 / gamma)
    return spec, prim_to_cons(rho, u, v, p, gamma)


def cylinder_blunt(ni: int = 160, nj: int = 20, mach: float = 20.0, recon: int = RECON_FIRST,
                   gamma: float = GAMMA) -> Tuple[GridSpec, np.ndarray]:
    """Hypersonic flow onto the front half of a unit cylinder (Section 7.5, carbuncle test):
    ni cells around the half circle (theta from 3 pi / 2 down to pi / 2, so i runs clockwise
    from the bottom shoulder over the stagnation point to the top), nj equal radial cells out
    to r_out(phi) = 1.6 + 1.4 sin^2 phi (phi = angle from the stagnation line), outside the bow
    shock at Mach 20. S: cylinder wall; N: supersonic free stream (INFLOW); W/E: supersonic
    outflow (zero gradient). Free stream rho = 1, p = 1/gamma, u = mach along +x, imposed in
    every cell at t = 0 (impulsive start)."""
    th = 1.5 * np.pi - np.pi * np.arange(ni + 1, dtype=np.float64) / ni
    phi = th - np.pi
    r_out = 1.6 + 1.4 * np.sin(phi) ** 2
    s = np.arange(nj + 1, dtype=np.float64) / nj
    R = 1.0 + s[:, None] * (r_out[None, :] - 1.0)
    xv = R * np.cos(th)[None, :]
    yv = R * np.sin(th)[None, :]
    p_inf = 1.0 / gamma
    spec = GridSpec(ni=ni, nj=nj, dx=0.0, dy=0.0, bc=(OUTFLOW, OUTFLOW, WALL, INFLOW),
                    inflow=(1.0, mach, 0.0, p_inf), xv=xv, yv=yv,
                    params=SchemeParams(gamma=gamma, m_ref=min(mach, 1.0), u_ref=mach, recon=recon))
    z = np.zeros((nj, ni))
    return spec, prim_to_cons(z + 1.0, z + mach, z, z + p_inf, gamma)


# Mach-5.09 and Mach-10 shocks into rho = 1.4, p = 1 (c = 1): post-shock (rho, u, v, p).
CORNER_POST = (7.04108, 4.07794, 0.0, 30.05942)    # Section 7.3
DMR_POST = (8.0, 8.25, 0.0, 116.5)                  # Mach 10 (Section 7.4)
STILL_AIR = (1.4, 0.0, 0.0, 1.0)


def supersonic_corner(n: int = 400, x_shock: float = 0.05, y_corner: float = 0.5,
                      recon: int = RECON_FIRST) -> Tuple[GridSpec, np.ndarray]:
    """Shock diffraction over a 90-degree corner (Section 7.3): [0,1]^2 with n x n cells, the
    block x < x_shock, y < y_corner solid; a Mach-5.09 shock at x = x_shock above the corner
    with the paper's post-shock state behind it. W: post-shock INFLOW; N: wall; E, S:
    zero-gradient outflow."""
    spec = GridSpec(ni=n, nj=n, dx=1.0 / n, dy=1.0 / n, bc=(INFLOW, OUTFLOW, OUTFLOW, WALL), inflow=CORNER_POST,
                    params=SchemeParams(m_ref=1.0, u_ref=CORNER_POST[1], recon=recon))
    xc, yc = spec.cell_centres()
    spec.solid = ((xc < x_shock) & (yc < y_corner)).astype(np.uint8)
    post = xc < x_shock
    rho = np.where(post, CORNER_POST[0], STILL_AIR[0])
    u = np.where(post, CORNER_POST[1], 0.0)
    p = np.where(post, CORNER_POST[3], STILL_AIR[3])
    return spec, prim_to_cons(rho, u, 0.0 * rho, p)


def wedge_dmr(ni: int = 800, nj: int = 200, x_tip: float = 0.5, ramp: float = 3.0, height: float = 2.8,
              recon: int = RECON_FIRST) -> Tuple[GridSpec, np.ndarray]:
    """Double-Mach reflection (Section 7.4) in the wedge frame: a Mach-10 shock, normal to a flat
    wall, meets a 30-degree ramp at x_tip, so that relative to the ramp it is inclined at 60
    degrees (the usual rotated set-up). Curvilinear ni x nj grid: columns x uniform on
    [0, x_tip + ramp cos 30], rows from the wall (flat, then the ramp) to a flat upper wall at
    `height`. The shock starts 0.05 before the tip. W: post-shock INFLOW; E: outflow; S, N:
    walls."""
    L = x_tip + ramp * math.cos(math.pi / 6)
    x = np.linspace(0.0, L, ni + 1)
    yb = np.where(x > x_tip, (x - x_tip) * math.tan(math.pi / 6), 0.0)
    s = np.arange(nj + 1, dtype=np.float64)[:, None] / nj
    xv = np.broadcast_to(x[None, :], (nj + 1, ni + 1)).copy()
    yv = yb[None, :] + s * (height - yb[None, :])
    spec = GridSpec(ni=ni, nj=nj, dx=L / ni, dy=height / nj, bc=(INFLOW, OUTFLOW, WALL, WALL), inflow=DMR_POST,
                    xv=xv, yv=yv, params=SchemeParams(m_ref=1.0, u_ref=DMR_POST[1], recon=recon))
    xc, _ = spec.cell_centres()
    post = xc < x_tip - 0.05
    rho = np.where(post, DMR_POST[0], STILL_AIR[0])
    u = np.where(post, DMR_POST[1], 0.0)
    p = np.where(post, DMR_POST[3], STILL_AIR[3])
    return spec, prim_to_cons(rho, u, 0.0 * rho, p)


# ----------------------------------------------------------------------------- 3D with scalars
@dataclass
class GridSpec3:
    """One structured 3D Cartesian grid: ni x nj x nk cells of dx x dy x dz, boundary types
    (W, E, S, N, B, T) = (-x, +x, -y, +y, -z, +z), nscal passive scalars. State arrays are
    (5 + nscal, nk, nj, ni): rho, rho u, rho v, rho w, rho E, rho k_1.. . inflow is the
    primitive (rho, u, v, w, p, k_1..) state imposed on INFLOW sides."""
    ni: int
    nj: int
    nk: int
    dx: float = 1.0
    dy: float = 1.0
    dz: float = 1.0
    bc: Tuple[int, ...] = (PERIODIC,) * 6
    inflow: Tuple[float, ...] = (1.0, 0.0, 0.0, 0.0, 1.0)
    nscal: int = 0
    params: SchemeParams = field(default_factory=SchemeParams)

    @property
    def ncells(self) -> int:
        return self.ni * self.nj * self.nk

    def cell_centres(self):
        """(x, y, z) cell centres, each of shape (nk, nj, ni)."""
        z, y, x = np.meshgrid((np.arange(self.nk) + 0.5) * self.dz, (np.arange(self.nj) + 0.5) * self.dy,
                              (np.arange(self.ni) + 0.5) * self.dx, indexing="ij")
        return x, y, z


def prim_to_cons3(rho, u, v, w, p, scalars=(), gamma=GAMMA) -> np.ndarray:
    """(rho, u, v, w, p, k..) -> (rho, rho u, rho v, rho w, rho E, rho k..)."""
    rho = np.asarray(rho, dtype=np.float64)
    b = np.broadcast_to
    u, v, w, p = (b(np.asarray(a, dtype=np.float64), rho.shape) for a in (u, v, w, p))
    E = p / ((gamma - 1.0) * rho) + 0.5 * (u * u + v * v + w * w)
    out = [rho, rho * u, rho * v, rho * w, rho * E] + [rho * b(np.asarray(k, dtype=np.float64), rho.shape)
                                                          for k in scalars]
    return np.stack(out)


def cons_to_prim3(U: np.ndarray, gamma=GAMMA):
    """(rho, u, v, w, p, [k..])."""
    rho = U[0]
    u, v, w = U[1] / rho, U[2] / rho, U[3] / rho
    p = (gamma - 1.0) * (U[4] - 0.5 * rho * (u * u + v * v + w * w))
    return (rho, u, v, w, p) + tuple(U[5 + s] / rho for s in range(U.shape[0] - 5))


def random_rough_state3(spec: GridSpec3, seed: int = DEFAULT_SEED, mach: float = 1.0,
                        jump: float = 0.5) -> np.ndarray:
    """Cell-by-cell seeded random 3D state: rho, p log-uniform within exp(+-jump), velocity
    components uniform in +-mach c, scalars uniform in [0, 1]."""
    rng = SplitMix64(seed)
    shape = (spec.nk, spec.nj, spec.ni)
    g = spec.params.gamma
    r = rng.uniforms((5 + spec.nscal) * spec.ncells).reshape((5 + spec.nscal,) + shape)
    rho = np.exp(jump * (2 * r[0] - 1))
    p = np.exp(jump * (2 * r[4] - 1))
    c = np.sqrt(g * p / rho)
    u, v, w = (mach * c * (2 * r[k] - 1) for k in (1, 2, 3))
    return prim_to_cons3(rho, u, v, w, p, [r[5 + s] for s in range(spec.nscal)], gamma=g)


def random_smooth_state3(spec: GridSpec3, seed: int = DEFAULT_SEED, mach: float = 0.5, amp: float = 0.2,
                         modes: int = 3) -> np.ndarray:
    """A seeded smooth periodic perturbation of a uniform flow: `modes` random Fourier modes in
    each primitive variable; scalars smooth in [0, 1]."""
    rng = SplitMix64(seed)
    g = spec.params.gamma
    x, y, z = spec.cell_centres()
    L = (spec.ni * spec.dx, spec.nj * spec.dy, spec.nk * spec.dz)
    cs = math.sqrt(g)
    base = (1.0, mach * cs, -0.5 * mach * cs, 0.3 * mach * cs, 1.0) + (0.5,) * spec.nscal
    out = []
    for k in range(5 + spec.nscal):
        f = np.full_like(x, base[k])
        for _ in range(modes):
            kk = [1 + int(rng.uniform() * 3) for _ in range(3)]
            ph = 2 * math.pi * rng.uniform()
            a = amp * (rng.uniform() - 0.5) * (mach * cs if k in (1, 2, 3) else 1.0)
            f = f + a * np.sin(2 * math.pi * (kk[0] * x / L[0] + kk[1] * y / L[1] + kk[2] * z / L[2]) + ph)
        out.append(f)
    return prim_to_cons3(*out[:5], out[5:], gamma=g)


def taylor_green3(n: int = 64, mach: float = 0.1, nscal: int = 1, recon: int = RECON_FIRST,
                  gamma: float = GAMMA) -> Tuple[GridSpec3, np.ndarray]:
    """Taylor-Green vortex on the periodic cube [0, 2 pi]^3 (n^3 cells): u = U0 sin x cos y cos z,
    v = -U0 cos x sin y cos z, w = 0, p = p0 + (rho0 U0^2 / 16)(cos 2x + cos 2y)(cos 2z + 2),
    rho0 = 1, U0 = 1, p0 = 1 / (gamma M^2); scalar k_s = (1 + sin(x + s) sin(y) sin(z)) / 2."""
    h = 2 * math.pi / n
    spec = GridSpec3(ni=n, nj=n, nk=n, dx=h, dy=h, dz=h, nscal=nscal,
                     params=SchemeParams(gamma=gamma, m_ref=mach, u_ref=1.0, recon=recon))
    x, y, z = spec.cell_centres()
    p0 = 1.0 / (gamma * mach * mach)
    u = np.sin(x) * np.cos(y) * np.cos(z)
    v = -np.cos(x) * np.sin(y) * np.cos(z)
    p = p0 + (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2) / 16.0
    ks = [0.5 * (1 + np.sin(x + s) * np.sin(y) * np.sin(z)) for s in range(nscal)]
    return spec, prim_to_cons3(np.ones_like(x), u, v, 0.0 * x, p, ks, gamma=gamma)


def shock_tube3(name: str, n: int = 200, axis: int = 0, nt: int = 2, nscal: int = 1) -> Tuple[GridSpec3, np.ndarray]:
    """A Section 7.1 tube along `axis` (0, 1, 2) of a 3D grid with nt cells in the two other
    (periodic) directions, zero-gradient ends; scalar k = 1 on the left, 0 on the right (a
    contact marker)."""
    (rl, ul, pl), (rr, ur, pr), x0, _ = SHOCK_TUBES[name]
    dims = [nt, nt, nt]
    dims[axis] = n
    bc = [PERIODIC] * 6
    bc[2 * axis] = bc[2 * axis + 1] = OUTFLOW
    spec = GridSpec3(ni=dims[0], nj=dims[1], nk=dims[2], dx=1.0 / n, dy=1.0 / n, dz=1.0 / n, bc=tuple(bc),
                     nscal=nscal, params=SchemeParams(m_ref=1.0, u_ref=max(abs(ul), abs(ur), 1.0)))
    c = spec.cell_centres()[axis]
    left = c < x0
    vel = [0.0 * c, 0.0 * c, 0.0 * c]
    vel[axis] = np.where(left, ul, ur)
    return spec, prim_to_cons3(np.where(left, rl, rr), *vel, np.where(left, pl, pr),
                               [np.where(left, 1.0, 0.0)] * nscal)


def with_params(spec: GridSpec, **kw) -> GridSpec:
    return replace(spec, params=replace(spec.params, **kw))
