/*
 * roeam_oracle.c — plain, slow CPU oracle of the Roe-AM finite-volume step.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this code. The product library never calls it and
 * shares no code, header, table or helper with it.
 *
 * Precision: `real` is double by default (FP64 oracle). Built a second time with
 * -DORC_LONG=1 it runs in long double, which the tests use to bound the rounding
 * error of the double build.
 *
 * What it computes (Li, Ren & Gu, "An improved Roe scheme for all Mach-number
 * flows simultaneously curing known problems"):
 *   - the 2D Euler conservative variables and face fluxes of Eqs. 1, 3, 4;
 *   - the Roe-AM dissipation of Section 6.2, Eqs. 85-109, term by term, in the
 *     paper's order; the classical Roe scale form of Eqs. 7, 13-17 as a control;
 *   - a cell-centred finite-volume residual R_i = -(1/V_i) sum_f F_f |S_f| built
 *     by a loop over faces that scatters to the two cells (the CUDA path gathers
 *     per cell instead);
 *   - MUSCL reconstruction on primitive variables (minmod / van Leer), the
 *     pressure-density detector of Eqs. 95-97 on cell-centre values, and the
 *     three-stage SSP Runge-Kutta update of Shu & Osher.
 *
 * Readings where the paper is silent or inconsistent (each is a documented choice):
 *   xi      — Eq. 86 with the [1 - f^8(Mbar)] factor of Eq. 68 on dU/2 (xi_form = 0);
 *             xi_form = 1 evaluates Eq. 86 literally.
 *   |U|'    — Eq. 92 with f(Mbar), clamped at 0.
 *   face U, c, rho in Eqs. 87-94 — Roe averages; sgn(0) = 0.
 *   n2      — Eq. 109 normalised to unit length (0 when n1 is parallel to n).
 *   detector on a 2D grid — the 5-face form of Eq. 96; P = 1 on a face with a
 *             solid side; ghost cells take their boundary-condition values.
 *   walls   — a wall face takes the first-order fluid state and its mirror image
 *             about the face normal; a reconstruction stencil that reaches into a
 *             solid cell uses the mirror of the adjacent fluid cell instead.
 *   MUSCL   — if a reconstructed rho or p is <= 0 on either side, that face falls
 *             back to first order.
 *   dt      — dt = CFL / max_i sum_dir (|U| + max(c, c~/theta))_dir |S_dir| / V_i, with
 *             S_dir the means of opposite face vectors and theta, c~ of Eqs. 99-101 on
 *             the cell state, taken from U^n (the preconditioned delta U_p of Eq. 89
 *             makes the dissipation's fastest speed ~ c / M_ref at low Mach); the
 *             classical Roe scheme takes theta = 1, i.e. |U| + c.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORC_LONG
#define ORC_LONG 0
#endif

#if ORC_LONG
typedef long double real;
#define RSQRT_(x) sqrtl(x)
#define RABS_(x) fabsl(x)
#define ORC_API(name) name##_ld
#else
typedef double real;
#define RSQRT_(x) sqrt(x)
#define RABS_(x) fabs(x)
#define ORC_API(name) name
#endif

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_INFLOW = 2, BC_OUTFLOW = 3 };
enum { SIDE_W = 0, SIDE_E = 1, SIDE_S = 2, SIDE_N = 3 };

typedef struct {
    double gamma, m_ref, u_ref, eps2;
    int eps1;      /* Eq. 111 */
    int use_s1;    /* 1: detector of Eq. 95; 0: s1 = 1 (Eq. 110) */
    int recon;     /* 0 first order, 1 MUSCL minmod, 2 MUSCL van Leer */
    int xi_form;   /* 0: Eq. 86 with the Eq. 68 factor; 1: Eq. 86 literal */
    int scheme;    /* 0 Roe-AM (Eqs. 85-109); 1 classical Roe (Eq. 7 with Eqs. 8-12) */
    int dup_mode;  /* Roe-AM delta U_p: 0 Eq. 89; 1 zero; 2 the Roe term max(0, c - |U|) dp / (rho c^2)
                      as Section 7.6 writes it */
    int ufix;      /* 1 |U|' of Eq. 92; 0 |U|' = |U| (Section 7.1.1 variant) */
    int xi_roe;    /* Roe-AM with xi = |U| of Eq. 13 instead of Eq. 86 (Section 7.2 variants) */
    double harten; /* classical Roe: eps_lambda of the entropy fix of Eqs. 114-115 (0 = none) */
} orc_params;

typedef struct {
    int ni, nj;
    int bc[4];              /* W, E, S, N */
    double inflow[4];       /* rho, u, v, p on INFLOW sides */
    const double *xv, *yv;  /* (nj+1) x (ni+1) vertices, i fastest; NULL => Cartesian */
    double dx, dy;
    const unsigned char *solid; /* nj x ni, NULL => none */
    orc_params prm;
} orc_grid;

/* ------------------------------------------------------------------ scalar helpers */
static real rmin(real a, real b) { return a < b ? a : b; }
static real rmax(real a, real b) { return a > b ? a : b; }
static real sgn(real a) { return (real)((a > 0) - (a < 0)); }   /* sgn(0) = 0 */
static real pow8(real a) { real a2 = a * a, a4 = a2 * a2; return a4 * a4; }

/* Eq. 98 (also Eq. 25): f(phi) = min(phi sqrt(4 + (1 - phi^2)^2) / (1 + phi^2), 1). */
static real fmach(real phi)
{
    real p2 = phi * phi;
    real t = 1 - p2;
    return rmin(phi * RSQRT_(4 + t * t) / (1 + p2), 1);
}

double ORC_API(orc_f)(double phi) { return (double)fmach((real)phi); }

/* Eq. 97: ratio indicator of the face between cells a and b (cell-centre rho, p). */
static real ratio_P(real ra, real pa, real rb, real pb)
{
    return rmin(rmin(pa / pb, pb / pa), rmin(ra / rb, rb / ra));
}

/* ------------------------------------------------------------------ the face flux */
typedef struct { real rho, u, v, H, c2, c, U; } roe_state;

/* Roe averages with sqrt(rho) weights (Roe 1981; the paper adopts them, Section 4.2). */
static roe_state roe_average(const real WL[4], const real WR[4], real nx, real ny, real g)
{
    roe_state s;
    real sL = RSQRT_(WL[0]), sR = RSQRT_(WR[0]);
    real HL = g / (g - 1) * WL[3] / WL[0] + (real)0.5 * (WL[1] * WL[1] + WL[2] * WL[2]);
    real HR = g / (g - 1) * WR[3] / WR[0] + (real)0.5 * (WR[1] * WR[1] + WR[2] * WR[2]);
    real w = 1 / (sL + sR);
    s.rho = sL * sR;
    s.u = (sL * WL[1] + sR * WR[1]) * w;
    s.v = (sL * WL[2] + sR * WR[2]) * w;
    s.H = (sL * HL + sR * HR) * w;
    s.c2 = (g - 1) * (s.H - (real)0.5 * (s.u * s.u + s.v * s.v));
    s.c = RSQRT_(s.c2);
    s.U = nx * s.u + ny * s.v;
    return s;
}

/* Numerical flux per unit face length through a face with unit normal (nx, ny) pointing
 * from L to R. W = (rho, u, v, p). s1 is the detector value of Eq. 95 (or 1). */
static void face_flux(const orc_params *P, const real WL[4], const real WR[4], real nx, real ny, real s1,
                      real F[4])
{
    const real g = (real)P->gamma;
    /* Each side: normal velocity, total enthalpy, sound speed (Eqs. 1, 4, 54). */
    real UL = nx * WL[1] + ny * WL[2], UR = nx * WR[1] + ny * WR[2];
    real HL = g / (g - 1) * WL[3] / WL[0] + (real)0.5 * (WL[1] * WL[1] + WL[2] * WL[2]);
    real HR = g / (g - 1) * WR[3] / WR[0] + (real)0.5 * (WR[1] * WR[1] + WR[2] * WR[2]);
    real cL = RSQRT_(g * WL[3] / WL[0]), cR = RSQRT_(g * WR[3] / WR[0]);
    /* Vectors (rho, rho u, rho v, rho H) of both sides: energy slot carries rho H (Eq. 49). */
    real QL[4] = {WL[0], WL[0] * WL[1], WL[0] * WL[2], WL[0] * HL};
    real QR[4] = {WR[0], WR[0] * WR[1], WR[0] * WR[2], WR[0] * HR};
    real pn[4] = {0, nx, ny, 0};
    int k;

    /* Central term, Eqs. 3-4. */
    real Fc[4];
    for (k = 0; k < 4; ++k)
        Fc[k] = (real)0.5 * ((UL * QL[k] + WL[3] * pn[k]) + (UR * QR[k] + WR[3] * pn[k]));

    roe_state h = roe_average(WL, WR, nx, ny, g);
    real dU = UR - UL, dp = WR[3] - WL[3];
    real hv[4] = {h.rho, h.rho * h.u, h.rho * h.v, h.rho * h.H};

    if (P->scheme == 1) {
        /* Classical Roe in the scale framework: Eq. 7 with the eigenvalue forms Eqs. 8-12
         * (Eqs. 13-17 when no entropy fix); Delta(rho E) in the xi term and U in the energy slot
         * of the pressure vector. The entropy fix of Eqs. 114-115 replaces every eigenvalue
         * below h = eps_lambda max(lambda_i) by (lambda^2 / h + h) / 2. */
        real aU = RABS_(h.U);
        real l1 = aU, l4 = RABS_(h.U - h.c), l5 = RABS_(h.U + h.c);
        if (P->harten > 0) {
            real hh = (real)P->harten * rmax(l1, rmax(l4, l5));
            if (l1 < hh) l1 = (real)0.5 * (l1 * l1 / hh + hh);
            if (l4 < hh) l4 = (real)0.5 * (l4 * l4 / hh + hh);
            if (l5 < hh) l5 = (real)0.5 * (l5 * l5 / hh + hh);
        }
        real xi = l1;                                               /* Eq. 8 */
        real dpu = ((l5 + l4) / 2 - l1) * h.rho * dU;               /* Eq. 9 */
        real dpp = (l5 - l4) / 2 * dp / h.c;                        /* Eq. 10 */
        real dUu = (l5 - l4) / 2 * dU / h.c;                        /* Eq. 11 */
        real dUp = ((l5 + l4) / 2 - l1) * dp / (h.rho * h.c2);      /* Eq. 12 */
        real EL = WL[3] / (g - 1) + (real)0.5 * WL[0] * (WL[1] * WL[1] + WL[2] * WL[2]);
        real ER = WR[3] / (g - 1) + (real)0.5 * WR[0] * (WR[1] * WR[1] + WR[2] * WR[2]);
        real dQ[4] = {WR[0] - WL[0], QR[1] - QL[1], QR[2] - QL[2], ER - EL};
        real pv[4] = {0, nx, ny, h.U};
        for (k = 0; k < 4; ++k)
            F[k] = Fc[k] - (real)0.5 * (xi * dQ[k] + (dpu + dpp) * pv[k] + (dUu + dUp) * hv[k]);
        return;
    }

    /* Roe-AM, Section 6.2. */
    real qL = RSQRT_(WL[1] * WL[1] + WL[2] * WL[2]), qR = RSQRT_(WR[1] * WR[1] + WR[2] * WR[2]);
    real M = (real)0.5 * (qL / cL + qR / cR);                     /* Eq. 93 */
    real aU = RABS_(h.U);
    real Mb = aU / h.c;                                           /* Eq. 94 */
    real fM = fmach(M), fMb = fmach(Mb);                          /* Eq. 98 */
    real fM8 = pow8(fM), fMb8 = pow8(fMb);

    /* Eq. 92: expansion-shock fix of |U| (clamped at zero). */
    real Up = aU;
    if (P->ufix) {
        real e = rmax(0, dU);
        Up = aU - fMb * (sgn(h.U + h.c) * e - sgn(h.U - h.c) * e) / 4;
        Up = rmax(Up, 0);
    }

    /* Eqs. 99-101. */
    real Mr2 = (real)P->m_ref * (real)P->m_ref;
    real theta = rmin(rmax(Mr2, M * M), 1);
    real om = 1 - theta;
    real ct = (real)0.5 * RSQRT_(4 * h.c2 * theta + om * om * h.U * h.U);
    real Ut = (real)0.5 * (1 + theta) * h.U;

    /* Eq. 86: basic upwind dissipation xi. */
    real xi_fac = (P->xi_form == 0) ? (1 - fMb8) : 1;
    real xi1 = RABS_((real)0.5 * (UR + UL)) + xi_fac * (real)0.5 * dU;
    real xi2 = 0;
    if (P->eps1) {
        real fef = (real)P->eps2 * h.c;                           /* Eq. 102 */
        /* Eqs. 103-109: rotated-Riemann estimate. */
        real du = WR[1] - WL[1], dv = WR[2] - WL[2];
        real dq = RSQRT_(du * du + dv * dv);
        real n1x = nx, n1y = ny;
        if (!(dq < (real)1e-5 * (real)P->u_ref)) { n1x = du / dq; n1y = dv / dq; }   /* Eq. 108 */
        real kz = n1x * ny - n1y * nx;                            /* (n1 x n) . e_z */
        real sk = sgn(kz);
        real n2x = -sk * n1y, n2y = sk * n1x;                     /* Eq. 109, normalised */
        real a1 = n1x * nx + n1y * ny, a2 = n2x * nx + n2y * ny;  /* Eqs. 106-107 */
        real U1 = n1x * h.u + n1y * h.v, U2 = n2x * h.u + n2y * h.v;   /* Eqs. 104-105 */
        real frr = RABS_(a1 * U1) + RABS_(a2 * U2);               /* Eq. 103 */
        xi2 = (1 - fMb8) * fM8 * rmin(fef, frr);
    }
    real xi = rmax(xi1, xi2);
    if (P->xi_roe) xi = aU;                                       /* Eq. 13 (Section 7.2 variant) */

    real mn = rmin(Up, h.c);
    real dpp = sgn(h.U) * mn * dp / h.c;                                  /* Eq. 87 */
    real dpu = (1 - s1 + s1 * fM) * rmax(0, h.c - Up) * h.rho * dU;        /* Eq. 88 */
    real dUp;
    if (P->dup_mode == 1)
        dUp = 0;
    else if (P->dup_mode == 2)
        dUp = rmax(0, h.c - aU) * dp / (h.rho * h.c2);                     /* Eq. 17 as in Section 7.6 */
    else
        dUp = s1 * (1 - fM8) *
              (rmax(0, ct - Up) + om * (Up - h.U / (2 * ct) * sgn(Ut) * rmin(RABS_(Ut), ct))) *
              dp / (h.rho * theta * h.c2);                                 /* Eq. 89 */
    real dUu = (real)0.5 * sgn(h.U) * mn * dU / h.c;                      /* Eqs. 90-91 */

    /* Eq. 85 (with Eq. 49: Delta(rho H) in the xi term, 0 in the pressure vector's energy slot). */
    for (k = 0; k < 4; ++k) {
        real dQ = QR[k] - QL[k];
        real Fd = -(real)0.5 * (xi * dQ + (dpp + dpu) * pn[k] + dUp * hv[k] + dUu * QR[k] + dUu * QL[k]);
        F[k] = Fc[k] + Fd;
    }
}

/* Batched face flux for tests: n faces, W arrays n x 4, normals n x 2 (unit), s1 n. */
void ORC_API(orc_face_flux)(const orc_params *P, int n, const double *WL, const double *WR, const double *nrm,
                            const double *s1, double *F)
{
    for (int f = 0; f < n; ++f) {
        real L[4], R[4], out[4];
        for (int k = 0; k < 4; ++k) { L[k] = WL[4 * f + k]; R[k] = WR[4 * f + k]; }
        face_flux(P, L, R, nrm[2 * f], nrm[2 * f + 1], s1 ? s1[f] : 1, out);
        for (int k = 0; k < 4; ++k) F[4 * f + k] = (double)out[k];
    }
}

/* Roe-averaged state (rho, u, v, H, c) per face, for tests. */
void ORC_API(orc_roe_average)(int n, const double *WL, const double *WR, double gamma, double *out)
{
    for (int f = 0; f < n; ++f) {
        real L[4], R[4];
        for (int k = 0; k < 4; ++k) { L[k] = WL[4 * f + k]; R[k] = WR[4 * f + k]; }
        roe_state h = roe_average(L, R, 1, 0, gamma);
        out[5 * f + 0] = h.rho; out[5 * f + 1] = h.u; out[5 * f + 2] = h.v;
        out[5 * f + 3] = h.H; out[5 * f + 4] = h.c;
    }
}

/* ------------------------------------------------------------------ grid access */
typedef struct {
    const orc_grid *g;
    real *W;          /* primitives (rho, u, v, p), 4 planes of nj x ni */
} field;

static int solid_at(const orc_grid *g, int i, int j) { return g->solid ? g->solid[(size_t)j * g->ni + i] : 0; }

static real vx(const orc_grid *g, int i, int j) { return g->xv ? g->xv[(size_t)j * (g->ni + 1) + i] : i * g->dx; }
static real vy(const orc_grid *g, int i, int j) { return g->yv ? g->yv[(size_t)j * (g->ni + 1) + i] : j * g->dy; }

/* Face vector of the x-face on vertex column ic (between cells ic-1 and ic), row j,
 * pointing towards +i: S = (dy, -dx) of the edge from vertex (ic, j) to (ic, j+1). */
static void xface_S(const orc_grid *g, int ic, int j, real *Sx, real *Sy)
{
    *Sx = vy(g, ic, j + 1) - vy(g, ic, j);
    *Sy = -(vx(g, ic, j + 1) - vx(g, ic, j));
}
/* Face vector of the y-face on vertex row jc (between cells jc-1 and jc), column i,
 * pointing towards +j: S = (-dy, dx) of the edge from vertex (i, jc) to (i+1, jc). */
static void yface_S(const orc_grid *g, int i, int jc, real *Sx, real *Sy)
{
    *Sx = -(vy(g, i + 1, jc) - vy(g, i, jc));
    *Sy = vx(g, i + 1, jc) - vx(g, i, jc);
}
static real cell_V(const orc_grid *g, int i, int j)
{
    real d1x = vx(g, i + 1, j + 1) - vx(g, i, j), d1y = vy(g, i + 1, j + 1) - vy(g, i, j);
    real d2x = vx(g, i, j + 1) - vx(g, i + 1, j), d2y = vy(g, i, j + 1) - vy(g, i + 1, j);
    return (real)0.5 * (d1x * d2y - d1y * d2x);
}

static void mirror(const real in[4], real nx, real ny, real out[4])
{
    real un = in[1] * nx + in[2] * ny;
    out[0] = in[0];
    out[1] = in[1] - 2 * un * nx;
    out[2] = in[2] - 2 * un * ny;
    out[3] = in[3];
}

static int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

/* State of cell (i, j) for i in [-2, ni+1], j in [-2, nj+1]: interior values, or ghost
 * values from the boundary conditions, resolving the i direction first, then j.
 * *is_solid reports whether the resolved cell is solid; *is_wall whether a WALL side
 * produced it. */
static void ext_state(const field *fd, int i, int j, real out[4], int *is_solid, int *is_wall)
{
    const orc_grid *g = fd->g;
    const int ni = g->ni, nj = g->nj;
    if (i < 0 || i >= ni) {
        int side = i < 0 ? SIDE_W : SIDE_E;
        int bc = g->bc[side];
        if (bc == BC_INFLOW) {
            for (int k = 0; k < 4; ++k) out[k] = (real)g->inflow[k];
            *is_solid = 0; *is_wall = 0;
            return;
        }
        int ii;
        if (bc == BC_PERIODIC) ii = ((i % ni) + ni) % ni;
        else if (bc == BC_OUTFLOW) ii = i < 0 ? 0 : ni - 1;
        else ii = i < 0 ? -1 - i : 2 * ni - 1 - i;
        ext_state(fd, ii, j, out, is_solid, is_wall);
        if (bc == BC_WALL) {
            real Sx, Sy;
            xface_S(g, i < 0 ? 0 : ni, clampi(j, 0, nj - 1), &Sx, &Sy);
            real L = RSQRT_(Sx * Sx + Sy * Sy);
            real tmp[4];
            mirror(out, Sx / L, Sy / L, tmp);
            memcpy(out, tmp, sizeof(tmp));
            *is_wall = 1;
        }
        return;
    }
    if (j < 0 || j >= nj) {
        int side = j < 0 ? SIDE_S : SIDE_N;
        int bc = g->bc[side];
        if (bc == BC_INFLOW) {
            for (int k = 0; k < 4; ++k) out[k] = (real)g->inflow[k];
            *is_solid = 0; *is_wall = 0;
            return;
        }
        int jj;
        if (bc == BC_PERIODIC) jj = ((j % nj) + nj) % nj;
        else if (bc == BC_OUTFLOW) jj = j < 0 ? 0 : nj - 1;
        else jj = j < 0 ? -1 - j : 2 * nj - 1 - j;
        ext_state(fd, i, jj, out, is_solid, is_wall);
        if (bc == BC_WALL) {
            real Sx, Sy;
            yface_S(g, i, j < 0 ? 0 : nj, &Sx, &Sy);
            real L = RSQRT_(Sx * Sx + Sy * Sy);
            real tmp[4];
            mirror(out, Sx / L, Sy / L, tmp);
            memcpy(out, tmp, sizeof(tmp));
            *is_wall = 1;
        }
        return;
    }
    size_t c = (size_t)j * ni + i, N = (size_t)ni * nj;
    for (int k = 0; k < 4; ++k) out[k] = fd->W[k * N + c];
    *is_solid = solid_at(g, i, j);
    *is_wall = 0;
}

/* Eq. 97 on the face between two (possibly ghost) cells; 1 if either side is solid. */
static real P_between(const field *fd, int ia, int ja, int ib, int jb)
{
    real a[4], b[4];
    int sa, wa, sb, wb;
    ext_state(fd, ia, ja, a, &sa, &wa);
    ext_state(fd, ib, jb, b, &sb, &wb);
    if (sa || sb) return 1;
    return ratio_P(a[0], a[3], b[0], b[3]);
}

/* Eqs. 95-96 in 2D for the face between cell A = (i, j) and cell B = (i+di, j+dj):
 * a = min over the face itself and the four transverse faces of A and B. */
static real detector_s1(const field *fd, int i, int j, int di, int dj)
{
    if (!fd->g->prm.use_s1) return 1;                   /* Eq. 110 */
    int ti = dj, tj = di;                               /* transverse direction */
    int bi = i + di, bj = j + dj;
    real a = P_between(fd, i, j, bi, bj);
    a = rmin(a, P_between(fd, bi, bj, bi - ti, bj - tj));
    a = rmin(a, P_between(fd, bi, bj, bi + ti, bj + tj));
    a = rmin(a, P_between(fd, i, j, i - ti, j - tj));
    a = rmin(a, P_between(fd, i, j, i + ti, j + tj));
    return pow8(fmach(a));
}

static real limiter(int kind, real a, real b)
{
    if (kind == 1) return (real)0.5 * (sgn(a) + sgn(b)) * rmin(RABS_(a), RABS_(b));   /* minmod */
    if (a * b <= 0) return 0;                                                          /* van Leer */
    return (a * RABS_(b) + RABS_(a) * b) / (RABS_(a) + RABS_(b));
}

/* Left and right states of the face between cells A = (i, j) and B = (i+di, j+dj), (di, dj)
 * in {(1,0), (0,1)}, with unit normal (nx, ny) from A to B. A wall face (a solid or WALL-ghost
 * side) takes the first-order fluid state and its mirror image about the face; otherwise the
 * cell states, reconstructed by MUSCL when recon != 0. Returns 0 when both sides are solid
 * (no face), else 1. */
static int face_states(const field *fd, int i, int j, int di, int dj, real nx, real ny, real WL[4], real WR[4])
{
    const orc_grid *g = fd->g;
    real A[4], B[4];
    int sA, wA, sB, wB;
    ext_state(fd, i, j, A, &sA, &wA);
    ext_state(fd, i + di, j + dj, B, &sB, &wB);
    if (sA && sB) return 0;
    if (sA || sB || wA || wB) {
        /* Wall face: first-order fluid state and its mirror image about this face. */
        if (sA || wA) { memcpy(WR, B, sizeof(B)); mirror(B, nx, ny, WL); }
        else { memcpy(WL, A, sizeof(A)); mirror(A, nx, ny, WR); }
        return 1;
    }
    memcpy(WL, A, sizeof(A));
    memcpy(WR, B, sizeof(B));
    if (g->prm.recon) {
        real Am[4], Bp[4];
        int s, w;
        ext_state(fd, i - di, j - dj, Am, &s, &w);
        if (s) {   /* stencil cell is solid: mirror of A about the face between them */
            real tx, ty;
            if (di) xface_S(g, i, j, &tx, &ty); else yface_S(g, i, j, &tx, &ty);
            real l = RSQRT_(tx * tx + ty * ty);
            mirror(A, tx / l, ty / l, Am);
        }
        ext_state(fd, i + 2 * di, j + 2 * dj, Bp, &s, &w);
        if (s) {
            real tx, ty;
            if (di) xface_S(g, i + 2, j, &tx, &ty); else yface_S(g, i, j + 2, &tx, &ty);
            real l = RSQRT_(tx * tx + ty * ty);
            mirror(B, tx / l, ty / l, Bp);
        }
        real rL[4], rR[4];
        for (int k = 0; k < 4; ++k) {
            rL[k] = A[k] + (real)0.5 * limiter(g->prm.recon, A[k] - Am[k], B[k] - A[k]);
            rR[k] = B[k] - (real)0.5 * limiter(g->prm.recon, B[k] - A[k], Bp[k] - B[k]);
        }
        /* Positivity of the reconstructed density and pressure, else first order. */
        if (rL[0] > 0 && rL[3] > 0 && rR[0] > 0 && rR[3] > 0) {
            memcpy(WL, rL, sizeof(rL));
            memcpy(WR, rR, sizeof(rR));
        }
    }
    return 1;
}

/* Flux F*|S| through the face between cells A = (i, j) and B = (i+di, j+dj), (di, dj) in
 * {(1,0), (0,1)}, with face vector S pointing from A to B. Returns 0 and F = 0 when both
 * sides are solid. */
static int face_flux_grid(const field *fd, int i, int j, int di, int dj, real Sx, real Sy, real F[4])
{
    real len = RSQRT_(Sx * Sx + Sy * Sy);
    real nx = Sx / len, ny = Sy / len;
    real WL[4], WR[4];
    for (int k = 0; k < 4; ++k) F[k] = 0;
    if (!face_states(fd, i, j, di, dj, nx, ny, WL, WR)) return 0;
    real s1 = detector_s1(fd, i, j, di, dj);
    face_flux(&fd->g->prm, WL, WR, nx, ny, s1, F);
    for (int k = 0; k < 4; ++k) F[k] *= len;
    return 1;
}

static void to_prim(const orc_grid *g, const double *U, real *W)
{
    size_t N = (size_t)g->ni * g->nj;
    real gm1 = (real)g->prm.gamma - 1;
    for (size_t c = 0; c < N; ++c) {
        real r = U[c], ru = U[N + c], rv = U[2 * N + c], rE = U[3 * N + c];
        real u = ru / r, v = rv / r;
        W[c] = r; W[N + c] = u; W[2 * N + c] = v;
        W[3 * N + c] = gm1 * (rE - (real)0.5 * r * (u * u + v * v));
    }
}

/* R = -(1/V) sum_f F_f |S_f| (outward), by a loop over every face scattering to its cells. */
static void residual(const orc_grid *g, const double *U, real *R, real *W)
{
    const int ni = g->ni, nj = g->nj;
    const size_t N = (size_t)ni * nj;
    field fd = {g, W};
    to_prim(g, U, W);
    for (size_t c = 0; c < 4 * N; ++c) R[c] = 0;

    /* x-faces: vertex columns ic = 0..ni (periodic: ic = 0 is the same face as ic = ni). */
    int ic0 = g->bc[SIDE_W] == BC_PERIODIC ? 1 : 0;
    for (int j = 0; j < nj; ++j)
        for (int ic = ic0; ic <= ni; ++ic) {
            real Sx, Sy, F[4];
            xface_S(g, ic, j, &Sx, &Sy);
            if (!face_flux_grid(&fd, ic - 1, j, 1, 0, Sx, Sy, F)) continue;
            int il = ic - 1, ir = ic;
            if (g->bc[SIDE_W] == BC_PERIODIC && ir == ni) ir = 0;
            if (il >= 0 && il < ni && !solid_at(g, il, j))
                for (int k = 0; k < 4; ++k) R[k * N + (size_t)j * ni + il] -= F[k];
            if (ir >= 0 && ir < ni && !solid_at(g, ir, j))
                for (int k = 0; k < 4; ++k) R[k * N + (size_t)j * ni + ir] += F[k];
        }
    /* y-faces: vertex rows jc = 0..nj. */
    int jc0 = g->bc[SIDE_S] == BC_PERIODIC ? 1 : 0;
    for (int jc = jc0; jc <= nj; ++jc)
        for (int i = 0; i < ni; ++i) {
            real Sx, Sy, F[4];
            yface_S(g, i, jc, &Sx, &Sy);
            if (!face_flux_grid(&fd, i, jc - 1, 0, 1, Sx, Sy, F)) continue;
            int jl = jc - 1, jr = jc;
            if (g->bc[SIDE_S] == BC_PERIODIC && jr == nj) jr = 0;
            if (jl >= 0 && jl < nj && !solid_at(g, i, jl))
                for (int k = 0; k < 4; ++k) R[k * N + (size_t)jl * ni + i] -= F[k];
            if (jr >= 0 && jr < nj && !solid_at(g, i, jr))
                for (int k = 0; k < 4; ++k) R[k * N + (size_t)jr * ni + i] += F[k];
        }
    for (int j = 0; j < nj; ++j)
        for (int i = 0; i < ni; ++i) {
            real V = cell_V(g, i, j);
            for (int k = 0; k < 4; ++k) R[k * N + (size_t)j * ni + i] /= V;
        }
}

void ORC_API(orc_residual)(const orc_grid *g, const double *U, double *Rout)
{
    size_t N = (size_t)g->ni * g->nj;
    real *R = (real *)malloc(4 * N * sizeof(real));
    real *W = (real *)malloc(4 * N * sizeof(real));
    residual(g, U, R, W);
    for (size_t c = 0; c < 4 * N; ++c) Rout[c] = (double)R[c];
    free(R);
    free(W);
}

/* Largest signal speed of the Roe-AM dissipation normal to a face with unit normal n:
 * |U| + max(c, c~/theta), with theta and c~ of Eqs. 99-101 evaluated on the cell state
 * (M = |q|/c). For theta = 1 this is the classical |U| + c; at low Mach the preconditioned
 * delta U_p of Eq. 89 makes c~/theta ~ c/M_ref the fastest dissipative speed. */
static real signal_speed(real Un, real c, real q2, real mref)
{
    real th = rmin(rmax(mref * mref, q2 / (c * c)), 1);
    real om = 1 - th;
    real ct = (real)0.5 * RSQRT_(4 * c * c * th + om * om * Un * Un);
    return RABS_(Un) + rmax(c, ct / th);
}

/* Largest sum_dir speed_dir |S_dir| / V over fluid cells (S_dir the mean of opposite face
 * vectors), from the state U: the explicit step is dt = CFL / max_rate. */
double ORC_API(orc_max_rate)(const orc_grid *g, const double *U)
{
    const int ni = g->ni, nj = g->nj;
    const size_t N = (size_t)ni * nj;
    real gm = (real)g->prm.gamma;
    /* the classical Roe scheme has no preconditioned term: theta = 1 gives |U| + c */
    real mref = g->prm.scheme == 1 ? 1 : (real)g->prm.m_ref;
    real best = 0;
    for (int j = 0; j < nj; ++j)
        for (int i = 0; i < ni; ++i) {
            if (solid_at(g, i, j)) continue;
            size_t c = (size_t)j * ni + i;
            real r = U[c], u = U[N + c] / r, v = U[2 * N + c] / r;
            real p = (gm - 1) * (U[3 * N + c] - (real)0.5 * r * (u * u + v * v));
            real cs = RSQRT_(gm * p / r);
            real ax, ay, bx, by;
            xface_S(g, i, j, &ax, &ay);
            xface_S(g, i + 1, j, &bx, &by);
            real Xx = (real)0.5 * (ax + bx), Xy = (real)0.5 * (ay + by);
            yface_S(g, i, j, &ax, &ay);
            yface_S(g, i, j + 1, &bx, &by);
            real Yx = (real)0.5 * (ax + bx), Yy = (real)0.5 * (ay + by);
            real lx = RSQRT_(Xx * Xx + Xy * Xy), ly = RSQRT_(Yx * Yx + Yy * Yy);
            real q2 = u * u + v * v;
            real lam = signal_speed((u * Xx + v * Xy) / lx, cs, q2, mref) * lx +
                       signal_speed((u * Yx + v * Yy) / ly, cs, q2, mref) * ly;
            lam /= cell_V(g, i, j);
            best = rmax(best, lam);
        }
    return (double)best;
}

/* One SSP-RK3 step (Shu & Osher): U1 = U + dt R(U); U2 = 3/4 U + 1/4 (U1 + dt R(U1));
 * U <- 1/3 U + 2/3 (U2 + dt R(U2)). dt = dt_fixed if > 0, else cfl / max_rate(U).
 * Solid cells are left unchanged. Returns the dt used. */
double ORC_API(orc_rk_step)(const orc_grid *g, double *U, double cfl, double dt_fixed)
{
    const size_t N = (size_t)g->ni * g->nj;
    double dt = dt_fixed > 0 ? dt_fixed : cfl / ORC_API(orc_max_rate)(g, U);
    real *R = (real *)malloc(4 * N * sizeof(real));
    real *W = (real *)malloc(4 * N * sizeof(real));
    double *U0 = (double *)malloc(4 * N * sizeof(double));
    double *Uk = (double *)malloc(4 * N * sizeof(double));
    memcpy(U0, U, 4 * N * sizeof(double));
    memcpy(Uk, U, 4 * N * sizeof(double));
    static const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
    static const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
    for (int s = 0; s < 3; ++s) {
        residual(g, Uk, R, W);
        for (size_t c = 0; c < 4 * N; ++c) {
            real upd = (real)Uk[c] + (real)dt * R[c];
            Uk[c] = (double)((real)ca[s] * (real)U0[c] + (real)cb[s] * upd);
        }
    }
    memcpy(U, Uk, 4 * N * sizeof(double));
    free(R); free(W); free(U0); free(Uk);
    return dt;
}

/* Conserved totals sum_i V_i Q_i over fluid cells. */
void ORC_API(orc_totals)(const orc_grid *g, const double *U, double out[4])
{
    const size_t N = (size_t)g->ni * g->nj;
    real acc[4] = {0, 0, 0, 0};
    for (int j = 0; j < g->nj; ++j)
        for (int i = 0; i < g->ni; ++i) {
            if (solid_at(g, i, j)) continue;
            real V = cell_V(g, i, j);
            size_t c = (size_t)j * g->ni + i;
            for (int k = 0; k < 4; ++k) acc[k] += V * (real)U[k * N + c];
        }
    for (int k = 0; k < 4; ++k) out[k] = (double)acc[k];
}

/* Detector s1 (Eq. 95) of every face, for tests: sx is nj x (ni+1) (x-face on vertex column ic
 * at index j*(ni+1)+ic), sy is (nj+1) x ni. */
void ORC_API(orc_detector)(const orc_grid *g, const double *U, double *sx, double *sy)
{
    const size_t N = (size_t)g->ni * g->nj;
    real *W = (real *)malloc(4 * N * sizeof(real));
    field fd = {g, W};
    to_prim(g, U, W);
    for (int j = 0; j < g->nj; ++j)
        for (int ic = 0; ic <= g->ni; ++ic)
            sx[(size_t)j * (g->ni + 1) + ic] = (double)detector_s1(&fd, ic - 1, j, 1, 0);
    for (int jc = 0; jc <= g->nj; ++jc)
        for (int i = 0; i < g->ni; ++i)
            sy[(size_t)jc * g->ni + i] = (double)detector_s1(&fd, i, jc - 1, 0, 1);
    free(W);
}

/* Left and right primitive states (rho, u, v, p) of n faces, for tests: face f lies between
 * cell (ij[2f], ij[2f+1]) and its neighbour in +i (dir[f] = 0) or +j (dir[f] = 1); WL and WR
 * receive 4 values per face. A face with two solid sides gives zeros. */
void ORC_API(orc_face_states)(const orc_grid *g, const double *U, int n, const int *ij, const int *dir, double *WL,
                              double *WR)
{
    const size_t N = (size_t)g->ni * g->nj;
    real *W = (real *)malloc(4 * N * sizeof(real));
    field fd = {g, W};
    to_prim(g, U, W);
    for (int f = 0; f < n; ++f) {
        const int i = ij[2 * f], j = ij[2 * f + 1], di = dir[f] ? 0 : 1, dj = dir[f] ? 1 : 0;
        real Sx, Sy;
        if (di) xface_S(g, i + 1, j, &Sx, &Sy); else yface_S(g, i, j + 1, &Sx, &Sy);
        real len = RSQRT_(Sx * Sx + Sy * Sy);
        real L[4] = {0, 0, 0, 0}, R[4] = {0, 0, 0, 0};
        face_states(&fd, i, j, di, dj, Sx / len, Sy / len, L, R);
        for (int k = 0; k < 4; ++k) { WL[4 * f + k] = (double)L[k]; WR[4 * f + k] = (double)R[k]; }
    }
    free(W);
}
