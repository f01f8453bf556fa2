/*
 * roeam_oracle3.c — plain, slow CPU oracle of the complete Roe-AM scheme in 3D with passive
 * scalars (the form of Eq. 85 with rho w and rho k rows, and the 9-face detector of Eq. 96).
 *
 * TEST INFRASTRUCTURE ONLY, like roeam_oracle.c: only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; it shares no code with the product library.
 * It is also independent of the 2D oracle (its own small helpers); a test checks that the two
 * agree on 2D data.
 *
 * Scope: structured Cartesian 3D grids, first-order face states, the SSP-RK3 update.
 * Variables: W = (rho, u, v, w, p, k_1..k_S) and Q = (rho, rho u, rho v, rho w, rho E,
 * rho k_1..rho k_S), S <= 3 passive scalars, each carried by the flow (Eq. 85's last rows).
 * Host layout [nv][nk][nj][ni], i fastest, nv = 5 + S.
 *
 * Readings (the same as the 2D oracle where they overlap):
 *   xi      — Eq. 86 with the [1 - f^8(Mbar)] factor of Eq. 68 on dU/2 (xi_form = 0).
 *   |U|'    — Eq. 92 with f(Mbar), clamped at 0. Face U, c, rho: Roe averages; sgn(0) = 0.
 *   k^      — the scalars of the delta U_p vector take Roe (sqrt(rho)-weighted) averages,
 *             like u, v, w and H.
 *   n2      — Eq. 109 read in 3D: n2 is the unit vector along n - (n . n1) n1, the part of the
 *             face normal perpendicular to n1 (0 when n1 is parallel to n).
 *   ghosts  — a neighbour outside the grid is resolved axis by axis (x, then y, then z) with
 *             that axis's boundary condition: periodic wrap, zero-gradient copy, the INFLOW
 *             state, or the WALL mirror (normal velocity component negated, scalars copied).
 *   dt      — CFL / max_i sum_dir (|U_dir| + max(c, c~/theta)) / h_dir with theta, c~ of
 *             Eqs. 99-101 on the cell state.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORC_LONG
#define ORC_LONG 0
#endif

#if ORC_LONG
typedef long double real;
#define SQRT3_(x) sqrtl(x)
#define ABS3_(x) fabsl(x)
#define ORC3_API(name) name##_ld
#else
typedef double real;
#define SQRT3_(x) sqrt(x)
#define ABS3_(x) fabs(x)
#define ORC3_API(name) name
#endif

#define MAXS 3
#define MAXV (5 + MAXS)

enum { B3_PERIODIC = 0, B3_WALL = 1, B3_INFLOW = 2, B3_OUTFLOW = 3 };

typedef struct {
    double gamma, m_ref, u_ref, eps2;
    int eps1, use_s1, xi_form, nscal;
} orc3_params;

typedef struct {
    int ni, nj, nk;
    int bc[6];              /* W, E (x); S, N (y); B, T (z) */
    double inflow[MAXV];    /* rho, u, v, w, p, k_1.. on INFLOW sides */
    double dx, dy, dz;
    orc3_params prm;
} orc3_grid;

static real mn3(real a, real b) { return a < b ? a : b; }
static real mx3(real a, real b) { return a > b ? a : b; }
static real sg3(real a) { return (real)((a > 0) - (a < 0)); }
static real p8(real a) { real a2 = a * a, a4 = a2 * a2; return a4 * a4; }

/* Eq. 98. */
static real fm3(real phi)
{
    real p2 = phi * phi, t = 1 - p2;
    return mn3(phi * SQRT3_(4 + t * t) / (1 + p2), 1);
}

/* Eq. 97 between two cells given their (rho, p). */
static real ratio3(real ra, real pa, real rb, real pb)
{
    return mn3(mn3(pa / pb, pb / pa), mn3(ra / rb, rb / ra));
}

/* Numerical flux per unit area through a face with unit normal n, from primitive states
 * W = (rho, u, v, w, p, k..) and detector value s1. Section 6.2 term by term. */
static void face_flux3(const orc3_params *P, const real *WL, const real *WR, const real n[3], real s1, real *F)
{
    const int ns = P->nscal, nv = 5 + ns;
    const real g = (real)P->gamma;
    real UL = n[0] * WL[1] + n[1] * WL[2] + n[2] * WL[3];
    real UR = n[0] * WR[1] + n[1] * WR[2] + n[2] * WR[3];
    real q2L = WL[1] * WL[1] + WL[2] * WL[2] + WL[3] * WL[3];
    real q2R = WR[1] * WR[1] + WR[2] * WR[2] + WR[3] * WR[3];
    real HL = g / (g - 1) * WL[4] / WL[0] + (real)0.5 * q2L;
    real HR = g / (g - 1) * WR[4] / WR[0] + (real)0.5 * q2R;
    real cL = SQRT3_(g * WL[4] / WL[0]), cR = SQRT3_(g * WR[4] / WR[0]);
    real QL[MAXV], QR[MAXV], pn[MAXV];
    int k;
    /* (rho, rho u, rho v, rho w, rho H, rho k..): energy slot carries rho H (Eq. 49) */
    QL[0] = WL[0]; QR[0] = WR[0];
    for (k = 1; k <= 3; ++k) { QL[k] = WL[0] * WL[k]; QR[k] = WR[0] * WR[k]; }
    QL[4] = WL[0] * HL; QR[4] = WR[0] * HR;
    for (k = 0; k < ns; ++k) { QL[5 + k] = WL[0] * WL[5 + k]; QR[5 + k] = WR[0] * WR[5 + k]; }
    for (k = 0; k < nv; ++k) pn[k] = 0;
    pn[1] = n[0]; pn[2] = n[1]; pn[3] = n[2];

    /* central part, Eqs. 3-4 */
    real Fc[MAXV];
    for (k = 0; k < nv; ++k) Fc[k] = (real)0.5 * (UL * QL[k] + WL[4] * pn[k] + UR * QR[k] + WR[4] * pn[k]);

    /* Roe averages (sqrt(rho) weights) of u, v, w, H and the scalars */
    real sL = SQRT3_(WL[0]), sR = SQRT3_(WR[0]), wgt = 1 / (sL + sR);
    real rh = sL * sR;
    real qh[3];
    for (k = 0; k < 3; ++k) qh[k] = (sL * WL[1 + k] + sR * WR[1 + k]) * wgt;
    real Hh = (sL * HL + sR * HR) * wgt;
    real kh[MAXS];
    for (k = 0; k < ns; ++k) kh[k] = (sL * WL[5 + k] + sR * WR[5 + k]) * wgt;
    real c2h = (g - 1) * (Hh - (real)0.5 * (qh[0] * qh[0] + qh[1] * qh[1] + qh[2] * qh[2]));
    real ch = SQRT3_(c2h);
    real Uh = n[0] * qh[0] + n[1] * qh[1] + n[2] * qh[2];
    real dU = UR - UL, dp = WR[4] - WL[4];

    real M = (real)0.5 * (SQRT3_(q2L) / cL + SQRT3_(q2R) / cR);   /* Eq. 93 */
    real aU = ABS3_(Uh);
    real Mb = aU / ch;                                             /* Eq. 94 */
    real fM = fm3(M), fMb = fm3(Mb), fM8 = p8(fM), fMb8 = p8(fMb);

    /* Eq. 92, clamped at 0 */
    real e = mx3(0, dU);
    real Up = mx3(aU - fMb * (sg3(Uh + ch) * e - sg3(Uh - ch) * e) / 4, 0);

    /* Eqs. 99-101 */
    real Mr2 = (real)P->m_ref * (real)P->m_ref;
    real th = mn3(mx3(Mr2, M * M), 1), om = 1 - th;
    real ct = (real)0.5 * SQRT3_(4 * c2h * th + om * om * Uh * Uh);
    real Ut = (real)0.5 * (1 + th) * Uh;

    /* Eq. 86 */
    real xi = ABS3_((real)0.5 * (UR + UL)) + (P->xi_form == 0 ? 1 - fMb8 : 1) * (real)0.5 * dU;
    real xi2 = 0;
    if (P->eps1) {
        real fef = (real)P->eps2 * ch;                                            /* Eq. 102 */
        real dq[3] = {WR[1] - WL[1], WR[2] - WL[2], WR[3] - WL[3]};
        real dqn = SQRT3_(dq[0] * dq[0] + dq[1] * dq[1] + dq[2] * dq[2]);
        real n1[3] = {n[0], n[1], n[2]};
        if (!(dqn < (real)1e-5 * (real)P->u_ref))                                 /* Eq. 108 */
            for (k = 0; k < 3; ++k) n1[k] = dq[k] / dqn;
        real a1 = n1[0] * n[0] + n1[1] * n[1] + n1[2] * n[2];                     /* Eq. 106 */
        real t[3] = {n[0] - a1 * n1[0], n[1] - a1 * n1[1], n[2] - a1 * n1[2]};
        real tn = SQRT3_(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
        real n2[3] = {0, 0, 0};
        if (tn > 0) for (k = 0; k < 3; ++k) n2[k] = t[k] / tn;                     /* Eq. 109 */
        real a2 = n2[0] * n[0] + n2[1] * n[1] + n2[2] * n[2];                     /* Eq. 107 */
        real U1 = n1[0] * qh[0] + n1[1] * qh[1] + n1[2] * qh[2];                  /* Eq. 104 */
        real U2 = n2[0] * qh[0] + n2[1] * qh[1] + n2[2] * qh[2];                  /* Eq. 105 */
        real frr = ABS3_(a1 * U1) + ABS3_(a2 * U2);                               /* Eq. 103 */
        xi2 = (1 - fMb8) * fM8 * mn3(fef, frr);
    }
    xi = mx3(xi, xi2);

    real mnU = mn3(Up, ch);
    real dpp = sg3(Uh) * mnU * dp / ch;                                           /* Eq. 87 */
    real dpu = (1 - s1 + s1 * fM) * mx3(0, ch - Up) * rh * dU;                    /* Eq. 88 */
    real dUp = s1 * (1 - fM8) *
               (mx3(0, ct - Up) + om * (Up - Uh / (2 * ct) * sg3(Ut) * mn3(ABS3_(Ut), ct))) *
               dp / (rh * th * c2h);                                              /* Eq. 89 */
    real dUu = (real)0.5 * sg3(Uh) * mnU * dU / ch;                               /* Eqs. 90-91 */

    real hv[MAXV];
    hv[0] = rh;
    for (k = 0; k < 3; ++k) hv[1 + k] = rh * qh[k];
    hv[4] = rh * Hh;
    for (k = 0; k < ns; ++k) hv[5 + k] = rh * kh[k];
    for (k = 0; k < nv; ++k)                                                      /* Eq. 85 */
        F[k] = Fc[k] - (real)0.5 * (xi * (QR[k] - QL[k]) + (dpp + dpu) * pn[k] + dUp * hv[k] +
                                    dUu * QR[k] + dUu * QL[k]);
}

void ORC3_API(orc3_face_flux)(const orc3_params *P, int n, const double *WL, const double *WR, const double *nrm,
                              const double *s1, double *F)
{
    const int nv = 5 + P->nscal;
    for (int f = 0; f < n; ++f) {
        real L[MAXV], R[MAXV], out[MAXV], nn[3];
        for (int k = 0; k < nv; ++k) { L[k] = WL[nv * f + k]; R[k] = WR[nv * f + k]; }
        for (int k = 0; k < 3; ++k) nn[k] = nrm[3 * f + k];
        face_flux3(P, L, R, nn, s1 ? s1[f] : 1, out);
        for (int k = 0; k < nv; ++k) F[nv * f + k] = (double)out[k];
    }
}

/* ------------------------------------------------------------------ the grid */
typedef struct {
    const orc3_grid *g;
    const real *W;   /* primitives [nv][nk][nj][ni] */
} field3;

static size_t cidx(const orc3_grid *g, int i, int j, int k)
{
    return ((size_t)k * g->nj + j) * g->ni + i;
}

/* Primitive state of cell (i, j, k), indices possibly outside the grid: resolved axis by
 * axis with each axis's boundary condition (see the readings above). */
static void ext3(const field3 *fd, int i, int j, int k, real *out)
{
    const orc3_grid *g = fd->g;
    const int nv = 5 + g->prm.nscal;
    const size_t N = (size_t)g->ni * g->nj * g->nk;
    int idx[3] = {i, j, k};
    const int n[3] = {g->ni, g->nj, g->nk};
    int flip[3] = {0, 0, 0}, inflow = 0;
    for (int ax = 0; ax < 3; ++ax) {
        int x = idx[ax];
        if (x >= 0 && x < n[ax]) continue;
        int bc = g->bc[2 * ax + (x < 0 ? 0 : 1)];
        if (bc == B3_PERIODIC) x = ((x % n[ax]) + n[ax]) % n[ax];
        else if (bc == B3_INFLOW) { inflow = 1; x = x < 0 ? 0 : n[ax] - 1; }
        else if (bc == B3_OUTFLOW) x = x < 0 ? 0 : n[ax] - 1;
        else { flip[ax] ^= 1; x = x < 0 ? -1 - x : 2 * n[ax] - 1 - x; }
        if (x < 0) x = 0;
        if (x >= n[ax]) x = n[ax] - 1;
        idx[ax] = x;
    }
    if (inflow) {
        for (int v = 0; v < nv; ++v) out[v] = (real)g->inflow[v];
        return;
    }
    size_t c = cidx(g, idx[0], idx[1], idx[2]);
    for (int v = 0; v < nv; ++v) out[v] = fd->W[(size_t)v * N + c];
    for (int ax = 0; ax < 3; ++ax)
        if (flip[ax]) out[1 + ax] = -out[1 + ax];
}

static real P3(const field3 *fd, int ia, int ja, int ka, int ib, int jb, int kb)
{
    real A[MAXV], B[MAXV];
    ext3(fd, ia, ja, ka, A);
    ext3(fd, ib, jb, kb, B);
    return ratio3(A[0], A[4], B[0], B[4]);
}

/* s1 of Eq. 95 on the face between cell (i,j,k) and its +axis neighbour: a is the minimum of
 * P over that face and the 8 faces of the two cells along the other two axes (Eq. 96). */
static real detector3(const field3 *fd, int i, int j, int k, int ax)
{
    if (!fd->g->prm.use_s1) return 1;
    int d[3] = {0, 0, 0};
    d[ax] = 1;
    int i2 = i + d[0], j2 = j + d[1], k2 = k + d[2];
    real a = P3(fd, i, j, k, i2, j2, k2);
    for (int t = 0; t < 3; ++t) {
        if (t == ax) continue;
        int e[3] = {0, 0, 0};
        e[t] = 1;
        /* transverse faces of both cells, at -1/2 and +1/2 along axis t */
        a = mn3(a, P3(fd, i - e[0], j - e[1], k - e[2], i, j, k));
        a = mn3(a, P3(fd, i, j, k, i + e[0], j + e[1], k + e[2]));
        a = mn3(a, P3(fd, i2 - e[0], j2 - e[1], k2 - e[2], i2, j2, k2));
        a = mn3(a, P3(fd, i2, j2, k2, i2 + e[0], j2 + e[1], k2 + e[2]));
    }
    return a >= 1 ? 1 : p8(fm3(a));
}

static void to_prim3(const orc3_grid *g, const double *U, real *W)
{
    const int ns = g->prm.nscal;
    const size_t N = (size_t)g->ni * g->nj * g->nk;
    const real gm = (real)g->prm.gamma;
    for (size_t c = 0; c < N; ++c) {
        real r = U[c], u = U[N + c] / r, v = U[2 * N + c] / r, w = U[3 * N + c] / r;
        W[c] = r; W[N + c] = u; W[2 * N + c] = v; W[3 * N + c] = w;
        W[4 * N + c] = (gm - 1) * (U[4 * N + c] - (real)0.5 * r * (u * u + v * v + w * w));
        for (int s = 0; s < ns; ++s) W[(5 + s) * N + c] = U[(5 + s) * N + c] / r;
    }
}

/* R = -(1/V) sum_f F |S| by a loop over faces scattering to both cells. */
static void residual3(const orc3_grid *g, const double *U, real *R, real *W)
{
    const int nv = 5 + g->prm.nscal;
    const int ni = g->ni, nj = g->nj, nk = g->nk;
    const size_t N = (size_t)ni * nj * nk;
    const real h[3] = {(real)g->dx, (real)g->dy, (real)g->dz};
    const real area[3] = {h[1] * h[2], h[0] * h[2], h[0] * h[1]};
    const real vol = h[0] * h[1] * h[2];
    to_prim3(g, U, W);
    field3 fd = {g, W};
    memset(R, 0, sizeof(real) * nv * N);
    for (int ax = 0; ax < 3; ++ax) {
        real nrm[3] = {0, 0, 0};
        nrm[ax] = 1;
        int d[3] = {0, 0, 0};
        d[ax] = 1;
        /* faces between cell (i,j,k) - d and (i,j,k), for index i..(n) along ax */
        for (int k = 0; k < nk + d[2]; ++k)
            for (int j = 0; j < nj + d[1]; ++j)
                for (int i = 0; i < ni + d[0]; ++i) {
                    int il = i - d[0], jl = j - d[1], kl = k - d[2];
                    real A[MAXV], B[MAXV], F[MAXV];
                    ext3(&fd, il, jl, kl, A);
                    ext3(&fd, i, j, k, B);
                    face_flux3(&g->prm, A, B, nrm, detector3(&fd, il, jl, kl, ax), F);
                    int inL = il >= 0 && jl >= 0 && kl >= 0;
                    int inR = i < ni && j < nj && k < nk;
                    for (int v = 0; v < nv; ++v) {
                        if (inL) R[(size_t)v * N + cidx(g, il, jl, kl)] -= F[v] * area[ax];
                        if (inR) R[(size_t)v * N + cidx(g, i, j, k)] += F[v] * area[ax];
                    }
                }
    }
    for (size_t c = 0; c < (size_t)nv * N; ++c) R[c] /= vol;
}

void ORC3_API(orc3_residual)(const orc3_grid *g, const double *U, double *Rout)
{
    const size_t N = (size_t)g->ni * g->nj * g->nk, nv = 5 + g->prm.nscal;
    real *R = (real *)malloc(nv * N * sizeof(real)), *W = (real *)malloc(nv * N * sizeof(real));
    residual3(g, U, R, W);
    for (size_t c = 0; c < nv * N; ++c) Rout[c] = (double)R[c];
    free(R);
    free(W);
}

/* max over cells of sum_dir (|U_dir| + max(c, c~/theta)) / h_dir */
double ORC3_API(orc3_max_rate)(const orc3_grid *g, const double *U)
{
    const size_t N = (size_t)g->ni * g->nj * g->nk;
    const real gm = (real)g->prm.gamma, mr = (real)g->prm.m_ref;
    const real h[3] = {(real)g->dx, (real)g->dy, (real)g->dz};
    real best = 0;
    for (size_t c = 0; c < N; ++c) {
        real r = U[c], q[3] = {U[N + c] / r, U[2 * N + c] / r, U[3 * N + c] / r};
        real q2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
        real p = (gm - 1) * (U[4 * N + c] - (real)0.5 * r * q2);
        real c2 = gm * p / r, cs = SQRT3_(c2);
        real th = mn3(mx3(mr * mr, q2 / c2), 1), om = 1 - th;
        real lam = 0;
        for (int ax = 0; ax < 3; ++ax) {
            real ct = (real)0.5 * SQRT3_(4 * c2 * th + om * om * q[ax] * q[ax]);
            lam += (ABS3_(q[ax]) + mx3(cs, ct / th)) / h[ax];
        }
        best = mx3(best, lam);
    }
    return (double)best;
}

/* One SSP-RK3 step (Shu & Osher) in place; returns dt. */
double ORC3_API(orc3_rk_step)(const orc3_grid *g, double *U, double cfl, double dt_fixed)
{
    const size_t N = (size_t)g->ni * g->nj * g->nk, nv = 5 + g->prm.nscal, M = nv * N;
    double dt = dt_fixed > 0 ? dt_fixed : cfl / ORC3_API(orc3_max_rate)(g, U);
    double *U0 = (double *)malloc(M * sizeof(double)), *Us = (double *)malloc(M * sizeof(double));
    real *R = (real *)malloc(M * sizeof(real)), *W = (real *)malloc(M * sizeof(real));
    const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0};
    memcpy(U0, U, M * sizeof(double));
    memcpy(Us, U, M * sizeof(double));
    for (int s = 0; s < 3; ++s) {
        residual3(g, Us, R, W);
        for (size_t c = 0; c < M; ++c) Us[c] = (double)(ca[s] * (real)U0[c] + cb[s] * ((real)Us[c] + dt * R[c]));
    }
    memcpy(U, Us, M * sizeof(double));
    free(U0); free(Us); free(R); free(W);
    return dt;
}

void ORC3_API(orc3_totals)(const orc3_grid *g, const double *U, double *out)
{
    const size_t N = (size_t)g->ni * g->nj * g->nk, nv = 5 + g->prm.nscal;
    const real vol = (real)g->dx * (real)g->dy * (real)g->dz;
    for (size_t v = 0; v < nv; ++v) {
        real s = 0;
        for (size_t c = 0; c < N; ++c) s += vol * U[v * N + c];
        out[v] = (double)s;
    }
}

/* s1 of every face along axis ax between cell c and its +ax neighbour (faces leaving the
 * grid included: (ni x nj x nk) values, ghost neighbours resolved by the boundary conditions). */
void ORC3_API(orc3_detector)(const orc3_grid *g, const double *U, int ax, double *s1)
{
    const size_t N = (size_t)g->ni * g->nj * g->nk, nv = 5 + g->prm.nscal;
    real *W = (real *)malloc(nv * N * sizeof(real));
    to_prim3(g, U, W);
    field3 fd = {g, W};
    for (int k = 0; k < g->nk; ++k)
        for (int j = 0; j < g->nj; ++j)
            for (int i = 0; i < g->ni; ++i) s1[cidx(g, i, j, k)] = (double)detector3(&fd, i, j, k, ax);
    free(W);
}
