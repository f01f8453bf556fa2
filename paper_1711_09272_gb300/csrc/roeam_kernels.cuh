// roeam_kernels.cuh — sm_103a kernels of the Roe-AM finite-volume step.
//
// One fused kernel evaluates a whole Runge-Kutta stage per tile of TX x TY cells:
//   1. halo load: the tile plus a 1-cell (first order) or 2-cell (MUSCL) halo is read
//      once from HBM (structure-of-arrays planes, coalesced along i); ghost cells are
//      generated on the fly from the boundary conditions (periodic wrap, wall mirror,
//      inflow state, zero-gradient outflow), so no separate boundary kernel runs;
//   2. the ratio indicator P of Eq. 97 on every face the tile's detectors need;
//   3. the Roe-AM flux of Section 6.2 (Eqs. 85-109) on each x- and y-face of the tile,
//      with the detector s1 of Eqs. 95-96, MUSCL reconstruction when enabled;
//   4. the residual R = -(1/V) sum_f F_f |S_f| and the SSP-RK3 combination with U^n,
//      plus the next step's time-step rate and the positivity/finiteness status.
// The kernel is persistent: each CTA strides over the flattened tile list of every grid
// of the batch, so ragged batches of uneven grids run in one launch.
#pragma once

#include <cstdint>

#include "roeam_internal.h"

namespace roeam {

// ------------------------------------------------------------------ scalar helpers
template <typename T> __device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }
template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }
template <typename T> __device__ __forceinline__ T tabs(T a) { return a < T(0) ? -a : a; }
template <typename T> __device__ __forceinline__ T sgn(T a) { return T(int(a > T(0)) - int(a < T(0))); }
template <typename T> __device__ __forceinline__ T pow8(T a) { T a2 = a * a, a4 = a2 * a2; return a4 * a4; }

// Eq. 98: f(phi) = min(phi sqrt(4 + (1 - phi^2)^2) / (1 + phi^2), 1); exactly 1 for phi >= 1.
template <typename T> __device__ __forceinline__ T fmach(T phi)
{
    if (phi >= T(1)) return T(1);
    T p2 = phi * phi, t = T(1) - p2;
    return tmin(phi * sqrt(T(4) + t * t) / (T(1) + p2), T(1));
}

// Mirror image of a velocity about a unit normal (wall ghost state).
template <typename T> __device__ __forceinline__ void mirror_vel(T &u, T &v, T nx, T ny)
{
    T un = u * nx + v * ny;
    u -= T(2) * un * nx;
    v -= T(2) * un * ny;
}

// Scheme constants of one grid in the working precision.
template <typename T> struct Coef {
    T g, gm1, gm1i, mr2, rr_thr, eps2;
    int eps1, xi_form;
};

template <typename T> __device__ __forceinline__ Coef<T> make_coef(const GridDev &G)
{
    Coef<T> c;
    c.g = T(G.gamma);
    c.gm1 = T(G.gamma - 1.0);
    c.gm1i = T(1.0 / (G.gamma - 1.0));
    c.mr2 = T(G.m_ref * G.m_ref);
    c.rr_thr = T(1e-5 * G.u_ref);
    c.eps2 = T(G.eps2);
    c.eps1 = G.eps1;
    c.xi_form = G.xi_form;
    return c;
}

// Per-side quantities of a face state W = (rho, u, v, p).
template <typename T> struct Side { T r, u, v, p, c2, H, sr, Un, Mq; };

template <typename T> __device__ __forceinline__ Side<T> make_side(T r, T u, T v, T p, T nx, T ny, const Coef<T> &K)
{
    Side<T> s;
    s.r = r; s.u = u; s.v = v; s.p = p;
    s.c2 = K.g * p / r;
    T q2 = u * u + v * v;
    s.H = s.c2 * K.gm1i + T(0.5) * q2;
    s.sr = sqrt(r);
    s.Un = nx * u + ny * v;
    s.Mq = sqrt(q2 / s.c2);    // |q| / c
    return s;
}

// Roe-AM numerical flux per unit face length (Section 6.2), unit normal n from L to R.
template <typename T>
__device__ __forceinline__ void roeam_flux(const Side<T> &L, const Side<T> &R, T nx, T ny, T s1, const Coef<T> &K,
                                           T F[4])
{
    // Central term, Eqs. 3-4.
    const T mL = L.r * L.Un, mR = R.r * R.Un;
    T Fc0 = T(0.5) * (mL + mR);
    T Fc1 = T(0.5) * (mL * L.u + L.p * nx + mR * R.u + R.p * nx);
    T Fc2 = T(0.5) * (mL * L.v + L.p * ny + mR * R.v + R.p * ny);
    T Fc3 = T(0.5) * (mL * L.H + mR * R.H);

    // Roe averages; c^2 in the sum-of-positives form (no cancellation at high Mach).
    const T w = T(1) / (L.sr + R.sr);
    const T rh = L.sr * R.sr;
    const T uh = (L.sr * L.u + R.sr * R.u) * w;
    const T vh = (L.sr * L.v + R.sr * R.v) * w;
    const T Hh = (L.sr * L.H + R.sr * R.H) * w;
    const T du = R.u - L.u, dv = R.v - L.v;
    const T c2h = (L.sr * L.c2 + R.sr * R.c2) * w + T(0.5) * K.gm1 * rh * w * w * (du * du + dv * dv);
    const T ch = sqrt(c2h);
    const T chi = T(1) / ch;
    const T Uh = nx * uh + ny * vh;
    const T aU = tabs(Uh);

    const T M = T(0.5) * (L.Mq + R.Mq);         // Eq. 93
    const T Mb = aU * chi;                       // Eq. 94
    const T fM = fmach(M), fMb = fmach(Mb);
    const T fM8 = pow8(fM), fMb8 = pow8(fMb);
    const T dUn = R.Un - L.Un, dp = R.p - L.p;

    // Eq. 92, clamped at zero.
    const T e = tmax(dUn, T(0));
    T Up = aU - fMb * (sgn(Uh + ch) - sgn(Uh - ch)) * e * T(0.25);
    Up = tmax(Up, T(0));

    // Eq. 86 (with the Eq. 68 factor unless xi_form = 1).
    const T xfac = K.xi_form ? T(1) : T(1) - fMb8;
    T xi = tabs(T(0.5) * (R.Un + L.Un)) + xfac * T(0.5) * dUn;
    if (K.eps1) {
        const T fef = K.eps2 * ch;                                   // Eq. 102
        const T dq = sqrt(du * du + dv * dv);
        T n1x = nx, n1y = ny;
        if (!(dq < K.rr_thr)) { const T dqi = T(1) / dq; n1x = du * dqi; n1y = dv * dqi; }   // Eq. 108
        const T sk = sgn(n1x * ny - n1y * nx);
        const T n2x = -sk * n1y, n2y = sk * n1x;                     // Eq. 109 (unit length)
        const T frr = tabs((n1x * nx + n1y * ny) * (n1x * uh + n1y * vh)) +
                      tabs((n2x * nx + n2y * ny) * (n2x * uh + n2y * vh));   // Eqs. 103-107
        xi = tmax(xi, (T(1) - fMb8) * fM8 * tmin(fef, frr));
    }
    xi = tmax(xi, T(0));

    const T mn = tmin(Up, ch);
    const T dpp = sgn(Uh) * mn * dp * chi;                                       // Eq. 87
    const T dpu = (T(1) - s1 + s1 * fM) * tmax(ch - Up, T(0)) * rh * dUn;       // Eq. 88
    T dUp = T(0);                                                                // Eq. 89
    const T sw = s1 * (T(1) - fM8);
    if (sw != T(0) && dp != T(0)) {
        const T theta = tmin(tmax(K.mr2, M * M), T(1));                          // Eq. 101
        const T om = T(1) - theta;
        const T ct = T(0.5) * sqrt(T(4) * c2h * theta + om * om * Uh * Uh);      // Eq. 99
        const T Ut = T(0.5) * (T(1) + theta) * Uh;                               // Eq. 100
        dUp = sw * (tmax(ct - Up, T(0)) + om * (Up - Uh / (T(2) * ct) * sgn(Ut) * tmin(tabs(Ut), ct))) * dp /
              (rh * theta * c2h);
    }
    const T dUu = T(0.5) * sgn(Uh) * mn * dUn * chi;                            // Eqs. 90-91

    // Eq. 85 with the energy convention of Eq. 49.
    const T pp = dpp + dpu;
    const T QL0 = L.r, QL1 = L.r * L.u, QL2 = L.r * L.v, QL3 = L.r * L.H;
    const T QR0 = R.r, QR1 = R.r * R.u, QR2 = R.r * R.v, QR3 = R.r * R.H;
    F[0] = Fc0 - T(0.5) * (xi * (QR0 - QL0) + dUp * rh + dUu * (QR0 + QL0));
    F[1] = Fc1 - T(0.5) * (xi * (QR1 - QL1) + pp * nx + dUp * rh * uh + dUu * (QR1 + QL1));
    F[2] = Fc2 - T(0.5) * (xi * (QR2 - QL2) + pp * ny + dUp * rh * vh + dUu * (QR2 + QL2));
    F[3] = Fc3 - T(0.5) * (xi * (QR3 - QL3) + dUp * rh * Hh + dUu * (QR3 + QL3));
}

// Largest dissipative signal speed normal to a face: |U| + max(c, c~/theta), Eqs. 99-101 on
// the cell state (classical |U| + c when theta = 1).
template <typename T> __device__ __forceinline__ T signal_speed(T Un, T c, T q2, T mr2)
{
    const T th = tmin(tmax(mr2, q2 / (c * c)), T(1));
    const T om = T(1) - th;
    const T ct = T(0.5) * sqrt(T(4) * c * c * th + om * om * Un * Un);
    return tabs(Un) + tmax(c, ct / th);
}

// ------------------------------------------------------------------ geometry
// Vertex (I, J) of a curvilinear grid sits at (I dx + dX(I, J), J dy + dY(I, J)).
// x-face on vertex column I, row J: S = (dy + dY(I,J+1) - dY(I,J), -(dX(I,J+1) - dX(I,J))).
// y-face on vertex row J, column I: S = (-(dY(I+1,J) - dY(I,J)), dx + dX(I+1,J) - dX(I,J)).
template <typename T> struct CellGeom { T Xx, Xy, Yx, Yy, V; };

template <typename T>
__device__ __forceinline__ CellGeom<T> cell_geom(T x00, T x10, T x01, T x11, T y00, T y10, T y01, T y11, T dx, T dy)
{
    CellGeom<T> c;
    c.Xx = dy + T(0.5) * ((y01 - y00) + (y11 - y10));
    c.Xy = -T(0.5) * ((x01 - x00) + (x11 - x10));
    c.Yx = -T(0.5) * ((y10 - y00) + (y11 - y01));
    c.Yy = dx + T(0.5) * ((x10 - x00) + (x11 - x01));
    const T d1x = dx + (x11 - x00), d1y = dy + (y11 - y00);
    const T d2x = -dx + (x01 - x10), d2y = dy + (y01 - y10);
    c.V = T(0.5) * (d1x * d2y - d1y * d2x);
    return c;
}

template <typename T>
__device__ __forceinline__ T cell_rate(T r, T u, T v, T p, const CellGeom<T> &cg, const Coef<T> &K)
{
    const T c = sqrt(K.g * p / r);
    const T q2 = u * u + v * v;
    const T lx = sqrt(cg.Xx * cg.Xx + cg.Xy * cg.Xy), ly = sqrt(cg.Yx * cg.Yx + cg.Yy * cg.Yy);
    const T sx = signal_speed((u * cg.Xx + v * cg.Xy) / lx, c, q2, K.mr2);
    const T sy = signal_speed((u * cg.Yx + v * cg.Yy) / ly, c, q2, K.mr2);
    return (sx * lx + sy * ly) / cg.V;
}

__device__ __forceinline__ int find_grid(const int *tile_base, int ngrids, int t)
{
    int lo = 0, hi = ngrids - 1;   // largest g with tile_base[g] <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(tile_base + mid) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

// State of cell (i, j) of grid G for i in [-2, ni+1], j in [-2, nj+1] as primitives, from
// the interior or, outside it, from the boundary conditions: the i direction is resolved
// first, then j; a WALL side mirrors the velocity about the boundary face normal. flag bit 0:
// the resolved cell is solid; bit 1: a WALL side produced it. Indices beyond the two ghost
// layers (ragged tiles) are clamped into the grid; their values are never used.
template <typename T, bool CURV>
__device__ __forceinline__ void load_ext(const StageArgs<T> &a, const GridDev &G, int i, int j, T w[4], uint8_t &fl)
{
    const int ni = G.ni, nj = G.nj;
    int ii = i, jj = j, mx = 0, my = 0;
    bool inflow = false;
    if (i < 0 || i >= ni) {
        const int bc = G.bc[i < 0 ? 0 : 1];
        if (bc == BC_INFLOW) inflow = true;
        else if (bc == BC_PERIODIC) ii = ((i % ni) + ni) % ni;
        else if (bc == BC_OUTFLOW) ii = i < 0 ? 0 : ni - 1;
        else { ii = i < 0 ? -1 - i : 2 * ni - 1 - i; mx = i < 0 ? 1 : 2; }
    }
    if (!inflow && (j < 0 || j >= nj)) {
        const int bc = G.bc[j < 0 ? 2 : 3];
        if (bc == BC_INFLOW) inflow = true;
        else if (bc == BC_PERIODIC) jj = ((j % nj) + nj) % nj;
        else if (bc == BC_OUTFLOW) jj = j < 0 ? 0 : nj - 1;
        else { jj = j < 0 ? -1 - j : 2 * nj - 1 - j; my = j < 0 ? 1 : 2; }
    }
    ii = clampi(ii, 0, ni - 1);
    jj = clampi(jj, 0, nj - 1);
    fl = 0;
    if (inflow) {
        w[0] = T(G.inflow[0]); w[1] = T(G.inflow[1]); w[2] = T(G.inflow[2]); w[3] = T(G.inflow[3]);
    } else {
        const long long c = G.off + (long long)jj * G.pitch + ii;
        const T r = a.src[c], ru = a.src[c + G.plane], rv = a.src[c + 2 * G.plane], rE = a.src[c + 3 * G.plane];
        const T u = ru / r, v = rv / r;
        w[0] = r; w[1] = u; w[2] = v;
        w[3] = T(G.gamma - 1.0) * (rE - T(0.5) * r * (u * u + v * v));
        if (G.soff >= 0 && a.solid[G.soff + (long long)jj * ni + ii]) fl |= 1;
    }
    if (my) {
        T nx = T(0), ny = T(1);
        if (CURV) {
            const int J = my == 1 ? 0 : nj;
            const long long b = G.voff + (long long)J * G.vpitch + ii;
            const T sx = -(a.vdy[b + 1] - a.vdy[b]), sy = T(G.dx) + (a.vdx[b + 1] - a.vdx[b]);
            const T l = sqrt(sx * sx + sy * sy);
            nx = sx / l; ny = sy / l;
        }
        mirror_vel(w[1], w[2], nx, ny);
    }
    if (mx) {
        T nx = T(1), ny = T(0);
        if (CURV) {
            const int I = mx == 1 ? 0 : ni;
            const int jr = clampi(j, 0, nj - 1);
            const long long b = G.voff + (long long)jr * G.vpitch + I;
            const T sx = T(G.dy) + (a.vdy[b + G.vpitch] - a.vdy[b]), sy = -(a.vdx[b + G.vpitch] - a.vdx[b]);
            const T l = sqrt(sx * sx + sy * sy);
            nx = sx / l; ny = sy / l;
        }
        mirror_vel(w[1], w[2], nx, ny);
    }
    if (mx || my) fl |= 2;
}

// ------------------------------------------------------------------ shared-memory tile
template <typename T, int TX, int TY, int H, bool CURV> struct Tile {
    static constexpr int HX = TX + 2 * H, HY = TY + 2 * H;
    static constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1);
    static constexpr int VX = CURV ? TX + 3 : 1, VY = CURV ? TY + 3 : 1;
    T W[4][HY][HX];            // primitives of the halo tile; cell (a, b) at [b + H][a + H]
    T Px[TY + 2][TX + 1];      // Eq. 97 on x-face column c between cells c-1, c; rows b = -1..TY at [b + 1]
    T Py[TY + 1][TX + 2];      // Eq. 97 on y-face row r between rows r-1, r; columns a = -1..TX at [a + 1]
    T Fx[4][TY][TX + 1];       // F |S| through x-face column c of row b
    T Fy[4][TY + 1][TX];       // F |S| through y-face row r of column a
    T vx[VY][VX], vy[VY][VX];  // vertex displacements, vertices i0-1..i0+TX+1, j0-1..j0+TY+1
    uint8_t flag[HY][HX];      // bit 0 solid, bit 1 wall ghost
};

// Smallest sizeof that holds a tile of each variant (dynamic shared memory per CTA).
template <typename T, int TX, int TY, bool MUSCL, bool CURV>
constexpr size_t tile_smem_bytes() { return sizeof(Tile<T, TX, TY, MUSCL ? 2 : 1, CURV>); }

template <typename T> __device__ __forceinline__ unsigned long long rate_bits(T r)
{
    return (unsigned long long)__double_as_longlong((double)r);
}

// Block-wide max of a non-negative value (all threads must call).
template <int NT> __device__ __forceinline__ double block_max(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    }
    return r;   // valid in thread 0
}

// ------------------------------------------------------------------ the fused stage kernel
template <typename T, int TX, int TY, int NT, bool MUSCL, bool CURV>
__global__ void __launch_bounds__(NT) stage_kernel(const StageArgs<T> a)
{
    constexpr int H = MUSCL ? 2 : 1;
    using TL = Tile<T, TX, TY, H, CURV>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TL &S = *reinterpret_cast<TL *>(smem_raw);
    __shared__ double red[NT / 32];
    const int tid = threadIdx.x;

    if (a.rate_zero && blockIdx.x == 0)
        for (int g = tid; g < a.ngrids; g += NT) a.rate_zero[g] = 0ull;

    double acc_s[4] = {0.0, 0.0, 0.0, 0.0}, acc_m[4] = {0.0, 0.0, 0.0, 0.0};

    for (int t = a.tile_lo + blockIdx.x; t < a.tile_hi; t += gridDim.x) {
        const int g = find_grid(a.tile_base, a.ngrids, t);
        const GridDev &G = a.grids[g];
        const int lt = t - G.tile_base;
        const int i0 = (lt % G.ntx) * TX, j0 = (lt / G.ntx) * TY;
        const int ni = G.ni, nj = G.nj;
        const Coef<T> K = make_coef<T>(G);
        const T dx = T(G.dx), dy = T(G.dy);
        const bool has_solid = G.soff >= 0;

        __syncthreads();   // the previous tile's readers of S are done
        // ---- 1. halo tile of primitives (ghosts from the boundary conditions)
        for (int idx = tid; idx < TL::HX * TL::HY; idx += NT) {
            const int la = idx % TL::HX, lb = idx / TL::HX;
            T w[4];
            uint8_t fl;
            load_ext<T, CURV>(a, G, i0 + la - H, j0 + lb - H, w, fl);
            S.W[0][lb][la] = w[0]; S.W[1][lb][la] = w[1]; S.W[2][lb][la] = w[2]; S.W[3][lb][la] = w[3];
            S.flag[lb][la] = fl;
        }
        if (CURV) {
            for (int idx = tid; idx < TL::VX * TL::VY; idx += NT) {
                const int va = idx % TL::VX, vb = idx / TL::VX;
                const int I = clampi(i0 - 1 + va, 0, ni), J = clampi(j0 - 1 + vb, 0, nj);
                const long long b = G.voff + (long long)J * G.vpitch + I;
                S.vx[vb][va] = a.vdx[b];
                S.vy[vb][va] = a.vdy[b];
            }
        }
        __syncthreads();

        // ---- 2. ratio indicator P (Eq. 97) on the faces the detectors read
        if (G.use_s1) {
            for (int idx = tid; idx < (TY + 2) * (TX + 1); idx += NT) {
                const int c = idx % (TX + 1), bb = idx / (TX + 1) - 1;     // cells (c-1, bb), (c, bb)
                const int ya = bb + H, xa = c - 1 + H;
                T P = T(1);
                if (!((S.flag[ya][xa] | S.flag[ya][xa + 1]) & 1)) {
                    const T p0 = S.W[3][ya][xa], p1 = S.W[3][ya][xa + 1];
                    const T r0 = S.W[0][ya][xa], r1 = S.W[0][ya][xa + 1];
                    P = tmin(tmin(p0, p1) / tmax(p0, p1), tmin(r0, r1) / tmax(r0, r1));
                }
                S.Px[bb + 1][c] = P;
            }
            for (int idx = tid; idx < (TY + 1) * (TX + 2); idx += NT) {
                const int aa = idx % (TX + 2) - 1, r = idx / (TX + 2);     // cells (aa, r-1), (aa, r)
                const int xa = aa + H, ya = r - 1 + H;
                T P = T(1);
                if (!((S.flag[ya][xa] | S.flag[ya + 1][xa]) & 1)) {
                    const T p0 = S.W[3][ya][xa], p1 = S.W[3][ya + 1][xa];
                    const T r0 = S.W[0][ya][xa], r1 = S.W[0][ya + 1][xa];
                    P = tmin(tmin(p0, p1) / tmax(p0, p1), tmin(r0, r1) / tmax(r0, r1));
                }
                S.Py[r][aa + 1] = P;
            }
            __syncthreads();
        }

        // ---- 3. Roe-AM flux through every x- and y-face of the tile
        for (int f = tid; f < TL::NFX + TL::NFY; f += NT) {
            const bool isx = f < TL::NFX;
            int fa, fb;          // x-face: column c, row b; y-face: column a, row r
            int Ax, Ay, dxs, dys;   // tile-array index of cell A and the step to B
            T Sx, Sy;
            bool inside;
            if (isx) {
                fa = f % (TX + 1); fb = f / (TX + 1);
                inside = (j0 + fb < nj) && (i0 + fa <= ni);
                Ax = fa - 1 + H; Ay = fb + H; dxs = 1; dys = 0;
                if (CURV) {
                    Sx = dy + (S.vy[fb + 2][fa + 1] - S.vy[fb + 1][fa + 1]);
                    Sy = -(S.vx[fb + 2][fa + 1] - S.vx[fb + 1][fa + 1]);
                } else { Sx = dy; Sy = T(0); }
            } else {
                const int ff = f - TL::NFX;
                fa = ff % TX; fb = ff / TX;
                inside = (i0 + fa < ni) && (j0 + fb <= nj);
                Ax = fa + H; Ay = fb - 1 + H; dxs = 0; dys = 1;
                if (CURV) {
                    Sx = -(S.vy[fb + 1][fa + 2] - S.vy[fb + 1][fa + 1]);
                    Sy = dx + (S.vx[fb + 1][fa + 2] - S.vx[fb + 1][fa + 1]);
                } else { Sx = T(0); Sy = dx; }
            }
            T F[4] = {T(0), T(0), T(0), T(0)};
            const uint8_t fA = S.flag[Ay][Ax], fB = S.flag[Ay + dys][Ax + dxs];
            if (inside && !((fA & fB) & 1)) {
                const T len = sqrt(Sx * Sx + Sy * Sy);
                const T nx = Sx / len, ny = Sy / len;
                T WL[4], WR[4];
                for (int k = 0; k < 4; ++k) { WL[k] = S.W[k][Ay][Ax]; WR[k] = S.W[k][Ay + dys][Ax + dxs]; }
                if ((fA | fB) != 0) {
                    // Wall face: the first-order fluid state and its mirror image about this face.
                    if (fA) { for (int k = 0; k < 4; ++k) WL[k] = WR[k]; mirror_vel(WL[1], WL[2], nx, ny); }
                    else { for (int k = 0; k < 4; ++k) WR[k] = WL[k]; mirror_vel(WR[1], WR[2], nx, ny); }
                } else if (MUSCL) {
                    T Am[4], Bp[4];
                    for (int k = 0; k < 4; ++k) {
                        Am[k] = S.W[k][Ay - dys][Ax - dxs];
                        Bp[k] = S.W[k][Ay + 2 * dys][Ax + 2 * dxs];
                    }
                    if (S.flag[Ay - dys][Ax - dxs] & 1) {   // solid stencil cell: mirror of A about their face
                        T tx, ty;
                        if (isx) {
                            if (CURV) { tx = dy + (S.vy[fb + 2][fa] - S.vy[fb + 1][fa]); ty = -(S.vx[fb + 2][fa] - S.vx[fb + 1][fa]); }
                            else { tx = dy; ty = T(0); }
                        } else {
                            if (CURV) { tx = -(S.vy[fb][fa + 2] - S.vy[fb][fa + 1]); ty = dx + (S.vx[fb][fa + 2] - S.vx[fb][fa + 1]); }
                            else { tx = T(0); ty = dx; }
                        }
                        const T l = sqrt(tx * tx + ty * ty);
                        for (int k = 0; k < 4; ++k) Am[k] = WL[k];
                        mirror_vel(Am[1], Am[2], tx / l, ty / l);
                    }
                    if (S.flag[Ay + 2 * dys][Ax + 2 * dxs] & 1) {
                        T tx, ty;
                        if (isx) {
                            if (CURV) { tx = dy + (S.vy[fb + 2][fa + 2] - S.vy[fb + 1][fa + 2]); ty = -(S.vx[fb + 2][fa + 2] - S.vx[fb + 1][fa + 2]); }
                            else { tx = dy; ty = T(0); }
                        } else {
                            if (CURV) { tx = -(S.vy[fb + 2][fa + 2] - S.vy[fb + 2][fa + 1]); ty = dx + (S.vx[fb + 2][fa + 2] - S.vx[fb + 2][fa + 1]); }
                            else { tx = T(0); ty = dx; }
                        }
                        const T l = sqrt(tx * tx + ty * ty);
                        for (int k = 0; k < 4; ++k) Bp[k] = WR[k];
                        mirror_vel(Bp[1], Bp[2], tx / l, ty / l);
                    }
                    T rL[4], rR[4], lLs[4], lRs[4];
                    const bool vl = G.limiter == 2;
                    for (int k = 0; k < 4; ++k) {
                        const T d0 = WL[k] - Am[k], d1 = WR[k] - WL[k], d2 = Bp[k] - WR[k];
                        T lL, lR;
                        if (vl) {
                            lL = (d0 * d1 <= T(0)) ? T(0) : (d0 * tabs(d1) + tabs(d0) * d1) / (tabs(d0) + tabs(d1));
                            lR = (d1 * d2 <= T(0)) ? T(0) : (d1 * tabs(d2) + tabs(d1) * d2) / (tabs(d1) + tabs(d2));
                        } else {
                            lL = T(0.5) * (sgn(d0) + sgn(d1)) * tmin(tabs(d0), tabs(d1));
                            lR = T(0.5) * (sgn(d1) + sgn(d2)) * tmin(tabs(d1), tabs(d2));
                        }
                        lLs[k] = lL;
                        lRs[k] = lR;
                        rL[k] = WL[k] + T(0.5) * lL;
                        rR[k] = WR[k] - T(0.5) * lR;
                    }
                    // Positivity of the reconstructed density and pressure, else first order. In
                    // FP32 a value within rounding of zero is re-decided exactly in FP64.
                    bool pos = rL[0] > T(0) && rL[3] > T(0) && rR[0] > T(0) && rR[3] > T(0);
                    if (sizeof(T) == 4 && pos) {
                        const T eps = T(1e-6);
                        if (rL[0] < eps * WL[0] || rL[3] < eps * WL[3] || rR[0] < eps * WR[0] || rR[3] < eps * WR[3]) {
                            pos = ((double)WL[0] + 0.5 * (double)lLs[0] > 0.0) && ((double)WL[3] + 0.5 * (double)lLs[3] > 0.0) &&
                                  ((double)WR[0] - 0.5 * (double)lRs[0] > 0.0) && ((double)WR[3] - 0.5 * (double)lRs[3] > 0.0);
                        }
                    }
                    if (pos) for (int k = 0; k < 4; ++k) { WL[k] = rL[k]; WR[k] = rR[k]; }
                }
                T s1 = T(1);
                if (G.use_s1) {
                    T am;
                    if (isx) {   // face column fa, row fb: cells A = (fa-1, fb), B = (fa, fb)
                        am = tmin(tmin(S.Px[fb + 1][fa], S.Py[fb][fa]), tmin(S.Py[fb + 1][fa], S.Py[fb][fa + 1]));
                        am = tmin(am, S.Py[fb + 1][fa + 1]);
                    } else {     // face row fb, column fa: cells A = (fa, fb-1), B = (fa, fb)
                        am = tmin(tmin(S.Py[fb][fa + 1], S.Px[fb][fa]), tmin(S.Px[fb][fa + 1], S.Px[fb + 1][fa]));
                        am = tmin(am, S.Px[fb + 1][fa + 1]);
                    }
                    s1 = pow8(fmach(am));
                }
                const Side<T> sl = make_side(WL[0], WL[1], WL[2], WL[3], nx, ny, K);
                const Side<T> sr = make_side(WR[0], WR[1], WR[2], WR[3], nx, ny, K);
                roeam_flux(sl, sr, nx, ny, s1, K, F);
                for (int k = 0; k < 4; ++k) F[k] *= len;
            }
            if (isx) { for (int k = 0; k < 4; ++k) S.Fx[k][fb][fa] = F[k]; }
            else { for (int k = 0; k < 4; ++k) S.Fy[k][fb][fa] = F[k]; }
        }
        __syncthreads();

        // ---- 4. residual, stage combination, next-step rate, status
        double dt = 0.0;
        if (a.mode == MODE_STAGE)
            dt = a.dt_fixed > 0.0 ? a.dt_fixed : a.cfl / __longlong_as_double((long long)a.rate_rd[g]);
        const T tdt = T(dt);
        double my_rate = 0.0;
        for (int cidx = tid; cidx < TX * TY; cidx += NT) {
            const int ca = cidx % TX, cb = cidx / TX;
            const int i = i0 + ca, j = j0 + cb;
            if (i >= ni || j >= nj) continue;
            const bool solid = has_solid && (S.flag[cb + H][ca + H] & 1);
            CellGeom<T> cg;
            if (CURV) {
                cg = cell_geom(S.vx[cb + 1][ca + 1], S.vx[cb + 1][ca + 2], S.vx[cb + 2][ca + 1], S.vx[cb + 2][ca + 2],
                               S.vy[cb + 1][ca + 1], S.vy[cb + 1][ca + 2], S.vy[cb + 2][ca + 1], S.vy[cb + 2][ca + 2],
                               dx, dy);
            } else {
                cg.Xx = dy; cg.Xy = T(0); cg.Yx = T(0); cg.Yy = dx; cg.V = dx * dy;
            }
            T R[4];
            for (int k = 0; k < 4; ++k)
                R[k] = solid ? T(0)
                             : ((S.Fx[k][cb][ca] - S.Fx[k][cb][ca + 1]) + (S.Fy[k][cb][ca] - S.Fy[k][cb + 1][ca])) / cg.V;
            const long long c = G.off + (long long)j * G.pitch + i;
            if (a.mode == MODE_STAGE) {
                T out[4];
                for (int k = 0; k < 4; ++k) {
                    const T upd = a.src[c + k * G.plane] + tdt * R[k];
                    out[k] = (a.alpha == T(0)) ? a.beta * upd : a.alpha * a.un[c + k * G.plane] + a.beta * upd;
                }
                for (int k = 0; k < 4; ++k) a.dst[c + k * G.plane] = out[k];
                if (!solid) {
                    const T u = out[1] / out[0], v = out[2] / out[0];
                    const T p = K.gm1 * (out[3] - T(0.5) * out[0] * (u * u + v * v));
                    if (!(out[0] > T(0)) || !(p > T(0))) {
                        const bool fin = isfinite((double)out[0]) && isfinite((double)p);
                        atomicOr(a.status, fin ? ST_NONPOSITIVE : ST_NONFINITE);
                    } else if (a.want_rate) {
                        my_rate = fmax(my_rate, (double)cell_rate(out[0], u, v, p, cg, K));
                    }
                }
            } else if (a.mode == MODE_RESIDUAL) {
                for (int k = 0; k < 4; ++k) a.dst[c + k * G.plane] = R[k];
            } else if (!solid) {
                for (int k = 0; k < 4; ++k) {
                    const double rk = (double)R[k];
                    acc_s[k] += rk * rk;
                    acc_m[k] = fmax(acc_m[k], fabs(rk));
                }
            }
        }
        if (a.want_rate) {
            const double m = block_max<NT>(my_rate, red);
            if (tid == 0 && m > 0.0) atomicMax(a.rate_wr + g, rate_bits(m));
        }
    }

    if (a.mode == MODE_NORM) {
        // Fixed-order block reduction of the FP64 partials: warp shuffles, then warp 0.
        __shared__ double wred[NT / 32][8];
        double v[8];
        for (int k = 0; k < 4; ++k) { v[k] = acc_s[k]; v[4 + k] = acc_m[k]; }
        for (int o = 16; o > 0; o >>= 1)
            for (int k = 0; k < 8; ++k) {
                const double x = __shfl_xor_sync(0xffffffffu, v[k], o);
                v[k] = k < 4 ? v[k] + x : fmax(v[k], x);
            }
        __syncthreads();
        if ((tid & 31) == 0)
            for (int k = 0; k < 8; ++k) wred[tid >> 5][k] = v[k];
        __syncthreads();
        if (tid < 8) {
            double r = tid < 4 ? 0.0 : 0.0;
            for (int w = 0; w < NT / 32; ++w) r = tid < 4 ? r + wred[w][tid] : fmax(r, wred[w][tid]);
            a.partials[(size_t)blockIdx.x * 8 + tid] = r;
        }
    }
}

// ------------------------------------------------------------------ small kernels
// Largest rate of every fluid cell of grids [g_lo, g_hi) (blockIdx.y = grid).
template <typename T, bool CURV>
__global__ void __launch_bounds__(256) rate_kernel(const GridDev *grids, int g_lo, const T *U, const T *vdx,
                                                   const T *vdy, const uint8_t *solid, unsigned long long *rate)
{
    __shared__ double red[8];
    const int g = g_lo + blockIdx.y;
    const GridDev &G = grids[g];
    const Coef<T> K = make_coef<T>(G);
    const T dx = T(G.dx), dy = T(G.dy);
    const long long n = (long long)G.ni * G.nj;
    double m = 0.0;
    for (long long q = (long long)blockIdx.x * 256 + threadIdx.x; q < n; q += (long long)gridDim.x * 256) {
        const int i = (int)(q % G.ni), j = (int)(q / G.ni);
        if (G.soff >= 0 && solid[G.soff + q]) continue;
        const long long c = G.off + (long long)j * G.pitch + i;
        const T r = U[c], u = U[c + G.plane] / r, v = U[c + 2 * G.plane] / r;
        const T p = K.gm1 * (U[c + 3 * G.plane] - T(0.5) * r * (u * u + v * v));
        CellGeom<T> cg;
        if (CURV) {
            const long long b = G.voff + (long long)j * G.vpitch + i;
            cg = cell_geom(vdx[b], vdx[b + 1], vdx[b + G.vpitch], vdx[b + G.vpitch + 1], vdy[b], vdy[b + 1],
                           vdy[b + G.vpitch], vdy[b + G.vpitch + 1], dx, dy);
        } else {
            cg.Xx = dy; cg.Xy = T(0); cg.Yx = T(0); cg.Yy = dx; cg.V = dx * dy;
        }
        m = fmax(m, (double)cell_rate(r, u, v, p, cg, K));
    }
    m = block_max<256>(m, red);
    if (threadIdx.x == 0 && m > 0.0) atomicMax(rate + g, rate_bits(m));
}

template <typename T>
__global__ void __launch_bounds__(256) pack_kernel(const GridDev *grids, int g_lo, const double *packed, T *U)
{
    const GridDev &G = grids[g_lo + blockIdx.y];
    const long long n = (long long)G.ni * G.nj;
    for (long long q = (long long)blockIdx.x * 256 + threadIdx.x; q < n; q += (long long)gridDim.x * 256) {
        const int i = (int)(q % G.ni), j = (int)(q / G.ni);
        const long long c = G.off + (long long)j * G.pitch + i;
        for (int k = 0; k < 4; ++k) U[c + k * G.plane] = T(packed[G.poff + k * n + q]);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) unpack_kernel(const GridDev *grids, int g_lo, const T *U, double *packed)
{
    const GridDev &G = grids[g_lo + blockIdx.y];
    const long long n = (long long)G.ni * G.nj;
    for (long long q = (long long)blockIdx.x * 256 + threadIdx.x; q < n; q += (long long)gridDim.x * 256) {
        const int i = (int)(q % G.ni), j = (int)(q / G.ni);
        const long long c = G.off + (long long)j * G.pitch + i;
        for (int k = 0; k < 4; ++k) packed[G.poff + k * n + q] = (double)U[c + k * G.plane];
    }
}

// FP64 block partials of sum V Q over the fluid cells of grid g (4 doubles per block).
template <typename T, bool CURV>
__global__ void __launch_bounds__(256) totals_kernel(const GridDev *grids, int g, const T *U, const T *vdx,
                                                     const T *vdy, const uint8_t *solid, double *partials)
{
    __shared__ double wred[8][4];
    const GridDev &G = grids[g];
    const long long n = (long long)G.ni * G.nj;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long q = (long long)blockIdx.x * 256 + threadIdx.x; q < n; q += (long long)gridDim.x * 256) {
        const int i = (int)(q % G.ni), j = (int)(q / G.ni);
        if (G.soff >= 0 && solid[G.soff + q]) continue;
        double V;
        if (CURV) {
            const long long b = G.voff + (long long)j * G.vpitch + i;
            V = (double)cell_geom(vdx[b], vdx[b + 1], vdx[b + G.vpitch], vdx[b + G.vpitch + 1], vdy[b], vdy[b + 1],
                                  vdy[b + G.vpitch], vdy[b + G.vpitch + 1], T(G.dx), T(G.dy)).V;
        } else {
            V = G.dx * G.dy;
        }
        const long long c = G.off + (long long)j * G.pitch + i;
        for (int k = 0; k < 4; ++k) s[k] += V * (double)U[c + k * G.plane];
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 4; ++k) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 4; ++k) wred[threadIdx.x >> 5][k] = s[k];
    __syncthreads();
    if (threadIdx.x < 4) {
        double r = 0.0;
        for (int w = 0; w < 8; ++w) r += wred[w][threadIdx.x];
        partials[(size_t)blockIdx.x * 4 + threadIdx.x] = r;
    }
}

// ------------------------------------------------------------------ launchers
template <typename T, int CFG, bool MUSCL, bool CURV> struct StageVariant {
    static constexpr int TX = TILE_CFGS[CFG].tx, TY = TILE_CFGS[CFG].ty, NT = TILE_CFGS[CFG].nt;
    static constexpr size_t SMEM = tile_smem_bytes<T, TX, TY, MUSCL, CURV>();
    // Opts the kernel in to its dynamic shared-memory size (once per process; the handle
    // calls occupancy() at creation, before any launch or graph capture).
    static cudaError_t prepare()
    {
        static cudaError_t done = cudaErrorNotReady;
        if (done != cudaSuccess)
            done = cudaFuncSetAttribute(stage_kernel<T, TX, TY, NT, MUSCL, CURV>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        return done;
    }
    static cudaError_t launch(const StageArgs<T> &a, int nblocks, cudaStream_t s)
    {
        cudaError_t e = prepare();
        if (e != cudaSuccess) return e;
        stage_kernel<T, TX, TY, NT, MUSCL, CURV><<<nblocks, NT, SMEM, s>>>(a);
        return cudaGetLastError();
    }
    static int occupancy()
    {
        if (prepare() != cudaSuccess) return 1;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage_kernel<T, TX, TY, NT, MUSCL, CURV>, NT, SMEM) !=
            cudaSuccess)
            return 1;
        return n > 0 ? n : 1;
    }
};

template <typename T, bool MUSCL, bool CURV>
static cudaError_t stage_dispatch_cfg(const StageArgs<T> &a, int cfg, int nblocks, cudaStream_t s)
{
    switch (cfg) {
    case 0: return StageVariant<T, 0, MUSCL, CURV>::launch(a, nblocks, s);
    case 1: return StageVariant<T, 1, MUSCL, CURV>::launch(a, nblocks, s);
    default: return StageVariant<T, 2, MUSCL, CURV>::launch(a, nblocks, s);
    }
}

template <typename T, bool MUSCL, bool CURV>
static int stage_occ_cfg(int cfg)
{
    switch (cfg) {
    case 0: return StageVariant<T, 0, MUSCL, CURV>::occupancy();
    case 1: return StageVariant<T, 1, MUSCL, CURV>::occupancy();
    default: return StageVariant<T, 2, MUSCL, CURV>::occupancy();
    }
}

template <typename T>
cudaError_t Launchers<T>::stage(const StageArgs<T> &a, int muscl, int curv, int cfg, int nblocks, cudaStream_t s)
{
    if (a.tile_hi <= a.tile_lo) return cudaSuccess;
    if (muscl) return curv ? stage_dispatch_cfg<T, true, true>(a, cfg, nblocks, s) : stage_dispatch_cfg<T, true, false>(a, cfg, nblocks, s);
    return curv ? stage_dispatch_cfg<T, false, true>(a, cfg, nblocks, s) : stage_dispatch_cfg<T, false, false>(a, cfg, nblocks, s);
}

template <typename T>
int Launchers<T>::stage_occupancy(int muscl, int curv, int cfg)
{
    if (muscl) return curv ? stage_occ_cfg<T, true, true>(cfg) : stage_occ_cfg<T, true, false>(cfg);
    return curv ? stage_occ_cfg<T, false, true>(cfg) : stage_occ_cfg<T, false, false>(cfg);
}

template <typename T>
cudaError_t Launchers<T>::rate(const GridDev *grids, int g_lo, int g_hi, const T *U, const T *vdx, const T *vdy,
                               const uint8_t *solid, unsigned long long *rate, int curv, cudaStream_t s)
{
    if (g_hi <= g_lo) return cudaSuccess;
    dim3 grid(64, g_hi - g_lo);
    if (curv) rate_kernel<T, true><<<grid, 256, 0, s>>>(grids, g_lo, U, vdx, vdy, solid, rate);
    else rate_kernel<T, false><<<grid, 256, 0, s>>>(grids, g_lo, U, vdx, vdy, solid, rate);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launchers<T>::pack(const GridDev *grids, int g_lo, int g_hi, int max_cells, const double *packed, T *U,
                               cudaStream_t s)
{
    if (g_hi <= g_lo) return cudaSuccess;
    int bx = (max_cells + 255) / 256;
    bx = bx < 1 ? 1 : (bx > 1024 ? 1024 : bx);
    pack_kernel<T><<<dim3(bx, g_hi - g_lo), 256, 0, s>>>(grids, g_lo, packed, U);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launchers<T>::unpack(const GridDev *grids, int g_lo, int g_hi, int max_cells, const T *U, double *packed,
                                 cudaStream_t s)
{
    if (g_hi <= g_lo) return cudaSuccess;
    int bx = (max_cells + 255) / 256;
    bx = bx < 1 ? 1 : (bx > 1024 ? 1024 : bx);
    unpack_kernel<T><<<dim3(bx, g_hi - g_lo), 256, 0, s>>>(grids, g_lo, U, packed);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launchers<T>::totals(const GridDev *grids, int g, const T *U, const T *vdx, const T *vdy,
                                 const uint8_t *solid, double *partials, int nblocks, int curv, cudaStream_t s)
{
    if (curv) totals_kernel<T, true><<<nblocks, 256, 0, s>>>(grids, g, U, vdx, vdy, solid, partials);
    else totals_kernel<T, false><<<nblocks, 256, 0, s>>>(grids, g, U, vdx, vdy, solid, partials);
    return cudaGetLastError();
}

}  // namespace roeam
