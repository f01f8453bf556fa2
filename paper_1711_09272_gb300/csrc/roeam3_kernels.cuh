// roeam3_kernels.cuh — the 3D Roe-AM path: Cartesian grids, first-order faces, up to three
// passive scalars (the complete form of Eq. 85, the 9-face detector of Eq. 96), fused with the
// residual and the SSP-RK3 stage update like the 2D kernels.
//
// Decomposition: a CTA of TY3 = ty3<T>() warps (16 in FP32, 8 in FP64) holds a 32 x TY3 tile of
// an (x, y) plane, lane = column, warp = row (one halo column and row on each side), and marches
// along z over a segment of planes. Each thread keeps its cell's primitives for planes k-1, k, k+1 in registers (the
// z-faces and their detector values), exchanges plane k with its x-neighbours by shuffles and
// with its y-neighbours through shared memory (double-buffered by plane parity, one block
// barrier per plane: the row above's south flux of plane k is read after the barrier of
// plane k + 1), and evaluates the west x-face, the south y-face and the bottom z-face of its
// cell; a cell's east, north and top fluxes come from the neighbouring lane, warp and the
// next plane.
#pragma once

#include "roeam_kernels.cuh"
#include "roeam3_internal.h"

namespace roeam {

// Primitive and derived values of one cell: c2 = gamma p / rho, H total enthalpy,
// sr = sqrt(rho), Mq = |q| / c, scalars k.
template <typename T, int NS> struct C3 {
    T r, u, v, w, p, c2, H, sr, Mq;
    T k[NS > 0 ? NS : 1];
};

template <typename T, int NS>
__device__ __forceinline__ void derive3(C3<T, NS> &c, const GridCoef3<T> &K)
{
    const T ri = rcp(c.r);
    c.c2 = K.g * c.p * ri;
    const T q2 = c.u * c.u + c.v * c.v + c.w * c.w;
    c.H = vfma(c.c2, K.gm1i, T(0.5) * q2);
    c.sr = c.r * rsq(c.r);
    c.Mq = sqrt0(q2 * rcp(c.c2));
}

// Raw conserved values of the cell a thread loads for one plane, and how its indices resolved
// (kinds of resolve_index: 0 source cell, 1 WALL mirror, 2 INFLOW).
template <typename T, int NS> struct Pend3 {
    T q[5 + NS];
    int kz;
};

template <typename T, int NS>
__device__ __forceinline__ void issue3(const T *src, long long vol, long long xy, int pitch, int nj, int ksrc, int kz,
                                       bool inflow_xy, Pend3<T, NS> &p)
{
    p.kz = kz;
    if (!inflow_xy && kz != 2) {
        const long long x = (long long)ksrc * nj * pitch + xy;
#pragma unroll
        for (int v = 0; v < 5 + NS; ++v) p.q[v] = __ldg(src + x + v * vol);
    }
}

template <typename T, int NS>
__device__ __forceinline__ void finish3(const Pend3<T, NS> &p, bool inflow_xy, int kx, int ky, const GridCoef3<T> &K,
                                        C3<T, NS> &c)
{
    if (inflow_xy || p.kz == 2) {
        c.r = K.inflow[0]; c.u = K.inflow[1]; c.v = K.inflow[2]; c.w = K.inflow[3]; c.p = K.inflow[4];
#pragma unroll
        for (int s = 0; s < NS; ++s) c.k[s] = K.inflow[5 + s];
    } else {
        const T ri = rcp(p.q[0]);
        c.r = p.q[0];
        c.u = p.q[1] * ri; c.v = p.q[2] * ri; c.w = p.q[3] * ri;
        c.p = K.gm1 * (p.q[4] - T(0.5) * p.q[0] * (c.u * c.u + c.v * c.v + c.w * c.w));
#pragma unroll
        for (int s = 0; s < NS; ++s) c.k[s] = p.q[5 + s] * ri;
        if (kx == 1) c.u = -c.u;
        if (ky == 1) c.v = -c.v;
        if (p.kz == 1) c.w = -c.w;
    }
    derive3(c, K);
}

// One side of a face in the face frame: normal velocity un, tangential ut, uw. V is the
// working precision, or V2 for two faces evaluated together in packed FP32.
template <typename V, int NS> struct FS3 {
    V r, un, ut, uw, p, c2, H, sr, Mq;
    V k[NS > 0 ? NS : 1];
};

template <typename T, int NS>
__device__ __forceinline__ FS3<T, NS> side3(const C3<T, NS> &c, int axis)
{
    FS3<T, NS> s;
    s.r = c.r; s.p = c.p; s.c2 = c.c2; s.H = c.H; s.sr = c.sr; s.Mq = c.Mq;
    if (axis == 0) { s.un = c.u; s.ut = c.v; s.uw = c.w; }
    else if (axis == 1) { s.un = c.v; s.ut = c.u; s.uw = c.w; }
    else { s.un = c.w; s.ut = c.u; s.uw = c.v; }
#pragma unroll
    for (int q = 0; q < NS; ++q) s.k[q] = c.k[q];
    return s;
}

// The sides of an x-face (component x) and a y-face (component y) packed together.
template <int NS>
__device__ __forceinline__ FS3<V2, NS> side3_xy(const C3<float, NS> &cx, const C3<float, NS> &cy)
{
    FS3<V2, NS> s;
    s.r = mk2(cx.r, cy.r); s.p = mk2(cx.p, cy.p); s.c2 = mk2(cx.c2, cy.c2); s.H = mk2(cx.H, cy.H);
    s.sr = mk2(cx.sr, cy.sr); s.Mq = mk2(cx.Mq, cy.Mq);
    s.un = mk2(cx.u, cy.v); s.ut = mk2(cx.v, cy.u); s.uw = mk2(cx.w, cy.w);
#pragma unroll
    for (int q = 0; q < NS; ++q) s.k[q] = mk2(cx.k[q], cy.k[q]);
    return s;
}

// Twice the Roe-AM flux per unit area in the face frame (mass, normal momentum, the two
// tangential momenta, energy, scalars): Section 6.2 term by term as in roeam_flux2, with the
// w rows and Eq. 85's scalar rows; the rotated-Riemann estimate of Eqs. 103-109 in 3D
// (n2 the unit part of n perpendicular to n1, so |a2 U2| = |U - a1 U1|).
template <typename V, typename S, int NS>
__device__ __forceinline__ void roeam_flux3(const FS3<V, NS> &L, const FS3<V, NS> &R, V s1, const GridCoef3<S> &K,
                                            int eps1, int xi_form, V F[5 + NS])
{
    const V zero = splat<V>(0), one = splat<V>(1), half = splat<V>(S(0.5));

    const V w = rcp(L.sr + R.sr);
    const V rh = L.sr * R.sr;
    const V uh = vfma(L.sr, L.un, R.sr * R.un) * w;
    const V vh = vfma(L.sr, L.ut, R.sr * R.ut) * w;
    const V wh = vfma(L.sr, L.uw, R.sr * R.uw) * w;
    const V Hh = vfma(L.sr, L.H, R.sr * R.H) * w;
    const V du = R.un - L.un, dv = R.ut - L.ut, dw = R.uw - L.uw;
    const V dq2 = vfma(du, du, vfma(dv, dv, dw * dw));
    const V c2h = vfma(vfma(L.sr, L.c2, R.sr * R.c2), w, splat<V>(K.hgm1) * rh * w * w * dq2);
    const V chi = rsq(c2h);
    const V ch = c2h * chi;
    const V aU = vabs(uh);

    const V M = half * (L.Mq + R.Mq);
    const V Mb = aU * chi;
    const V fM = fmach(M), fMb = fmach(Mb);
    const V fM8 = pow8(fM), fMb8 = pow8(fMb);
    const V dp = R.p - L.p;

    const V br = bracket(aU, ch);
    const V Up = vmx(vfma(splat<V>(S(-0.25)) * fMb * br, vmx(du, zero), aU), zero);   // du <= 0 leaves |U|

    const V xfh = xi_form ? half : vfma(splat<V>(S(-0.5)), fMb8, half);   // [1 - f^8(Mbar)] / 2
    V xi = vmx(vfma(xfh, du, vabs(half * (L.un + R.un))), zero);
    if (eps1) {
        const V dq = sqrt0(dq2);
        const auto big = ge(dq, splat<V>(K.rr_thr));
        const V dqi = rcp(sel(big, dq, one));
        const V n1x = sel(big, du * dqi, one);
        const V U1 = sel(big, vfma(du, uh, vfma(dv, vh, dw * wh)) * dqi, uh);
        const V frr = vabs(n1x * U1) + vabs(vfma(-n1x, U1, uh));
        xi = vmx(xi, (one - fMb8) * fM8 * vmn(splat<V>(K.eps2) * ch, frr));
    }

    const V mn = vmn(Up, ch);
    const V smc = vcopysign(mn, uh) * chi;
    const V pp = vfma(smc, dp, (one - s1 + s1 * fM) * vmx(ch - Up, zero) * rh * du);
    const V th = vmn(vmx(splat<V>(K.mr2), M * M), one);
    const V om = one - th;
    const V ou = om * uh;
    const V X = vfma(ou, ou, (splat<V>(4) * c2h) * th);
    const V rX = rsq(X);
    const V ct = half * X * rX;
    const V aUt = vfma(half, th, half) * aU;   // |U~| = (1 + theta) |U| / 2
    const V term = vfma(om, Up - aU * rX * vmn(aUt, ct), vmx(ct - Up, zero));
    const V nA = s1 * (fM8 - one) * term * dp * chi * chi * rcp(th);   // -rho delta U_p
    const V dUu = half * smc * du;

    // Eq. 85 per side (as in roeam_flux2): rho_side (U_side +- xi - dUu) times the side's
    // (1, U, V, W, H, k), plus the pressure and delta U_p terms.
    const V gL = L.r * (L.un + (xi - dUu)), gR = R.r * (R.un - (xi + dUu));
    F[0] = (gL + gR) + nA;
    F[1] = vfma(gL, L.un, vfma(gR, R.un, vfma(nA, uh, L.p + R.p) - pp));
    F[2] = vfma(gL, L.ut, vfma(gR, R.ut, nA * vh));
    F[3] = vfma(gL, L.uw, vfma(gR, R.uw, nA * wh));
    F[4] = vfma(gL, L.H, vfma(gR, R.H, nA * Hh));
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const V kh = vfma(L.sr, L.k[s], R.sr * R.k[s]) * w;
        F[5 + s] = vfma(gL, L.k[s], vfma(gR, R.k[s], nA * kh));
    }
}

// Flux through a Cartesian face along `axis`, times area/2, in global components.
template <typename T, int NS>
__device__ __forceinline__ void face3(const C3<T, NS> &a, const C3<T, NS> &b, int axis, T s1, T area,
                                      const GridCoef3<T> &K, int eps1, int xi_form, T F[5 + NS])
{
    T G2[5 + NS];
    roeam_flux3<T, T, NS>(side3(a, axis), side3(b, axis), s1, K, eps1, xi_form, G2);
    const T h = T(0.5) * area;
    F[0] = h * G2[0];
    F[4] = h * G2[4];
    if (axis == 0) { F[1] = h * G2[1]; F[2] = h * G2[2]; F[3] = h * G2[3]; }
    else if (axis == 1) { F[1] = h * G2[2]; F[2] = h * G2[1]; F[3] = h * G2[3]; }
    else { F[1] = h * G2[2]; F[2] = h * G2[3]; F[3] = h * G2[1]; }
#pragma unroll
    for (int s = 0; s < NS; ++s) F[5 + s] = h * G2[5 + s];
}

// The x-face (Lx | B) and the y-face (Ly | B) of one cell together in packed FP32.
template <int NS>
__device__ __forceinline__ void faces3_xy(const C3<float, NS> &Lx, const C3<float, NS> &Ly, const C3<float, NS> &B,
                                          float s1x, float s1y, const GridCoef3<float> &K, int eps1, int xi_form,
                                          float Fx[5 + NS], float Fy[5 + NS])
{
    V2 G2[5 + NS];
    roeam_flux3<V2, float, NS>(side3_xy(Lx, Ly), side3_xy(B, B), mk2(s1x, s1y), K, eps1, xi_form, G2);
    const float hx = 0.5f * K.ax, hy = 0.5f * K.ay;
    Fx[0] = hx * G2[0].v.x; Fx[1] = hx * G2[1].v.x; Fx[2] = hx * G2[2].v.x; Fx[3] = hx * G2[3].v.x;
    Fx[4] = hx * G2[4].v.x;
    Fy[0] = hy * G2[0].v.y; Fy[1] = hy * G2[2].v.y; Fy[2] = hy * G2[1].v.y; Fy[3] = hy * G2[3].v.y;
    Fy[4] = hy * G2[4].v.y;
#pragma unroll
    for (int s = 0; s < NS; ++s) { Fx[5 + s] = hx * G2[5 + s].v.x; Fy[5 + s] = hy * G2[5 + s].v.y; }
}

template <typename T> __device__ __forceinline__ T min9(T a, T b, T c, T d, T e, T f, T g, T h, T i)
{
    return fmn3(fmn3(a, b, c), fmn3(d, e, f), fmn3(g, h, i));   // (positive ratios, never NaN)
}

// Velocity, |q|^2 and pressure of a conserved 3D state, with explicit rounding (the stage
// epilogue's positivity check and the time-step rate share them).
template <typename T> struct Prims3 { T ri, u, v, w, q2, p; };
template <typename T>
__device__ __forceinline__ Prims3<T> cell_prims3(T r, T ru, T rv, T rw, T rE, const GridCoef3<T> &K)
{
    Prims3<T> s;
    s.ri = rcp(r);
    s.u = rmul(ru, s.ri); s.v = rmul(rv, s.ri); s.w = rmul(rw, s.ri);
    s.q2 = radd(radd(rmul(s.u, s.u), rmul(s.v, s.v)), rmul(s.w, s.w));
    s.p = rmul(K.gm1, rsub(rE, rmul(rmul(T(0.5), r), s.q2)));
    return s;
}

// Time-step rate of one 3D cell (the 2D rule with three directions; theta shared).
template <typename T>
__device__ __forceinline__ T cell_rate3(const Prims3<T> &s, const GridCoef3<T> &K)
{
    const T c2 = rmul(rmul(K.g, s.p), s.ri);
    const T c = sqrt0(c2);
    const T th = vmin(vmax(K.mr2, rmul(s.q2, rcp(c2))), T(1));
    T wx = c, wy = c, wz = c;
    if (th < T(1)) {
        const T om = rsub(T(1), th), ith = rcp(th);
        const T a = rmul(rmul(T(4), c2), th), o2 = rmul(om, om);
        wx = vmax(c, rmul(rmul(T(0.5), sqrt0(radd(a, rmul(o2, rmul(s.u, s.u))))), ith));
        wy = vmax(c, rmul(rmul(T(0.5), sqrt0(radd(a, rmul(o2, rmul(s.v, s.v))))), ith));
        wz = vmax(c, rmul(rmul(T(0.5), sqrt0(radd(a, rmul(o2, rmul(s.w, s.w))))), ith));
    }
    return radd(radd(rmul(radd(vabs(s.u), wx), K.idx), rmul(radd(vabs(s.v), wy), K.idy)),
                rmul(radd(vabs(s.w), wz), K.idz));
}

// Shared-memory exchange of one plane: fields [9 + NS cell values][3 detector values][NV flux
// values], each TY3 x 32, double-buffered by plane parity.
template <typename T, int NS> struct Smem3 {
    static constexpr int NC = 9 + NS, NP = 3, NV = 5 + NS, PER = (NC + NP + NV) * ty3<T>() * 32;
    static __host__ __device__ constexpr size_t bytes() { return sizeof(T) * 2 * (size_t)PER; }
};

// FP32: 16-warp CTAs, one per SM (128 registers); FP64: 8-warp CTAs.
template <typename T, int NS>
__global__ void __launch_bounds__(32 * ty3<T>(), (sizeof(T) == 4 && ty3<T>() <= 8) ? 2 : 1) stage3_kernel(const StageArgs3<T> a)
{
    constexpr int TY3 = ty3<T>();
    using SM = Smem3<T, NS>;
    constexpr int NV = 5 + NS, NC = SM::NC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int ys = wy > 0 ? wy - 1 : 0, yn = wy < TY3 - 1 ? wy + 1 : TY3 - 1;   // clamped neighbour rows
    const int le = lane < 31 ? lane + 1 : 31;
    auto at = [&](int buf, int f, int row, int col) -> T & {
        return sm[(size_t)buf * SM::PER + ((size_t)f * TY3 + row) * 32 + col];
    };

    if (a.rate_zero && blockIdx.x == 0)
        for (int g = threadIdx.x; g < a.ngrids; g += blockDim.x) a.rate_zero[g] = 0ull;

    for (int u = blockIdx.x; u < a.nunits; u += gridDim.x) {
        const int4 unit = a.units[u];
        const int g = unit.x;
        const int i = unit.y - 1 + lane, j = unit.z - 1 + wy;
        const int k0 = unit.w & 0xffff, k1 = unit.w >> 16;
        const GridDev3 &G = a.grids[g];
        const GridCoef3<T> K = a.coef[g];
        const T *src = a.src + G.off;
        const T *un = a.un + G.off;
        T *dst = a.dst + G.off;
        const long long vol = G.vol;
        const int ni = G.ni, nj = G.nj, nk = G.nk, pitch = G.pitch;
        int kx, ky;
        const int isrc = resolve_index(i, ni, G.bc[0], G.bc[1], kx);
        const int jsrc = resolve_index(j, nj, G.bc[2], G.bc[3], ky);
        const bool inflow_xy = kx == 2 || ky == 2;
        const long long xy = (long long)jsrc * pitch + isrc;
        const bool out_cell = lane >= 1 && lane <= 30 && wy >= 1 && wy <= TY3 - 2 && i < ni && j < nj;
        const int eps1 = G.eps1, xi_form = G.xi_form;
        const bool use_s1 = G.use_s1 != 0;
        T dt = T(0);
        if (a.mode == MODE_STAGE) dt = a.dt_fixed_t > T(0) ? a.dt_fixed_t : a.cfl_t / rate_value<T>(__ldg(a.rate_rd + g));
        const bool stage_mode = a.mode == MODE_STAGE;
        const bool combine = stage_mode && a.alpha != T(0);

        // window: planes k-1 (Wm), k (W0), k+1 (Wp); loads of k+2 in flight
        C3<T, NS> Wm, W0, Wp;
        Pend3<T, NS> pend;
        {
            int kk;
            int ks = resolve_index(k0 - 1, nk, G.bc[4], G.bc[5], kk);
            issue3<T, NS>(src, vol, xy, pitch, nj, ks, kk, inflow_xy, pend);
            finish3<T, NS>(pend, inflow_xy, kx, ky, K, Wm);
            ks = resolve_index(k0, nk, G.bc[4], G.bc[5], kk);
            issue3<T, NS>(src, vol, xy, pitch, nj, ks, kk, inflow_xy, pend);
            finish3<T, NS>(pend, inflow_xy, kx, ky, K, W0);
            ks = resolve_index(k0 + 1, nk, G.bc[4], G.bc[5], kk);
            issue3<T, NS>(src, vol, xy, pitch, nj, ks, kk, inflow_xy, pend);
            finish3<T, NS>(pend, inflow_xy, kx, ky, K, Wp);
            ks = resolve_index(k0 + 2, nk, G.bc[4], G.bc[5], kk);
            issue3<T, NS>(src, vol, xy, pitch, nj, ks, kk, inflow_xy, pend);
        }
        // detector values of plane k0 - 1 (x and y faces), for the first z-face
        T Px_m, Pxe_m, Py_m, Pyn_m;
        {
            // (through the buffer of plane k0 - 1's parity: plane k0 writes the other one)
            const int bp = (k0 + 1) & 1;
            Px_m = ratio_P(shup(Wm.r, 1), shup(Wm.p, 1), Wm.r, Wm.p);
            Pxe_m = shdn(Px_m, 1);
            __syncthreads();   // the previous unit's readers are done with both buffers
            at(bp, 0, wy, lane) = Wm.r;
            at(bp, 4, wy, lane) = Wm.p;
            __syncthreads();
            Py_m = ratio_P(at(bp, 0, ys, lane), at(bp, 4, ys, lane), Wm.r, Wm.p);
            Pyn_m = ratio_P(Wm.r, Wm.p, at(bp, 0, yn, lane), at(bp, 4, yn, lane));
        }
        T acc[NV];
        T Un[NV];
        T my_rate = T(0);
        T Pz_carry = ratio_P(Wm.r, Wm.p, W0.r, W0.p);   // bottom z-face of plane k0

        for (int k = k0; k <= k1; ++k) {
            const int b = k & 1;
            // U^n of plane k for the combination at the next iteration
            T Un_next[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) Un_next[v] = T(0);
            if (combine && out_cell && k < k1) {
                const long long x = (long long)k * nj * pitch + (long long)j * pitch + i;
#pragma unroll
                for (int v = 0; v < NV; ++v) Un_next[v] = un[x + v * vol];
            }

            // detector values of plane k known to this thread
            const T Px = ratio_P(shup(W0.r, 1), shup(W0.p, 1), W0.r, W0.p);   // west x-face
            const T Pxe = shdn(Px, 1);                                        // east x-face
            const T Pz = Pz_carry;                                            // bottom z-face
            const T Pzt = ratio_P(W0.r, W0.p, Wp.r, Wp.p);                    // top z-face

            // exchange plane k with the rows above and below
            at(b, 0, wy, lane) = W0.r; at(b, 1, wy, lane) = W0.u; at(b, 2, wy, lane) = W0.v;
            at(b, 3, wy, lane) = W0.w; at(b, 4, wy, lane) = W0.p; at(b, 5, wy, lane) = W0.c2;
            at(b, 6, wy, lane) = W0.H; at(b, 7, wy, lane) = W0.sr; at(b, 8, wy, lane) = W0.Mq;
#pragma unroll
            for (int s = 0; s < NS; ++s) at(b, 9 + s, wy, lane) = W0.k[s];
            at(b, NC, wy, lane) = Px;
            at(b, NC + 1, wy, lane) = Pz;
            at(b, NC + 2, wy, lane) = Pzt;
            __syncthreads();
            // the north neighbour's south flux of plane k - 1 (written after the previous barrier)
            if (k > k0) {
#pragma unroll
                for (int v = 0; v < NV; ++v) acc[v] -= at(b ^ 1, NC + 3 + v, yn, lane);
            }
            C3<T, NS> S;   // the cell below (row j - 1)
            S.r = at(b, 0, ys, lane); S.u = at(b, 1, ys, lane); S.v = at(b, 2, ys, lane); S.w = at(b, 3, ys, lane);
            S.p = at(b, 4, ys, lane); S.c2 = at(b, 5, ys, lane); S.H = at(b, 6, ys, lane); S.sr = at(b, 7, ys, lane);
            S.Mq = at(b, 8, ys, lane);
#pragma unroll
            for (int s = 0; s < NS; ++s) S.k[s] = at(b, 9 + s, ys, lane);
            const T Py = ratio_P(S.r, S.p, W0.r, W0.p);
            const T Pyn = ratio_P(W0.r, W0.p, at(b, 0, yn, lane), at(b, 4, yn, lane));

            // s1 of the three faces (Eq. 96: the face and the 8 transverse faces of its cells)
            T s1x = T(1), s1y = T(1), s1z = T(1);
            if (use_s1) {
                const T ax = min9(Px, shup(Py, 1), shup(Pyn, 1), Py, Pyn, shup(Pz, 1), shup(Pzt, 1), Pz, Pzt);
                const T ay = min9(Py, at(b, NC, ys, lane), at(b, NC, ys, le), Px, Pxe, at(b, NC + 1, ys, lane),
                                  at(b, NC + 2, ys, lane), Pz, Pzt);
                const T az = min9(Pz, Px_m, Pxe_m, Px, Pxe, Py_m, Pyn_m, Py, Pyn);
                if constexpr (sizeof(T) == 4) {
                    const V2 sxy = detector_of(mk2(ax, ay));
                    s1x = sxy.v.x; s1y = sxy.v.y;
                } else {
                    s1x = detector_of(ax);
                    s1y = detector_of(ay);
                }
                s1z = detector_of(az);
            }

            // the three faces of this cell
            C3<T, NS> Wl;   // the cell to the west (lane - 1)
            Wl.r = shup(W0.r, 1); Wl.u = shup(W0.u, 1); Wl.v = shup(W0.v, 1); Wl.w = shup(W0.w, 1);
            Wl.p = shup(W0.p, 1); Wl.c2 = shup(W0.c2, 1); Wl.H = shup(W0.H, 1); Wl.sr = shup(W0.sr, 1);
            Wl.Mq = shup(W0.Mq, 1);
#pragma unroll
            for (int s = 0; s < NS; ++s) Wl.k[s] = shup(W0.k[s], 1);
            // (the halo rows need none of their faces but the top row's south face; FP32 evaluates
            //  the x- and y-faces together as packed pairs)
            T Fw[NV], Fs[NV], Fb[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) Fw[v] = Fs[v] = Fb[v] = T(0);
            if constexpr (sizeof(T) == 4) {
                if (wy > 0) faces3_xy<NS>(Wl, S, W0, s1x, s1y, K, eps1, xi_form, Fw, Fs);
            } else {
                if (wy > 0) face3<T, NS>(S, W0, 1, s1y, K.ay, K, eps1, xi_form, Fs);
                if (wy > 0 && wy < TY3 - 1) face3<T, NS>(Wl, W0, 0, s1x, K.ax, K, eps1, xi_form, Fw);
            }
            // U^(k) of plane k - 1 for the epilogue, issued before the z-face in FP32 (its latency
            // then hides behind the z-face: 18.8 -> 19.3 Gcell-updates/s per stage on the 256^3
            // Taylor-Green vortex, and fewer spills); FP64 reads it in the epilogue
            T Uk[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) Uk[v] = T(0);
            if (sizeof(T) == 4 && stage_mode && out_cell && k > k0) {
                const long long x = (long long)(k - 1) * nj * pitch + (long long)j * pitch + i;
#pragma unroll
                for (int v = 0; v < NV; ++v) Uk[v] = __ldg(src + x + v * vol);
            }
            if (wy > 0 && wy < TY3 - 1) face3<T, NS>(Wm, W0, 2, s1z, K.az, K, eps1, xi_form, Fb);

            // this plane's south flux, read by the row below after the next plane's barrier
#pragma unroll
            for (int v = 0; v < NV; ++v) at(b, NC + 3 + v, wy, lane) = Fs[v];

            // finish plane k - 1: R = (acc - F_top) / V, then the stage combination
            if (k > k0 && out_cell) {
                T Rs[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) Rs[v] = (acc[v] - Fb[v]) * K.Vi;
                const long long x = (long long)(k - 1) * nj * pitch + (long long)j * pitch + i;
                if (stage_mode) {
                    T out[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        const T uk = sizeof(T) == 4 ? Uk[v] : __ldg(src + x + v * vol);
                        const T upd = uk + dt * Rs[v];
                        out[v] = combine ? a.alpha * Un[v] + a.beta * upd : upd;
                    }
#pragma unroll
                    for (int v = 0; v < NV; ++v) dst[x + v * vol] = out[v];
                    if (a.want_rate) {
                        const Prims3<T> cp = cell_prims3(out[0], out[1], out[2], out[3], out[4], K);
                        if (!(out[0] > T(0)) || !(cp.p > T(0))) {
                            const bool fin = isfinite((double)out[0]) && isfinite((double)cp.p);
                            atomicOr(a.status, fin ? ST_NONPOSITIVE : ST_NONFINITE);
                        } else {
                            my_rate = vmax(my_rate, cell_rate3(cp, K));
                        }
                    } else {
                        // p > 0 without the division: 2 rho (rho E) > |rho q|^2; a cell that fails
                        // it (rare: also products beyond the FP32 range) is decided by its pressure
                        const T e2 = T(2) * out[0] * out[4];
                        const T m2 = out[1] * out[1] + out[2] * out[2] + out[3] * out[3];
                        if (!(out[0] > T(0)) || !(e2 > m2)) {
                            const Prims3<T> cp = cell_prims3(out[0], out[1], out[2], out[3], out[4], K);
                            if (!(out[0] > T(0)) || !(cp.p > T(0))) {
                                const bool fin = isfinite((double)out[0]) && isfinite((double)cp.p);
                                atomicOr(a.status, fin ? ST_NONPOSITIVE : ST_NONFINITE);
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < NV; ++v) dst[x + v * vol] = Rs[v];
                }
            }
            if (k == k1) break;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                Un[v] = Un_next[v];
                acc[v] = Fw[v] - shdn(Fw[v], 1) + Fs[v] + Fb[v];
            }

            // advance the window
            Px_m = Px; Pxe_m = Pxe; Py_m = Py; Pyn_m = Pyn;
            Pz_carry = Pzt;   // the top z-face of plane k is the bottom one of plane k + 1
            Wm = W0;
            W0 = Wp;
            finish3<T, NS>(pend, inflow_xy, kx, ky, K, Wp);
            int kk;
            const int ks = resolve_index(k + 3, nk, G.bc[4], G.bc[5], kk);
            issue3<T, NS>(src, vol, xy, pitch, nj, ks, kk, inflow_xy, pend);
        }
        if (a.want_rate) {
            for (int o = 16; o > 0; o >>= 1) my_rate = vmax(my_rate, __shfl_xor_sync(0xffffffffu, my_rate, o));
            if (lane == 0 && my_rate > T(0)) atomicMax(a.rate_wr + g, rate_bits(my_rate));
        }
    }
}

// Largest rate over every cell of grids [g_lo, g_hi) (blockIdx.y = grid).
template <typename T>
__global__ void __launch_bounds__(256) rate3_kernel(const GridDev3 *grids, const GridCoef3<T> *coef, int g_lo,
                                                    const T *U, unsigned long long *rate)
{
    __shared__ T red[8];
    const int g = g_lo + blockIdx.y;
    const GridDev3 &G = grids[g];
    const GridCoef3<T> K = coef[g];
    const long long n = (long long)G.ni * G.nj * G.nk;
    T m = T(0);
    for (long long q = (long long)blockIdx.x * 256 + threadIdx.x; q < n; q += (long long)gridDim.x * 256) {
        const long long i = q % G.ni, jk = q / G.ni;
        const long long c = G.off + jk * G.pitch + i;
        m = vmax(m, cell_rate3(cell_prims3(U[c], U[c + G.vol], U[c + 2 * G.vol], U[c + 3 * G.vol], U[c + 4 * G.vol], K),
                               K));
    }
    m = block_max<256>(m, red);
    if (threadIdx.x == 0 && m > T(0)) atomicMax(rate + g, rate_bits(m));
}

template <typename T>
__global__ void __launch_bounds__(256) pack3_kernel(const GridDev3 *grids, int g_lo, int nv, const double *packed, T *U)
{
    const GridDev3 &G = grids[g_lo + blockIdx.y];
    const long long n = (long long)G.ni * G.nj * G.nk;
    for (long long q = (long long)blockIdx.x * 256 + threadIdx.x; q < n; q += (long long)gridDim.x * 256) {
        const long long c = G.off + (q / G.ni) * G.pitch + q % G.ni;
        for (int v = 0; v < nv; ++v) U[c + v * G.vol] = T(packed[G.poff + v * n + q]);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) unpack3_kernel(const GridDev3 *grids, int g_lo, int nv, const T *U, double *packed)
{
    const GridDev3 &G = grids[g_lo + blockIdx.y];
    const long long n = (long long)G.ni * G.nj * G.nk;
    for (long long q = (long long)blockIdx.x * 256 + threadIdx.x; q < n; q += (long long)gridDim.x * 256) {
        const long long c = G.off + (q / G.ni) * G.pitch + q % G.ni;
        for (int v = 0; v < nv; ++v) packed[G.poff + v * n + q] = (double)U[c + v * G.vol];
    }
}

// FP64 block partials of sum V Q over grid g (gridDim.x x MAX_VARS3 doubles).
template <typename T>
__global__ void __launch_bounds__(256) totals3_kernel(const GridDev3 *grids, int g, const T *U, int nv, double *partials)
{
    __shared__ double wred[8][MAX_VARS3];
    const GridDev3 &G = grids[g];
    const long long n = (long long)G.ni * G.nj * G.nk;
    const double V = G.dx * G.dy * G.dz;
    double s[MAX_VARS3];
    for (int v = 0; v < MAX_VARS3; ++v) s[v] = 0.0;
    for (long long q = (long long)blockIdx.x * 256 + threadIdx.x; q < n; q += (long long)gridDim.x * 256) {
        const long long c = G.off + (q / G.ni) * G.pitch + q % G.ni;
        for (int v = 0; v < nv; ++v) s[v] += V * (double)U[c + v * G.vol];
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int v = 0; v < MAX_VARS3; ++v) s[v] += __shfl_xor_sync(0xffffffffu, s[v], o);
    if ((threadIdx.x & 31) == 0)
        for (int v = 0; v < MAX_VARS3; ++v) wred[threadIdx.x >> 5][v] = s[v];
    __syncthreads();
    if (threadIdx.x < MAX_VARS3) {
        double r = 0.0;
        for (int w = 0; w < 8; ++w) r += wred[w][threadIdx.x];
        partials[(size_t)blockIdx.x * MAX_VARS3 + threadIdx.x] = r;
    }
}

// ------------------------------------------------------------------ launchers
template <typename T, int NS> struct Stage3Variant {
    static cudaError_t launch(const StageArgs3<T> &a, int nblocks, cudaStream_t s)
    {
        // (per device and cheap, so set on every launch)
        cudaError_t e = cudaFuncSetAttribute(stage3_kernel<T, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Smem3<T, NS>::bytes());
        if (e != cudaSuccess) return e;
        stage3_kernel<T, NS><<<nblocks, 32 * ty3<T>(), Smem3<T, NS>::bytes(), s>>>(a);
        return cudaGetLastError();
    }
    static int occupancy()
    {
        cudaFuncSetAttribute(stage3_kernel<T, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Smem3<T, NS>::bytes());
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage3_kernel<T, NS>, 32 * ty3<T>(), Smem3<T, NS>::bytes()) !=
            cudaSuccess)
            return 1;
        return n > 0 ? n : 1;
    }
};

template <typename T>
cudaError_t Launchers3<T>::stage(const StageArgs3<T> &a, int nscal, int nblocks, cudaStream_t s)
{
    if (a.nunits <= 0) return cudaSuccess;
    switch (nscal) {
    case 0: return Stage3Variant<T, 0>::launch(a, nblocks, s);
    case 1: return Stage3Variant<T, 1>::launch(a, nblocks, s);
    case 2: return Stage3Variant<T, 2>::launch(a, nblocks, s);
    default: return Stage3Variant<T, 3>::launch(a, nblocks, s);
    }
}

template <typename T>
int Launchers3<T>::stage_occupancy(int nscal)
{
    switch (nscal) {
    case 0: return Stage3Variant<T, 0>::occupancy();
    case 1: return Stage3Variant<T, 1>::occupancy();
    case 2: return Stage3Variant<T, 2>::occupancy();
    default: return Stage3Variant<T, 3>::occupancy();
    }
}

template <typename T>
cudaError_t Launchers3<T>::rate(const GridDev3 *grids, const GridCoef3<T> *coef, int g_lo, int g_hi, const T *U,
                                int nscal, unsigned long long *rate, cudaStream_t s)
{
    (void)nscal;
    if (g_hi <= g_lo) return cudaSuccess;
    rate3_kernel<T><<<dim3(64, g_hi - g_lo), 256, 0, s>>>(grids, coef, g_lo, U, rate);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launchers3<T>::pack(const GridDev3 *grids, int g_lo, int g_hi, int nv, long long max_cells,
                                const double *packed, T *U, cudaStream_t s)
{
    if (g_hi <= g_lo) return cudaSuccess;
    long long bx = (max_cells + 255) / 256;
    bx = bx < 1 ? 1 : (bx > 1024 ? 1024 : bx);
    pack3_kernel<T><<<dim3((unsigned)bx, g_hi - g_lo), 256, 0, s>>>(grids, g_lo, nv, packed, U);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launchers3<T>::unpack(const GridDev3 *grids, int g_lo, int g_hi, int nv, long long max_cells, const T *U,
                                  double *packed, cudaStream_t s)
{
    if (g_hi <= g_lo) return cudaSuccess;
    long long bx = (max_cells + 255) / 256;
    bx = bx < 1 ? 1 : (bx > 1024 ? 1024 : bx);
    unpack3_kernel<T><<<dim3((unsigned)bx, g_hi - g_lo), 256, 0, s>>>(grids, g_lo, nv, U, packed);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launchers3<T>::totals(const GridDev3 *grids, int g, const T *U, int nv, double *partials, int nblocks,
                                  cudaStream_t s)
{
    totals3_kernel<T><<<nblocks, 256, 0, s>>>(grids, g, U, nv, partials);
    return cudaGetLastError();
}

}  // namespace roeam
