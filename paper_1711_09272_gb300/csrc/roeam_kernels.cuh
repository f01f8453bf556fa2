// roeam_kernels.cuh — sm_103a kernels of the Roe-AM finite-volume step.
//
// The stage kernel evaluates a whole Runge-Kutta stage: face fluxes of Section 6.2
// (Eqs. 85-109), the finite-volume residual, and the SSP-RK3 combination, in one pass
// over the state. Its work unit is one warp sweeping a strip of 32 columns (H halo lanes
// on each side, H = 1 at first order, 2 with MUSCL) over a segment of rows in +j:
//   - each lane keeps a rolling window of H+2 rows of its column in registers and
//     prefetches the next row while it computes the current one, so every cell state is
//     read from HBM once per stage (plus halo lanes and H+1 warm-up rows per segment);
//   - neighbour states, detector ratios and fluxes move between lanes with warp shuffles:
//     no shared memory and no block barrier;
//   - ghost cells come from the boundary conditions on the fly (periodic wrap, wall
//     mirror, inflow state, zero-gradient outflow), so no separate boundary kernel runs;
//   - the flux is evaluated in the face frame (normal velocity first), which makes the
//     Cartesian x- and y-faces the same computation; in FP32 a lane evaluates its west
//     x-face and its south y-face together as packed float2 arithmetic (FFMA2, FADD2,
//     FMUL2 on sm_100-class GPUs).
#pragma once

#include <cstdint>

#include "roeam_internal.h"

namespace roeam {

__device__ __forceinline__ int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

// ------------------------------------------------------------------ math on scalars and pairs
// V is float, double, or V2 (two floats evaluated as one packed pair). Comparisons give a
// mask (bool, or B2 for pairs); sel(mask, a, b) picks per component.
struct V2 { float2 v; };
struct B2 { bool x, y; };

__device__ __forceinline__ V2 mk2(float a, float b) { V2 r; r.v = make_float2(a, b); return r; }
__device__ __forceinline__ V2 operator+(V2 a, V2 b) { V2 r; r.v = __fadd2_rn(a.v, b.v); return r; }
__device__ __forceinline__ V2 operator*(V2 a, V2 b) { V2 r; r.v = __fmul2_rn(a.v, b.v); return r; }
__device__ __forceinline__ V2 operator-(V2 a, V2 b) { V2 r; r.v = __ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v); return r; }
__device__ __forceinline__ V2 operator-(V2 a) { return mk2(-a.v.x, -a.v.y); }
__device__ __forceinline__ V2 vfma(V2 a, V2 b, V2 c) { V2 r; r.v = __ffma2_rn(a.v, b.v, c.v); return r; }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
// c - a b: one fused operation on scalars; on pairs the product and the packed subtraction.
__device__ __forceinline__ float vfnma(float a, float b, float c) { return fmaf(-a, b, c); }
__device__ __forceinline__ double vfnma(double a, double b, double c) { return fma(-a, b, c); }
__device__ __forceinline__ V2 vfnma(V2 a, V2 b, V2 c) { return c - a * b; }

template <typename V> struct Sc;
template <> struct Sc<float> { using S = float; using M = bool; };
template <> struct Sc<double> { using S = double; using M = bool; };
template <> struct Sc<V2> { using S = float; using M = B2; };

template <typename V> __device__ __forceinline__ V splat(typename Sc<V>::S c) { return V(c); }
template <> __device__ __forceinline__ V2 splat<V2>(float c) { return mk2(c, c); }

template <typename T> __device__ __forceinline__ T vmin(T a, T b) { return a < b ? a : b; }
template <typename T> __device__ __forceinline__ T vmax(T a, T b) { return a > b ? a : b; }
__device__ __forceinline__ V2 vmin(V2 a, V2 b) { return mk2(fminf(a.v.x, b.v.x), fminf(a.v.y, b.v.y)); }
__device__ __forceinline__ V2 vmax(V2 a, V2 b) { return mk2(fmaxf(a.v.x, b.v.x), fmaxf(a.v.y, b.v.y)); }
// Minimum and maximum as single instructions (the a < b ? a : b forms above must keep their
// NaN and signed-zero behaviour, which costs a compare and a select). For the positive ratios
// of the detector, whose operands are never NaN, the results are the same; the three-operand
// minimum is one instruction on sm_100-class GPUs.
__device__ __forceinline__ float fmn(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double fmn(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float fmx(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double fmx(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float fmn3(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ double fmn3(double a, double b, double c) { return fmin(fmin(a, b), c); }
// Minimum and maximum inside the flux, whose operands are finite: single instructions for
// every operand type (the V2 forms above already are).
__device__ __forceinline__ float vmn(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double vmn(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ V2 vmn(V2 a, V2 b) { return vmin(a, b); }
__device__ __forceinline__ float vmx(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double vmx(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ V2 vmx(V2 a, V2 b) { return vmax(a, b); }
// 1 where a < b (a <= b), else 0, as one instruction each (PTX set).
__device__ __forceinline__ float setlt(float a, float b) { float r; asm("set.lt.f32.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b)); return r; }
__device__ __forceinline__ float setle(float a, float b) { float r; asm("set.le.f32.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b)); return r; }
__device__ __forceinline__ float vabs(float a) { return fabsf(a); }
__device__ __forceinline__ double vabs(double a) { return fabs(a); }
__device__ __forceinline__ V2 vabs(V2 a) { return mk2(fabsf(a.v.x), fabsf(a.v.y)); }

template <typename T> __device__ __forceinline__ bool lt(T a, T b) { return a < b; }
template <typename T> __device__ __forceinline__ bool gt(T a, T b) { return a > b; }
template <typename T> __device__ __forceinline__ bool ge(T a, T b) { return a >= b; }
template <typename T> __device__ __forceinline__ bool eq(T a, T b) { return a == b; }
__device__ __forceinline__ B2 lt(V2 a, V2 b) { return {a.v.x < b.v.x, a.v.y < b.v.y}; }
__device__ __forceinline__ B2 gt(V2 a, V2 b) { return {a.v.x > b.v.x, a.v.y > b.v.y}; }
__device__ __forceinline__ B2 ge(V2 a, V2 b) { return {a.v.x >= b.v.x, a.v.y >= b.v.y}; }
__device__ __forceinline__ B2 eq(V2 a, V2 b) { return {a.v.x == b.v.x, a.v.y == b.v.y}; }
__device__ __forceinline__ B2 operator&&(B2 a, B2 b) { return {a.x && b.x, a.y && b.y}; }
template <typename T> __device__ __forceinline__ T sel(bool m, T a, T b) { return m ? a : b; }
__device__ __forceinline__ V2 sel(B2 m, V2 a, V2 b) { return mk2(m.x ? a.v.x : b.v.x, m.y ? a.v.y : b.v.y); }

// The 2D kernel translation units compile with -fmad=false: every fused multiply-add is
// written out (vfma, vfnma), so a value comes out bit for bit the same wherever it is
// evaluated (in a loop's prologue or body, in either copy of an unrolled body, in any work-unit
// layout), and results do not depend on the tile shape or on how a grid is split into slabs.

// Reciprocal, reciprocal square root and square root (of a non-negative value). FP32 uses
// the single-instruction hardware approximations (PTX rcp/rsqrt/sqrt .approx). FP64 starts
// from the hardware approximations (PTX rcp.approx.ftz.f64, rsqrt.approx.ftz.f64) and refines
// them by two Newton-Raphson steps, each of which squares the relative error (y <- y + y e
// with e = 1 - x y for 1/x, y <- y + y e / 2 with e = 1 - x y^2 for 1/sqrt(x)): within two
// ulp of the correctly rounded results for the positive normal arguments the scheme produces
// (roeam_math_check compares them with the IEEE operations), at a fraction of their cost.
__device__ __forceinline__ float rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsq(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt0(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp(double x)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}
__device__ __forceinline__ double rsq(double x)
{
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x * y, y, 1.0);
    y = fma(0.5 * y, e, y);
    e = fma(-x * y, y, 1.0);
    return fma(0.5 * y, e, y);
}
__device__ __forceinline__ double sqrt0(double x) { return x > 0.0 ? x * rsq(x) : 0.0; }
__device__ __forceinline__ V2 rcp(V2 x) { return mk2(rcp(x.v.x), rcp(x.v.y)); }
__device__ __forceinline__ V2 rsq(V2 x) { return mk2(rsq(x.v.x), rsq(x.v.y)); }
__device__ __forceinline__ V2 sqrt0(V2 x) { return mk2(sqrt0(x.v.x), sqrt0(x.v.y)); }

// copysign(a, b): magnitude of a, sign of b.
__device__ __forceinline__ float vcopysign(float a, float b) { return copysignf(a, b); }
__device__ __forceinline__ double vcopysign(double a, double b) { return copysign(a, b); }
__device__ __forceinline__ V2 vcopysign(V2 a, V2 b) { return mk2(copysignf(a.v.x, b.v.x), copysignf(a.v.y, b.v.y)); }

// sgn with sgn(0) = 0.
template <typename V> __device__ __forceinline__ V sgnv(V a)
{
    const V z = splat<V>(0);
    return sel(gt(a, z), splat<V>(1), sel(lt(a, z), splat<V>(-1), z));
}
template <typename V> __device__ __forceinline__ V pow8(V a) { V a2 = a * a, a4 = a2 * a2; return a4 * a4; }

// Eq. 98: f(phi) = min(phi sqrt(4 + (1 - phi^2)^2) / (1 + phi^2), 1). The argument is clamped
// at 2 (f = 1 for every phi >= 1, and the clamp keeps the powers below in range), and the
// square root and the division share one reciprocal square root:
// sqrt(s) / q = s / sqrt(s q^2) with s = 4 + (1 - phi^2)^2, q = 1 + phi^2.
template <typename V> __device__ __forceinline__ V fmach(V phi)
{
    const V one = splat<V>(1);
    const V p = vmn(phi, splat<V>(2));
    const V t = vfnma(p, p, one);
    const V s = vfma(t, t, splat<V>(4));
    const V q = vfma(p, p, one);
    return vmn(p * s * rsq(s * q * q), one);
}

// Eq. 95 (with P values of Eq. 97 already reduced to their minimum a by Eq. 96). The
// argument is a ratio of positive values (at most 1, plus the rounding of a reciprocal), so
// Eq. 98 needs no clamp of its argument here; its result is still clamped at 1.
template <typename V> __device__ __forceinline__ V detector_of(V a)
{
    const V one = splat<V>(1);
    const V t = vfnma(a, a, one);
    const V s = vfma(t, t, splat<V>(4));
    const V q = vfma(a, a, one);
    const V f = vmn(a * s * rsq(s * q * q), one);
    return sel(ge(a, one), one, pow8(f));
}

// Mirror image of a velocity about a unit normal (wall ghost state).
template <typename T> __device__ __forceinline__ void mirror_vel(T &u, T &v, T nx, T ny)
{
    const T un2 = T(2) * vfma(u, nx, v * ny);
    u = vfnma(un2, nx, u);
    v = vfnma(un2, ny, v);
}

// ------------------------------------------------------------------ the Roe-AM flux
// Quantities of one side of a face, in the face frame: un is the velocity along the unit
// normal (from L to R), ut the tangential one. c2 = gamma p / rho, H total enthalpy,
// sr = sqrt(rho), Mq = |q| / c.
template <typename V> struct FS { V r, un, ut, p, c2, H, sr, Mq; };

template <typename V, typename S>
__device__ __forceinline__ FS<V> side_from_prims(V r, V un, V ut, V p, const GridCoef<S> &K)
{
    FS<V> s;
    s.r = r; s.un = un; s.ut = ut; s.p = p;
    const V ri = rcp(r);
    s.c2 = splat<V>(K.g) * p * ri;
    const V q2 = vfma(un, un, ut * ut);
    s.H = vfma(s.c2, splat<V>(K.gm1i), splat<V>(S(0.5)) * q2);
    s.sr = r * rsq(r);
    s.Mq = sqrt0(q2 * rcp(s.c2));
    return s;
}

// The bracket sgn(U + c) - sgn(U - c) of Eq. 92 for |U| and c >= 0: 2 for |U| < c, 1 for
// |U| = c, 0 above (in FP32 as the sum of two set instructions).
__device__ __forceinline__ float bracket(float aU, float c) { return setlt(aU, c) + setle(aU, c); }
__device__ __forceinline__ double bracket(double aU, double c) { return aU < c ? 2.0 : (aU == c ? 1.0 : 0.0); }
__device__ __forceinline__ V2 bracket(V2 aU, V2 c)
{
    return mk2(setlt(aU.v.x, c.v.x), setlt(aU.v.y, c.v.y)) + mk2(setle(aU.v.x, c.v.x), setle(aU.v.y, c.v.y));
}

// Ablation variants of the flux (the schemes Section 7 compares with), read per grid by the
// ablation kernels only: scheme 1 is classical Roe (Eq. 7 with Eqs. 8-12, entropy fix of
// Eqs. 114-115 with GridCoef::harten); for Roe-AM, dup_mode 1 sets delta U_p = 0 and 2 takes
// the Roe term of Eq. 17, ufix = 0 drops Eq. 92, xi_roe = 1 takes xi = |U| (Eq. 13).
struct Variant { int scheme = 0, dup_mode = 0, ufix = 1, xi_roe = 0; };

// Twice the Roe-AM numerical flux per unit face length, in the face frame (components:
// mass, normal momentum, tangential momentum, energy). Section 6.2, term by term:
// central part (Eqs. 3-4), Roe averages, M (Eq. 93), Mbar (Eq. 94), f (Eq. 98), |U|'
// (Eq. 92, clamped at 0), xi (Eq. 86 with the Eq. 68 factor unless xi_form = 1; the eps1
// floor with Eqs. 102-109), delta p_p + delta p_u (Eqs. 87-88), rho delta U_p (Eq. 89 with
// Eqs. 99-101), delta U_u (Eqs. 90-91), assembled as Eq. 85 with the energy convention of
// Eq. 49. With ABL the Variant switches apply (scalar V only).
template <bool ABL = false, typename V, typename S>
__device__ __forceinline__ void roeam_flux2(const FS<V> &L, const FS<V> &R, V s1, const GridCoef<S> &K, int eps1,
                                            int xi_form, V F[4], const Variant &var = Variant())
{
    const V zero = splat<V>(0), one = splat<V>(1), half = splat<V>(S(0.5));

    // Roe averages; c^2 in the sum-of-positives form (no cancellation at high Mach).
    const V w = rcp(L.sr + R.sr);
    const V rh = L.sr * R.sr;
    const V uh = vfma(L.sr, L.un, R.sr * R.un) * w;
    const V vh = vfma(L.sr, L.ut, R.sr * R.ut) * w;
    const V Hh = vfma(L.sr, L.H, R.sr * R.H) * w;
    const V du = R.un - L.un, dv = R.ut - L.ut;
    const V dq2 = vfma(du, du, dv * dv);
    const V c2h = vfma(splat<V>(K.hgm1) * rh * w, dq2, vfma(L.sr, L.c2, R.sr * R.c2)) * w;
    const V chi = rsq(c2h);
    const V ch = c2h * chi;
    const V aU = vabs(uh);

    if constexpr (ABL) {
        if (var.scheme == 1) {
            // Classical Roe: |lambda| = |U|, |U - c|, |U + c|, each raised to (l^2 / h + h) / 2
            // below h = eps_lambda max|lambda| (Eqs. 114-115); xi = l1 (Eq. 8), delta p_u +
            // delta p_p (Eqs. 9-10) and rho (delta U_u + delta U_p) (Eqs. 11-12); the xi term
            // acts on Delta(rho E) = Delta(rho H) - Delta p and the pressure vector carries U
            // in its energy slot.
            V l1 = aU, l4 = vabs(uh - ch), l5 = vabs(uh + ch);
            const V hh = splat<V>(K.harten) * vmx(l1, vmx(l4, l5));
            if (gt(hh, zero)) {
                const V hi = rcp(hh);
                l1 = sel(lt(l1, hh), half * vfma(l1 * l1, hi, hh), l1);
                l4 = sel(lt(l4, hh), half * vfma(l4 * l4, hi, hh), l4);
                l5 = sel(lt(l5, hh), half * vfma(l5 * l5, hi, hh), l5);
            }
            const V mL = L.r * L.un, mR = R.r * R.un;
            const V F0c = mL + mR;
            const V F1c = vfma(mL, L.un, vfma(mR, R.un, L.p + R.p));
            const V F2c = vfma(mL, L.ut, mR * R.ut);
            const V F3c = vfma(mL, L.H, mR * R.H);
            const V dp = R.p - L.p;
            const V spp = vfma(half, l5 + l4, -l1), smm = half * (l5 - l4);
            const V pp = vfma(spp * rh, du, smm * dp * chi);
            const V A = vfma(smm * rh * chi, du, spp * dp * chi * chi);
            const V QL2 = L.r * L.ut, QR2 = R.r * R.ut, QL3 = L.r * L.H, QR3 = R.r * R.H;
            F[0] = F0c - vfma(l1, R.r - L.r, A);
            F[1] = F1c - vfma(l1, mR - mL, vfma(A, uh, pp));
            F[2] = F2c - vfma(l1, QR2 - QL2, A * vh);
            F[3] = F3c - vfma(l1, (QR3 - QL3) - dp, vfma(A, Hh, pp * uh));
            return;
        }
    }

    const V M = half * (L.Mq + R.Mq);
    const V Mb = aU * chi;
    const V fM = fmach(M), fMb = fmach(Mb);
    const V fM8 = pow8(fM), fMb8 = pow8(fMb);
    const V dp = R.p - L.p;

    // |U|': the bracket sgn(U + c) - sgn(U - c) is 2 for |U| < c, 1 for |U| = c, 0 above.
    const V br = bracket(aU, ch);
    // (du <= 0 leaves |U|: the correction is applied to max(du, 0))
    V Up = vmx(vfma(splat<V>(S(-0.25)) * fMb * br, vmx(du, zero), aU), zero);
    if constexpr (ABL) {
        if (!var.ufix) Up = aU;
    }

    // xi's factor [1 - f^8(Mbar)] / 2 on dU (1/2 with xi_form = 1)
    const V xfh = xi_form ? half : vfma(splat<V>(S(-0.5)), fMb8, half);
    V xi = vmx(vfma(xfh, du, vabs(half * (L.un + R.un))), zero);
    if (eps1) {
        // Rotated-Riemann estimate in the face frame (n = (1, 0)): n1 = dq / |dq| unless
        // |dq| < 1e-5 U_ref; |alpha1 U1| + |alpha2 U2| with the unit n2 perpendicular to n1.
        const V dq = sqrt0(dq2);
        const auto big = ge(dq, splat<V>(K.rr_thr));
        const V dqi = rcp(sel(big, dq, one));
        const V n1x = sel(big, du * dqi, one), n1y = sel(big, dv * dqi, zero);
        const V frr = vabs(n1x * vfma(n1x, uh, n1y * vh)) + vabs(n1y * (vfma(n1x, vh, -(n1y * uh))));
        xi = vmx(xi, (one - fMb8) * fM8 * vmn(splat<V>(K.eps2) * ch, frr));
    }
    if constexpr (ABL) {
        if (var.xi_roe) xi = aU;
    }

    // sgn(U) min(|U|', c): min(|U|', c) = 0 whenever U = 0 (then |U|' = 0), so the sign can
    // be copied onto it
    const V mn = vmn(Up, ch);
    const V smc = vcopysign(mn, uh) * chi;
    const V pp = vfma(smc, dp, vfma(s1, fM, one - s1) * vmx(ch - Up, zero) * rh * du);
    const V th = vmn(vmx(splat<V>(K.mr2), M * M), one);
    const V om = one - th;
    const V ou = om * uh;
    const V X = vfma(ou, ou, (splat<V>(4) * c2h) * th);
    const V rX = rsq(X);           // 1 / (2 c~)
    const V ct = half * X * rX;    // c~
    // |U~| = (1 + theta) |U| / 2, and U sgn(U~) min(|U~|, c~) = |U| min(|U~|, c~): U~ has the
    // sign of U
    const V aUt = vfma(half, th, half) * aU;
    const V term = vfma(om, vfnma(aU * rX, vmn(aUt, ct), Up), vmx(ct - Up, zero));
    // -rho delta U_p (the sign is taken into the factor 1 - f^8(M))
    V nA = s1 * (fM8 - one) * term * dp * chi * chi * rcp(th);
    if constexpr (ABL) {
        if (var.dup_mode == 1) nA = zero;
        else if (var.dup_mode == 2) nA = -(vmx(ch - aU, zero) * dp * chi * chi);   // rho x Eq. 17
    }
    const V dUu = half * smc * du;

    // Eq. 85 assembled per side: the central flux, the xi and delta U_u terms of a side carry
    // the same factor rho_side (U_side + xi - dUu) or rho_side (U_side - xi - dUu) times the
    // side's (1, U, V, H), so each component is two products of that factor plus the
    // pressure and delta U_p terms.
    const V gL = L.r * (L.un + (xi - dUu)), gR = R.r * (R.un - (xi + dUu));
    F[0] = (gL + gR) + nA;
    F[1] = vfma(gL, L.un, vfma(gR, R.un, vfma(nA, uh, L.p + R.p) - pp));
    F[2] = vfma(gL, L.ut, vfma(gR, R.ut, nA * vh));
    F[3] = vfma(gL, L.H, vfma(gR, R.H, nA * Hh));
}

// ------------------------------------------------------------------ geometry
// Vertex (I, J) of a curvilinear grid sits at (I dx + dX(I, J), J dy + dY(I, J)).
// x-face on vertex column I, row J: S = (dy + dY(I,J+1) - dY(I,J), -(dX(I,J+1) - dX(I,J))).
// y-face on vertex row J, column I: S = (-(dY(I+1,J) - dY(I,J)), dx + dX(I+1,J) - dX(I,J)).
template <typename T> struct CellGeom { T Xx, Xy, Yx, Yy, V; };

// Arithmetic with explicit rounding (no FMA contraction), so that the time-step rate of a
// state comes out bit-identical wherever it is evaluated (the stage-3 epilogue and the rate
// kernel after a restart from a saved state).
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
template <typename T> __device__ __forceinline__ T rsub(T a, T b) { return radd(a, -b); }

template <typename T>
__device__ __forceinline__ CellGeom<T> cell_geom(T x00, T x10, T x01, T x11, T y00, T y10, T y01, T y11, T dx, T dy)
{
    const T h = T(0.5);
    CellGeom<T> c;
    c.Xx = radd(dy, rmul(h, radd(rsub(y01, y00), rsub(y11, y10))));
    c.Xy = -rmul(h, radd(rsub(x01, x00), rsub(x11, x10)));
    c.Yx = -rmul(h, radd(rsub(y10, y00), rsub(y11, y01)));
    c.Yy = radd(dx, rmul(h, radd(rsub(x10, x00), rsub(x11, x01))));
    const T d1x = radd(dx, rsub(x11, x00)), d1y = radd(dy, rsub(y11, y00));
    const T d2x = radd(-dx, rsub(x01, x10)), d2y = radd(dy, rsub(y01, y10));
    c.V = rmul(h, rsub(rmul(d1x, d2y), rmul(d1y, d2x)));
    return c;
}

// Velocity, |q|^2 and pressure of a conserved state, with explicit rounding: the stage
// epilogue's positivity check and the time-step rate share them.
template <typename T> struct CellPrims { T ri, u, v, q2, p; };
template <typename T>
__device__ __forceinline__ CellPrims<T> cell_prims(T r, T ru, T rv, T rE, const GridCoef<T> &K)
{
    CellPrims<T> s;
    s.ri = rcp(r);
    s.u = rmul(ru, s.ri);
    s.v = rmul(rv, s.ri);
    s.q2 = radd(rmul(s.u, s.u), rmul(s.v, s.v));
    s.p = rmul(K.gm1, rsub(rE, rmul(rmul(T(0.5), r), s.q2)));
    return s;
}

// The rate sum_dir speed_dir |S_dir| / V of one cell (the time step is CFL / max rate). The
// speed normal to a direction is |U| + max(c, c~/theta), with theta and c~ of Eqs. 99-101 on
// the cell state: theta depends only on the cell's Mach number, so both directions share it
// (classical |U| + c when theta = 1).
template <bool CURV, typename T>
__device__ __forceinline__ T cell_rate(const CellPrims<T> &s, const CellGeom<T> &cg, const GridCoef<T> &K)
{
    const T c2 = rmul(rmul(K.g, s.p), s.ri);
    const T c = sqrt0(c2);
    const T th = vmin(vmax(K.mr2, rmul(s.q2, rcp(c2))), T(1));
    T Ux = s.u, Uy = s.v, lx = T(1), ly = T(1);
    if constexpr (CURV) {
        lx = sqrt0(radd(rmul(cg.Xx, cg.Xx), rmul(cg.Xy, cg.Xy)));
        ly = sqrt0(radd(rmul(cg.Yx, cg.Yx), rmul(cg.Yy, cg.Yy)));
        Ux = rmul(radd(rmul(s.u, cg.Xx), rmul(s.v, cg.Xy)), rcp(lx));
        Uy = rmul(radd(rmul(s.u, cg.Yx), rmul(s.v, cg.Yy)), rcp(ly));
    }
    T wx = c, wy = c;
    if (th < T(1)) {
        const T om = rsub(T(1), th), ith = rcp(th);
        const T a = rmul(rmul(T(4), c2), th), o2 = rmul(om, om);
        wx = vmax(c, rmul(rmul(T(0.5), sqrt0(radd(a, rmul(o2, rmul(Ux, Ux))))), ith));
        wy = vmax(c, rmul(rmul(T(0.5), sqrt0(radd(a, rmul(o2, rmul(Uy, Uy))))), ith));
    }
    const T sx = radd(vabs(Ux), wx), sy = radd(vabs(Uy), wy);
    if constexpr (CURV) return rmul(radd(rmul(sx, lx), rmul(sy, ly)), rcp(cg.V));
    else return radd(rmul(sx, K.idx), rmul(sy, K.idy));
}

// Rate slots hold a non-negative rate as the bit pattern of the working precision (float bits
// in the low word for FP32), so that an unsigned atomicMax orders them like the values.
__device__ __forceinline__ unsigned long long rate_bits(float r) { return (unsigned long long)__float_as_uint(r); }
__device__ __forceinline__ unsigned long long rate_bits(double r) { return (unsigned long long)__double_as_longlong(r); }
template <typename T> __device__ __forceinline__ T rate_value(unsigned long long b);
template <> __device__ __forceinline__ float rate_value<float>(unsigned long long b) { return __uint_as_float((unsigned)b); }
template <> __device__ __forceinline__ double rate_value<double>(unsigned long long b) { return __longlong_as_double((long long)b); }

// Boundary resolution of one index direction: a cell index outside [0, n) maps to the
// source index of its ghost value and a kind: 0 interior/periodic/outflow (a plain copy of
// the source cell), 1 WALL (the source cell mirrored about the boundary face), 2 INFLOW (the
// prescribed state), 3 EXCHANGE (the ghost row itself, j = -2, -1, n or n + 1: a grid with an
// EXCHANGE side stores those rows in its state planes, set by the caller from the
// neighbouring slab). Indices beyond the two ghost layers (ragged strips) are clamped into the
// grid; their values are never used.
__device__ __forceinline__ int resolve_index(int x, int n, int bc_lo, int bc_hi, int &kind)
{
    kind = 0;
    if (x >= 0 && x < n) return x;
    const int bc = x < 0 ? bc_lo : bc_hi;
    int s;
    if (bc == BC_INFLOW) { kind = 2; s = 0; }
    else if (bc == BC_EXCHANGE) { kind = 3; return clampi(x, -2, n + 1); }   // a ghost row kept in the planes
    else if (bc == BC_PERIODIC) s = ((x % n) + n) % n;
    else if (bc == BC_OUTFLOW) s = x < 0 ? 0 : n - 1;
    else { kind = 1; s = x < 0 ? -1 - x : 2 * n - 1 - x; }
    return clampi(s, 0, n - 1);
}

// ------------------------------------------------------------------ face evaluation
template <typename T> __device__ __forceinline__ T shup(T v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
template <typename T> __device__ __forceinline__ T shdn(T v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }

template <typename T> __device__ __forceinline__ T ratio_P(T r0, T p0, T r1, T p1)
{
    // Eq. 97; in FP32 each ratio is the smaller value times the reciprocal of the larger
    if constexpr (sizeof(T) == 4)
        return fmn(fmn(p0, p1) * rcp(fmx(p0, p1)), fmn(r0, r1) * rcp(fmx(r0, r1)));
    else
        return fmn(fmn(p0, p1) / fmx(p0, p1), fmn(r0, r1) / fmx(r0, r1));
}

// MUSCL limited slope: minmod(a, b) = (sgn a + sgn b)/2 min(|a|, |b|); van Leer
// (a|b| + |a|b) / (|a|+|b|) = 2 a |b| / (|a| + |b|), 0 when ab <= 0. The sign test and the van
// Leer quotient avoid the product a b, which in FP32 underflows for differences below ~1e-19
// (a state scaled by 1e-24 is as valid as the unscaled one).
template <typename V> __device__ __forceinline__ V limiter(bool vanleer, V a, V b)
{
    const V zero = splat<V>(0);
    const auto keep = gt(a * vcopysign(splat<V>(1), b), zero);   // same signs, a != 0
    if (vanleer) {
        const V aa = vabs(a), ab = vabs(b);
        return sel(keep, (a + a) * (ab * rcp(aa + ab)), zero);
    }
    return sel(keep, sel(gt(a, zero), vmin(a, b), vmax(a, b)), zero);
}

// Cell-window entry: primitives (rho, u, v, p) in the global frame, the derived face
// quantities (first order: computed once per cell), the conserved rho u, rho v, rho E as
// loaded (the first-order kernels' stage epilogue takes U^(k) from here instead of reading it
// again), and the flags (bit 0 solid, bit 1 wall).
template <typename T> struct WC {
    T r, u, v, p, c2, H, sr, Mq;
    T q1, q2, q3;
    uint8_t fl;
};

template <typename T, bool MUSCL>
__device__ __forceinline__ void derive(WC<T> &c, const GridCoef<T> &K)
{
    if constexpr (!MUSCL) {
        const FS<T> s = side_from_prims(c.r, c.u, c.v, c.p, K);
        c.c2 = s.c2; c.H = s.H; c.sr = s.sr; c.Mq = s.Mq;
    } else {
        c.c2 = c.H = c.sr = c.Mq = T(0);
    }
}

// A face as seen by one lane: left/right cells A, B, MUSCL stencil cells Am (before A) and
// Bp (after B), the unit normal from A to B, the length, the unit normals of the faces Am|A
// and B|Bp (for mirrors at solid stencil cells), and the detector value.
template <typename T> struct Face {
    WC<T> A, B, Am, Bp;
    T nx, ny, len, nAmx, nAmy, nBpx, nBpy, s1;
};

template <typename T> __device__ __forceinline__ bool face_is_wall(const Face<T> &f, bool muscl)
{
    return (f.A.fl | f.B.fl) != 0 || (muscl && ((f.Am.fl | f.Bp.fl) & 1));
}

// Face-frame side from global primitives (rotation by the face normal).
template <typename V, typename S>
__device__ __forceinline__ FS<V> side_rot(V r, V u, V v, V p, V nx, V ny, const GridCoef<S> &K)
{
    return side_from_prims(r, vfma(nx, u, ny * v), vfma(nx, v, -(ny * u)), p, K);
}

// Packed reconstruction. A face's left state is its left cell plus half that cell's limited
// slope, its right state its right cell minus half that cell's slope, so the slope is a
// per-cell quantity: a lane evaluates its cell's x- and y-slopes as one packed pair, takes the
// west cell's x-slope from its neighbour lane and the south cell's y-slope from the row before
// (the same operands, and so the same values, as evaluating both slopes per face). Both
// limiters keep a reconstructed value between the two cells of the face (minmod: within half
// the smaller slope; van Leer: the harmonic mean is below twice either slope), so positive
// density and pressure stay positive. The packed path runs only on faces whose two cells'
// densities and pressures are within a factor 1e5 of each other, where that bound holds in
// FP32 with a wide margin (rounding moves a value by a few ulps of the larger cell value, far
// less than the smaller one); the positivity fallback to first order therefore never fires
// there, and the scalar path keeps it for every other face.

// Scalar evaluation of one face: walls (first-order state and its mirror), MUSCL with solid
// mirrors and the FP64 positivity decision in FP32, rotation to the face frame, flux, and the
// rotation back. Returns F |S| in the global frame.
template <typename T, bool MUSCL, bool ABL = false>
__device__ __forceinline__ void face_scalar(const Face<T> &f, const GridCoef<T> &K, int eps1, int xi_form,
                                            bool vanleer, T F[4], const Variant &var = Variant())
{
    F[0] = F[1] = F[2] = F[3] = T(0);
    if ((f.A.fl & f.B.fl) & 1) return;
    T WL[4] = {f.A.r, f.A.u, f.A.v, f.A.p}, WR[4] = {f.B.r, f.B.u, f.B.v, f.B.p};
    if ((f.A.fl | f.B.fl) != 0) {
        if (f.A.fl) { for (int k = 0; k < 4; ++k) WL[k] = WR[k]; mirror_vel(WL[1], WL[2], f.nx, f.ny); }
        else { for (int k = 0; k < 4; ++k) WR[k] = WL[k]; mirror_vel(WR[1], WR[2], f.nx, f.ny); }
    } else if constexpr (MUSCL) {
        T M0[4] = {f.Am.r, f.Am.u, f.Am.v, f.Am.p}, M3[4] = {f.Bp.r, f.Bp.u, f.Bp.v, f.Bp.p};
        if (f.Am.fl & 1) { for (int k = 0; k < 4; ++k) M0[k] = WL[k]; mirror_vel(M0[1], M0[2], f.nAmx, f.nAmy); }
        if (f.Bp.fl & 1) { for (int k = 0; k < 4; ++k) M3[k] = WR[k]; mirror_vel(M3[1], M3[2], f.nBpx, f.nBpy); }
        T lL[4], lR[4], rL[4], rR[4];
        for (int k = 0; k < 4; ++k) {
            lL[k] = limiter(vanleer, WL[k] - M0[k], WR[k] - WL[k]);
            lR[k] = limiter(vanleer, WR[k] - WL[k], M3[k] - WR[k]);
            rL[k] = vfma(T(0.5), lL[k], WL[k]);
            rR[k] = vfnma(T(0.5), lR[k], WR[k]);
        }
        // Positivity of the reconstructed density and pressure, else first order. In FP32 a
        // density or pressure that comes out within rounding of zero (or below it) is
        // reconstructed again in FP64 from the same cell values and decided there: a limited
        // reconstruction lies between the face's two cells, which FP32 cannot resolve across a
        // jump of seven or more orders of magnitude, while FP64 decides as the FP64 path does.
        bool pos = rL[0] > T(0) && rL[3] > T(0) && rR[0] > T(0) && rR[3] > T(0);
        if constexpr (sizeof(T) == 4) {
            const T eps = T(1e-6);
            if (!(rL[0] > eps * WL[0]) || !(rL[3] > eps * WL[3]) || !(rR[0] > eps * WR[0]) || !(rR[3] > eps * WR[3])) {
                double dL[4], dR[4];
                for (int k = 0; k < 4; ++k) {
                    const double wl = WL[k], wr = WR[k], m0 = M0[k], m3 = M3[k];
                    dL[k] = fma(0.5, limiter(vanleer, wl - m0, wr - wl), wl);
                    dR[k] = fma(-0.5, limiter(vanleer, wr - wl, m3 - wr), wr);
                }
                pos = dL[0] > 0.0 && dL[3] > 0.0 && dR[0] > 0.0 && dR[3] > 0.0;
                if (pos)
                    for (int k = 0; k < 4; ++k) { rL[k] = (T)dL[k]; rR[k] = (T)dR[k]; }
            }
        }
        if (pos) for (int k = 0; k < 4; ++k) { WL[k] = rL[k]; WR[k] = rR[k]; }
    }
    FS<T> L, R;
    if (!MUSCL && (f.A.fl | f.B.fl) == 0) {
        L = {f.A.r, vfma(f.nx, f.A.u, f.ny * f.A.v), vfma(f.nx, f.A.v, -(f.ny * f.A.u)), f.A.p, f.A.c2, f.A.H, f.A.sr, f.A.Mq};
        R = {f.B.r, vfma(f.nx, f.B.u, f.ny * f.B.v), vfma(f.nx, f.B.v, -(f.ny * f.B.u)), f.B.p, f.B.c2, f.B.H, f.B.sr, f.B.Mq};
    } else {
        L = side_rot(WL[0], WL[1], WL[2], WL[3], f.nx, f.ny, K);
        R = side_rot(WR[0], WR[1], WR[2], WR[3], f.nx, f.ny, K);
    }
    T G2[4];
    roeam_flux2<ABL>(L, R, f.s1, K, eps1, xi_form, G2, var);
    const T h = T(0.5) * f.len;
    F[0] = h * G2[0];
    F[1] = h * vfnma(f.ny, G2[2], f.nx * G2[1]);
    F[2] = h * vfma(f.ny, G2[1], f.nx * G2[2]);
    F[3] = h * G2[3];
}

// Packed FP32 evaluation of a lane's x-face (component x) and y-face (component y), both free
// of walls. Cartesian faces enter with their normal velocity first (the y-face's (v, u) is a
// relabelling, undone on output); curvilinear faces are rotated by their normals. WL / WR are
// the reconstructed states (global frame) of the reconstructing kernels.
template <bool MUSCL, bool CURV>
__device__ __forceinline__ void faces_packed(const Face<float> &fx, const Face<float> &fy, const GridCoef<float> &K,
                                             int eps1, int xi_form, const V2 WL[4], const V2 WR[4], float Fx[4],
                                             float Fy[4])
{
    FS<V2> L, R;
    if constexpr (!MUSCL) {
        const WC<float> &a = fx.A, &b = fx.B, &c = fy.A, &d = fy.B;
        if constexpr (CURV) {
            const V2 nx = mk2(fx.nx, fy.nx), ny = mk2(fx.ny, fy.ny);
            const V2 uL = mk2(a.u, c.u), vL = mk2(a.v, c.v), uR = mk2(b.u, d.u), vR = mk2(b.v, d.v);
            L = {mk2(a.r, c.r), vfma(nx, uL, ny * vL), vfma(nx, vL, -(ny * uL)), mk2(a.p, c.p), mk2(a.c2, c.c2),
                 mk2(a.H, c.H), mk2(a.sr, c.sr), mk2(a.Mq, c.Mq)};
            R = {mk2(b.r, d.r), vfma(nx, uR, ny * vR), vfma(nx, vR, -(ny * uR)), mk2(b.p, d.p), mk2(b.c2, d.c2),
                 mk2(b.H, d.H), mk2(b.sr, d.sr), mk2(b.Mq, d.Mq)};
        } else {
            L = {mk2(a.r, c.r), mk2(a.u, c.v), mk2(a.v, c.u), mk2(a.p, c.p), mk2(a.c2, c.c2), mk2(a.H, c.H),
                 mk2(a.sr, c.sr), mk2(a.Mq, c.Mq)};
            R = {mk2(b.r, d.r), mk2(b.u, d.v), mk2(b.v, d.u), mk2(b.p, d.p), mk2(b.c2, d.c2), mk2(b.H, d.H),
                 mk2(b.sr, d.sr), mk2(b.Mq, d.Mq)};
        }
    } else {
        if constexpr (CURV) {
            const V2 nx = mk2(fx.nx, fy.nx), ny = mk2(fx.ny, fy.ny);
            L = side_rot(WL[0], WL[1], WL[2], WL[3], nx, ny, K);
            R = side_rot(WR[0], WR[1], WR[2], WR[3], nx, ny, K);
        } else {
            L = side_from_prims(WL[0], mk2(WL[1].v.x, WL[2].v.y), mk2(WL[2].v.x, WL[1].v.y), WL[3], K);
            R = side_from_prims(WR[0], mk2(WR[1].v.x, WR[2].v.y), mk2(WR[2].v.x, WR[1].v.y), WR[3], K);
        }
    }
    V2 G2[4];
    roeam_flux2(L, R, mk2(fx.s1, fy.s1), K, eps1, xi_form, G2);
    if constexpr (CURV) {
        const float hx = 0.5f * fx.len, hy = 0.5f * fy.len;
        Fx[0] = hx * G2[0].v.x;
        Fx[3] = hx * G2[3].v.x;
        Fy[0] = hy * G2[0].v.y;
        Fy[3] = hy * G2[3].v.y;
        Fx[1] = hx * vfnma(fx.ny, G2[2].v.x, fx.nx * G2[1].v.x);
        Fx[2] = hx * vfma(fx.ny, G2[1].v.x, fx.nx * G2[2].v.x);
        Fy[1] = hy * vfnma(fy.ny, G2[2].v.y, fy.nx * G2[1].v.y);
        Fy[2] = hy * vfma(fy.ny, G2[1].v.y, fy.nx * G2[2].v.y);
    } else {
        // (twice the flux: the residual applies the half lengths)
        Fx[0] = G2[0].v.x;
        Fx[1] = G2[1].v.x;
        Fx[2] = G2[2].v.x;
        Fx[3] = G2[3].v.x;
        Fy[0] = G2[0].v.y;
        Fy[1] = G2[2].v.y;
        Fy[2] = G2[1].v.y;
        Fy[3] = G2[3].v.y;
    }
}

// ------------------------------------------------------------------ the fused stage kernel
// Per-grid values a warp keeps in registers while it sweeps a strip.
// Bounds-checked debug builds (-DROEAM_DEBUG): every state, mask and vertex access of the
// stage kernel is checked against its whole buffer; an access outside it sets ST_BOUNDS in the
// status word (reported as ROEAM_E_BOUNDS) and reads zeros or is skipped instead of faulting.
#ifdef ROEAM_DEBUG
__device__ __align__(16) unsigned char dbg_sink[16];
struct DbgBufs {
    const unsigned char *lo[6];   // src, un, dst, vdx, vdy, solid
    unsigned long long bytes[6];
    unsigned *status;
};
template <typename P> __device__ __forceinline__ bool dbg_ok(const DbgBufs &d, int buf, P *p)
{
    const unsigned char *q = (const unsigned char *)p;
    if (d.lo[buf] && q >= d.lo[buf] && q + sizeof(P) <= d.lo[buf] + d.bytes[buf]) return true;
    atomicOr(d.status, ST_BOUNDS);
    return false;
}
#define DBG_LD(R, buf, p) (dbg_ok((R).dbg, (buf), (p)) ? (p) : (decltype(p))dbg_sink)
#define DBG_ST(R, buf, p) dbg_ok((R).dbg, (buf), (p))
#else
#define DBG_LD(R, buf, p) (p)
#define DBG_ST(R, buf, p) true
#endif
enum { DB_SRC = 0, DB_UN = 1, DB_DST = 2, DB_VDX = 3, DB_VDY = 4, DB_SOLID = 5 };

template <typename T> struct GridRegs {
    const T *src, *un;
    T *dst;
    const T *vdx, *vdy;         // vertex displacement planes of this grid (curvilinear)
    const uint8_t *solid;       // solid mask of this grid, or null
    int ni, nj, pitch, plane, vpitch;
    int bcW, bcE, bcS, bcN;
#ifdef ROEAM_DEBUG
    DbgBufs dbg;
#endif
};

// Cell loads of the reconstructing kernels carry the L1 priority evict_last: their window is
// deeper, so a row is read again by the stage epilogue several rows after its first load, and
// without the hint most of those reads missed L1 (measured faster on the Cartesian and the
// curvilinear reconstructing workloads; the first-order kernels measured slower with it).
__device__ __forceinline__ float ld_keep(const float *p) { float v; asm("ld.global.nc.L1::evict_last.f32 %0, [%1];" : "=f"(v) : "l"(p)); return v; }
__device__ __forceinline__ double ld_keep(const double *p) { double v; asm("ld.global.nc.L1::evict_last.f64 %0, [%1];" : "=d"(v) : "l"(p)); return v; }
template <bool KEEP, typename T> __device__ __forceinline__ T ld_row(const T *p) { if constexpr (KEEP) return ld_keep(p); else return __ldg(p); }

// Loading a cell is split in two so that the next row's HBM loads are in flight while the
// current row is computed: issue_cell resolves row j (the column is resolved once per unit
// into isrc / kx) and starts the loads; finish_cell turns them into primitives, derived face
// quantities and flags. Resolution order: an INFLOW side in i gives the inflow state;
// otherwise an INFLOW side in j gives it (then mirrored by a WALL side in i); otherwise the
// source cell, mirrored about the S/N boundary face by a WALL side in j, then about the W/E
// boundary face by a WALL side in i.
template <typename T> struct Pending {
    T raw[4];
    int jsrc, ky;
    int solid;   // the cell's solid-mask byte (kernels with walls)
};

template <typename T, bool WALLS, bool KEEP = false>
__device__ __forceinline__ void issue_cell(const GridRegs<T> &R, int isrc, int kx, int j, Pending<T> &q)
{
    q.jsrc = resolve_index(j, R.nj, R.bcS, R.bcN, q.ky);
    q.solid = 0;
    if (kx != 2 && q.ky != 2) {
        const int x = q.jsrc * R.pitch + isrc;
        q.raw[0] = ld_row<KEEP>(DBG_LD(R, DB_SRC, R.src + x));
        q.raw[1] = ld_row<KEEP>(DBG_LD(R, DB_SRC, R.src + x + R.plane));
        q.raw[2] = ld_row<KEEP>(DBG_LD(R, DB_SRC, R.src + x + 2 * R.plane));
        q.raw[3] = ld_row<KEEP>(DBG_LD(R, DB_SRC, R.src + x + 3 * R.plane));
        // (jsrc is a grid row, or an EXCHANGE ghost row, whose mask rows the grid also keeps)
        if constexpr (WALLS)
            if (R.solid) q.solid = __ldg(DBG_LD(R, DB_SOLID, R.solid + q.jsrc * R.ni + isrc));
    }
}

// LATE_SOLID reads the solid-mask byte here instead of taking the one issue_cell prefetched
// (the ablation kernels, whose scalar path measured faster that way; the main kernels hide
// that load's latency behind a row of work).
template <typename T, bool MUSCL, bool CURV, bool WALLS, bool LATE_SOLID = false>
__device__ __forceinline__ void finish_cell(const GridRegs<T> &R, const GridCoef<T> &K, int i, int isrc, int kx, int j,
                                            const Pending<T> &q, WC<T> &c)
{
    const int ky = q.ky;
    c.fl = 0;
    if (kx == 2 || ky == 2) {
        c.r = K.inflow[0]; c.u = K.inflow[1]; c.v = K.inflow[2]; c.p = K.inflow[3];
        // (q1..q3 stay unset: an inflow ghost cell is never written)
    } else {
        const T ri = rcp(q.raw[0]);
        c.r = q.raw[0]; c.u = q.raw[1] * ri; c.v = q.raw[2] * ri;
        c.q1 = q.raw[1]; c.q2 = q.raw[2]; c.q3 = q.raw[3];
        c.p = K.gm1 * vfnma(T(0.5) * q.raw[0], vfma(c.u, c.u, c.v * c.v), q.raw[3]);
        if constexpr (WALLS) {
            if constexpr (LATE_SOLID) { if (R.solid && *DBG_LD(R, DB_SOLID, R.solid + q.jsrc * R.ni + isrc)) c.fl = 1; }
            else if (q.solid) c.fl = 1;
        }
    }
    if constexpr (WALLS) {
        if (ky == 1 && kx != 2) {
            T nx = T(0), ny = T(1);
            if constexpr (CURV) {
                const int b = (j < 0 ? 0 : R.nj) * R.vpitch + isrc;
                const T sx = -(*DBG_LD(R, DB_VDY, R.vdy + (b + 1)) - *DBG_LD(R, DB_VDY, R.vdy + b)),
                        sy = K.dx + (*DBG_LD(R, DB_VDX, R.vdx + (b + 1)) - *DBG_LD(R, DB_VDX, R.vdx + b));
                const T l = rsq(vfma(sx, sx, sy * sy));
                nx = sx * l; ny = sy * l;
            }
            mirror_vel(c.u, c.v, nx, ny);
        }
        if (kx == 1) {
            T nx = T(1), ny = T(0);
            if constexpr (CURV) {
                // (the W/E boundary face of row j, ghost rows of EXCHANGE sides included)
                const int b = clampi(j, R.bcS == BC_EXCHANGE ? -2 : 0, R.bcN == BC_EXCHANGE ? R.nj + 1 : R.nj - 1) *
                                  R.vpitch + (i < 0 ? 0 : R.ni);
                const T sx = K.dy + (*DBG_LD(R, DB_VDY, R.vdy + (b + R.vpitch)) - *DBG_LD(R, DB_VDY, R.vdy + b)),
                        sy = -(*DBG_LD(R, DB_VDX, R.vdx + (b + R.vpitch)) - *DBG_LD(R, DB_VDX, R.vdx + b));
                const T l = rsq(vfma(sx, sx, sy * sy));
                nx = sx * l; ny = sy * l;
            }
            mirror_vel(c.u, c.v, nx, ny);
        }
        if ((kx == 1 || ky == 1) && kx != 2) c.fl |= 2;
    }
    derive<T, MUSCL>(c, K);
}

template <bool WALLS, typename T> __device__ __forceinline__ WC<T> shup_c(const WC<T> &c, int d, bool derived)
{
    WC<T> o;
    o.r = shup(c.r, d); o.u = shup(c.u, d); o.v = shup(c.v, d); o.p = shup(c.p, d);
    if (derived) { o.c2 = shup(c.c2, d); o.H = shup(c.H, d); o.sr = shup(c.sr, d); o.Mq = shup(c.Mq, d); }
    else { o.c2 = o.H = o.sr = o.Mq = T(0); }
    // (q1..q3 stay unset: a neighbour's conserved values are never read)
    o.fl = WALLS ? (uint8_t)__shfl_up_sync(0xffffffffu, (int)c.fl, d) : (uint8_t)0;
    return o;
}
template <bool WALLS, typename T> __device__ __forceinline__ WC<T> shdn_c(const WC<T> &c, int d)
{
    WC<T> o;
    o.r = shdn(c.r, d); o.u = shdn(c.u, d); o.v = shdn(c.v, d); o.p = shdn(c.p, d);
    o.c2 = o.H = o.sr = o.Mq = T(0);
    o.fl = WALLS ? (uint8_t)__shfl_down_sync(0xffffffffu, (int)c.fl, d) : (uint8_t)0;
    return o;
}

// Dynamic unit scheduling (StageArgs::work): the unit after u for this warp. DYN = false keeps
// the static round robin (the reconstructing curvilinear kernels: their units are of equal size
// on the grids they serve, and the claim's registers made them spill, -16 % on the warped step).
template <bool DYN, typename T>
__device__ __forceinline__ int next_unit(const StageArgs<T> &a, int u, int nwarps, int lane)
{
    if (!DYN || !a.work) return u + nwarps;
    unsigned n = 0;
    if (lane == 0) n = atomicAdd(a.work, 1u);
    return a.tile_lo + nwarps + (int)__shfl_sync(0xffffffffu, n, 0);
}
// A warp that has run out of units counts itself done; the last one resets the counters (every
// warp's final claim precedes its count, fenced).
template <bool DYN, typename T>
__device__ __forceinline__ void finish_units(const StageArgs<T> &a, int nwarps, int lane)
{
    if (!DYN || !a.work || lane != 0) return;
    __threadfence();
    if (atomicAdd(a.work + 1, 1u) == (unsigned)nwarps - 1u) {
        __threadfence();
        atomicExch(a.work, 0u);
        atomicExch(a.work + 1, 0u);
    }
}

template <typename T, bool MUSCL, bool CURV, bool WALLS, int NT, bool ABL>
__global__ void __launch_bounds__(NT, (stage_min_blocks<T, MUSCL, CURV, ABL>())) stage_kernel(const StageArgs<T> a)
{
    constexpr int H = MUSCL ? 2 : 1;
    constexpr int NW = H + 2;          // window rows j-H .. j+1
    constexpr int NV = 4;              // vertex rows j-1 .. j+2 (curvilinear)
    constexpr int WIDTH = 32 - 2 * H;  // interior columns per strip
    constexpr bool PACKED = sizeof(T) == 4;
    const int lane = threadIdx.x & 31;
    const int warp = blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
    const int nwarps = gridDim.x * (NT / 32);

    if (a.rate_zero && blockIdx.x == 0)
        for (int g = threadIdx.x; g < a.ngrids; g += NT) a.rate_zero[g] = 0ull;

    // MODE_NORM: each thread's FP64 sums of R^2 [k] and maxima of |R| [4 + k] in dynamic shared
    // memory (slot k * NT + thread; only norm launches ask for it), rather than in sixteen
    // registers that every launch would hold
    extern __shared__ __align__(16) unsigned char norm_smem[];
    double *const nacc = reinterpret_cast<double *>(norm_smem) + threadIdx.x;
    if (a.mode == MODE_NORM)
        for (int k = 0; k < 8; ++k) nacc[k * NT] = 0.0;

    // Each warp takes unit tile_lo + warp first, then (dynamic scheduling) the next unclaimed
    // one, in the order of the unit table (whole-batch launches: by decreasing height), so that
    // warps that drew short units take more of them and the launch ends evenly.
    constexpr bool DYN = stage_dynamic(MUSCL, CURV);
    for (int u = a.tile_lo + warp; u < a.tile_hi; u = next_unit<DYN>(a, u, nwarps, lane)) {
        const int4 unit = __ldg(a.units + u);   // (grid, first lane's column, j0, j1)
        const int g = unit.x;
        const int i = unit.y + lane;            // this lane's column
        const int j0 = unit.z, j1 = unit.w;
        const GridDev &G = a.grids[g];
        const GridCoef<T> K = a.coef[g];
        GridRegs<T> R;
        R.src = a.src + G.off;
        R.un = a.un + G.off;
        R.dst = a.dst + (G.off - a.dst_shift);
        R.ni = G.ni; R.nj = G.nj; R.pitch = G.pitch; R.plane = (int)G.plane;
        R.bcW = G.bc[0]; R.bcE = G.bc[1]; R.bcS = G.bc[2]; R.bcN = G.bc[3];
        if constexpr (CURV) { R.vdx = a.vdx + G.voff; R.vdy = a.vdy + G.voff; R.vpitch = G.vpitch; }
        else { R.vdx = R.vdy = nullptr; R.vpitch = 0; }
#ifdef ROEAM_DEBUG
        R.dbg.lo[DB_SRC] = (const unsigned char *)a.src; R.dbg.bytes[DB_SRC] = sizeof(T) * a.n_state;
        R.dbg.lo[DB_UN] = (const unsigned char *)a.un; R.dbg.bytes[DB_UN] = sizeof(T) * a.n_state;
        R.dbg.lo[DB_DST] = (const unsigned char *)a.dst; R.dbg.bytes[DB_DST] = sizeof(T) * a.n_dst;
        R.dbg.lo[DB_VDX] = (const unsigned char *)a.vdx; R.dbg.bytes[DB_VDX] = sizeof(T) * a.n_vert;
        R.dbg.lo[DB_VDY] = (const unsigned char *)a.vdy; R.dbg.bytes[DB_VDY] = sizeof(T) * a.n_vert;
        R.dbg.lo[DB_SOLID] = a.solid; R.dbg.bytes[DB_SOLID] = a.n_solid;
        R.dbg.status = a.status;
#endif
        R.solid = (WALLS && G.soff >= 0) ? a.solid + G.soff : nullptr;
        const int ni = R.ni, nj = R.nj;
        const bool use_s1 = G.use_s1 != 0;
        const int eps1 = G.eps1, xi_form = G.xi_form;
        const bool vanleer = G.limiter == 2;
        Variant var;
        if constexpr (ABL) {
            var.scheme = G.scheme; var.dup_mode = G.dup_mode; var.ufix = G.ufix; var.xi_roe = G.xi_roe;
        }
        int kx;
        const int isrc = resolve_index(i, ni, R.bcW, R.bcE, kx);
        const bool icol = i >= 0 && i < ni;
        const bool out_lane = lane >= H && lane < H + WIDTH && icol;
        const T rxy = K.dy / K.dx, cy = T(0.5) * K.dx * K.Vi;   // Cartesian residual weights
        T dt = T(0);
        if (a.mode == MODE_STAGE) {
            if (a.dt_fixed_t > T(0)) dt = a.dt_fixed_t;
            else dt = a.cfl_t / rate_value<T>(__ldg(a.rate_rd + g));
        }

        WC<T> Wn[NW];
        T Px[NW], Py[NW - 1];
        T vX[NV], vY[NV];
        Pending<T> pend;
        // vertex rows 0..nj, and the two ghost vertex rows beyond an EXCHANGE side
        const int vjlo = R.bcS == BC_EXCHANGE ? -2 : 0, vjhi = R.bcN == BC_EXCHANGE ? nj + 2 : nj;
        auto vload = [&](int J, T &x, T &y) {
            if constexpr (CURV) {
                const int b = clampi(J, vjlo, vjhi) * R.vpitch + clampi(i, 0, ni);
                x = __ldg(DBG_LD(R, DB_VDX, R.vdx + b)); y = __ldg(DBG_LD(R, DB_VDY, R.vdy + b));
            } else { x = y = T(0); }
        };
        auto px_of = [&](const WC<T> &c) {   // Eq. 97 on this lane's west face; 1 at solid sides
            const T rl = shup(c.r, 1), pl = shup(c.p, 1);
            if constexpr (WALLS) {
                const int fl = __shfl_up_sync(0xffffffffu, (int)c.fl, 1);
                if ((c.fl | fl) & 1) return T(1);
            }
            return ratio_P(rl, pl, c.r, c.p);
        };
        auto py_of = [&](const WC<T> &lo, const WC<T> &hi) {
            if constexpr (WALLS) {
                if ((lo.fl | hi.fl) & 1) return T(1);
            }
            return ratio_P(lo.r, lo.p, hi.r, hi.p);
        };
        // window rows j0-H .. j0+1, each row's loads issued one row ahead (the last issue is
        // the loop's first prefetch, row j0+2)
        for (int v = 0; v < NV; ++v) vload(j0 - 1 + v, vX[v], vY[v]);
        issue_cell<T, WALLS && !ABL, MUSCL>(R, isrc, kx, j0 - H, pend);
        for (int w = 0; w < NW; ++w) {
            const int jr = j0 - H + w;
            const Pending<T> cur = pend;
            issue_cell<T, WALLS && !ABL, MUSCL>(R, isrc, kx, jr + 1, pend);
            finish_cell<T, MUSCL, CURV, WALLS, ABL>(R, K, i, isrc, kx, jr, cur, Wn[w]);
            Px[w] = px_of(Wn[w]);
            if (w > 0) Py[w - 1] = py_of(Wn[w - 1], Wn[w]);
        }
        // the y-slope of row j0 - 1 (packed reconstruction), as the loop would have left it
        float sy_prev[4] = {0.f, 0.f, 0.f, 0.f};
        if constexpr (PACKED && MUSCL) {
            const WC<T> &a0 = Wn[H - 2], &b0 = Wn[H - 1], &c0 = Wn[H];
            const V2 lo = limiter(vanleer, mk2(b0.r, b0.u) - mk2(a0.r, a0.u), mk2(c0.r, c0.u) - mk2(b0.r, b0.u));
            const V2 hi = limiter(vanleer, mk2(b0.v, b0.p) - mk2(a0.v, a0.p), mk2(c0.v, c0.p) - mk2(b0.v, b0.p));
            sy_prev[0] = lo.v.x; sy_prev[1] = lo.v.y; sy_prev[2] = hi.v.x; sy_prev[3] = hi.v.y;
        }
        T Un[4] = {T(0), T(0), T(0), T(0)};
        T acc[4] = {T(0), T(0), T(0), T(0)};
        T my_rate = T(0);
        const bool stage_mode = a.mode == MODE_STAGE;
        const bool combine = stage_mode && a.alpha != T(0);

        // two rows per trip for the first-order kernels (measured faster; the reconstructing ones
        // are not)
#pragma unroll (MUSCL ? 1 : 2)
        for (int j = j0; j <= j1; ++j) {
            // U^n of row j (combined at iteration j+1), issued early
            T Un_next[4] = {T(0), T(0), T(0), T(0)};
            if (combine && out_lane && j < j1) {
                const int x = j * R.pitch + i;
                for (int k = 0; k < 4; ++k) Un_next[k] = *DBG_LD(R, DB_UN, R.un + (x + k * R.plane));
            }

            // ---- the two faces of this lane: west x-face of row j (cells lane-1 | lane) and
            //      the y-face between rows j-1 and j (window H-1 | H)
            Face<T> fx, fy;
            fx.A = shup_c<WALLS>(Wn[H], 1, !MUSCL);
            fx.B = Wn[H];
            fy.A = Wn[H - 1];
            fy.B = Wn[H];
            if constexpr (MUSCL) {
                // (fx.Am's values are shuffled in on the scalar path, the only one that reads them)
                fx.Am.fl = WALLS ? (uint8_t)__shfl_up_sync(0xffffffffu, (int)Wn[H].fl, 2) : (uint8_t)0;
                fx.Bp = shdn_c<WALLS>(Wn[H], 1);
                fy.Am = Wn[H - 2];
                fy.Bp = Wn[H + 1];
            } else {
                fx.Am = fx.Bp = fx.A;
                fy.Am = fy.Bp = fy.A;
            }
            if (use_s1) {
                // Eq. 96 in 2D: the face and the transverse faces of both cells.
                const T pym_l = shup(Py[H - 1], 1), pyp_l = shup(Py[H], 1);
                const T pxm_r = shdn(Px[H - 1], 1), px0_r = shdn(Px[H], 1);
                T ax = fmn3(fmn3(Px[H], pym_l, pyp_l), Py[H - 1], Py[H]);
                T ay = fmn3(fmn3(Py[H - 1], Px[H - 1], pxm_r), Px[H], px0_r);
                if constexpr (PACKED) {
                    const V2 s1 = detector_of(mk2(ax, ay));
                    fx.s1 = s1.v.x; fy.s1 = s1.v.y;
                } else {
                    fx.s1 = detector_of(ax); fy.s1 = detector_of(ay);
                }
            } else {
                fx.s1 = fy.s1 = T(1);
            }
            if constexpr (CURV) {
                // x-face: vertices (i, j), (i, j+1); y-face: vertices (i, j), (i+1, j)
                T sx = K.dy + (vY[2] - vY[1]), sy = -(vX[2] - vX[1]);
                fx.len = sqrt0(vfma(sx, sx, sy * sy));
                T li = rcp(fx.len);
                fx.nx = sx * li; fx.ny = sy * li;
                const T xr = shdn(vX[1], 1), yr = shdn(vY[1], 1);
                sx = -(yr - vY[1]); sy = K.dx + (xr - vX[1]);
                fy.len = sqrt0(vfma(sx, sx, sy * sy));
                li = rcp(fy.len);
                fy.nx = sx * li; fy.ny = sy * li;
                if constexpr (!MUSCL) {
                    fx.nAmx = fx.nBpx = fx.nx; fx.nAmy = fx.nBpy = fx.ny;
                    fy.nAmx = fy.nBpx = fy.nx; fy.nAmy = fy.nBpy = fy.ny;
                }   // (reconstructing: set on the scalar path, the only one that reads them)
            } else {
                // (Cartesian faces leave the length out: len = 2 makes the face's factor
                //  len / 2 one, and the residual applies dy / 2 and dx / 2 per direction)
                fx.nx = T(1); fx.ny = T(0); fx.len = T(2);
                fy.nx = T(0); fy.ny = T(1); fy.len = T(2);
                fx.nAmx = fx.nBpx = T(1); fx.nAmy = fx.nBpy = T(0);
                fy.nAmx = fy.nBpx = T(0); fy.nAmy = fy.nBpy = T(1);
            }

            // per-cell limited slopes (packed reconstruction): this cell's (x, y) pair, the
            // west cell's x-slope and the south cell's y-slope (carried from the row before)
            V2 WLp[4], WRp[4];
            if constexpr (PACKED && MUSCL) {
                const float Ax[4] = {fx.A.r, fx.A.u, fx.A.v, fx.A.p}, Ay[4] = {fy.A.r, fy.A.u, fy.A.v, fy.A.p};
                const float Bc[4] = {fx.B.r, fx.B.u, fx.B.v, fx.B.p};
                const float Px_[4] = {fx.Bp.r, fx.Bp.u, fx.Bp.v, fx.Bp.p}, Py_[4] = {fy.Bp.r, fy.Bp.u, fy.Bp.v, fy.Bp.p};
                const V2 half = mk2(0.5f, 0.5f);
                for (int k = 0; k < 4; ++k) {
                    const V2 A2 = mk2(Ax[k], Ay[k]), B2 = mk2(Bc[k], Bc[k]);
                    const V2 sg = limiter(vanleer, B2 - A2, mk2(Px_[k], Py_[k]) - B2);
                    WRp[k] = B2 - half * sg;
                    WLp[k] = vfma(half, mk2(shup(sg.v.x, 1), sy_prev[k]), A2);
                    sy_prev[k] = sg.v.y;
                }
            }
            T Fw[4], Fs[4];
            // walls, solid cells (and FP64, and the ablation variants) take the scalar path;
            // batches without walls or solid cells never do in FP32
            bool scalar = !PACKED || ABL;
            if constexpr (PACKED && WALLS && !ABL)
                scalar = __any_sync(0xffffffffu, face_is_wall(fx, MUSCL) || face_is_wall(fy, MUSCL));
            if constexpr (PACKED && MUSCL) {
                // faces across a density or pressure jump of 1e5 or more take the scalar path,
                // where a reconstruction within rounding of zero is decided in FP64 (the
                // reconstruction's bounds depend only on the face's two cells)
                if (!scalar) {
                    // (the faces' Eq. 97 ratios min/max of rho and p, already at hand for the
                    //  detector, say whether the jump is 1e5 or more)
                    const T eps = T(1e-5);
                    const bool marginal = Px[H] < eps || Py[H - 1] < eps;
                    scalar = __any_sync(0xffffffffu, marginal);
                }
            }
            // U^(k) of row j-1 for this iteration's epilogue, issued just before the faces are
            // evaluated (the reconstructing curvilinear kernel, which is latency-bound: +2.4 %
            // over the epilogue read when issued at the top of the iteration, +2 % more and 36
            // instead of 60 bytes of spills here, after the slopes and the screens; the other
            // kernels measured slower with it and read it again in the epilogue)
            T Uk[4] = {T(0), T(0), T(0), T(0)};
            if constexpr (MUSCL && CURV) {
                if (stage_mode && out_lane && j > j0) {
                    const int x = (j - 1) * R.pitch + i;
                    for (int k = 0; k < 4; ++k) Uk[k] = __ldg(DBG_LD(R, DB_SRC, R.src + x + k * R.plane));
                }
            }
            if (scalar) {
                if constexpr (MUSCL) {
                    const uint8_t fl = fx.Am.fl;
                    fx.Am = shup_c<WALLS>(Wn[H], 2, false);
                    fx.Am.fl = fl;
                }
                if constexpr (CURV && MUSCL) {
                    // normals of the faces Am|A and B|Bp of both faces (mirrors at solid cells;
                    // the branch is warp-uniform, so the shuffles are safe here)
                    fx.nAmx = shup(fx.nx, 1); fx.nAmy = shup(fx.ny, 1);
                    fx.nBpx = shdn(fx.nx, 1); fx.nBpy = shdn(fx.ny, 1);
                    const T x0 = shdn(vX[0], 1), y0 = shdn(vY[0], 1), x3 = shdn(vX[3], 1), y3 = shdn(vY[3], 1);
                    T tx = -(y0 - vY[0]), ty = K.dx + (x0 - vX[0]), l = rsq(vfma(tx, tx, ty * ty));
                    fy.nAmx = tx * l; fy.nAmy = ty * l;
                    tx = -(y3 - vY[3]); ty = K.dx + (x3 - vX[3]); l = rsq(vfma(tx, tx, ty * ty));
                    fy.nBpx = tx * l; fy.nBpy = ty * l;
                }
                if constexpr (!PACKED || WALLS || MUSCL) {
                    face_scalar<T, MUSCL, ABL>(fx, K, eps1, xi_form, vanleer, Fw, var);
                    face_scalar<T, MUSCL, ABL>(fy, K, eps1, xi_form, vanleer, Fs, var);
                }
            } else if constexpr (PACKED) {
                faces_packed<MUSCL, CURV>(fx, fy, K, eps1, xi_form, WLp, WRp, Fw, Fs);
            }
            // (faces of lanes or rows outside the grid are computed from clamped or ghost states
            //  and never reach a written cell: a written cell's faces all lie in the grid)

            // ---- finish row j-1: R = (acc - F_north) / V, then the stage combination
            if (j > j0) {
                CellGeom<T> cg;
                if constexpr (CURV) {
                    const T x00 = vX[0], y00 = vY[0], x01 = vX[1], y01 = vY[1];
                    const T x10 = shdn(x00, 1), y10 = shdn(y00, 1), x11 = shdn(x01, 1), y11 = shdn(y01, 1);
                    cg = cell_geom(x00, x10, x01, x11, y00, y10, y01, y11, K.dx, K.dy);
                } else {
                    cg.Xx = K.dy; cg.Xy = T(0); cg.Yx = T(0); cg.Yy = K.dx; cg.V = K.V;
                }
                if (out_lane) {
                    const bool solid = WALLS && (Wn[H - 1].fl & 1);
                    // R = D sc: the face sum D and its scale (1 / V, or 1 / (2 dy) for Cartesian
                    // faces); a stage applies dt sc to D in one product
                    T D[4];
                    for (int k = 0; k < 4; ++k) D[k] = solid ? T(0) : acc[k] - Fs[k];
                    const T sc = CURV ? rcp(cg.V) : cy;
                    const int x = (j - 1) * R.pitch + i;
                    if (stage_mode) {
                        T out[4];
                        const WC<T> &self = Wn[H - 1];
                        const T Uw[4] = {self.r, self.q1, self.q2, self.q3};
                        for (int k = 0; k < 4; ++k) {
                            // U^(k) of this cell: kept in the window (FP32 first order without
                            // walls, +1.2 % on the benchmark batch; the walls and FP64 kernels then
                            // spill), loaded above (reconstructing curvilinear), or loaded again
                            // (mostly an L1 hit)
                            const T uk = (!MUSCL && !WALLS && sizeof(T) == 4) ? Uw[k]
                                                            : ((MUSCL && CURV) ? Uk[k] : __ldg(DBG_LD(R, DB_SRC, R.src + x + k * R.plane)));
                            const T upd = vfma(dt * sc, D[k], uk);
                            out[k] = combine ? vfma(a.alpha, Un[k], a.beta * upd) : upd;
                        }
                        for (int k = 0; k < 4; ++k)
                            if (DBG_ST(R, DB_DST, R.dst + (x + k * R.plane))) R.dst[x + k * R.plane] = out[k];
                        if (!solid && a.want_rate) {
                            const CellPrims<T> cp = cell_prims(out[0], out[1], out[2], out[3], K);
                            if (!(out[0] > T(0)) || !(cp.p > T(0))) {
                                const bool fin = isfinite((double)out[0]) && isfinite((double)cp.p);
                                atomicOr(a.status, fin ? ST_NONPOSITIVE : ST_NONFINITE);
                            } else {
                                my_rate = vmax(my_rate, cell_rate<CURV>(cp, cg, K));
                            }
                        } else if (!solid) {
                            // p > 0 without the division: 2 rho (rho E) > (rho u)^2 + (rho v)^2; a cell
                            // that fails it (rare: also products beyond the FP32 range) is decided
                            // by its pressure
                            const T e2 = T(2) * out[0] * out[3], m2 = vfma(out[1], out[1], out[2] * out[2]);
                            if (!(out[0] > T(0)) || !(e2 > m2)) {
                                const CellPrims<T> cp = cell_prims(out[0], out[1], out[2], out[3], K);
                                if (!(out[0] > T(0)) || !(cp.p > T(0))) {
                                    const bool fin = isfinite((double)out[0]) && isfinite((double)cp.p);
                                    atomicOr(a.status, fin ? ST_NONPOSITIVE : ST_NONFINITE);
                                }
                            }
                        }
                    } else if (a.mode == MODE_RESIDUAL) {
                        for (int k = 0; k < 4; ++k)
                            if (DBG_ST(R, DB_DST, R.dst + (x + k * R.plane))) R.dst[x + k * R.plane] = D[k] * sc;
                    } else if (!solid) {
                        for (int k = 0; k < 4; ++k) {
                            const double rk = (double)(D[k] * sc);
                            nacc[k * NT] = fma(rk, rk, nacc[k * NT]);
                            nacc[(4 + k) * NT] = fmax(nacc[(4 + k) * NT], fabs(rk));
                        }
                    }
                }
            }
            if (j == j1) break;
            for (int k = 0; k < 4; ++k) Un[k] = Un_next[k];
            // (curvilinear faces carry their lengths; Cartesian ones twice the flux: the x-face
            //  difference is weighted by dy / dx here and the sum scaled by 1 / (2 dy) above,
            //  so that equal fluxes on opposite faces cancel exactly)
            if constexpr (CURV) {
                for (int k = 0; k < 4; ++k) acc[k] = Fw[k] - shdn(Fw[k], 1) + Fs[k];
            } else {
                for (int k = 0; k < 4; ++k) acc[k] = vfma(Fw[k] - shdn(Fw[k], 1), rxy, Fs[k]);
            }

            // ---- advance the window: row j+2 enters from the prefetch
            for (int w = 0; w < NW - 1; ++w) { Wn[w] = Wn[w + 1]; Px[w] = Px[w + 1]; }
            for (int w = 0; w < NW - 2; ++w) Py[w] = Py[w + 1];
            finish_cell<T, MUSCL, CURV, WALLS, ABL>(R, K, i, isrc, kx, j + NW - H, pend, Wn[NW - 1]);
            Px[NW - 1] = px_of(Wn[NW - 1]);
            Py[NW - 2] = py_of(Wn[NW - 2], Wn[NW - 1]);
            issue_cell<T, WALLS && !ABL, MUSCL>(R, isrc, kx, j + NW - H + 1, pend);
            if constexpr (CURV) {
                for (int v = 0; v < NV - 1; ++v) { vX[v] = vX[v + 1]; vY[v] = vY[v + 1]; }
                vload(j + NV - 1, vX[NV - 1], vY[NV - 1]);
            }
        }
        if (a.want_rate) {
            for (int o = 16; o > 0; o >>= 1) my_rate = vmax(my_rate, __shfl_xor_sync(0xffffffffu, my_rate, o));
            if (lane == 0 && my_rate > T(0)) atomicMax(a.rate_wr + g, rate_bits(my_rate));
        }
    }

    finish_units<DYN>(a, nwarps, lane);

    if (a.mode == MODE_NORM) {
        // Fixed-order block reduction of the FP64 partials: warp shuffles, then warp 0.
        __shared__ double wred[NT / 32][8];
        double v[8];
        for (int k = 0; k < 8; ++k) v[k] = nacc[k * NT];
        for (int o = 16; o > 0; o >>= 1)
            for (int k = 0; k < 8; ++k) {
                const double x = __shfl_xor_sync(0xffffffffu, v[k], o);
                v[k] = k < 4 ? v[k] + x : fmax(v[k], x);
            }
        if (lane == 0)
            for (int k = 0; k < 8; ++k) wred[threadIdx.x >> 5][k] = v[k];
        __syncthreads();
        if (threadIdx.x < 8) {
            double r = 0.0;
            for (int w = 0; w < NT / 32; ++w) r = threadIdx.x < 4 ? r + wred[w][threadIdx.x] : fmax(r, wred[w][threadIdx.x]);
            a.partials[(size_t)blockIdx.x * 8 + threadIdx.x] = r;
        }
    }
}

// Block-wide max of a non-negative value (all threads must call); valid in thread 0.
template <int NT, typename T> __device__ __forceinline__ T block_max(T v, T *red)
{
    for (int o = 16; o > 0; o >>= 1) v = vmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    T r = T(0);
    if (threadIdx.x < 32) {
        r = threadIdx.x < NT / 32 ? red[threadIdx.x] : T(0);
        for (int o = 16; o > 0; o >>= 1) r = vmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    }
    return r;
}

// ------------------------------------------------------------------ small kernels
// Host layout [4][nj][ni] per grid (H: float64 or float) <-> pitched planes, blockIdx.y = grid.
// Each thread moves IO_PER cells a stride of gridDim.x * 256 apart, all of their loads issued
// before the first store, so that a thread has IO_PER x 4 loads in flight instead of one DRAM
// latency per cell; indices are 32-bit (a grid holds at most 2^28 cells). With RATE the pack
// also takes the time-step rate of the state it writes, the largest cell_rate over the fluid
// cells (the functions the stage kernel's third stage applies to the state it writes, so a state
// loaded from the host gives the dt bit for bit that the same state gives once stepped into),
// in the same pass.
constexpr int IO_PER = 4;

template <typename T, typename H, bool RATE, bool CURV>
__global__ void __launch_bounds__(256) pack_kernel(const GridDev *grids, int g_lo, const H *__restrict__ packed,
                                                   T *__restrict__ U, long long p_shift, RateOut<T> ro)
{
    __shared__ T red[8];
    const int g = g_lo + blockIdx.y;
    const GridDev &G = grids[g];
    const unsigned ni = (unsigned)G.ni, n = ni * (unsigned)G.nj, stride = gridDim.x * 256u;
    const H *__restrict__ src = packed + (G.poff - p_shift);
    T *__restrict__ dst = U + G.off;
    const long long pitch = G.pitch, plane = G.plane;
    T m = T(0);
    for (unsigned q0 = blockIdx.x * 256u + threadIdx.x; q0 < n; q0 += IO_PER * stride) {
        T v[IO_PER][4];
#pragma unroll
        for (int e = 0; e < IO_PER; ++e) {
            const unsigned q = q0 + e * stride;
            if (q < n)
                for (int k = 0; k < 4; ++k) v[e][k] = T(src[(long long)k * n + q]);
        }
#pragma unroll
        for (int e = 0; e < IO_PER; ++e) {
            const unsigned q = q0 + e * stride;
            if (q >= n) break;
            const unsigned j = q / ni, i = q - j * ni;
            const long long c = (long long)j * pitch + i;
            for (int k = 0; k < 4; ++k) dst[c + k * plane] = v[e][k];
            if constexpr (RATE) {
                if (G.soff >= 0 && ro.solid[G.soff + q]) continue;
                const GridCoef<T> &K = ro.coef[g];
                CellGeom<T> cg;
                if constexpr (CURV) {
                    const T *vx = ro.vdx + G.voff, *vy = ro.vdy + G.voff;
                    const long long b = (long long)j * G.vpitch + i;
                    cg = cell_geom(vx[b], vx[b + 1], vx[b + G.vpitch], vx[b + G.vpitch + 1], vy[b], vy[b + 1],
                                   vy[b + G.vpitch], vy[b + G.vpitch + 1], K.dx, K.dy);
                } else {
                    cg.Xx = K.dy; cg.Xy = T(0); cg.Yx = T(0); cg.Yy = K.dx; cg.V = K.V;
                }
                m = vmax(m, cell_rate<CURV>(cell_prims(v[e][0], v[e][1], v[e][2], v[e][3], K), cg, K));
            }
        }
    }
    if constexpr (RATE) {
        m = block_max<256>(m, red);
        if (threadIdx.x == 0 && m > T(0)) atomicMax(ro.rate + g, rate_bits(m));
    }
}

template <typename T, typename H>
__global__ void __launch_bounds__(256) unpack_kernel(const GridDev *grids, int g_lo, const T *__restrict__ U,
                                                     H *__restrict__ packed, long long u_shift, long long p_shift)
{
    const GridDev &G = grids[g_lo + blockIdx.y];
    const unsigned ni = (unsigned)G.ni, n = ni * (unsigned)G.nj, stride = gridDim.x * 256u;
    const T *__restrict__ src = U + (G.off - u_shift);
    H *__restrict__ dst = packed + (G.poff - p_shift);
    const long long pitch = G.pitch, plane = G.plane;
    for (unsigned q0 = blockIdx.x * 256u + threadIdx.x; q0 < n; q0 += IO_PER * stride) {
        T v[IO_PER][4];
#pragma unroll
        for (int e = 0; e < IO_PER; ++e) {
            const unsigned q = q0 + e * stride;
            if (q < n) {
                const unsigned j = q / ni, i = q - j * ni;
                const long long c = (long long)j * pitch + i;
                for (int k = 0; k < 4; ++k) v[e][k] = src[c + k * plane];
            }
        }
#pragma unroll
        for (int e = 0; e < IO_PER; ++e) {
            const unsigned q = q0 + e * stride;
            if (q < n)
                for (int k = 0; k < 4; ++k) dst[(long long)k * n + q] = (H)v[e][k];
        }
    }
}

// FP64 block partials of sum V Q over the fluid cells of grid g (4 doubles per block).
template <typename T, bool CURV>
__global__ void __launch_bounds__(256) totals_kernel(const GridDev *grids, const GridCoef<T> *coef, int g, const T *U,
                                                     const T *vdx, const T *vdy, const uint8_t *solid,
                                                     double *partials)
{
    __shared__ double wred[8][4];
    const GridDev &G = grids[g];
    const GridCoef<T> K = coef[g];
    const long long n = (long long)G.ni * G.nj;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long q = (long long)blockIdx.x * 256 + threadIdx.x; q < n; q += (long long)gridDim.x * 256) {
        const int i = (int)(q % G.ni), j = (int)(q / G.ni);
        if (G.soff >= 0 && solid[G.soff + q]) continue;
        double V;
        if (CURV) {
            const long long b = G.voff + (long long)j * G.vpitch + i;
            V = (double)cell_geom(vdx[b], vdx[b + 1], vdx[b + G.vpitch], vdx[b + G.vpitch + 1], vdy[b], vdy[b + 1],
                                  vdy[b + G.vpitch], vdy[b + G.vpitch + 1], K.dx, K.dy).V;
        } else {
            V = G.dx * G.dy;
        }
        const long long c = G.off + (long long)j * G.pitch + i;
        for (int k = 0; k < 4; ++k) s[k] = fma(V, (double)U[c + k * G.plane], s[k]);
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
template <typename T, bool MUSCL, bool CURV, bool WALLS, bool ABL = false> struct StageVariant {
    static constexpr int NT = STAGE_THREADS;
    static cudaError_t launch(const StageArgs<T> &a, int nblocks, cudaStream_t s)
    {
        const size_t smem = a.mode == MODE_NORM ? 8 * NT * sizeof(double) : 0;   // (the norm accumulators)
        stage_kernel<T, MUSCL, CURV, WALLS, NT, ABL><<<nblocks, NT, smem, s>>>(a);
        return cudaGetLastError();
    }
    static int occupancy()
    {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage_kernel<T, MUSCL, CURV, WALLS, NT, ABL>, NT, 0) !=
            cudaSuccess)
            return 1;
        return n > 0 ? n : 1;
    }
};

template <typename T, bool MUSCL, bool CURV>
static cudaError_t stage_walls(const StageArgs<T> &a, int walls, int nblocks, cudaStream_t s)
{
    return walls ? StageVariant<T, MUSCL, CURV, true>::launch(a, nblocks, s)
                 : StageVariant<T, MUSCL, CURV, false>::launch(a, nblocks, s);
}
template <typename T, bool MUSCL, bool CURV>
static int occ_walls(int walls)
{
    return walls ? StageVariant<T, MUSCL, CURV, true>::occupancy() : StageVariant<T, MUSCL, CURV, false>::occupancy();
}

template <typename T>
cudaError_t Launchers<T>::stage(const StageArgs<T> &a, int muscl, int curv, int kind, int nblocks, cudaStream_t s)
{
    if (a.tile_hi <= a.tile_lo) return cudaSuccess;
    if (kind == KIND_ABLATION) return AblationLaunchers<T>::stage(a, muscl, curv, nblocks, s);
    const int walls = kind == KIND_WALLS;
    if (muscl) return curv ? stage_walls<T, true, true>(a, walls, nblocks, s) : stage_walls<T, true, false>(a, walls, nblocks, s);
    return curv ? stage_walls<T, false, true>(a, walls, nblocks, s) : stage_walls<T, false, false>(a, walls, nblocks, s);
}

template <typename T>
int Launchers<T>::stage_occupancy(int muscl, int curv, int kind)
{
    if (kind == KIND_ABLATION) return AblationLaunchers<T>::stage_occupancy(muscl, curv);
    const int walls = kind == KIND_WALLS;
    if (muscl) return curv ? occ_walls<T, true, true>(walls) : occ_walls<T, true, false>(walls);
    return curv ? occ_walls<T, false, true>(walls) : occ_walls<T, false, false>(walls);
}

// The ablation kernels handle walls and solid cells too (every face takes the scalar path).
template <typename T>
cudaError_t AblationLaunchers<T>::stage(const StageArgs<T> &a, int muscl, int curv, int nblocks, cudaStream_t s)
{
    if (a.tile_hi <= a.tile_lo) return cudaSuccess;
    if (muscl)
        return curv ? StageVariant<T, true, true, true, true>::launch(a, nblocks, s)
                    : StageVariant<T, true, false, true, true>::launch(a, nblocks, s);
    return curv ? StageVariant<T, false, true, true, true>::launch(a, nblocks, s)
                : StageVariant<T, false, false, true, true>::launch(a, nblocks, s);
}

template <typename T>
int AblationLaunchers<T>::stage_occupancy(int muscl, int curv)
{
    if (muscl)
        return curv ? StageVariant<T, true, true, true, true>::occupancy()
                    : StageVariant<T, true, false, true, true>::occupancy();
    return curv ? StageVariant<T, false, true, true, true>::occupancy()
                : StageVariant<T, false, false, true, true>::occupancy();
}

// IO_PER cells per thread of a block of 256 for the largest grid (one pass over it), at most
// 1024 blocks per grid.
static inline int io_blocks(int max_cells)
{
    const int bx = (max_cells + 256 * IO_PER - 1) / (256 * IO_PER);
    return bx < 1 ? 1 : (bx > 1024 ? 1024 : bx);
}

template <typename T, typename H>
static cudaError_t launch_pack(const GridDev *grids, int g_lo, int g_hi, int max_cells, const H *packed, T *U,
                               cudaStream_t s, long long p_shift, const RateOut<T> *ro)
{
    if (g_hi <= g_lo) return cudaSuccess;
    const dim3 grid(io_blocks(max_cells), g_hi - g_lo);
    if (!ro) pack_kernel<T, H, false, false><<<grid, 256, 0, s>>>(grids, g_lo, packed, U, p_shift, RateOut<T>());
    else if (ro->curv) pack_kernel<T, H, true, true><<<grid, 256, 0, s>>>(grids, g_lo, packed, U, p_shift, *ro);
    else pack_kernel<T, H, true, false><<<grid, 256, 0, s>>>(grids, g_lo, packed, U, p_shift, *ro);
    return cudaGetLastError();
}

template <typename T, typename H>
static cudaError_t launch_unpack(const GridDev *grids, int g_lo, int g_hi, int max_cells, const T *U, H *packed,
                                 cudaStream_t s, long long u_shift, long long p_shift)
{
    if (g_hi <= g_lo) return cudaSuccess;
    unpack_kernel<T, H><<<dim3(io_blocks(max_cells), g_hi - g_lo), 256, 0, s>>>(grids, g_lo, U, packed, u_shift,
                                                                                 p_shift);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launchers<T>::pack(const GridDev *grids, int g_lo, int g_hi, int max_cells, const double *packed, T *U,
                               cudaStream_t s, long long p_shift, const RateOut<T> *ro)
{
    return launch_pack<T, double>(grids, g_lo, g_hi, max_cells, packed, U, s, p_shift, ro);
}
template <typename T>
cudaError_t Launchers<T>::pack(const GridDev *grids, int g_lo, int g_hi, int max_cells, const float *packed, T *U,
                               cudaStream_t s, long long p_shift, const RateOut<T> *ro)
{
    return launch_pack<T, float>(grids, g_lo, g_hi, max_cells, packed, U, s, p_shift, ro);
}

template <typename T>
cudaError_t Launchers<T>::unpack(const GridDev *grids, int g_lo, int g_hi, int max_cells, const T *U, double *packed,
                                 cudaStream_t s, long long u_shift, long long p_shift)
{
    return launch_unpack<T, double>(grids, g_lo, g_hi, max_cells, U, packed, s, u_shift, p_shift);
}
template <typename T>
cudaError_t Launchers<T>::unpack(const GridDev *grids, int g_lo, int g_hi, int max_cells, const T *U, float *packed,
                                 cudaStream_t s, long long u_shift, long long p_shift)
{
    return launch_unpack<T, float>(grids, g_lo, g_hi, max_cells, U, packed, s, u_shift, p_shift);
}

template <typename T>
cudaError_t Launchers<T>::totals(const GridDev *grids, const GridCoef<T> *coef, int g, const T *U, const T *vdx,
                                 const T *vdy, const uint8_t *solid, double *partials, int nblocks, int curv,
                                 cudaStream_t s)
{
    if (curv) totals_kernel<T, true><<<nblocks, 256, 0, s>>>(grids, coef, g, U, vdx, vdy, solid, partials);
    else totals_kernel<T, false><<<nblocks, 256, 0, s>>>(grids, coef, g, U, vdx, vdy, solid, partials);
    return cudaGetLastError();
}

}  // namespace roeam
