// roeam3_internal.h — device-side descriptors and launch entry points of the 3D path (Cartesian
// grids with passive scalars), shared by roeam3_api.cu and the 3D kernel translation units.
// Not part of the public ABI.
#pragma once

#include "roeam_internal.h"

namespace roeam {

constexpr int MAX_SCALARS = 3;
constexpr int MAX_VARS3 = 5 + MAX_SCALARS;

// Per-grid descriptor of a 3D grid, resident in device memory.
struct GridDev3 {
    long long off;     // element offset of this grid's variable-0 volume in the state buffers
    long long vol;     // elements per variable volume (nk * nj * pitch)
    long long poff;    // element offset of this grid in the packed host layout [nv][nk][nj][ni]
    int ni, nj, nk, pitch;
    int bc[6];         // W, E, S, N, B, T
    int eps1, use_s1, xi_form, pad_;
    double inflow[MAX_VARS3];   // rho, u, v, w, p, k_1..
    double gamma, m_ref, u_ref, eps2;
    double dx, dy, dz;
};

// Per-grid constants in the working precision.
template <typename T>
struct GridCoef3 {
    T g, gm1, gm1i, hgm1, mr2, rr_thr, eps2;
    T ax, ay, az, Vi;            // face areas dy dz, dx dz, dx dy; 1 / (dx dy dz)
    T idx, idy, idz;             // 1/dx, 1/dy, 1/dz
    T inflow[MAX_VARS3];
};

// Work-unit shape of the 3D stage kernel: a CTA of ty3<T>() warps covers 32 columns (30
// written) by ty3<T>() rows (two fewer written) and marches along z over a segment of planes.
// FP32 takes 16-row tiles, one 512-thread CTA per SM at 128 registers (30 x 14 of its 32 x 16
// cells written; 8-row tiles, two CTAs per SM, write 30 x 6 of 32 x 8 and measured 3.4 % slower
// on the 256^3 Taylor-Green vortex); FP64, which needs up to 255 registers, 8-row tiles.
#ifndef ROEAM_TY3_F32
#define ROEAM_TY3_F32 16
#endif
#ifndef ROEAM_TY3_F64
#define ROEAM_TY3_F64 8
#endif
template <typename T> __host__ __device__ constexpr int ty3() { return sizeof(T) == 4 ? ROEAM_TY3_F32 : ROEAM_TY3_F64; }
template <typename T> __host__ __device__ constexpr int tile3_y() { return ty3<T>() - 2; }
constexpr int TILE3_X = 30;

template <typename T>
struct StageArgs3 {
    const GridDev3 *grids;
    const GridCoef3<T> *coef;
    const int4 *units;       // (grid, column of lane 0 + 1, row of warp 0 + 1, k0 | k1 << 16)
    int ngrids, nunits;
    const T *src, *un;
    T *dst;
    T alpha, beta;
    int mode;                // MODE_STAGE or MODE_RESIDUAL
    int want_rate;
    const unsigned long long *rate_rd;
    unsigned long long *rate_wr, *rate_zero;
    T cfl_t, dt_fixed_t;
    unsigned *status;
};

template <typename T>
struct Launchers3 {
    static cudaError_t stage(const StageArgs3<T> &a, int nscal, int nblocks, cudaStream_t s);
    static int stage_occupancy(int nscal);
    static cudaError_t rate(const GridDev3 *grids, const GridCoef3<T> *coef, int g_lo, int g_hi, const T *U, int nscal,
                            unsigned long long *rate, cudaStream_t s);
    static cudaError_t pack(const GridDev3 *grids, int g_lo, int g_hi, int nv, long long max_cells,
                            const double *packed, T *U, cudaStream_t s);
    static cudaError_t unpack(const GridDev3 *grids, int g_lo, int g_hi, int nv, long long max_cells, const T *U,
                              double *packed, cudaStream_t s);
    static cudaError_t totals(const GridDev3 *grids, int g, const T *U, int nv, double *partials, int nblocks,
                              cudaStream_t s);
};

}  // namespace roeam
