// roeam_internal.h — device-side descriptors and launch entry points shared by the
// library's host code (roeam_api.cu) and its kernel translation units (roeam_k32.cu,
// roeam_k64.cu and their ablation-variant companions). Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace roeam {

constexpr int BC_PERIODIC = 0, BC_WALL = 1, BC_INFLOW = 2, BC_OUTFLOW = 3, BC_EXCHANGE = 4;

// Status bits raised by kernels (read back by the host at synchronising calls).
constexpr unsigned ST_NONPOSITIVE = 1u, ST_NONFINITE = 2u;
constexpr unsigned ST_BOUNDS = 4u;   // an index outside its buffer (bounds-checked debug builds only)

// Per-grid descriptor, resident in device memory, read-only in kernels.
struct GridDev {
    long long off;    // element offset of this grid's row 0 of variable 0 in the state buffers
    long long plane;  // elements per variable plane (nj * pitch; (nj + 4) * pitch with an
                      // EXCHANGE side, whose planes also hold the ghost rows j = -2, -1, nj, nj+1)
    long long voff;   // element offset of this grid's vertex displacement planes (-1: Cartesian)
    long long soff;   // byte offset of this grid's solid mask (-1: none)
    long long poff;   // element offset of this grid in the packed host layout [4][nj][ni]
    int ni, nj, pitch, vpitch;
    int ntx, nty, tile_base, ntiles;
    int bc[4];        // W, E, S, N
    int limiter;      // 1 minmod, 2 van Leer (MUSCL kernels)
    int eps1, use_s1, xi_form;
    int scheme, dup_mode, ufix, xi_roe;   // ablation variants (0, 0, 1, 0: Roe-AM)
    double inflow[4]; // rho, u, v, p
    double gamma, m_ref, u_ref, eps2;
    double harten;    // classical Roe: eps_lambda of the entropy fix (0: none)
    double dx, dy;    // Cartesian spacings / reference-grid spacings of a curvilinear grid
    double nfluid;    // number of fluid cells
};

enum Mode { MODE_STAGE = 0, MODE_RESIDUAL = 1, MODE_NORM = 2 };

// Per-grid constants in the working precision, computed once on the host so that the
// FP32 kernels execute no FP64 arithmetic on their hot path.
template <typename T>
struct GridCoef {
    T g, gm1, gm1i, hgm1, mr2, rr_thr, eps2;   // gamma, gamma-1, 1/(gamma-1), (gamma-1)/2, M_ref^2, 1e-5 U_ref, eps2
    T dx, dy, V, Vi;                     // spacings (reference spacings if curvilinear), dx*dy, 1/(dx*dy)
    T idx, idy;                          // 1/dx, 1/dy (Cartesian)
    T inflow[4];                         // rho, u, v, p of INFLOW sides
    T harten;                            // classical Roe: eps_lambda (0: no entropy fix)
};

template <typename T>
struct StageArgs {
    const GridDev *grids;
    const GridCoef<T> *coef;
    const int4 *units;      // work units: (grid, column of lane 0, first row, end row)
    int ngrids;
    int tile_lo, tile_hi;   // work units [tile_lo, tile_hi) of the batch processed by this launch
    const T *src;           // U^(k): the state whose residual is evaluated (halo source)
    const T *un;            // U^n for the stage combination
    T *dst;                 // stage output, or the residual in MODE_RESIDUAL
    long long dst_shift;    // grid g's output starts at dst + (G.off - dst_shift) (0: the state layout)
    const T *vdx, *vdy;     // vertex displacement planes (curvilinear grids)
    const uint8_t *solid;   // solid masks
    T alpha, beta;          // dst = alpha * U^n + beta * (U^(k) + dt R(U^(k)))
    int mode;
    int want_rate;          // write each grid's max signal-speed rate of dst into rate_wr
    const unsigned long long *rate_rd;  // per-grid max rate of U^n (working-precision bits)
    unsigned long long *rate_wr;        // per-grid max rate of the stage output
    unsigned long long *rate_zero;      // per-grid slots to reset (the next step's rate_wr), may be null
    double cfl, dt_fixed;
    T cfl_t, dt_fixed_t;    // the same in the working precision
    unsigned *status;
    double *partials;       // MODE_NORM: gridDim.x * 8 (sum R^2 [4], max |R| [4])
    // Dynamic unit scheduling (null: static round robin): work[0] counts the units claimed past
    // each warp's first, work[1] the warps that have finished; the last warp to finish resets
    // both, so that the next launch on the handle's stream starts from zero.
    unsigned *work;
#ifdef ROEAM_DEBUG
    // buffer sizes (elements of each state buffer and of dst, of each vertex plane buffer; bytes of
    // the solid masks), read by the bounds checks of debug builds
    long long n_state, n_dst, n_vert, n_solid;
#endif
};

// Work-unit shapes of the stage kernel: a warp sweeps a strip tx = 32 lanes wide (2H of
// them halo) over ty rows; nt threads per CTA. The autotuner picks among these.
// One warp per CTA: registers are then allocated warp by warp, so every 8 registers saved
// per thread buys another resident warp.
#ifndef STAGE_THREADS_DEF
#define STAGE_THREADS_DEF 32
#endif
constexpr int STAGE_THREADS = STAGE_THREADS_DEF;
// Resident CTAs per SM the compiler is asked to fit (register budget): 13 keeps the FP32
// first-order Cartesian kernel at 128 registers without spills (16 warps per SM); the
// reconstructing and curvilinear FP32 variants are held to 128 registers as well (16 warps
// per SM: the 4096^2 warped step runs 10 % faster than at 168 registers and 12 warps, although
// it spills 60 bytes there); FP64 and the ablation variants are left to the compiler.
#ifndef STAGE_MIN_BLOCKS_FAST
#define STAGE_MIN_BLOCKS_FAST 13
#endif
#ifndef STAGE_MIN_BLOCKS_OTHER
#define STAGE_MIN_BLOCKS_OTHER 16
#endif
template <typename T, bool MUSCL, bool CURV, bool ABL = false>
constexpr int stage_min_blocks()
{
    return (sizeof(T) != 4 || ABL) ? 1 : ((!MUSCL && !CURV) ? STAGE_MIN_BLOCKS_FAST : STAGE_MIN_BLOCKS_OTHER);
}
// dyn: dynamic unit scheduling (the kernels that support it claim units from a counter after
// their first; 0 = static round robin over the unit table).
struct TileCfg { int tx, ty, nt, dyn; };
constexpr int NUM_TILE_CFGS = 10;
constexpr TileCfg TILE_CFGS[NUM_TILE_CFGS] = {
    {32, 32, STAGE_THREADS, 1}, {32, 64, STAGE_THREADS, 1}, {32, 16, STAGE_THREADS, 1}, {32, 128, STAGE_THREADS, 1},
    {32, 256, STAGE_THREADS, 1}, {32, 32, STAGE_THREADS, 0}, {32, 64, STAGE_THREADS, 0}, {32, 16, STAGE_THREADS, 0},
    {32, 128, STAGE_THREADS, 0}, {32, 256, STAGE_THREADS, 0}};
// Whether a stage-kernel family claims units dynamically when asked to (the reconstructing
// curvilinear kernels keep the static round robin).
__host__ __device__ constexpr bool stage_dynamic(int muscl, int curv) { return !(muscl && curv); }

// Stage-kernel families: no walls anywhere in the batch; some WALL side or solid cells; some
// grid uses an ablation variant of the flux (every face on the scalar path).
enum StageKind { KIND_PLAIN = 0, KIND_WALLS = 1, KIND_ABLATION = 2 };

// What a pack needs to take the time-step rate of the state it writes: the grids' coefficients,
// vertex displacements and solid masks, and the rate slots it raises with atomicMax.
template <typename T> struct RateOut {
    const GridCoef<T> *coef = nullptr;
    const T *vdx = nullptr, *vdy = nullptr;
    const uint8_t *solid = nullptr;
    unsigned long long *rate = nullptr;
    int curv = 0;
};

template <typename T>
struct Launchers {
    // Fused face-flux / residual / stage kernel over tiles [tile_lo, tile_hi).
    static cudaError_t stage(const StageArgs<T> &a, int muscl, int curv, int kind, int nblocks, cudaStream_t s);
    // Largest resident CTAs per SM of a stage-kernel variant (for persistent launches).
    static int stage_occupancy(int muscl, int curv, int kind);
    // Packed float64 [4][nj][ni] per grid <-> pitched working-precision planes.
    // (pack reads grid g at packed + G.poff - p_shift; the host-side layout in float64 or float;
    //  with ro it also writes the packed state's rate into ro->rate[g], zeroed by the caller)
    static cudaError_t pack(const GridDev *grids, int g_lo, int g_hi, int max_cells, const double *packed, T *U,
                            cudaStream_t s, long long p_shift = 0, const RateOut<T> *ro = nullptr);
    static cudaError_t pack(const GridDev *grids, int g_lo, int g_hi, int max_cells, const float *packed, T *U,
                            cudaStream_t s, long long p_shift = 0, const RateOut<T> *ro = nullptr);
    // (unpack reads grid g at U + G.off - u_shift and writes it at packed + G.poff - p_shift)
    static cudaError_t unpack(const GridDev *grids, int g_lo, int g_hi, int max_cells, const T *U, double *packed,
                              cudaStream_t s, long long u_shift = 0, long long p_shift = 0);
    static cudaError_t unpack(const GridDev *grids, int g_lo, int g_hi, int max_cells, const T *U, float *packed,
                              cudaStream_t s, long long u_shift = 0, long long p_shift = 0);
    // FP64 block partials of sum V*U over the fluid cells of one grid (gridDim.x * 4 doubles).
    static cudaError_t totals(const GridDev *grids, const GridCoef<T> *coef, int g, const T *U, const T *vdx,
                              const T *vdy, const uint8_t *solid, double *partials, int nblocks, int curv,
                              cudaStream_t s);
};

// The ablation-variant stage kernels, instantiated in their own translation units.
template <typename T>
struct AblationLaunchers {
    static cudaError_t stage(const StageArgs<T> &a, int muscl, int curv, int nblocks, cudaStream_t s);
    static int stage_occupancy(int muscl, int curv);
};

// The kernels' reciprocal, rsqrt and sqrt on n device values (n rows of 6 doubles; test hook).
cudaError_t launch_math_check(int n, const double *x, double *out, cudaStream_t s);

// Sets the thread's roeam_last_error() message and returns `status` (host).
int record_error(int status, const char *msg);

// Fixed-order reduction of nblocks x 8 norm partials into out[8] (sum[4], max[4]).
cudaError_t launch_reduce_partials(const double *partials, int nblocks, int width, double *out, cudaStream_t s);

}  // namespace roeam
