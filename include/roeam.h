/*
 * roeam.h — C ABI of the GB300 (sm_103a) Roe-AM finite-volume library.
 *
 * The library advances the 2D compressible Euler equations (the 2D form of Eq. 1 of
 * Li, Ren & Gu, "An improved Roe scheme for all Mach-number flows simultaneously
 * curing known problems") on structured Cartesian or curvilinear grids with the
 * Roe-AM numerical flux of Section 6.2 (Eqs. 85-109), a cell-centred finite-volume
 * residual and a three-stage SSP Runge-Kutta update. Every step of that path runs
 * in the library's CUDA kernels on one GPU.
 *
 * Conventions used by every call:
 *   - A handle holds a batch of `count` >= 1 independent grids that advance together.
 *     All grids of one handle share the precision, the reconstruction order
 *     (first order vs MUSCL) and the geometry kind (Cartesian vs curvilinear).
 *   - Host state arrays are float64, structure of arrays, shape [4][nj][ni] with i
 *     fastest, variables (rho, rho*u, rho*v, rho*E). With grid_idx = -1 the call
 *     covers every grid of the batch, concatenated in grid order.
 *   - Host arrays are owned by the caller and only read/written during the call
 *     (the library copies them; page-locked memory makes the copies asynchronous-fast).
 *     All device memory belongs to the handle and is released by roeam_destroy_grid.
 *   - Calls return a status code; nothing crosses the ABI as an exception. After a
 *     non-OK status, roeam_last_error() gives a human-readable message (thread-local).
 *   - Errors raised on the device (non-positive or non-finite state after a step) are
 *     reported by the next call that synchronises with the GPU (get_state,
 *     residual_norm, conserved_totals, check, rk_step with dt_last).
 *   - One host thread uses a handle at a time. Work is ordered on the CUDA stream
 *     given at creation (NULL: the legacy default stream).
 */
#ifndef ROEAM_H
#define ROEAM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct roeam_grid roeam_grid; /* opaque batch handle */

typedef enum {
    ROEAM_OK = 0,
    ROEAM_E_ARG = 1,          /* invalid argument (message says which) */
    ROEAM_E_CUDA = 2,         /* a CUDA runtime call failed */
    ROEAM_E_OOM = 3,          /* device allocation failed */
    ROEAM_E_NONPOSITIVE = 4,  /* density or pressure <= 0 after a step */
    ROEAM_E_NONFINITE = 5,    /* NaN or Inf in the state after a step */
    ROEAM_E_TIMEOUT = 6,      /* a bounded device wait gave up */
    ROEAM_E_STATE = 7,        /* call not valid in the handle's current state */
    ROEAM_E_BOUNDS = 8        /* a kernel index left its buffer (only libraries built with
                                 ROEAM_DEBUG check; the access was skipped, nothing trapped) */
} roeam_status;

enum { ROEAM_BC_PERIODIC = 0, ROEAM_BC_WALL = 1, ROEAM_BC_INFLOW = 2, ROEAM_BC_OUTFLOW = 3, ROEAM_BC_EXCHANGE = 4 };
enum { ROEAM_RECON_FIRST = 0, ROEAM_RECON_MINMOD = 1, ROEAM_RECON_VANLEER = 2 };
enum { ROEAM_NORM_L2 = 0, ROEAM_NORM_LINF = 1 };

/* Scheme parameters (Section 6.2).
 *   gamma    ratio of specific heats (> 1).
 *   m_ref    global reference Mach number M_ref of Eq. 101 (> 0).
 *   u_ref    reference speed U_ref of Eq. 108 (> 0); sets the rotated-direction threshold.
 *   eps2     entropy-fix constant of Eqs. 102 and 112 (suggested 0.05).
 *   eps1     0 or 1 (Eq. 111): 1 adds the entropy-fix / rotated-Riemann floor of Eq. 86.
 *   use_s1   1 evaluates the pressure-density detector s1 of Eqs. 95-97; 0 sets s1 = 1 (Eq. 110).
 *   recon    ROEAM_RECON_*: first order, or MUSCL on primitive variables with the minmod
 *            or van Leer limiter (a face whose reconstructed rho or p is not positive
 *            falls back to first order).
 *   xi_form  0: xi of Eq. 86 with the [1 - f^8(Mbar)] factor of Eq. 68 on dU/2 (exact
 *            full upwinding for supersonic faces, Eq. 44); 1: Eq. 86 as printed.
 *   precision 32 (state and flux arithmetic in FP32; FP64 reductions) or 64.
 *
 * Ablation variants (the schemes Section 7 compares Roe-AM with; zero everywhere gives
 * Roe-AM as defined above). A batch whose grids use any of them runs a slower kernel that
 * evaluates every face on its scalar path.
 *   scheme   ROEAM_SCHEME_ROEAM, or ROEAM_SCHEME_ROE: the classical Roe flux (Eq. 7 with the
 *            eigenvalue forms of Eqs. 8-12, Delta(rho E) in the xi term). The flux then ignores
 *            m_ref, eps1, eps2, use_s1 and xi_form, the time-step rule becomes the classical
 *            |U| + c (theta = 1), and dup_mode, no_ufix and xi_roe must be 0.
 *   harten   classical Roe only: eps_lambda of the entropy fix of Eqs. 114-115, in [0, 1)
 *            (0 = no fix).
 *   dup_mode Roe-AM delta U_p: ROEAM_DUP_ROEAM (Eq. 89), ROEAM_DUP_ZERO, or ROEAM_DUP_ROE
 *            (max(0, c - |U|) dp / (rho c^2), the classical term of Eq. 17).
 *   no_ufix  1: |U|' = |U| (Roe-AM without the expansion-shock fix of Eq. 92).
 *   xi_roe   1: xi = |U| (Eq. 13) instead of Eq. 86.
 * Out-of-range values give ROEAM_E_ARG. */
enum { ROEAM_SCHEME_ROEAM = 0, ROEAM_SCHEME_ROE = 1 };
enum { ROEAM_DUP_ROEAM = 0, ROEAM_DUP_ZERO = 1, ROEAM_DUP_ROE = 2 };
typedef struct {
    double gamma, m_ref, u_ref, eps2;
    int eps1, use_s1, recon, xi_form;
    int precision;
    int scheme, dup_mode, no_ufix, xi_roe;
    int reserved_;   /* must be 0 */
    double harten;
} roeam_params;

/* One grid of ni x nj cells.
 *   bc[4]      boundary type of the W (i = 0), E (i = ni-1), S (j = 0), N (j = nj-1) sides.
 *              PERIODIC must be set on both sides of a direction. WALL mirrors the
 *              adjacent state about the face normal; INFLOW imposes `inflow`;
 *              OUTFLOW copies the adjacent state (zero gradient). EXCHANGE (S and N only)
 *              takes the two ghost rows beyond the side from roeam_set_halo: the grid is a row
 *              slab of a larger grid whose neighbouring slab lives elsewhere (another GPU).
 *   inflow     (rho, u, v, p) used by INFLOW sides.
 *   xv, yv     host float64 vertex coordinates, shape [nj+1][ni+1], or both NULL for a
 *              Cartesian grid with spacings dx, dy (> 0). For curvilinear grids dx, dy >= 0
 *              give the uniform reference grid x = i*dx, y = j*dy that the library stores
 *              the vertices relative to (the displacement from it is kept in the working
 *              precision): the mean spacings for a gently warped grid; 0, 0 (absolute
 *              coordinates) for grids such as O-grids, whose cells shrink towards the
 *              origin. Every cell must have positive area (the vertex order turns
 *              counter-clockwise from +i to +j), else ROEAM_E_ARG. A periodic direction
 *              should repeat its first vertex column (row) in the last one up to the
 *              period shift, bit for bit after the subtraction of the reference grid, so
 *              that both sides of the seam see the same face.
 *   solid      host uint8 mask [nj][ni] (1 = solid wall cell, never updated) or NULL.
 *              Solid cells may not be combined with PERIODIC in the same direction. A grid
 *              with an EXCHANGE side takes the mask rows beyond it from roeam_set_halo_solid. */
typedef struct {
    int ni, nj;
    int bc[4];
    double inflow[4];
    const double *xv, *yv;
    double dx, dy;
    const uint8_t *solid;
    roeam_params p;
} roeam_grid_desc;

/* Creates a batch handle of `count` (1..65535) grids on CUDA device `device`, ordering its work on
 * `cuda_stream` (a cudaStream_t, or NULL). Copies every descriptor array. The state is
 * zero until roeam_set_state. On success *out receives the handle. */
roeam_status roeam_create_grid(int count, const roeam_grid_desc *descs, int device, void *cuda_stream,
                               roeam_grid **out);

/* Releases the handle and all its device memory. NULL is ignored. */
void roeam_destroy_grid(roeam_grid *g);

/* Copies the conserved state of grid `grid_idx` (or all grids with -1) from the host,
 * converting to the handle's precision, and refreshes the time-step estimate. */
roeam_status roeam_set_state(roeam_grid *g, int grid_idx, const double *cons);

/* Copies the conserved state of grid `grid_idx` (or all grids) to the host as float64.
 * Synchronises; reports pending device errors. */
roeam_status roeam_get_state(roeam_grid *g, int grid_idx, double *cons_out);

/* Device-pointer forms of roeam_set_state / roeam_get_state, for callers whose state already
 * lives on the GPU (a PyTorch tensor, another solver's buffer): the paper has no counterpart;
 * the survey of this library's interface lists them as the optional device variants of the
 * state calls. cons_dev / cons_out_dev is float64 device memory of the handle's device (or
 * managed memory), 8-byte aligned, laid out like the host arrays ([4][nj][ni] per grid, grids
 * concatenated for grid_idx = -1); the caller owns it. cuda_stream (a cudaStream_t, or NULL
 * for the legacy default stream) orders the call with the caller's work: what the caller
 * submitted to it before the call completes before the library reads (set) or writes (get)
 * the array, and what the caller submits to it afterwards runs after the library has
 * finished with the array. The host does not wait; device errors of earlier steps are
 * reported by the next synchronising call. Wrong pointers (host memory, another device,
 * misaligned) give ROEAM_E_ARG. set refreshes the time-step estimate like roeam_set_state. */
roeam_status roeam_set_state_device(roeam_grid *g, int grid_idx, const double *cons_dev, void *cuda_stream);
roeam_status roeam_get_state_device(roeam_grid *g, int grid_idx, double *cons_out_dev, void *cuda_stream);

/* Evaluates the finite-volume residual R(U) = -(1/V) sum_f F_f |S_f| (outward faces,
 * Roe-AM flux of Eqs. 85-109) of grid `grid_idx` (or all) for the current state and
 * copies it to res_out (same layout as the state; solid cells get 0). res_out may be
 * NULL (the residual is then only computed). Synchronises when res_out is not NULL. */
roeam_status roeam_flux_residual(roeam_grid *g, int grid_idx, double *res_out);

/* Advances every grid by nsteps SSP-RK3 steps (Shu & Osher; each stage one fused kernel:
 * face fluxes, residual, stage combination). Each grid's dt is dt_fixed if > 0, else
 * cfl / max_i sum_dir (|U| + max(c, c~/theta))|S_dir| / V_i evaluated on the state at the
 * start of the step (theta, c~ of Eqs. 99-101; theta = 1 on classical-Roe grids).
 * dt_last (nullable, `count` doubles) receives each grid's dt of the last step (this
 * synchronises). */
roeam_status roeam_rk_step(roeam_grid *g, double cfl, double dt_fixed, int nsteps, double *dt_last);

/* Test hook (the paper has no counterpart): evaluates, on CUDA device `device`, the
 * reciprocal, reciprocal square root and square root that the kernels use, for n (1..2^24)
 * host values x > 0. out (6 n doubles) receives per value: 1/x, 1/sqrt(x), sqrt(x) in FP64,
 * then the same three in FP32 of (float)x. Used to check them against the IEEE operations. */
roeam_status roeam_math_check(int device, int n, const double *x, double *out);

/* Stage-by-stage stepping, for a grid split into row slabs over several GPUs (one handle per
 * slab, S/N sides between slabs of type EXCHANGE). One SSP-RK3 step is three calls, stage =
 * 0, 1, 2 in order, each advancing every grid of the handle with the same dt (> 0); between
 * them the caller refreshes the ghost rows of EXCHANGE sides: before stage s, copy the
 * neighbour's roeam_edge_rows(..., s, ...) into roeam_set_halo(..., s, ...). A step begun this way must be
 * finished before roeam_rk_step runs (ROEAM_E_STATE otherwise). The global time step is
 * CFL / max over all slabs of roeam_max_rate. */
roeam_status roeam_rk_stage(roeam_grid *g, int stage, double dt);

/* The same stage in two launches, so that a slab's ghost-row exchange can overlap its interior:
 * part ROEAM_PART_INTERIOR updates every cell whose stencil stays inside the grid (all but the
 * 1 (first order) or 2 (MUSCL) rows next to each EXCHANGE side), part ROEAM_PART_EDGES the rest;
 * the caller sets the ghost rows (roeam_set_halo) after the first and before the second. Called
 * in that order, the two parts give the same bits as ROEAM_PART_ALL (= roeam_rk_stage). */
enum { ROEAM_PART_ALL = 0, ROEAM_PART_INTERIOR = 1, ROEAM_PART_EDGES = 2 };
roeam_status roeam_rk_stage_part(roeam_grid *g, int stage, double dt, int part);

/* Per-grid largest signal-speed rate sum_dir (|U| + max(c, c~/theta))|S_dir| / V of the current
 * state (rate_out: `count` doubles); CFL / rate is the grid's time step. Synchronises and reports
 * pending device errors. */
roeam_status roeam_max_rate(roeam_grid *g, double *rate_out);

/* Copies the two rows of grid grid_idx nearest side (2 = S: rows 0, 1; 3 = N: rows nj-2, nj-1)
 * of the state that stage `stage` (0, 1, 2) reads (U^n, U1, U2) into dst, laid out
 * [4 variables][2 rows, j increasing][ni] in the handle's precision (float or double). dst may
 * be host or device memory; the copy is ordered on the handle's stream and, for host memory,
 * complete on return. */
roeam_status roeam_edge_rows(roeam_grid *g, int grid_idx, int side, int stage, void *dst);

/* Sets the two ghost rows beyond the EXCHANGE side `side` (2 = S: j = -2, -1; 3 = N: j = nj,
 * nj+1) of grid grid_idx, in the state that stage `stage` (0, 1, 2) reads, from src laid out
 * like roeam_edge_rows' output (host or device memory; ordered on the handle's stream and, for
 * host memory, complete on return, so the buffer may be reused at once). A grid
 * with an EXCHANGE side keeps these rows in its own state planes; they start at zero, so each
 * must be set before the stage that reads it. */
roeam_status roeam_set_halo(roeam_grid *g, int grid_idx, int side, int stage, const void *src);

/* Static ghost rows of a grid with an EXCHANGE side whose neighbouring slab has solid cells or
 * curvilinear geometry (set once, after roeam_create_grid; they do not change from step to step).
 *   roeam_set_halo_solid: the solid-mask rows beyond side `side` (2 = S: rows j = -2, -1; 3 = N:
 *     rows nj, nj+1), host uint8 [2][ni], j increasing. The grid must have a solid mask (pass an
 *     all-zero one if its own cells are all fluid). Without it the ghost rows are fluid.
 *   roeam_set_halo_vertices: the vertex rows beyond side `side` (2 = S: J = -2, -1; 3 = N:
 *     J = nj+1, nj+2), host float64 [2][ni+1] each, J increasing, in the coordinates of the
 *     grid's own xv, yv (the library stores them relative to the reference grid x = I dx,
 *     y = J dy like the others). Curvilinear handles only. Without it the ghost vertices sit on
 *     the reference grid. They give the normals of the faces beyond the side (mirror images of
 *     solid reconstruction-stencil cells, wall ghost cells of the W/E sides in the ghost rows).
 * Both copy synchronously and return ROEAM_E_ARG for a side that is not EXCHANGE. */
roeam_status roeam_set_halo_solid(roeam_grid *g, int grid_idx, int side, const uint8_t *rows);
roeam_status roeam_set_halo_vertices(roeam_grid *g, int grid_idx, int side, const double *xv, const double *yv);

/* The host-resident form of a step: loads every grid from cons_in (host float64, the layout of
 * roeam_set_state with grid_idx = -1), advances nsteps SSP-RK3 steps as roeam_rk_step does, and
 * writes the result to cons_out (same layout; it may equal cons_in), overlapping the copies
 * with the computation: the grids go through in ten chunks of whole grids, small at both ends
 * (about 1:2:3:4:4:4:4:3:2:1 of the cells), on three internal streams (copies in, computation,
 * copies out), so that one chunk is copied in while the one before it is stepped and an earlier
 * one is copied out.
 * Page-locked host arrays make the copies asynchronous. The device state afterwards equals
 * cons_out. dt_last as in roeam_rk_step. Synchronises; reports device errors. */
roeam_status roeam_step_host(roeam_grid *g, double cfl, double dt_fixed, int nsteps, const double *cons_in,
                             double *cons_out, double *dt_last);

/* Single-precision host arrays: the same calls as roeam_set_state, roeam_get_state and
 * roeam_step_host with float [4][nj][ni] host arrays (the paper has no counterpart). For an
 * FP32 handle nothing is lost, the state being FP32, and half the bytes of the float64 calls
 * cross the host link; an FP64 handle widens the input and rounds the output. */
roeam_status roeam_set_state_f32(roeam_grid *g, int grid_idx, const float *cons);
roeam_status roeam_get_state_f32(roeam_grid *g, int grid_idx, float *cons_out);
roeam_status roeam_step_host_f32(roeam_grid *g, double cfl, double dt_fixed, int nsteps, const float *cons_in,
                                 float *cons_out, double *dt_last);

/* FP64 norm of the residual R(U) of grid `grid_idx` over its fluid cells, per variable:
 * kind ROEAM_NORM_L2 gives sqrt(mean R^2), ROEAM_NORM_LINF gives max |R|. Synchronises. */
roeam_status roeam_residual_norm(roeam_grid *g, int grid_idx, int kind, double out[4]);

/* FP64 conserved totals sum_i V_i Q_i over the fluid cells of grid `grid_idx`. Synchronises. */
roeam_status roeam_conserved_totals(roeam_grid *g, int grid_idx, double out[4]);

/* Synchronises and returns the first device error recorded since the last call
 * (ROEAM_E_NONPOSITIVE / ROEAM_E_NONFINITE), clearing it; ROEAM_OK if none. */
roeam_status roeam_check(roeam_grid *g);

/* Residual of one grid, like roeam_flux_residual (res_out non-null, grid_idx >= 0), for
 * callers that cannot allocate device memory when they need it: a host that runs this
 * library inside a fixed device-memory budget with no allocation after start-up, or a
 * monitor next to a solver whose memory pool owns the device. The paper has no counterpart;
 * it is a service of this library. The call allocates nothing: its scratch is a fixed
 * 24 MiB array that every GPU loading the library holds until the process exits. A grid
 * fits if 4 x nj x pitch working-precision values (pitch = ni rounded up to 32) plus
 * 4 x ni x nj doubles fit in it (about 512 x 512 cells); larger grids get ROEAM_E_ARG with
 * a message saying so. The array is committed on a device when the first handle on that
 * device is created (roeam_create_grid looks it up there, which makes CUDA load the module
 * holding it), so a caller that creates its handles at start-up has the array before it
 * stops allocating, and this call itself allocates nothing. Calls share the array and it
 * keeps the last call's contents (each call writes all it reads); calls whose work overlaps
 * on the GPU race. Synchronises. */
roeam_status roeam_flux_residual_noalloc(roeam_grid *g, int grid_idx, double *res_out);

/* Number of tile shapes (stage-kernel work-unit layouts and schedules) the library is built
 * with: 10. Shapes 0-4 cut each grid into warp strips of 32 lanes and segments of 32, 64, 16,
 * 128 and 256 rows and let warps claim units dynamically in the order of the unit table
 * (tallest first); shapes 5-9 are the same heights with a static round robin of units over
 * warps. (Kernels that do not claim units dynamically treat 0-4 as 5-9; a batch too small to
 * give every resident warp a unit halves the height, down to 4 rows, and on to 2 rows while the
 * units still fit one round of the resident warps.) Results are bit-identical across shapes. */
int roeam_tile_config_count(void);

/* Describes tile shape `cfg`: strip width tx, segment height ty (cells) and threads per CTA. */
roeam_status roeam_tile_config_info(int cfg, int *tx, int *ty, int *threads);

/* Selects tile shape `cfg` for this handle's stage kernels (default 0). Captured graphs
 * are rebuilt on the next step. */
roeam_status roeam_set_tile_config(roeam_grid *g, int cfg);

/* Autotuner: times `steps` SSP-RK3 steps at `cfl` with every tile shape on the current
 * state (best of two timings; shapes that give the same units and schedule are timed once),
 * restores the state after each trial, and keeps the fastest shape. best_cfg (nullable)
 * receives it; ms_per_step (nullable, roeam_tile_config_count() doubles) the measured time
 * per step of each shape. The result is kept for the process: a later call on any handle
 * with the same workload (device, kernel family, every grid's sizes, boundary kinds and
 * scheme switches) applies it without timing and returns the same figures. Synchronises;
 * allocates a temporary copy of the state when it times. */
roeam_status roeam_autotune(roeam_grid *g, double cfl, int steps, int *best_cfg, double *ms_per_step);

/* Number of kernels this handle has launched (graph nodes count one each per replay). */
unsigned long long roeam_launch_count(const roeam_grid *g);

/* Total cells of grid `grid_idx` (or of the batch with -1), or -1 on a bad argument. */
long long roeam_cell_count(const roeam_grid *g, int grid_idx);

/* Message of the last failing call on this thread ("" if none). */
const char *roeam_last_error(void);

/* ABI version (major * 10000 + minor * 100 + patch). */
int roeam_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ROEAM_H */
