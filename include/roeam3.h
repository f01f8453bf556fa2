/*
 * roeam3.h — C ABI of the 3D path of the GB300 (sm_103a) Roe-AM library: the complete form of
 * the scheme's dissipation, Eq. 85 of Li, Ren & Gu ("An improved Roe scheme for all
 * Mach-number flows simultaneously curing known problems"), with the w-momentum row and
 * passive-scalar rows rho k (the rows "such as the turbulence model" that Section 6.2 appends),
 * the 9-face pressure-density detector of Eq. 96, and the SSP-RK3 update, on structured
 * Cartesian 3D grids with first-order face states.
 *
 * Conventions (as in roeam.h, whose status codes and roeam_last_error() this header shares):
 *   - A handle holds `count` >= 1 independent grids advancing together; all share the
 *     precision and the number of scalars.
 *   - Host state arrays are float64, shape [5 + nscal][nk][nj][ni], i fastest, variables
 *     (rho, rho u, rho v, rho w, rho E, rho k_1, ..); grid_idx = -1 covers every grid,
 *     concatenated. The caller owns host arrays; the handle owns its device memory.
 *   - Device-side failures (non-positive or non-finite states) are reported by the next call
 *     that synchronises (get_state, conserved_totals, check, rk_step with dt_last).
 *   - One host thread uses a handle at a time; work is ordered on the stream given at
 *     creation (NULL: the legacy default stream).
 */
#ifndef ROEAM3_H
#define ROEAM3_H

#include "roeam.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct roeam3_grid roeam3_grid; /* opaque batch handle */

enum { ROEAM3_MAX_SCALARS = 3 };

/* One 3D grid of ni x nj x nk cells of dx x dy x dz (all > 0; ni, nj, nk in 1..65535, at most
 * 2^28 cells).
 *   bc[6]     boundary type of the -x, +x, -y, +y, -z, +z sides (ROEAM_BC_*; PERIODIC on both
 *             sides of an axis or neither). WALL mirrors the adjacent state (normal velocity
 *             component negated, scalars copied); INFLOW imposes `inflow`; OUTFLOW copies.
 *   inflow    primitive (rho, u, v, w, p, k_1, .., k_nscal) of INFLOW sides.
 *   nscal     passive scalars, 0..ROEAM3_MAX_SCALARS, the same for every grid of a handle.
 *   p         scheme parameters as in roeam.h; recon must be ROEAM_RECON_FIRST and the
 *             ablation fields (scheme, dup_mode, no_ufix, xi_roe, harten) must be zero.
 * Otherwise roeam3_create_grid returns ROEAM_E_ARG. */
typedef struct {
    int ni, nj, nk;
    int bc[6];
    double inflow[5 + ROEAM3_MAX_SCALARS];
    double dx, dy, dz;
    int nscal;
    int reserved_;   /* must be 0 */
    roeam_params p;
} roeam3_grid_desc;

/* Creates a handle of `count` (1..65535) grids on CUDA device `device`, ordering its work on
 * `cuda_stream` (a cudaStream_t, or NULL). The state is zero until roeam3_set_state. */
roeam_status roeam3_create_grid(int count, const roeam3_grid_desc *descs, int device, void *cuda_stream,
                                roeam3_grid **out);

/* Releases the handle and its device memory. NULL is ignored. */
void roeam3_destroy_grid(roeam3_grid *g);

/* Copies the conserved state of grid grid_idx (or all with -1) from the host. */
roeam_status roeam3_set_state(roeam3_grid *g, int grid_idx, const double *cons);

/* Copies the conserved state of grid grid_idx (or all) to the host. Synchronises. */
roeam_status roeam3_get_state(roeam3_grid *g, int grid_idx, double *cons_out);

/* Residual R(U) = -(1/V) sum_f F_f |S_f| of grid grid_idx (or all) for the current state, copied
 * to res_out (same layout as the state) when not NULL. */
roeam_status roeam3_flux_residual(roeam3_grid *g, int grid_idx, double *res_out);

/* Advances every grid by nsteps SSP-RK3 steps; each grid's dt is dt_fixed if > 0, else
 * cfl / max_i sum_dir (|U_dir| + max(c, c~/theta)) / h_dir on the state at the start of the
 * step (theta, c~ of Eqs. 99-101). dt_last (nullable, count doubles) receives each grid's last
 * dt (this synchronises). */
roeam_status roeam3_rk_step(roeam3_grid *g, double cfl, double dt_fixed, int nsteps, double *dt_last);

/* FP64 totals sum_i V Q_i of grid grid_idx: 5 + nscal values. Synchronises. */
roeam_status roeam3_conserved_totals(roeam3_grid *g, int grid_idx, double *out);

/* Synchronises and returns (and clears) the first device error since the last call. */
roeam_status roeam3_check(roeam3_grid *g);

/* Kernel launches issued by the handle so far. */
unsigned long long roeam3_launch_count(const roeam3_grid *g);

#ifdef __cplusplus
}
#endif

#endif /* ROEAM3_H */
