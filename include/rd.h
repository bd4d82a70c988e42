/*
 * rd.h -- C ABI of the tumour forward model in libdbq.so: the
 * reaction-diffusion equation of Ezhov et al. (2022), Section 2.1, Eq. 1-2,
 *
 *     du/dt = div(D grad u) + rho u (1 - u)   in the brain Omega,
 *     n . grad u = 0                           on the boundary of Omega,
 *     u(r, 0) = u0 at the seed point r*, 0 elsewhere,
 *
 * solved on the GPU for many parameter sets theta = (x, y, z, D_w, rho, T_end)
 * (the parameters the paper samples to build its database, Section 3).
 * Thresholding the result at u_T1Gd and u_FLAIR (db_load_volumes +
 * db_build_masks of dbq.h) gives a database entry.
 *
 * Discretisation (the paper names none):
 *   * unit voxel spacing on an nx x ny x nz grid, volumes [nz][ny][nx] with x
 *     fastest; D(x) = D_w m(x) with m the caller's tissue map of relative
 *     diffusivities (e.g. 1 in white matter, 0.1 in grey matter, 0 in CSF and
 *     background); Omega = {m > 0};
 *   * the flux through the face between neighbours i and j is
 *     D_w h(m_i, m_j) (u_j - u_i), h the harmonic mean 2 m_i m_j / (m_i + m_j),
 *     which is 0 when either voxel is outside Omega (the no-flux condition);
 *     the grid's outer faces carry no flux;
 *   * explicit Euler: n = ceil(T_end (6 D_w max(m) + rho) / cfl) steps of
 *     dt = T_end / n (n = 0 if T_end = 0), each voxel updated from the
 *     previous step as u + dt (D_w sum_j h (u_j - u_i) + rho u (1 - u));
 *     0 < cfl <= 1 keeps 0 <= u <= 1;
 *   * the seed voxel is (floor(x + 0.5), floor(y + 0.5), floor(z + 0.5)).
 * The GPU computes in binary32 (u, the face coefficients, dt D_w and
 * dt rho); the step count is computed on the host in binary64.
 *
 * Errors: the status codes of dbq.h (DBQ_OK, DBQ_EINVAL, DBQ_ENOMEM,
 * DBQ_ECUDA); db_last_error() describes the last failure of the thread.
 */
#ifndef DBQ_RD_H
#define DBQ_RD_H

#include <stdint.h>

#include "dbq.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rd_solver rd_solver;

/*
 * rd_create -- a solver for one grid and tissue map on the current device.
 *   nx, ny, nz   grid (each >= 1, nx*ny*nz < 2^31).
 *   tissue       [nz][ny][nx] float32 relative diffusivity, every value
 *                finite and >= 0 (DBQ_EINVAL otherwise); host or device
 *                memory, copied.
 *   batch        simulation slots advanced together, 1..1024 (0: 16): each
 *                launch advances every busy slot by one explicit step, and a
 *                slot whose simulation has ended takes the next one (longest
 *                first) between two launches.  Device memory held:
 *                2 * batch * V * 4 bytes of ping-pong fields plus
 *                5 * V * 4 bytes (map and face coefficients).
 * Returns DBQ_OK and *out, or DBQ_EINVAL / DBQ_ENOMEM / DBQ_ECUDA.
 */
int rd_create(rd_solver** out, int nx, int ny, int nz, const float* tissue, int batch);

/*
 * rd_simulate -- u(T_end) for `count` parameter sets.
 *   theta   host [count][6] doubles (x, y, z, D_w, rho, T_end): seed point in
 *           voxel coordinates (its voxel must be in the grid and in Omega),
 *           D_w >= 0 in voxel^2 per time unit, rho >= 0 per time unit,
 *           T_end >= 0, all finite.
 *   u0      initial density at the seed, in (0, 1].
 *   cfl     in (0, 1].
 *   out     [count][nz][ny][nx] float32, host or device memory.
 *   steps   host [count] int64 step counts n, or NULL.
 * Every argument is checked before any work; outputs are written only on
 * DBQ_OK.  Synchronous on `stream`: returns after `out` is written.
 */
int rd_simulate(rd_solver* rs, int count, const double* theta, float u0, double cfl,
                float* out, int64_t* steps, void* stream);

/*
 * rd_stats -- measurements of the last rd_simulate on this solver:
 * out[0] GPU milliseconds from the first slot fill to the last launch
 * (CUDA events; step launches and slot refills), out[1] step launches,
 * out[2] voxel updates computed (tiles not skipped), out[3] slots used.
 * DBQ_ESTATE before any run.
 */
int rd_stats(const rd_solver* rs, double out[4]);

/* rd_destroy -- frees the solver (NULL-safe). */
int rd_destroy(rd_solver* rs);

#ifdef __cplusplus
}
#endif

#endif /* DBQ_RD_H */
