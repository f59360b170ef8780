/* Initial iterate x-bar for NTVS (arXiv 1803.01112): filtered back-projection of binned
 * proton histories, a median filter and a threshold hull, on the GPU in FP64.
 *
 * The paper starts the reconstruction from x-bar (Appendix A), an FBP image (FBP is the
 * transform method of Sec. II; Sec. III-D leaves the preprocessing to earlier work) to
 * which a median filter of radius 2 is applied (Sec. V-A).  The paper defines none of
 * these steps; this library specifies them as follows.
 *
 *   1. Binning (ntvs_fbp_bin).  A history is taken as its chord P_in -> P_out (the path
 *      record of ntvs_load_paths, [M][10] floats; the four bend parameters are ignored).
 *      The line's normal is the chord direction turned by +90 degrees, theta = its angle,
 *      t = P_in . (cos theta, sin theta), z = (z_in + z_out) / 2.  The angle is rebased,
 *      phi = theta - theta0 brought into [0, pi) by steps of pi with t negated at each
 *      step (the same line).  Angle bin a covers phi in [a, a+1) pi/n_theta, lateral bin k
 *      covers t in [k - n_t/2, k + 1 - n_t/2) dt, slice iz covers z in [iz, iz+1) dz
 *      (half-open; histories outside are dropped).  A bin holds the mean WEPL of its
 *      histories, 0 when empty.
 *   2. Filtering (ntvs_fbp_filter).  The discrete Ram-Lak filter along t of every
 *      (slice, angle) row: q_k = dt sum_n p_n h(k - n), h(0) = 1/(4 dt^2),
 *      h(m) = -1/(pi^2 m^2 dt^2) for odd m, 0 for even m != 0.
 *   3. Back-projection (ntvs_fbp_backproject).  f(x, y) = (pi/n_theta) sum_a
 *      Q_a(x cos theta_a + y sin theta_a) at each voxel centre, theta_a = theta0 +
 *      (a + 1/2) pi/n_theta, voxel centres x = (ix + 1/2) dx - nx dx/2 (y alike; the grid
 *      is centred in-plane).  Q_a is linear between the bin centres (k + 1/2 - n_t/2) dt,
 *      with Q = 0 at every k outside [0, n_t).
 *   4. Median filter (ntvs_median_filter), radius r: over the window offsets in
 *      [-r, r] with ox^2 + oy^2 + oz^2 <= r^2 + 1 (oz = 0 per slice; all three in the ball
 *      mode; r = 0 is the voxel alone), the
 *      in-image neighbours only; the result is element floor(n/2), counted from 0, of
 *      the n sorted values (21 pixels per slice and 57 voxels in the ball at r = 2).
 *   5. Hull (ntvs_hull): voxels whose value is <= tau become 0.
 *
 * Conventions: every pointer is device memory of the current CUDA device (the caller
 * owns it); work is queued on cuda_stream (a cudaStream_t, NULL for the legacy default
 * stream) and nothing synchronizes; arrays are C order with x fastest (voxel
 * (iz*ny + iy)*nx + ix, sinogram bin (iz*n_theta + a)*n_t + k).  Each call returns
 * NTVS_OK or a negative NTVS_ERR_* code of ntvs.h, with the text in ntvs_last_error();
 * NTVS_ERR_ARG for a null pointer, a size below 1, a non-positive or non-finite
 * spacing, |theta0| > 16 pi or non-finite, n_t > 8192, n_theta > 4096, nz > 65535, more
 * than 2^31 - 1 voxels or bins, a median radius outside [0, 3], overlapping input and
 * output, or a NaN tau; NTVS_ERR_CUDA when a launch fails.  No call allocates device
 * memory.
 */
#ifndef NTVS_FBP_H
#define NTVS_FBP_H

#include <stdint.h>

#include "ntvs.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t nx, ny, nz;     /* image grid; in-plane centred on (0,0); slice iz covers z in [iz dz, (iz+1) dz) */
    int32_t n_theta, n_t;   /* angle bins of width pi/n_theta from theta0; lateral bins centred on t = 0 */
    int32_t reserved;       /* must be 0 */
    double dx, dy, dz;      /* voxel size, mm */
    double dt;              /* lateral bin width, mm */
    double theta0;          /* angular origin of the bins, radians */
} ntvs_fbp_geom;

/* Step 1.  paths: [M][10] float records (only P_in and P_out are read); wepl: [M] double.
 * Writes sino [nz][n_theta][n_t] double (mean WEPL per bin, 0 when empty) and count
 * [nz][n_theta][n_t] int32 (histories per bin).  M = 0 gives a zero sinogram.  Bin sums
 * are accumulated with atomics, so the rounding of a mean may differ between runs. */
int ntvs_fbp_bin(const ntvs_fbp_geom* g, const float* paths, const double* wepl, int64_t M, double* sino,
                 int32_t* count, void* cuda_stream);

/* Step 2.  sino, q: [nz][n_theta][n_t] double; q must not overlap sino. */
int ntvs_fbp_filter(const ntvs_fbp_geom* g, const double* sino, double* q, void* cuda_stream);

/* Step 3.  q: [nz][n_theta][n_t] double (filtered); img: [nz][ny][nx] double. */
int ntvs_fbp_backproject(const ntvs_fbp_geom* g, const double* q, double* img, void* cuda_stream);

/* Step 4 (and 5 when use_hull != 0: the result is set to 0 where it is <= tau).  in, out:
 * [nz][ny][nx] double, not overlapping; radius 0..3 (0 copies); ball != 0 for the 3D
 * window. */
int ntvs_median_filter(const double* in, double* out, int nx, int ny, int nz, int radius, int ball, int use_hull,
                       double tau, void* cuda_stream);

/* Step 5 in place on V voxels. */
int ntvs_hull(double* img, int64_t V, double tau, void* cuda_stream);

/* Device workspace in bytes that ntvs_initial_iterate needs for g (sinogram, counts,
 * filtered sinogram and the unfiltered image, each 256-byte aligned); negative
 * NTVS_ERR_ARG for an invalid geometry. */
int64_t ntvs_fbp_workspace_bytes(const ntvs_fbp_geom* g);

/* Steps 1-5: out = hull(median(backproject(filter(bin(paths, wepl))))).  median_radius 0
 * skips the median filter, use_hull 0 the hull.  workspace: workspace_bytes >=
 * ntvs_fbp_workspace_bytes(g) of device memory (256-byte aligned), reused freely by the
 * call.  out: [nz][ny][nx] double. */
int ntvs_initial_iterate(const ntvs_fbp_geom* g, const float* paths, const double* wepl, int64_t M, int median_radius,
                         int median_ball, int use_hull, double tau, void* workspace, int64_t workspace_bytes,
                         double* out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* NTVS_FBP_H */
