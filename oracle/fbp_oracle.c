/* FP64 CPU oracle of the initial iterate x-bar -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the CPU baseline of the benchmark use this file;
 * the product library shares no code with it.
 *
 * The paper reconstructs from an initial iterate x-bar (Appendix A) made by filtered
 * back-projection (FBP, the transform method of Sec. II; the preprocessing itself is left
 * to earlier work in Sec. III-D), to which a median filter of radius r = 2 is applied
 * (Sec. V-A).  It gives no formulas, so the library states its own specification and
 * this file is each step's plain definition, in the order of that specification:
 *   1. binning: every history by its chord (straight-line approximation), into
 *      (slice, angle, lateral) bins of a parallel-beam sinogram; a bin holds the mean
 *      WEPL of its histories (0 when empty);
 *   2. filtering: the discrete Ram-Lak ramp filter (Kak & Slaney, "Principles of
 *      Computerized Tomographic Imaging", ch. 3) by direct convolution along t;
 *   3. back-projection: linear interpolation between lateral bin centres, weight
 *      pi / n_theta;
 *   4. median filter: a disc window (per slice) or a ball window (3D), in-image
 *      neighbours only, the element floor(n/2) of the n sorted values;
 *   5. threshold hull: voxels at or below tau become 0.
 *
 * Pins (tests/test_oracle_fbp.py): analytic disc projections reconstruct to the disc
 * (levels, centroid of an off-centre disc, scale), hand-placed histories land in the
 * bins worked out by hand (the angle fold included), hand-made median cases and the
 * library median filter on interior voxels, the hull rule, and the end-to-end FBP of
 * noise-free straight histories through the synthetic phantom.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int32_t nx, ny, nz;     /* image grid; in-plane centred on (0,0), slice iz covers z in [iz dz, (iz+1) dz) */
    int32_t n_theta, n_t;   /* angle bins over [0, pi), lateral bins centred on t = 0 */
    int32_t reserved;
    double dx, dy, dz;      /* voxel size, mm */
    double dt;              /* lateral bin width, mm */
    double theta0;          /* angle bin a covers theta0 + [a, a+1) pi/n_theta (mod pi) */
} orc_fbp_geom;

/* ---------------------------------------------------------------- 1. binning */

/* The line of a history's chord P_in -> P_out (record: P_in xyz, P_out xyz, then four
 * bend parameters that FBP ignores) as (theta, t): theta the direction of the line's
 * normal, the chord direction turned by +90 degrees, folded into [0, pi) (the line at
 * theta >= pi is the line at theta - pi with t negated); t = P_in . (cos theta, sin theta);
 * z the mean of the two heights.  Returns 0 for a record whose chord has no in-plane
 * extent (an empty row). */
int orc_fbp_line(const float* rec, double* theta_out, double* t_out, double* z_out) {
    const double px = rec[0], py = rec[1], pz = rec[2], qx = rec[3], qy = rec[4], qz = rec[5];
    const double ddx = qx - px, ddy = qy - py;
    const double len = sqrt(ddx * ddx + ddy * ddy);
    if (!(len > 0.0)) return 0;
    const double cx = -ddy / len, cy = ddx / len;   /* (cos theta, sin theta) before the fold */
    double theta = atan2(cy, cx);
    double t = px * cx + py * cy;
    if (theta < 0.0) theta += 2.0 * M_PI;
    if (theta >= M_PI) {
        theta -= M_PI;
        t = -t;
    }
    *theta_out = theta;
    *t_out = t;
    *z_out = 0.5 * (pz + qz);
    return 1;
}

/* The line (theta, t) relative to the first angle bin: phi = theta - theta0 brought into
 * [0, pi) by steps of pi, t negated at every step (the same line). */
static void orc_fbp_rebase(double theta, double t, double theta0, double* phi_out, double* t_out) {
    double phi = theta - theta0;
    while (phi < 0.0) {
        phi += M_PI;
        t = -t;
    }
    while (phi >= M_PI) {
        phi -= M_PI;
        t = -t;
    }
    *phi_out = phi;
    *t_out = t;
}

/* Bin of one history: returns 1 and its (slice, angle bin, lateral bin), or 0 when it
 * falls outside the bins.  Angle bin a covers phi in [a, a+1) pi/n_theta (a rounding up
 * to phi = pi lands in the last bin); lateral bin k covers t in [k - n_t/2, k + 1 - n_t/2) dt
 * (t taken for the rebased angle); slice iz covers z in [iz, iz+1) dz. */
int orc_fbp_bin_of(const float* rec, const orc_fbp_geom* g, int64_t* iz, int64_t* ia, int64_t* it) {
    double theta, t0, z, theta_r, t;
    if (!orc_fbp_line(rec, &theta, &t0, &z)) return 0;
    orc_fbp_rebase(theta, t0, g->theta0, &theta_r, &t);
    int64_t a = (int64_t)floor(theta_r / (M_PI / g->n_theta));
    if (a < 0) a = 0;
    if (a > g->n_theta - 1) a = g->n_theta - 1;
    const double u = t / g->dt + 0.5 * g->n_t;
    if (!(u >= 0.0 && u < (double)g->n_t)) return 0;
    const double v = z / g->dz;
    if (!(v >= 0.0 && v < (double)g->nz)) return 0;
    *iz = (int64_t)floor(v);
    *ia = a;
    *it = (int64_t)floor(u);
    if (*it > g->n_t - 1) *it = g->n_t - 1;
    if (*iz > g->nz - 1) *iz = g->nz - 1;
    return 1;
}

/* Sinogram p[iz][a][k] = mean WEPL of the histories in the bin (0 for an empty bin) and
 * its history count.  Histories are taken in their stored order. */
void orc_fbp_bin(const float* paths, const double* wepl, int64_t M, const orc_fbp_geom* g, double* sino,
                 int64_t* count) {
    const int64_t S = (int64_t)g->nz * g->n_theta * g->n_t;
    for (int64_t i = 0; i < S; ++i) {
        sino[i] = 0.0;
        count[i] = 0;
    }
    for (int64_t h = 0; h < M; ++h) {
        int64_t iz, ia, it;
        if (!orc_fbp_bin_of(paths + 10 * h, g, &iz, &ia, &it)) continue;
        const int64_t s = (iz * g->n_theta + ia) * g->n_t + it;
        sino[s] += wepl[h];
        count[s] += 1;
    }
    for (int64_t i = 0; i < S; ++i)
        if (count[i] > 0) sino[i] = sino[i] / (double)count[i];
}

/* ---------------------------------------------------------------- 2. filtering */

/* Discrete Ram-Lak kernel at lag m: 1/(4 dt^2) at m = 0, -1/(pi^2 m^2 dt^2) at odd m,
 * 0 at even m != 0. */
double orc_ramlak(int64_t m, double dt) {
    if (m == 0) return 1.0 / (4.0 * dt * dt);
    if (m % 2 == 0) return 0.0;
    const double md = (double)m;
    return -1.0 / (M_PI * M_PI * md * md * dt * dt);
}

/* q_k = dt * sum_n p_n h(k - n) along every (slice, angle) row of n_t bins. */
void orc_fbp_filter(const double* sino, const orc_fbp_geom* g, double* q) {
    const int64_t rows = (int64_t)g->nz * g->n_theta, nt = g->n_t;
    for (int64_t r = 0; r < rows; ++r) {
        const double* p = sino + r * nt;
        for (int64_t k = 0; k < nt; ++k) {
            double s = 0.0;
            for (int64_t n = 0; n < nt; ++n) s += p[n] * orc_ramlak(k - n, g->dt);
            q[r * nt + k] = g->dt * s;
        }
    }
}

/* ---------------------------------------------------------------- 3. back-projection */

/* f(x, y) = (pi / n_theta) sum_a Q_a(x cos theta_a + y sin theta_a) at every voxel centre,
 * theta_a = theta0 + (a + 1/2) pi / n_theta, x = (ix + 1/2) dx - nx dx / 2 (y alike).  Q_a(t) is
 * linear between bin centres t_k = (k + 1/2 - n_t/2) dt with Q = 0 at every k outside
 * [0, n_t). */
void orc_fbp_backproject(const double* q, const orc_fbp_geom* g, double* img) {
    const int64_t nx = g->nx, ny = g->ny, nz = g->nz, na = g->n_theta, nt = g->n_t;
    for (int64_t iz = 0; iz < nz; ++iz)
        for (int64_t iy = 0; iy < ny; ++iy)
            for (int64_t ix = 0; ix < nx; ++ix) {
                const double x = ((double)ix + 0.5) * g->dx - 0.5 * (double)nx * g->dx;
                const double y = ((double)iy + 0.5) * g->dy - 0.5 * (double)ny * g->dy;
                double s = 0.0;
                for (int64_t a = 0; a < na; ++a) {
                    const double th = g->theta0 + ((double)a + 0.5) * M_PI / (double)na;
                    const double t = x * cos(th) + y * sin(th);
                    const double u = t / g->dt + 0.5 * (double)nt - 0.5;
                    const double k0 = floor(u);
                    const double w = u - k0;
                    const int64_t k = (int64_t)k0;
                    const double* row = q + (iz * na + a) * nt;
                    const double v0 = (k >= 0 && k < nt) ? row[k] : 0.0;
                    const double v1 = (k + 1 >= 0 && k + 1 < nt) ? row[k + 1] : 0.0;
                    s += (1.0 - w) * v0 + w * v1;
                }
                img[(iz * ny + iy) * nx + ix] = s * M_PI / (double)na;
            }
}

/* ---------------------------------------------------------------- 4. median filter */

static int cmp_double(const void* a, const void* b) {
    const double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Window offsets (ox, oy, oz) with ox^2 + oy^2 + oz^2 <= r^2 + 1 (oz = 0 unless ball). */
int orc_median_window(int r, int ball, int* off) {
    int n = 0;
    const int rz = ball ? r : 0;
    for (int oz = -rz; oz <= rz; ++oz)
        for (int oy = -r; oy <= r; ++oy)
            for (int ox = -r; ox <= r; ++ox)
                if (ox * ox + oy * oy + oz * oz <= r * r + 1) {
                    if (off) {
                        off[3 * n] = ox;
                        off[3 * n + 1] = oy;
                        off[3 * n + 2] = oz;
                    }
                    ++n;
                }
    return n;
}

/* out[v] = element floor(n/2) of the sorted values of the n in-image voxels of v's window. */
void orc_median(const double* in, int nx, int ny, int nz, int r, int ball, double* out) {
    const int W = orc_median_window(r, ball, NULL);
    int* off = (int*)malloc(sizeof(int) * 3 * (size_t)W);
    double* buf = (double*)malloc(sizeof(double) * (size_t)W);
    orc_median_window(r, ball, off);
    for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix) {
                int n = 0;
                for (int w = 0; w < W; ++w) {
                    const int jx = ix + off[3 * w], jy = iy + off[3 * w + 1], jz = iz + off[3 * w + 2];
                    if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz) continue;
                    buf[n++] = in[((int64_t)jz * ny + jy) * nx + jx];
                }
                qsort(buf, (size_t)n, sizeof(double), cmp_double);
                out[((int64_t)iz * ny + iy) * nx + ix] = buf[n / 2];
            }
    free(buf);
    free(off);
}

/* ---------------------------------------------------------------- 5. hull */

void orc_hull(double* img, int64_t V, double tau) {
    for (int64_t v = 0; v < V; ++v)
        if (img[v] <= tau) img[v] = 0.0;
}

/* ---------------------------------------------------------------- the chain */

/* x-bar = hull(median(backproject(filter(bin(paths, wepl))))); median_r = 0 skips the
 * median filter, use_hull = 0 the hull. */
void orc_initial_iterate(const float* paths, const double* wepl, int64_t M, const orc_fbp_geom* g, int median_r,
                         int median_ball, int use_hull, double tau, double* out) {
    const int64_t S = (int64_t)g->nz * g->n_theta * g->n_t;
    const int64_t V = (int64_t)g->nx * g->ny * g->nz;
    double* sino = (double*)malloc(sizeof(double) * (size_t)(S > 0 ? S : 1));
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)(S > 0 ? S : 1));
    double* q = (double*)malloc(sizeof(double) * (size_t)(S > 0 ? S : 1));
    double* img = (double*)malloc(sizeof(double) * (size_t)(V > 0 ? V : 1));
    orc_fbp_bin(paths, wepl, M, g, sino, cnt);
    orc_fbp_filter(sino, g, q);
    orc_fbp_backproject(q, g, img);
    if (median_r > 0)
        orc_median(img, g->nx, g->ny, g->nz, median_r, median_ball, out);
    else
        memcpy(out, img, sizeof(double) * (size_t)V);
    if (use_hull) orc_hull(out, V, tau);
    free(img);
    free(q);
    free(cnt);
    free(sino);
}
