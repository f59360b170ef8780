/*
 * Seeded synthetic proton-CT system generator.
 *
 * Stand-in for the paper's Geant4 / experimental CTP404 data (Sec. III-C, Table I):
 * a cylinder phantom with cylindrical inserts is voxelised, proton histories are
 * drawn per projection angle, each history's path through the voxel grid is
 * traced (straight line, or a cubic-Hermite bent path split into straight
 * segments) with exact voxel intersection lengths (Siddon-style plane-crossing
 * traversal), and the measured WEPL is the line integral of the voxelised
 * phantom plus Gaussian noise.
 *
 * This module only builds inputs: it holds none of the reconstruction's
 * arithmetic (no DROP step, no TV).  Both the CUDA library and the CPU oracle
 * consume its output; it imports neither.
 *
 * Randomness: every draw is SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) used
 * in counter mode, output n of stream `seed` = mix(seed + (n+1)*golden_gamma),
 * keyed by the global history index, so the result does not depend on the
 * number of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t nx, ny, nz;
    double dx, dy, dz;          /* voxel size, mm */
    double cyl_r, cyl_rsp;      /* phantom cylinder radius (mm) and RSP */
    int32_t n_ins;
    const double* ins_cx;       /* insert centres (mm, in-plane), radii, RSP */
    const double* ins_cy;
    const double* ins_r;
    const double* ins_rsp;
    int64_t n_hist;
    int32_t n_angles;
    double angle_span_deg;      /* angles a*span/n_angles, a = 0..n_angles-1 */
    int32_t curved;             /* 0 straight, 1 cubic-Hermite bent paths */
    int32_t n_seg;              /* straight segments per bent path */
    double dev_max;             /* max deviation from the chord (mm), lateral and z */
    double noise_sigma;         /* relative WEPL noise */
    double min_len;             /* intersection lengths below this are dropped (mm) */
    double lateral_width;       /* lateral offsets t ~ U(-w/2, w/2) (mm) */
    uint64_t seed;
} syn_cfg;

/* ---------------------------------------------------------------- RNG */
static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static inline uint64_t sm64_at(uint64_t seed, uint64_t n) {
    return sm64_mix(seed + (n + 1) * 0x9E3779B97F4A7C15ULL);
}
/* uniform in [0,1) with 53 random bits */
static inline double u01(uint64_t seed, uint64_t n) {
    return (double)(sm64_at(seed, n) >> 11) * (1.0 / 9007199254740992.0);
}

enum { DRAWS_PER_HIST = 8 };

/* ----------------------------------------------------------- phantom */
static double rsp_at(const syn_cfg* c, double x, double y) {
    if (x * x + y * y > c->cyl_r * c->cyl_r) return 0.0;
    for (int i = 0; i < c->n_ins; ++i) {
        double ex = x - c->ins_cx[i], ey = y - c->ins_cy[i];
        if (ex * ex + ey * ey <= c->ins_r[i] * c->ins_r[i]) return c->ins_rsp[i];
    }
    return c->cyl_rsp;
}

/* xstar: phantom RSP averaged over a 4x4 in-plane supersample of each voxel.
 * xbar : 1 where the voxel centre is inside the cylinder, 0 outside (hull stand-in).
 * label: insert index at the voxel centre, n_ins for cylinder background, -1 outside. */
void syn_phantom(const syn_cfg* c, double* xstar, double* xbar, int32_t* label) {
    const double ox = -0.5 * c->nx * c->dx, oy = -0.5 * c->ny * c->dy;
    for (int iy = 0; iy < c->ny; ++iy)
        for (int ix = 0; ix < c->nx; ++ix) {
            double acc = 0.0;
            for (int sy = 0; sy < 4; ++sy)
                for (int sx = 0; sx < 4; ++sx) {
                    double x = ox + (ix + (sx + 0.5) / 4.0) * c->dx;
                    double y = oy + (iy + (sy + 0.5) / 4.0) * c->dy;
                    acc += rsp_at(c, x, y);
                }
            double xc = ox + (ix + 0.5) * c->dx, yc = oy + (iy + 0.5) * c->dy;
            int lab = -1;
            if (xc * xc + yc * yc <= c->cyl_r * c->cyl_r) {
                lab = c->n_ins;
                for (int i = 0; i < c->n_ins; ++i) {
                    double ex = xc - c->ins_cx[i], ey = yc - c->ins_cy[i];
                    if (ex * ex + ey * ey <= c->ins_r[i] * c->ins_r[i]) { lab = i; break; }
                }
            }
            for (int iz = 0; iz < c->nz; ++iz) {
                int64_t j = ((int64_t)iz * c->ny + iy) * c->nx + ix;
                if (xstar) xstar[j] = acc / 16.0;
                if (xbar) xbar[j] = (lab >= 0) ? 1.0 : 0.0;
                if (label) label[j] = lab;
            }
        }
}

/* ------------------------------------------------------ history plan */
typedef struct { double t, z; uint64_t key; int64_t zbin; } hist_t;

static int cmp_hist(const void* a, const void* b) {
    const hist_t* p = (const hist_t*)a; const hist_t* q = (const hist_t*)b;
    if (p->zbin != q->zbin) return p->zbin < q->zbin ? -1 : 1;
    if (p->t != q->t) return p->t < q->t ? -1 : 1;
    return p->key < q->key ? -1 : (p->key > q->key);
}

static int64_t hist_per_angle(const syn_cfg* c, int a) {
    int64_t base = c->n_hist / c->n_angles, rem = c->n_hist % c->n_angles;
    return base + (a < rem ? 1 : 0);
}
static int64_t angle_first_row(const syn_cfg* c, int a) {
    int64_t base = c->n_hist / c->n_angles, rem = c->n_hist % c->n_angles;
    return (int64_t)a * base + (a < rem ? a : rem);
}

/* Rows are emitted angle by angle; within an angle, histories are ordered by
 * (z slice, lateral offset) - a binned acquisition order.  plan[r] gives the
 * lateral offset t, height z and RNG key of row r. */
void syn_plan(const syn_cfg* c, double* t_out, double* z_out, uint64_t* key_out, int32_t* angle_out) {
    const double Z = c->nz * c->dz;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int a = 0; a < c->n_angles; ++a) {
        int64_t m = hist_per_angle(c, a), r0 = angle_first_row(c, a);
        hist_t* h = (hist_t*)malloc(sizeof(hist_t) * (size_t)(m > 0 ? m : 1));
        for (int64_t k = 0; k < m; ++k) {
            uint64_t key = (uint64_t)(r0 + k);
            h[k].t = (u01(c->seed, key * DRAWS_PER_HIST + 0) - 0.5) * c->lateral_width;
            h[k].z = u01(c->seed, key * DRAWS_PER_HIST + 1) * Z;
            h[k].key = key;
            h[k].zbin = (int64_t)floor(h[k].z / c->dz);
        }
        qsort(h, (size_t)m, sizeof(hist_t), cmp_hist);
        for (int64_t k = 0; k < m; ++k) {
            t_out[r0 + k] = h[k].t; z_out[r0 + k] = h[k].z; key_out[r0 + k] = h[k].key;
            if (angle_out) angle_out[r0 + k] = a;
        }
        free(h);
    }
}

/* ---------------------------------------------------- path tracing */
static int seg_axis_cap(const syn_cfg* c) {
    int m = c->nx > c->ny ? c->nx : c->ny;
    if (c->nz > m) m = c->nz;
    return m + 4;
}
static int seg_scratch(const syn_cfg* c) { return 3 * seg_axis_cap(c); }

typedef struct {
    int32_t* col; double* len; int n, cap;
    int32_t* hkey; int32_t* hpos; int hcap;   /* open-addressing map voxel -> position */
} rowbuf;

static void rb_init(rowbuf* rb) {
    rb->cap = 4096; rb->n = 0;
    rb->col = (int32_t*)malloc(sizeof(int32_t) * rb->cap);
    rb->len = (double*)malloc(sizeof(double) * rb->cap);
    rb->hcap = 8192;
    rb->hkey = (int32_t*)malloc(sizeof(int32_t) * rb->hcap);
    rb->hpos = (int32_t*)malloc(sizeof(int32_t) * rb->hcap);
    for (int i = 0; i < rb->hcap; ++i) rb->hkey[i] = -1;
}
static void rb_free(rowbuf* rb) { free(rb->col); free(rb->len); free(rb->hkey); free(rb->hpos); }
/* erase the hash slots of every stored entry (whole probe clusters: all belong to this row) */
static void rb_erase_hash(rowbuf* rb) {
    for (int i = 0; i < rb->n; ++i) {
        uint32_t h = ((uint32_t)rb->col[i] * 2654435761u) & (uint32_t)(rb->hcap - 1);
        while (rb->hkey[h] != -1) { rb->hkey[h] = -1; h = (h + 1) & (uint32_t)(rb->hcap - 1); }
    }
}
static void rb_add(rowbuf* rb, int32_t j, double l) {
    uint32_t h = ((uint32_t)j * 2654435761u) & (uint32_t)(rb->hcap - 1);
    while (rb->hkey[h] != -1) {
        if (rb->hkey[h] == j) { rb->len[rb->hpos[h]] += l; return; }
        h = (h + 1) & (uint32_t)(rb->hcap - 1);
    }
    if (rb->n == rb->cap) {
        rb->cap *= 2;
        rb->col = (int32_t*)realloc(rb->col, sizeof(int32_t) * rb->cap);
        rb->len = (double*)realloc(rb->len, sizeof(double) * rb->cap);
    }
    if (2 * (rb->n + 1) > rb->hcap) {   /* grow and rehash */
        int nh = rb->hcap * 2;
        free(rb->hkey); free(rb->hpos);
        rb->hkey = (int32_t*)malloc(sizeof(int32_t) * nh);
        rb->hpos = (int32_t*)malloc(sizeof(int32_t) * nh);
        for (int i = 0; i < nh; ++i) rb->hkey[i] = -1;
        rb->hcap = nh;
        for (int i = 0; i < rb->n; ++i) {
            uint32_t g = ((uint32_t)rb->col[i] * 2654435761u) & (uint32_t)(nh - 1);
            while (rb->hkey[g] != -1) g = (g + 1) & (uint32_t)(nh - 1);
            rb->hkey[g] = rb->col[i]; rb->hpos[g] = i;
        }
        h = ((uint32_t)j * 2654435761u) & (uint32_t)(rb->hcap - 1);
        while (rb->hkey[h] != -1) h = (h + 1) & (uint32_t)(rb->hcap - 1);
    }
    rb->hkey[h] = j; rb->hpos[h] = rb->n;
    rb->col[rb->n] = j; rb->len[rb->n] = l; rb->n++;
}

/* Plane-crossing parameters s in (lo, hi) of axis a for P + s*D, in increasing order. */
static int crossings(double p, double d, double o, double h, int n, double lo, double hi, double* out) {
    if (d == 0.0) return 0;
    double u0 = (p + lo * d - o) / h, u1 = (p + hi * d - o) / h;
    double umin = u0 < u1 ? u0 : u1, umax = u0 < u1 ? u1 : u0;
    long k0 = (long)ceil(umin), k1 = (long)floor(umax);
    if (k0 < 0) k0 = 0;
    if (k1 > n) k1 = n;
    int m = 0;
    if (d > 0.0) {
        for (long k = k0; k <= k1; ++k) {
            double s = (o + k * h - p) / d;
            if (s > lo && s < hi) out[m++] = s;
        }
    } else {
        for (long k = k1; k >= k0; --k) {
            double s = (o + k * h - p) / d;
            if (s > lo && s < hi) out[m++] = s;
        }
    }
    return m;
}

/* Exact intersection lengths of segment P->Q with the voxel grid: the segment is
 * clipped to the grid box, cut at every voxel plane it crosses, and each piece is
 * credited to the voxel containing its midpoint (Siddon, Med. Phys. 12, 1985). */
static void trace_segment(const syn_cfg* c, const double P[3], const double Q[3], rowbuf* rb, double* sbuf) {
    const double o[3] = {-0.5 * c->nx * c->dx, -0.5 * c->ny * c->dy, 0.0};
    const double h[3] = {c->dx, c->dy, c->dz};
    const int n[3] = {c->nx, c->ny, c->nz};
    double D[3] = {Q[0] - P[0], Q[1] - P[1], Q[2] - P[2]};
    double L = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
    if (L <= 0.0) return;
    double lo = 0.0, hi = 1.0;
    for (int a = 0; a < 3; ++a) {
        double e0 = o[a], e1 = o[a] + n[a] * h[a];
        if (D[a] == 0.0) {
            if (P[a] < e0 || P[a] > e1) return;
        } else {
            double s0 = (e0 - P[a]) / D[a], s1 = (e1 - P[a]) / D[a];
            if (s0 > s1) { double t = s0; s0 = s1; s1 = t; }
            if (s0 > lo) lo = s0;
            if (s1 < hi) hi = s1;
        }
    }
    if (!(hi > lo)) return;
    const int cap = seg_axis_cap(c);
    double* ax[3] = {sbuf, sbuf + cap, sbuf + 2 * cap};
    int na[3], ia[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) na[a] = crossings(P[a], D[a], o[a], h[a], n[a], lo, hi, ax[a]);
    double s0 = lo;
    for (;;) {
        /* next crossing of the three increasing sequences, else the segment end */
        double s1 = hi; int w = -1;
        for (int a = 0; a < 3; ++a)
            if (ia[a] < na[a] && ax[a][ia[a]] < s1) { s1 = ax[a][ia[a]]; w = a; }
        double ds = s1 - s0;
        if (ds > 1e-14) {
            double sm = 0.5 * (s0 + s1);
            int idx[3];
            for (int a = 0; a < 3; ++a) {
                int i = (int)floor((P[a] + sm * D[a] - o[a]) / h[a]);
                if (i < 0) i = 0;
                if (i >= n[a]) i = n[a] - 1;
                idx[a] = i;
            }
            int32_t j = (int32_t)(((int64_t)idx[2] * n[1] + idx[1]) * n[0] + idx[0]);
            rb_add(rb, j, ds * L);
        }
        if (w < 0) break;
        ia[w]++;
        s0 = s1;
    }
}

static inline double h10(double s) { return s * s * s - 2.0 * s * s + s; }
static inline double h11(double s) { return s * s * s - s * s; }

/* Trace row r into rb (lengths merged per voxel, short ones dropped).
 * Path: chord of the in-plane line {t*n + s*u} across the grid square at height z;
 * bent paths add A*h10(sigma)+B*h11(sigma) along n and along z (|offset| <= dev_max). */
static void trace_row(const syn_cfg* c, double t, double z, uint64_t key, int a, rowbuf* rb, double* sbuf) {
    rb->n = 0;   /* invariant: the hash is empty between rows */
    double th = (c->angle_span_deg * a / c->n_angles) * (M_PI / 180.0);
    double ux = cos(th), uy = sin(th), nxv = -sin(th), nyv = cos(th);
    double hx = 0.5 * c->nx * c->dx, hy = 0.5 * c->ny * c->dy;
    /* chord parameter range where the in-plane line is inside the grid square */
    double lo = -1e300, hi = 1e300;
    double px = t * nxv, py = t * nyv;
    if (ux != 0.0) {
        double s0 = (-hx - px) / ux, s1 = (hx - px) / ux;
        if (s0 > s1) { double q = s0; s0 = s1; s1 = q; }
        if (s0 > lo) lo = s0;
        if (s1 < hi) hi = s1;
    } else if (px < -hx || px > hx) return;
    if (uy != 0.0) {
        double s0 = (-hy - py) / uy, s1 = (hy - py) / uy;
        if (s0 > s1) { double q = s0; s0 = s1; s1 = q; }
        if (s0 > lo) lo = s0;
        if (s1 < hi) hi = s1;
    } else if (py < -hy || py > hy) return;
    if (!(hi > lo)) return;
    lo -= 1.0; hi += 1.0;    /* start and end just outside the grid */
    if (!c->curved) {
        double P[3] = {px + lo * ux, py + lo * uy, z}, Q[3] = {px + hi * ux, py + hi * uy, z};
        trace_segment(c, P, Q, rb, sbuf);
    } else {
        double k = (27.0 / 8.0) * c->dev_max;
        double Al = (2.0 * u01(c->seed, key * DRAWS_PER_HIST + 2) - 1.0) * k;
        double Bl = (2.0 * u01(c->seed, key * DRAWS_PER_HIST + 3) - 1.0) * k;
        double Az = (2.0 * u01(c->seed, key * DRAWS_PER_HIST + 4) - 1.0) * k;
        double Bz = (2.0 * u01(c->seed, key * DRAWS_PER_HIST + 5) - 1.0) * k;
        double prev[3];
        for (int q = 0; q <= c->n_seg; ++q) {
            double sg = (double)q / c->n_seg;
            double s = lo + sg * (hi - lo);
            double ol = Al * h10(sg) + Bl * h11(sg), oz = Az * h10(sg) + Bz * h11(sg);
            double cur[3] = {px + s * ux + ol * nxv, py + s * uy + ol * nyv, z + oz};
            if (q > 0) trace_segment(c, prev, cur, rb, sbuf);
            prev[0] = cur[0]; prev[1] = cur[1]; prev[2] = cur[2];
        }
    }
    rb_erase_hash(rb);
    int w = 0;   /* drop short intersections (keeps stored-precision hit counts stable) */
    for (int i = 0; i < rb->n; ++i)
        if (rb->len[i] >= c->min_len) { rb->col[w] = rb->col[i]; rb->len[w] = rb->len[i]; ++w; }
    rb->n = w;
}


/* pass 1: nonzeros of rows 0..n-1 of the plan arrays passed */
void syn_count(const syn_cfg* c, int64_t n, const double* t, const double* z, const uint64_t* key,
               const int32_t* angle, int64_t* row_nnz) {
    #pragma omp parallel
    {
        rowbuf rb; rb_init(&rb);
        double* sbuf = (double*)malloc(sizeof(double) * (size_t)seg_scratch(c));
        #pragma omp for schedule(dynamic, 1024)
        for (int64_t r = 0; r < n; ++r) {
            trace_row(c, t[r], z[r], key[r], angle[r], &rb, sbuf);
            row_nnz[r] = rb.n;
        }
        free(sbuf); rb_free(&rb);
    }
}

/* pass 2: write col / val (val_dtype 0 = f64, 1 = f32) and b of rows 0..n-1 of the plan
 * arrays passed.  b_r = (sum_j len_rj * xstar_j) * (1 + noise_sigma * N(0,1)), from the
 * f64 lengths. */
void syn_fill(const syn_cfg* c, int64_t n, const double* t, const double* z, const uint64_t* key,
              const int32_t* angle, const int64_t* row_ptr, int32_t* col, void* val, int32_t val_dtype,
              double* b, const double* xstar) {
    #pragma omp parallel
    {
        rowbuf rb; rb_init(&rb);
        double* sbuf = (double*)malloc(sizeof(double) * (size_t)seg_scratch(c));
        #pragma omp for schedule(dynamic, 1024)
        for (int64_t r = 0; r < n; ++r) {
            trace_row(c, t[r], z[r], key[r], angle[r], &rb, sbuf);
            int64_t p = row_ptr[r];
            double wepl = 0.0;
            for (int i = 0; i < rb.n; ++i) {
                col[p + i] = rb.col[i];
                if (val_dtype == 0) ((double*)val)[p + i] = rb.len[i];
                else ((float*)val)[p + i] = (float)rb.len[i];
                wepl += rb.len[i] * xstar[rb.col[i]];
            }
            double u1 = 1.0 - u01(c->seed, key[r] * DRAWS_PER_HIST + 6);   /* (0,1] */
            double u2 = u01(c->seed, key[r] * DRAWS_PER_HIST + 7);
            double gauss = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);       /* Box-Muller */
            b[r] = wepl * (1.0 + c->noise_sigma * gauss);
        }
        free(sbuf); rb_free(&rb);
    }
}

/* raw SplitMix64 stream value, exported for tests of the generator itself */
uint64_t syn_splitmix64_at(uint64_t seed, uint64_t n) { return sm64_at(seed, n); }

/* ------------------------------------------------------------ path records */
/* The path of row r as 10 floats: chord start P_in (x, y, z), chord end P_out (x, y, z),
 * and the cubic-Hermite offset coefficients (A_lat, B_lat, A_z, B_z): the path is
 *   P(s) = P_in + s (P_out - P_in) + (A_lat h10(s) + B_lat h11(s)) n + (A_z h10(s) + B_z h11(s)) e_z,
 * s in [0, 1], n the in-plane unit normal (-u_y, u_x) of the chord direction u, split into
 * n_seg straight segments at s = q / n_seg.  Rows whose line misses the grid get
 * P_in = P_out (an empty row). */
void syn_paths(const syn_cfg* c, int64_t n, const double* t, const double* z, const uint64_t* key,
               const int32_t* angle, float* out) {
    #pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n; ++r) {
        float* o = out + 10 * r;
        double th = (c->angle_span_deg * angle[r] / c->n_angles) * (M_PI / 180.0);
        double ux = cos(th), uy = sin(th), nxv = -sin(th), nyv = cos(th);
        double hx = 0.5 * c->nx * c->dx, hy = 0.5 * c->ny * c->dy;
        double lo = -1e300, hi = 1e300;
        double px = t[r] * nxv, py = t[r] * nyv;
        int miss = 0;
        if (ux != 0.0) {
            double s0 = (-hx - px) / ux, s1 = (hx - px) / ux;
            if (s0 > s1) { double q = s0; s0 = s1; s1 = q; }
            if (s0 > lo) lo = s0;
            if (s1 < hi) hi = s1;
        } else if (px < -hx || px > hx) miss = 1;
        if (uy != 0.0) {
            double s0 = (-hy - py) / uy, s1 = (hy - py) / uy;
            if (s0 > s1) { double q = s0; s0 = s1; s1 = q; }
            if (s0 > lo) lo = s0;
            if (s1 < hi) hi = s1;
        } else if (py < -hy || py > hy) miss = 1;
        if (miss || !(hi > lo)) {
            for (int k = 0; k < 10; ++k) o[k] = 0.0f;
            continue;
        }
        lo -= 1.0; hi += 1.0;
        o[0] = (float)(px + lo * ux); o[1] = (float)(py + lo * uy); o[2] = (float)z[r];
        o[3] = (float)(px + hi * ux); o[4] = (float)(py + hi * uy); o[5] = (float)z[r];
        if (c->curved) {
            double k = (27.0 / 8.0) * c->dev_max;
            o[6] = (float)((2.0 * u01(c->seed, key[r] * DRAWS_PER_HIST + 2) - 1.0) * k);
            o[7] = (float)((2.0 * u01(c->seed, key[r] * DRAWS_PER_HIST + 3) - 1.0) * k);
            o[8] = (float)((2.0 * u01(c->seed, key[r] * DRAWS_PER_HIST + 4) - 1.0) * k);
            o[9] = (float)((2.0 * u01(c->seed, key[r] * DRAWS_PER_HIST + 5) - 1.0) * k);
        } else {
            o[6] = o[7] = o[8] = o[9] = 0.0f;
        }
    }
}

/* b of rows 0..n-1 without storing them: the same trace and noise as syn_fill. */
void syn_rhs(const syn_cfg* c, int64_t n, const double* t, const double* z, const uint64_t* key,
             const int32_t* angle, double* b, const double* xstar) {
    #pragma omp parallel
    {
        rowbuf rb; rb_init(&rb);
        double* sbuf = (double*)malloc(sizeof(double) * (size_t)seg_scratch(c));
        #pragma omp for schedule(dynamic, 1024)
        for (int64_t r = 0; r < n; ++r) {
            trace_row(c, t[r], z[r], key[r], angle[r], &rb, sbuf);
            double wepl = 0.0;
            for (int i = 0; i < rb.n; ++i) wepl += rb.len[i] * xstar[rb.col[i]];
            double u1 = 1.0 - u01(c->seed, key[r] * DRAWS_PER_HIST + 6);
            double u2 = u01(c->seed, key[r] * DRAWS_PER_HIST + 7);
            double gauss = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
            b[r] = wepl * (1.0 + c->noise_sigma * gauss);
        }
        free(sbuf); rb_free(&rb);
    }
}
