/*
 * FP64 CPU oracle for NTVS reconstruction (arXiv 1803.01112).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously-correct
 * restatement of the method, used by the tests, by the smoke check and by the
 * CPU-baseline leg of the benchmark.  The product library never links, loads or
 * calls it, and it shares no code with the CUDA path.
 *
 * What it follows:
 *   - NTVS outer loop, without and with the TV-reduction check: Appendix C
 *     (Algorithm "NTVS" and its variant with the TV reduction requirement),
 *     notation of Appendix A.
 *   - ell schedule: ell_k = rand(k, ell_{k-1}), Sec. III-B (item 4) and Appendix C.
 *   - step size beta_{k,n} = alpha^{ell_k}, Sec. III-B and Appendix A; the paper's
 *     beta_0 = 1 is exposed as beta0.
 *   - OTVS (Appendix B): ell is never reset between cycles, beta = (1/2)^ell.
 *   - decoupled step size beta_{k,n} = alpha^n gamma^{f(k)}, f(k) = k (Sec. VI).
 *   - phi = TV, the sum over the voxels of the local variation (introduced in Sec. II
 *     with ref. CCCNP10);
 *     v = -grad phi / ||grad phi|| (Appendix A).
 *   - P_T = one sweep of block-DROP (Sec. III-D cites the DROP algorithm of ref.
 *     CEHN08 without printing its update).
 * Readings where the paper is silent or garbled (all listed in the design notes):
 *   - DROP step for block t (rows B_t, all using the same x):
 *       x_j <- x_j + lambda * (1/s_j) * sum_{i in B_t} a_ij (b_i - <a_i,x>) / ||a_i||^2
 *     with s_j = number of rows of B_t with a_ij != 0; voxels with s_j = 0 and rows
 *     with ||a_i|| = 0 contribute nothing.
 *   - TV: isotropic forward differences on index spacing with a Neumann boundary
 *     (a difference past the last index is 0); phi has no epsilon; the gradient is
 *     that of phi_eps(x) = sum_p sqrt(eps + |forward differences at p|^2).
 *   - rand(a, b): uniform integer in [min(a,b), max(a,b)], drawn for cycle k as
 *     lo + (SplitMix64 output k of stream `seed`) mod (hi - lo + 1).
 *   - check variant: beta is recomputed as beta0*alpha^ell after each ell++ (the
 *     printed loop never updates beta); a tie phi(z) == phi(x) accepts; after
 *     max_retries rejected tries x is left unchanged.
 *   - decoupled rule: n and k are counted from 0 as in the Appendix C loops, so the
 *     first step of the first cycle is beta0; it is stated without the check, and is
 *     only defined here without it.
 */
/* The OpenMP pragmas below only act in the separate timing build (compiled with
 * -fopenmp, used to time the method on all host cores); the checker is compiled without
 * OpenMP, where they are ignored and every loop runs in the order written. */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
static int orc_nthreads(void) { return omp_get_max_threads(); }
static int orc_thread(void) { return omp_get_thread_num(); }
#else
static int orc_nthreads(void) { return 1; }
static int orc_thread(void) { return 0; }
#endif

/* ------------------------------------------------------------------ RNG */
/* SplitMix64 (Steele, Lea, Flood 2014), counter form: output n of stream seed. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t n) {
    uint64_t z = seed + (n + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* ell_k = rand(k, ell_{k-1}) : uniform integer between the two, inclusive. */
int64_t orc_rand_ell(uint64_t seed, int64_t k, int64_t ell_prev) {
    int64_t lo = k < ell_prev ? k : ell_prev;
    int64_t hi = k < ell_prev ? ell_prev : k;
    uint64_t span = (uint64_t)(hi - lo) + 1u;
    return lo + (int64_t)(orc_splitmix64(seed, (uint64_t)k) % span);
}

/* ------------------------------------------------------------------- TV */
static int64_t vid(int nx, int ny, int ix, int iy, int iz) {
    return ((int64_t)iz * ny + iy) * nx + ix;
}

/* forward differences at voxel (ix,iy,iz); zero past the last index */
static void fwd_diff(const double* x, int nx, int ny, int nz, int ix, int iy, int iz, double d[3]) {
    double c = x[vid(nx, ny, ix, iy, iz)];
    d[0] = (ix + 1 < nx) ? x[vid(nx, ny, ix + 1, iy, iz)] - c : 0.0;
    d[1] = (iy + 1 < ny) ? x[vid(nx, ny, ix, iy + 1, iz)] - c : 0.0;
    d[2] = (iz + 1 < nz) ? x[vid(nx, ny, ix, iy, iz + 1)] - c : 0.0;
}

/* phi_eps(x) = sum_p sqrt(eps + sum_a d_a(p)^2); eps = 0 gives the TV phi. */
double orc_tv(const double* x, int nx, int ny, int nz, double eps) {
    double s = 0.0;
#pragma omp parallel for collapse(2) reduction(+ : s) schedule(static)
    for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix) {
                double d[3];
                fwd_diff(x, nx, ny, nz, ix, iy, iz, d);
                s += sqrt(eps + d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            }
    return s;
}

/* D_c = sqrt(eps + |d(c)|^2) */
static double Dval(const double* x, int nx, int ny, int nz, int ix, int iy, int iz, double eps) {
    double d[3];
    fwd_diff(x, nx, ny, nz, ix, iy, iz, d);
    return sqrt(eps + d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
}

/* g = grad phi_eps(x):
 *   g_q = sum_a [q+e_a inside] (x_q - x_{q+e_a}) / D_q
 *       + sum_a [q-e_a inside] (x_q - x_{q-e_a}) / D_{q-e_a}
 * A term whose D is 0 is 0 (its numerator is 0 as well). */
void orc_tv_grad(const double* x, int nx, int ny, int nz, double eps, double* g) {
    const int n[3] = {nx, ny, nz};
#pragma omp parallel for collapse(2) schedule(static)
    for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix) {
                int q[3] = {ix, iy, iz};
                double xq = x[vid(nx, ny, ix, iy, iz)];
                double Dq = Dval(x, nx, ny, nz, ix, iy, iz, eps);
                double acc = 0.0;
                for (int a = 0; a < 3; ++a) {
                    int p[3] = {q[0], q[1], q[2]};
                    p[a] = q[a] + 1;
                    if (p[a] < n[a] && Dq > 0.0)
                        acc += (xq - x[vid(nx, ny, p[0], p[1], p[2])]) / Dq;
                    p[a] = q[a] - 1;
                    if (p[a] >= 0) {
                        double Dm = Dval(x, nx, ny, nz, p[0], p[1], p[2], eps);
                        if (Dm > 0.0) acc += (xq - x[vid(nx, ny, p[0], p[1], p[2])]) / Dm;
                    }
                }
                g[vid(nx, ny, ix, iy, iz)] = acc;
            }
}

/* ----------------------------------------------------------------- DROP */
/* One block-DROP step over rows [r0, r1): every row uses the x on entry.
 * Returns sum_i (b_i - <a_i,x>)^2 over the block (x on entry) in *resid_ss. */
void orc_drop_block(const int64_t* row_ptr, const int32_t* col, const double* val, const double* b,
                    int64_t r0, int64_t r1, int64_t V, double lambda, double* x, double* resid_ss) {
    int64_t m = r1 - r0;
    double* r = (double*)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    double* num = (double*)calloc((size_t)V, sizeof(double));
    int64_t* s = (int64_t*)calloc((size_t)V, sizeof(int64_t));
    double ss = 0.0;
#pragma omp parallel for reduction(+ : ss) schedule(static)
    for (int64_t i = r0; i < r1; ++i) {
        double dot = 0.0, nrm2 = 0.0;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            dot += val[p] * x[col[p]];
            nrm2 += val[p] * val[p];
        }
        double res = b[i] - dot;
        ss += res * res;
        r[i - r0] = (nrm2 > 0.0) ? res / nrm2 : 0.0;
    }
    /* num_j = sum_i a_ij r_i and s_j: each thread sums its rows into its own arrays, which
     * are then added voxel by voxel (one thread: the rows in order, then 0 + that sum) */
    const int nt = orc_nthreads();
    double** pn = (double**)calloc((size_t)nt, sizeof(double*));
    int64_t** ps = (int64_t**)calloc((size_t)nt, sizeof(int64_t*));
#pragma omp parallel num_threads(nt)
    {
        const int t = orc_thread();
        double* num_t = pn[t] = (double*)calloc((size_t)V, sizeof(double));
        int64_t* s_t = ps[t] = (int64_t*)calloc((size_t)V, sizeof(int64_t));
#pragma omp for schedule(static)
        for (int64_t i = r0; i < r1; ++i)
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
                num_t[col[p]] += val[p] * r[i - r0];
                if (val[p] != 0.0) s_t[col[p]] += 1;
            }
#pragma omp for schedule(static)
        for (int64_t j = 0; j < V; ++j) {
            double a = 0.0;
            int64_t c = 0;
            for (int u = 0; u < nt; ++u) {
                a += pn[u][j];
                c += ps[u][j];
            }
            num[j] = a;
            s[j] = c;
        }
    }
    for (int u = 0; u < nt; ++u) { free(pn[u]); free(ps[u]); }
    free(pn); free(ps);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < V; ++j)
        if (s[j] > 0) x[j] += lambda * num[j] / (double)s[j];
    if (resid_ss) *resid_ss = ss;
    free(r); free(num); free(s);
}

/* P_T: blocks t = 0..B-1 in order, block t = rows [block_ptr[t], block_ptr[t+1]). */
void orc_drop_sweep(const int64_t* row_ptr, const int32_t* col, const double* val, const double* b,
                    const int64_t* block_ptr, int B, int64_t V, double lambda, double* x, double* resid_ss) {
    for (int t = 0; t < B; ++t)
        orc_drop_block(row_ptr, col, val, b, block_ptr[t], block_ptr[t + 1], V, lambda, x,
                       resid_ss ? resid_ss + t : NULL);
}

/* The DROP block of orc_drop_block evaluated only at the listed voxels: out[q] is the
 * updated value of voxel vox[q], x is not modified.  For checks at sizes where the
 * full block is too slow; same formula, same order of terms per voxel. */
void orc_drop_block_at(const int64_t* row_ptr, const int32_t* col, const double* val, const double* b,
                       int64_t r0, int64_t r1, int64_t V, double lambda, const double* x,
                       int64_t n_vox, const int64_t* vox, double* out) {
    char* want = (char*)calloc((size_t)V, 1);
    double* num = (double*)calloc((size_t)V, sizeof(double));
    int64_t* s = (int64_t*)calloc((size_t)V, sizeof(int64_t));
    for (int64_t q = 0; q < n_vox; ++q) want[vox[q]] = 1;
    for (int64_t i = r0; i < r1; ++i) {
        int hit = 0;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) hit |= want[col[p]];
        if (!hit) continue;
        double dot = 0.0, nrm2 = 0.0;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            dot += val[p] * x[col[p]];
            nrm2 += val[p] * val[p];
        }
        double ri = (nrm2 > 0.0) ? (b[i] - dot) / nrm2 : 0.0;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
            if (want[col[p]]) {
                num[col[p]] += val[p] * ri;
                if (val[p] != 0.0) s[col[p]] += 1;
            }
    }
    for (int64_t q = 0; q < n_vox; ++q) {
        int64_t j = vox[q];
        out[q] = x[j] + ((s[j] > 0) ? lambda * num[j] / (double)s[j] : 0.0);
    }
    free(want); free(num); free(s);
}

/* ----------------------------------------------------------------- NTVS */
/* step_rule: how the step sizes of cycle k are chosen.
 *   0  NTVS (Appendix C): ell_k = rand(k, ell_{k-1}); step n uses beta0 * alpha^ell, ell++
 *      after every try.
 *   1  OTVS (Appendix B): ell is never reset: ell_k = ell_{k-1}, and otherwise as rule 0.
 *      The paper's OTVS is this rule with N = 1, alpha = 1/2, beta0 = 1 and the TV check.
 *   2  decoupled (Sec. VI): beta_{k,n} = beta0 * alpha^n * gamma^k for n = 0..N-1, with no
 *      ell; defined without the TV check. */
typedef struct {
    double lambda, alpha, beta0, eps_tv;
    int32_t N, tv_check, max_retries, step_rule;
    uint64_t seed;
    double gamma;
} orc_params;

typedef struct {
    int64_t* ell_k;        /* [K]   ell_k drawn at the start of cycle k (or replayed)   */
    int64_t* ell_step;     /* [K*N] ell used by the accepted / last try of step n      */
    int32_t* tries;        /* [K*N] tries made at step n (1 without the check)         */
    int32_t* accepted;     /* [K*N] 1 if step n changed x                              */
    double* tv;            /* [K]   phi(x^{k+1})                                       */
    double* resid_ss;      /* [K*B] per-block residual sum of squares                  */
    double* beta_step;     /* [K*N] beta of the accepted / last try of step n          */
} orc_trace;

/* x <- x + beta * v, v = -g/||g|| (v = 0 when ||g|| = 0). */
static void perturb(double* z, const double* x, const double* g, double gnorm, double beta, int64_t V) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < V; ++j) z[j] = x[j] + ((gnorm > 0.0) ? beta * (-g[j] / gnorm) : 0.0);
}

/* K cycles of NTVS (Appendix C) from x (in/out).  ell_override: if not NULL, ell_k is
 * taken from it instead of being drawn (replays a recorded schedule).  ell_prev_io
 * carries ell_{k-1} between calls (start with 0); k0 is the index of the first cycle.
 * Under the decoupled rule ell_k records k and ell_prev_io is left as it is.  Returns -1
 * (nothing done) for an unknown rule or the decoupled rule with the TV check. */
int orc_ntvs(const int64_t* row_ptr, const int32_t* col, const double* val, const double* b,
             const int64_t* block_ptr, int B, int nx, int ny, int nz, const orc_params* prm,
             int K, int k0, int64_t* ell_prev_io, const int64_t* ell_override, double* x, orc_trace* tr) {
    const int64_t V = (int64_t)nx * ny * nz;
    const int N = prm->N;
    const int rule = prm->step_rule;
    if (rule < 0 || rule > 2 || (rule == 2 && prm->tv_check)) return -1;
    double* g = (double*)malloc(sizeof(double) * (size_t)(V > 0 ? V : 1));
    double* z = (double*)malloc(sizeof(double) * (size_t)(V > 0 ? V : 1));
    int64_t ell_prev = *ell_prev_io;
    for (int kk = 0; kk < K; ++kk) {
        int64_t k = k0 + kk;
        int64_t ell;
        if (ell_override) ell = ell_override[kk];
        else if (rule == 0) ell = orc_rand_ell(prm->seed, k, ell_prev);
        else if (rule == 1) ell = ell_prev;
        else ell = k;
        if (tr && tr->ell_k) tr->ell_k[kk] = ell;
        for (int n = 0; n < N; ++n) {
            orc_tv_grad(x, nx, ny, nz, prm->eps_tv, g);
            double gn = 0.0;
#pragma omp parallel for reduction(+ : gn) schedule(static)
            for (int64_t j = 0; j < V; ++j) gn += g[j] * g[j];
            gn = sqrt(gn);
            double beta = (rule == 2) ? prm->beta0 * pow(prm->alpha, (double)n) * pow(prm->gamma, (double)k)
                                      : prm->beta0 * pow(prm->alpha, (double)ell);
            double beta_used = beta;
            int tries = 0, acc = 0;
            int64_t ell_used = ell;
            if (!prm->tv_check) {
                perturb(x, x, g, gn, beta, V);
                ell_used = ell;
                if (rule != 2) ell += 1;
                tries = 1; acc = 1;
            } else {
                double phi_x = orc_tv(x, nx, ny, nz, 0.0);
                for (;;) {
                    perturb(z, x, g, gn, beta, V);
                    ell_used = ell;
                    beta_used = beta;
                    ell += 1;
                    tries += 1;
                    if (orc_tv(z, nx, ny, nz, 0.0) <= phi_x) {
                        memcpy(x, z, sizeof(double) * (size_t)V);
                        acc = 1;
                        break;
                    }
                    if (tries >= prm->max_retries) break;
                    beta = prm->beta0 * pow(prm->alpha, (double)ell);
                }
            }
            if (tr && tr->ell_step) tr->ell_step[(int64_t)kk * N + n] = ell_used;
            if (tr && tr->tries) tr->tries[(int64_t)kk * N + n] = tries;
            if (tr && tr->accepted) tr->accepted[(int64_t)kk * N + n] = acc;
            if (tr && tr->beta_step) tr->beta_step[(int64_t)kk * N + n] = beta_used;
        }
        if (rule != 2) ell_prev = ell;
        orc_drop_sweep(row_ptr, col, val, b, block_ptr, B, V, prm->lambda, x,
                       (tr && tr->resid_ss) ? tr->resid_ss + (int64_t)kk * B : NULL);
        if (tr && tr->tv) tr->tv[kk] = orc_tv(x, nx, ny, nz, 0.0);
    }
    *ell_prev_io = ell_prev;
    free(g); free(z);
    return 0;
}
