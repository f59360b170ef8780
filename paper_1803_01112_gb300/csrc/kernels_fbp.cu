// Initial iterate x-bar (arXiv 1803.01112: x-bar of Appendix A, FBP of Sec. II, median
// filter of radius 2 on the initial iterate in Sec. V-A): chord binning, Ram-Lak filter,
// back-projection, median filter and threshold hull, all in FP64.  The steps follow the
// specification in include/ntvs_fbp.h.
//
// Kernels and their bounds (CTP404 scale: 10M histories, 16 x 180 x 200 bins, 200x200x16
// voxels):
//   fbp_bin_kernel       one thread per history; 24 B read per history; bin sums by
//                        one FP64 atomic per run of equal bins in a warp (segmented suffix
//                        sum; acquisition order gives runs); FP32 atan2 with an FP64 recheck
//                        near angle-bin edges, FP64 sqrt and three FP64 divisions.
//   fbp_filter_kernel    one CTA per (slice, angle) row; the row and the odd-lag kernel in
//                        shared memory; n_t^2/2 FMAs per row.
//   fbp_backproject_kernel one thread per 4 voxels of a row, 128x8 tiles of a slice;
//                        cos/sin of every angle in shared memory; two L1/L2-resident loads
//                        and 7 FP64-pipe operations per (voxel, angle) (FMA, two
//                        conversions, three adds, FMA): FP64-pipe bound on GB300.
//   median_kernel        one thread per voxel; the window as monotone 64-bit integer keys
//                        in registers, the element floor(n/2) by rank counting (W^2
//                        integer compares, no FP64 pipe); the hull fused into the store.
#include <math.h>

#include <string>

#include "common.cuh"
#include "ntvs_fbp.h"

namespace ntvs {

namespace {

constexpr int kMaxNt = 8192;
constexpr int kMaxNtheta = 4096;
constexpr int kMaxMedianRadius = 3;
constexpr double kPi = 3.14159265358979323846;

int fbp_fail(int code, const std::string& msg) {
    set_last_error(msg);   // read back with ntvs_last_error()
    return code;
}

int launch_status(const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fbp_fail(NTVS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return NTVS_OK;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

int check_geom(const ntvs_fbp_geom* g, const char* where) {
    if (!g) return fbp_fail(NTVS_ERR_ARG, std::string(where) + ": null geometry");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1 || g->n_theta < 1 || g->n_t < 1)
        return fbp_fail(NTVS_ERR_ARG, std::string(where) + ": grid and bin counts must be >= 1");
    if (g->reserved != 0) return fbp_fail(NTVS_ERR_ARG, std::string(where) + ": reserved must be 0");
    if (g->n_t > kMaxNt) return fbp_fail(NTVS_ERR_ARG, std::string(where) + ": n_t > 8192");
    if (g->n_theta > kMaxNtheta) return fbp_fail(NTVS_ERR_ARG, std::string(where) + ": n_theta > 4096");
    if (g->nz > 65535) return fbp_fail(NTVS_ERR_ARG, std::string(where) + ": nz > 65535");
    if (!finite_pos(g->dx) || !finite_pos(g->dy) || !finite_pos(g->dz) || !finite_pos(g->dt))
        return fbp_fail(NTVS_ERR_ARG, std::string(where) + ": dx, dy, dz and dt must be finite and > 0");
    if (!std::isfinite(g->theta0) || fabs(g->theta0) > 16.0 * kPi)
        return fbp_fail(NTVS_ERR_ARG, std::string(where) + ": theta0 must be finite with |theta0| <= 16 pi");
    const int64_t V = (int64_t)g->nx * g->ny * g->nz;
    const int64_t S = (int64_t)g->nz * g->n_theta * g->n_t;
    if (V > INT32_MAX || S > INT32_MAX)
        return fbp_fail(NTVS_ERR_ARG, std::string(where) + ": more than 2^31 - 1 voxels or bins");
    return NTVS_OK;
}

// ---------------------------------------------------------------- 1. binning

// (phi, t) of a line whose normal is at angle theta (any value in [-pi, 2 pi)) with
// lateral offset t: the fold into [0, pi) and the rebase to theta0 of step 1.
__device__ __forceinline__ double fold_rebase(double theta, double& t, double theta0) {
    if (theta < 0.0) theta += 2.0 * kPi;
    if (theta >= kPi) {
        theta -= kPi;
        t = -t;
    }
    double phi = theta - theta0;   // |theta0| <= 16 pi is checked by the host: at most 18 steps
    for (int i = 0; i < 64 && phi < 0.0; ++i) {
        phi += kPi;
        t = -t;
    }
    for (int i = 0; i < 64 && phi >= kPi; ++i) {
        phi -= kPi;
        t = -t;
    }
    return phi;
}

// Flat bin of one chord record, or -1 when it falls outside the bins (step 1), decided in
// FP64.  The normal's angle is first taken from the FP32 atan2 of the chord direction
// (error below 1e-6 rad, the FP32 rounding of the direction included): when the rebased
// angle lies more than 1e-5 rad from every angle-bin edge (the fold at theta = pi is
// continuous in the bin it gives, except where it is itself an edge), the FP64 angle gives
// the same bin; otherwise the angle is recomputed with the FP64 atan2.  t is the FP64
// projection of P_in on the unit normal.
__device__ __forceinline__ int64_t bin_of(const float* __restrict__ rec, const ntvs_fbp_geom& g) {
    const double px = __ldg(rec + 0), py = __ldg(rec + 1), pz = __ldg(rec + 2);
    const double qx = __ldg(rec + 3), qy = __ldg(rec + 4), qz = __ldg(rec + 5);
    const double ddx = qx - px, ddy = qy - py;
    const double len = sqrt(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)));
    if (!(len > 0.0)) return -1;
    const double t0 = __dadd_rn(__dmul_rn(px, -ddy), __dmul_rn(py, ddx)) / len;   // normal (-ddy, ddx)/len
    const double w = kPi / g.n_theta;
    double t = t0;
    double phi = fold_rebase((double)atan2f((float)ddx, (float)-ddy), t, g.theta0);
    const double f = phi / w - floor(phi / w);
    if (fmin(f, 1.0 - f) * w < 1e-5 || len < 1e-30) {   // near an edge, or FP32 would underflow
        t = t0;
        phi = fold_rebase(atan2(ddx, -ddy), t, g.theta0);
    }
    if (!(phi >= 0.0 && phi < kPi)) return -1;   // unreachable for |theta0| <= 16 pi
    int64_t a = (int64_t)floor(phi / w);
    a = a < 0 ? 0 : (a > g.n_theta - 1 ? g.n_theta - 1 : a);
    const double u = __dadd_rn(t / g.dt, 0.5 * g.n_t);
    if (!(u >= 0.0 && u < (double)g.n_t)) return -1;
    const double v = __dmul_rn(0.5, pz + qz) / g.dz;
    if (!(v >= 0.0 && v < (double)g.nz)) return -1;
    int64_t k = (int64_t)floor(u), iz = (int64_t)floor(v);
    if (k > g.n_t - 1) k = g.n_t - 1;
    if (iz > g.nz - 1) iz = g.nz - 1;
    return (iz * g.n_theta + a) * g.n_t + k;
}

// Bin sums and counts.  Every lane of a warp takes one history.  Lanes with equal bins
// next to each other form a run (histories in acquisition order give runs of one bin);
// a segmented suffix sum over each run (five shuffle steps) leaves the run's sum in its
// first lane, which adds it and the run length with one atomic each.  Equal bins that are
// not adjacent make separate runs, which is still correct.  The loop bound is warp-
// uniform so that every shuffle has all 32 lanes.
__global__ void __launch_bounds__(256) fbp_bin_kernel(ntvs_fbp_geom g, const float* __restrict__ paths,
                                                      const double* __restrict__ wepl, int64_t M,
                                                      double* __restrict__ sum, int32_t* __restrict__ count) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * 32; base < M; base += nwarps * 32) {
        const int64_t h = base + lane;
        int64_t key = -1;
        double w = 0.0;
        if (h < M) {
            key = bin_of(paths + 10 * h, g);
            w = __ldg(wepl + h);
        }
        const int64_t next = __shfl_down_sync(0xffffffffu, key, 1);
        const unsigned last = __ballot_sync(0xffffffffu, lane == 31 || next != key);   // bit l: run ends at l
        const int end = __ffs(last & (0xffffffffu << lane)) - 1;                     // this lane's run end
        double s = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double v = __shfl_down_sync(0xffffffffu, s, o);
            if (lane + o <= end) s += v;
        }
        const bool head = lane == 0 || ((last >> (lane - 1)) & 1u);
        if (head && key >= 0) {
            atomicAdd(sum + key, s);
            atomicAdd(count + key, end - lane + 1);
        }
    }
}

__global__ void fbp_mean_kernel(double* __restrict__ sino, const int32_t* __restrict__ count, int64_t S) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = count[i];
        sino[i] = c > 0 ? sino[i] / (double)c : 0.0;
    }
}

// ---------------------------------------------------------------- 2. filtering

// One CTA per (slice, angle) row: the row p and the odd-lag kernel values
// hodd[j] = h(2j + 1) in shared memory; q_k = dt (p_k h(0) + sum over odd lags), the
// terms taken in ascending n as in the definition (even lags add exact zeros there).
__global__ void __launch_bounds__(256) fbp_filter_kernel(const double* __restrict__ sino, double* __restrict__ q,
                                                         int nt, double dt) {
    extern __shared__ double fsm[];
    double* p = fsm;            // [nt]
    double* hodd = fsm + nt;    // [nt/2 + 1]
    const int64_t row = blockIdx.x;
    const double* src = sino + row * nt;
    for (int i = threadIdx.x; i < nt; i += blockDim.x) p[i] = src[i];
    const int nh = nt / 2 + 1;
    for (int j = threadIdx.x; j < nh; j += blockDim.x) {
        const double m = (double)(2 * j + 1);
        hodd[j] = -1.0 / (kPi * kPi * m * m * dt * dt);
    }
    __syncthreads();
    const double h0 = 1.0 / (4.0 * dt * dt);
    for (int k = threadIdx.x; k < nt; k += blockDim.x) {
        double s = 0.0;
        // n < k with k - n odd: n = k-1, k-3, ... taken in ascending order
        for (int n = (k & 1) ^ 1; n < k; n += 2) s += p[n] * hodd[(k - n - 1) >> 1];
        s += p[k] * h0;
        for (int n = k + 1; n < nt; n += 2) s += p[n] * hodd[(n - k - 1) >> 1];
        q[row * nt + k] = dt * s;
    }
}

// ---------------------------------------------------------------- 3. back-projection

constexpr int kBpTx = 32, kBpTy = 8, kBpVx = 4;   // a CTA covers 128 x 8 voxels of one slice

// One thread per 4 voxels of a row (x = ix, ix+32, ix+64, ix+96 within the CTA's 128).
// Shared memory holds, per bin angle, cos(theta_a)/dt and sin(theta_a)/dt; the position of
// voxel (x, y) in bin units is u = x cos/dt + (y sin/dt + n_t/2 - 1/2): one FMA per voxel
// once the row's y term is formed.  The angles are summed in ascending order, as defined;
// the interpolation is v0 + w (v1 - v0).
__global__ void __launch_bounds__(kBpTx * kBpTy) fbp_backproject_kernel(ntvs_fbp_geom g, const double* __restrict__ q,
                                                                         double* __restrict__ img) {
    extern __shared__ double bsm[];
    double* cs = bsm;                 // [n_theta] cos(theta_a) / dt
    double* sn = bsm + g.n_theta;     // [n_theta] sin(theta_a) / dt
    const int na = g.n_theta, nt = g.n_t;
    const double inv_dt = 1.0 / g.dt;
    for (int a = threadIdx.y * kBpTx + threadIdx.x; a < na; a += kBpTx * kBpTy) {
        const double th = g.theta0 + ((double)a + 0.5) * kPi / (double)na;
        double sa, ca;
        sincos(th, &sa, &ca);
        cs[a] = ca * inv_dt;
        sn[a] = sa * inv_dt;
    }
    __syncthreads();
    const int iy = blockIdx.y * kBpTy + threadIdx.y, iz = blockIdx.z;
    if (iy >= g.ny) return;
    const int ix0 = blockIdx.x * (kBpTx * kBpVx) + threadIdx.x;
    const double y = ((double)iy + 0.5) * g.dy - 0.5 * (double)g.ny * g.dy;
    const double off = 0.5 * (double)nt - 0.5;
    double x[kBpVx], s[kBpVx];
#pragma unroll
    for (int v = 0; v < kBpVx; ++v) {
        x[v] = ((double)(ix0 + kBpTx * v) + 0.5) * g.dx - 0.5 * (double)g.nx * g.dx;
        s[v] = 0.0;
    }
    const double* qs = q + (int64_t)iz * na * nt;
    for (int a = 0; a < na; ++a) {
        const double base = fma(y, sn[a], off);
        const double c = cs[a];
        const double* row = qs + (int64_t)a * nt;
#pragma unroll
        for (int v = 0; v < kBpVx; ++v) {
            const double u = fma(x[v], c, base);
            const int k = __double2int_rd(u);         // floor; saturates far outside the row
            const double w = u - (double)k;
            const double v0 = (k >= 0 && k < nt) ? __ldg(row + k) : 0.0;
            const double v1 = (k >= -1 && k < nt - 1) ? __ldg(row + k + 1) : 0.0;
            s[v] += fma(w, v1 - v0, v0);
        }
    }
    const double scale = kPi / (double)na;
#pragma unroll
    for (int v = 0; v < kBpVx; ++v) {
        const int ix = ix0 + kBpTx * v;
        if (ix < g.nx) img[((int64_t)iz * g.ny + iy) * g.nx + ix] = s[v] * scale;
    }
}

// ---------------------------------------------------------------- 4. median filter (+ 5. hull)

// Order-preserving map of a double onto unsigned 64-bit integers (negative values have
// their bits inverted, the others their sign bit set), so that the window's values can be
// compared on the integer pipes.  -0.0 sorts just below +0.0; both are the value 0.
__device__ __forceinline__ uint64_t mono_key(double v) {
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double mono_value(uint64_t k) {
    const uint64_t b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

__host__ __device__ constexpr int window_size(int r, bool ball) {
    int n = 0;
    for (int oz = -(ball ? r : 0); oz <= (ball ? r : 0); ++oz)
        for (int oy = -r; oy <= r; ++oy)
            for (int ox = -r; ox <= r; ++ox)
                if (ox * ox + oy * oy + oz * oz <= r * r + 1) ++n;
    return n;
}

// One thread per voxel.  The W window values become keys in registers (a neighbour
// outside the image becomes the largest key, above every value); with n in-image
// neighbours the result is the key whose rank range [#less, #less-or-equal) holds
// floor(n/2).
template <int R, bool BALL>
__global__ void __launch_bounds__(128) median_kernel(const double* __restrict__ in, double* __restrict__ out, int nx,
                                                     int ny, int nz, int use_hull, double tau) {
    constexpr int W = window_size(R, BALL);
    constexpr int RZ = BALL ? R : 0;
    const int64_t V = (int64_t)nx * ny * nz;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= V) return;
    const int ix = (int)(p % nx);
    const int64_t r_ = p / nx;
    const int iy = (int)(r_ % ny), iz = (int)(r_ / ny);
    uint64_t key[W];
    int n = 0;
    {
        int w = 0;
#pragma unroll
        for (int oz = -RZ; oz <= RZ; ++oz)
#pragma unroll
            for (int oy = -R; oy <= R; ++oy)
#pragma unroll
                for (int ox = -R; ox <= R; ++ox) {
                    if (ox * ox + oy * oy + oz * oz <= R * R + 1) {
                        const int jx = ix + ox, jy = iy + oy, jz = iz + oz;
                        const bool ok = jx >= 0 && jx < nx && jy >= 0 && jy < ny && jz >= 0 && jz < nz;
                        key[w] = ok ? mono_key(__ldg(in + ((int64_t)jz * ny + jy) * nx + jx)) : ~0ull;
                        n += ok ? 1 : 0;
                        ++w;
                    }
                }
    }
    const int m = n >> 1;
    uint64_t res = 0;
    // windows up to 64 values stay in registers (loops fully unrolled); the 147-voxel
    // ball of radius 3 is ranked from local memory
#pragma unroll(W <= 64 ? W : 1)
    for (int i = 0; i < W; ++i) {
        int lt = 0, le = 0;
#pragma unroll(W <= 64 ? W : 4)
        for (int j = 0; j < W; ++j) {
            lt += key[j] < key[i] ? 1 : 0;
            le += key[j] <= key[i] ? 1 : 0;
        }
        if (lt <= m && m < le) res = key[i];
    }
    double v = mono_value(res);
    if (use_hull && v <= tau) v = 0.0;
    out[p] = v;
}

__global__ void hull_kernel(double* __restrict__ img, int64_t V, double tau) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x)
        if (img[i] <= tau) img[i] = 0.0;
}

__global__ void copy_hull_kernel(const double* __restrict__ in, double* __restrict__ out, int64_t V, int use_hull,
                                 double tau) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = in[i];
        out[i] = (use_hull && v <= tau) ? 0.0 : v;
    }
}

int grid_for(int64_t n, int threads) {
    const int64_t g = (n + threads - 1) / threads;
    return (int)(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
}

}  // namespace
}  // namespace ntvs

using namespace ntvs;

namespace {

int median_launch(const double* in, double* out, int nx, int ny, int nz, int r, bool ball, int use_hull, double tau,
                  cudaStream_t s) {
    const int64_t V = (int64_t)nx * ny * nz;
    const int grid = (int)((V + 127) / 128);
#define NTVS_MEDIAN_CASE(RR, BB) median_kernel<RR, BB><<<grid, 128, 0, s>>>(in, out, nx, ny, nz, use_hull, tau)
    if (r == 1) {
        if (ball) NTVS_MEDIAN_CASE(1, true); else NTVS_MEDIAN_CASE(1, false);
    } else if (r == 2) {
        if (ball) NTVS_MEDIAN_CASE(2, true); else NTVS_MEDIAN_CASE(2, false);
    } else {
        if (ball) NTVS_MEDIAN_CASE(3, true); else NTVS_MEDIAN_CASE(3, false);
    }
#undef NTVS_MEDIAN_CASE
    return launch_status("median_kernel launch");
}

int filter_launch(const ntvs_fbp_geom* g, const double* sino, double* q, cudaStream_t s) {
    const size_t smem = sizeof(double) * ((size_t)g->n_t + (size_t)(g->n_t / 2 + 1));
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fbp_filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return fbp_fail(NTVS_ERR_CUDA, std::string("filter smem attribute: ") + cudaGetErrorString(e));
    }
    const int rows = g->nz * g->n_theta;
    fbp_filter_kernel<<<rows, 256, smem, s>>>(sino, q, g->n_t, g->dt);
    return launch_status("fbp_filter_kernel launch");
}

int backproject_launch(const ntvs_fbp_geom* g, const double* q, double* img, cudaStream_t s) {
    const size_t smem = sizeof(double) * 2 * (size_t)g->n_theta;
    if (smem > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(fbp_backproject_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return fbp_fail(NTVS_ERR_CUDA, std::string("back-projection smem attribute: ") + cudaGetErrorString(e));
    }
    dim3 grid((g->nx + kBpTx * kBpVx - 1) / (kBpTx * kBpVx), (g->ny + kBpTy - 1) / kBpTy, g->nz);
    fbp_backproject_kernel<<<grid, dim3(kBpTx, kBpTy), smem, s>>>(*g, q, img);
    return launch_status("fbp_backproject_kernel launch");
}

int bin_launch(const ntvs_fbp_geom* g, const float* paths, const double* wepl, int64_t M, double* sino,
               int32_t* count, cudaStream_t s) {
    const int64_t S = (int64_t)g->nz * g->n_theta * g->n_t;
    cudaError_t e = cudaMemsetAsync(sino, 0, sizeof(double) * (size_t)S, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(int32_t) * (size_t)S, s);
    if (e != cudaSuccess) return fbp_fail(NTVS_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    if (M > 0) {
        const int64_t warps = (M + 31) / 32;
        const int64_t want = (warps + 7) / 8;   // 8 warps per 256-thread CTA
        const int grid = (int)(want < 1 ? 1 : (want > 152 * 16 ? 152 * 16 : want));
        fbp_bin_kernel<<<grid, 256, 0, s>>>(*g, paths, wepl, M, sino, count);
        int rc = launch_status("fbp_bin_kernel launch");
        if (rc != NTVS_OK) return rc;
    }
    fbp_mean_kernel<<<grid_for(S, 256), 256, 0, s>>>(sino, count, S);
    return launch_status("fbp_mean_kernel launch");
}

int64_t align256(int64_t b) { return (b + 255) / 256 * 256; }

}  // namespace

extern "C" int ntvs_fbp_bin(const ntvs_fbp_geom* g, const float* paths, const double* wepl, int64_t M, double* sino,
                            int32_t* count, void* cuda_stream) {
    int rc = check_geom(g, "ntvs_fbp_bin");
    if (rc != NTVS_OK) return rc;
    if (M < 0) return fbp_fail(NTVS_ERR_ARG, "ntvs_fbp_bin: M < 0");
    if (!sino || !count || (M > 0 && (!paths || !wepl))) return fbp_fail(NTVS_ERR_ARG, "ntvs_fbp_bin: null pointer");
    return bin_launch(g, paths, wepl, M, sino, count, (cudaStream_t)cuda_stream);
}

extern "C" int ntvs_fbp_filter(const ntvs_fbp_geom* g, const double* sino, double* q, void* cuda_stream) {
    int rc = check_geom(g, "ntvs_fbp_filter");
    if (rc != NTVS_OK) return rc;
    if (!sino || !q) return fbp_fail(NTVS_ERR_ARG, "ntvs_fbp_filter: null pointer");
    const int64_t S = (int64_t)g->nz * g->n_theta * g->n_t;
    if (((uintptr_t)sino < (uintptr_t)(q + S)) && ((uintptr_t)q < (uintptr_t)(sino + S)))
        return fbp_fail(NTVS_ERR_ARG, "ntvs_fbp_filter: q must not overlap sino");
    return filter_launch(g, sino, q, (cudaStream_t)cuda_stream);
}

extern "C" int ntvs_fbp_backproject(const ntvs_fbp_geom* g, const double* q, double* img, void* cuda_stream) {
    int rc = check_geom(g, "ntvs_fbp_backproject");
    if (rc != NTVS_OK) return rc;
    if (!q || !img) return fbp_fail(NTVS_ERR_ARG, "ntvs_fbp_backproject: null pointer");
    return backproject_launch(g, q, img, (cudaStream_t)cuda_stream);
}

extern "C" int ntvs_median_filter(const double* in, double* out, int nx, int ny, int nz, int radius, int ball,
                                  int use_hull, double tau, void* cuda_stream) {
    if (!in || !out) return fbp_fail(NTVS_ERR_ARG, "ntvs_median_filter: null pointer");
    if (nx < 1 || ny < 1 || nz < 1) return fbp_fail(NTVS_ERR_ARG, "ntvs_median_filter: sizes must be >= 1");
    if ((int64_t)nx * ny * nz > INT32_MAX) return fbp_fail(NTVS_ERR_ARG, "ntvs_median_filter: more than 2^31 - 1 voxels");
    if (((uintptr_t)in < (uintptr_t)(out + (int64_t)nx * ny * nz)) && ((uintptr_t)out < (uintptr_t)(in + (int64_t)nx * ny * nz)))
        return fbp_fail(NTVS_ERR_ARG, "ntvs_median_filter: out must not overlap in");
    if (radius < 0 || radius > kMaxMedianRadius) return fbp_fail(NTVS_ERR_ARG, "ntvs_median_filter: radius must be 0..3");
    if (use_hull && std::isnan(tau)) return fbp_fail(NTVS_ERR_ARG, "ntvs_median_filter: tau is NaN");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int64_t V = (int64_t)nx * ny * nz;
    if (radius == 0) {
        copy_hull_kernel<<<grid_for(V, 256), 256, 0, s>>>(in, out, V, use_hull, tau);
        return launch_status("copy_hull_kernel launch");
    }
    return median_launch(in, out, nx, ny, nz, radius, ball != 0, use_hull, tau, s);
}

extern "C" int ntvs_hull(double* img, int64_t V, double tau, void* cuda_stream) {
    if (!img) return fbp_fail(NTVS_ERR_ARG, "ntvs_hull: null image");
    if (V < 1) return fbp_fail(NTVS_ERR_ARG, "ntvs_hull: V must be >= 1");
    if (std::isnan(tau)) return fbp_fail(NTVS_ERR_ARG, "ntvs_hull: tau is NaN");
    hull_kernel<<<grid_for(V, 256), 256, 0, (cudaStream_t)cuda_stream>>>(img, V, tau);
    return launch_status("hull_kernel launch");
}

extern "C" int64_t ntvs_fbp_workspace_bytes(const ntvs_fbp_geom* g) {
    int rc = check_geom(g, "ntvs_fbp_workspace_bytes");
    if (rc != NTVS_OK) return rc;
    const int64_t S = (int64_t)g->nz * g->n_theta * g->n_t;
    const int64_t V = (int64_t)g->nx * g->ny * g->nz;
    return align256(8 * S) + align256(4 * S) + align256(8 * S) + align256(8 * V);
}

extern "C" int ntvs_initial_iterate(const ntvs_fbp_geom* g, const float* paths, const double* wepl, int64_t M,
                                    int median_radius, int median_ball, int use_hull, double tau, void* workspace,
                                    int64_t workspace_bytes, double* out, void* cuda_stream) {
    int rc = check_geom(g, "ntvs_initial_iterate");
    if (rc != NTVS_OK) return rc;
    if (M < 0) return fbp_fail(NTVS_ERR_ARG, "ntvs_initial_iterate: M < 0");
    if (!out || !workspace || (M > 0 && (!paths || !wepl)))
        return fbp_fail(NTVS_ERR_ARG, "ntvs_initial_iterate: null pointer");
    if (median_radius < 0 || median_radius > kMaxMedianRadius)
        return fbp_fail(NTVS_ERR_ARG, "ntvs_initial_iterate: median radius must be 0..3");
    if (use_hull && std::isnan(tau)) return fbp_fail(NTVS_ERR_ARG, "ntvs_initial_iterate: tau is NaN");
    const int64_t need = ntvs_fbp_workspace_bytes(g);
    if (workspace_bytes < need)
        return fbp_fail(NTVS_ERR_ARG, "ntvs_initial_iterate: workspace of " + std::to_string(workspace_bytes) +
                                          " bytes, " + std::to_string(need) + " needed");
    if (((uintptr_t)workspace & 255) != 0)
        return fbp_fail(NTVS_ERR_ARG, "ntvs_initial_iterate: workspace must be 256-byte aligned");
    const int64_t S = (int64_t)g->nz * g->n_theta * g->n_t;
    char* w = (char*)workspace;
    double* sino = (double*)w;
    w += align256(8 * S);
    int32_t* cnt = (int32_t*)w;
    w += align256(4 * S);
    double* q = (double*)w;
    w += align256(8 * S);
    double* img = (double*)w;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if ((rc = bin_launch(g, paths, wepl, M, sino, cnt, s)) != NTVS_OK) return rc;
    if ((rc = filter_launch(g, sino, q, s)) != NTVS_OK) return rc;
    if ((rc = backproject_launch(g, q, img, s)) != NTVS_OK) return rc;
    return ntvs_median_filter(img, out, g->nx, g->ny, g->nz, median_radius, median_ball, use_hull, tau, cuda_stream);
}
