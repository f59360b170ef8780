// On-the-fly DROP rows (P_T of arXiv 1803.01112 Appendix C with the system never stored):
// row i is the intersection-length vector of history i's path with the voxel grid
// (Sec. I: a row holds the lengths of one tracked proton's path through the voxels).
// A path is a chord P_in -> P_out plus cubic-Hermite offsets A h10(s) + B h11(s) along the
// in-plane normal and along z, split into n_seg straight segments; every sweep traces it
// again, in FP32: each segment is cut at every voxel plane it crosses (three per-axis
// crossing sequences merged in order) and each piece is credited to the voxel holding its
// midpoint.  Pieces shorter than min_len are dropped.  Only 44 bytes per history live in
// HBM (10 path floats + b); the work is ALU (tracing) and L2 atomics (scatter).
//
// Load time: one thread per row traces the whole path in order, merges consecutive pieces
// of one voxel (segment joins), and accumulates ||a_i||^2 (FP64) and the per-block hit
// counts s_j^t.
#include "common.cuh"

namespace ntvs {

namespace {

struct Grid3 {
    float ox, oy, oz, hx, hy, hz;
    float ihx, ihy, ihz;   // 1 / voxel size
    int nx, ny, nz;
    int ltx, lty, ntx;     // internal voxel order: tiles of 2^ltx x 2^lty, ntx tiles per row
    int slice_p;           // voxels per padded slice
};

// internal index (see VoxMap) of voxel (ix, iy, iz)
__device__ __forceinline__ int grid_index(const Grid3& g, int ix, int iy, int iz) {
    const int tile = (iy >> g.lty) * g.ntx + (ix >> g.ltx);
    return iz * g.slice_p + (tile << (g.ltx + g.lty)) + ((iy & ((1 << g.lty) - 1)) << g.ltx) +
           (ix & ((1 << g.ltx) - 1));
}

__device__ __forceinline__ float h10f(float s) { return s * s * s - 2.f * s * s + s; }
__device__ __forceinline__ float h11f(float s) { return s * s * s - s * s; }

// point of the path at parameter s
__device__ __forceinline__ void path_point(const float* pr, float nxv, float nyv, float s, float out[3]) {
    const float ol = pr[6] * h10f(s) + pr[7] * h11f(s), oz = pr[8] * h10f(s) + pr[9] * h11f(s);
    out[0] = pr[0] + s * (pr[3] - pr[0]) + ol * nxv;
    out[1] = pr[1] + s * (pr[4] - pr[1]) + ol * nyv;
    out[2] = pr[2] + s * (pr[5] - pr[2]) + oz;
}

// in-plane unit normal (-u_y, u_x) of the chord
__device__ __forceinline__ void chord_normal(const float* pr, float& nxv, float& nyv) {
    const float ux = pr[3] - pr[0], uy = pr[4] - pr[1];
    const float l = sqrtf(ux * ux + uy * uy);
    if (l > 0.f) { nxv = -uy / l; nyv = ux / l; }
    else { nxv = 1.f; nyv = 0.f; }
}

// Calls f(voxel, length) for every piece of segment P -> Q inside the grid.  The segment is
// clipped to the grid, the crossings of the three plane families are merged in order of
// their parameter t (each from its plane index: t = (o + k h - P) / D, computed with the
// reciprocal of D), and a piece between consecutive crossings is credited to the voxel
// between those planes: the voxel before the first crossing of each axis follows from
// that crossing's plane index, and the index is stepped by one along the axis of every
// crossing, so the voxel of a piece is always the one bounded by the planes around it
// (the voxel holding the piece's midpoint).
template <typename F>
__device__ __forceinline__ void trace_segment(const Grid3& g, const float P[3], const float Q[3], F&& f) {
    const float D[3] = {Q[0] - P[0], Q[1] - P[1], Q[2] - P[2]};
    const float L = sqrtf(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
    if (!(L > 0.f)) return;
    const float o[3] = {g.ox, g.oy, g.oz}, h[3] = {g.hx, g.hy, g.hz}, ih[3] = {g.ihx, g.ihy, g.ihz};
    const int n[3] = {g.nx, g.ny, g.nz};
    float inv[3];
    float lo = 0.f, hi = 1.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float e0 = o[a], e1 = o[a] + n[a] * h[a];
        inv[a] = D[a] != 0.f ? 1.f / D[a] : 0.f;
        if (D[a] == 0.f) {
            if (P[a] < e0 || P[a] > e1) return;
        } else {
            float s0 = (e0 - P[a]) * inv[a], s1 = (e1 - P[a]) * inv[a];
            if (s0 > s1) { const float t = s0; s0 = s1; s1 = t; }
            lo = fmaxf(lo, s0);
            hi = fminf(hi, s1);
        }
    }
    if (!(hi > lo)) return;
    // next crossing of each axis: plane index k, parameter tn
    int k[3], step[3];
    float tn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (D[a] == 0.f) { tn[a] = 2.f; step[a] = 0; k[a] = 0; continue; }
        const float u = (P[a] + lo * D[a] - o[a]) * ih[a];
        step[a] = D[a] > 0.f ? 1 : -1;
        k[a] = D[a] > 0.f ? (int)floorf(u) + 1 : (int)ceilf(u) - 1;
        tn[a] = (o[a] + k[a] * h[a] - P[a]) * inv[a];
        if (tn[a] <= lo) {   // the start lies on plane k: move to the next one
            k[a] += step[a];
            tn[a] = (o[a] + k[a] * h[a] - P[a]) * inv[a];
        }
    }
    int idx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int i = step[a] > 0 ? k[a] - 1 : step[a] < 0 ? k[a] : (int)floorf((P[a] - o[a]) * ih[a]);
        idx[a] = min(max(i, 0), n[a] - 1);
    }
    float t0 = lo;
    for (int guard = 0; guard < 4 * (g.nx + g.ny + g.nz) + 8; ++guard) {
        int w = 0;
        float t1 = tn[0];
        if (tn[1] < t1) { t1 = tn[1]; w = 1; }
        if (tn[2] < t1) { t1 = tn[2]; w = 2; }
        const bool last = !(t1 < hi);
        if (last) t1 = hi;
        if (t1 - t0 > 1e-7f) f(grid_index(g, idx[0], idx[1], idx[2]), (t1 - t0) * L);
        if (last) break;
#pragma unroll
        for (int a = 0; a < 3; ++a) {   // constant indices keep the arrays in registers
            if (a == w) {
                idx[a] = min(max(idx[a] + step[a], 0), n[a] - 1);
                k[a] += step[a];
                tn[a] = (o[a] + k[a] * h[a] - P[a]) * inv[a];
            }
        }
        t0 = t1;
    }
}

// ---------------------------------------------------------------- load-time row statistics
__global__ void otf_prep_kernel(const float* __restrict__ paths, int64_t r0, int64_t r1, Grid3 g, int n_seg,
                                float min_len, float* __restrict__ inv_norm2, int32_t* __restrict__ cnt) {
    for (int64_t i = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < r1;
         i += (int64_t)gridDim.x * blockDim.x) {
        float pr[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) pr[q] = paths[i * 10 + q];
        float nxv, nyv;
        chord_normal(pr, nxv, nyv);
        double n2 = 0.0;
        int cur = -1;
        float acc = 0.f;
        auto close = [&]() {
            if (cur >= 0 && acc >= min_len) {
                n2 += (double)acc * (double)acc;
                atomicAdd(cnt + cur, 1);
            }
        };
        float A[3], B[3];
        path_point(pr, nxv, nyv, 0.f, A);
        for (int sg = 0; sg < n_seg; ++sg) {
            path_point(pr, nxv, nyv, (float)(sg + 1) / (float)n_seg, B);
            trace_segment(g, A, B, [&](int v, float l) {
                if (v == cur) { acc += l; return; }
                close();
                cur = v;
                acc = l;
            });
            A[0] = B[0]; A[1] = B[1]; A[2] = B[2];
        }
        close();
        inv_norm2[i] = n2 > 0.0 ? (float)(1.0 / n2) : 0.f;
    }
}

// ---------------------------------------------------------------- stored rows from paths
// Row i as the load-time statistics see it: the path traced in order by one thread,
// consecutive pieces of one voxel merged, merged pieces shorter than min_len dropped.
// Pass 1 counts the entries of every row; pass 2 writes them (voxel index in the order of
// g, length) from row_ptr[i].  Both passes run the same code, so they agree entry by entry.
template <bool FILL>
__global__ void otf_rows_kernel(const float* __restrict__ paths, int64_t M, Grid3 g, int n_seg, float min_len,
                                int32_t* __restrict__ nnz_row, const int64_t* __restrict__ row_ptr,
                                int32_t* __restrict__ col, float* __restrict__ val) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        float pr[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) pr[q] = paths[i * 10 + q];
        float nxv, nyv;
        chord_normal(pr, nxv, nyv);
        int64_t pos = FILL ? row_ptr[i] : 0;
        int n = 0;
        int cur = -1;
        float acc = 0.f;
        auto close = [&]() {
            if (cur >= 0 && acc >= min_len) {
                if (FILL) {
                    col[pos] = cur;
                    val[pos] = acc;
                    ++pos;
                }
                ++n;
            }
        };
        float A[3], B[3];
        path_point(pr, nxv, nyv, 0.f, A);
        for (int sg = 0; sg < n_seg; ++sg) {
            path_point(pr, nxv, nyv, (float)(sg + 1) / (float)n_seg, B);
            trace_segment(g, A, B, [&](int v, float l) {
                if (v == cur) { acc += l; return; }
                close();
                cur = v;
                acc = l;
            });
            A[0] = B[0]; A[1] = B[1]; A[2] = B[2];
        }
        close();
        if (!FILL) nnz_row[i] = n;
    }
}

// ---------------------------------------------------------------- the DROP block
// A group of 16 lanes per row (2 rows per warp); lane s traces segments s, s + 16, ...
// The dot-product pass keeps the first kOtfCache accepted pieces of each lane (voxel,
// length) in shared memory, and the scatter pass replays them; a lane with more pieces
// traces its segments again and scatters only the pieces past the cached ones.
// Four CTAs per SM: 64 registers per thread (no spills) and 4 x 48 KB of piece caches.
constexpr int kOtfThreads = 256;
constexpr int kOtfCache = 24;

__global__ void __launch_bounds__(kOtfThreads, 4) otf_drop_kernel(const float* __restrict__ paths,
                                                                const float* __restrict__ b,
                                                                const float* __restrict__ inv_norm2, int64_t r0,
                                                                int64_t r1, Grid3 g, int n_seg, float min_len,
                                                                const float* __restrict__ x, float* __restrict__ delta,
                                                                float lambda, double* resid_ss) {
    constexpr int LPR = 16;
    extern __shared__ __align__(16) unsigned char otf_smem[];
    int32_t* cv = reinterpret_cast<int32_t*>(otf_smem);                 // [kOtfCache][kOtfThreads]
    float* cl = reinterpret_cast<float*>(cv + kOtfCache * kOtfThreads);  // [kOtfCache][kOtfThreads]
    const int tid = threadIdx.x;
    const int lane = tid & 31, sub = lane % LPR;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + tid) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double ss = 0.0;
    for (int64_t base = r0 + warp * 2; base < r1; base += nwarps * 2) {
        const int64_t i = base + lane / LPR;
        const bool valid = i < r1;
        float pr[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) pr[q] = valid ? __ldg(paths + i * 10 + q) : 0.f;
        float nxv, nyv;
        chord_normal(pr, nxv, nyv);
        float acc = 0.f;
        int np = 0;   // accepted pieces of this lane
        if (valid) {
            for (int sg = sub; sg < n_seg; sg += LPR) {
                float A[3], B[3];
                path_point(pr, nxv, nyv, (float)sg / (float)n_seg, A);
                path_point(pr, nxv, nyv, (float)(sg + 1) / (float)n_seg, B);
                trace_segment(g, A, B, [&](int v, float l) {
                    if (l >= min_len) {
                        if (np < kOtfCache) {
                            cv[np * kOtfThreads + tid] = v;
                            cl[np * kOtfThreads + tid] = l;
                        } else {
                            acc += l * __ldg(x + v);
                        }
                        ++np;
                    }
                });
            }
            // the cached pieces' gathers are independent: issued back to back, four in flight
            const int nc = np < kOtfCache ? np : kOtfCache;
            int q = 0;
            for (; q + 4 <= nc; q += 4) {
                float xv[4], lv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    xv[u] = __ldg(x + cv[(q + u) * kOtfThreads + tid]);
                    lv[u] = cl[(q + u) * kOtfThreads + tid];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) acc += lv[u] * xv[u];
            }
            for (; q < nc; ++q) acc += cl[q * kOtfThreads + tid] * __ldg(x + cv[q * kOtfThreads + tid]);
        }
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (!valid) continue;   // both halves of the warp are past their shuffles
        const float res = __ldg(b + i) - acc;
        const float r = lambda * res * __ldg(inv_norm2 + i);
        if (sub == 0) ss += (double)res * (double)res;
        const int nc = np < kOtfCache ? np : kOtfCache;
        for (int q = 0; q < nc; ++q) atomicAdd(delta + cv[q * kOtfThreads + tid], r * cl[q * kOtfThreads + tid]);
        if (np > kOtfCache) {
            int seen = 0;
            for (int sg = sub; sg < n_seg; sg += LPR) {
                float A[3], B[3];
                path_point(pr, nxv, nyv, (float)sg / (float)n_seg, A);
                path_point(pr, nxv, nyv, (float)(sg + 1) / (float)n_seg, B);
                trace_segment(g, A, B, [&](int v, float l) {
                    if (l >= min_len) {
                        if (seen >= kOtfCache) atomicAdd(delta + v, r * l);
                        ++seen;
                    }
                });
            }
        }
    }
    __shared__ double sh[32];
    const double tot = block_sum(ss, sh);
    if (threadIdx.x == 0 && tot != 0.0) atomicAdd(resid_ss, tot);
}

// ---------------------------------------------------------------- forward projection
// out_i = sum of l * x_v over the accepted pieces (voxel v, length l >= min_len) of history
// i's path, the rows the DROP sweeps use; 16 lanes per row, each tracing every 16th segment.
__global__ void __launch_bounds__(256) otf_project_kernel(const float* __restrict__ paths, int64_t M, Grid3 g,
                                                           int n_seg, float min_len, const float* __restrict__ x,
                                                           float* __restrict__ out) {
    constexpr int LPR = 16;
    const int lane = threadIdx.x & 31, sub = lane % LPR;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * 2; base < M; base += nwarps * 2) {
        const int64_t i = base + lane / LPR;
        const bool valid = i < M;
        float acc = 0.f;
        if (valid) {
            float pr[10];
#pragma unroll
            for (int q = 0; q < 10; ++q) pr[q] = __ldg(paths + i * 10 + q);
            float nxv, nyv;
            chord_normal(pr, nxv, nyv);
            for (int sg = sub; sg < n_seg; sg += LPR) {
                float A[3], B[3];
                path_point(pr, nxv, nyv, (float)sg / (float)n_seg, A);
                path_point(pr, nxv, nyv, (float)(sg + 1) / (float)n_seg, B);
                trace_segment(g, A, B, [&](int v, float l) {
                    if (l >= min_len) acc += l * __ldg(x + v);
                });
            }
        }
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (valid && sub == 0) out[i] = acc;
    }
}

// History data (P_in, P_out, d_in, d_out) -> path record (P_in, P_out, A_lat, B_lat, A_z, B_z):
// end tangents m = L d / |d| (chord direction for a zero d), deviations m - c projected on
// the chord's in-plane normal and on z.  flags |= 32 on a non-finite history value.
__global__ void hist_to_paths_kernel(const float* __restrict__ hist, int64_t M, float* __restrict__ rec, int* flags) {
    int f = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        float h[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            h[q] = hist[i * 12 + q];
            if (!isfinite(h[q])) f |= 32;
        }
        const float c[3] = {h[3] - h[0], h[4] - h[1], h[5] - h[2]};
        const float L = sqrtf(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        float pr[10] = {h[0], h[1], h[2], h[3], h[4], h[5], 0.f, 0.f, 0.f, 0.f};
        float nxv, nyv;
        chord_normal(pr, nxv, nyv);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float* d = h + 6 + 3 * e;
            const float dl = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            float m[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) m[a] = dl > 0.f ? L * (d[a] / dl) : c[a];
            const float dev[3] = {m[0] - c[0], m[1] - c[1], m[2] - c[2]};
            pr[6 + e] = dev[0] * nxv + dev[1] * nyv;   // A_lat, B_lat
            pr[8 + e] = dev[2];                         // A_z, B_z
        }
#pragma unroll
        for (int q = 0; q < 10; ++q) rec[i * 10 + q] = pr[q];
    }
    if (f) atomicOr(flags, f);
}

// paths finite, n_seg sane: flags |= 32 on a non-finite path value, 16 on a non-finite b
__global__ void otf_validate_kernel(const float* __restrict__ paths, const float* __restrict__ b, int64_t M,
                                    int* flags) {
    int f = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        for (int q = 0; q < 10; ++q)
            if (!isfinite(paths[i * 10 + q])) f |= 32;
        if (!isfinite(b[i])) f |= 16;
    }
    if (f) atomicOr(flags, f);
}

}  // namespace

static Grid3 make_grid(const OtfArgs& a) {
    Grid3 g;
    g.nx = a.nx; g.ny = a.ny; g.nz = a.nz;
    g.hx = (float)a.dx; g.hy = (float)a.dy; g.hz = (float)a.dz;
    g.ihx = 1.f / g.hx; g.ihy = 1.f / g.hy; g.ihz = 1.f / g.hz;
    g.ltx = a.vm.ltx; g.lty = a.vm.lty;
    g.ntx = a.vm.nxp >> a.vm.ltx;
    g.slice_p = (int)a.vm.slice_p;
    g.ox = (float)(-0.5 * a.nx * a.dx); g.oy = (float)(-0.5 * a.ny * a.dy); g.oz = 0.f;
    return g;
}

cudaError_t k_hist_to_paths(const float* hist, int64_t M, float* rec, int* flags, int grid, cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    hist_to_paths_kernel<<<grid, 256, 0, s>>>(hist, M, rec, flags);
    return cudaGetLastError();
}

cudaError_t k_otf_validate(const OtfArgs& a, int* flags, cudaStream_t s) {
    if (a.M <= 0) return cudaSuccess;
    otf_validate_kernel<<<a.grid, 256, 0, s>>>(a.paths, a.b, a.M, flags);
    return cudaGetLastError();
}

cudaError_t k_otf_prep(const OtfArgs& a, int64_t r0, int64_t r1, float* inv_norm2, int32_t* cnt, cudaStream_t s) {
    if (r1 <= r0) return cudaSuccess;
    otf_prep_kernel<<<a.grid, 128, 0, s>>>(a.paths, r0, r1, make_grid(a), a.n_seg, a.min_len, inv_norm2, cnt);
    return cudaGetLastError();
}

cudaError_t k_otf_drop(const OtfArgs& a, int64_t r0, int64_t r1, const float* inv_norm2, const float* x, float* delta,
                       double lambda, double* resid_ss, cudaStream_t s) {
    if (r1 <= r0) return cudaSuccess;
    const size_t smem = (size_t)kOtfCache * kOtfThreads * (sizeof(int32_t) + sizeof(float));
    cudaError_t e = cudaFuncSetAttribute(otf_drop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    otf_drop_kernel<<<a.grid, kOtfThreads, smem, s>>>(a.paths, a.b, inv_norm2, r0, r1, make_grid(a), a.n_seg,
                                                      a.min_len, x, delta, (float)lambda, resid_ss);
    return cudaGetLastError();
}

cudaError_t k_otf_count_rows(const OtfArgs& a, int32_t* nnz_row, cudaStream_t s) {
    if (a.M <= 0) return cudaSuccess;
    otf_rows_kernel<false><<<a.grid, 128, 0, s>>>(a.paths, a.M, make_grid(a), a.n_seg, a.min_len, nnz_row, nullptr,
                                                  nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t k_otf_fill_rows(const OtfArgs& a, const int64_t* row_ptr, int32_t* col, float* val, cudaStream_t s) {
    if (a.M <= 0) return cudaSuccess;
    otf_rows_kernel<true><<<a.grid, 128, 0, s>>>(a.paths, a.M, make_grid(a), a.n_seg, a.min_len, nullptr, row_ptr,
                                                 col, val);
    return cudaGetLastError();
}

cudaError_t k_otf_project(const OtfArgs& a, const float* x, float* out, cudaStream_t s) {
    if (a.M <= 0) return cudaSuccess;
    otf_project_kernel<<<a.grid, 256, 0, s>>>(a.paths, a.M, make_grid(a), a.n_seg, a.min_len, x, out);
    return cudaGetLastError();
}

}  // namespace ntvs
