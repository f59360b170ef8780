// Batched NTVS: many independent reconstructions (each with its own grid, system, block
// partition and (lambda, N, alpha, beta0, eps, seed)) advanced together, one kernel
// launch per step type per cycle instead of one per reconstruction (arXiv 1803.01112,
// Appendix C, applied to every reconstruction of the batch; the variant without the TV
// check, whose control flow is the same for every member).
//
// Work lists pack the members: a TV item is a run of <= kTvItem voxels of one member, a
// DROP item a run of <= kDropItem rows of one member's block b.  One cycle is
//     for n < N_max:  grad (items of members with n < N_r) ; apply
//     for b < B_max:  drop block b (items of members with b < B_r) ; apply block b
//     phi of every member
// Per-member reductions (||g||^2, phi) are FP64 partials per item, summed in a fixed order
// by the last item of the member to finish (per-member ticket): deterministic.
// The cycle's launches are captured once in a CUDA graph; what changes from cycle to cycle
// (the step sizes beta_{k,n} of every member) is a device table refreshed by one copy.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "voxel_coords.cuh"
#include "ntvs.h"
#include "step_rule.h"

namespace ntvs {
namespace {

constexpr int kTvItem = 2048;     // voxels per TV item (256 threads x 8)
constexpr int kDropItem = 256;    // rows per DROP item (enough CTAs to fill every SM)

struct MemberDev {
    const int64_t* row_ptr;
    const int32_t* col;
    const float* val;
    const float* b;
    const float* inv_norm2;
    const float* inv_s;   // [B][vint], internal voxel order
    double* x;
    float* x32;           // fl32(x), internal voxel order (the DROP gathers)
    float* xh;            // fl32(x) and fl32(x - xh), canonical order: the TV stencil
    float* xl;            //   differences are formed from both
    float* delta;
    float* g;
    double* resid;        // [B]
    double* tv_hist;      // [cap]
    int nx, ny, nz, B, N;
    int64_t V;
    VoxMap vm;            // internal order of x32, delta, inv_s and the stored columns
    float lambda, eps;
    int item0, nitems;    // this member's TV items
};

struct Item {
    int member;
    int pad;
    int64_t i0, i1;   // voxel or row range
};

__device__ __forceinline__ double block_sum_d(double v, double* sh) { return block_sum(v, sh); }

// per-member deterministic reduction of one value: partials[item], ticket per member
__device__ __forceinline__ void member_reduce(double v, int item, const MemberDev& m, int r, double* partials,
                                              unsigned* tickets, double* out) {
    __shared__ double sh[32];
    __shared__ bool last;
    const double tot = block_sum_d(v, sh);
    if (threadIdx.x == 0) {
        partials[item] = tot;
        __threadfence();
        const unsigned t = atomicAdd(tickets + r, 1u);
        last = (t == (unsigned)m.nitems - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = 0.0;
    for (int q = threadIdx.x; q < m.nitems; q += blockDim.x) a += __ldcg(partials + m.item0 + q);
    a = block_sum_d(a, sh);
    if (threadIdx.x == 0) {
        *out = a;
        tickets[r] = 0u;
    }
}

// grad phi_eps of member r over the item's voxels; ||g||^2 into gnorm2[r]
__global__ void __launch_bounds__(256) tvb_grad_kernel(const MemberDev* __restrict__ mem, const Item* __restrict__ items,
                                                       int n_step, double* partials, unsigned* tickets,
                                                       double* gnorm2) {
    const Item it = items[blockIdx.x];
    const MemberDev m = mem[it.member];
    if (n_step >= m.N) return;   // uniform over the CTA: no reduction for this member
    const int nx = m.nx, ny = m.ny, nz = m.nz;
    const int64_t sxy = (int64_t)nx * ny;
    const float* xh = m.xh;
    const float* xl = m.xl;
    const float eps = m.eps;
    auto dif = [&](int64_t a, int64_t b) -> float {
        return (__ldg(xh + a) - __ldg(xh + b)) + (__ldg(xl + a) - __ldg(xl + b));
    };
    double acc = 0.0;
    for (int64_t p = it.i0 + threadIdx.x; p < it.i1; p += blockDim.x) {
        int ix, iy, iz;
        voxel_coords(p, nx, ny, ix, iy, iz);
        const bool hx = ix + 1 < nx, hy = iy + 1 < ny, hz = iz + 1 < nz;
        const float dx = hx ? dif(p + 1, p) : 0.f, dy = hy ? dif(p + nx, p) : 0.f, dz = hz ? dif(p + sxy, p) : 0.f;
        const float D = sqrtf(eps + (dx * dx + dy * dy + dz * dz));
        float gq = (D > 0.f) ? -(dx + dy + dz) / D : 0.f;
        if (ix > 0) {
            const int64_t q = p - 1;
            const float a = dif(p, q), bb = hy ? dif(q + nx, q) : 0.f, c = hz ? dif(q + sxy, q) : 0.f;
            const float Dm = sqrtf(eps + (a * a + bb * bb + c * c));
            if (Dm > 0.f) gq += a / Dm;
        }
        if (iy > 0) {
            const int64_t q = p - nx;
            const float a = dif(p, q), bb = hx ? dif(q + 1, q) : 0.f, c = hz ? dif(q + sxy, q) : 0.f;
            const float Dm = sqrtf(eps + (a * a + bb * bb + c * c));
            if (Dm > 0.f) gq += a / Dm;
        }
        if (iz > 0) {
            const int64_t q = p - sxy;
            const float a = dif(p, q), bb = hx ? dif(q + 1, q) : 0.f, c = hy ? dif(q + nx, q) : 0.f;
            const float Dm = sqrtf(eps + (a * a + bb * bb + c * c));
            if (Dm > 0.f) gq += a / Dm;
        }
        m.g[p] = gq;
        acc += (double)gq * (double)gq;
    }
    member_reduce(acc, blockIdx.x, m, it.member, partials, tickets, gnorm2 + it.member);
}

// x <- x - beta_r / ||g_r|| * g on the items' voxels (members with n_step < N_r)
__global__ void __launch_bounds__(256) tvb_apply_kernel(const MemberDev* __restrict__ mem,
                                                        const Item* __restrict__ items, int n_step,
                                                        const double* __restrict__ beta, int R,
                                                        const double* __restrict__ gnorm2) {
    const Item it = items[blockIdx.x];
    const MemberDev m = mem[it.member];
    if (n_step >= m.N) return;
    const double sc = step_scale(beta[(int64_t)n_step * R + it.member], gnorm2 + it.member);
    for (int64_t p = it.i0 + threadIdx.x; p < it.i1; p += blockDim.x) {
        const double z = perturbed(m.x[p], sc, (double)m.g[p]);
        m.x[p] = z;
        const float h = (float)z;
        m.x32[vox_internal(m.vm, p)] = h;
        m.xh[p] = h;
        m.xl[p] = (float)(z - (double)h);
    }
}

// DROP block b of every member with b < B_r: a group of LPR lanes per row; the first
// CH * LPR entries of a row stay in registers between the dot product and the scatter
// (the matrix is read once), longer rows re-read their tail; global reductions.
template <int LPR, int CH>
__global__ void __launch_bounds__(256) dropb_block_kernel(const MemberDev* __restrict__ mem,
                                                          const Item* __restrict__ items) {
    const Item it = items[blockIdx.x];
    const MemberDev m = mem[it.member];
    constexpr int G = 32 / LPR;
    const int lane = threadIdx.x & 31, sub = lane % LPR;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double ss = 0.0;
    for (int64_t base = it.i0 + (int64_t)warp * G; base < it.i1; base += (int64_t)nw * G) {
        const int64_t i = base + lane / LPR;
        const bool valid = i < it.i1;
        int64_t p0 = 0, p1 = 0;
        if (valid) { p0 = __ldg(m.row_ptr + i); p1 = __ldg(m.row_ptr + i + 1); }
        int32_t c[CH];
        float a[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const int64_t q = p0 + (int64_t)u * LPR + sub;
            if (q < p1) { c[u] = __ldcs(m.col + q); a[u] = __ldcs(m.val + q); }
            else { c[u] = -1; a[u] = 0.f; }
        }
        float acc = 0.f;
#pragma unroll
        for (int u = 0; u < CH; ++u)
            if (c[u] >= 0) acc += a[u] * __ldg(m.x32 + c[u]);
        const int64_t tail0 = p0 + (int64_t)CH * LPR;
        for (int64_t p = tail0 + sub; p < p1; p += LPR) acc += m.val[p] * __ldg(m.x32 + m.col[p]);
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        float r = 0.f;
        if (valid) {
            const float res = __ldg(m.b + i) - acc;
            r = m.lambda * res * __ldg(m.inv_norm2 + i);
            if (sub == 0) ss += (double)res * (double)res;
        }
#pragma unroll
        for (int u = 0; u < CH; ++u)
            if (c[u] >= 0) atomicAdd(m.delta + c[u], r * a[u]);
        for (int64_t p = tail0 + sub; p < p1; p += LPR) atomicAdd(m.delta + m.col[p], r * m.val[p]);
    }
    __shared__ double sh[32];
    const double tot = block_sum(ss, sh);
    if (threadIdx.x == 0 && tot != 0.0) atomicAdd(m.resid + it.pad, tot);   // pad carries the block index
}

// x += delta / s for block b of members with b < B_r (TV items cover every voxel)
__global__ void __launch_bounds__(256) dropb_apply_kernel(const MemberDev* __restrict__ mem,
                                                          const Item* __restrict__ items, int b) {
    const Item it = items[blockIdx.x];
    const MemberDev m = mem[it.member];
    if (b >= m.B) return;
    const float* inv_s = m.inv_s + (int64_t)b * m.vm.vint;
    const bool last = b == m.B - 1;   // xh, xl are read by the next gradient only: written after the last block
    for (int64_t j = it.i0 + threadIdx.x; j < it.i1; j += blockDim.x) {
        const int64_t p = vox_internal(m.vm, j);
        const double v = m.x[j] + (double)m.delta[p] * (double)inv_s[p];
        m.x[j] = v;
        const float h = (float)v;
        m.x32[p] = h;
        if (last) {
            m.xh[j] = h;
            m.xl[j] = (float)(v - (double)h);
        }
        m.delta[p] = 0.f;
    }
}

// phi of every member into tv_hist[k]
__global__ void __launch_bounds__(256) tvb_value_kernel(const MemberDev* __restrict__ mem,
                                                        const Item* __restrict__ items, const int64_t* __restrict__ kk,
                                                        double* partials, unsigned* tickets) {
    const Item it = items[blockIdx.x];
    const MemberDev m = mem[it.member];
    const int nx = m.nx, ny = m.ny, nz = m.nz;
    const int64_t sxy = (int64_t)nx * ny;
    double acc = 0.0;
    for (int64_t p = it.i0 + threadIdx.x; p < it.i1; p += blockDim.x) {
        int ix, iy, iz;
        voxel_coords(p, nx, ny, ix, iy, iz);
        const double xc = m.x[p];
        const double ex = (ix + 1 < nx) ? m.x[p + 1] - xc : 0.0, ey = (iy + 1 < ny) ? m.x[p + nx] - xc : 0.0,
                     ez = (iz + 1 < nz) ? m.x[p + sxy] - xc : 0.0;
        acc += sqrt(ex * ex + ey * ey + ez * ez);
    }
    member_reduce(acc, blockIdx.x, m, it.member, partials, tickets, m.tv_hist + kk[it.member]);
}

__global__ void zero_resid_kernel(const MemberDev* __restrict__ mem, int R, int b) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < R && b < mem[r].B) mem[r].resid[b] = 0.0;
}

__global__ void advance_k_kernel(int64_t* kk, int R) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < R) kk[r] += 1;
}

// ------------------------------------------------------------------ host side
int bfail(int code, const std::string& m) {
    set_last_error(m);
    return code;
}
#define BCUDA(expr)                                                                                     \
    do {                                                                                                \
        cudaError_t e_ = (expr);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return bfail(e_ == cudaErrorMemoryAllocation ? NTVS_ERR_OOM : NTVS_ERR_CUDA,                \
                         std::string(#expr) + ": " + cudaGetErrorString(e_));                          \
    } while (0)
#define BTRY(expr)                    \
    do {                              \
        int r_ = (expr);              \
        if (r_ != NTVS_OK) return r_; \
    } while (0)

template <typename P>
int balloc(P** p, size_t bytes, const char* what) {
    *p = nullptr;
    cudaError_t e = cudaMalloc((void**)p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(e == cudaErrorMemoryAllocation ? NTVS_ERR_OOM : NTVS_ERR_CUDA,
                     std::string("batch allocation of ") + what + ": " + cudaGetErrorString(e));
    }
    return NTVS_OK;
}

}  // namespace
}  // namespace ntvs

using namespace ntvs;

struct ntvs_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool finalized = false;
    struct Member {
        MemberDev d{};
        ntvs_params p{};
        std::vector<int64_t> block_ptr;
        int64_t M = 0, nnz = 0, k = 0, ell_prev = 0;
        std::vector<void*> owned;
    };
    std::vector<Member> m;
    // device tables
    MemberDev* dmem = nullptr;
    Item* tv_items = nullptr;
    int n_tv_items = 0;
    std::vector<Item*> drop_items;   // per block step b
    std::vector<int> n_drop_items;
    double* partials = nullptr;
    unsigned* tickets = nullptr;
    double* gnorm2 = nullptr;
    double* beta = nullptr;          // [N_max][R]
    double* hbeta[2] = {nullptr, nullptr};
    int64_t* kk = nullptr;           // per-member cycle index (tv_hist slot)
    int N_max = 0, B_max = 0;
    int lpr = 32;
    int64_t tv_cap = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    cudaEvent_t used[2] = {nullptr, nullptr};
    int next = 0;
    int64_t launches = 0, cycles = 0;
};

namespace {

// lanes per row 8 / 16 / 32 with 16 / 10 / 6 register steps (128 / 160 / 192 entries)
void launch_dropb(int lpr, int n_items, const MemberDev* mem, const Item* items, cudaStream_t s) {
    switch (lpr) {
        case 8: dropb_block_kernel<8, 16><<<n_items, 256, 0, s>>>(mem, items); break;
        case 16: dropb_block_kernel<16, 10><<<n_items, 256, 0, s>>>(mem, items); break;
        default: dropb_block_kernel<32, 6><<<n_items, 256, 0, s>>>(mem, items); break;
    }
}

int launch_cycle(ntvs_batch* bt, const double* beta_src) {
    cudaStream_t s = bt->stream;
    const int R = (int)bt->m.size();
    BCUDA(cudaMemcpyAsync(bt->beta, beta_src, sizeof(double) * (size_t)bt->N_max * R, cudaMemcpyHostToDevice, s));
    for (int n = 0; n < bt->N_max; ++n) {
        tvb_grad_kernel<<<bt->n_tv_items, 256, 0, s>>>(bt->dmem, bt->tv_items, n, bt->partials, bt->tickets,
                                                        bt->gnorm2);
        tvb_apply_kernel<<<bt->n_tv_items, 256, 0, s>>>(bt->dmem, bt->tv_items, n, bt->beta, R, bt->gnorm2);
    }
    for (int b = 0; b < bt->B_max; ++b) {
        zero_resid_kernel<<<(R + 127) / 128, 128, 0, s>>>(bt->dmem, R, b);
        if (bt->n_drop_items[b] > 0) launch_dropb(bt->lpr, bt->n_drop_items[b], bt->dmem, bt->drop_items[b], s);
        dropb_apply_kernel<<<bt->n_tv_items, 256, 0, s>>>(bt->dmem, bt->tv_items, b);
    }
    tvb_value_kernel<<<bt->n_tv_items, 256, 0, s>>>(bt->dmem, bt->tv_items, bt->kk, bt->partials, bt->tickets);
    advance_k_kernel<<<(R + 127) / 128, 128, 0, s>>>(bt->kk, R);
    BCUDA(cudaGetLastError());
    return NTVS_OK;
}

int kernels_per_cycle(const ntvs_batch* bt) {
    int n = 2 * bt->N_max + 2;
    for (int b = 0; b < bt->B_max; ++b) n += 2 + (bt->n_drop_items[b] > 0 ? 1 : 0);
    return n;
}

}  // namespace

extern "C" {

int ntvs_batch_create(ntvs_batch** out, int device, void* cuda_stream) {
    if (!out) return bfail(NTVS_ERR_ARG, "null output");
    *out = nullptr;
    int ndev = 0;
    BCUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return bfail(NTVS_ERR_ARG, "device index out of range");
    BCUDA(cudaSetDevice(device));
    ntvs_batch* bt = new ntvs_batch();
    bt->device = device;
    if (cuda_stream) {
        bt->stream = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete bt;
            return bfail(NTVS_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
        }
        bt->own_stream = true;
    }
    *out = bt;
    return NTVS_OK;
}

int ntvs_batch_destroy(ntvs_batch* bt) {
    if (!bt) return NTVS_OK;
    cudaSetDevice(bt->device);
    if (bt->stream) cudaStreamSynchronize(bt->stream);
    for (auto& mm : bt->m)
        for (void* p : mm.owned) cudaFree(p);
    cudaFree(bt->dmem);
    cudaFree(bt->tv_items);
    for (Item* p : bt->drop_items) cudaFree(p);
    cudaFree(bt->partials);
    cudaFree(bt->tickets);
    cudaFree(bt->gnorm2);
    cudaFree(bt->beta);
    cudaFree(bt->kk);
    for (int j = 0; j < 2; ++j) {
        if (bt->hbeta[j]) cudaFreeHost(bt->hbeta[j]);
        if (bt->graph[j]) cudaGraphExecDestroy(bt->graph[j]);
        if (bt->used[j]) cudaEventDestroy(bt->used[j]);
    }
    if (bt->own_stream && bt->stream) cudaStreamDestroy(bt->stream);
    delete bt;
    return NTVS_OK;
}

int ntvs_batch_add(ntvs_batch* bt, const ntvs_system* s, const ntvs_params* p, const void* x0, int x0_dtype,
                   int x0_mem, int* index) {
    if (!bt || !s || !p || !x0) return bfail(NTVS_ERR_ARG, "null argument");
    if (bt->finalized) return bfail(NTVS_ERR_STATE, "batch already finalized");
    BCUDA(cudaSetDevice(bt->device));
    if (s->val_dtype != NTVS_F32 || s->storage != NTVS_CSR32)
        return bfail(NTVS_ERR_ARG, "batched members take FP32 values in CSR32 storage");
    if (p->tv_check) return bfail(NTVS_ERR_ARG, "batched members run NTVS without the TV check");
    if (p->N < 0 || !(p->alpha > 0 && p->alpha < 1) || !(p->beta0 >= 0) || !(p->eps_tv >= 0))
        return bfail(NTVS_ERR_ARG, "bad parameters");
    if (p->step_rule < NTVS_STEP_NTVS || p->step_rule > NTVS_STEP_DECOUPLED)
        return bfail(NTVS_ERR_ARG, "unknown step_rule");
    if (p->step_rule == NTVS_STEP_DECOUPLED && !(p->gamma > 0 && p->gamma < 1))
        return bfail(NTVS_ERR_ARG, "gamma must lie in (0, 1)");
    if (s->nx < 1 || s->ny < 1 || s->nz < 1 || s->n_rows < 0) return bfail(NTVS_ERR_ARG, "bad sizes");
    if (x0_dtype != NTVS_F64 && x0_dtype != NTVS_F32) return bfail(NTVS_ERR_ARG, "x0 dtype must be F64 or F32");
    const int64_t V = (int64_t)s->nx * s->ny * s->nz;
    if (V > 0x7fffffffLL) return bfail(NTVS_ERR_ARG, "V too large");
    const int64_t M = s->n_rows;
    // host copies of the structure (blocks are planned on the host)
    std::vector<int64_t> rp((size_t)M + 1);
    const bool host = s->mem_kind == NTVS_MEM_HOST;
    if (host) std::memcpy(rp.data(), s->row_ptr, sizeof(int64_t) * rp.size());
    else BCUDA(cudaMemcpy(rp.data(), s->row_ptr, sizeof(int64_t) * rp.size(), cudaMemcpyDeviceToHost));
    if (rp[0] != 0) return bfail(NTVS_ERR_CSR, "row_ptr[0] != 0");
    for (int64_t i = 0; i < M; ++i)
        if (rp[i] > rp[i + 1]) return bfail(NTVS_ERR_CSR, "row_ptr decreases");
    const int64_t nnz = rp[M];
    std::vector<int32_t> col((size_t)nnz);
    std::vector<float> val((size_t)nnz), b((size_t)M);
    if (host) {
        std::memcpy(col.data(), s->col, sizeof(int32_t) * col.size());
        std::memcpy(val.data(), s->val, sizeof(float) * val.size());
        std::memcpy(b.data(), s->b, sizeof(float) * b.size());
    } else {
        BCUDA(cudaMemcpy(col.data(), s->col, sizeof(int32_t) * col.size(), cudaMemcpyDeviceToHost));
        BCUDA(cudaMemcpy(val.data(), s->val, sizeof(float) * val.size(), cudaMemcpyDeviceToHost));
        BCUDA(cudaMemcpy(b.data(), s->b, sizeof(float) * b.size(), cudaMemcpyDeviceToHost));
    }
    for (int64_t q = 0; q < nnz; ++q)
        if (col[q] < 0 || col[q] >= V || !std::isfinite(val[q])) return bfail(NTVS_ERR_CSR, "bad column or value");
    for (int64_t i = 0; i < M; ++i)
        if (!std::isfinite(b[i])) return bfail(NTVS_ERR_CSR, "non-finite right-hand side");
    // blocks, norms, hit counts (host, FP64)
    std::vector<int64_t> bp;
    if (s->block_ptr) {
        bp.assign(s->block_ptr, s->block_ptr + s->n_blocks + 1);
        if (bp.front() != 0 || bp.back() != M) return bfail(NTVS_ERR_ARG, "block_ptr must run from 0 to n_rows");
    } else {
        if (s->n_blocks < 1) return bfail(NTVS_ERR_ARG, "n_blocks must be >= 1");
        const int64_t per = (M + s->n_blocks - 1) / s->n_blocks;
        for (int t = 0; t <= s->n_blocks; ++t) bp.push_back(std::min<int64_t>((int64_t)t * per, M));
    }
    const int B = (int)bp.size() - 1;
    // internal voxel order (4x4 in-plane tiles, as the single-context FP32 path)
    VoxMap vm = make_voxmap(s->nx, s->ny, s->nz, 4, 4);
    if (vm.vint > 0x7fffffffLL) vm = make_voxmap(s->nx, s->ny, s->nz, 1, 1);
    const int64_t VI = vm.vint;
    std::vector<float> inn((size_t)M), inv_s((size_t)B * VI, 0.f);
    for (int64_t i = 0; i < M; ++i) {
        double n2 = 0.0;
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) n2 += (double)val[q] * (double)val[q];
        inn[i] = n2 > 0.0 ? (float)(1.0 / n2) : 0.f;
    }
    {
        std::vector<int32_t> cnt((size_t)V);
        for (int t = 0; t < B; ++t) {
            std::fill(cnt.begin(), cnt.end(), 0);
            for (int64_t q = rp[bp[t]]; q < rp[bp[t + 1]]; ++q)
                if (val[q] != 0.f) cnt[col[q]] += 1;
            for (int64_t j = 0; j < V; ++j)
                inv_s[(size_t)t * VI + vox_internal_host(vm, j)] = cnt[j] ? (float)(1.0 / cnt[j]) : 0.f;
        }
    }
    ntvs_batch::Member mm;
    MemberDev& d = mm.d;
    auto up = [&](void** dst, const void* src, size_t bytes, const char* what) -> int {
        BTRY(balloc(dst, bytes, what));
        mm.owned.push_back(*dst);
        if (src && bytes) BCUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
        return NTVS_OK;
    };
    std::vector<double> x((size_t)V);
    if (x0_mem == NTVS_MEM_HOST) {
        if (x0_dtype == NTVS_F64) std::memcpy(x.data(), x0, sizeof(double) * V);
        else for (int64_t j = 0; j < V; ++j) x[j] = ((const float*)x0)[j];
    } else {
        if (x0_dtype == NTVS_F64) BCUDA(cudaMemcpy(x.data(), x0, sizeof(double) * V, cudaMemcpyDeviceToHost));
        else {
            std::vector<float> t((size_t)V);
            BCUDA(cudaMemcpy(t.data(), x0, sizeof(float) * V, cudaMemcpyDeviceToHost));
            for (int64_t j = 0; j < V; ++j) x[j] = t[j];
        }
    }
    std::vector<float> x32((size_t)VI, 0.f), xh((size_t)V), xl((size_t)V);
    for (int64_t j = 0; j < V; ++j) {
        xh[j] = (float)x[j];
        xl[j] = (float)(x[j] - (double)xh[j]);
        x32[(size_t)vox_internal_host(vm, j)] = xh[j];
    }
    for (auto& c : col) c = (int32_t)vox_internal_host(vm, c);   // validated above
    int rc = NTVS_OK;
    if ((rc = up((void**)&d.row_ptr, rp.data(), sizeof(int64_t) * rp.size(), "row_ptr")) ||
        (rc = up((void**)&d.col, col.data(), sizeof(int32_t) * col.size(), "col")) ||
        (rc = up((void**)&d.val, val.data(), sizeof(float) * val.size(), "val")) ||
        (rc = up((void**)&d.b, b.data(), sizeof(float) * b.size(), "b")) ||
        (rc = up((void**)&d.inv_norm2, inn.data(), sizeof(float) * inn.size(), "inv_norm2")) ||
        (rc = up((void**)&d.inv_s, inv_s.data(), sizeof(float) * inv_s.size(), "inv_s")) ||
        (rc = up((void**)&d.x, x.data(), sizeof(double) * V, "x")) ||
        (rc = up((void**)&d.x32, x32.data(), sizeof(float) * VI, "x32")) ||
        (rc = up((void**)&d.xh, xh.data(), sizeof(float) * V, "xh")) ||
        (rc = up((void**)&d.xl, xl.data(), sizeof(float) * V, "xl")) ||
        (rc = up((void**)&d.delta, nullptr, sizeof(float) * VI, "delta")) ||
        (rc = up((void**)&d.g, nullptr, sizeof(float) * V, "g")) ||
        (rc = up((void**)&d.resid, nullptr, sizeof(double) * std::max(B, 1), "resid"))) {
        for (void* q : mm.owned) cudaFree(q);
        return rc;
    }
    BCUDA(cudaMemset((void*)d.delta, 0, sizeof(float) * VI));
    BCUDA(cudaMemset((void*)d.resid, 0, sizeof(double) * std::max(B, 1)));
    d.nx = s->nx; d.ny = s->ny; d.nz = s->nz; d.B = B; d.N = p->N; d.V = V;
    d.vm = vm;
    d.lambda = (float)p->lambda;
    d.eps = (float)p->eps_tv;
    mm.p = *p;
    mm.block_ptr = bp;
    mm.M = M;
    mm.nnz = nnz;
    bt->m.push_back(std::move(mm));
    if (index) *index = (int)bt->m.size() - 1;
    return NTVS_OK;
}

int ntvs_batch_finalize(ntvs_batch* bt, int max_cycles) {
    if (!bt) return bfail(NTVS_ERR_ARG, "null batch");
    if (bt->finalized) return bfail(NTVS_ERR_STATE, "batch already finalized");
    if (bt->m.empty()) return bfail(NTVS_ERR_STATE, "empty batch");
    if (max_cycles < 1) return bfail(NTVS_ERR_ARG, "max_cycles must be >= 1");
    BCUDA(cudaSetDevice(bt->device));
    const int R = (int)bt->m.size();
    // TV items (every voxel of every member) and DROP items per block step
    std::vector<Item> tv;
    bt->N_max = 0;
    bt->B_max = 0;
    for (int r = 0; r < R; ++r) {
        MemberDev& d = bt->m[r].d;
        d.item0 = (int)tv.size();
        for (int64_t v = 0; v < d.V; v += kTvItem) tv.push_back({r, 0, v, std::min<int64_t>(d.V, v + kTvItem)});
        d.nitems = (int)tv.size() - d.item0;
        bt->N_max = std::max(bt->N_max, d.N);
        bt->B_max = std::max(bt->B_max, d.B);
        BTRY(balloc(&d.tv_hist, sizeof(double) * (size_t)max_cycles, "tv history"));
        bt->m[r].owned.push_back(d.tv_hist);
    }
    bt->tv_cap = max_cycles;
    bt->n_tv_items = (int)tv.size();
    BTRY(balloc(&bt->tv_items, sizeof(Item) * tv.size(), "TV items"));
    BCUDA(cudaMemcpy(bt->tv_items, tv.data(), sizeof(Item) * tv.size(), cudaMemcpyHostToDevice));
    for (int b = 0; b < bt->B_max; ++b) {
        std::vector<Item> it;
        for (int r = 0; r < R; ++r) {
            const auto& mm = bt->m[r];
            if (b >= mm.d.B) continue;
            for (int64_t i = mm.block_ptr[b]; i < mm.block_ptr[b + 1]; i += kDropItem)
                it.push_back({r, b, i, std::min<int64_t>(mm.block_ptr[b + 1], i + kDropItem)});
        }
        Item* di = nullptr;
        BTRY(balloc(&di, sizeof(Item) * std::max<size_t>(it.size(), 1), "DROP items"));
        if (!it.empty()) BCUDA(cudaMemcpy(di, it.data(), sizeof(Item) * it.size(), cudaMemcpyHostToDevice));
        bt->drop_items.push_back(di);
        bt->n_drop_items.push_back((int)it.size());
    }
    std::vector<MemberDev> md;
    for (auto& mm : bt->m) md.push_back(mm.d);
    BTRY(balloc(&bt->dmem, sizeof(MemberDev) * R, "member table"));
    BCUDA(cudaMemcpy(bt->dmem, md.data(), sizeof(MemberDev) * R, cudaMemcpyHostToDevice));
    BTRY(balloc(&bt->partials, sizeof(double) * std::max(bt->n_tv_items, 1), "partials"));
    BTRY(balloc(&bt->tickets, sizeof(unsigned) * R, "tickets"));
    BTRY(balloc(&bt->gnorm2, sizeof(double) * R, "gnorm2"));
    BTRY(balloc(&bt->beta, sizeof(double) * std::max(bt->N_max, 1) * R, "beta table"));
    BTRY(balloc(&bt->kk, sizeof(int64_t) * R, "cycle index"));
    BCUDA(cudaMemset(bt->tickets, 0, sizeof(unsigned) * R));
    BCUDA(cudaMemset(bt->kk, 0, sizeof(int64_t) * R));
    for (int j = 0; j < 2; ++j) {
        BCUDA(cudaHostAlloc((void**)&bt->hbeta[j], sizeof(double) * std::max(bt->N_max, 1) * R, cudaHostAllocDefault));
        std::memset(bt->hbeta[j], 0, sizeof(double) * std::max(bt->N_max, 1) * R);
        BCUDA(cudaEventCreateWithFlags(&bt->used[j], cudaEventDisableTiming));
    }
    // autotune lanes per row on block step 0 (delta is cleared afterwards; x is untouched)
    if (bt->B_max > 0 && bt->n_drop_items[0] > 0) {
        cudaEvent_t e0, e1;
        BCUDA(cudaEventCreate(&e0));
        BCUDA(cudaEventCreate(&e1));
        float best = 1e30f;
        for (int lpr : {8, 16, 32}) {
            float total = 0.f;
            for (int rep = 0; rep < 2; ++rep) {
                BCUDA(cudaEventRecord(e0, bt->stream));
                launch_dropb(lpr, bt->n_drop_items[0], bt->dmem, bt->drop_items[0], bt->stream);
                BCUDA(cudaEventRecord(e1, bt->stream));
                BCUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                BCUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (rep) total += ms;
            }
            if (total < best) { best = total; bt->lpr = lpr; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        for (auto& mm : bt->m) {
            BCUDA(cudaMemsetAsync(mm.d.delta, 0, sizeof(float) * mm.d.vm.vint, bt->stream));
            BCUDA(cudaMemsetAsync(mm.d.resid, 0, sizeof(double) * std::max(mm.d.B, 1), bt->stream));
        }
        BCUDA(cudaStreamSynchronize(bt->stream));
    }
    // one graph per pinned beta buffer
    for (int j = 0; j < 2; ++j) {
        cudaGraph_t g = nullptr;
        BCUDA(cudaStreamBeginCapture(bt->stream, cudaStreamCaptureModeThreadLocal));
        int rc = launch_cycle(bt, bt->hbeta[j]);
        cudaError_t e = cudaStreamEndCapture(bt->stream, &g);
        if (rc != NTVS_OK) return rc;
        if (e != cudaSuccess) return bfail(NTVS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&bt->graph[j], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bfail(NTVS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    bt->finalized = true;
    return NTVS_OK;
}

int ntvs_batch_run(ntvs_batch* bt, int k_iters) {
    if (!bt) return bfail(NTVS_ERR_ARG, "null batch");
    if (!bt->finalized) return bfail(NTVS_ERR_STATE, "batch not finalized");
    if (k_iters < 0) return bfail(NTVS_ERR_ARG, "k_iters < 0");
    BCUDA(cudaSetDevice(bt->device));
    const int R = (int)bt->m.size();
    for (int it = 0; it < k_iters; ++it) {
        if (bt->cycles >= bt->tv_cap) return bfail(NTVS_ERR_STATE, "more cycles than finalize's max_cycles");
        const int j = bt->next;
        BCUDA(cudaEventSynchronize(bt->used[j]));   // the graph that last read this buffer has copied it
        double* hb = bt->hbeta[j];
        for (int r = 0; r < R; ++r) {
            auto& mm = bt->m[r];
            const int64_t k = mm.k;
            int64_t ell = cycle_ell(mm.p, k, mm.ell_prev);
            const int64_t adv = ell_advances(mm.p) ? 1 : 0;
            for (int n = 0; n < bt->N_max; ++n) {
                hb[(size_t)n * R + r] = (n < mm.p.N) ? step_beta(mm.p, k, n, ell) : 0.0;
                if (n < mm.p.N) ell += adv;
            }
            if (adv) mm.ell_prev = ell;
            mm.k = k + 1;
        }
        BCUDA(cudaGraphLaunch(bt->graph[j], bt->stream));
        BCUDA(cudaEventRecord(bt->used[j], bt->stream));
        bt->next ^= 1;
        bt->cycles += 1;
        bt->launches += kernels_per_cycle(bt);
    }
    return NTVS_OK;
}

int ntvs_batch_get_image(ntvs_batch* bt, int index, void* out, int dtype, int mem_kind) {
    if (!bt || !out) return bfail(NTVS_ERR_ARG, "null argument");
    if (index < 0 || index >= (int)bt->m.size()) return bfail(NTVS_ERR_ARG, "member index out of range");
    if (dtype != NTVS_F64 && dtype != NTVS_F32) return bfail(NTVS_ERR_ARG, "dtype must be F64 or F32");
    BCUDA(cudaSetDevice(bt->device));
    const MemberDev& d = bt->m[index].d;
    std::vector<double> x((size_t)d.V);
    BCUDA(cudaMemcpyAsync(x.data(), d.x, sizeof(double) * d.V, cudaMemcpyDeviceToHost, bt->stream));
    BCUDA(cudaStreamSynchronize(bt->stream));
    if (mem_kind == NTVS_MEM_HOST) {
        if (dtype == NTVS_F64) std::memcpy(out, x.data(), sizeof(double) * d.V);
        else for (int64_t j = 0; j < d.V; ++j) ((float*)out)[j] = (float)x[j];
        return NTVS_OK;
    }
    if (dtype == NTVS_F64) {
        BCUDA(cudaMemcpy(out, x.data(), sizeof(double) * d.V, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f((size_t)d.V);
        for (int64_t j = 0; j < d.V; ++j) f[j] = (float)x[j];
        BCUDA(cudaMemcpy(out, f.data(), sizeof(float) * d.V, cudaMemcpyHostToDevice));
    }
    return NTVS_OK;
}

int ntvs_batch_get_tv(ntvs_batch* bt, int index, double* tv) {
    if (!bt || !tv) return bfail(NTVS_ERR_ARG, "null argument");
    if (index < 0 || index >= (int)bt->m.size()) return bfail(NTVS_ERR_ARG, "member index out of range");
    const auto& mm = bt->m[index];
    if (mm.k == 0) return bfail(NTVS_ERR_STATE, "no cycle run yet");
    BCUDA(cudaSetDevice(bt->device));
    BCUDA(cudaMemcpyAsync(tv, mm.d.tv_hist + (mm.k - 1), sizeof(double), cudaMemcpyDeviceToHost, bt->stream));
    BCUDA(cudaStreamSynchronize(bt->stream));
    return NTVS_OK;
}

int ntvs_batch_get_stats(ntvs_batch* bt, ntvs_batch_stats* st) {
    if (!bt || !st) return bfail(NTVS_ERR_ARG, "null argument");
    std::memset(st, 0, sizeof(*st));
    st->members = (int32_t)bt->m.size();
    st->lanes_per_row = bt->lpr;
    st->cycles = bt->cycles;
    st->n_launches = bt->launches;
    st->kernels_per_cycle = bt->finalized ? kernels_per_cycle(bt) : 0;
    for (const auto& mm : bt->m) {
        st->total_rows += mm.M;
        st->total_nnz += mm.nnz;
        st->total_voxels += mm.d.V;
    }
    return NTVS_OK;
}

}  // extern "C"
