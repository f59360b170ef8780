// Batched NTVS: many independent reconstructions (each with its own grid, system, block
// partition and (lambda, N, alpha, beta0, eps, seed, TV check)) advanced together by one
// persistent kernel per cycle (arXiv 1803.01112, Appendix C, for every member; the TV
// check of Sec. III-E as a per-member option).
//
// Work model.  A member's cycle is a sequence of phases,
//     [GRAD(n), (TRY(n) ...), APPLY(n)] for n < N,  [DROP(b), DAPPLY(b)] for b < B,  PHI,
// each cut into items: runs of kTvItem voxels (GRAD, TRY, APPLY, DAPPLY, PHI) or of a
// member-specific number of rows of block b (DROP).  Phases of one member run in order;
// phases of different members overlap.  Every member has a 64-bit word (phase epoch |
// items in the phase | cursor); a CTA takes an item with one atomic add on the cursor,
// processes it without waiting on anything, and counts it done.  The CTA that finishes a
// phase's last item does the phase's reductions (in a fixed order: deterministic), decides
// the next phase and publishes it with one atomic exchange of the word.  A CTA that finds
// no item waits (polling, bounded by %globaltimer); since no item ever waits, every taken
// item completes and the cycle ends without co-residency or grid barriers.  When the wait
// runs out the CTA records an error and every CTA leaves (NTVS_ERR_TIMEOUT on the host).
//
// Memory ordering.  Data written inside the kernel (the image and its copies, g, delta,
// partials) is read with plain loads, which may be served by the SM's L1: every item is
// taken by an atomic on the schedule word followed by a gpu-scope fence and a CTA barrier
// (an acquire), and every phase is published by a fence before the exchange (a release),
// so by the PTX memory model the loads of an item see everything its member's earlier
// phases wrote.  The non-coherent read-only path (__ldg) is used only for data that no
// phase writes (rows, b, 1/||a||^2, 1/s, tables).
//
// TV check (TRY): each pass evaluates phi(z_t), z_t = x - beta_{ell+t} g / ||g||, for
// kSpec consecutive tries t at once (x and g read once for all of them); the first t with
// phi(z_t) <= phi(x) is the accepted try, as if the tries had run one by one; a pass with
// no acceptance is followed by another until max_retries tries were made.
//
// DROP items process rows with LPR lanes per row (8, 16 or 32, per member from its row
// length) holding the row's first CH*LPR entries in registers between the dot product
// and the scatter; a member's entries are stored as {column, value} pairs, one 8-byte
// load each.  The scatter either goes to global memory (FP32 reductions) or is staged
// in a shared window of the CTA (the item's whole column range when it fits, else the
// range centred on its mean column, whose outside entries still go to global memory),
// flushed once per item: only the window's nonzero entries become global reductions.
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

constexpr int kThreads = 256;     // threads per CTA of the persistent kernel
constexpr int kTvItem = 2048;     // voxels per voxel item (256 threads x 8)
constexpr int kSpec = 4;          // TV-check tries evaluated per pass
constexpr int kBetaTab = 4096;    // beta0 alpha^ell from the host for ell < kBetaTab
constexpr unsigned long long kM24 = 0xffffffull;
constexpr int kErrBatchStall = 16;   // error word: an idle CTA's bounded wait ran out

enum : int { PH_GRAD = 0, PH_TRY = 1, PH_APPLY = 2, PH_DROP = 3, PH_DAPPLY = 4, PH_PHI = 5, PH_DONE = 6 };

// Read-only description of one member (pointers owned by the batch).
struct MemberDev {
    const int64_t* row_ptr;
    const int32_t* col;        // internal voxel order (until the member is prepared)
    const float* val;
    const int2* ent;           // [nnz] {column, value bits}: the prepared member's entries
    const float* b;
    const float* inv_norm2;
    const float* inv_s;        // [B][vint], internal voxel order
    const int64_t* block_ptr;  // [B+1]
    const int32_t* win_lo;     // [n_drop_items] first column of each DROP item's window, -1: none
    const int32_t* item0;      // [B] index of block b's first DROP item in win_lo
    const double* beta_tab;    // [kBetaTab] beta0 alpha^ell (TV check)
    double* x;                 // master image, canonical order
    float* x32;                // fl32(x), internal order (the DROP gathers)
    float* xh;                 // fl32(x) and fl32(x - xh), canonical order (gradient stencil)
    float* xl;
    float* delta;              // internal order
    float* g;                  // canonical order
    double* resid;             // [B]
    float* wstat;              // [4B] per block: lmax, bound, observed max (float bits), amax (the
                               // fixed-point DROP window's scale, as in the single-context kernel)
    double* tv_hist;           // [cap]
    int nx, ny, nz, B, N;
    int64_t V;
    VoxMap vm;
    float lambda, eps;
    double beta0, alpha;
    int check, max_retries, rule;
    uint64_t seed;
    int lpr, rows_per_item, n_vox_items, part_off;
};

// Mutable per-member state of the schedule.
struct MemberState {
    unsigned long long word;   // [63:48] epoch, [47:24] items of the phase, [23:0] cursor
    unsigned done;             // items of the phase finished
    int phase, n, b, tries;    // tries: of the current TV step (TV check)
    int64_t ell, k;            // ell (TV check, carried across cycles); cycles completed
    double gnorm2, phi_x, sc;
    int64_t n_tries, n_accepted, n_steps;
};

struct RunState {
    unsigned members_done;
    int err, err_member, err_phase;
};

struct CycleArgs {
    const MemberDev* mem;
    MemberState* st;
    RunState* run;
    int R;
    double* part;      // [total voxel items] ||g||^2 or phi partials
    double* part2;     // [total voxel items] phi(x) partials (TV check)
    double* part_try;  // [total voxel items][kSpec] phi(z_t) partials
    const double* beta;   // [N_max][R] beta_{k,n} of the cycle (no TV check)
    uint64_t wait_ns;
    int starve;        // test hook: member 0's first phase never ends
    int win_cap;       // floats of the shared scatter window (0: global scatter only)
};

__device__ __forceinline__ unsigned long long pack_word(unsigned epoch, unsigned items) {
    return ((unsigned long long)(epoch & 0xffffu) << 48) | ((unsigned long long)(items & kM24) << 24);
}

__device__ __forceinline__ unsigned long long ld_word(const unsigned long long* p) {
    return *(volatile const unsigned long long*)p;
}

// sum over i < n of a[i * stride] in a fixed order (every thread a strided subset, then the
// block tree): the same order whichever CTA does it
__device__ __forceinline__ double ordered_sum(const double* a, int n, int stride, double* sh) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += a[(size_t)i * stride];
    return block_sum(s, sh);   // valid in thread 0
}

// ---------------------------------------------------------------- voxel items

// gradient of phi_eps (FP32 stencil on x = xh + xl) on the item's voxels; partials of
// ||g||^2 and (TV check) of phi(x) from the FP64 image
__device__ void grad_item(const MemberDev& m, int idx, double* part, double* part2, double* sh) {
    const int nx = m.nx, ny = m.ny, nz = m.nz;
    const int64_t sxy = (int64_t)nx * ny;
    const int64_t i0 = (int64_t)idx * kTvItem, i1 = min(m.V, i0 + kTvItem);
    const float* xh = m.xh;
    const float* xl = m.xl;
    const float eps = m.eps;
    auto dif = [&](int64_t a, int64_t b) -> float {
        return (xh[a] - xh[b]) + (xl[a] - xl[b]);
    };
    double acc = 0.0, phi = 0.0;
    for (int64_t p = i0 + threadIdx.x; p < i1; p += blockDim.x) {
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
        if (m.check) {
            const double xc = m.x[p];
            const double ex = hx ? m.x[p + 1] - xc : 0.0, ey = hy ? m.x[p + nx] - xc : 0.0,
                         ez = hz ? m.x[p + sxy] - xc : 0.0;
            phi += sqrt(ex * ex + ey * ey + ez * ez);
        }
    }
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) part[m.part_off + idx] = t;
    if (m.check) {
        const double tp = block_sum(phi, sh);
        if (threadIdx.x == 0) part2[m.part_off + idx] = tp;
    }
}

__device__ __forceinline__ double beta_of(const MemberDev& m, int64_t ell) {
    return (ell >= 0 && ell < kBetaTab) ? __ldg(m.beta_tab + ell) : m.beta0 * pow(m.alpha, (double)ell);
}

// phi(z_t) partials of the item's voxels for the pass's tries t < T (z_t = x - sc_t g)
__device__ void try_item(const MemberDev& m, int idx, int64_t ell, int T, double gnorm2, double* part_try, double* sh) {
    const int nx = m.nx, ny = m.ny, nz = m.nz;
    const int64_t sxy = (int64_t)nx * ny;
    const int64_t i0 = (int64_t)idx * kTvItem, i1 = min(m.V, i0 + kTvItem);
    double sc[kSpec], acc[kSpec];
#pragma unroll
    for (int t = 0; t < kSpec; ++t) {
        sc[t] = (t < T && gnorm2 > 0.0) ? beta_of(m, ell + t) / sqrt(gnorm2) : 0.0;
        acc[t] = 0.0;
    }
    for (int64_t p = i0 + threadIdx.x; p < i1; p += blockDim.x) {
        int ix, iy, iz;
        voxel_coords(p, nx, ny, ix, iy, iz);
        const double xc = m.x[p], gc = (double)m.g[p];
        const bool hx = ix + 1 < nx, hy = iy + 1 < ny, hz = iz + 1 < nz;
        const double xx = hx ? m.x[p + 1] : 0.0, gx = hx ? (double)m.g[p + 1] : 0.0;
        const double xy = hy ? m.x[p + nx] : 0.0, gy = hy ? (double)m.g[p + nx] : 0.0;
        const double xz = hz ? m.x[p + sxy] : 0.0, gz = hz ? (double)m.g[p + sxy] : 0.0;
#pragma unroll
        for (int t = 0; t < kSpec; ++t) {
            if (t < T) {
                const double zc = perturbed(xc, sc[t], gc);
                const double ex = hx ? perturbed(xx, sc[t], gx) - zc : 0.0;
                const double ey = hy ? perturbed(xy, sc[t], gy) - zc : 0.0;
                const double ez = hz ? perturbed(xz, sc[t], gz) - zc : 0.0;
                acc[t] += sqrt(ex * ex + ey * ey + ez * ez);
            }
        }
    }
#pragma unroll
    for (int t = 0; t < kSpec; ++t) {
        if (t < T) {
            const double s = block_sum(acc[t], sh);
            if (threadIdx.x == 0) part_try[(size_t)(m.part_off + idx) * kSpec + t] = s;
        }
    }
}

// x <- x - sc g on the item's voxels, and the FP32 copies
__device__ void apply_item(const MemberDev& m, int idx, double sc) {
    const int64_t i0 = (int64_t)idx * kTvItem, i1 = min(m.V, i0 + kTvItem);
    for (int64_t p = i0 + threadIdx.x; p < i1; p += blockDim.x) {
        const double z = perturbed(m.x[p], sc, (double)m.g[p]);
        m.x[p] = z;
        const float h = (float)z;
        m.x32[vox_internal(m.vm, p)] = h;
        m.xh[p] = h;
        m.xl[p] = (float)(z - (double)h);
    }
}

// x += delta / s for block b on the item's voxels; delta cleared; after the last block
// also xh, xl (read by the next cycle's gradient only)
__device__ void dapply_item(const MemberDev& m, int idx, int b) {
    const int64_t i0 = (int64_t)idx * kTvItem, i1 = min(m.V, i0 + kTvItem);
    const float* inv_s = m.inv_s + (int64_t)b * m.vm.vint;
    const bool last = b == m.B - 1;
    for (int64_t j = i0 + threadIdx.x; j < i1; j += blockDim.x) {
        const int64_t p = vox_internal(m.vm, j);
        const double v = m.x[j] + (double)m.delta[p] * (double)__ldg(inv_s + p);
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

// phi(x) partial of the item's voxels (FP64)
__device__ void phi_item(const MemberDev& m, int idx, double* part, double* sh) {
    const int nx = m.nx, ny = m.ny, nz = m.nz;
    const int64_t sxy = (int64_t)nx * ny;
    const int64_t i0 = (int64_t)idx * kTvItem, i1 = min(m.V, i0 + kTvItem);
    double acc = 0.0;
    for (int64_t p = i0 + threadIdx.x; p < i1; p += blockDim.x) {
        int ix, iy, iz;
        voxel_coords(p, nx, ny, ix, iy, iz);
        const double xc = m.x[p];
        const double ex = (ix + 1 < nx) ? m.x[p + 1] - xc : 0.0, ey = (iy + 1 < ny) ? m.x[p + nx] - xc : 0.0,
                     ez = (iz + 1 < nz) ? m.x[p + sxy] - xc : 0.0;
        acc += sqrt(ex * ex + ey * ey + ez * ez);
    }
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) part[m.part_off + idx] = t;
}

// ---------------------------------------------------------------- DROP items

extern __shared__ float batch_win[];   // the shared scatter window (win_cap floats)

// rows [i0, i1) of member m: LPR lanes per row, CH register steps; when w0 >= 0 the
// entries with columns in [w0, w0 + win_cap) are scattered into the shared window and the
// others into global delta, else every entry into global delta
template <int LPR, int CH>
__device__ void drop_rows(const MemberDev& m, int64_t i0, int64_t i1, int w0, int win_cap, double* resid_b,
                          double* sh, float invQ, float bnd, unsigned* obs) {
    constexpr int G = 32 / LPR;
    const int lane = threadIdx.x & 31, sub = lane % LPR;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const bool win = w0 >= 0;
    double ss = 0.0;
    for (int64_t base = i0 + (int64_t)warp * G; base < i1; base += (int64_t)nw * G) {
        const int64_t i = base + lane / LPR;
        const bool valid = i < i1;
        int64_t p0 = 0, p1 = 0;
        if (valid) { p0 = __ldg(m.row_ptr + i); p1 = __ldg(m.row_ptr + i + 1); }
        int32_t c[CH];
        float a[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const int64_t q = p0 + (int64_t)u * LPR + sub;
            if (q < p1) {
                const int2 e = __ldcs(m.ent + q);   // one 8-byte load per entry
                c[u] = e.x;
                a[u] = __int_as_float(e.y);
            } else {
                c[u] = -1;
                a[u] = 0.f;
            }
        }
        float acc = 0.f;
#pragma unroll
        for (int u = 0; u < CH; ++u)
            if (c[u] >= 0) acc += a[u] * m.x32[c[u]];
        const int64_t tail0 = p0 + (int64_t)CH * LPR;
        for (int64_t q = tail0 + sub; q < p1; q += LPR) {
            const int2 e = __ldg(m.ent + q);
            acc += __int_as_float(e.y) * m.x32[e.x];
        }
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        float r = 0.f, rn = 0.f;
        if (valid) {
            const float res = __ldg(m.b + i) - acc;
            rn = res * __ldg(m.inv_norm2 + i);
            r = m.lambda * rn;
            if (sub == 0) ss += (double)res * (double)res;
            // the block's largest |r / lambda| (the next sweep's window bound); a plain read
            // first skips the atomic for most rows
            const unsigned arn = __float_as_uint(fabsf(rn));
            if (sub == 0 && obs && arn > *(volatile unsigned*)obs) atomicMax(obs, arn);
        }
        // a row within the bound adds its terms to the window as int32 multiples of the
        // quantum (every term below 2^22 quanta, every slot below 2^30): r / Q = r * invQ
        const bool rowfix = invQ > 0.f && fabsf(rn) <= bnd;
        const float rq = r * invQ;
        int* wint = reinterpret_cast<int*>(batch_win);
        if (win) {   // entries inside the window to shared memory, the others to global memory
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                if (c[u] >= 0) {
                    const unsigned o = (unsigned)(c[u] - w0);
                    if (rowfix && o < (unsigned)win_cap)   // adding 1.5 * 2^23 rounds to the nearest integer
                        atomicAdd(wint + o, __float_as_int(fmaf(rq, a[u], 12582912.0f)) - 0x4B400000);
                    else
                        atomicAdd(m.delta + c[u], r * a[u]);
                }
            }
            for (int64_t q = tail0 + sub; q < p1; q += LPR) {
                const int2 e = __ldg(m.ent + q);
                const unsigned o = (unsigned)(e.x - w0);
                const float av = __int_as_float(e.y);
                if (rowfix && o < (unsigned)win_cap)
                    atomicAdd(wint + o, __float_as_int(fmaf(rq, av, 12582912.0f)) - 0x4B400000);
                else
                    atomicAdd(m.delta + e.x, r * av);
            }
        } else {
#pragma unroll
            for (int u = 0; u < CH; ++u)
                if (c[u] >= 0) atomicAdd(m.delta + c[u], r * a[u]);
            for (int64_t q = tail0 + sub; q < p1; q += LPR) {
                const int2 e = __ldg(m.ent + q);
                atomicAdd(m.delta + e.x, r * __int_as_float(e.y));
            }
        }
    }
    const double tot = block_sum(ss, sh);
    if (threadIdx.x == 0 && tot != 0.0) atomicAdd(resid_b, tot);
}

__device__ void drop_item(const MemberDev& m, int b, int idx, int win_cap, double* sh) {
    const int64_t r0 = __ldg(m.block_ptr + b) + (int64_t)idx * m.rows_per_item;
    const int64_t r1 = min(__ldg(m.block_ptr + b + 1), r0 + m.rows_per_item);
    const int w0 = win_cap > 0 ? __ldg(m.win_lo + __ldg(m.item0 + b) + idx) : -1;
    // the window's quantum Q = |lambda| bound lmax / 2^30 from the block's statistics (lmax:
    // the largest column sum of |a_ij| over the block's rows, so no slot passes 2^30 Q);
    // rows above min(bound, 2^22 Q / (|lambda| amax)) go to global memory
    float Q = 0.f, invQ = 0.f, bnd = 0.f;
    unsigned* obs = m.wstat ? reinterpret_cast<unsigned*>(m.wstat + 2 * m.B + b) : nullptr;
    if (w0 >= 0 && m.wstat) {
        const float lmax = m.wstat[b], bound = m.wstat[m.B + b], amax = m.wstat[3 * m.B + b];
        const float lam = fabsf(m.lambda);
        Q = lam * bound * lmax * 0x1p-30f;
        const float iq = 1.f / Q;
        if (bound > 0.f && amax > 0.f && Q > 0.f && isfinite(Q) && isfinite(iq)) {
            invQ = iq;
            bnd = fminf(bound, 0x1p22f * Q / (lam * amax));
        }
    }
    if (w0 >= 0) {
        for (int j = threadIdx.x; j < win_cap; j += blockDim.x) batch_win[j] = 0.f;   // int 0 has the bits of 0.0f
        __syncthreads();
    }
    switch (m.lpr) {
        case 8: drop_rows<8, 16>(m, r0, r1, w0, win_cap, m.resid + b, sh, invQ, bnd, obs); break;
        case 16: drop_rows<16, 10>(m, r0, r1, w0, win_cap, m.resid + b, sh, invQ, bnd, obs); break;
        default: drop_rows<32, 6>(m, r0, r1, w0, win_cap, m.resid + b, sh, invQ, bnd, obs); break;
    }
    if (w0 >= 0) {
        __syncthreads();
        const int64_t n = min((int64_t)win_cap, m.vm.vint - (int64_t)w0);
        const int* wint = reinterpret_cast<const int*>(batch_win);
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const int v = wint[j];
            if (v != 0) atomicAdd(m.delta + w0 + j, (float)v * Q);
        }
    }
}

// ---------------------------------------------------------------- the phase machine

__device__ __forceinline__ int drop_items_of(const MemberDev& m, int b) {
    const int64_t rows = __ldg(m.block_ptr + b + 1) - __ldg(m.block_ptr + b);
    return (int)((rows + m.rows_per_item - 1) / m.rows_per_item);
}

// The first phase at or after (phase, n, b) that has items (DROP of an empty block is
// skipped; its DAPPLY still runs); returns its item count, 0 for DONE.
__device__ int settle(const MemberDev& m, int& phase, int& n, int& b) {
    for (int guard = 0; guard < 4; ++guard) {
        if (phase == PH_GRAD && n >= m.N) {
            phase = PH_DROP;
            b = 0;
        }
        if (phase == PH_DROP && b >= m.B) phase = PH_PHI;
        if (phase == PH_DROP) {
            const int k = drop_items_of(m, b);
            if (k > 0) return k;
            phase = PH_DAPPLY;
        }
        if (phase == PH_DONE) return 0;
        return m.n_vox_items;
    }
    return 0;
}

// Reductions of the phase just finished (all threads), then thread 0 sets the next phase
// and publishes it.  items: the finished phase's item count; word: its schedule word.
__device__ void finish_phase(const CycleArgs& a, int r, int phase, int items, unsigned long long word, int tries_done,
                             double* sh) {
    const MemberDev& m = a.mem[r];
    double t0 = 0.0, t1 = 0.0;
    double tt[kSpec];
    int T = 0;
    if (phase == PH_GRAD || phase == PH_PHI) t0 = ordered_sum(a.part + m.part_off, items, 1, sh);
    if (phase == PH_GRAD && m.check) t1 = ordered_sum(a.part2 + m.part_off, items, 1, sh);
    if (phase == PH_TRY) {
        T = min(kSpec, m.max_retries - tries_done);
#pragma unroll
        for (int t = 0; t < kSpec; ++t)
            tt[t] = (t < T) ? ordered_sum(a.part_try + (size_t)m.part_off * kSpec + t, items, kSpec, sh) : 0.0;
    }
    if (threadIdx.x != 0) return;
    if (a.starve && r == 0) return;   // test hook: member 0 never leaves its first phase
    MemberState* st = a.st + r;
    volatile MemberState* vs = st;
    int ph = phase, n = vs->n, b = vs->b;
    switch (phase) {
        case PH_GRAD:
            st->gnorm2 = t0;
            if (m.check) {
                st->phi_x = t1;
                st->tries = 0;
                ph = PH_TRY;
            } else {
                st->sc = step_scale(__ldg(a.beta + (size_t)n * a.R + r), &st->gnorm2);
                st->n_steps += 1;
                st->n_tries += 1;
                if (st->sc != 0.0) st->n_accepted += 1;
                ph = PH_APPLY;
            }
            break;
        case PH_TRY: {
            const double gn2 = vs->gnorm2, px = vs->phi_x;
            int acc = -1;
            for (int t = 0; t < T; ++t)
                if (tt[t] <= px) { acc = t; break; }   // ties accept
            const int64_t ell = vs->ell;
            if (acc >= 0) {
                st->sc = gn2 > 0.0 ? beta_of(m, ell + acc) / sqrt(gn2) : 0.0;
                st->ell = ell + acc + 1;
                st->tries = tries_done + acc + 1;
                st->n_tries += acc + 1;
                st->n_accepted += 1;
                st->n_steps += 1;
                ph = PH_APPLY;
            } else {
                st->ell = ell + T;
                st->tries = tries_done + T;
                st->n_tries += T;
                if (tries_done + T >= m.max_retries) {   // the step is skipped
                    st->n_steps += 1;
                    ph = PH_GRAD;
                    n += 1;
                }
            }
            break;
        }
        case PH_APPLY:
            ph = PH_GRAD;
            n += 1;
            break;
        case PH_DROP:   // the block's next window bound: twice the largest |r / lambda| of this sweep
            if (m.wstat) {
                const float o = __uint_as_float(atomicExch(reinterpret_cast<unsigned*>(m.wstat + 2 * m.B + b), 0u));
                if (o > 0.f) m.wstat[m.B + b] = 2.f * o;
            }
            ph = PH_DAPPLY;
            break;
        case PH_DAPPLY:
            ph = PH_DROP;
            b += 1;
            break;
        case PH_PHI: {
            const int64_t k = vs->k;
            m.tv_hist[k] = t0;
            st->k = k + 1;
            ph = PH_DONE;
            break;
        }
        default:
            break;
    }
    const int nitems = settle(m, ph, n, b);
    st->phase = ph;
    st->n = n;
    st->b = b;
    st->done = 0u;
    __threadfence();
    atomicExch(&st->word, pack_word((unsigned)(word >> 48) + 1u, (unsigned)nitems));
    if (ph == PH_DONE) atomicAdd(&a.run->members_done, 1u);
}

// Start of a cycle (one thread per member): ell_k of checked members, residual sums
// cleared, the first phase published.
__global__ void cycle_setup_kernel(const MemberDev* __restrict__ mem, MemberState* st, RunState* run, int R) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r == 0) run->members_done = 0u;
    if (r >= R) return;
    const MemberDev& m = mem[r];
    MemberState& s = st[r];
    if (m.check && m.rule == NTVS_STEP_NTVS) s.ell = draw_ell(m.seed, s.k, s.ell);
    for (int b = 0; b < m.B; ++b) m.resid[b] = 0.0;
    int ph = PH_GRAD, n = 0, b = 0;
    const int items = settle(m, ph, n, b);
    s.phase = ph;
    s.n = n;
    s.b = b;
    s.tries = 0;
    s.done = 0u;
    s.word = pack_word((unsigned)(s.word >> 48) + 1u, (unsigned)items);
}

// One cycle of every member (see the file comment).  MINB: CTAs per SM the register
// allocation is fitted to (3: no spills; 4: 64 registers, a few spills).
template <int MINB>
__global__ void __launch_bounds__(kThreads, MINB) batch_cycle_kernel(CycleArgs a) {
    __shared__ double sh[32];
    __shared__ int s_r, s_idx, s_items, s_last, s_exit, s_phase, s_b, s_tries;
    __shared__ unsigned long long s_word;
    __shared__ int64_t s_ell;
    __shared__ double s_gnorm2, s_sc;
    const int lane = threadIdx.x & 31;
    int start = blockIdx.x % a.R;
    uint64_t idle0 = 0;
    for (;;) {
        if (threadIdx.x < 32) {   // warp 0 looks for an item, 32 members per probe
            int got = -1, gidx = 0, gitems = 0;
            unsigned long long gword = 0ull;
            for (int base = 0; base < a.R && got < 0; base += 32) {
                int r = start + base + lane;
                if (r >= a.R) r -= a.R;
                bool avail = false;
                if (base + lane < a.R) {
                    const unsigned long long w = ld_word(&a.st[r].word);
                    avail = (w & kM24) < ((w >> 24) & kM24);
                }
                unsigned bal = __ballot_sync(0xffffffffu, avail);
                while (bal != 0u) {
                    const int L = __ffs(bal) - 1;
                    bal &= bal - 1u;
                    const int rr = __shfl_sync(0xffffffffu, r, L);
                    unsigned long long old = 0ull;
                    if (lane == 0) old = atomicAdd(&a.st[rr].word, 1ull);
                    old = __shfl_sync(0xffffffffu, old, 0);
                    const unsigned cur = (unsigned)(old & kM24), n = (unsigned)((old >> 24) & kM24);
                    if (cur < n) {
                        got = rr;
                        gidx = (int)cur;
                        gitems = (int)n;
                        gword = old;
                        break;
                    }
                }
            }
            if (lane == 0) {
                s_r = got;
                s_idx = gidx;
                s_items = gitems;
                s_word = gword;
            }
        }
        __syncthreads();
        const int r = s_r;
        if (r < 0) {   // nothing to take: done, failed, or wait (bounded) for a phase to end
            if (threadIdx.x == 0) {
                int ex = 0;
                if (*(volatile int*)&a.run->err != 0 || *(volatile unsigned*)&a.run->members_done >= (unsigned)a.R) {
                    ex = 1;
                } else {
                    const uint64_t now = globaltimer_ns();
                    if (idle0 == 0) {
                        idle0 = now;
                    } else if (now - idle0 > a.wait_ns) {
                        if (atomicCAS(&a.run->err, 0, kErrBatchStall) == 0) {
                            // the first member that has not finished its cycle, for the report
                            for (int q = 0; q < a.R; ++q)
                                if (((volatile MemberState*)(a.st + q))->phase != PH_DONE) {
                                    a.run->err_member = q;
                                    a.run->err_phase = ((volatile MemberState*)(a.st + q))->phase;
                                    break;
                                }
                        }
                        ex = 1;
                    }
                    if (!ex) __nanosleep(256);
                }
                s_exit = ex;
            }
            __syncthreads();
            if (s_exit) break;
            continue;
        }
        idle0 = 0;
        start = r;
        if (threadIdx.x == 0) {
            __threadfence();
            const volatile MemberState* vs = a.st + r;
            s_phase = vs->phase;
            s_b = vs->b;
            s_tries = vs->tries;
            s_ell = vs->ell;
            s_gnorm2 = vs->gnorm2;
            s_sc = vs->sc;
        }
        __syncthreads();
        const MemberDev& m = a.mem[r];
        const int idx = s_idx, phase = s_phase;
        switch (phase) {
            case PH_GRAD: grad_item(m, idx, a.part, a.part2, sh); break;
            case PH_TRY: try_item(m, idx, s_ell, min(kSpec, m.max_retries - s_tries), s_gnorm2, a.part_try, sh); break;
            case PH_APPLY: apply_item(m, idx, s_sc); break;
            case PH_DROP: drop_item(m, s_b, idx, a.win_cap, sh); break;
            case PH_DAPPLY: dapply_item(m, idx, s_b); break;
            case PH_PHI: phi_item(m, idx, a.part, sh); break;
            default: break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned d = atomicAdd(&a.st[r].done, 1u);
            s_last = (d + 1u == (unsigned)s_items) ? 1 : 0;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            finish_phase(a, r, phase, s_items, s_word, s_tries, sh);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- member preparation

// flags |= 1 row_ptr not non-decreasing from 0 to nnz, 2 column outside [0, V),
// 4 non-finite value, 8 non-finite right-hand side
__global__ void validate_kernel(const int64_t* __restrict__ rp, int64_t M, const int32_t* __restrict__ col,
                                const float* __restrict__ val, int64_t nnz, const float* __restrict__ b, int64_t V,
                                int* flags) {
    int f = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x, t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = t0; i < M; i += stride) {
        if (rp[i] > rp[i + 1]) f |= 1;
        if (!isfinite(b[i])) f |= 8;
    }
    if (t0 == 0 && (rp[0] != 0 || rp[M] != nnz)) f |= 1;
    for (int64_t q = t0; q < nnz; q += stride) {
        const int32_t c = col[q];
        if (c < 0 || (int64_t)c >= V) f |= 2;
        if (!isfinite(val[q])) f |= 4;
    }
    if (f) atomicOr(flags, f);
}

__global__ void remap_kernel(int32_t* __restrict__ col, int64_t nnz, VoxMap vm) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x)
        col[q] = (int32_t)vox_internal(vm, col[q]);
}

// canonical index of internal slot p (the inverse of vox_internal on real voxels)
__device__ __forceinline__ int64_t vox_canonical(const VoxMap& m, int64_t p) {
    if (m.tx == 1 && m.ty == 1 && !m.sw) return p;
    const int64_t iz = p / m.slice_p;
    int64_t rem = p - iz * m.slice_p;
    if (m.sw) rem ^= (rem >> 5) & 31;   // the swizzle is its own inverse
    const int64_t tile = rem >> (m.ltx + m.lty), in = rem & ((1 << (m.ltx + m.lty)) - 1);
    const int64_t ntx = m.nxp >> m.ltx;
    const int64_t ty = tile / ntx, tx = tile - ty * ntx;
    const int64_t ix = (tx << m.ltx) + (in & (m.tx - 1)), iy = (ty << m.lty) + (in >> m.ltx);
    return (iz * m.ny + iy) * m.nx + ix;
}

// the canonical columns and the values of a member's packed entries
__global__ void unmap_kernel(const int2* __restrict__ ent, int32_t* __restrict__ col, float* __restrict__ val,
                             int64_t nnz, VoxMap vm) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x) {
        const int2 e = ent[q];
        if (col) col[q] = (int32_t)vox_canonical(vm, e.x);
        if (val) val[q] = __int_as_float(e.y);
    }
}

// ent[q] = {col[q], bits of val[q]}
__global__ void pack_pairs_kernel(const int32_t* __restrict__ col, const float* __restrict__ val, int64_t nnz,
                                  int2* __restrict__ ent) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x)
        ent[q] = make_int2(col[q], __float_as_int(val[q]));
}

// 1 / ||a_i||^2 (FP64 sum), a warp per row
__global__ void norm_kernel(const int64_t* __restrict__ rp, const float* __restrict__ val, int64_t M,
                            float* __restrict__ inn) {
    const int lane = threadIdx.x & 31;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < M;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        double s = 0.0;
        for (int64_t q = rp[i] + lane; q < rp[i + 1]; q += 32) s += (double)val[q] * (double)val[q];
        s = warp_sum(s);
        if (lane == 0) inn[i] = s > 0.0 ? (float)(1.0 / s) : 0.f;
    }
}

// hit counts of rows [r0, r1): cnt[col] += 1 per nonzero entry (internal order)
__global__ void count_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                             const float* __restrict__ val, int64_t r0, int64_t r1, int32_t* __restrict__ cnt) {
    const int64_t q0 = rp[r0], q1 = rp[r1];
    for (int64_t q = q0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < q1; q += (int64_t)gridDim.x * blockDim.x)
        if (val[q] != 0.f) atomicAdd(cnt + col[q], 1);
}

// The window statistics of one block (rows [r0, r1)), each a non-negative float kept as its
// bits so that an unsigned atomic max orders them: colsum[j] += |a_ij| and *amax = max |a_ij|
__global__ void colsum_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                              const float* __restrict__ val, int64_t r0, int64_t r1, float* __restrict__ colsum,
                              unsigned* __restrict__ amax) {
    const int64_t q0 = rp[r0], q1 = rp[r1];
    unsigned mx = 0u;
    for (int64_t q = q0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < q1; q += (int64_t)gridDim.x * blockDim.x) {
        const float a = fabsf(val[q]);
        if (a != 0.f) atomicAdd(colsum + col[q], a);
        mx = max(mx, __float_as_uint(a));
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(amax, mx);
}

// *out = max(*out, largest of v[0..n)) for non-negative v
__global__ void max_bits_kernel(const float* __restrict__ v, int64_t n, unsigned* __restrict__ out) {
    unsigned mx = 0u;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        mx = max(mx, __float_as_uint(v[j]));
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

// *out = max over rows [r0, r1) of |b_i| / ||a_i||^2: the residual bound at x = 0, the first
// sweep's window bound
__global__ void seed_bound_kernel(const float* __restrict__ b, const float* __restrict__ inn, int64_t r0, int64_t r1,
                                  unsigned* __restrict__ out) {
    unsigned mx = 0u;
    for (int64_t i = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < r1; i += (int64_t)gridDim.x * blockDim.x)
        mx = max(mx, __float_as_uint(fabsf(b[i]) * inn[i]));
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

__global__ void inv_count_kernel(const int32_t* __restrict__ cnt, float* __restrict__ inv_s, int64_t n) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = cnt[p];
        inv_s[p] = c ? (float)(1.0 / (double)c) : 0.f;
    }
}

// image copies from x0 (canonical, F64 or F32)
__global__ void image_init_kernel(const void* __restrict__ x0, int f64, int64_t V, VoxMap vm, double* __restrict__ x,
                                  float* __restrict__ x32, float* __restrict__ xh, float* __restrict__ xl) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < V; j += (int64_t)gridDim.x * blockDim.x) {
        const double v = f64 ? ((const double*)x0)[j] : (double)((const float*)x0)[j];
        x[j] = v;
        const float h = (float)v;
        x32[vox_internal(vm, j)] = h;
        xh[j] = h;
        xl[j] = (float)(v - (double)h);
    }
}

// column range and mean column (internal order) of each DROP item of one block
__global__ void item_range_kernel(const int64_t* __restrict__ rp, const int2* __restrict__ ent, int64_t r0,
                                  int64_t r1, int rows_per_item, int32_t* __restrict__ lo, int32_t* __restrict__ hi,
                                  int32_t* __restrict__ mean) {
    const int it = blockIdx.x;
    const int64_t a = r0 + (int64_t)it * rows_per_item, e = min(r1, a + rows_per_item);
    int mn = INT32_MAX, mx = -1;
    long long sum = 0;
    for (int64_t q = rp[a] + threadIdx.x; q < rp[e]; q += blockDim.x) {
        const int c = ent[q].x;
        mn = min(mn, c);
        mx = max(mx, c);
        sum += c;
    }
    for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
    }
    __shared__ int smn[32], smx[32];
    __shared__ long long ssum[32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { smn[w] = mn; smx[w] = mx; ssum[w] = sum; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) { mn = min(mn, smn[q]); mx = max(mx, smx[q]); sum += ssum[q]; }
        const int64_t n = rp[e] - rp[a];
        lo[it] = mn;
        hi[it] = mx;
        mean[it] = n > 0 ? (int32_t)(sum / n) : -1;
    }
}

// window start of each item for a window of cap floats: lo when all of the item's columns
// fit; otherwise the window centred on the item's mean column, clamped to [0, vint - cap]
// (the item's other entries go to global memory); -1 without entries or without a window
__global__ void window_kernel(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                              const int32_t* __restrict__ mean, int n, int cap, int64_t vint,
                              int32_t* __restrict__ win) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int32_t w = -1;
        if (cap > 0 && hi[i] >= lo[i]) {
            if (hi[i] - lo[i] < cap) {
                w = lo[i];
            } else {
                const int64_t top = vint > cap ? vint - cap : 0;
                w = (int32_t)max((int64_t)0, min(top, (int64_t)mean[i] - cap / 2));
            }
        }
        win[i] = w;
    }
}

}  // namespace
}  // namespace ntvs

// ------------------------------------------------------------------ host side
namespace ntvs {
namespace {

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

int grid_of(int64_t n, int threads = 256) {
    const int64_t g = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
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
        int64_t M = 0, nnz = 0, k = 0, ell_prev = 0;   // k, ell_prev: host schedule (no TV check)
        std::vector<void*> owned;
        int32_t* item_lo = nullptr;   // [n_drop_items] column range of each DROP item
        int32_t* item_hi = nullptr;
        int32_t* item_mean = nullptr;
        int32_t* win = nullptr;
        int32_t* item0 = nullptr;     // [B]
        int n_drop_items = 0;
        int lpr_own = 32;             // lanes per row from the member's mean row length
    };
    std::vector<Member> m;
    MemberDev* dmem = nullptr;
    MemberState* dst = nullptr;
    RunState* drun = nullptr;
    double* part = nullptr;
    double* part2 = nullptr;
    double* part_try = nullptr;
    double* beta = nullptr;          // [N_max][R]
    double* hbeta[2] = {nullptr, nullptr};
    int N_max = 0;
    int total_vox_items = 0;
    int64_t tv_cap = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    cudaEvent_t used[2] = {nullptr, nullptr};
    int next = 0;
    int64_t launches = 0, cycles = 0;
    // schedule of the persistent kernel (fixed by the caller or tuned at finalize)
    int grid = 0, win_cap = -1, rows_per_item = 0, minb = 3;
    int req_rows = 0, req_win = -1;
    uint64_t wait_ns = 2000000000ull;
    int hook = 0;
    std::vector<int32_t> tune_cand;   // (rows per item, window floats, CTAs per SM, lanes per row) per
                                      // timed candidate; lanes per row 0: each member's own (from its rows)
    std::vector<float> tune_ms;       // its cycle time
    int lpr_policy = 0;               // lanes per row of every member, 0: each member's own
};

namespace {

void free_member(ntvs_batch::Member& mm) {
    for (void* q : mm.owned) cudaFree(q);
    mm.owned.clear();
}

int member_alloc(ntvs_batch::Member& mm, void** dst, size_t bytes, const char* what) {
    BTRY(balloc(dst, bytes, what));
    mm.owned.push_back(*dst);
    return NTVS_OK;
}

// frees one of the member's buffers before the member is destroyed
void member_release(ntvs_batch::Member& mm, const void* q) {
    for (size_t i = 0; i < mm.owned.size(); ++i)
        if (mm.owned[i] == q) {
            cudaFree(mm.owned[i]);
            mm.owned.erase(mm.owned.begin() + (long)i);
            return;
        }
}

// lanes per row: the smallest LPR whose register-held entries (LPR x CH) cover 1.15x the
// member's mean row length
int pick_lpr(int64_t M, int64_t nnz) {
    const double mean = M > 0 ? (double)nnz / (double)M : 0.0;
    if (1.15 * mean <= 8 * 16) return 8;
    if (1.15 * mean <= 16 * 10) return 16;
    return 32;
}

int check_params(const ntvs_params* p) {
    if (p->N < 0 || !(p->alpha > 0 && p->alpha < 1) || !(p->beta0 >= 0) || !(p->eps_tv >= 0) || !(p->lambda == p->lambda))
        return bfail(NTVS_ERR_ARG, "bad parameters");
    if (p->step_rule < NTVS_STEP_NTVS || p->step_rule > NTVS_STEP_DECOUPLED)
        return bfail(NTVS_ERR_ARG, "unknown step_rule");
    if (p->step_rule == NTVS_STEP_DECOUPLED && !(p->gamma > 0 && p->gamma < 1))
        return bfail(NTVS_ERR_ARG, "gamma must lie in (0, 1)");
    if (p->tv_check && p->step_rule == NTVS_STEP_DECOUPLED)
        return bfail(NTVS_ERR_ARG, "the decoupled rule is defined without the TV check");
    if (p->tv_check && p->max_retries < 1) return bfail(NTVS_ERR_ARG, "max_retries must be >= 1");
    return NTVS_OK;
}

int plan_blocks(const int64_t* block_ptr, int n_blocks, int64_t M, std::vector<int64_t>& bp) {
    bp.clear();
    if (block_ptr) {
        if (n_blocks < 1) return bfail(NTVS_ERR_ARG, "n_blocks must be >= 1");
        bp.assign(block_ptr, block_ptr + n_blocks + 1);
        if (bp.front() != 0 || bp.back() != M) return bfail(NTVS_ERR_ARG, "block_ptr must run from 0 to n_rows");
        for (int t = 0; t < n_blocks; ++t)
            if (bp[t] > bp[t + 1]) return bfail(NTVS_ERR_ARG, "block_ptr decreases");
    } else {
        if (n_blocks < 1) return bfail(NTVS_ERR_ARG, "n_blocks must be >= 1");
        const int64_t per = (M + n_blocks - 1) / n_blocks;
        for (int t = 0; t <= n_blocks; ++t) bp.push_back(std::min<int64_t>((int64_t)t * per, M));
    }
    return NTVS_OK;
}

// Everything after the rows are on the device in internal column order: norms, per-block
// hit counts, block table, image copies, scratch.
int member_prep(ntvs_batch* bt, ntvs_batch::Member& mm, const void* x0, int x0_dtype, int x0_mem) {
    MemberDev& d = mm.d;
    cudaStream_t s = bt->stream;
    const int64_t M = mm.M, nnz = mm.nnz, V = d.V, VI = d.vm.vint;
    const int B = (int)mm.block_ptr.size() - 1;
    BTRY(member_alloc(mm, (void**)&d.inv_norm2, sizeof(float) * std::max<int64_t>(M, 1), "inv_norm2"));
    BTRY(member_alloc(mm, (void**)&d.inv_s, sizeof(float) * (size_t)B * VI, "inv_s"));
    BTRY(member_alloc(mm, (void**)&d.block_ptr, sizeof(int64_t) * (B + 1), "block_ptr"));
    BTRY(member_alloc(mm, (void**)&d.x, sizeof(double) * V, "x"));
    BTRY(member_alloc(mm, (void**)&d.x32, sizeof(float) * VI, "x32"));
    BTRY(member_alloc(mm, (void**)&d.xh, sizeof(float) * V, "xh"));
    BTRY(member_alloc(mm, (void**)&d.xl, sizeof(float) * V, "xl"));
    BTRY(member_alloc(mm, (void**)&d.delta, sizeof(float) * VI, "delta"));
    BTRY(member_alloc(mm, (void**)&d.g, sizeof(float) * V, "g"));
    BTRY(member_alloc(mm, (void**)&d.resid, sizeof(double) * B, "resid"));
    BCUDA(cudaMemcpyAsync((void*)d.block_ptr, mm.block_ptr.data(), sizeof(int64_t) * (B + 1), cudaMemcpyHostToDevice, s));
    if (M > 0) norm_kernel<<<grid_of(M * 32), 256, 0, s>>>(d.row_ptr, d.val, M, (float*)d.inv_norm2);
    int32_t* cnt = nullptr;
    BTRY(balloc(&cnt, sizeof(int32_t) * VI, "hit counts"));
    BTRY(member_alloc(mm, (void**)&d.wstat, sizeof(float) * 4 * (size_t)B, "window statistics"));
    cudaMemsetAsync(d.wstat, 0, sizeof(float) * 4 * (size_t)B, s);
    for (int t = 0; t < B; ++t) {
        cudaMemsetAsync(cnt, 0, sizeof(int32_t) * VI, s);
        if (mm.block_ptr[t + 1] > mm.block_ptr[t]) {
            count_kernel<<<grid_of(nnz), 256, 0, s>>>(d.row_ptr, d.col, d.val, mm.block_ptr[t], mm.block_ptr[t + 1], cnt);
            // the window statistics: column sums of |a| into the (reused) count buffer as floats
            inv_count_kernel<<<grid_of(VI), 256, 0, s>>>(cnt, (float*)d.inv_s + (size_t)t * VI, VI);
            cudaMemsetAsync(cnt, 0, sizeof(int32_t) * VI, s);
            unsigned* w = reinterpret_cast<unsigned*>(d.wstat);
            colsum_kernel<<<grid_of(nnz), 256, 0, s>>>(d.row_ptr, d.col, d.val, mm.block_ptr[t], mm.block_ptr[t + 1],
                                                       reinterpret_cast<float*>(cnt), w + 3 * B + t);
            max_bits_kernel<<<grid_of(VI), 256, 0, s>>>(reinterpret_cast<const float*>(cnt), VI, w + t);
            seed_bound_kernel<<<grid_of(mm.block_ptr[t + 1] - mm.block_ptr[t]), 256, 0, s>>>(
                d.b, d.inv_norm2, mm.block_ptr[t], mm.block_ptr[t + 1], w + B + t);
        } else {
            inv_count_kernel<<<grid_of(VI), 256, 0, s>>>(cnt, (float*)d.inv_s + (size_t)t * VI, VI);
        }
    }
    // x0 on the device (copied when it is host memory)
    const size_t xb = (x0_dtype == NTVS_F64 ? sizeof(double) : sizeof(float)) * (size_t)V;
    void* xdev = (void*)x0;
    void* xtmp = nullptr;
    if (x0_mem == NTVS_MEM_HOST) {
        cudaError_t e = cudaMalloc(&xtmp, xb);
        if (e != cudaSuccess) {
            cudaFree(cnt);
            return bfail(NTVS_ERR_OOM, "batch: x0 staging");
        }
        cudaMemcpyAsync(xtmp, x0, xb, cudaMemcpyHostToDevice, s);
        xdev = xtmp;
    }
    cudaMemsetAsync(d.x32, 0, sizeof(float) * VI, s);
    image_init_kernel<<<grid_of(V), 256, 0, s>>>(xdev, x0_dtype == NTVS_F64 ? 1 : 0, V, d.vm, d.x, d.x32, d.xh, d.xl);
    cudaMemsetAsync(d.delta, 0, sizeof(float) * VI, s);
    cudaMemsetAsync(d.resid, 0, sizeof(double) * B, s);
    cudaError_t e = cudaGetLastError();
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(cnt);
    if (xtmp) cudaFree(xtmp);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return bfail(NTVS_ERR_CUDA, std::string("batch member preparation: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    // the entries as {column, value} pairs (one 8-byte load each in the DROP items); the
    // separate arrays are released
    BTRY(member_alloc(mm, (void**)&d.ent, sizeof(int2) * (size_t)std::max<int64_t>(nnz, 1), "packed entries"));
    if (nnz > 0) pack_pairs_kernel<<<grid_of(nnz), 256, 0, s>>>(d.col, d.val, nnz, (int2*)d.ent);
    e = cudaGetLastError();
    e2 = cudaStreamSynchronize(s);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return bfail(NTVS_ERR_CUDA, std::string("batch entry packing: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    member_release(mm, d.col);
    member_release(mm, d.val);
    d.col = nullptr;
    d.val = nullptr;
    d.B = B;
    d.lpr = pick_lpr(M, nnz);
    mm.lpr_own = d.lpr;
    return NTVS_OK;
}

void set_member_params(ntvs_batch::Member& mm, int nx, int ny, int nz, const ntvs_params* p) {
    MemberDev& d = mm.d;
    d.nx = nx; d.ny = ny; d.nz = nz;
    d.V = (int64_t)nx * ny * nz;
    d.N = p->N;
    d.lambda = (float)p->lambda;
    d.eps = (float)p->eps_tv;
    d.beta0 = p->beta0;
    d.alpha = p->alpha;
    d.check = p->tv_check ? 1 : 0;
    d.max_retries = p->tv_check ? p->max_retries : 1;
    d.rule = p->step_rule;
    d.seed = p->seed;
    d.vm = make_voxmap(nx, ny, nz, 4, 4);
    if (d.vm.vint > 0x7fffffffLL) d.vm = make_voxmap(nx, ny, nz, 1, 1);
    mm.p = *p;
}

int common_checks(ntvs_batch* bt, const ntvs_params* p, int nx, int ny, int nz, int x0_dtype, int x0_mem) {
    if (bt->finalized) return bfail(NTVS_ERR_STATE, "batch already finalized");
    BTRY(check_params(p));
    if (nx < 1 || ny < 1 || nz < 1) return bfail(NTVS_ERR_ARG, "bad sizes");
    if ((int64_t)nx * ny * nz > 0x7fffffffLL) return bfail(NTVS_ERR_ARG, "V too large");
    if (x0_dtype != NTVS_F64 && x0_dtype != NTVS_F32) return bfail(NTVS_ERR_ARG, "x0 dtype must be F64 or F32");
    if (x0_mem != NTVS_MEM_HOST && x0_mem != NTVS_MEM_DEVICE) return bfail(NTVS_ERR_ARG, "bad x0 memory kind");
    return NTVS_OK;
}

// Item tables of every member for a number of rows per item, and the windows for cap.
int build_items(ntvs_batch* bt, int rows_per_item, int cap) {
    cudaStream_t s = bt->stream;
    for (auto& mm : bt->m) {
        MemberDev& d = mm.d;
        const int B = d.B;
        std::vector<int32_t> item0(B);
        int n = 0;
        for (int t = 0; t < B; ++t) {
            item0[t] = n;
            n += (int)((mm.block_ptr[t + 1] - mm.block_ptr[t] + rows_per_item - 1) / rows_per_item);
        }
        if (mm.item_lo) {
            cudaFree(mm.item_lo); cudaFree(mm.item_hi); cudaFree(mm.item_mean); cudaFree(mm.win); cudaFree(mm.item0);
        }
        mm.item_lo = mm.item_hi = mm.item_mean = mm.win = mm.item0 = nullptr;
        BTRY(balloc(&mm.item_lo, sizeof(int32_t) * std::max(n, 1), "item ranges"));
        BTRY(balloc(&mm.item_hi, sizeof(int32_t) * std::max(n, 1), "item ranges"));
        BTRY(balloc(&mm.item_mean, sizeof(int32_t) * std::max(n, 1), "item ranges"));
        BTRY(balloc(&mm.win, sizeof(int32_t) * std::max(n, 1), "item windows"));
        BTRY(balloc(&mm.item0, sizeof(int32_t) * std::max(B, 1), "item table"));
        BCUDA(cudaMemcpyAsync(mm.item0, item0.data(), sizeof(int32_t) * B, cudaMemcpyHostToDevice, s));
        for (int t = 0; t < B; ++t) {
            const int k = (t + 1 < B ? item0[t + 1] : n) - item0[t];
            if (k > 0)
                item_range_kernel<<<k, 256, 0, s>>>(d.row_ptr, d.ent, mm.block_ptr[t], mm.block_ptr[t + 1], rows_per_item,
                                                    mm.item_lo + item0[t], mm.item_hi + item0[t],
                                                    mm.item_mean + item0[t]);
        }
        if (n > 0)
            window_kernel<<<grid_of(n), 256, 0, s>>>(mm.item_lo, mm.item_hi, mm.item_mean, n, cap, d.vm.vint, mm.win);
        mm.n_drop_items = n;
        d.rows_per_item = rows_per_item;
        d.win_lo = mm.win;
        d.item0 = mm.item0;
    }
    std::vector<MemberDev> md;
    for (auto& mm : bt->m) md.push_back(mm.d);
    BCUDA(cudaMemcpyAsync(bt->dmem, md.data(), sizeof(MemberDev) * md.size(), cudaMemcpyHostToDevice, s));
    BCUDA(cudaStreamSynchronize(s));
    BCUDA(cudaGetLastError());
    return NTVS_OK;
}

CycleArgs cycle_args(ntvs_batch* bt, bool hooks) {
    CycleArgs a;
    a.mem = bt->dmem;
    a.st = bt->dst;
    a.run = bt->drun;
    a.R = (int)bt->m.size();
    a.part = bt->part;
    a.part2 = bt->part2;
    a.part_try = bt->part_try;
    a.beta = bt->beta;
    a.wait_ns = bt->wait_ns;
    a.starve = hooks && (bt->hook & NTVS_HOOK_STARVE_BATCH) ? 1 : 0;
    a.win_cap = bt->win_cap;
    return a;
}

int launch_cycle(ntvs_batch* bt, const double* beta_src, bool hooks) {
    cudaStream_t s = bt->stream;
    const int R = (int)bt->m.size();
    BCUDA(cudaMemcpyAsync(bt->beta, beta_src, sizeof(double) * (size_t)std::max(bt->N_max, 1) * R,
                          cudaMemcpyHostToDevice, s));
    cycle_setup_kernel<<<(R + 127) / 128, 128, 0, s>>>(bt->dmem, bt->dst, bt->drun, R);
    const size_t smem = sizeof(float) * (size_t)bt->win_cap;
    if (bt->minb == 4) batch_cycle_kernel<4><<<bt->grid, kThreads, smem, s>>>(cycle_args(bt, hooks));
    else batch_cycle_kernel<3><<<bt->grid, kThreads, smem, s>>>(cycle_args(bt, hooks));
    BCUDA(cudaGetLastError());
    return NTVS_OK;
}

// beta_{k,n} of the next cycle of every member without the TV check (host ell schedule)
void fill_betas(ntvs_batch* bt, double* hb, bool advance) {
    const int R = (int)bt->m.size();
    for (int r = 0; r < R; ++r) {
        auto& mm = bt->m[r];
        const int64_t k = mm.k;
        int64_t ell = mm.p.tv_check ? 0 : cycle_ell(mm.p, k, mm.ell_prev);
        const int64_t adv = ell_advances(mm.p) ? 1 : 0;
        for (int n = 0; n < std::max(bt->N_max, 1); ++n) {
            hb[(size_t)n * R + r] = (!mm.p.tv_check && n < mm.p.N) ? step_beta(mm.p, k, n, ell) : 0.0;
            if (!mm.p.tv_check && n < mm.p.N) ell += adv;
        }
        if (advance) {
            if (!mm.p.tv_check && adv) mm.ell_prev = ell;
            mm.k = k + 1;
        }
    }
}

int device_error(ntvs_batch* bt) {
    RunState rs;
    BCUDA(cudaMemcpyAsync(&rs, bt->drun, sizeof(RunState), cudaMemcpyDeviceToHost, bt->stream));
    BCUDA(cudaStreamSynchronize(bt->stream));
    if (rs.err != 0)
        return bfail(NTVS_ERR_TIMEOUT, "batch: an idle CTA's bounded wait ran out (member " +
                                           std::to_string(rs.err_member) + " stopped in phase " +
                                           std::to_string(rs.err_phase) + "); the batch's images are undefined");
    return NTVS_OK;
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
    for (auto& mm : bt->m) {
        free_member(mm);
        cudaFree(mm.item_lo);
        cudaFree(mm.item_hi);
        cudaFree(mm.item_mean);
        cudaFree(mm.win);
        cudaFree(mm.item0);
    }
    cudaFree(bt->dmem);
    cudaFree(bt->dst);
    cudaFree(bt->drun);
    cudaFree(bt->part);
    cudaFree(bt->part2);
    cudaFree(bt->part_try);
    cudaFree(bt->beta);
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
    BTRY(common_checks(bt, p, s->nx, s->ny, s->nz, x0_dtype, x0_mem));
    BCUDA(cudaSetDevice(bt->device));
    if (s->val_dtype != NTVS_F32 || s->storage != NTVS_CSR32)
        return bfail(NTVS_ERR_ARG, "batched members take FP32 values in CSR32 storage");
    if (s->n_rows < 0) return bfail(NTVS_ERR_ARG, "n_rows < 0");
    if (s->mem_kind != NTVS_MEM_HOST && s->mem_kind != NTVS_MEM_DEVICE) return bfail(NTVS_ERR_ARG, "bad mem_kind");
    if (!s->row_ptr || (s->n_rows > 0 && !s->b)) return bfail(NTVS_ERR_ARG, "null row_ptr or b");
    ntvs_batch::Member mm;
    set_member_params(mm, s->nx, s->ny, s->nz, p);
    const int64_t M = s->n_rows;
    mm.M = M;
    const cudaMemcpyKind kind = s->mem_kind == NTVS_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    int64_t nnz = 0;
    if (s->mem_kind == NTVS_MEM_HOST) nnz = s->row_ptr[M];
    else BCUDA(cudaMemcpy(&nnz, s->row_ptr + M, sizeof(int64_t), cudaMemcpyDeviceToHost));
    if (nnz < 0) return bfail(NTVS_ERR_CSR, "row_ptr[M] < 0");
    if (nnz > 0 && (!s->col || !s->val)) return bfail(NTVS_ERR_ARG, "null col or val");
    mm.nnz = nnz;
    int rc = plan_blocks(s->block_ptr, s->n_blocks, M, mm.block_ptr);
    if (rc != NTVS_OK) return rc;
    MemberDev& d = mm.d;
    int* flags = nullptr;
    cudaStream_t st = bt->stream;
    if ((rc = member_alloc(mm, (void**)&d.row_ptr, sizeof(int64_t) * (M + 1), "row_ptr")) ||
        (rc = member_alloc(mm, (void**)&d.col, sizeof(int32_t) * std::max<int64_t>(nnz, 1), "col")) ||
        (rc = member_alloc(mm, (void**)&d.val, sizeof(float) * std::max<int64_t>(nnz, 1), "val")) ||
        (rc = member_alloc(mm, (void**)&d.b, sizeof(float) * std::max<int64_t>(M, 1), "b")) ||
        (rc = balloc(&flags, sizeof(int), "flags"))) {
        free_member(mm);
        return rc;
    }
    cudaMemsetAsync(flags, 0, sizeof(int), st);
    cudaMemcpyAsync((void*)d.row_ptr, s->row_ptr, sizeof(int64_t) * (M + 1), kind, st);
    if (nnz > 0) {
        cudaMemcpyAsync((void*)d.col, s->col, sizeof(int32_t) * nnz, kind, st);
        cudaMemcpyAsync((void*)d.val, s->val, sizeof(float) * nnz, kind, st);
    }
    if (M > 0) cudaMemcpyAsync((void*)d.b, s->b, sizeof(float) * M, kind, st);
    validate_kernel<<<grid_of(std::max(M, nnz)), 256, 0, st>>>(d.row_ptr, M, d.col, d.val, nnz, d.b, d.V, flags);
    int hf = 0;
    cudaMemcpyAsync(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(flags);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        free_member(mm);
        return bfail(NTVS_ERR_CUDA, std::string("batch: copying or validating the system: ") + cudaGetErrorString(e));
    }
    if (hf) {
        free_member(mm);
        return bfail(NTVS_ERR_CSR, (hf & 1) ? "row_ptr must run non-decreasing from 0 to nnz"
                                   : (hf & 2) ? "column outside [0, V)"
                                   : (hf & 4) ? "non-finite value" : "non-finite right-hand side");
    }
    if (nnz > 0) remap_kernel<<<grid_of(nnz), 256, 0, st>>>((int32_t*)d.col, nnz, d.vm);
    if ((rc = member_prep(bt, mm, x0, x0_dtype, x0_mem)) != NTVS_OK) {
        free_member(mm);
        return rc;
    }
    bt->m.push_back(std::move(mm));
    if (index) *index = (int)bt->m.size() - 1;
    return NTVS_OK;
}

int ntvs_batch_add_paths(ntvs_batch* bt, const ntvs_paths* p, const ntvs_params* prm, const void* x0, int x0_dtype,
                         int x0_mem, int* index) {
    if (!bt || !p || !prm || !x0) return bfail(NTVS_ERR_ARG, "null argument");
    BTRY(common_checks(bt, prm, p->nx, p->ny, p->nz, x0_dtype, x0_mem));
    BCUDA(cudaSetDevice(bt->device));
    if (p->n_rows < 0 || p->n_seg < 1 || p->n_seg > 64 || !(p->min_len >= 0) || !(p->dx > 0) || !(p->dy > 0) ||
        !(p->dz > 0))
        return bfail(NTVS_ERR_ARG, "bad path geometry");
    if (p->mem_kind != NTVS_MEM_HOST && p->mem_kind != NTVS_MEM_DEVICE) return bfail(NTVS_ERR_ARG, "bad mem_kind");
    if (p->n_rows > 0 && (!p->paths || !p->b)) return bfail(NTVS_ERR_ARG, "null paths or b");
    ntvs_batch::Member mm;
    set_member_params(mm, p->nx, p->ny, p->nz, prm);
    const int64_t M = p->n_rows;
    mm.M = M;
    int rc = plan_blocks(p->block_ptr, p->n_blocks, M, mm.block_ptr);
    if (rc != NTVS_OK) return rc;
    MemberDev& d = mm.d;
    cudaStream_t st = bt->stream;
    const cudaMemcpyKind kind = p->mem_kind == NTVS_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    // the path records on the device (borrowed when they already are), b copied
    float* paths = (float*)p->paths;
    float* ptmp = nullptr;
    int* flags = nullptr;
    int32_t* nrow = nullptr;
    auto cleanup = [&]() {
        if (ptmp) cudaFree(ptmp);
        if (flags) cudaFree(flags);
        if (nrow) cudaFree(nrow);
    };
    if ((rc = member_alloc(mm, (void**)&d.b, sizeof(float) * std::max<int64_t>(M, 1), "b")) ||
        (rc = member_alloc(mm, (void**)&d.row_ptr, sizeof(int64_t) * (M + 1), "row_ptr")) ||
        (rc = balloc(&flags, sizeof(int), "flags")) ||
        (rc = balloc(&nrow, sizeof(int32_t) * std::max<int64_t>(M, 1), "row lengths"))) {
        cleanup();
        free_member(mm);
        return rc;
    }
    if (p->mem_kind == NTVS_MEM_HOST && M > 0) {
        if ((rc = balloc(&ptmp, sizeof(float) * 10 * (size_t)M, "path staging")) != NTVS_OK) {
            cleanup();
            free_member(mm);
            return rc;
        }
        cudaMemcpyAsync(ptmp, p->paths, sizeof(float) * 10 * (size_t)M, cudaMemcpyHostToDevice, st);
        paths = ptmp;
    }
    if (M > 0) cudaMemcpyAsync((void*)d.b, p->b, sizeof(float) * M, kind, st);
    cudaMemsetAsync(flags, 0, sizeof(int), st);
    OtfArgs oa;
    oa.paths = paths;
    oa.b = d.b;
    oa.M = M;
    oa.nx = p->nx; oa.ny = p->ny; oa.nz = p->nz;
    oa.dx = p->dx; oa.dy = p->dy; oa.dz = p->dz;
    oa.n_seg = p->n_seg;
    oa.min_len = (float)p->min_len;
    oa.grid = grid_of(M, 128);
    oa.vm = d.vm;   // rows traced straight into the internal voxel order
    k_otf_validate(oa, flags, st);
    k_otf_count_rows(oa, nrow, st);
    int hf = 0;
    std::vector<int32_t> lens((size_t)M);
    cudaMemcpyAsync(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (M > 0) cudaMemcpyAsync(lens.data(), nrow, sizeof(int32_t) * M, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        cleanup();
        free_member(mm);
        return bfail(NTVS_ERR_CUDA, std::string("batch: tracing the paths: ") + cudaGetErrorString(e));
    }
    if (hf) {
        cleanup();
        free_member(mm);
        return bfail(NTVS_ERR_CSR, (hf & 32) ? "non-finite path value" : "non-finite right-hand side");
    }
    std::vector<int64_t> rp((size_t)M + 1, 0);
    for (int64_t i = 0; i < M; ++i) rp[i + 1] = rp[i] + lens[i];
    const int64_t nnz = rp[M];
    mm.nnz = nnz;
    if ((rc = member_alloc(mm, (void**)&d.col, sizeof(int32_t) * std::max<int64_t>(nnz, 1), "col")) ||
        (rc = member_alloc(mm, (void**)&d.val, sizeof(float) * std::max<int64_t>(nnz, 1), "val"))) {
        cleanup();
        free_member(mm);
        return rc;
    }
    cudaMemcpyAsync((void*)d.row_ptr, rp.data(), sizeof(int64_t) * (M + 1), cudaMemcpyHostToDevice, st);
    k_otf_fill_rows(oa, d.row_ptr, (int32_t*)d.col, (float*)d.val, st);
    e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        free_member(mm);
        return bfail(NTVS_ERR_CUDA, std::string("batch: writing the traced rows: ") + cudaGetErrorString(e));
    }
    if ((rc = member_prep(bt, mm, x0, x0_dtype, x0_mem)) != NTVS_OK) {
        free_member(mm);
        return rc;
    }
    bt->m.push_back(std::move(mm));
    if (index) *index = (int)bt->m.size() - 1;
    return NTVS_OK;
}

int ntvs_batch_set_schedule(ntvs_batch* bt, int rows_per_item, int window_floats) {
    if (!bt) return bfail(NTVS_ERR_ARG, "null batch");
    if (bt->finalized) return bfail(NTVS_ERR_STATE, "batch already finalized");
    if (rows_per_item < 0 || rows_per_item > (1 << 20)) return bfail(NTVS_ERR_ARG, "rows_per_item out of range");
    if (window_floats < -1 || window_floats > 49152) return bfail(NTVS_ERR_ARG, "window_floats out of range");
    bt->req_rows = rows_per_item;
    bt->req_win = window_floats;
    return NTVS_OK;
}

int ntvs_batch_set_fault_hook(ntvs_batch* bt, int64_t wait_ns, int flags) {
    if (!bt) return bfail(NTVS_ERR_ARG, "null batch");
    if (bt->finalized) return bfail(NTVS_ERR_STATE, "set the hook before ntvs_batch_finalize");
    if (flags & ~NTVS_HOOK_STARVE_BATCH) return bfail(NTVS_ERR_ARG, "unknown hook flags");
    if (wait_ns < 0) return bfail(NTVS_ERR_ARG, "wait_ns < 0");
    bt->wait_ns = wait_ns > 0 ? (uint64_t)wait_ns : 2000000000ull;
    bt->hook = flags;
    return NTVS_OK;
}

int ntvs_batch_finalize(ntvs_batch* bt, int max_cycles) {
    if (!bt) return bfail(NTVS_ERR_ARG, "null batch");
    if (bt->finalized) return bfail(NTVS_ERR_STATE, "batch already finalized");
    if (bt->m.empty()) return bfail(NTVS_ERR_STATE, "empty batch");
    if (max_cycles < 1) return bfail(NTVS_ERR_ARG, "max_cycles must be >= 1");
    BCUDA(cudaSetDevice(bt->device));
    const int R = (int)bt->m.size();
    if (R > (1 << 20)) return bfail(NTVS_ERR_ARG, "too many members");
    cudaStream_t s = bt->stream;
    constexpr int kTrialCycles = 2;   // per tuning candidate: one warm-up, one timed
    bt->tv_cap = max_cycles;
    bt->N_max = 0;
    int off = 0;
    for (auto& mm : bt->m) {
        MemberDev& d = mm.d;
        d.n_vox_items = (int)((d.V + kTvItem - 1) / kTvItem);
        if ((int64_t)d.n_vox_items > (int64_t)(kM24 >> 1)) return bfail(NTVS_ERR_ARG, "member too large");
        d.part_off = off;
        off += d.n_vox_items;
        bt->N_max = std::max(bt->N_max, d.N);
        BTRY(member_alloc(mm, (void**)&d.tv_hist, sizeof(double) * (size_t)(max_cycles + kTrialCycles), "tv history"));
        if (d.check) {
            std::vector<double> tab(kBetaTab);
            for (int l = 0; l < kBetaTab; ++l) tab[l] = mm.p.beta0 * std::pow(mm.p.alpha, (double)l);
            BTRY(member_alloc(mm, (void**)&d.beta_tab, sizeof(double) * kBetaTab, "beta table"));
            BCUDA(cudaMemcpy((void*)d.beta_tab, tab.data(), sizeof(double) * kBetaTab, cudaMemcpyHostToDevice));
        }
    }
    bt->total_vox_items = off;
    BTRY(balloc(&bt->dmem, sizeof(MemberDev) * R, "member table"));
    BTRY(balloc(&bt->dst, sizeof(MemberState) * R, "member states"));
    BTRY(balloc(&bt->drun, sizeof(RunState), "run state"));
    BTRY(balloc(&bt->part, sizeof(double) * off, "partials"));
    BTRY(balloc(&bt->part2, sizeof(double) * off, "partials"));
    BTRY(balloc(&bt->part_try, sizeof(double) * off * kSpec, "partials"));
    BTRY(balloc(&bt->beta, sizeof(double) * std::max(bt->N_max, 1) * R, "beta table"));
    BCUDA(cudaMemset(bt->dst, 0, sizeof(MemberState) * R));
    BCUDA(cudaMemset(bt->drun, 0, sizeof(RunState)));
    for (int j = 0; j < 2; ++j) {
        BCUDA(cudaHostAlloc((void**)&bt->hbeta[j], sizeof(double) * std::max(bt->N_max, 1) * R, cudaHostAllocDefault));
        std::memset(bt->hbeta[j], 0, sizeof(double) * std::max(bt->N_max, 1) * R);
        BCUDA(cudaEventCreateWithFlags(&bt->used[j], cudaEventDisableTiming));
    }
    int sms = 0;
    BCUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, bt->device));
    BCUDA(cudaFuncSetAttribute(batch_cycle_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 49152 * 4));
    BCUDA(cudaFuncSetAttribute(batch_cycle_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 49152 * 4));
    auto set_grid = [&](int cap, int minb) -> int {
        int per = 0;
        if (minb == 4)
            BCUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_cycle_kernel<4>, kThreads, sizeof(float) * cap));
        else
            BCUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_cycle_kernel<3>, kThreads, sizeof(float) * cap));
        if (per < 1) return bfail(NTVS_ERR_CUDA, "batch: the persistent kernel does not fit on an SM");
        bt->grid = per * sms;
        bt->minb = minb;
        return NTVS_OK;
    };
    // schedule: fixed by the caller, else timed over kTrialCycles cycles per candidate
    // (images and schedule state saved before and restored after)
    std::vector<int> rows_c = bt->req_rows > 0 ? std::vector<int>{bt->req_rows} : std::vector<int>{256, 512, 1024};
    std::vector<int> win_c = bt->req_win >= 0 ? std::vector<int>{bt->req_win} : std::vector<int>{0, 8192, 12288, 16384};
    std::vector<int> minb_c = (bt->req_rows > 0 && bt->req_win >= 0) ? std::vector<int>{3} : std::vector<int>{3, 4};
    if (rows_c.size() * win_c.size() * minb_c.size() == 1) {
        bt->rows_per_item = rows_c[0];
        bt->win_cap = win_c[0];
        bt->minb = minb_c[0];
    } else {
        std::vector<void*> saved;
        auto save = [&](const void* src, size_t bytes) -> int {
            void* q = nullptr;
            BTRY(balloc(&q, bytes, "tuning snapshot"));
            saved.push_back(q);
            BCUDA(cudaMemcpyAsync(q, src, bytes, cudaMemcpyDeviceToDevice, s));
            return NTVS_OK;
        };
        auto restore = [&]() -> int {
            size_t i = 0;
            for (auto& mm : bt->m) {
                const MemberDev& d = mm.d;
                BCUDA(cudaMemcpyAsync(d.x, saved[i++], sizeof(double) * d.V, cudaMemcpyDeviceToDevice, s));
                BCUDA(cudaMemcpyAsync(d.x32, saved[i++], sizeof(float) * d.vm.vint, cudaMemcpyDeviceToDevice, s));
                BCUDA(cudaMemcpyAsync(d.xh, saved[i++], sizeof(float) * d.V, cudaMemcpyDeviceToDevice, s));
                BCUDA(cudaMemcpyAsync(d.xl, saved[i++], sizeof(float) * d.V, cudaMemcpyDeviceToDevice, s));
            }
            BCUDA(cudaMemsetAsync(bt->dst, 0, sizeof(MemberState) * R, s));
            BCUDA(cudaMemsetAsync(bt->drun, 0, sizeof(RunState), s));
            return NTVS_OK;
        };
        for (auto& mm : bt->m) {
            const MemberDev& d = mm.d;
            BTRY(save(d.x, sizeof(double) * d.V));
            BTRY(save(d.x32, sizeof(float) * d.vm.vint));
            BTRY(save(d.xh, sizeof(float) * d.V));
            BTRY(save(d.xl, sizeof(float) * d.V));
        }
        cudaEvent_t e0, e1;
        BCUDA(cudaEventCreate(&e0));
        BCUDA(cudaEventCreate(&e1));
        float best = 1e30f;
        int best_rows = rows_c[0], best_win = win_c[0], best_minb = minb_c[0];
        int rc = NTVS_OK;
        for (int rows : rows_c) {
            if ((rc = build_items(bt, rows, 0)) != NTVS_OK) break;
            for (int cap : win_c) {
                if (cap > 0 && (rc = build_items(bt, rows, cap)) != NTVS_OK) break;
                for (int minb : minb_c) {
                    if ((rc = set_grid(cap, minb)) != NTVS_OK) break;
                    bt->win_cap = cap;
                    if ((rc = launch_cycle(bt, bt->hbeta[0], false)) != NTVS_OK) break;   // warm-up
                    cudaEventRecord(e0, s);
                    for (int c = 1; c < kTrialCycles && rc == NTVS_OK; ++c) rc = launch_cycle(bt, bt->hbeta[0], false);
                    cudaEventRecord(e1, s);
                    if (rc != NTVS_OK) break;
                    if (cudaEventSynchronize(e1) != cudaSuccess) { rc = bfail(NTVS_ERR_CUDA, "batch tuning"); break; }
                    if ((rc = device_error(bt)) != NTVS_OK) break;
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    bt->tune_cand.insert(bt->tune_cand.end(), {rows, cap, minb, 0});
                    bt->tune_ms.push_back(ms / (float)(kTrialCycles - 1));
                    if (ms < best) { best = ms; best_rows = rows; best_win = cap; best_minb = minb; }
                    if ((rc = restore()) != NTVS_OK) break;
                }
                if (rc != NTVS_OK) break;
            }
            if (rc != NTVS_OK) break;
        }
        // then the rows per warp: every member with 1 row per warp, 2 or 4 (lanes per row 32,
        // 16, 8) against each member's own choice, on the best schedule found
        int best_lpr = 0;
        for (int lpr : {32, 16, 8}) {
            if (rc != NTVS_OK) break;
            for (auto& mm : bt->m) mm.d.lpr = lpr;
            if ((rc = build_items(bt, best_rows, best_win)) != NTVS_OK || (rc = set_grid(best_win, best_minb)) != NTVS_OK)
                break;
            bt->win_cap = best_win;
            if ((rc = launch_cycle(bt, bt->hbeta[0], false)) != NTVS_OK) break;   // warm-up
            cudaEventRecord(e0, s);
            for (int c = 1; c < kTrialCycles && rc == NTVS_OK; ++c) rc = launch_cycle(bt, bt->hbeta[0], false);
            cudaEventRecord(e1, s);
            if (rc != NTVS_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = bfail(NTVS_ERR_CUDA, "batch tuning"); break; }
            if ((rc = device_error(bt)) != NTVS_OK) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            bt->tune_cand.insert(bt->tune_cand.end(), {best_rows, best_win, best_minb, lpr});
            bt->tune_ms.push_back(ms / (float)(kTrialCycles - 1));
            if (ms < best) { best = ms; best_lpr = lpr; }
            if ((rc = restore()) != NTVS_OK) break;
        }
        for (auto& mm : bt->m) mm.d.lpr = mm.lpr_own;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc == NTVS_OK) rc = restore();
        cudaStreamSynchronize(s);
        for (void* q : saved) cudaFree(q);
        if (rc != NTVS_OK) return rc;
        bt->rows_per_item = best_rows;
        bt->win_cap = best_win;
        bt->minb = best_minb;
        bt->lpr_policy = best_lpr;
    }
    if (bt->lpr_policy > 0)
        for (auto& mm : bt->m) mm.d.lpr = bt->lpr_policy;
    BTRY(build_items(bt, bt->rows_per_item, bt->win_cap));
    BTRY(set_grid(bt->win_cap, bt->minb));
    // one graph per pinned beta buffer: beta copy, cycle setup, the persistent kernel
    for (int j = 0; j < 2; ++j) {
        cudaGraph_t g = nullptr;
        BCUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int rc = launch_cycle(bt, bt->hbeta[j], true);
        cudaError_t e = cudaStreamEndCapture(s, &g);
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
    if (bt->cycles + k_iters > bt->tv_cap) return bfail(NTVS_ERR_STATE, "more cycles than finalize's max_cycles");
    BCUDA(cudaSetDevice(bt->device));
    for (int it = 0; it < k_iters; ++it) {
        const int j = bt->next;
        BCUDA(cudaEventSynchronize(bt->used[j]));   // the graph that last read this buffer has copied it
        fill_betas(bt, bt->hbeta[j], true);
        BCUDA(cudaGraphLaunch(bt->graph[j], bt->stream));
        BCUDA(cudaEventRecord(bt->used[j], bt->stream));
        bt->next ^= 1;
        bt->cycles += 1;
        bt->launches += 2;
    }
    return NTVS_OK;
}

int ntvs_batch_sync(ntvs_batch* bt) {
    if (!bt) return bfail(NTVS_ERR_ARG, "null batch");
    BCUDA(cudaSetDevice(bt->device));
    BCUDA(cudaStreamSynchronize(bt->stream));
    if (!bt->finalized) return NTVS_OK;
    return device_error(bt);
}

int ntvs_batch_get_image(ntvs_batch* bt, int index, void* out, int dtype, int mem_kind) {
    if (!bt || !out) return bfail(NTVS_ERR_ARG, "null argument");
    if (index < 0 || index >= (int)bt->m.size()) return bfail(NTVS_ERR_ARG, "member index out of range");
    if (dtype != NTVS_F64 && dtype != NTVS_F32) return bfail(NTVS_ERR_ARG, "dtype must be F64 or F32");
    if (mem_kind != NTVS_MEM_HOST && mem_kind != NTVS_MEM_DEVICE) return bfail(NTVS_ERR_ARG, "bad mem_kind");
    BTRY(ntvs_batch_sync(bt));
    const MemberDev& d = bt->m[index].d;
    std::vector<double> x((size_t)d.V);
    BCUDA(cudaMemcpy(x.data(), d.x, sizeof(double) * d.V, cudaMemcpyDeviceToHost));
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
    if (bt->cycles == 0) return bfail(NTVS_ERR_STATE, "no cycle run yet");
    BTRY(ntvs_batch_sync(bt));
    BCUDA(cudaMemcpy(tv, bt->m[index].d.tv_hist + (bt->cycles - 1), sizeof(double), cudaMemcpyDeviceToHost));
    return NTVS_OK;
}

int ntvs_batch_get_member(ntvs_batch* bt, int index, int64_t* out5) {
    if (!bt || !out5) return bfail(NTVS_ERR_ARG, "null argument");
    if (index < 0 || index >= (int)bt->m.size()) return bfail(NTVS_ERR_ARG, "member index out of range");
    if (!bt->finalized) return bfail(NTVS_ERR_STATE, "batch not finalized");
    BTRY(ntvs_batch_sync(bt));
    MemberState st;
    BCUDA(cudaMemcpy(&st, bt->dst + index, sizeof(MemberState), cudaMemcpyDeviceToHost));
    const auto& mm = bt->m[index];
    out5[0] = st.k;
    out5[1] = mm.p.tv_check ? st.ell : mm.ell_prev;
    out5[2] = st.n_steps;
    out5[3] = st.n_accepted;
    out5[4] = st.n_tries;
    return NTVS_OK;
}

int ntvs_batch_get_rows(ntvs_batch* bt, int index, int64_t* n_rows, int64_t* nnz, int64_t* row_ptr, int32_t* col,
                        float* val) {
    if (!bt) return bfail(NTVS_ERR_ARG, "null batch");
    if (index < 0 || index >= (int)bt->m.size()) return bfail(NTVS_ERR_ARG, "member index out of range");
    BCUDA(cudaSetDevice(bt->device));
    const auto& mm = bt->m[index];
    if (n_rows) *n_rows = mm.M;
    if (nnz) *nnz = mm.nnz;
    BCUDA(cudaStreamSynchronize(bt->stream));
    if (row_ptr) BCUDA(cudaMemcpy(row_ptr, mm.d.row_ptr, sizeof(int64_t) * (mm.M + 1), cudaMemcpyDeviceToHost));
    if ((col || val) && mm.nnz > 0) {   // unpacked from the pairs, columns back in canonical order
        int32_t* tc = nullptr;
        float* tv = nullptr;
        if (col) BTRY(balloc(&tc, sizeof(int32_t) * mm.nnz, "column read-back"));
        if (val) {
            const int rc = balloc(&tv, sizeof(float) * mm.nnz, "value read-back");
            if (rc != NTVS_OK) {
                cudaFree(tc);
                return rc;
            }
        }
        unmap_kernel<<<grid_of(mm.nnz), 256, 0, bt->stream>>>(mm.d.ent, tc, tv, mm.nnz, mm.d.vm);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && col)
            e = cudaMemcpyAsync(col, tc, sizeof(int32_t) * mm.nnz, cudaMemcpyDeviceToHost, bt->stream);
        if (e == cudaSuccess && val)
            e = cudaMemcpyAsync(val, tv, sizeof(float) * mm.nnz, cudaMemcpyDeviceToHost, bt->stream);
        cudaError_t e2 = cudaStreamSynchronize(bt->stream);
        cudaFree(tc);
        cudaFree(tv);
        if (e != cudaSuccess || e2 != cudaSuccess) return bfail(NTVS_ERR_CUDA, "batch: row read-back");
    }
    return NTVS_OK;
}

int ntvs_batch_get_tuning(ntvs_batch* bt, int32_t* cand, float* ms, int cap, int* n) {
    if (!bt || !n) return bfail(NTVS_ERR_ARG, "null argument");
    if (cap < 0 || (cap > 0 && (!cand || !ms))) return bfail(NTVS_ERR_ARG, "bad output arrays");
    const int k = (int)bt->tune_ms.size();
    *n = k;
    for (int i = 0; i < std::min(k, cap); ++i) {
        for (int q = 0; q < 4; ++q) cand[4 * i + q] = bt->tune_cand[4 * (size_t)i + q];
        ms[i] = bt->tune_ms[i];
    }
    return NTVS_OK;
}

int ntvs_batch_get_stats(ntvs_batch* bt, ntvs_batch_stats* st) {
    if (!bt || !st) return bfail(NTVS_ERR_ARG, "null argument");
    std::memset(st, 0, sizeof(*st));
    st->members = (int32_t)bt->m.size();
    st->cycles = bt->cycles;
    st->n_launches = bt->launches;
    st->kernels_per_cycle = bt->finalized ? 2 : 0;
    st->rows_per_item = bt->rows_per_item;
    st->window_floats = bt->win_cap < 0 ? 0 : bt->win_cap;
    st->ctas = bt->grid;
    st->ctas_per_sm = bt->minb;
    int lmin = 32, lmax = 0;
    for (const auto& mm : bt->m) {
        st->total_rows += mm.M;
        st->total_nnz += mm.nnz;
        st->total_voxels += mm.d.V;
        lmin = std::min(lmin, mm.d.lpr);
        lmax = std::max(lmax, mm.d.lpr);
    }
    st->lanes_per_row = bt->m.empty() ? 0 : lmax;
    st->lanes_per_row_min = bt->m.empty() ? 0 : lmin;
    st->lanes_per_row_all = bt->lpr_policy;
    return NTVS_OK;
}

}  // extern "C"
