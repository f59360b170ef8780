// Block-DROP kernels (P_T of arXiv 1803.01112 Appendix C; DROP of ref. CEHN08, Sec. III-D).
//
// drop_block: for every row i of block t (all rows see the same x):
//     d_i = <a_i, x>                    (CSR gather, x is L2/L1-resident)
//     r_i = lambda (b_i - d_i) / ||a_i||^2
//     delta_j += r_i a_ij               (scatter-add)
//   A group of LPR lanes owns a row; each lane loads VW consecutive entries per step
//   (16-byte column and value vectors for 4-byte values), and the row's entries stay in
//   registers between the dot product and the scatter, so the matrix streams from HBM
//   exactly once.
//
//   Windowed variant (one 1024-thread CTA per SM): the CTA owns a list of row segments
//   that share a "home" z-slice (assigned at load time), keeps delta for that slice in
//   shared memory and scatters there with shared-memory atomics; entries outside the
//   slice go to global memory.  When the home slice changes, and at the end, the window
//   is flushed into delta with one global reduction per touched voxel.  This replaces
//   ~1 global L2 atomic per matrix entry by ~0.2.
//   Plain variant (any row order): every scatter is a global reduction.
// drop_apply: x_j += delta_j / s_j^t (inverse counts precomputed), delta_j = 0.
#include <type_traits>

#include "common.cuh"

namespace ntvs {

// 4 consecutive values from an 8- or 16-byte aligned address, streamed (evict-first)
__device__ __forceinline__ void load4(const float* p, float (&o)[4]) {
    const float4 v = __ldcs(reinterpret_cast<const float4*>(p));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void load4(const __half* p, float (&o)[4]) {
    const uint2 v = __ldcs(reinterpret_cast<const uint2*>(p));
    const __half2 h0 = *reinterpret_cast<const __half2*>(&v.x), h1 = *reinterpret_cast<const __half2*>(&v.y);
    const float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
    o[0] = f0.x; o[1] = f0.y; o[2] = f1.x; o[3] = f1.y;
}
__device__ __forceinline__ void load4(const __nv_bfloat16* p, float (&o)[4]) {
    const uint2 v = __ldcs(reinterpret_cast<const uint2*>(p));
    const __nv_bfloat162 h0 = *reinterpret_cast<const __nv_bfloat162*>(&v.x);
    const __nv_bfloat162 h1 = *reinterpret_cast<const __nv_bfloat162*>(&v.y);
    const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
    o[0] = f0.x; o[1] = f0.y; o[2] = f1.x; o[3] = f1.y;
}

// The windowed kernel's dynamic shared memory: the slice window, voxels [w0, w0 + W).
extern __shared__ __align__(16) unsigned char drop_win_smem[];

struct Window {
    int w0;        // voxel indices stay below 2^31
    int W;
};

// Scale of the FP32 fixed-point window, uniform over the CTA (kept in shared memory so
// that the row loop's registers hold the matrix entries): quantum Q = 1 / invQ; rows with
// |r_i / lambda| above `bound` scatter globally (invQ = 0 sends every row there), which
// keeps every window slot below 2^30 Q and every converted term below 2^22 in magnitude;
// `obs` collects the largest |r_i / lambda| seen (float bits, atomic max).
struct WinScale {
    float invQ;
    float bound;
    unsigned obs;
};

// Shared-memory slot of window offset j: the low 5 bits are XORed with the next 5, a
// bijection inside each group of 32 slots.  Paths along y step the offset by nx (200: 8
// mod 32), which without the swizzle puts a warp's 32 updates into 4 banks.
__device__ __forceinline__ int swz(int j) { return j ^ ((j >> 5) & 31); }

// delta_c += r * a.  In the window: FP32 compute adds round(rq * a) (rq = r / Q) to the
// int32 fixed-point slot with a native shared-memory integer atomic when the row is
// within the bound (rowfix), else the row's entries take the global path; FP64 compute
// adds r * a to a double slot.  Outside the window: a global reduction.
template <typename T, bool WIN>
__device__ __forceinline__ void scatter(T* delta, const Window& w, int32_t c, T r, T a, bool rowfix, float rq) {
    if (WIN) {
        const int rel = c - w.w0;
        if ((unsigned)rel < (unsigned)w.W) {
            if constexpr (sizeof(T) == 4) {
                if (rowfix) {   // |rq a| < 2^22: adding 1.5 * 2^23 rounds it to the nearest integer
                    const int y = __float_as_int(fmaf(rq, (float)a, 12582912.0f)) - 0x4B400000;
                    atomicAdd(reinterpret_cast<int*>(drop_win_smem) + swz(rel), y);
                    return;
                }
            } else {
                atomicAdd(reinterpret_cast<T*>(drop_win_smem) + swz(rel), r * a);
                return;
            }
        }
    }
    atomicAdd(delta + c, r * a);
}

// the row's r = lambda * res / ||a||^2, whether its windowed entries go to the fixed-point
// window, and r / Q; the row's first lane records |res / ||a||^2| of a valid row in ws->obs
template <typename T, bool WIN>
__device__ __forceinline__ void row_factor(bool valid, bool first_lane, T res, T inv, T lambda, WinScale* ws,
                                           T& r, bool& rowfix, float& rq) {
    const T rn = res * inv;
    r = lambda * rn;
    rowfix = false;
    rq = 0.f;
    if constexpr (WIN && sizeof(T) == 4) {
        const float arn = fabsf((float)rn);
        const float iq = ws->invQ;
        rowfix = iq > 0.f && arn <= ws->bound;
        rq = (float)r * iq;
        if (valid && first_lane && arn > 0.f) atomicMax(&ws->obs, __float_as_uint(arn));
    }
}

// A row's extent, loaded one row ahead of its use by the row loops (the row pointer,
// col/val and x gathers are otherwise three dependent round trips per row).
struct RowHead {
    int64_t p0, p1;
};

__device__ __forceinline__ RowHead load_head(int64_t i, bool valid, const int64_t* __restrict__ row_ptr) {
    RowHead h{0, 0};
    if (valid) {
        h.p0 = __ldg(row_ptr + i);
        h.p1 = __ldg(row_ptr + i + 1);
    }
    return h;
}

// One row per group of LPR lanes (all lanes of the warp call this together).
// VW entries per lane per step from aligned addresses; CH steps held in registers.
template <typename T, typename V, int LPR, int CH, int VW, bool WIN>
__device__ __forceinline__ void drop_row(int64_t i, const RowHead& h, bool valid, int sub,
                                         const int32_t* __restrict__ col, const V* __restrict__ val,
                                         const T* __restrict__ b, const T* __restrict__ inv_norm2,
                                         const T* __restrict__ x, T* __restrict__ delta, T lambda, const Window& w,
                                         double& ss, WinScale* ws) {
    const int64_t p0 = h.p0, p1 = h.p1;
    const int64_t pa = p0 & ~(int64_t)(VW - 1);
    // entries relative to the aligned start in 32 bits (the register steps cover far fewer
    // than 2^31 entries; the tail loop below runs in 64 bits)
    const int32_t* colr = col + pa;
    const V* valr = val + pa;
    const int lo = (int)(p0 - pa);
    const int hi = (int)((p1 - pa) < (int64_t)0x7fffffff ? (p1 - pa) : (int64_t)0x7fffffff);
    // Every register step is predicated rather than skipped: with a branch per step the
    // gathers of later steps could not be issued ahead of the earlier steps' arithmetic
    // (measured 0.47 against 0.33 ms per 500k-row block).
    int32_t c[CH][VW];
    T a[CH][VW];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
        const int q = (u * LPR + sub) * VW;
        if (q < hi) {
            if constexpr (VW == 4) {
                const int4 cv = __ldcs(reinterpret_cast<const int4*>(colr + q));
                float av[4];
                load4(valr + q, av);
                c[u][0] = cv.x; c[u][1] = cv.y; c[u][2] = cv.z; c[u][3] = cv.w;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    a[u][e] = (T)av[e];
                    if (q + e < lo || q + e >= hi) c[u][e] = -1;
                }
            } else {
                c[u][0] = __ldcs(colr + q);
                a[u][0] = (T)to_compute(valr[q]);
            }
        } else {
#pragma unroll
            for (int e = 0; e < VW; ++e) { c[u][e] = -1; a[u][e] = (T)0; }
        }
    }
    T acc = (T)0;
#pragma unroll
    for (int u = 0; u < CH; ++u)
#pragma unroll
        for (int e = 0; e < VW; ++e)
            if (c[u][e] >= 0) acc += a[u][e] * __ldg(x + c[u][e]);
    // entries beyond the register-held steps (long rows): scalar, re-read for the scatter
    const int64_t tail0 = pa + (int64_t)CH * LPR * VW;
    for (int64_t p = (tail0 > p0 ? tail0 : p0) + sub; p < p1; p += LPR)
        acc += (T)to_compute(val[p]) * __ldg(x + col[p]);
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    T res = (T)0, inv = (T)0;
    if (valid) {
        res = __ldg(b + i) - acc;
        inv = __ldg(inv_norm2 + i);
        if (sub == 0) ss += (double)res * (double)res;
    }
    T r;
    bool rowfix;
    float rq;
    row_factor<T, WIN>(valid, sub == 0, res, inv, lambda, ws, r, rowfix, rq);
#pragma unroll
    for (int u = 0; u < CH; ++u)
#pragma unroll
        for (int e = 0; e < VW; ++e)
            if (c[u][e] >= 0) scatter<T, WIN>(delta, w, c[u][e], r, a[u][e], rowfix, rq);
    for (int64_t p = (tail0 > p0 ? tail0 : p0) + sub; p < p1; p += LPR)
        scatter<T, WIN>(delta, w, col[p], r, (T)to_compute(val[p]), rowfix, rq);
}

// drop_row on DELTA16 storage, a warp per row: each 32-entry chunk is decoded once (warp
// prefix sum of the int16 differences, escapes from the row's exception list) into the
// same registers the CSR32 path loads; long-row tails decode on the fly.
template <typename T, typename V, int CH, bool WIN>
__device__ __forceinline__ void drop_row_d16(int64_t i, bool valid, const int64_t* __restrict__ row_ptr,
                                             const Delta16& d16, const V* __restrict__ val, const T* __restrict__ b,
                                             const T* __restrict__ inv_norm2, const T* __restrict__ x,
                                             T* __restrict__ delta, T lambda, const Window& w, double& ss,
                                             WinScale* ws) {
    const int lane = threadIdx.x & 31;
    int64_t p0 = 0, p1 = 0;
    int32_t base = 0;
    int e0 = 0, ne = 0;
    if (valid) {
        p0 = __ldg(row_ptr + i);
        p1 = __ldg(row_ptr + i + 1);
        base = __ldg(d16.base + i);
        e0 = __ldg(d16.exc_off + i);
        ne = __ldg(d16.exc_off + i + 1) - e0;
    }
    const int2* ex = d16.exc + e0;
    int32_t c[CH];
    T a[CH];
    int carry = base;
#pragma unroll
    for (int u = 0; u < CH; ++u) {
        const int64_t p = p0 + lane + (int64_t)u * 32;
        const bool ok = p < p1;
        int dd = 0;
        if (ok) { dd = __ldcs(d16.col16 + p); a[u] = (T)to_compute(val[p]); } else { a[u] = (T)0; }
        const int cc = decode_delta16(dd, ok, (int)(p - p0), ex, ne, carry);
        c[u] = ok ? cc : -1;
    }
    const int tail_carry = carry;
    const int64_t tail0 = p0 + (int64_t)CH * 32;
    T acc = (T)0;
#pragma unroll
    for (int u = 0; u < CH; ++u)
        if (c[u] >= 0) acc += a[u] * __ldg(x + c[u]);
    carry = tail_carry;
    for (int64_t pb = tail0; pb < p1; pb += 32) {
        const int64_t p = pb + lane;
        const bool ok = p < p1;
        const int cc = decode_delta16(ok ? (int)d16.col16[p] : 0, ok, (int)(p - p0), ex, ne, carry);
        if (ok) acc += (T)to_compute(val[p]) * __ldg(x + cc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    T res = (T)0, inv = (T)0;
    if (valid) {
        res = __ldg(b + i) - acc;
        inv = __ldg(inv_norm2 + i);
        if (lane == 0) ss += (double)res * (double)res;
    }
    T r;
    bool rowfix;
    float rq;
    row_factor<T, WIN>(valid, lane == 0, res, inv, lambda, ws, r, rowfix, rq);
#pragma unroll
    for (int u = 0; u < CH; ++u)
        if (c[u] >= 0) scatter<T, WIN>(delta, w, c[u], r, a[u], rowfix, rq);
    carry = tail_carry;
    for (int64_t pb = tail0; pb < p1; pb += 32) {
        const int64_t p = pb + lane;
        const bool ok = p < p1;
        const int cc = decode_delta16(ok ? (int)d16.col16[p] : 0, ok, (int)(p - p0), ex, ne, carry);
        if (ok) scatter<T, WIN>(delta, w, cc, r, (T)to_compute(val[p]), rowfix, rq);
    }
}

// Plain variant: grid-stride over the rows of the block.
template <typename T, typename V, int LPR, int CH, int VW>
__global__ void __launch_bounds__(256)
drop_block_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, const V* __restrict__ val,
                  const T* __restrict__ b, const T* __restrict__ inv_norm2, int64_t r0, int64_t r1,
                  const T* __restrict__ x, T* __restrict__ delta, T lambda, double* resid_ss) {
    constexpr int G = 32 / LPR;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const Window w{0, 0};
    double ss = 0.0;
    int64_t i = r0 + warp * G + lane / LPR;
    RowHead h = load_head(i, i < r1, row_ptr);
    for (int64_t base = r0 + warp * G; base < r1; base += nwarps * G) {
        const int64_t in = i + nwarps * G;
        const RowHead hn = load_head(in, in < r1, row_ptr);   // next row, ahead of use
        drop_row<T, V, LPR, CH, VW, false>(i, h, i < r1, lane % LPR, col, val, b, inv_norm2, x, delta, lambda, w, ss,
                                           nullptr);
        i = in;
        h = hn;
    }
    __shared__ double sh[32];
    const double tot = block_sum(ss, sh);
    if (threadIdx.x == 0 && tot != 0.0) atomicAdd(resid_ss, tot);
}

// Windowed variant: CTA b processes segments [seg_begin[b], seg_begin[b+1]) in order.
// The window holds Wp = W rounded up to 32 slots (swizzled); slots past W stay 0.  FP32
// compute keeps int32 multiples of the quantum Q, FP64 compute doubles.
template <typename T>
__device__ __forceinline__ void flush_window(void* winp, int Wp, T* delta, int w0, float Q) {
    if constexpr (sizeof(T) == 4) {
        int* win = reinterpret_cast<int*>(winp);
        for (int jj = threadIdx.x; jj < Wp; jj += blockDim.x) {
            const int v = win[jj];
            if (v != 0) {
                atomicAdd(delta + w0 + swz(jj), (float)v * Q);
                win[jj] = 0;
            }
        }
    } else {
        T* win = reinterpret_cast<T*>(winp);
        for (int jj = threadIdx.x; jj < Wp; jj += blockDim.x) {
            const T v = win[jj];
            if (v != (T)0) {
                atomicAdd(delta + w0 + swz(jj), v);
                win[jj] = (T)0;
            }
        }
    }
}

template <typename T, typename V, int LPR, int CH, int VW, bool D16>
__global__ void __launch_bounds__(1024, 1)
drop_block_window_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                         const V* __restrict__ val, const T* __restrict__ b, const T* __restrict__ inv_norm2,
                         const DropSegment* __restrict__ segs, const int32_t* __restrict__ seg_begin,
                         int64_t slice, const T* __restrict__ x, T* __restrict__ delta, T lambda,
                         double* resid_ss, Delta16 d16, const float* wlmax, const float* wbound, float* wobs,
                         const float* wamax) {
    T* win = reinterpret_cast<T*>(drop_win_smem);
    __shared__ WinScale ws;
    __shared__ double ss_grp[32][32 / LPR];                     // per row group: sum of res^2 (one writer)
    const int W = (int)slice;
    const int Wp = (W + 31) & ~31;
    constexpr int G = 32 / LPR;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    for (int j = threadIdx.x; j < Wp; j += blockDim.x) win[j] = (T)0;   // int 0 has the bits of 0.0f
    for (int q = threadIdx.x; q < 32 * G; q += blockDim.x) (&ss_grp[0][0])[q] = 0.0;
    // rows with |r/lambda| <= bound keep |window slot| <= |lambda| bound lmax = 2^30 Q (no
    // int32 overflow); rows also below 2^22 Q / (|lambda| amax) keep every term below 2^22
    const float bound = wbound ? *wbound : 0.f, lmax = wlmax ? *wlmax : 0.f, amax = wamax ? *wamax : 0.f;
    const float lam = fabsf((float)lambda);
    const float Q = lam * bound * lmax * 0x1p-30f;
    if (threadIdx.x == 0) {
        const float iq = 1.f / Q;
        const bool fix = sizeof(T) == 4 && bound > 0.f && amax > 0.f && Q > 0.f && isfinite(Q) && isfinite(iq);
        ws.invQ = fix ? iq : 0.f;
        ws.bound = fix ? fminf(bound, 0x1p22f * Q / (lam * amax)) : 0.f;
        ws.obs = 0u;
    }
    __syncthreads();
    const int s0 = seg_begin[blockIdx.x], s1 = seg_begin[blockIdx.x + 1];
    int cur = s0 < s1 ? segs[s0].home : 0;
    Window w{(int)(cur * slice), W};
    double ss = 0.0;   // DELTA16 rows
    for (int s = s0; s < s1; ++s) {
        const DropSegment sg = segs[s];
        if (sg.home != cur) {   // uniform across the CTA
            __syncthreads();
            flush_window<T>(win, Wp, delta, w.w0, Q);
            __syncthreads();
            cur = sg.home;
            w.w0 = (int)(cur * slice);
        }
        if constexpr (D16) {
            for (int64_t base = sg.r0 + (int64_t)warp * G; base < sg.r1; base += (int64_t)nwarps * G) {
                const int64_t i = base + lane / LPR;
                drop_row_d16<T, V, CH, true>(i, i < sg.r1, row_ptr, d16, val, b, inv_norm2, x, delta, lambda, w, ss,
                                             &ws);
            }
        } else {
            const int grp = lane / LPR;
            for (int64_t base = sg.r0 + (int64_t)warp * G; base < sg.r1; base += (int64_t)nwarps * G) {
                const int64_t i = base + grp;
                const RowHead h = load_head(i, i < sg.r1, row_ptr);
                drop_row<T, V, LPR, CH, VW, true>(i, h, i < sg.r1, lane % LPR, col, val, b, inv_norm2, x, delta,
                                                  lambda, w, ss_grp[warp][grp], &ws);
            }
        }
    }
    __syncthreads();
    flush_window<T>(win, Wp, delta, w.w0, Q);
    if (!D16 && lane < G) ss = ss_grp[warp][lane];
    __shared__ double sh[32];
    const double tot = block_sum(ss, sh);   // synchronizes the CTA
    if (threadIdx.x == 0) {
        if (tot != 0.0) atomicAdd(resid_ss, tot);
        if (wobs && ws.obs) atomicMax(reinterpret_cast<unsigned*>(wobs), ws.obs);
    }
}

// Plain variant on DELTA16 index storage: a warp per row; columns are decoded chunk by
// chunk with a warp prefix sum, once for the dot product and once for the scatter.
template <typename T, typename V>
__global__ void __launch_bounds__(256)
drop_block_d16_kernel(const int64_t* __restrict__ row_ptr, Delta16 d16, const V* __restrict__ val,
                      const T* __restrict__ b, const T* __restrict__ inv_norm2, int64_t r0, int64_t r1,
                      const T* __restrict__ x, T* __restrict__ delta, T lambda, double* resid_ss) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double ss = 0.0;
    for (int64_t i = r0 + warp; i < r1; i += nwarps) {
        const int64_t p0 = __ldg(row_ptr + i), p1 = __ldg(row_ptr + i + 1);
        const int32_t base = __ldg(d16.base + i);
        const int e0 = __ldg(d16.exc_off + i), ne = __ldg(d16.exc_off + i + 1) - e0;
        const int2* ex = d16.exc + e0;
        T acc = (T)0;
        int carry = base;
        for (int64_t pb = p0; pb < p1; pb += 32) {
            const int64_t p = pb + lane;
            const bool valid = p < p1;
            const int c = decode_delta16(valid ? (int)__ldcs(d16.col16 + p) : 0, valid, (int)(p - p0), ex, ne, carry);
            if (valid) acc += (T)to_compute(val[p]) * __ldg(x + c);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        const T res = __ldg(b + i) - acc;
        const T r = lambda * res * __ldg(inv_norm2 + i);
        if (lane == 0) ss += (double)res * (double)res;
        carry = base;
        for (int64_t pb = p0; pb < p1; pb += 32) {
            const int64_t p = pb + lane;
            const bool valid = p < p1;
            const int c = decode_delta16(valid ? (int)d16.col16[p] : 0, valid, (int)(p - p0), ex, ne, carry);
            if (valid) atomicAdd(delta + c, r * (T)to_compute(val[p]));
        }
    }
    __shared__ double sh[32];
    const double tot = block_sum(ss, sh);
    if (threadIdx.x == 0 && tot != 0.0) atomicAdd(resid_ss, tot);
}

template <typename T>
__global__ void drop_apply_kernel(double* __restrict__ x, ImgCopies c, T* __restrict__ delta,
                                  const T* __restrict__ inv_s, int64_t V, float* wbound, float* wobs) {
    if (wbound && blockIdx.x == 0 && threadIdx.x == 0) {   // the window bound of the next sweep
        const float o = *wobs;
        if (o > 0.f) *wbound = 2.f * o;
        *wobs = 0.f;
    }
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < V; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = vox_internal(c.m, j);
        const double v = x[j] + (double)delta[p] * (double)__ldg(inv_s + p);
        x[j] = v;
        store_copies(c, j, v);
        delta[p] = (T)0;
    }
}

// ------------------------------------------------------------------ launch
template <typename T, typename V, int LPR, int CH, int VW, bool D16>
static cudaError_t launch_window(const DropArgs& a, cudaStream_t s) {
    auto kern = drop_block_window_kernel<T, V, LPR, CH, VW, D16>;
    const size_t smem = (size_t)((a.slice + 31) & ~31LL) * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<a.grid, 1024, smem, s>>>(a.row_ptr, a.col, (const V*)a.val, (const T*)a.b, (const T*)a.inv_norm2, a.segs,
                                    a.seg_begin, a.slice, (const T*)a.x, (T*)a.delta, (T)a.lambda, a.resid_ss, a.d16,
                                    a.wlmax, a.wbound, a.wobs, a.wamax);
    return cudaGetLastError();
}

template <typename T, typename V, int LPR, int CH, int VW>
static cudaError_t launch_cfg(const DropArgs& a, cudaStream_t s) {
    if (a.segs) {
        return launch_window<T, V, LPR, CH, VW, false>(a, s);
    } else {
        drop_block_kernel<T, V, LPR, CH, VW><<<a.grid, 256, 0, s>>>(
            a.row_ptr, a.col, (const V*)a.val, (const T*)a.b, (const T*)a.inv_norm2, a.r0, a.r1, (const T*)a.x,
            (T*)a.delta, (T)a.lambda, a.resid_ss);
    }
    return cudaGetLastError();
}

template <typename T, typename V>
static cudaError_t dispatch(const DropArgs& a, cudaStream_t s) {
    if constexpr (sizeof(V) <= 4) {
        if (a.vector4) {
        switch (a.lanes_per_row) {
            case 4: return launch_cfg<T, V, 4, 2, 4>(a, s);
            case 8: return launch_cfg<T, V, 8, 2, 4>(a, s);
            case 16: return launch_cfg<T, V, 16, 3, 4>(a, s);
            case 32: return launch_cfg<T, V, 32, 3, 4>(a, s);
            default: return cudaErrorInvalidValue;
        }
        }
    }
    // windowed FP32 compute with a warp per row: as many register steps as the block's
    // longest row needs (8..12; longer rows finish in the tail loop), so blocks of short rows
    // do not evaluate empty steps
    if constexpr (sizeof(T) == 4 && (std::is_same<V, float>::value || std::is_same<V, __nv_bfloat16>::value)) {
        if (a.segs && a.lanes_per_row == 32) {
            const int need = (int)((a.max_row + 31) / 32);
            if (need <= 8) return launch_cfg<T, V, 32, 8, 1>(a, s);
            if (need == 9) return launch_cfg<T, V, 32, 9, 1>(a, s);
            if (need == 10) return launch_cfg<T, V, 32, 10, 1>(a, s);
            if (need == 11) return launch_cfg<T, V, 32, 11, 1>(a, s);
        }
    }
    switch (a.lanes_per_row) {
        case 4: return launch_cfg<T, V, 4, 8, 1>(a, s);
        case 8: return launch_cfg<T, V, 8, 8, 1>(a, s);
        case 16: return launch_cfg<T, V, 16, 10, 1>(a, s);
        case 32: return launch_cfg<T, V, 32, 12, 1>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, typename V>
static cudaError_t launch_d16(const DropArgs& a, cudaStream_t s) {
    drop_block_d16_kernel<T, V><<<a.grid, 256, 0, s>>>(a.row_ptr, a.d16, (const V*)a.val, (const T*)a.b,
                                                        (const T*)a.inv_norm2, a.r0, a.r1, (const T*)a.x, (T*)a.delta,
                                                        (T)a.lambda, a.resid_ss);
    return cudaGetLastError();
}

cudaError_t k_drop_block(const DropArgs& a, cudaStream_t s) {
    if (a.r1 <= a.r0) return cudaSuccess;
    if (a.use_d16) {
        if (a.segs) {   // windowed: a warp per row, 12 register chunks
            if (a.cdt == F64) return a.vdt == F64   ? launch_window<double, double, 32, 12, 1, true>(a, s)
                                     : a.vdt == F32 ? launch_window<double, float, 32, 12, 1, true>(a, s)
                                                    : cudaErrorInvalidValue;
            switch (a.vdt) {
                case F32: return launch_window<float, float, 32, 12, 1, true>(a, s);
                case F16: return launch_window<float, __half, 32, 12, 1, true>(a, s);
                case BF16: return launch_window<float, __nv_bfloat16, 32, 12, 1, true>(a, s);
                default: return cudaErrorInvalidValue;
            }
        }
        if (a.cdt == F64) return a.vdt == F64 ? launch_d16<double, double>(a, s)
                                              : a.vdt == F32 ? launch_d16<double, float>(a, s) : cudaErrorInvalidValue;
        switch (a.vdt) {
            case F32: return launch_d16<float, float>(a, s);
            case F16: return launch_d16<float, __half>(a, s);
            case BF16: return launch_d16<float, __nv_bfloat16>(a, s);
            default: return cudaErrorInvalidValue;
        }
    }
    if (a.cdt == F64) {   // FP64 arithmetic on FP64 or FP32 storage
        if (a.vector4) return cudaErrorInvalidValue;
        if (a.vdt == F64) return dispatch<double, double>(a, s);
        if (a.vdt == F32) return dispatch<double, float>(a, s);
        return cudaErrorInvalidValue;
    }
    switch (a.vdt) {
        case F32: return dispatch<float, float>(a, s);
        case F16: return dispatch<float, __half>(a, s);
        case BF16: return dispatch<float, __nv_bfloat16>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t k_drop_apply(int cdt, double* x, ImgCopies c, void* delta, const void* inv_s, int64_t V, int grid,
                         float* wbound, float* wobs, cudaStream_t s) {
    if (cdt == F64)
        drop_apply_kernel<double><<<grid, 256, 0, s>>>(x, c, (double*)delta, (const double*)inv_s, V, wbound, wobs);
    else
        drop_apply_kernel<float><<<grid, 256, 0, s>>>(x, c, (float*)delta, (const float*)inv_s, V, wbound, wobs);
    return cudaGetLastError();
}

// *out = max(*out, longest row of rows [r0, r1))
__global__ void row_maxlen_kernel(const int64_t* __restrict__ row_ptr, int64_t r0, int64_t r1, unsigned long long* out) {
    unsigned long long m = 0;
    for (int64_t i = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < r1; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = row_ptr[i + 1] - row_ptr[i];
        m = l > (int64_t)m ? (unsigned long long)l : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
        m = v > m ? v : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

cudaError_t k_row_maxlen(const int64_t* row_ptr, int64_t r0, int64_t r1, unsigned long long* out, int grid,
                         cudaStream_t s) {
    if (r1 <= r0) return cudaSuccess;
    row_maxlen_kernel<<<grid, 256, 0, s>>>(row_ptr, r0, r1, out);
    return cudaGetLastError();
}

// home slice of each row: the median of the z-slices of its first, middle and last
// entries (-1 for an empty row); a path that bends out of its slice and back keeps the
// slice it enters and leaves by
__global__ void row_home_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int64_t M,
                                int64_t slice, int32_t* __restrict__ home) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p0 = row_ptr[i], p1 = row_ptr[i + 1];
        if (p1 <= p0) { home[i] = -1; continue; }
        const int32_t a = (int32_t)(col[p0] / slice), m = (int32_t)(col[p0 + (p1 - p0) / 2] / slice),
                      c = (int32_t)(col[p1 - 1] / slice);
        home[i] = max(min(a, m), min(max(a, m), c));
    }
}

cudaError_t k_row_home(const int64_t* row_ptr, const int32_t* col, int64_t M, int64_t slice, int32_t* home, int grid,
                       cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    row_home_kernel<<<grid, 256, 0, s>>>(row_ptr, col, M, slice, home);
    return cudaGetLastError();
}

// A warp per chunk of rows [cs[q], cs[q+1]) (at most 64): the lower median (element n/2
// of the sorted values) of the home slices of its non-empty rows, -1 when all are empty.
// Rows i >= 1 whose home and the previous row's home are both defined and differ are
// counted into *changes.
__global__ void chunk_home_kernel(const int32_t* __restrict__ home, const int64_t* __restrict__ cs, int64_t nchunks,
                                  int32_t* __restrict__ out, unsigned long long* changes) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long ch = 0;
    for (int64_t q = w0; q < nchunks; q += nw) {
        const int64_t i0 = cs[q], i1 = cs[q + 1];
        const int64_t ia = i0 + lane, ib = i0 + 32 + lane;
        const int32_t ha = ia < i1 ? home[ia] : -1;
        const int32_t hb = ib < i1 ? home[ib] : -1;
        if (ia < i1 && ia > 0) { const int32_t p = home[ia - 1]; ch += (ha >= 0 && p >= 0 && ha != p) ? 1 : 0; }
        if (ib < i1) { const int32_t p = home[ib - 1]; ch += (hb >= 0 && p >= 0 && hb != p) ? 1 : 0; }
        const int nv = __popc(__ballot_sync(0xffffffffu, ha >= 0)) + __popc(__ballot_sync(0xffffffffu, hb >= 0));
        if (nv == 0) {
            if (lane == 0) out[q] = -1;
            continue;
        }
        const int k = nv / 2;
        int la = 0, ea = 0, lb = 0, eb = 0;   // defined values below / at most ha and hb
        for (int src = 0; src < 32; ++src) {
            const int32_t wa = __shfl_sync(0xffffffffu, ha, src), wb = __shfl_sync(0xffffffffu, hb, src);
            if (wa >= 0) { la += wa < ha; ea += wa <= ha; lb += wa < hb; eb += wa <= hb; }
            if (wb >= 0) { la += wb < ha; ea += wb <= ha; lb += wb < hb; eb += wb <= hb; }
        }
        const unsigned ma = __ballot_sync(0xffffffffu, ha >= 0 && la <= k && k < ea);
        const unsigned mb = __ballot_sync(0xffffffffu, hb >= 0 && lb <= k && k < eb);
        const int32_t va = __shfl_sync(0xffffffffu, ha, ma ? __ffs(ma) - 1 : 0);
        const int32_t vb = __shfl_sync(0xffffffffu, hb, mb ? __ffs(mb) - 1 : 0);
        if (lane == 0) out[q] = ma ? va : vb;
    }
    for (int o = 16; o > 0; o >>= 1) ch += __shfl_xor_sync(0xffffffffu, ch, o);
    if (lane == 0 && ch) atomicAdd(changes, ch);
}

cudaError_t k_chunk_home(const int32_t* home, const int64_t* chunk_start, int64_t nchunks, int32_t* out,
                         unsigned long long* changes, int grid, cudaStream_t s) {
    if (nchunks <= 0) return cudaSuccess;
    chunk_home_kernel<<<grid, 256, 0, s>>>(home, chunk_start, nchunks, out, changes);
    return cudaGetLastError();
}

}  // namespace ntvs
