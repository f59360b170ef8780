// Block-DROP kernel templates (P_T of arXiv 1803.01112 Appendix C; DROP of ref. CEHN08,
// Sec. III-D), shared by the CSR32 and DELTA16 translation units.
//
// drop_block: for every row i of block t (all rows see the same x):
//     d_i = <a_i, x>                    (CSR gather, x is L2/L1-resident)
//     r_i = lambda (b_i - d_i) / ||a_i||^2
//     delta_j += r_i a_ij               (scatter-add)
//   A group of LPR lanes owns a row; each lane loads one entry per step (FP32 values:
//   the packed {column, value} pair, one 8-byte load), and the row's entries stay in
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
#pragma once
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

// The windowed kernel's dynamic shared memory: the stage of the current run of
// row_stage<D16>() rows (row pointers, b, 1/||a||^2) at fixed offsets, then the slice
// window, voxels [w0, w0 + W).  Fixed offsets keep the addresses out of the row loop's
// registers.  DELTA16 rows stage 5 more bytes each, so their stage is shorter: with the
// 160 KB window of a 200x200 slice both fit the 196 KB shared-memory carve-out, and the
// x gathers keep the L1 that a larger allocation would take (2048 DELTA16 rows measured
// 0.2652 against 0.2588 ms with 1600; FP32 rows 0.2346 with 1600 against 0.2329 with 2048).
extern __shared__ __align__(16) unsigned char drop_win_smem[];
template <bool D16>
__host__ __device__ constexpr int row_stage() { return D16 ? 1600 : 2048; }   // rows staged at once
constexpr int kPrefetchRows = 1;  // the windowed kernel asks L2 for the entries of the row this many ahead
constexpr int kShortSteps = kShortBody;   // register steps of the windowed kernel's body for short rows

// L2 prefetch of the 128-byte lines holding entries [q0, q1) of the index array (int32
// columns or DELTA16 offsets) and of val, one line per lane (rows longer than the warp's
// 32 lines prefetch their first lines only)
template <typename I, typename V>
__device__ __forceinline__ void prefetch_row_l2(const I* col, const V* val, int64_t q0, int64_t q1, int lane) {
    const uintptr_t c0 = (uintptr_t)(col + q0) & ~(uintptr_t)127, c1 = (uintptr_t)(col + q1);
    const uintptr_t v0 = (uintptr_t)(val + q0) & ~(uintptr_t)127, v1 = (uintptr_t)(val + q1);
    const int nc = (int)((c1 - c0 + 127) >> 7), nv = (int)((v1 - v0 + 127) >> 7);
    if (lane < nc) asm volatile("prefetch.global.L2 [%0];" ::"l"(c0 + ((uintptr_t)lane << 7)));
    else if (lane - nc < nv) asm volatile("prefetch.global.L2 [%0];" ::"l"(v0 + ((uintptr_t)(lane - nc) << 7)));
}
// the same for entries [q0, q1) of one array (packed pairs)
template <typename E>
__device__ __forceinline__ void prefetch_lines_l2(const E* a, int64_t q0, int64_t q1, int lane) {
    const uintptr_t a0 = (uintptr_t)(a + q0) & ~(uintptr_t)127, a1 = (uintptr_t)(a + q1);
    const int na = (int)((a1 - a0 + 127) >> 7);
    if (lane < na) asm volatile("prefetch.global.L2 [%0];" ::"l"(a0 + ((uintptr_t)lane << 7)));
}
template <typename T, bool D16>
__host__ __device__ constexpr size_t stage_bytes() {
    return ((sizeof(int64_t) * (row_stage<D16>() + 1) + 15) & ~(size_t)15) + 2 * sizeof(T) * row_stage<D16>();
}
// DELTA16 rows also stage their flags (1 byte) and their first chunk base (the base of a
// narrow row), so that neither is a dependent global load at the start of a row
template <typename T, bool D16>
__host__ __device__ constexpr size_t stage_bytes_all() {
    return stage_bytes<T, D16>() + (D16 ? ((size_t)row_stage<D16>() + 4 * (size_t)row_stage<D16>()) : 0);
}
template <typename T, bool D16>
__device__ __forceinline__ int64_t* stage_rp() { return reinterpret_cast<int64_t*>(drop_win_smem); }
template <typename T, bool D16>
__device__ __forceinline__ T* stage_b() {
    return reinterpret_cast<T*>(drop_win_smem + ((sizeof(int64_t) * (row_stage<D16>() + 1) + 15) & ~(size_t)15));
}
template <typename T, bool D16>
__device__ __forceinline__ T* stage_inv() { return stage_b<T, D16>() + row_stage<D16>(); }
template <typename T, bool D16>
__device__ __forceinline__ uint8_t* stage_fl() { return drop_win_smem + stage_bytes<T, D16>(); }
template <typename T, bool D16>
__device__ __forceinline__ int32_t* stage_rb() {
    return reinterpret_cast<int32_t*>(drop_win_smem + stage_bytes<T, D16>() + row_stage<D16>());
}
template <typename T, bool D16>
__device__ __forceinline__ unsigned char* window_base() { return drop_win_smem + stage_bytes_all<T, D16>(); }
inline size_t window_smem_bytes(int64_t slice, size_t tsize, bool d16) {
    const size_t stage = tsize == 8 ? (d16 ? stage_bytes_all<double, true>() : stage_bytes_all<double, false>())
                                    : (d16 ? stage_bytes_all<float, true>() : stage_bytes_all<float, false>());
    return stage + (size_t)((slice + 31) & ~31LL) * tsize;
}

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

// Shared-memory slot of window offset j.  Paths along y step the offset by nx (200: 8
// mod 32), which with slot = offset puts a warp's 32 updates into 4 banks; XORing the low
// 5 bits with the next 5 (a bijection inside each group of 32 slots) spreads them.  The
// FP32 path's internal voxel order already carries that swizzle inside each slice (the
// window starts at a slice), so its slot is the offset itself; the FP64 path gathers the
// canonical order and swizzles here.
__device__ __forceinline__ int swz(int j) { return j ^ ((j >> 5) & 31); }
// A DELTA16 word read without allocating in L1, which the x gathers then keep (0.2504 ->
// 0.2481 ms per 500k-row BF16 block; the FP32 pairs measured slower this way, 0.2307 ->
// 0.2325 ms, and keep the streaming load)
__device__ __forceinline__ uint32_t ld_no_l1(const uint32_t* p) {
    uint32_t v;
    asm("ld.global.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
template <typename T>
__device__ __forceinline__ int win_slot(int j) {
    if constexpr (sizeof(T) == 4) return j;
    else return swz(j);
}

// delta_c += r * a.  In the window: FP32 compute adds round(rq * a) (rq = r / Q) to the
// int32 fixed-point slot with a native shared-memory integer atomic when the row is
// within the bound (rowfix), else the row's entries take the global path; FP64 compute
// adds r * a to a double slot.  Outside the window: a global reduction.
template <typename T, bool WIN, bool D16>
__device__ __forceinline__ void scatter(T* delta, const Window& w, int32_t c, T r, T a, bool rowfix, float rq) {
    if (WIN) {
        const int rel = c - w.w0;
        if ((unsigned)rel < (unsigned)w.W) {
            if constexpr (sizeof(T) == 4) {
                if (rowfix) {   // |rq a| < 2^22: adding 1.5 * 2^23 rounds it to the nearest integer
                    const int y = __float_as_int(fmaf(rq, (float)a, 12582912.0f)) - 0x4B400000;
                    atomicAdd(reinterpret_cast<int*>(window_base<T, D16>()) + win_slot<T>(rel), y);
                    return;
                }
            } else {
                atomicAdd(reinterpret_cast<T*>(window_base<T, D16>()) + win_slot<T>(rel), r * a);
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
        // the block's largest |r/lambda|: a plain read first skips the atomic for most rows
        if (valid && first_lane && __float_as_uint(arn) > *(volatile unsigned*)&ws->obs)
            atomicMax(&ws->obs, __float_as_uint(arn));
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

// Column of entry q (counted from the row's first entry) of a DELTA16 row whose chunk bases
// start at cbr: the chunk's base plus the entry's offset, or, when the row has escaped
// chunks (ESC), the full column of an escaped chunk.
template <bool ESC>
__device__ __forceinline__ int32_t d16_col_o(const Delta16& d, const int32_t* cbr, int o, int q) {
    const int32_t base = __ldg(cbr + (q >> 5));
    if constexpr (ESC) return base >= 0 ? base + o : __ldg(d.exc + ((int64_t)(-1 - base) << 5) + (q & 31));
    return base + o;
}
template <bool ESC>
__device__ __forceinline__ int32_t d16_col(const Delta16& d, const int32_t* cbr, const uint16_t* offr, int q) {
    return d16_col_o<ESC>(d, cbr, (int)__ldcs(offr + q), q);
}

// entry p of a row (q = p minus the row's aligned start) as column and value, from whichever
// storage the kernel has: packed pairs, DELTA16 words, DELTA16 offsets with values, or int32
// columns with values
template <typename T, typename V, bool D16>
__device__ __forceinline__ void entry_any(const int32_t* col, const Delta16& d16, const V* val, const int32_t* cbr,
                                          int64_t p, int q, int32_t& c, T& a) {
    if constexpr (packed_entries<V, D16>()) {
        const int2 e = reinterpret_cast<const int2*>(col)[p];
        c = e.x;
        a = (T)__int_as_float(e.y);
    } else if constexpr (delta16_words<V, D16>()) {
        const uint32_t e = d16.word[p];
        c = d16_col_o<true>(d16, cbr, (int)(e & 0xffffu), q);
        a = (T)word_value<V>(e);
    } else if constexpr (D16) {
        c = d16_col_o<true>(d16, cbr, (int)d16.off[p], q);
        a = (T)to_compute(val[p]);
    } else {
        c = col[p];
        a = (T)to_compute(val[p]);
    }
}

template <typename T, typename V, int LPR, int CH, int VW, bool WIN, bool D16, bool ESC = false,
          bool NARROW = false>
__device__ __forceinline__ void drop_row(int64_t i, const RowHead& h, bool valid, int sub,
                                         const int32_t* __restrict__ col, const Delta16& d16,
                                         const V* __restrict__ val, T bval, T ival, const T* __restrict__ x,
                                         T* __restrict__ delta, T lambda, const Window& w, double& ss, WinScale* ws,
                                         int32_t rbase = 0) {
    static_assert(!D16 || VW == 1, "DELTA16 rows are read one entry per lane");
    constexpr bool PK = packed_entries<V, D16>();   // {column, value} pairs: one 8-byte load per entry
    constexpr bool W16 = delta16_words<V, D16>();   // DELTA16 {offset, value} words: one 4-byte load
    static_assert(!PK || VW == 1, "packed pairs are read one entry per lane");
    const int64_t p0 = h.p0, p1 = h.p1;
    const int64_t pa = p0 & ~(int64_t)(VW - 1);
    // entries relative to the aligned start in 32 bits (the register steps cover far fewer
    // than 2^31 entries; the tail loop below runs in 64 bits)
    const int32_t* colr = (D16 || PK) ? nullptr : col + pa;
    const int2* entr = PK ? reinterpret_cast<const int2*>(col) + pa : nullptr;
    // DELTA16: the row's offsets (or words) and its chunk bases (slot (p0 >> 5) + i + k), in 32 bits
    const uint16_t* offr = (D16 && !W16) ? d16.off + pa : nullptr;
    const uint32_t* wr = W16 ? d16.word + pa : nullptr;
    const int32_t* cbr = D16 ? d16.cbase + (pa >> 5) + i : nullptr;
    const V* valr = (PK || W16) ? nullptr : val + pa;
    const int lo = (int)(p0 - pa);
    const int hi = (int)((p1 - pa) < (int64_t)0x7fffffff ? (p1 - pa) : (int64_t)0x7fffffff);
    // Every register step is predicated rather than skipped: with a branch per step the
    // gathers of later steps could not be issued ahead of the earlier steps' arithmetic
    // (measured 0.47 against 0.33 ms per 500k-row block).
    int32_t c[CH][VW];
    T a[CH][VW];
    // a narrow DELTA16 row: all its chunk bases are rbase, the row's base (staged by the caller)
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
                if constexpr (W16) {
                    const uint32_t e = ld_no_l1(wr + q);
                    if constexpr (NARROW) c[u][0] = rbase + (int)(e & 0xffffu);
                    else c[u][0] = d16_col_o<ESC>(d16, cbr, (int)(e & 0xffffu), q);
                    a[u][0] = (T)word_value<V>(e);
                } else if constexpr (D16 && NARROW) {
                    c[u][0] = rbase + (int)__ldcs(offr + q);
                } else if constexpr (D16) {
                    c[u][0] = d16_col<ESC>(d16, cbr, offr, q);   // with a warp per row: one base per step
                } else if constexpr (PK) {
                    const int2 e = __ldcs(entr + q);
                    c[u][0] = e.x;
                    a[u][0] = (T)__int_as_float(e.y);
                } else {
                    c[u][0] = __ldcs(colr + q);
                }
                if constexpr (!PK && !W16) a[u][0] = (T)to_compute(valr[q]);
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
    for (int64_t p = (tail0 > p0 ? tail0 : p0) + sub; p < p1; p += LPR) {
        int32_t cp;
        T ap;
        entry_any<T, V, D16>(col, d16, val, cbr, p, (int)(p - pa), cp, ap);
        acc += ap * __ldg(x + cp);
    }
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    T res = (T)0, inv = (T)0;
    if (valid) {
        res = bval - acc;
        inv = ival;
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
            if (c[u][e] >= 0) scatter<T, WIN, D16>(delta, w, c[u][e], r, a[u][e], rowfix, rq);
    for (int64_t p = (tail0 > p0 ? tail0 : p0) + sub; p < p1; p += LPR) {
        int32_t cp;
        T ap;
        entry_any<T, V, D16>(col, d16, val, cbr, p, (int)(p - pa), cp, ap);
        scatter<T, WIN, D16>(delta, w, cp, r, ap, rowfix, rq);
    }
}

// One row, DELTA16 rows touching an escaped chunk through the checked body (a branch that
// is uniform over the row's lanes; the rows without escapes decode with one add).
template <typename T, typename V, int LPR, int CH, int VW, bool WIN, bool D16>
__device__ __forceinline__ void drop_row_any(int64_t i, const RowHead& h, bool valid, int sub,
                                             const int32_t* __restrict__ col, const Delta16& d16,
                                             const V* __restrict__ val, T bval, T ival, const T* __restrict__ x,
                                             T* __restrict__ delta, T lambda, const Window& w, double& ss,
                                             WinScale* ws, int fl_staged = -1, int32_t rbase = 0) {
    if constexpr (D16) {
        // DELTA16 row flags: staged by the windowed kernel, else read here
        const unsigned fl = fl_staged >= 0 ? (unsigned)fl_staged : (valid ? __ldg(d16.rowesc + i) : 0u);
        if (fl & 1u)
            drop_row<T, V, LPR, CH, VW, WIN, true, true>(i, h, valid, sub, col, d16, val, bval, ival, x, delta,
                                                        lambda, w, ss, ws);
        else if (WIN && LPR == 32 && fl_staged >= 0 && (fl & 2u)) {   // narrow rows: the staged base
            if (CH > kShortSteps && h.p1 - h.p0 <= (int64_t)kShortSteps * 32)
                drop_row<T, V, LPR, (CH > kShortSteps ? kShortSteps : CH), VW, WIN, true, false, true>(
                    i, h, valid, sub, col, d16, val, bval, ival, x, delta, lambda, w, ss, ws, rbase);
            else if (CH > kMidBody && h.p1 - h.p0 <= (int64_t)kMidBody * 32)   // 0.2681 -> 0.2657 ms
                drop_row<T, V, LPR, (CH > kMidBody ? kMidBody : CH), VW, WIN, true, false, true>(
                    i, h, valid, sub, col, d16, val, bval, ival, x, delta, lambda, w, ss, ws, rbase);
            else
                drop_row<T, V, LPR, CH, VW, WIN, true, false, true>(i, h, valid, sub, col, d16, val, bval, ival, x,
                                                                   delta, lambda, w, ss, ws, rbase);
        } else if (WIN && LPR == 32 && CH > kShortSteps && h.p1 - h.p0 <= (int64_t)kShortSteps * 32)
            drop_row<T, V, LPR, (CH > kShortSteps ? kShortSteps : CH), VW, WIN, true, false>(
                i, h, valid, sub, col, d16, val, bval, ival, x, delta, lambda, w, ss, ws);
        else
            drop_row<T, V, LPR, CH, VW, WIN, true, false>(i, h, valid, sub, col, d16, val, bval, ival, x, delta,
                                                         lambda, w, ss, ws);
    } else if constexpr (WIN && LPR == 32 && VW == 1 && CH > kShortSteps) {
        // rows of at most kShortSteps x 32 entries take a body with fewer register steps:
        // with the block's deepest body a short row would issue its empty steps predicated off;
        // in blocks deeper than kMidBody steps a middle body takes the rows that fit it
        // (measured 0.2356 -> 0.2326 ms per 500k-row block)
        if (h.p1 - h.p0 <= (int64_t)kShortSteps * 32)
            drop_row<T, V, LPR, kShortSteps, VW, WIN, false>(i, h, valid, sub, col, d16, val, bval, ival, x, delta,
                                                            lambda, w, ss, ws);
        else if (CH > kMidBody && h.p1 - h.p0 <= (int64_t)kMidBody * 32)
            drop_row<T, V, LPR, (CH > kMidBody ? kMidBody : CH), VW, WIN, false>(i, h, valid, sub, col, d16, val, bval,
                                                                                ival, x, delta, lambda, w, ss, ws);
        else
            drop_row<T, V, LPR, CH, VW, WIN, false>(i, h, valid, sub, col, d16, val, bval, ival, x, delta, lambda, w,
                                                    ss, ws);
    } else {
        drop_row<T, V, LPR, CH, VW, WIN, false>(i, h, valid, sub, col, d16, val, bval, ival, x, delta, lambda, w,
                                                ss, ws);
    }
}

// Plain variant: grid-stride over the rows of the block.
template <typename T, typename V, int LPR, int CH, int VW, bool D16>
__global__ void __launch_bounds__(256)
drop_block_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, const V* __restrict__ val,
                  const T* __restrict__ b, const T* __restrict__ inv_norm2, int64_t r0, int64_t r1,
                  const T* __restrict__ x, T* __restrict__ delta, T lambda, double* resid_ss, Delta16 d16) {
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
        const bool valid = i < r1;
        const T bi = valid ? __ldg(b + i) : (T)0, ii = valid ? __ldg(inv_norm2 + i) : (T)0;
        drop_row_any<T, V, LPR, CH, VW, false, D16>(i, h, valid, lane % LPR, col, d16, val, bi, ii, x, delta, lambda,
                                                    w, ss, nullptr);
        i = in;
        h = hn;
    }
    __shared__ double sh[32];
    const double tot = block_sum(ss, sh);
    if (threadIdx.x == 0 && tot != 0.0) atomicAdd(resid_ss, tot);
}

// Windowed variant: CTA b processes segments [seg_begin[b], seg_begin[b+1]) in order.
// The window holds Wp = W rounded up to 32 slots (win_slot); slots past W stay 0.  FP32
// compute keeps int32 multiples of the quantum Q, FP64 compute doubles.
// 4 consecutive floats added to global memory with one vector reduction (16-byte aligned)
__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

template <typename T>
__device__ __forceinline__ void flush_window(void* winp, int W, int Wp, T* delta, int w0, float Q) {
    if constexpr (sizeof(T) == 4) {
        int* win = reinterpret_cast<int*>(winp);
        // slot j holds voxel w0 + j (win_slot<float> is the identity)
        if (((w0 | W) & 3) == 0 && ((uintptr_t)delta & 15) == 0) {
            // one 16-byte shared load and one vector reduction per four voxels
            for (int j = 4 * threadIdx.x; j < W; j += 4 * blockDim.x) {
                int4* slot = reinterpret_cast<int4*>(win + j);
                const int4 v4 = *slot;
                if ((v4.x | v4.y | v4.z | v4.w) == 0) continue;
                red_add_v4(reinterpret_cast<float*>(delta) + w0 + j, (float)v4.x * Q, (float)v4.y * Q,
                           (float)v4.z * Q, (float)v4.w * Q);
                *slot = make_int4(0, 0, 0, 0);
            }
            return;
        }
        for (int jj = threadIdx.x; jj < W; jj += blockDim.x) {
            const int v = win[jj];
            if (v != 0) {
                atomicAdd(delta + w0 + jj, (float)v * Q);
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
    T* win = reinterpret_cast<T*>(window_base<T, D16>());
    const int W = (int)slice;
    const int Wp = (W + 31) & ~31;
    __shared__ WinScale ws;
    __shared__ double ss_grp[32][32 / LPR];                     // per row group: sum of res^2 (one writer)
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
    double ss = 0.0;
    for (int s = s0; s < s1; ++s) {
        const DropSegment sg = segs[s];
        if (sg.home != cur) {   // uniform across the CTA
            __syncthreads();
            flush_window<T>(win, W, Wp, delta, w.w0, Q);
            __syncthreads();
            cur = sg.home;
            w.w0 = (int)(cur * slice);
        }
        const int grp = lane / LPR;
        // the segment's rows in runs of row_stage<D16>(): one coalesced load of their row
        // pointers, b and 1/||a||^2 into shared memory, so that a row starts from its
        // entries' addresses instead of a round trip to HBM for its row pointer
        for (int64_t c0 = sg.r0; c0 < sg.r1; c0 += row_stage<D16>()) {
            const int n = (int)min((int64_t)row_stage<D16>(), sg.r1 - c0);
            __syncthreads();   // the previous run's rows are done with the stage
            for (int j = threadIdx.x; j <= n; j += blockDim.x) {
                const int64_t rp = __ldg(row_ptr + c0 + j);
                stage_rp<T, D16>()[j] = rp;
                if (j < n) {
                    stage_b<T, D16>()[j] = __ldg(b + c0 + j);
                    stage_inv<T, D16>()[j] = __ldg(inv_norm2 + c0 + j);
                    if constexpr (D16) {
                        stage_fl<T, D16>()[j] = __ldg(d16.rowesc + c0 + j);
                        stage_rb<T, D16>()[j] = __ldg(d16.cbase + (rp >> 5) + c0 + j);   // the row's first chunk base
                    }
                }
            }
            __syncthreads();
            for (int base = warp * G; base < n; base += nwarps * G) {
                const int k = base + grp;
                const bool valid = k < n;
                if constexpr (kPrefetchRows > 0 && LPR == 32) {
                    const int kp = k + kPrefetchRows * nwarps;   // this warp's row that many iterations ahead
                    if (kp < n) {
                        const int64_t q0 = stage_rp<T, D16>()[kp], q1 = stage_rp<T, D16>()[kp + 1];
                        if constexpr (D16) {
                            if constexpr (delta16_words<V, D16>()) prefetch_lines_l2(d16.word, q0, q1, lane);
                            else prefetch_row_l2(d16.off, val, q0, q1, lane);
                            // and the chunk bases of a row that is not narrow (one short run)
                            if (lane == 31 && !(stage_fl<T, D16>()[kp] & 2))
                                asm volatile("prefetch.global.L2 [%0];" ::"l"(d16.cbase + (q0 >> 5) + c0 + kp));
                        } else if constexpr (packed_entries<V, D16>()) {
                            prefetch_lines_l2(reinterpret_cast<const int2*>(col), q0, q1, lane);
                        } else {
                            prefetch_row_l2(col, val, q0, q1, lane);
                        }
                    }
                }
                const RowHead h{valid ? stage_rp<T, D16>()[k] : 0, valid ? stage_rp<T, D16>()[k + 1] : 0};
                drop_row_any<T, V, LPR, CH, VW, true, D16>(
                    c0 + k, h, valid, lane % LPR, col, d16, val, valid ? stage_b<T, D16>()[k] : (T)0,
                    valid ? stage_inv<T, D16>()[k] : (T)0, x, delta, lambda, w, ss_grp[warp][grp], &ws,
                    D16 ? (valid ? (int)stage_fl<T, D16>()[k] : 0) : -1, (D16 && valid) ? stage_rb<T, D16>()[k] : 0);
            }
        }
    }
    __syncthreads();
    flush_window<T>(win, W, Wp, delta, w.w0, Q);
    if (lane < G) ss = ss_grp[warp][lane];
    __shared__ double sh[32];
    const double tot = block_sum(ss, sh);   // synchronizes the CTA
    if (threadIdx.x == 0) {
        if (tot != 0.0) atomicAdd(resid_ss, tot);
        if (wobs && ws.obs) atomicMax(reinterpret_cast<unsigned*>(wobs), ws.obs);
    }
}

// ------------------------------------------------------------------ launch
template <typename T, typename V, int LPR, int CH, int VW, bool D16>
cudaError_t launch_window(const DropArgs& a, cudaStream_t s) {
    auto kern = drop_block_window_kernel<T, V, LPR, CH, VW, D16>;
    const size_t smem = window_smem_bytes(a.slice, sizeof(T), D16);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<a.grid, 1024, smem, s>>>(a.row_ptr, a.col, (const V*)a.val, (const T*)a.b, (const T*)a.inv_norm2, a.segs,
                                    a.seg_begin, a.slice, (const T*)a.x, (T*)a.delta, (T)a.lambda, a.resid_ss, a.d16,
                                    a.wlmax, a.wbound, a.wobs, a.wamax);
    return cudaGetLastError();
}

template <typename T, typename V, int LPR, int CH, int VW, bool D16>
static cudaError_t launch_cfg(const DropArgs& a, cudaStream_t s) {
    if (a.segs) {
        return launch_window<T, V, LPR, CH, VW, D16>(a, s);
    } else {
        drop_block_kernel<T, V, LPR, CH, VW, D16><<<a.grid, 256, 0, s>>>(
            a.row_ptr, a.col, (const V*)a.val, (const T*)a.b, (const T*)a.inv_norm2, a.r0, a.r1, (const T*)a.x,
            (T*)a.delta, (T)a.lambda, a.resid_ss, a.d16);
    }
    return cudaGetLastError();
}

template <typename T, typename V, bool D16>
static cudaError_t dispatch(const DropArgs& a, cudaStream_t s) {
    if (a.vector4) return cudaErrorInvalidValue;   // 4-entry vector loads measured slower; not built
    // windowed FP32 compute with a warp per row: as many register steps as the block's
    // longest row needs (window_register_steps: 8..12; longer rows finish in the tail loop),
    // so blocks of short rows do not evaluate empty steps; the schedule planner balances the
    // CTAs by the same rule
    if constexpr (sizeof(T) == 4 && (std::is_same<V, float>::value || std::is_same<V, __nv_bfloat16>::value)) {
        if (a.segs) {
            switch (window_register_steps(a.max_row, a.cdt, a.vdt, a.lanes_per_row)) {
                case 8: return launch_cfg<T, V, 32, 8, 1, D16>(a, s);
                case 9: return launch_cfg<T, V, 32, 9, 1, D16>(a, s);
                case 10: return launch_cfg<T, V, 32, 10, 1, D16>(a, s);
                case 11: return launch_cfg<T, V, 32, 11, 1, D16>(a, s);
                default: break;   // 12: the fixed depth below
            }
        }
    }
    switch (a.lanes_per_row) {
        case 4: return launch_cfg<T, V, 4, 8, 1, D16>(a, s);
        case 8: return launch_cfg<T, V, 8, 8, 1, D16>(a, s);
        case 16: return launch_cfg<T, V, 16, 10, 1, D16>(a, s);
        case 32: return launch_cfg<T, V, 32, 12, 1, D16>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ntvs
