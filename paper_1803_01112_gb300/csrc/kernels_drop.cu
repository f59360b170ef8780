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
#include "kernels_drop.cuh"

namespace ntvs {

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

int64_t k_window_smem_bytes(int64_t slice, int csz, bool d16) {
    return (int64_t)window_smem_bytes(slice, (size_t)csz, d16);
}

cudaError_t k_drop_block(const DropArgs& a, cudaStream_t s) {
    if (a.r1 <= a.r0) return cudaSuccess;
    if (a.use_d16) return k_drop_block_d16(a, s);
    if (a.cdt == F64) {   // FP64 arithmetic on FP64 or FP32 storage
        if (a.vector4) return cudaErrorInvalidValue;
        if (a.vdt == F64) return dispatch<double, double, false>(a, s);
        if (a.vdt == F32) return dispatch<double, float, false>(a, s);
        return cudaErrorInvalidValue;
    }
    switch (a.vdt) {
        case F32: return dispatch<float, float, false>(a, s);
        case F16: return dispatch<float, __half, false>(a, s);
        case BF16: return dispatch<float, __nv_bfloat16, false>(a, s);
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

// out_i = <a_i, x> for rows [0, M), a warp per row (x in the gather order of the stored
// columns), for CSR32 (packed pairs for FP32 values) or DELTA16 storage (words for 16-bit
// values); accumulated in the compute type T.
template <typename T, typename V, bool D16>
__global__ void __launch_bounds__(256)
project_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, Delta16 d16,
               const V* __restrict__ val, int64_t M, const T* __restrict__ x, T* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < M; i += nw) {
        const int64_t p0 = __ldg(row_ptr + i), p1 = __ldg(row_ptr + i + 1);
        const int32_t* cbr = D16 ? d16.cbase + (p0 >> 5) + i : nullptr;
        T acc = (T)0;
        for (int64_t p = p0 + lane; p < p1; p += 32) {
            int32_t c;
            T a;
            entry_any<T, V, D16>(col, d16, val, cbr, p, (int)(p - p0), c, a);
            acc += a * __ldg(x + c);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) out[i] = acc;
    }
}

template <typename T, typename V>
static cudaError_t launch_project(const DropArgs& a, int64_t M, const void* x, void* out, cudaStream_t s) {
    if (a.use_d16)
        project_kernel<T, V, true><<<a.grid, 256, 0, s>>>(a.row_ptr, a.col, a.d16, (const V*)a.val, M,
                                                          (const T*)x, (T*)out);
    else
        project_kernel<T, V, false><<<a.grid, 256, 0, s>>>(a.row_ptr, a.col, a.d16, (const V*)a.val, M,
                                                           (const T*)x, (T*)out);
    return cudaGetLastError();
}

// ent[p] = {col[p], bits of val[p]} for entries [0, n)
__global__ void pack_entries_kernel(const int32_t* __restrict__ col, const float* __restrict__ val, int64_t n,
                                    int2* __restrict__ ent) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        ent[p] = make_int2(__ldcs(col + p), __float_as_int(__ldcs(val + p)));
}

cudaError_t k_pack_entries(const int32_t* col, const float* val, int64_t n, int32_t* ent, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t need = (n + 255) / 256;
    const int grid = (int)(need < 4096 ? need : 4096);
    pack_entries_kernel<<<grid, 256, 0, s>>>(col, val, n, reinterpret_cast<int2*>(ent));
    return cudaGetLastError();
}

// word[p] = off[p] | val[p] << 16 (16-bit value bits) for entries [0, n)
__global__ void pack_words_kernel(const uint16_t* __restrict__ off, const uint16_t* __restrict__ val, int64_t n,
                                  uint32_t* __restrict__ word) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        word[p] = (uint32_t)__ldcs(off + p) | ((uint32_t)__ldcs(val + p) << 16);
}

cudaError_t k_pack_words(const uint16_t* off, const uint16_t* val, int64_t n, uint32_t* word, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t need = (n + 255) / 256;
    const int grid = (int)(need < 4096 ? need : 4096);
    pack_words_kernel<<<grid, 256, 0, s>>>(off, val, n, word);
    return cudaGetLastError();
}

cudaError_t k_project(const DropArgs& a, int64_t M, const void* x, void* out, cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    if (a.cdt == F64) {
        if (a.vdt == F64) return launch_project<double, double>(a, M, x, out, s);
        if (a.vdt == F32) return launch_project<double, float>(a, M, x, out, s);
        return cudaErrorInvalidValue;
    }
    switch (a.vdt) {
        case F32: return launch_project<float, float>(a, M, x, out, s);
        case F16: return launch_project<float, __half>(a, M, x, out, s);
        case BF16: return launch_project<float, __nv_bfloat16>(a, M, x, out, s);
        default: return cudaErrorInvalidValue;
    }
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
// slice it enters and leaves by.  Entry p's column is col[stride * p] (stride 2: the
// packed pairs).
__global__ void row_home_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int stride,
                                int64_t M, int64_t slice, int32_t* __restrict__ home) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p0 = row_ptr[i], p1 = row_ptr[i + 1];
        if (p1 <= p0) { home[i] = -1; continue; }
        const int32_t a = (int32_t)(col[stride * p0] / slice), m = (int32_t)(col[stride * (p0 + (p1 - p0) / 2)] / slice),
                      c = (int32_t)(col[stride * (p1 - 1)] / slice);
        home[i] = max(min(a, m), min(max(a, m), c));
    }
}

cudaError_t k_row_home(const int64_t* row_ptr, const int32_t* col, int stride, int64_t M, int64_t slice, int32_t* home,
                       int grid, cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    row_home_kernel<<<grid, 256, 0, s>>>(row_ptr, col, stride, M, slice, home);
    return cudaGetLastError();
}

// A warp per chunk of rows: the chunk's work in issued register steps (k_chunk_cost); a
// chunk of a block without a per-block depth (ch = 0) counts its rows
__global__ void chunk_cost_kernel(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ cs,
                                  const int8_t* __restrict__ ch, int mid, int64_t nchunks, int64_t* __restrict__ cost) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q = w0; q < nchunks; q += nw) {
        const int64_t r0 = cs[q], r1 = cs[q + 1];
        const int64_t d = ch[q];
        long long acc = 0;
        for (int64_t i = r0 + lane; i < r1; i += 32) {
            if (d <= 0) {
                acc += 4;
                continue;
            }
            const int64_t steps = (row_ptr[i + 1] - row_ptr[i] + 31) / 32;
            const int64_t body = (steps <= kShortBody && d > kShortBody) ? kShortBody
                                 : (mid > 0 && d > mid && steps <= mid) ? mid : d;
            const int64_t live = steps < body ? steps : body;
            acc += 4 + 4 * live + (body - live) + 8 * (steps > d ? steps - d : 0);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) cost[q] = acc;
    }
}

cudaError_t k_chunk_cost(const int64_t* row_ptr, const int64_t* cs, const int8_t* ch, int mid, int64_t nchunks,
                         int64_t* cost, int grid, cudaStream_t s) {
    if (nchunks <= 0) return cudaSuccess;
    chunk_cost_kernel<<<grid, 256, 0, s>>>(row_ptr, cs, ch, mid, nchunks, cost);
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
