// Load-time preparation of the system (runs once per ntvs_load_system, outside the
// iteration): validation, FP64 row norms ||a_i||^2 of the stored values, and the
// per-block hit counts s_j^t of the block-DROP weights (Sec. III-D, DROP of ref. CEHN08).
#include "common.cuh"

namespace ntvs {

template <typename V> __device__ __forceinline__ double as_f64(V v) { return (double)to_compute(v); }

__global__ void validate_rows_kernel(const int64_t* __restrict__ row_ptr, int64_t M, int* flags) {
    int f = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
        if (row_ptr[i] > row_ptr[i + 1]) f |= 1;
    if (blockIdx.x == 0 && threadIdx.x == 0 && row_ptr[0] != 0) f |= 2;
    if (f) atomicOr(flags, f);
}

template <typename T>
__global__ void inv_counts_kernel(const int32_t* __restrict__ cnt, T* __restrict__ inv_s, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = cnt[j];
        inv_s[j] = c > 0 ? (T)(1.0 / (double)c) : (T)0;
    }
}

static int prep_grid() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (sms > 0 ? sms : 1) * 8;
}

cudaError_t k_validate_rows(const int64_t* row_ptr, int64_t M, int* flags, cudaStream_t s) {
    validate_rows_kernel<<<prep_grid(), 256, 0, s>>>(row_ptr, M, flags);
    return cudaGetLastError();
}

__global__ void remap_cols_kernel(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t nnz, VoxMap m,
                                  int* flags) {
    const int64_t V = (int64_t)m.nx * m.ny * m.nz;
    int f = 0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = in[p];
        if (c < 0 || (int64_t)c >= V) {
            f |= 4;
            out[p] = 0;
        } else {
            out[p] = (int32_t)vox_internal(m, c);
        }
    }
    if (f) atomicOr(flags, f);
}

cudaError_t k_remap_cols(const int32_t* col_in, int32_t* col_out, int64_t nnz, VoxMap m, int* flags, cudaStream_t s) {
    if (nnz <= 0) return cudaSuccess;
    remap_cols_kernel<<<prep_grid(), 256, 0, s>>>(col_in, col_out, nnz, m, flags);
    return cudaGetLastError();
}

cudaError_t k_inv_counts(const int32_t* cnt, void* inv_s, int cdt, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (cdt == F64) inv_counts_kernel<double><<<prep_grid(), 256, 0, s>>>(cnt, (double*)inv_s, n);
    else inv_counts_kernel<float><<<prep_grid(), 256, 0, s>>>(cnt, (float*)inv_s, n);
    return cudaGetLastError();
}

}  // namespace ntvs

namespace ntvs {

// ------------------------------------------------------------------ fused block pass
// One pass over the rows [r0, r1) of a block, a warp per row: flags |= 4 for a column
// outside [0, V) (the entry is then skipped), 8 for a non-finite value, 16 for a
// non-finite b; inv_norm2[i] = 1 / sum a^2 (FP64 sum of the stored values, 0 for a zero
// row); cnt[j] += 1 for every entry with a != 0.  Requires a validated row_ptr.
// With colsum != nullptr it also accumulates colsum[j] += |a_ij| (the block's column sums
// of lengths), rb[0] = max over the rows of |b_i| / ||a_i||^2 and rb[1] = max |a_ij| (as
// float bits, atomic maxima of non-negative floats): the scale statistics of the
// fixed-point DROP window.
template <typename V, typename T>
__global__ void __launch_bounds__(256) prep_block_kernel(const int64_t* __restrict__ row_ptr,
                                                         const int32_t* __restrict__ col, const V* __restrict__ val,
                                                         int64_t e0, const T* __restrict__ b, int64_t r0, int64_t r1,
                                                         int64_t nvox,
                                                         T* __restrict__ inv_norm2, int32_t* __restrict__ cnt,
                                                         int* flags, float* __restrict__ colsum, unsigned* rb) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int f = 0;
    float bmax = 0.f, amax = 0.f;
    for (int64_t i = r0 + w0; i < r1; i += nw) {
        const int64_t p0 = __ldg(row_ptr + i), p1 = __ldg(row_ptr + i + 1);
        double sq = 0.0;
#pragma unroll 4
        for (int64_t p = p0 + lane; p < p1; p += 32) {
            const int32_t c = __ldcs(col + (p - e0));
            const double a = as_f64(val[p - e0]);
            if (!isfinite(a)) f |= 8;
            sq += a * a;
            if (c < 0 || (int64_t)c >= nvox) f |= 4;
            else if (a != 0.0) {
                atomicAdd(cnt + c, 1);
                if (colsum) {
                    atomicAdd(colsum + c, (float)fabs(a));
                    amax = fmaxf(amax, (float)fabs(a));
                }
            }
        }
        sq = warp_sum(sq);
        if (lane == 0) {
            const double inv = (sq > 0.0 && isfinite(sq)) ? 1.0 / sq : 0.0;
            inv_norm2[i] = (T)inv;
            const double bi = (double)b[i];
            if (!isfinite(bi)) f |= 16;
            else bmax = fmaxf(bmax, (float)(fabs(bi) * inv));
        }
    }
    if (f) atomicOr(flags, f);
    if (rb) {
        for (int o = 16; o > 0; o >>= 1) {
            bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
            amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        }
        if (lane == 0 && bmax > 0.f) atomicMax(rb, __float_as_uint(bmax));
        if (lane == 0 && amax > 0.f) atomicMax(rb + 1, __float_as_uint(amax));
    }
}

// *out = max(*out, max_j v[j]) for non-negative v (float bits compared as unsigned)
__global__ void colmax_kernel(const float* __restrict__ v, int64_t n, unsigned* out) {
    float m = 0.f;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, v[j]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(out, __float_as_uint(m));
}

cudaError_t k_colmax(const float* v, int64_t n, float* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    colmax_kernel<<<prep_grid(), 256, 0, s>>>(v, n, reinterpret_cast<unsigned*>(out));
    return cudaGetLastError();
}

template <typename V>
static cudaError_t launch_prep(const int64_t* rp, const int32_t* col, const V* val, int64_t e0, const void* b,
                               int64_t r0, int64_t r1, int64_t nvox, void* inn, int cdt, int32_t* cnt, int* flags,
                               float* colsum, float* rb, cudaStream_t s) {
    unsigned* rbu = reinterpret_cast<unsigned*>(rb);
    if (cdt == F64)
        prep_block_kernel<V, double><<<prep_grid(), 256, 0, s>>>(rp, col, val, e0, (const double*)b, r0, r1, nvox,
                                                                 (double*)inn, cnt, flags, colsum, rbu);
    else
        prep_block_kernel<V, float><<<prep_grid(), 256, 0, s>>>(rp, col, val, e0, (const float*)b, r0, r1, nvox,
                                                                (float*)inn, cnt, flags, colsum, rbu);
    return cudaGetLastError();
}

cudaError_t k_prep_block(const int64_t* row_ptr, const int32_t* col, const void* val, int64_t e0, int vdt,
                         const void* b, int64_t r0, int64_t r1, int64_t nvox, void* inv_norm2, int cdt, int32_t* cnt,
                         int* flags, float* colsum, float* rb, cudaStream_t s) {
    if (r1 <= r0) return cudaSuccess;
    switch (vdt) {
        case F64:
            return launch_prep(row_ptr, col, (const double*)val, e0, b, r0, r1, nvox, inv_norm2, cdt, cnt, flags,
                               colsum, rb, s);
        case F32:
            return launch_prep(row_ptr, col, (const float*)val, e0, b, r0, r1, nvox, inv_norm2, cdt, cnt, flags,
                               colsum, rb, s);
        case F16:
            return launch_prep(row_ptr, col, (const __half*)val, e0, b, r0, r1, nvox, inv_norm2, cdt, cnt, flags,
                               colsum, rb, s);
        case BF16:
            return launch_prep(row_ptr, col, (const __nv_bfloat16*)val, e0, b, r0, r1, nvox, inv_norm2, cdt, cnt,
                               flags, colsum, rb, s);
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------ DELTA16 packing
// A warp per row.  A row whose columns span at most 65535 is narrow: every entry keeps its
// offset from the row's smallest column, which is the base of all of the row's chunks
// (rowesc bit 1).  Otherwise chunk by chunk: the chunk's smallest and largest column
// decide between base + 16-bit offsets and an escaped chunk of full columns (rowesc bit 0
// when the row has one).

__device__ __forceinline__ void chunk_range(const int32_t* __restrict__ col, int64_t p, int64_t p1, int32_t& c,
                                            int32_t& lo, int32_t& hi) {
    c = p < p1 ? col[p] : -1;
    lo = __reduce_min_sync(0xffffffffu, p < p1 ? c : 0x7fffffff);
    hi = __reduce_max_sync(0xffffffffu, c);
}

// smallest and largest column of row [p0, p1) (warp-uniform result; lo > hi for an empty row)
__device__ __forceinline__ void row_range(const int32_t* __restrict__ col, int64_t p0, int64_t p1, int lane,
                                          int32_t& lo, int32_t& hi) {
    lo = 0x7fffffff;
    hi = -1;
    for (int64_t pc = p0; pc < p1; pc += 32) {
        int32_t c, l, h;
        chunk_range(col, pc + lane, p1, c, l, h);
        lo = min(lo, l);
        hi = max(hi, h);
    }
}

__global__ void delta16_count_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int64_t M,
                                     unsigned long long* n_esc) {
    const int lane = threadIdx.x & 31;
    unsigned long long n = 0;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < M;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t p0 = row_ptr[i], p1 = row_ptr[i + 1];
        int32_t rlo, rhi;
        row_range(col, p0, p1, lane, rlo, rhi);
        if ((int64_t)rhi - (int64_t)rlo <= 65535) continue;   // narrow: no escaped chunk
        for (int64_t pc = p0; pc < p1; pc += 32) {
            int32_t c, lo, hi;
            chunk_range(col, pc + lane, p1, c, lo, hi);
            if ((int64_t)hi - (int64_t)lo > 65535) ++n;
        }
    }
    if (lane == 0 && n) atomicAdd(n_esc, n);
}

__global__ void delta16_fill_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int64_t M,
                                    uint16_t* __restrict__ off, int32_t* __restrict__ cbase, int32_t* __restrict__ exc,
                                    uint8_t* __restrict__ rowesc, unsigned long long* slot) {
    const int lane = threadIdx.x & 31;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < M;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t p0 = row_ptr[i], p1 = row_ptr[i + 1];
        int32_t* cb = cbase + (p0 >> 5) + i;
        int32_t rlo, rhi;
        row_range(col, p0, p1, lane, rlo, rhi);
        if ((int64_t)rhi - (int64_t)rlo <= 65535) {   // narrow row: one base for all of its chunks
            for (int64_t pc = p0, k = 0; pc < p1; pc += 32, ++k) {
                const int64_t p = pc + lane;
                if (p < p1) off[p] = (uint16_t)(col[p] - rlo);
                if (lane == 0) cb[k] = rlo;
            }
            if (lane == 0) rowesc[i] = 2;
            continue;
        }
        bool any = false;
        for (int64_t pc = p0, k = 0; pc < p1; pc += 32, ++k) {
            const int64_t p = pc + lane;
            int32_t c, lo, hi;
            chunk_range(col, p, p1, c, lo, hi);
            if ((int64_t)hi - (int64_t)lo <= 65535) {
                if (p < p1) off[p] = (uint16_t)(c - lo);
                if (lane == 0) cb[k] = lo;
            } else {
                unsigned long long e = 0;
                if (lane == 0) e = atomicAdd(slot, 1ull);
                e = __shfl_sync(0xffffffffu, e, 0);
                exc[(int64_t)(e << 5) + lane] = p < p1 ? c : 0;
                if (p < p1) off[p] = 0;
                if (lane == 0) cb[k] = -1 - (int32_t)e;
                any = true;
            }
        }
        if (lane == 0) rowesc[i] = any ? 1 : 0;
    }
}

cudaError_t k_delta16_count(const int64_t* row_ptr, const int32_t* col, int64_t M, unsigned long long* n_esc,
                            cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    delta16_count_kernel<<<prep_grid(), 256, 0, s>>>(row_ptr, col, M, n_esc);
    return cudaGetLastError();
}

cudaError_t k_delta16_fill(const int64_t* row_ptr, const int32_t* col, int64_t M, uint16_t* off, int32_t* cbase,
                           int32_t* exc, uint8_t* rowesc, unsigned long long* slot, cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    delta16_fill_kernel<<<prep_grid(), 256, 0, s>>>(row_ptr, col, M, off, cbase, exc, rowesc, slot);
    return cudaGetLastError();
}

}  // namespace ntvs

namespace ntvs {

// ------------------------------------------------------------------ row-sharded DROP
// Conversions between the internal voxel order of a block's accumulator / inverse hit
// counts and the canonical order of the public arrays (all V voxels, one pass each).

// out[j] = delta[internal(j)] (as F32 or F64), delta[internal(j)] = 0
template <typename T, typename O>
__global__ void delta_out_kernel(T* __restrict__ delta, VoxMap m, O* __restrict__ out, int64_t V) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < V; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = vox_internal(m, j);
        out[j] = (O)delta[p];
        delta[p] = (T)0;
    }
}

// x_j += d[j] * inv_s[internal(j)] on the FP64 master and its FP32 copies
template <typename T, typename D>
__global__ void apply_ext_kernel(double* __restrict__ x, ImgCopies c, const D* __restrict__ d,
                                 const T* __restrict__ inv_s, int64_t V) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < V; j += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[j] + (double)d[j] * (double)inv_s[vox_internal(c.m, j)];
        x[j] = v;
        store_copies(c, j, v);
    }
}

// counts <-> inverse counts over n slots of one order (1/(1/s) rounds back to s exactly in
// FP64, and in FP32 for every count below 2^22)
template <typename T>
__global__ void counts_from_inv_kernel(const T* __restrict__ inv_s, int32_t* __restrict__ cnt, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)inv_s[j];
        cnt[j] = v > 0.0 ? (int32_t)rint(1.0 / v) : 0;
    }
}

// the same between canonical counts and internal-order inverse counts
template <typename T>
__global__ void counts_out_kernel(const T* __restrict__ inv_s, VoxMap m, int32_t* __restrict__ cnt, int64_t V) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < V; j += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)inv_s[vox_internal(m, j)];
        cnt[j] = v > 0.0 ? (int32_t)rint(1.0 / v) : 0;
    }
}
template <typename T>
__global__ void counts_in_kernel(const int32_t* __restrict__ cnt, VoxMap m, T* __restrict__ inv_s, int64_t V) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < V; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = cnt[j];
        inv_s[vox_internal(m, j)] = s > 0 ? (T)(1.0 / (double)s) : (T)0;
    }
}

cudaError_t k_delta_out(int cdt, void* delta, VoxMap m, void* out, int odt, cudaStream_t s) {
    const int64_t V = (int64_t)m.nx * m.ny * m.nz;
    if (V <= 0) return cudaSuccess;
    if (cdt == F64 && odt == F64) delta_out_kernel<double, double><<<prep_grid(), 256, 0, s>>>((double*)delta, m, (double*)out, V);
    else if (cdt == F64 && odt == F32) delta_out_kernel<double, float><<<prep_grid(), 256, 0, s>>>((double*)delta, m, (float*)out, V);
    else if (cdt == F32 && odt == F64) delta_out_kernel<float, double><<<prep_grid(), 256, 0, s>>>((float*)delta, m, (double*)out, V);
    else if (cdt == F32 && odt == F32) delta_out_kernel<float, float><<<prep_grid(), 256, 0, s>>>((float*)delta, m, (float*)out, V);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t k_apply_ext(int cdt, double* x, ImgCopies c, const void* d, int ddt, const void* inv_s, cudaStream_t s) {
    const int64_t V = (int64_t)c.m.nx * c.m.ny * c.m.nz;
    if (V <= 0) return cudaSuccess;
    if (cdt == F64 && ddt == F64) apply_ext_kernel<double, double><<<prep_grid(), 256, 0, s>>>(x, c, (const double*)d, (const double*)inv_s, V);
    else if (cdt == F64 && ddt == F32) apply_ext_kernel<double, float><<<prep_grid(), 256, 0, s>>>(x, c, (const float*)d, (const double*)inv_s, V);
    else if (cdt == F32 && ddt == F64) apply_ext_kernel<float, double><<<prep_grid(), 256, 0, s>>>(x, c, (const double*)d, (const float*)inv_s, V);
    else if (cdt == F32 && ddt == F32) apply_ext_kernel<float, float><<<prep_grid(), 256, 0, s>>>(x, c, (const float*)d, (const float*)inv_s, V);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t k_counts_from_inv(int cdt, const void* inv_s, int32_t* cnt, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (cdt == F64) counts_from_inv_kernel<double><<<prep_grid(), 256, 0, s>>>((const double*)inv_s, cnt, n);
    else counts_from_inv_kernel<float><<<prep_grid(), 256, 0, s>>>((const float*)inv_s, cnt, n);
    return cudaGetLastError();
}

cudaError_t k_counts_out(int cdt, const void* inv_s, VoxMap m, int32_t* cnt, cudaStream_t s) {
    const int64_t V = (int64_t)m.nx * m.ny * m.nz;
    if (V <= 0) return cudaSuccess;
    if (cdt == F64) counts_out_kernel<double><<<prep_grid(), 256, 0, s>>>((const double*)inv_s, m, cnt, V);
    else counts_out_kernel<float><<<prep_grid(), 256, 0, s>>>((const float*)inv_s, m, cnt, V);
    return cudaGetLastError();
}

cudaError_t k_counts_in(int cdt, const int32_t* cnt, VoxMap m, void* inv_s, cudaStream_t s) {
    const int64_t V = (int64_t)m.nx * m.ny * m.nz;
    if (V <= 0) return cudaSuccess;
    if (cdt == F64) counts_in_kernel<double><<<prep_grid(), 256, 0, s>>>(cnt, m, (double*)inv_s, V);
    else counts_in_kernel<float><<<prep_grid(), 256, 0, s>>>(cnt, m, (float*)inv_s, V);
    return cudaGetLastError();
}

}  // namespace ntvs
