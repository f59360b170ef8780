// Block-DROP kernels (P_T of arXiv 1803.01112 Appendix C; DROP of ref. CEHN08, Sec. II-D).
//
// drop_block: for every row i of block t (all rows see the same x):
//     d_i = <a_i, x>                    (CSR gather, x is L2-resident)
//     r_i = lambda (b_i - d_i) / ||a_i||^2
//     delta_j += r_i a_ij               (scatter-add, fire-and-forget L2 reductions)
//   A group of LPR lanes owns a row; the row's entries stay in registers between the
//   dot product and the scatter, so the matrix streams from HBM exactly once.
// drop_apply: x_j += delta_j / s_j^t (inverse counts precomputed), delta_j = 0.
#include "common.cuh"

namespace ntvs {

template <typename T> __device__ __forceinline__ void red_add(T* p, T v) { atomicAdd(p, v); }

// CH chunks of LPR entries per row are kept in registers; longer rows re-read the tail.
template <typename T, typename V, int LPR, int CH>
__global__ void __launch_bounds__(256)
drop_block_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, const V* __restrict__ val,
                  const T* __restrict__ b, const T* __restrict__ inv_norm2, int64_t r0, int64_t r1,
                  const T* __restrict__ x, T* __restrict__ delta, T lambda, double* resid_ss) {
    constexpr int G = 32 / LPR;   // rows per warp pass
    const int lane = threadIdx.x & 31;
    const int sub = lane % LPR;
    const int grp = lane / LPR;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double ss = 0.0;
    for (int64_t base = r0 + warp * G; base < r1; base += nwarps * G) {
        const int64_t i = base + grp;
        const bool valid = i < r1;
        int64_t p0 = 0, p1 = 0;
        if (valid) { p0 = __ldg(row_ptr + i); p1 = __ldg(row_ptr + i + 1); }
        int32_t c[CH];
        T a[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const int64_t p = p0 + sub + (int64_t)u * LPR;
            if (p < p1) { c[u] = __ldcs(col + p); a[u] = (T)to_compute(val[p]); }
            else { c[u] = -1; a[u] = (T)0; }
        }
        T acc = (T)0;
#pragma unroll
        for (int u = 0; u < CH; ++u)
            if (c[u] >= 0) acc += a[u] * __ldg(x + c[u]);
        for (int64_t p = p0 + sub + (int64_t)CH * LPR; p < p1; p += LPR)
            acc += (T)to_compute(val[p]) * __ldg(x + col[p]);
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        T r = (T)0;
        if (valid) {
            const T res = __ldg(b + i) - acc;
            r = lambda * res * __ldg(inv_norm2 + i);
            if (sub == 0) ss += (double)res * (double)res;
        }
#pragma unroll
        for (int u = 0; u < CH; ++u)
            if (c[u] >= 0) red_add(delta + c[u], r * a[u]);
        for (int64_t p = p0 + sub + (int64_t)CH * LPR; p < p1; p += LPR)
            red_add(delta + col[p], r * (T)to_compute(val[p]));
    }
    __shared__ double sh[32];
    const double tot = block_sum(ss, sh);
    if (threadIdx.x == 0 && tot != 0.0) atomicAdd(resid_ss, tot);
}

template <typename T>
__global__ void drop_apply_kernel(double* __restrict__ x, float* __restrict__ x32, T* __restrict__ delta,
                                  const T* __restrict__ inv_s, int64_t V) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < V; j += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[j] + (double)delta[j] * (double)__ldg(inv_s + j);
        x[j] = v;
        if (x32) x32[j] = (float)v;
        delta[j] = (T)0;
    }
}

template <typename T, typename V, int LPR, int CH>
static void launch_block(const DropArgs& a, cudaStream_t s) {
    drop_block_kernel<T, V, LPR, CH><<<a.grid, 256, 0, s>>>(
        a.row_ptr, a.col, (const V*)a.val, (const T*)a.b, (const T*)a.inv_norm2, a.r0, a.r1, (const T*)a.x,
        (T*)a.delta, (T)a.lambda, a.resid_ss);
}

template <typename T, typename V>
static cudaError_t dispatch_lpr(const DropArgs& a, cudaStream_t s) {
    switch (a.lanes_per_row) {
        case 4: launch_block<T, V, 4, 8>(a, s); break;
        case 8: launch_block<T, V, 8, 8>(a, s); break;
        case 16: launch_block<T, V, 16, 10>(a, s); break;
        case 32: launch_block<T, V, 32, 12>(a, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t k_drop_block(const DropArgs& a, cudaStream_t s) {
    if (a.r1 <= a.r0) return cudaSuccess;
    if (a.cdt == F64) {
        if (a.vdt != F64) return cudaErrorInvalidValue;
        return dispatch_lpr<double, double>(a, s);
    }
    switch (a.vdt) {
        case F32: return dispatch_lpr<float, float>(a, s);
        case F16: return dispatch_lpr<float, __half>(a, s);
        case BF16: return dispatch_lpr<float, __nv_bfloat16>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t k_drop_apply(int cdt, double* x, float* x32, void* delta, const void* inv_s, int64_t V, int grid,
                         cudaStream_t s) {
    if (cdt == F64) drop_apply_kernel<double><<<grid, 256, 0, s>>>(x, x32, (double*)delta, (const double*)inv_s, V);
    else drop_apply_kernel<float><<<grid, 256, 0, s>>>(x, x32, (float*)delta, (const float*)inv_s, V);
    return cudaGetLastError();
}

}  // namespace ntvs
