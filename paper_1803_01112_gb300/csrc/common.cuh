// Device helpers shared by the kernel translation units.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ntvs_internal.h"

namespace ntvs {

template <typename T> struct StorageOf;
__device__ __forceinline__ float to_compute(float v) { return v; }
__device__ __forceinline__ double to_compute(double v) { return v; }
__device__ __forceinline__ float to_compute(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_compute(__nv_bfloat16 v) { return __bfloat162float(v); }

// the 16-bit value in the high half of a DELTA16 word: BF16 bits are the FP32 value's high half
template <typename V>
__device__ __forceinline__ float word_value(uint32_t e) {
    if constexpr (std::is_same<V, __nv_bfloat16>::value) return __uint_as_float(e & 0xffff0000u);
    else return __half2float(__ushort_as_half((unsigned short)(e >> 16)));
}

// fused x - s*g on the FP64 master image, spelled out so every kernel that forms a
// perturbed voxel rounds alike
__device__ __forceinline__ double perturbed(double x, double s, double g) { return __fma_rn(-s, g, x); }

// s = beta / ||g|| (0 when g = 0, i.e. v = 0)
__device__ __forceinline__ double step_scale(double beta, const double* gnorm2) {
    const double n2 = *gnorm2;
    return (n2 > 0.0) ? beta / sqrt(n2) : 0.0;
}

// internal index of canonical voxel j (see VoxMap); 32-bit arithmetic, as every index
// of either order is below 2^31
__device__ __forceinline__ int64_t vox_internal(const VoxMap& m, int64_t j) {
    if (m.tx == 1 && m.ty == 1 && !m.sw) return j;
    const uint32_t u = (uint32_t)j, nx = (uint32_t)m.nx, ny = (uint32_t)m.ny;
    const uint32_t t = u / nx, ix = u - t * nx;
    const uint32_t iz = t / ny, iy = t - iz * ny;
    const uint32_t ntx = (uint32_t)m.nxp >> m.ltx;
    const uint32_t tile = (iy >> m.lty) * ntx + (ix >> m.ltx);
    uint32_t p = (tile << (m.ltx + m.lty)) + ((iy & (uint32_t)(m.ty - 1)) << m.ltx) + (ix & (uint32_t)(m.tx - 1));
    if (m.sw) p ^= (p >> 5) & 31u;
    return (int64_t)(iz * (uint32_t)m.slice_p + p);
}

// the FP32 copies of master value v of canonical voxel j
__device__ __forceinline__ void store_copies(const ImgCopies& c, int64_t j, double v) {
    if (c.x32) c.x32[vox_internal(c.m, j)] = (float)v;
    if (c.xh) {
        const float h = (float)v;
        c.xh[j] = h;
        c.xl[j] = (float)(v - (double)h);
    }
}

// %globaltimer in nanoseconds (the clock of every bounded device-side wait)
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of v over the CTA (blockDim.x multiple of 32, <= 1024); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh /* >= 32 */) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// Deterministic grid reduction of NV values per CTA: CTA b writes partials[q*grid + b];
// the last CTA to finish sums each q in a fixed order into out[q] and resets the ticket.
// Returns true in the last CTA (all threads), after out[] is written.
template <int NV>
__device__ __forceinline__ bool grid_reduce(const double (&v)[NV], double* partials, unsigned* ticket,
                                            double* const (&out)[NV]) {
    __shared__ double sh[32];
    __shared__ bool last;
    double tot[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) tot[q] = block_sum(v[q], sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) partials[q * gridDim.x + blockIdx.x] = tot[q];
        __threadfence();
        unsigned t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double a = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) a += __ldcg(&partials[q * gridDim.x + i]);
        a = block_sum(a, sh);
        if (threadIdx.x == 0 && out[q]) *out[q] = a;
    }
    if (threadIdx.x == 0) *ticket = 0u;
    return true;
}

}  // namespace ntvs
