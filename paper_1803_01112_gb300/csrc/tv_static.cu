// TV value phi(x) with its reduction scratch in a file-scope device array, for callers
// that cannot allocate device memory.
//
// Who needs this: code that runs where cudaMalloc is off limits -- inside a host callback
// or a library hook that must not allocate, under a memory pool or allocator that owns
// every device allocation of the process, or on a path whose memory budget is fixed in
// advance.  ntvs_get_tv needs a context, and a context allocates its scratch; this entry
// point takes the caller's image and output pointers and allocates nothing.
//
// Scratch: kStaticCtas FP64 partials plus a ticket word, in one static __device__ array
// that every GPU loading the library holds until the process exits.  The grid is fixed by
// the image size (kVoxelsPerThread voxels per thread), so the largest image is
// kStaticCtas * 256 * kVoxelsPerThread voxels; larger images are rejected.
#include <string>

#include "common.cuh"
#include "ntvs.h"

namespace ntvs {

namespace {

constexpr int kStaticCtas = 4096;
constexpr int kVoxelsPerThread = 16;
constexpr int64_t kStaticMaxVoxels = (int64_t)kStaticCtas * kRedThreads * kVoxelsPerThread;   // 16,777,216

struct StaticScratch {
    double partials[kStaticCtas];
    unsigned ticket;
};

// Host code must not use this name as a device address: it is a host-side stand-in.
// The device address comes from cudaGetSymbolAddress on every call, below.
static __device__ __align__(256) StaticScratch g_static_scratch;

int static_fail(int code, const std::string& msg) {
    set_last_error(msg);   // read back with ntvs_last_error()
    return code;
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads)
tv_value_static_kernel(const T* __restrict__ x, int nx, int ny, int nz, StaticScratch* scratch, double* tv) {
    const int64_t sxy = (int64_t)nx * ny, V = sxy * nz;
    double acc[1] = {0.0};
    const int64_t first = (int64_t)blockIdx.x * blockDim.x * kVoxelsPerThread + threadIdx.x;
#pragma unroll 4
    for (int q = 0; q < kVoxelsPerThread; ++q) {
        const int64_t p = first + (int64_t)q * blockDim.x;
        if (p >= V) break;
        const int ix = (int)(p % nx);
        const int64_t t = p / nx;
        const int iy = (int)(t % ny), iz = (int)(t / ny);
        const double xc = (double)__ldg(x + p);
        const double ex = (ix + 1 < nx) ? (double)__ldg(x + p + 1) - xc : 0.0;
        const double ey = (iy + 1 < ny) ? (double)__ldg(x + p + nx) - xc : 0.0;
        const double ez = (iz + 1 < nz) ? (double)__ldg(x + p + sxy) - xc : 0.0;
        acc[0] += sqrt(ex * ex + ey * ey + ez * ez);
    }
    double* const outs[1] = {tv};
    grid_reduce<1>(acc, scratch->partials, &scratch->ticket, outs);
}

// Device address of the static scratch in the current device's current context.  It is
// looked up on every call (cudaGetSymbolAddress allocates nothing): each CUDA context
// loads its own copy of the module, so an address kept from an earlier call could belong
// to a context that has since been reset or is not the one current now.
int scratch_address(StaticScratch** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
        return static_fail(NTVS_ERR_CUDA, std::string("cudaGetSymbolAddress of the static TV scratch: ") +
                                              cudaGetErrorString(e));
    *out = (StaticScratch*)p;
    return NTVS_OK;
}

}  // namespace
}  // namespace ntvs

using namespace ntvs;

extern "C" int ntvs_tv_value_static(const void* x, int dtype, int nx, int ny, int nz, double* tv_out,
                                    void* cuda_stream) {
    if (!x || !tv_out) return static_fail(NTVS_ERR_ARG, "ntvs_tv_value_static: null image or output");
    if (dtype != NTVS_F64 && dtype != NTVS_F32)
        return static_fail(NTVS_ERR_ARG, "ntvs_tv_value_static: dtype must be NTVS_F64 or NTVS_F32");
    if (nx < 1 || ny < 1 || nz < 1) return static_fail(NTVS_ERR_ARG, "ntvs_tv_value_static: grid sizes must be >= 1");
    const int64_t V = (int64_t)nx * ny * nz;
    if (V > kStaticMaxVoxels)
        return static_fail(NTVS_ERR_ARG, "ntvs_tv_value_static: image of " + std::to_string(V) +
                                             " voxels exceeds the static scratch limit of " +
                                             std::to_string(kStaticMaxVoxels) + " voxels");
    StaticScratch* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != NTVS_OK) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the ticket must start at 0 (a launch that failed part-way could have left it set)
    cudaError_t e = cudaMemsetAsync(&scratch->ticket, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return static_fail(NTVS_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    const int64_t per_cta = (int64_t)kRedThreads * kVoxelsPerThread;
    const int grid = (int)((V + per_cta - 1) / per_cta);
    if (dtype == NTVS_F64)
        tv_value_static_kernel<double><<<grid, kRedThreads, 0, s>>>((const double*)x, nx, ny, nz, scratch, tv_out);
    else
        tv_value_static_kernel<float><<<grid, kRedThreads, 0, s>>>((const float*)x, nx, ny, nz, scratch, tv_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return static_fail(NTVS_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return NTVS_OK;
}
