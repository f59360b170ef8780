// TV kernels: gradient of phi_eps with its FP64 norm, phi in FP64, and the perturbation
// x <- x + beta v, v = -g/||g|| (arXiv 1803.01112, Appendix A/C; phi = TV as the sum of
// local variations, introduced in Sec. II).  Forward differences on index spacing, zero past the last
// index.  The image is tiny next to the system matrix (V floats), so these kernels live
// in L2; every reduction is FP64 with a fixed reduction order (deterministic).
#include "common.cuh"
#include "voxel_coords.cuh"

namespace ntvs {

int red_grid(int64_t n, int sm_count) {
    int64_t need = (n + kRedThreads - 1) / kRedThreads;
    int64_t cap = (int64_t)sm_count * 8;
    if (need < 1) need = 1;
    return (int)(need < cap ? need : cap);
}

// One voxel of grad phi_eps:
//   g_q = -sum_a d_a(q) / D_q + sum_{a: q-e_a inside} d_a(q-e_a) / D_{q-e_a}
// with d_a(c) = x_{c+e_a} - x_c (0 past the last index) and D_c = sqrt(eps + |d(c)|^2).
// The image is the FP64 master copy; differences are formed in FP64 (so nearly equal
// neighbours keep their difference) and the rest of the arithmetic runs in T.
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
tv_grad_kernel(const double* __restrict__ x, T* __restrict__ g, int nx, int ny, int nz, T eps,
               double* partials, unsigned* ticket, double* gnorm2, double* phi) {
    const int64_t sxy = (int64_t)nx * ny, V = sxy * nz;
    double acc[2] = {0.0, 0.0};
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < V; p += (int64_t)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        voxel_coords(p, nx, ny, ix, iy, iz);
        const bool hx = ix + 1 < nx, hy = iy + 1 < ny, hz = iz + 1 < nz;
        const double xc = __ldg(x + p);
        const double ex = hx ? __ldg(x + p + 1) - xc : 0.0;
        const double ey = hy ? __ldg(x + p + nx) - xc : 0.0;
        const double ez = hz ? __ldg(x + p + sxy) - xc : 0.0;
        const T dx = (T)ex, dy = (T)ey, dz = (T)ez;
        const T D = sqrt(eps + (dx * dx + dy * dy + dz * dz));
        T gq = (D > (T)0) ? -(dx + dy + dz) / D : (T)0;
        if (ix > 0) {
            const double xm = __ldg(x + p - 1);
            const T a = (T)(xc - xm);
            const T b = hy ? (T)(__ldg(x + p - 1 + nx) - xm) : (T)0;
            const T c = hz ? (T)(__ldg(x + p - 1 + sxy) - xm) : (T)0;
            const T Dm = sqrt(eps + (a * a + b * b + c * c));
            if (Dm > (T)0) gq += a / Dm;
        }
        if (iy > 0) {
            const double xm = __ldg(x + p - nx);
            const T a = (T)(xc - xm);
            const T b = hx ? (T)(__ldg(x + p - nx + 1) - xm) : (T)0;
            const T c = hz ? (T)(__ldg(x + p - nx + sxy) - xm) : (T)0;
            const T Dm = sqrt(eps + (a * a + b * b + c * c));
            if (Dm > (T)0) gq += a / Dm;
        }
        if (iz > 0) {
            const double xm = __ldg(x + p - sxy);
            const T a = (T)(xc - xm);
            const T b = hx ? (T)(__ldg(x + p - sxy + 1) - xm) : (T)0;
            const T c = hy ? (T)(__ldg(x + p - sxy + nx) - xm) : (T)0;
            const T Dm = sqrt(eps + (a * a + b * b + c * c));
            if (Dm > (T)0) gq += a / Dm;
        }
        g[p] = gq;
        acc[0] += (double)gq * (double)gq;
        if (phi) acc[1] += sqrt(ex * ex + ey * ey + ez * ez);
    }
    double* const outs[2] = {gnorm2, phi};
    grid_reduce<2>(acc, partials, ticket, outs);
}

// The same gradient on the FP32 path from the split copies xh + xl of the master image:
// every neighbour difference is (xh_a - xh_b) + (xl_a - xl_b) in FP32, so the stencil runs
// without FP64 arithmetic (only ||g||^2 is accumulated in FP64).
__global__ void __launch_bounds__(kRedThreads)
tv_grad_split_kernel(const float* __restrict__ xh, const float* __restrict__ xl, float* __restrict__ g, int nx,
                     int ny, int nz, float eps, double* partials, unsigned* ticket, double* gnorm2) {
    const int64_t sxy = (int64_t)nx * ny, V = sxy * nz;
    auto dif = [&](int64_t a, int64_t b) -> float {
        return (__ldg(xh + a) - __ldg(xh + b)) + (__ldg(xl + a) - __ldg(xl + b));
    };
    double acc[1] = {0.0};
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < V; p += (int64_t)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        voxel_coords(p, nx, ny, ix, iy, iz);
        const bool hx = ix + 1 < nx, hy = iy + 1 < ny, hz = iz + 1 < nz;
        const float dx = hx ? dif(p + 1, p) : 0.f, dy = hy ? dif(p + nx, p) : 0.f, dz = hz ? dif(p + sxy, p) : 0.f;
        const float D = sqrtf(eps + (dx * dx + dy * dy + dz * dz));
        float gq = (D > 0.f) ? -(dx + dy + dz) / D : 0.f;
        if (ix > 0) {
            const int64_t q = p - 1;
            const float a = dif(p, q), b = hy ? dif(q + nx, q) : 0.f, c = hz ? dif(q + sxy, q) : 0.f;
            const float Dm = sqrtf(eps + (a * a + b * b + c * c));
            if (Dm > 0.f) gq += a / Dm;
        }
        if (iy > 0) {
            const int64_t q = p - nx;
            const float a = dif(p, q), b = hx ? dif(q + 1, q) : 0.f, c = hz ? dif(q + sxy, q) : 0.f;
            const float Dm = sqrtf(eps + (a * a + b * b + c * c));
            if (Dm > 0.f) gq += a / Dm;
        }
        if (iz > 0) {
            const int64_t q = p - sxy;
            const float a = dif(p, q), b = hx ? dif(q + 1, q) : 0.f, c = hy ? dif(q + nx, q) : 0.f;
            const float Dm = sqrtf(eps + (a * a + b * b + c * c));
            if (Dm > 0.f) gq += a / Dm;
        }
        g[p] = gq;
        acc[0] += (double)gq * (double)gq;
    }
    double* const outs[1] = {gnorm2};
    grid_reduce<1>(acc, partials, ticket, outs);
}

// phi_0(z), z = x - sc*g (z = x if g is null), FP64 from the master image.
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
tv_value_kernel(const double* __restrict__ x, const T* __restrict__ g, const double* gnorm2, double beta, int nx,
                int ny, int nz, double* partials, unsigned* ticket, double* phi, const double* phi_ref, int* accept) {
    const int64_t sxy = (int64_t)nx * ny, V = sxy * nz;
    const double sc = g ? step_scale(beta, gnorm2) : 0.0;
    double acc[1] = {0.0};
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < V; p += (int64_t)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        voxel_coords(p, nx, ny, ix, iy, iz);
        auto zat = [&](int64_t q) -> double {
            return g ? perturbed(__ldg(x + q), sc, (double)__ldg(g + q)) : __ldg(x + q);
        };
        const double zc = zat(p);
        const double ex = (ix + 1 < nx) ? zat(p + 1) - zc : 0.0;
        const double ey = (iy + 1 < ny) ? zat(p + nx) - zc : 0.0;
        const double ez = (iz + 1 < nz) ? zat(p + sxy) - zc : 0.0;
        acc[0] += sqrt(ex * ex + ey * ey + ez * ez);
    }
    double* const outs[1] = {phi};
    if (grid_reduce<1>(acc, partials, ticket, outs)) {
        if (threadIdx.x == 0 && phi_ref && accept) {
            __threadfence();
            *accept = (__ldcg(phi) <= *phi_ref) ? 1 : 0;
        }
    }
}

// x <- x - sc*g on the master image (and its FP32 gather copy when present)
template <typename T>
__global__ void tv_apply_kernel(double* __restrict__ x, ImgCopies c, const T* __restrict__ g, const double* gnorm2,
                                double beta, const int* accept, int64_t V) {
    if (accept && *accept == 0) return;
    const double sc = step_scale(beta, gnorm2);
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < V; p += (int64_t)gridDim.x * blockDim.x) {
        const double z = perturbed(x[p], sc, (double)g[p]);
        x[p] = z;
        store_copies(c, p, z);
    }
}

__global__ void x32_from_x64_kernel(const double* __restrict__ x, ImgCopies c) {
    const int64_t V = (int64_t)c.m.nx * c.m.ny * c.m.nz;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < V; j += (int64_t)gridDim.x * blockDim.x)
        store_copies(c, j, x[j]);
}

static int g_sm_count = 0;
static int sm_count() {
    if (!g_sm_count) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (g_sm_count <= 0) g_sm_count = 1;
    }
    return g_sm_count;
}

cudaError_t k_tv_grad(int cdt, const double* x, const float* xh, const float* xl, void* g, int nx, int ny, int nz,
                      double eps, RedScratch r, double* gnorm2, double* phi, cudaStream_t s) {
    if (cdt == F32 && xh && xl && !phi)
        tv_grad_split_kernel<<<r.grid, kRedThreads, 0, s>>>(xh, xl, (float*)g, nx, ny, nz, (float)eps, r.partials,
                                                           r.ticket, gnorm2);
    else if (cdt == F64)
        tv_grad_kernel<double><<<r.grid, kRedThreads, 0, s>>>(x, (double*)g, nx, ny, nz, eps, r.partials, r.ticket,
                                                              gnorm2, phi);
    else
        tv_grad_kernel<float><<<r.grid, kRedThreads, 0, s>>>(x, (float*)g, nx, ny, nz, (float)eps, r.partials,
                                                             r.ticket, gnorm2, phi);
    return cudaGetLastError();
}

cudaError_t k_tv_value(int cdt, const double* x, const void* g, const double* gnorm2, double beta, int nx, int ny,
                       int nz, RedScratch r, double* phi, const double* phi_ref, int* accept, cudaStream_t s) {
    if (cdt == F64)
        tv_value_kernel<double><<<r.grid, kRedThreads, 0, s>>>(x, (const double*)g, gnorm2, beta, nx, ny, nz,
                                                               r.partials, r.ticket, phi, phi_ref, accept);
    else
        tv_value_kernel<float><<<r.grid, kRedThreads, 0, s>>>(x, (const float*)g, gnorm2, beta, nx, ny, nz,
                                                              r.partials, r.ticket, phi, phi_ref, accept);
    return cudaGetLastError();
}

cudaError_t k_tv_apply(int cdt, double* x, ImgCopies c, const void* g, const double* gnorm2, double beta,
                       const int* accept, int64_t V, cudaStream_t s) {
    const int grid = red_grid(V, sm_count());
    if (cdt == F64)
        tv_apply_kernel<double><<<grid, kRedThreads, 0, s>>>(x, c, (const double*)g, gnorm2, beta, accept, V);
    else
        tv_apply_kernel<float><<<grid, kRedThreads, 0, s>>>(x, c, (const float*)g, gnorm2, beta, accept, V);
    return cudaGetLastError();
}

cudaError_t k_x32_from_x64(const double* x, ImgCopies c, cudaStream_t s) {
    const int64_t V = (int64_t)c.m.nx * c.m.ny * c.m.nz;
    x32_from_x64_kernel<<<red_grid(V, sm_count()), kRedThreads, 0, s>>>(x, c);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ conversions
template <typename S, typename D>
__global__ void convert_kernel(const S* __restrict__ src, D* __restrict__ dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (D)src[i];
}

cudaError_t k_convert(const void* src, int sdt, void* dst, int ddt, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int grid = red_grid(n, sm_count());
    if (sdt == F64 && ddt == F32) convert_kernel<double, float><<<grid, 256, 0, s>>>((const double*)src, (float*)dst, n);
    else if (sdt == F32 && ddt == F64) convert_kernel<float, double><<<grid, 256, 0, s>>>((const float*)src, (double*)dst, n);
    else if (sdt == ddt) return cudaMemcpyAsync(dst, src, (size_t)n * dt_size(sdt), cudaMemcpyDeviceToDevice, s);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace ntvs
