// The TV-reduction check decided on the device (arXiv 1803.01112, Appendix C, NTVS with
// the TV check; Sec. III-B on the cost of its branches).
//
// One cycle of the checked variant: ell_k = rand(k, ell_{k-1}) (or ell_{k-1} under the
// OTVS rule, Appendix B), then for each of the N steps the gradient kernel forms g and
// phi(x), and one cooperative launch runs the whole retry loop:
//     try t: z = x - beta_t g/||g||, beta_t = beta0 * alpha^(ell + t)
//            phi(z) (FP64, a fixed reduction order); accept if phi(z) <= phi(x)
//            ell += 1 after every try, the accepted one included
//     on accept x <- z (and its FP32 copies); at most max_retries tries.
// The CTAs meet at one grid barrier per try (partials of phi(z) double-buffered by try
// parity, so one barrier suffices); after it every CTA sums the same partials in the
// same order, so all of them take the same decision without a second barrier.  The
// barrier wait is bounded by %globaltimer: on expiry the CTA records an error code and
// leaves (the host reports NTVS_ERR_TIMEOUT).  Nothing is read back per try: the host
// reads the traces (tries, accepted, ell_k) when it asks for them.
#include "common.cuh"
#include "step_rule.h"

namespace ntvs {

namespace {

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier of a co-resident grid on a monotone arrival counter: the CTA arrives
// (unless `skip`, a test hook that starves the barrier) and waits until `target`
// arrivals, at most wait_ns.  Returns false in every thread of a CTA that gave up.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target, uint64_t wait_ns, int* err, bool skip) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        if (!skip) atomicAdd(bar, 1u);
        if (ld_acquire(bar) < target) {
            const uint64_t t0 = globaltimer_ns();
            while (ld_acquire(bar) < target) {
                if (globaltimer_ns() - t0 > wait_ns) {
                    atomicExch(err, kErrCheckBarrier);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

__global__ void check_cycle_begin_kernel(CheckState* st, int rule, uint64_t seed, int64_t k, int has_override,
                                         int64_t override_ell, int64_t* ell_slot) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int64_t prev = st->ell;
    const int64_t ell = has_override ? override_ell : (rule == NTVS_STEP_OTVS ? prev : draw_ell(seed, k, prev));
    st->ell = ell;
    *ell_slot = ell;
}

// phi_0 contribution of voxel p of z = x - sc*g (the forward-difference length at p)
template <typename T>
__device__ __forceinline__ double phi_z_at(const double* __restrict__ x, const T* __restrict__ g, double sc, int64_t p,
                                           int nx, int ny, int nz, int64_t sxy) {
    int ix, iy, iz;
    {
        const uint32_t u = (uint32_t)p, t = u / (uint32_t)nx;
        ix = (int)(u - t * (uint32_t)nx);
        iz = (int)(t / (uint32_t)ny);
        iy = (int)(t - (uint32_t)iz * (uint32_t)ny);
    }
    auto zat = [&](int64_t q) -> double { return perturbed(__ldg(x + q), sc, (double)__ldg(g + q)); };
    const double zc = zat(p);
    const double ex = (ix + 1 < nx) ? zat(p + 1) - zc : 0.0;
    const double ey = (iy + 1 < ny) ? zat(p + nx) - zc : 0.0;
    const double ez = (iz + 1 < nz) ? zat(p + sxy) - zc : 0.0;
    return sqrt(ex * ex + ey * ey + ez * ez);
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads)
tv_check_loop_kernel(double* __restrict__ x, ImgCopies c, const T* __restrict__ g, const double* gnorm2,
                     const double* phi_x, CheckState* st, const double* __restrict__ beta_tab, int tab_len,
                     double beta0, double alpha, int max_retries, double* partials, int* err, uint64_t wait_ns,
                     int starve, int32_t* tries_out, int32_t* acc_out, int nx, int ny, int nz) {
    __shared__ double sh[32];
    __shared__ double tot_sh;
    const int64_t sxy = (int64_t)nx * ny, V = sxy * nz;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double n2 = *gnorm2, phi_ref = *phi_x;
    int64_t ell = st->ell;   // read by every CTA before its first barrier arrival
    int tries = 0, acc = 0;
    bool ok = true;
    for (int t = 0; t < max_retries; ++t) {
        const double beta = (ell >= 0 && ell < tab_len) ? beta_tab[ell] : beta0 * pow(alpha, (double)ell);
        const double sc = (n2 > 0.0) ? beta / sqrt(n2) : 0.0;
        double tot;
        if (sc == 0.0) {
            tot = phi_ref;   // z = x: phi(z) = phi(x) exactly, a tie, accepted below
        } else {
            double a = 0.0;
            for (int64_t p = first; p < V; p += stride) a += phi_z_at<T>(x, g, sc, p, nx, ny, nz, sxy);
            const double cta = block_sum(a, sh);
            double* buf = partials + (size_t)(t & 1) * gridDim.x;
            if (threadIdx.x == 0) buf[blockIdx.x] = cta;
            ok = grid_barrier(&st->bar, (unsigned)(t + 1) * gridDim.x, wait_ns, err,
                              starve != 0 && blockIdx.x == 0 && t == 0);
            if (!ok) break;
            double part = 0.0;
            for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) part += __ldcg(buf + i);
            const double s = block_sum(part, sh);
            if (threadIdx.x == 0) tot_sh = s;
            __syncthreads();
            tot = tot_sh;
        }
        ell += 1;
        tries += 1;
        if (tot <= phi_ref) {   // ties accept
            acc = 1;
            if (sc != 0.0) {
                for (int64_t p = first; p < V; p += stride) {
                    const double z = perturbed(x[p], sc, (double)g[p]);
                    x[p] = z;
                    store_copies(c, p, z);
                }
            }
            break;
        }
    }
    if (ok && blockIdx.x == 0 && threadIdx.x == 0) {
        st->ell = ell;
        *tries_out = tries;
        *acc_out = acc;
    }
}

}  // namespace

cudaError_t k_check_cycle_begin(CheckState* st, int rule, uint64_t seed, int64_t k, bool has_override,
                                int64_t override_ell, int64_t* ell_slot, cudaStream_t s) {
    check_cycle_begin_kernel<<<1, 32, 0, s>>>(st, rule, seed, k, has_override ? 1 : 0, override_ell, ell_slot);
    return cudaGetLastError();
}

int check_loop_max_grid(int cdt, int sms) {
    int per = 0;
    cudaError_t e = (cdt == F64)
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tv_check_loop_kernel<double>, kRedThreads, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tv_check_loop_kernel<float>, kRedThreads, 0);
    if (e != cudaSuccess || per < 1) return 0;
    return per * sms;
}

cudaError_t k_tv_check_loop(const CheckLoopArgs& a, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(&a.st->bar, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    double* x = a.x;
    ImgCopies c = a.copies;
    const double* gn = a.gnorm2;
    const double* px = a.phi_x;
    CheckState* st = a.st;
    const double* tab = a.beta_tab;
    int tab_len = a.tab_len;
    double beta0 = a.beta0, alpha = a.alpha;
    int mr = a.max_retries;
    double* part = a.partials;
    int* err = a.err;
    uint64_t wns = a.wait_ns;
    int starve = a.starve;
    int32_t* to = a.tries_out;
    int32_t* ao = a.acc_out;
    int nx = a.nx, ny = a.ny, nz = a.nz;
    if (a.cdt == F64) {
        const double* g = (const double*)a.g;
        void* args[] = {&x, &c, &g, &gn, &px, &st, &tab, &tab_len, &beta0, &alpha, &mr, &part, &err, &wns, &starve,
                        &to, &ao, &nx, &ny, &nz};
        return cudaLaunchCooperativeKernel((const void*)tv_check_loop_kernel<double>, a.grid, kRedThreads, args, 0, s);
    }
    const float* g = (const float*)a.g;
    void* args[] = {&x, &c, &g, &gn, &px, &st, &tab, &tab_len, &beta0, &alpha, &mr, &part, &err, &wns, &starve,
                    &to, &ao, &nx, &ny, &nz};
    return cudaLaunchCooperativeKernel((const void*)tv_check_loop_kernel<float>, a.grid, kRedThreads, args, 0, s);
}

}  // namespace ntvs
