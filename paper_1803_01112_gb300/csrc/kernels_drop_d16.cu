// Block-DROP on DELTA16 index storage (P_T of arXiv 1803.01112 Appendix C; DROP of ref.
// CEHN08, Sec. III-D): the kernels of kernels_drop.cuh with each column decoded as the
// 16-bit offset of the entry plus the base of its 32-entry chunk.  A separate translation
// unit so that the two storages compile in parallel.
#include "kernels_drop.cuh"

namespace ntvs {

cudaError_t k_drop_block_d16(const DropArgs& a, cudaStream_t s) {
    if (a.r1 <= a.r0) return cudaSuccess;
    if (a.cdt == F64) {   // FP64 arithmetic on FP64 or FP32 storage
        if (a.vdt == F64) return dispatch<double, double, true>(a, s);
        if (a.vdt == F32) return dispatch<double, float, true>(a, s);
        return cudaErrorInvalidValue;
    }
    switch (a.vdt) {
        case F32: return dispatch<float, float, true>(a, s);
        case F16: return dispatch<float, __half, true>(a, s);
        case BF16: return dispatch<float, __nv_bfloat16, true>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ntvs
