// Grid coordinates of a canonical voxel index, p = (iz * ny + iy) * nx + ix, in 32-bit
// arithmetic (every image holds fewer than 2^31 voxels).
#pragma once
#include <cstdint>

namespace ntvs {

__device__ __forceinline__ void voxel_coords(int64_t p, int nx, int ny, int& ix, int& iy, int& iz) {
    const uint32_t u = (uint32_t)p;
    const uint32_t t = u / (uint32_t)nx;
    ix = (int)(u - t * (uint32_t)nx);
    const uint32_t z = t / (uint32_t)ny;
    iy = (int)(t - z * (uint32_t)ny);
    iz = (int)z;
}

}  // namespace ntvs
