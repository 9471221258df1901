// hough_encode.cuh -- step A alone (hough_encode), included by hough_api.cu.
#pragma once

#include "hough_kernels.cuh"

namespace hk {

// Step A alone: strip addresses -> fixed-point (phi, z).
__global__ void encode_kernel(const int32_t *vane, const int32_t *strip, long long n, int vane_step,
                              int z_min_u, int z_pitch_u, int z_half, int32_t *phi_q, int32_t *z_q)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        phi_q[i] = (int32_t)((long long)vane_step * (long long)__ldg(vane + i));
        z_q[i] = (int32_t)((long long)z_min_u + (long long)z_pitch_u * (long long)__ldg(strip + i) +
                           z_half);
    }
}

}  // namespace hk
