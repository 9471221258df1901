// hough_find_fp64.cu -- the find kernel of the FP64 variant
// (HOUGH_FLAG_FP64), a translation unit of its own.
#include "hough_kernels.cuh"

namespace hk {

// Any CTA size up to 1024 threads.
__global__ void __launch_bounds__(1024, 1) find_kernel_fp64(KParams p)
{
    find_body<true>(p);
}

}  // namespace hk
