// hough_find.cu -- the fixed-point find kernels (a translation unit of their
// own, compiled in parallel with the rest of libhough).
#include "hough_kernels.cuh"

namespace hk {

// Any CTA size up to 1024 threads (64 registers a thread).
__global__ void __launch_bounds__(1024, 1) find_kernel(KParams p)
{
    find_body<false>(p);
}

// CTAs of at most 256 threads, three per SM: up to 80 registers a thread
// instead of 64, so that the vote loop and the candidate test keep their
// operands in registers (6% faster on the batched pileup windows).
__global__ void __launch_bounds__(256, 3) find_kernel_256(KParams p)
{
    find_body<false>(p);
}

}  // namespace hk
