// probe.cu -- measures the shared-memory atomic throughput of the GPU, the
// ceiling of the Hough vote loop (each vote is one 32-bit shared atomicAdd).
//
// Every lane adds into its own row of a 32 x 33 word array, so the 32 lanes of
// a warp always hit 32 distinct banks (no bank conflict, no same-address
// conflict): the best case the vote loop's layout aims for.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__global__ void __launch_bounds__(1024) smem_atomic_probe(int iters, unsigned *sink)
{
    __shared__ unsigned s[32 * 33];
    for (int i = threadIdx.x; i < 32 * 33; i += blockDim.x)
        s[i] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned *row = s + lane * 33;
    const int b = warp & 31;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            atomicAdd(row + ((b + k) & 31), 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0)
        sink[blockIdx.x] = s[0] + s[32 * 33 - 1];
}

}  // namespace

extern "C" {

// Runs the probe on the current device; *gops receives 10^9 atomics per second.
// Returns 0 or a CUDA error code.
int hough_probe_smem_atomics(int iters, int blocks_per_sm, int threads, double *gops, double *ms_out)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -1;
    if (iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 8 || threads < 32 || threads > 1024 ||
        threads % 32 != 0)
        return -2;
    int grid = sms * blocks_per_sm;
    unsigned *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(unsigned) * grid) != cudaSuccess)
        return -3;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    smem_atomic_probe<<<grid, threads>>>(iters / 4 + 1, sink);   // warm-up
    cudaEventRecord(e0);
    smem_atomic_probe<<<grid, threads>>>(iters, sink);
    cudaEventRecord(e1);
    int rc = cudaEventSynchronize(e1) == cudaSuccess ? 0 : -4;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc == 0) {
        double n = (double)grid * threads * (double)iters * 8.0;
        *gops = n / (ms * 1e-3) / 1e9;
        if (ms_out)
            *ms_out = ms;
    }
    return rc;
}

}  // extern "C"
