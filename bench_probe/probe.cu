// probe.cu -- measures the shared-memory atomic throughput of the GPU, the
// ceiling of the Hough vote loop (bench-side tooling; not part of libhough).
//
// Every lane adds into its own row of a 32 x 33 word array, so the 32 lanes of
// a warp always hit 32 distinct banks (no bank conflict, no same-address
// conflict): the best case the vote loop's layout aims for.  Two forms of the
// 32-bit add are measured, each written as the instruction itself:
//   op 0: atom.shared.add.u32 with the returned old value consumed -- the
//         form the find kernel's vote loop issues (the old value tells it
//         when a bin reaches the vote threshold);
//   op 1: red.shared.add.u32, no returned value -- the form of the
//         accumulator-only kernel.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

template <int OP>
__global__ void __launch_bounds__(1024) smem_atomic_probe(int iters, unsigned *sink)
{
    __shared__ unsigned s[32 * 33];
    for (int i = threadIdx.x; i < 32 * 33; i += blockDim.x)
        s[i] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned row = (unsigned)__cvta_generic_to_shared(s + lane * 33);
    const int b = warp & 31;
    unsigned acc = 0u;
    for (int i = 0; i < iters; ++i) {
        unsigned old[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const unsigned a = row + 4u * (unsigned)((b + k) & 31);
            if (OP == 0)
                asm volatile("atom.shared.add.u32 %0, [%1], 1;" : "=r"(old[k]) : "r"(a) : "memory");
            else
                asm volatile("red.shared.add.u32 [%0], 1;" :: "r"(a) : "memory");
        }
        if (OP == 0) {
            // the returned values are consumed, as the vote loop consumes them
#pragma unroll
            for (int k = 0; k < 8; ++k)
                acc += old[k];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0)
        sink[blockIdx.x] = s[0] + s[32 * 33 - 1];
    if (acc == 0xdeadbeefu)
        sink[0] = acc;
}

}  // namespace

extern "C" {

// Runs the probe on the current device; *gops receives 10^9 atomics per
// second.  op: 0 = atom with the old value used, 1 = red (no return).
// Returns 0 or a negative code.
int hough_probe_smem_atomics(int op, int iters, int blocks_per_sm, int threads, double *gops,
                             double *ms_out)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -1;
    if (op < 0 || op > 1 || iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 8 || threads < 32 ||
        threads > 1024 || threads % 32 != 0)
        return -2;
    int grid = sms * blocks_per_sm;
    unsigned *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(unsigned) * grid) != cudaSuccess)
        return -3;
    auto kern = op == 0 ? smem_atomic_probe<0> : smem_atomic_probe<1>;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    kern<<<grid, threads>>>(iters / 4 + 1, sink);   // warm-up
    cudaEventRecord(e0);
    kern<<<grid, threads>>>(iters, sink);
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
