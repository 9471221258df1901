// Time slicing on the device (Section 5: overlapping windows of a
// time-ordered readout).  Included by hough_api.cu after hough_kernels.cuh.
#pragma once

namespace hk {

// Window k holds the hits with t0 + k*step <= t < t0 + (k + m)*step (window
// length m steps).  With LB(j) = the first hit whose time is >= t0 + j*step
// (a lower bound on the sorted times), window k is hits [LB(k), LB(k + m)).
struct SliceParams {
    const long long *t;
    const int32_t *in0, *in1;
    long long n, t0, step, n_windows, cap;
    int m;
    int block;          // windows per CTA step, 32..kSliceBlock
    int32_t *out0, *out1;
    long long *out_index;
    long long *offsets;
    unsigned int *status;
};

// First index i in [0, n) with t[i] >= v (n if none), found by the whole
// warp: each step probes 32 evenly spaced positions at once and keeps the
// interval between the last probe below v and the first one not below, so
// the range shrinks about 33-fold per step.  Every lane returns the result.
__device__ long long warp_lower_bound(const long long *t, long long n, long long v)
{
    const int lane = threadIdx.x & 31;
    long long lo = 0, hi = n;
    while (hi - lo > 32) {
        const long long span = hi - lo;
        const long long pos = lo + span * (lane + 1) / 33;            // lo <= pos < hi
        const unsigned below = __ballot_sync(0xffffffffu, __ldg(t + pos) < v);
        const int c = __popc(below);                                   // probes below v (a prefix)
        const long long p_last = lo + span * c / 33;                   // probe c - 1
        const long long p_next = lo + span * (c + 1) / 33;             // probe c
        if (c > 0)
            lo = p_last + 1;
        if (c < 32)
            hi = p_next;
    }
    const bool in = lo + lane < hi;
    const unsigned below = __ballot_sync(0xffffffffu, in && __ldg(t + lo + lane) < v);
    return lo + __popc(below);
}

// floor(a / b) for b > 0
__device__ __forceinline__ long long floor_div_ll(long long a, long long b)
{
    const long long q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}

// Largest number of windows per CTA step of the slicer.
constexpr int kSliceBlock = 256;

// Time slicing (Section 5).  LB(k) = first hit with t >= s_k, s_k = t0 + k
// step; window k holds hits [LB(k), LB(k + m)) and starts at offsets[k] =
// sum_{i<m} LB(k + i) - sum_{i<m} LB(i).  A CTA takes the windows
// [k0, k0 + block) at a time: two warps find LB(k0) and the last LB it
// needs by search, then every hit between them sets, in one coalesced pass,
// LB(k) = i for the k with t[i-1] < s_k <= t[i] (t sorted); the warps then
// write the offsets and copy each window's hits.
__global__ void __launch_bounds__(256) slice_kernel(SliceParams q)
{
    __shared__ long long lbs[kSliceBlock + HOUGH_SLICE_MAX_OVERLAP + 1];
    __shared__ long long ends[2];
    __shared__ long long base_s[HOUGH_SLICE_MAX_OVERLAP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned full = 0xffffffffu;
    // sortedness, every adjacent pair once over the grid
    bool bad = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i + 1 < q.n;
         i += (long long)gridDim.x * blockDim.x)
        bad |= __ldg(q.t + i) > __ldg(q.t + i + 1);
    if (__any_sync(full, bad) && lane == 0 && q.status)
        atomicOr(q.status, HOUGH_SLICE_UNSORTED);
    // sum_{i<m} LB(i)
    for (int i = warp; i < q.m; i += nw) {
        const long long lb = warp_lower_bound(q.t, q.n, q.t0 + (long long)i * q.step);
        if (lane == 0)
            base_s[i] = lb;
    }
    __syncthreads();
    long long base = 0;
    for (int i = 0; i < q.m; ++i)
        base += base_s[i];

    const long long n_entries = q.n_windows + 1;          // offsets[0 .. n_windows]
    const int B = q.block;
    for (long long k0 = (long long)blockIdx.x * B; k0 < n_entries; k0 += (long long)gridDim.x * B) {
        const long long kend = min(k0 + (long long)B, n_entries);
        const int cnt = (int)(kend - k0) + q.m;            // LB(k0) .. LB(kend - 1 + m)
        if (warp < 2) {
            const long long kk = warp == 0 ? k0 : kend - 1 + q.m;
            const long long lb = warp_lower_bound(q.t, q.n, q.t0 + kk * q.step);
            if (lane == 0)
                ends[warp] = lb;
        }
        __syncthreads();
        const long long lo = ends[0];
        const long long hi = max(ends[1], lo);           // unsorted input: keep the range sane
        for (int x = threadIdx.x; x < cnt; x += blockDim.x)
            lbs[x] = hi;
        __syncthreads();
        // times clamped to [t0 - 1, t0 + lim + 1], which keeps every
        // comparison with a window start and makes t - t0 safe
        const long long lim = 0x7fffffffffffffffll / 4;
        auto rel = [&](long long t) { return min(max(t, q.t0 - 1), q.t0 + lim + 1) - q.t0; };
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            // the k with t[i-1] < s_k <= t[i], within [k0, k0 + cnt)
            long long ka = k0;
            if (i > lo)
                ka = max(ka, floor_div_ll(rel(__ldg(q.t + i - 1)), q.step) + 1);
            const long long kb = min(floor_div_ll(rel(__ldg(q.t + i)), q.step), k0 + cnt - 1);
            for (long long k = ka; k <= kb; ++k)
                lbs[k - k0] = i;
        }
        __syncthreads();
        for (long long k = k0 + warp; k < kend; k += nw) {
            const int x = (int)(k - k0);
            long long s = lane < q.m ? lbs[x + lane] : 0;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1)
                s += __shfl_xor_sync(full, s, d);
            const long long off = s - base;
            if (lane == 0)
                q.offsets[k] = off;
            if (k == q.n_windows)
                continue;                                  // offsets[n_windows] only
            const long long wlo = lbs[x], whi = lbs[x + q.m];
            // unsorted input can give any bounds and offsets: copy only what fits
            if (wlo < whi && wlo >= 0 && whi <= q.n && off >= 0 && off + (whi - wlo) <= q.cap) {
                for (long long j = lane; j < whi - wlo; j += 32) {
                    q.out0[off + j] = __ldg(q.in0 + wlo + j);
                    q.out1[off + j] = __ldg(q.in1 + wlo + j);
                    if (q.out_index)
                        q.out_index[off + j] = wlo + j;
                }
            }
        }
        __syncthreads();                                   // lbs and ends are reused
    }
}

}  // namespace hk
