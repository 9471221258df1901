// Steps A-B alone with every window's accumulator written out: the (theta,
// rho) histogram of Eq. (1) binned as in Section 5, one per time window
// (Section 6), without peaks or association.  Included by hough_api.cu after
// hough_kernels.cuh; shares its vote arithmetic (rho_bin) and hit staging
// with the find kernel, so the histograms equal the ones the find writes in
// export mode.
#pragma once

namespace hk {

__device__ __forceinline__ void red_add_shared(unsigned addr, unsigned v)
{
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}

// Every staged hit votes once in each of the tile's rows.  No vote needs its
// returned count here (nothing is listed), so the votes are reductions.
// FAST: every valid hit votes in range and the tile has no row past n_theta.
template <int P, bool FAST>
__device__ void acc_vote_tile(const KParams &p, uint32_t *acc, const int2 *stage, int nh, int t0,
                              bool &oor)
{
    constexpr int CW = 32 / P;
    const int WR = p.word_rows, G = WR >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int g = warp % G;
    const int wr = g * 32 + lane;
    const int hstep = nw / G;
    int c[P], s[P];
    bool act[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
        const int t = t0 + k * WR + wr;
        act[k] = t < p.n_theta;
        c[k] = act[k] ? __ldg(p.C + t) : 0;
        s[k] = act[k] ? __ldg(p.S + t) : 0;
    }
    // bank-private column of this lane: word (wr, b) at col_word0 + 32 b
    const unsigned col_word0 = (unsigned)(g * p.n_rho) * 32u + (unsigned)lane;
    const unsigned col = (unsigned)__cvta_generic_to_shared(acc) + 4u * col_word0;
    const int D = p.D, K = p.K;
    const unsigned nr = (unsigned)p.n_rho;
#pragma unroll 4
    for (int h = warp / G; h < nh; h += hstep) {
        const int2 hv = stage[h];
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const int b = rho_bin(hv.x, hv.y, c[k], s[k], D, K);
            bool in = true;
            if (!FAST) {
                in = act[k] && (unsigned)b < nr;
                oor |= act[k] && !in;
            }
            if (in)
                red_add_shared(col + (unsigned)b * 128u, 1u << (k * CW));
        }
    }
}

// Export of a tile that is not read again: each warp takes a block of 32
// word rows x 32 bins (1024 consecutive words of the bank-private layout),
// holds it in registers and writes it back transposed in place: word row r
// becomes 32 consecutive words (bins b0..b0+31), its 16-byte chunk c stored
// at chunk c ^ (r & 7), so that the 16-byte writes and reads that follow
// take the minimum four wavefronts.  Each lane then reads four bins of one
// word row and writes each of its P theta rows with one 16-byte store: a
// warp store covers four whole 128-byte lines.  Bins past the last whole
// block of 32 (n_rho not a multiple of 32) go out one lane per word row
// with 4-byte stores, as does everything when the accumulator is not
// 16-byte aligned or the tile has rows past n_theta (then row by row).
template <int P>
__device__ void export_tile_rows(const KParams &p, uint32_t *acc, int t0, int R, long long w)
{
    constexpr int CW = 32 / P;
    constexpr unsigned MASK = P == 1 ? 0xffffffffu : ((1u << CW) - 1u);
    const int WR = p.word_rows, G = WR >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nblk = p.n_rho >> 5;
    int32_t *out = p.acc + (size_t)w * p.n_theta * p.n_rho;
    const bool fast = t0 + R <= p.n_theta && (reinterpret_cast<uintptr_t>(p.acc) & 15u) == 0u;
    for (int item = warp; item < G * nblk; item += nw) {
        const int g = item / nblk, b0 = (item - g * nblk) * 32;
        uint32_t *blk = acc + (size_t)(g * p.n_rho + b0) * 32;
        uint32_t r[32];
#pragma unroll
        for (int j = 0; j < 32; ++j)
            r[j] = blk[j * 32 + lane];                 // word (g*32 + lane, b0 + j)
        __syncwarp();
#pragma unroll
        for (int c = 0; c < 8; ++c)
            *reinterpret_cast<uint4 *>(blk + lane * 32 + ((c ^ (lane & 7)) << 2)) =
                make_uint4(r[4 * c], r[4 * c + 1], r[4 * c + 2], r[4 * c + 3]);
        __syncwarp();
        if (fast) {
            // lane: word row q + (lane >> 3), bins b0 + 4 (lane & 7) .. + 3
            const int rs = lane >> 3, c = lane & 7;
            int32_t *o = out + (size_t)(t0 + g * 32 + rs) * p.n_rho + b0 + 4 * c;
            const int sstep = WR * p.n_rho;
#pragma unroll 4
            for (int q = 0; q < 32; q += 4) {
                const int row = q + rs;
                const uint4 v = *reinterpret_cast<const uint4 *>(blk + row * 32 + ((c ^ (row & 7)) << 2));
#pragma unroll
                for (int s = 0; s < P; ++s)
                    *reinterpret_cast<int4 *>(o + q * p.n_rho + s * sstep) = fields4<P>(v, s);
            }
        } else {
            for (int q = 0; q < 32; ++q) {
                const uint32_t v = blk[q * 32 + ((((lane >> 2) ^ (q & 7))) << 2) + (lane & 3)];
#pragma unroll
                for (int s = 0; s < P; ++s) {
                    const int i = s * WR + g * 32 + q, t = t0 + i;
                    if (i < R && t < p.n_theta)
                        out[(size_t)t * p.n_rho + b0 + lane] = (int)((v >> (s * CW)) & MASK);
                }
            }
        }
    }
    const int rb = nblk * 32;
    if (rb < p.n_rho) {
        for (int g = warp; g < G; g += nw) {
            const int wr = g * 32 + lane;
            for (int b = rb; b < p.n_rho; ++b) {
                const uint32_t v = acc[(size_t)(g * p.n_rho + b) * 32 + lane];
#pragma unroll
                for (int s = 0; s < P; ++s) {
                    const int i = s * WR + wr, t = t0 + i;
                    if (i < R && t < p.n_theta)
                        out[(size_t)t * p.n_rho + b] = (int)((v >> (s * CW)) & MASK);
                }
            }
        }
    }
}

// One window: P counters per word (H votes at most per bin), tiles of
// word_rows * P theta rows, each voted, then exported.
template <int P>
__device__ void acc_window(const KParams &p, long long beg, int H, uint32_t *acc, int2 *stage,
                           int *wtot, WinScalars &ws, long long w)
{
    const int WR = p.word_rows, R = WR * P;
    const int n_tiles = (p.n_theta + R - 1) / R;
    const bool single = H <= p.hit_stage;
    const int acc_words4 = (WR * p.n_rho) >> 2;
    int nv = 0;
    if (single)
        nv = stage_hits(p, beg, H, stage, wtot, ws);
    bool oor = false;
    for (int tile = 0; tile < n_tiles; ++tile) {
        const int t0 = tile * R;
        uint4 *acc4 = reinterpret_cast<uint4 *>(acc);
        for (int i = threadIdx.x; i < acc_words4; i += blockDim.x)
            acc4[i] = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
        if (single) {
            if (p.in_range && t0 + R <= p.n_theta)
                acc_vote_tile<P, true>(p, acc, stage, nv, t0, oor);
            else
                acc_vote_tile<P, false>(p, acc, stage, nv, t0, oor);
        } else {
            for (long long s0 = 0; s0 < H; s0 += p.hit_stage) {
                const int n = (int)min((long long)p.hit_stage, (long long)H - s0);
                const int ns = stage_hits(p, beg + s0, n, stage, wtot, ws);
                acc_vote_tile<P, false>(p, acc, stage, ns, t0, oor);
                __syncthreads();
            }
        }
        __syncthreads();
        export_tile_rows<P>(p, acc, t0, R, w);
        __syncthreads();
    }
    if (__syncthreads_or(oor) && threadIdx.x == 0)
        atomicOr(&ws.flags, HOUGH_WIN_VOTE_OUT_OF_RANGE);
}

// Persistent CTAs stride over the windows.  Shared memory: the tile
// (word_rows * n_rho words) then the stage of hit_stage (phi, z) pairs.
__global__ void __launch_bounds__(1024, 1) accumulate_kernel(KParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ WinScalars ws;
    __shared__ int wtot[32];
    uint32_t *acc = reinterpret_cast<uint32_t *>(smem);
    int2 *stage = reinterpret_cast<int2 *>(smem + align_up((size_t)p.word_rows * p.n_rho * 4, 16));
    for (long long w = blockIdx.x; w < p.n_windows; w += gridDim.x) {
        const long long beg = p.offsets[w], end = p.offsets[w + 1];
        if (!(beg >= 0 && beg <= end && end <= p.n_hits && end - beg < (1ll << 30))) {
            if (threadIdx.x == 0)
                p.status[w] = HOUGH_WIN_BAD_OFFSETS;
            continue;                                  // uniform
        }
        const int H = (int)(end - beg);
        if (threadIdx.x == 0)
            ws.flags = 0u;
        __syncthreads();
        if (H <= 255)
            acc_window<4>(p, beg, H, acc, stage, wtot, ws, w);
        else if (H <= 65535)
            acc_window<2>(p, beg, H, acc, stage, wtot, ws, w);
        else
            acc_window<1>(p, beg, H, acc, stage, wtot, ws, w);
        __syncthreads();
        if (threadIdx.x == 0)
            p.status[w] = ws.flags;
        __syncthreads();                               // ws is reused
    }
}

}  // namespace hk
