// hough_iterative.cuh -- device code of the iterative highest-bin search (the
// literal reading of the paper's peak step, repeated): vote the hits not yet
// assigned, take the accumulator's highest bin (ties: first in row-major
// order), stop below T, else give track k every remaining hit within tol
// bins of it in its row, remove them and vote again.
//
// One CTA per window (grid-stride).  The window's valid hits are staged in
// shared memory with their window-local indices; every iteration runs the
// theta tiles of the find kernel's vote loop (its narrowed tiles, vote_tile
// with candidate listing switched off) and a block maximum over each tile's
// counters, then marks the line's hits and compacts them out of the stage in
// order.
#pragma once

#include "hough_kernels.cuh"

namespace hk {

struct IterParams {
    KParams k;                  // hits, tables, shape, thresholds, launch shape
    int max_tracks;
    int4 *tracks;               // [n_windows * max_tracks]: theta, rho, votes, n_hits
    int32_t *n_tracks;          // [n_windows]
};

// Stage the window's valid hits (in order) with their window-local indices;
// invalid hits get hit_track = -2, valid ones -1.  Returns the staged count
// (uniform), or -1 when they do not fit in the stage.
__device__ int iter_stage(const KParams &p, long long beg, int H, int2 *stage, int *sidx,
                          int *wtot)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int total = 0;
    for (int c0 = 0; c0 < H; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        int phi = 0, z = 0;
        bool ok = false;
        if (i < H) {
            ok = load_hit(p, beg + i, phi, z);
            p.hit_track[beg + i] = ok ? -1 : -2;
        }
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (lane == 0)
            wtot[warp] = __popc(m);
        __syncthreads();
        int pre = 0, tot = 0;
        for (int k = 0; k < nw; ++k) {
            const int v = wtot[k];
            pre += k < warp ? v : 0;
            tot += v;
        }
        const int pos = total + pre + __popc(m & lanemask_lt());
        if (ok && pos < p.hit_stage) {
            stage[pos] = make_int2(phi, z);
            sidx[pos] = i;
        }
        total += tot;
        __syncthreads();
    }
    return total <= p.hit_stage ? total : -1;
}

// Highest counter of the voted tile as a key (count << 32 | ~(t << 16 | b)):
// the block maximum is the highest count, first in row-major order.
__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long k,
                                                            unsigned long long *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, k, d);
        k = o > k ? o : k;
    }
    __syncthreads();
    if (lane == 0)
        red[warp] = k;
    __syncthreads();
    unsigned long long m = 0ull;
    for (int i = 0; i < nw; ++i)
        m = red[i] > m ? red[i] : m;
    return m;
}

// Whether some P-bit field of w equals v (v < 2^(32/P)): the fields of
// y = w ^ (v in every field) that are zero, by the exact zero-field test
// (y - 0x..01..01) & ~y & 0x..80..80 (non-zero iff some field of y is zero).
template <int P>
__device__ __forceinline__ bool has_field(uint32_t w, unsigned v)
{
    if constexpr (P == 1) {
        return w == v;
    } else if constexpr (P == 2) {
        const uint32_t y = w ^ (v * 0x00010001u);
        return ((y - 0x00010001u) & ~y & 0x80008000u) != 0u;
    } else {
        const uint32_t y = w ^ (v * 0x01010101u);
        return ((y - 0x01010101u) & ~y & 0x80808080u) != 0u;
    }
}

// The tile's highest bin as the key (count << 32) | (2^32 - 1 - (t << 16 | b)):
// the highest count, then the first bin in row-major order.  Two passes over
// the counters: the highest count (fields only: rows past n_theta never get a
// vote, so every non-zero field is a bin of the accumulator), then the words
// holding that count.  Every thread gets the result.
template <int P>
__device__ unsigned long long tile_best(const KParams &p, const uint32_t *acc, int t0, int lo,
                                        unsigned long long *red)
{
    constexpr int CW = 32 / P;
    constexpr unsigned MASK = P == 1 ? 0xffffffffu : ((1u << CW) - 1u);
    const int words = p.word_rows * p.n_b;
    unsigned m = 0u;
    for (int f = threadIdx.x; f < words; f += blockDim.x) {
        const uint32_t wv = acc[f];
#pragma unroll
        for (int s = 0; s < P; ++s)
            m = max(m, (wv >> (s * CW)) & MASK);
    }
    const unsigned top = (unsigned)(block_max_u64(m, red) & 0xffffffffu);
    if (top == 0u)
        return 0ull;
    unsigned long long best = 0ull;
    for (int f = threadIdx.x; f < words; f += blockDim.x) {
        const uint32_t wv = acc[f];
        if (!has_field<P>(wv, top))
            continue;
        const int q = f >> 5;
        const int g = (int)__umulhi((unsigned)q, p.nb_inv);
        const int b = q - g * p.n_b + lo;                   // the tile stores bins lo ..
        const int wr = g * 32 + (f & 31);
#pragma unroll
        for (int s = 0; s < P; ++s) {
            if (((wv >> (s * CW)) & MASK) != top)
                continue;
            const int t = t0 + s * p.word_rows + wr;
            const unsigned long long key = ((unsigned long long)top << 32) |
                                           (unsigned long long)(0xffffffffu -
                                                                (((unsigned)t << 16) | (unsigned)b));
            best = key > best ? key : best;
        }
    }
    return block_max_u64(best, red);
}

// One pass over every tile: the highest bin of the remaining hits' votes.
// ub[tile]: an upper bound of the tile's highest count (its highest count
// when it was last voted: removing hits only lowers counts), valid while the
// counter width P, and so the tiling, stays the same.  The tiles are taken in
// decreasing order of their bound (ties: the earlier tile first), so that the
// best count is found early; a tile is voted only if it could still hold the
// highest bin: a bound of at least T and above the best count so far, or
// equal to it in a tile before the best bin's (the first bin in row-major
// order wins a tie).  done: one bit per tile, this call's visits.
template <int P>
__device__ unsigned long long iter_best(const KParams &p, uint32_t *acc, const int2 *stage, int nv,
                                        unsigned long long *red, WinScalars &ws, int *ub,
                                        unsigned *done, int T)
{
    const int R = p.word_rows * P;
    const int n_tiles = (p.n_theta + R - 1) / R;
    const int lane = threadIdx.x & 31;
    constexpr int lgP = P == 4 ? 2 : (P == 2 ? 1 : 0);
    const int32_t *lo_row = p.lo_tab ? p.lo_tab + lgP * p.lo_stride : nullptr;
    unsigned long long best = 0ull;
    int best_tile = n_tiles;
    int cnt = 0;
    const ListOvf none{&ws.n_sel, 0};
    for (int i = threadIdx.x; i < (n_tiles + 31) / 32; i += blockDim.x)
        done[i] = 0u;
    __syncthreads();
    for (;;) {
        // every warp picks the same tile: the largest (bound, -index) not yet visited
        unsigned long long pick = 0ull;
        for (int x = lane; x < n_tiles; x += 32) {
            if ((done[x >> 5] >> (x & 31)) & 1u)
                continue;
            const unsigned long long k = ((unsigned long long)(unsigned)ub[x] << 32) |
                                         (unsigned long long)(0xffffffffu - (unsigned)x);
            pick = k > pick ? k : pick;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, pick, d);
            pick = o > pick ? o : pick;
        }
        if (pick == 0ull)
            break;                                   // every tile visited
        const int tile = (int)(0xffffffffu - (unsigned)(pick & 0xffffffffu));
        const unsigned bound = (unsigned)(pick >> 32);
        const unsigned top = (unsigned)(best >> 32);
        if ((int)bound < T || bound < top || (bound == top && tile > best_tile))
            break;                                   // no unvisited tile can hold the highest bin
        const int t0 = tile * R;
        const int lo = lo_row ? __ldg(lo_row + tile) : 0;
        uint4 *acc4 = reinterpret_cast<uint4 *>(acc);
        for (int i = threadIdx.x; i < (p.word_rows * p.n_b) >> 2; i += blockDim.x)
            acc4[i] = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
        if (p.in_range && t0 + R <= p.n_theta)
            vote_tile<P, true>(p, acc, stage, nv, t0, lo, nullptr, 0, cnt, none, ws);
        else
            vote_tile<P, false>(p, acc, stage, nv, t0, lo, nullptr, 0, cnt, none, ws);
        __syncthreads();
        const unsigned long long k = tile_best<P>(p, acc, t0, lo, red);
        if (threadIdx.x == 0) {
            ub[tile] = (int)(k >> 32);
            done[tile >> 5] |= 1u << (tile & 31);
        }
        if (k > best) {
            best = k;
            best_tile = tile;
        }
        __syncthreads();
    }
    return best;
}

__global__ void __launch_bounds__(512, 1) iterative_kernel(IterParams q)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ WinScalars ws;
    __shared__ unsigned long long red[16];
    __shared__ int wtot[32];
    __shared__ int taken;
    __shared__ int ub[HOUGH_MAX_THETA / 32];      // per-tile bounds (at most n_theta / 32 tiles)
    __shared__ unsigned done[HOUGH_MAX_THETA / 32 / 32];
    KParams p = q.k;
    p.T = 0x7fffffff;               // the vote loop lists nothing
    const int T = q.k.T;
    uint32_t *acc = reinterpret_cast<uint32_t *>(smem);
    int2 *stage = reinterpret_cast<int2 *>(smem + (size_t)p.word_rows * p.n_b * 4);
    int *sidx = reinterpret_cast<int *>(stage + p.hit_stage);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (long long w = blockIdx.x; w < p.n_windows; w += gridDim.x) {
        const long long beg = p.offsets[w], end = p.offsets[w + 1];
        if (!(beg >= 0 && beg <= end && end <= p.n_hits && end - beg < (1ll << 30))) {
            if (threadIdx.x == 0) {
                p.status[w] = HOUGH_WIN_BAD_OFFSETS;
                q.n_tracks[w] = 0;
            }
            continue;
        }
        const int H = (int)(end - beg);
        if (threadIdx.x == 0)
            ws.flags = 0u;
        __syncthreads();
        int nv = iter_stage(p, beg, H, stage, sidx, wtot);
        int found = 0;
        unsigned flags = 0u;
        if (nv < 0) {
            flags |= HOUGH_WIN_TOO_LARGE;
            nv = 0;
        }
        int width = 0;                               // counter fields per word of the bounds
        while (found < q.max_tracks && nv > 0) {
            const int P = nv <= 255 ? 4 : (nv <= 65535 ? 2 : 1);
            if (P != width) {                        // new tiling: no bound known yet
                for (int i = threadIdx.x; i < HOUGH_MAX_THETA / 32; i += blockDim.x)
                    ub[i] = 0x7fffffff;
                __syncthreads();
                width = P;
            }
            unsigned long long best;
            if (P == 4)
                best = iter_best<4>(p, acc, stage, nv, red, ws, ub, done, T);
            else if (P == 2)
                best = iter_best<2>(p, acc, stage, nv, red, ws, ub, done, T);
            else
                best = iter_best<1>(p, acc, stage, nv, red, ws, ub, done, T);
            const int votes = (int)(best >> 32);
            if (votes < T)
                break;
            const unsigned tb = 0xffffffffu - (unsigned)(best & 0xffffffffu);
            const int bt = (int)(tb >> 16), bb = (int)(tb & 0xffffu);
            const int c = __ldg(p.C + bt), s = __ldg(p.S + bt);
            if (threadIdx.x == 0)
                taken = 0;
            __syncthreads();
            // mark the line's hits and compact the rest, in order, in place
            int kept = 0, mine = 0;
            for (int c0 = 0; c0 < nv; c0 += blockDim.x) {
                const int i = c0 + threadIdx.x;
                int2 h = make_int2(0, 0);
                int idx = 0;
                bool keep = false;
                if (i < nv) {
                    h = stage[i];
                    idx = sidx[i];
                    const int d = rho_bin(h.x, h.y, c, s, p.D, p.K) - bb;
                    if (d <= p.tol && d >= -p.tol) {
                        p.hit_track[beg + idx] = found;
                        ++mine;
                    } else {
                        keep = true;
                    }
                }
                const unsigned m = __ballot_sync(0xffffffffu, keep);
                if (lane == 0)
                    wtot[warp] = __popc(m);
                __syncthreads();
                int pre = 0, tot = 0;
                for (int k = 0; k < nw; ++k) {
                    const int v = wtot[k];
                    pre += k < warp ? v : 0;
                    tot += v;
                }
                if (keep) {
                    const int pos = kept + pre + __popc(m & lanemask_lt());
                    stage[pos] = h;
                    sidx[pos] = idx;
                }
                kept += tot;
                __syncthreads();
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1)
                mine += __shfl_xor_sync(0xffffffffu, mine, d);
            if (lane == 0 && mine)
                atomicAdd(&taken, mine);
            __syncthreads();
            if (threadIdx.x == 0)
                q.tracks[(size_t)w * q.max_tracks + found] = make_int4(bt, bb, votes, taken);
            nv = kept;
            ++found;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            q.n_tracks[w] = found;
            p.status[w] = flags | ws.flags;
        }
        __syncthreads();
    }
}

}  // namespace hk
