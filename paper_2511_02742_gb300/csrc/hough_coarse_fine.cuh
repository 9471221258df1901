// hough_coarse_fine.cuh -- device code of the paper's two-stage search
// (coarse 18 x 100 histogram, then a 10 x 10 fine block of the 180 x 1000
// grid; one line per window).  Uses the fixed-point bin of hough_kernels.cuh.
#pragma once

#include <climits>

#include "hough_kernels.cuh"

namespace hk {

// Coarse: every (hit, row) pair of the 18 coarse rows votes into an 18 x 100
// shared histogram; the maximum of (count, -index) gives the coarse bin
// (ties row-major).
// Fine: the (hit, row) pairs of the 10 fine rows inside it vote into a 10 x
// 10 histogram, keeping only the bins of the 10 fine columns; its maximum is
// the line.  Consecutive threads take the rows of one hit, so the lanes of a
// warp vote in different rows (few same-address atomics).
constexpr int kCfCoarseT = 18, kCfCoarseR = 100, kCfFineT = 180, kCfFineR = 1000, kCfBlock = 10;

struct CfParams {
    const int32_t *a, *b;          // as KParams
    long long n_hits;
    int raw, vane_step, z_min_u, z_pitch_u, z_half;
    long long phi_end, z_end;
    const long long *offsets;
    long long n_windows;
    const int32_t *Cc, *Sc, *Cf, *Sf;
    int Dc, Kc, Df, Kf;
    int T, tol;
    hough_line *lines;
    int32_t *hit_track;
};

__device__ __forceinline__ bool cf_load_hit(const CfParams &p, long long i, int &phi, int &z)
{
    const int a = __ldg(p.a + i), b = __ldg(p.b + i);
    if (p.raw) {
        phi = (int)((long long)p.vane_step * (long long)a);
        z = (int)((long long)p.z_min_u + (long long)p.z_pitch_u * (long long)b + p.z_half);
    } else {
        phi = a;
        z = b;
    }
    return phi >= 0 && (long long)phi < p.phi_end && z >= p.z_min_u && (long long)z <= p.z_end;
}

// Warp maximum of a 64-bit key (every lane gets it).
__device__ __forceinline__ unsigned long long cf_warp_max(unsigned long long k)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, k, d);
        k = o > k ? o : k;
    }
    return k;
}

// Windows per CTA (one warp each).
constexpr int kCfWarps = 4;

// One warp per window (grid-stride over windows), with its own coarse and
// fine histograms in shared memory, so that no phase waits for a block
// barrier.  The maxima use the key (count << 32) | (2^32 - 1 - index): the
// highest count, then the first bin in row-major order.
__global__ void __launch_bounds__(32 * kCfWarps) coarse_fine_kernel(CfParams p)
{
    __shared__ __align__(16) int coarse_s[kCfWarps][kCfCoarseT * kCfCoarseR];
    __shared__ __align__(16) int fine_s[kCfWarps][kCfBlock * kCfBlock];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int *coarse = coarse_s[warp], *fine = fine_s[warp];
    const long long n_warps = (long long)gridDim.x * kCfWarps;
    for (long long w = (long long)blockIdx.x * kCfWarps + warp; w < p.n_windows; w += n_warps) {
        const long long beg = p.offsets[w], end = p.offsets[w + 1];
        const bool ok_off = beg >= 0 && beg <= end && end <= p.n_hits;
        const int H = ok_off ? (int)min(end - beg, (long long)INT_MAX / kCfCoarseT) : 0;
        int4 *c4 = reinterpret_cast<int4 *>(coarse);
        for (int i = lane; i < kCfCoarseT * kCfCoarseR / 4; i += 32)
            c4[i] = make_int4(0, 0, 0, 0);
        for (int i = lane; i < kCfBlock * kCfBlock; i += 32)
            fine[i] = 0;
        __syncwarp();
        // coarse: a lane per hit (loaded and encoded once), over the 18 rows
        for (int h = lane; h < H; h += 32) {
            int phi, z;
            if (!cf_load_hit(p, beg + h, phi, z))
                continue;
#pragma unroll 6
            for (int t = 0; t < kCfCoarseT; ++t) {
                const int b = rho_bin(phi, z, __ldg(p.Cc + t), __ldg(p.Sc + t), p.Dc, p.Kc);
                if ((unsigned)b < (unsigned)kCfCoarseR)
                    atomicAdd(&coarse[t * kCfCoarseR + b], 1);
            }
        }
        __syncwarp();
        unsigned long long key = 0ull;
        for (int i = lane; i < kCfCoarseT * kCfCoarseR; i += 32) {
            const unsigned long long k = ((unsigned long long)(unsigned)coarse[i] << 32) |
                                         (unsigned long long)(0xffffffffu - (unsigned)i);
            key = k > key ? k : key;
        }
        const unsigned long long cmax = cf_warp_max(key);
        const int cidx = (int)(0xffffffffu - (unsigned)(cmax & 0xffffffffu));
        const int cvotes = (int)(cmax >> 32);
        const int tc = cidx / kCfCoarseR, bc = cidx - tc * kCfCoarseR;
        bool found = cvotes >= p.T;
        int tf = 0, bf = 0, fvotes = 0;
        if (found) {
            for (int h = lane; h < H; h += 32) {
                int phi, z;
                if (!cf_load_hit(p, beg + h, phi, z))
                    continue;
#pragma unroll 5
                for (int i = 0; i < kCfBlock; ++i) {
                    const int t = tc * kCfBlock + i;
                    const int b = rho_bin(phi, z, __ldg(p.Cf + t), __ldg(p.Sf + t), p.Df, p.Kf);
                    const int j = b - bc * kCfBlock;
                    if ((unsigned)j < (unsigned)kCfBlock)
                        atomicAdd(&fine[i * kCfBlock + j], 1);
                }
            }
            __syncwarp();
            unsigned long long fk = 0ull;
            for (int i = lane; i < kCfBlock * kCfBlock; i += 32) {
                const unsigned long long k = ((unsigned long long)(unsigned)fine[i] << 32) |
                                             (unsigned long long)(0xffffffffu - (unsigned)i);
                fk = k > fk ? k : fk;
            }
            const unsigned long long fmax = cf_warp_max(fk);
            const int fidx = (int)(0xffffffffu - (unsigned)(fmax & 0xffffffffu));
            fvotes = (int)(fmax >> 32);
            tf = tc * kCfBlock + fidx / kCfBlock;
            bf = bc * kCfBlock + fidx % kCfBlock;
            found = fvotes >= p.T;
        }
        // seeds
        int mine = 0;
        const int cft = __ldg(p.Cf + tf), sft = __ldg(p.Sf + tf);
        for (int h = lane; h < H; h += 32) {
            int phi, z;
            int v = -2;
            if (cf_load_hit(p, beg + h, phi, z)) {
                v = -1;
                if (found) {
                    const int d = rho_bin(phi, z, cft, sft, p.Df, p.Kf) - bf;
                    if (d <= p.tol && d >= -p.tol) {
                        v = 0;
                        ++mine;
                    }
                }
            }
            p.hit_track[beg + h] = v;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1)
            mine += __shfl_xor_sync(0xffffffffu, mine, d);
        if (lane == 0) {
            hough_line r;
            r.coarse_theta = ok_off ? tc : 0;
            r.coarse_rho = ok_off ? bc : 0;
            r.coarse_votes = ok_off ? cvotes : 0;
            r.fine_theta = tf;
            r.fine_rho = bf;
            r.fine_votes = fvotes;
            r.n_seeds = mine;
            r.found = found ? 1 : 0;
            p.lines[w] = r;
        }
        __syncwarp();                        // the histograms are cleared next
    }
}

}  // namespace hk
