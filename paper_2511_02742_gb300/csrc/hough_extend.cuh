// Track extension (Section 4): a seed of three hits on consecutive vanes,
// taken from a peak's associated hits, extrapolated vane by vane forward and
// backward through the window's hits.  One warp per window; windows are
// independent.  Included by hough_api.cu after hough_kernels.cuh.
#pragma once

namespace hk {

constexpr int kExtClaimed = 512;   // tag of a claimed hit: kExtClaimed + track index

struct ExtParams {
    KParams k;          // hits, geometry, windows and the find step's outputs
    int n_vanes;        // 3..HOUGH_EXT_MAX_VANES
    int tol_z;          // 0..HOUGH_EXT_MAX_TOL, z units
    int cap;            // hits a warp holds in shared memory in this launch (<= 4096)
    long long lo;       // this launch takes the windows with lo < n_hits <= cap
    int flag_large;     // windows above cap get HOUGH_WIN_TOO_LARGE (last launch)
    int4 *ext;          // [n_windows * max_peaks]: first_vane, n_hits, hit_begin, seed_mid
    int32_t *ext_track; // [n_hits] window-local track index, -1 none
    int32_t *ext_hits;  // [n_hits] window-local hit order
    uint32_t *status;   // [n_windows]
};

// Shared memory of one warp: z[cap] int32, vane[cap] int16 (-1: takes no
// part), tag[cap] int16 (the hit's peak from the find step, -1 none, or
// kExtClaimed + track once claimed), bucket[cap] int16 (hit indices grouped
// by vane), bstart[n_vanes + 1] and bcur[n_vanes] int32, line[2 n_vanes + 4]
// int16 (the track being built, in vane order).
__host__ __device__ inline size_t ext_smem_bytes(int cap, int n_vanes)
{
    return (size_t)cap * 10 + (size_t)(2 * n_vanes + 1) * 4 + (size_t)(2 * n_vanes + 4) * 2;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
        x = y < x ? y : x;
    }
    return x;
}

// The unclaimed hit of bucket [s0, s1) nearest to pred within tol, as the
// key (|z - pred| << 13) | (z > pred) << 12 | hit: the minimum is the nearest,
// then the lower z, then the lower index.  ~0u when there is none.
__device__ __forceinline__ unsigned ext_nearest(const int32_t *zs, const int16_t *tag,
                                                const int16_t *bucket, int s0, int s1,
                                                long long pred, int tol)
{
    unsigned best = 0xffffffffu;
    for (int i = s0 + (int)(threadIdx.x & 31); i < s1; i += 32) {
        const int h = bucket[i];
        if (tag[h] >= kExtClaimed)
            continue;
        long long d = (long long)zs[h] - pred;
        const unsigned side = d > 0 ? 1u : 0u;
        d = d < 0 ? -d : d;
        if (d > tol)
            continue;
        const unsigned key = ((unsigned)d << 13) | (side << 12) | (unsigned)h;
        best = key < best ? key : best;
    }
    return __reduce_min_sync(0xffffffffu, best);
}

__global__ void __launch_bounds__(32) extend_kernel(ExtParams q)
{
    extern __shared__ __align__(16) unsigned char ext_sm[];
    const KParams &p = q.k;
    const int lane = threadIdx.x & 31;
    const int nv = q.n_vanes, cap = q.cap, tol = q.tol_z;
    int32_t *zs = reinterpret_cast<int32_t *>(ext_sm);
    int16_t *vs = reinterpret_cast<int16_t *>(zs + cap);
    int16_t *tag = vs + cap;
    int16_t *bucket = tag + cap;
    int32_t *bstart = reinterpret_cast<int32_t *>(bucket + cap);   // cap is a multiple of 8
    int32_t *bcur = bstart + nv + 1;
    int16_t *line = reinterpret_cast<int16_t *>(bcur + nv);
    const int vstep = p.vane_step;

    for (long long w = blockIdx.x; w < p.n_windows; w += gridDim.x) {
        const long long beg = p.offsets[w], end = p.offsets[w + 1];
        if (!(beg >= 0 && beg <= end && end <= p.n_hits)) {
            if (q.lo < 0 && lane == 0)      // flagged once, by the first launch
                q.status[w] = HOUGH_WIN_BAD_OFFSETS;
            continue;
        }
        const long long n = end - beg;
        if (n <= q.lo)
            continue;                       // an earlier launch took it
        const int np = min(max(p.n_peaks[w], 0), p.max_peaks);
        int4 *ext = q.ext + w * (long long)p.max_peaks;
        if (n > cap) {
            if (q.flag_large) {
                for (int i = lane; i < np; i += 32)
                    ext[i] = make_int4(-1, 0, 0, -1);
                for (long long i = lane; i < n; i += 32) {
                    q.ext_track[beg + i] = -1;
                    q.ext_hits[beg + i] = (int)i;
                }
                if (lane == 0)
                    q.status[w] = HOUGH_WIN_TOO_LARGE;
            }
            continue;
        }
        const int H = (int)n;

        // ---- stage the window's hits and group them by vane
        for (int v = lane; v < nv; v += 32)
            bcur[v] = 0;
        __syncwarp();
        for (int i = lane; i < H; i += 32) {
            int phi, z;
            const bool ok = load_hit(p, beg + i, phi, z);
            const int ht = p.hit_track[beg + i];
            int v = -1;
            if (ok && ht != -2) {
                if (p.raw)
                    v = __ldg(p.a + beg + i);
                else if (phi % vstep == 0)
                    v = phi / vstep;
                if (v >= nv)
                    v = -1;
            }
            zs[i] = z;
            vs[i] = (int16_t)v;
            tag[i] = (int16_t)(ht >= 0 && ht < kExtClaimed ? ht : -1);
            if (v >= 0)
                atomicAdd(&bcur[v], 1);
        }
        __syncwarp();
        {
            // exclusive prefix over the vanes: lane l sums vanes [8l, 8l + 8)
            const int v0 = lane * 8;
            int s = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j)
                s += (v0 + j < nv) ? bcur[v0 + j] : 0;
            int incl = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o)
                    incl += y;
            }
            int run = incl - s;
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (v0 + j < nv) {
                    const int c = bcur[v0 + j];
                    bstart[v0 + j] = run;
                    bcur[v0 + j] = run;
                    run += c;
                }
            }
            if (lane == 31)
                bstart[nv] = incl;
        }
        __syncwarp();
        for (int i = lane; i < H; i += 32) {
            const int v = vs[i];
            if (v >= 0)
                bucket[atomicAdd(&bcur[v], 1)] = (int16_t)i;
        }
        __syncwarp();

        // ---- the peaks in order
        const hough_peak *pk = p.peaks + w * (long long)p.max_peaks;
        int pos = 0;
        for (int pi = 0; pi < np; ++pi) {
            const int hb = pk[pi].hit_begin, m = pk[pi].n_hits;
            const bool grp_ok = hb >= 0 && m >= 3 && (long long)hb + m <= H;
            if (!grp_ok) {                  // fewer than three hits: no seed
                if (lane == 0)
                    ext[pi] = make_int4(-1, 0, pos, -1);
                continue;
            }
            // seed: the smallest (bend, b, a, c) over the group's unclaimed triplets
            unsigned long long best = ~0ull;
            for (int j = lane; j < m; j += 32) {
                const int b = p.track_hits[beg + hb + j];
                if ((unsigned)b >= (unsigned)H || tag[b] != pi)
                    continue;
                const int vb = vs[b];
                if (vb < 0)
                    continue;
                const int va = vb == 0 ? nv - 1 : vb - 1;
                const int vc = vb + 1 == nv ? 0 : vb + 1;
                const long long zb2 = 2LL * zs[b];
                const int c0 = bstart[vc], c1 = bstart[vc + 1];
                for (int ia = bstart[va], ea = bstart[va + 1]; ia < ea; ++ia) {
                    const int a = bucket[ia];
                    if (tag[a] != pi)
                        continue;
                    const long long za = zs[a];
                    for (int ic = c0; ic < c1; ++ic) {
                        const int c = bucket[ic];
                        if (tag[c] != pi)
                            continue;
                        long long bend = za - zb2 + zs[c];
                        bend = bend < 0 ? -bend : bend;
                        if (bend > tol)
                            continue;
                        const unsigned long long key = ((unsigned long long)bend << 36) |
                                                       ((unsigned long long)b << 24) |
                                                       ((unsigned long long)a << 12) |
                                                       (unsigned long long)c;
                        best = key < best ? key : best;
                    }
                }
            }
            best = warp_min_u64(best);
            if (best == ~0ull) {
                if (lane == 0)
                    ext[pi] = make_int4(-1, 0, pos, -1);
                continue;
            }
            const int b = (int)((best >> 24) & 4095u);
            const int a = (int)((best >> 12) & 4095u);
            const int c = (int)(best & 4095u);
            const int16_t mine = (int16_t)(kExtClaimed + pi);
            int lo = nv + 1, hi = nv + 4;
            if (lane == 0) {
                tag[a] = tag[b] = tag[c] = mine;
                line[lo] = (int16_t)a;
                line[lo + 1] = (int16_t)b;
                line[lo + 2] = (int16_t)c;
            }
            __syncwarp();
            // forward: the parabola through the last three hits, one vane on
            {
                long long z0 = zs[a], z1 = zs[b], z2 = zs[c];
                int v2 = vs[c];
                while (hi - lo < nv) {
                    const int tv = v2 + 1 == nv ? 0 : v2 + 1;
                    const unsigned key = ext_nearest(zs, tag, bucket, bstart[tv], bstart[tv + 1],
                                                     3 * z2 - 3 * z1 + z0, tol);
                    if (key == 0xffffffffu)
                        break;
                    const int h = (int)(key & 4095u);
                    if (lane == 0) {
                        tag[h] = mine;
                        line[hi] = (int16_t)h;
                    }
                    ++hi;
                    z0 = z1;
                    z1 = z2;
                    z2 = zs[h];
                    v2 = tv;
                    __syncwarp();
                }
            }
            // backward, from the seed's first hit
            {
                long long z0 = zs[c], z1 = zs[b], z2 = zs[a];
                int v2 = vs[a];
                while (hi - lo < nv) {
                    const int tv = v2 == 0 ? nv - 1 : v2 - 1;
                    const unsigned key = ext_nearest(zs, tag, bucket, bstart[tv], bstart[tv + 1],
                                                     3 * z2 - 3 * z1 + z0, tol);
                    if (key == 0xffffffffu)
                        break;
                    const int h = (int)(key & 4095u);
                    --lo;
                    if (lane == 0) {
                        tag[h] = mine;
                        line[lo] = (int16_t)h;
                    }
                    z0 = z1;
                    z1 = z2;
                    z2 = zs[h];
                    v2 = tv;
                    __syncwarp();
                }
            }
            __syncwarp();
            const int cnt = hi - lo;
            for (int j = lane; j < cnt; j += 32)
                q.ext_hits[beg + pos + j] = line[lo + j];
            if (lane == 0)
                ext[pi] = make_int4(vs[line[lo]], cnt, pos, b);
            pos += cnt;
            __syncwarp();
        }

        // ---- per-hit track and the unclaimed hits in index order
        for (int base = 0; base < H; base += 32) {
            const int i = base + lane;
            const int t = i < H ? tag[i] : 0;
            const bool un = i < H && t < kExtClaimed;
            if (i < H)
                q.ext_track[beg + i] = un ? -1 : t - kExtClaimed;
            const unsigned m = __ballot_sync(0xffffffffu, un);
            if (un)
                q.ext_hits[beg + pos + __popc(m & ((1u << lane) - 1u))] = i;
            pos += __popc(m);
        }
        if (lane == 0)
            q.status[w] = 0u;
        __syncwarp();
    }
}

}  // namespace hk
