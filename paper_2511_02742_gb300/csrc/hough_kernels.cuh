// hough_kernels.cuh -- device code of the track-finding path (sm_103a).
//
// One persistent kernel processes whole time windows (Section 6: one window
// per unit of work).  Per window, in one CTA:
//   1. stage: the window's hits are loaded (encoded on the fly from strip
//      addresses if asked), checked against the detector box and compacted
//      into shared memory;
//   2. for each theta tile: zero the shared accumulator tile, vote (Eq. (1)),
//      optionally export it, scan it for 3x3 local maxima >= T and feed them
//      to an exact online top-k (Section 4 / Section 5 peak finding);
//   3. associate every hit with the first peak whose line it lies on and
//      compact the hits per peak (Section 5 seed finding).
//
// Accumulator tile layout.  The tile covers R = WR * P consecutive theta
// rows.  Shared memory holds WR "word rows" of `stride` 32-bit words; word
// (wr, b) packs P counters of cw = 32/P bits: counter s is the count of bin b
// in tile row s*WR + wr.  P = 4 (8-bit) when the window has <= 255 hits,
// P = 2 (16-bit) when <= 65535, else P = 1: a count never exceeds the number
// of hits, so the packed counters are exact.  stride = n_rho + pad with
// stride = 1 (mod 32), so that lanes voting into 32 consecutive word rows
// at nearby bins fall into distinct banks.
//
// Voting assigns lane l of a warp to word row 32*g + l and loops the warp over
// hits; each lane adds one vote per packed row.  No two lanes of a warp ever
// touch the same word, so no warp aggregation is needed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hough.h"

namespace hk {

constexpr int kFrac = HOUGH_FRAC_BITS;
constexpr int kKeyBuf = 2048;               // top-k region + candidate buffer (u64 keys)
constexpr unsigned long long kKeyMax = ~0ull;

struct KParams {
    // hits
    const int32_t *a;   // phi_q, or vane when raw
    const int32_t *b;   // z_q, or strip when raw
    long long n_hits;
    int raw;
    int vane_step;      // phi units per vane
    int z_min_u, z_pitch_u, z_half;
    long long phi_end;  // 360 deg in phi units
    long long z_end;    // z_min + n_z_strips * pitch
    // windows
    const long long *offsets;
    long long n_windows;
    // tables
    const int32_t *C;
    const int32_t *S;
    long long D;
    int n_theta, n_rho;
    int T, tol, max_peaks;
    int export_acc;
    // outputs
    hough_peak *peaks;
    int32_t *n_peaks;
    int32_t *n_found;
    int32_t *hit_track;
    int32_t *track_hits;
    uint32_t *status;
    int32_t *acc;
    // scheduling: [0] next-window counter, [1] finished-CTA counter
    unsigned int *work;
    // launch shape
    int word_rows;      // WR, multiple of 32
    int stride;         // words per word row
    int hit_stage;      // HS
    int kp;             // top-k region (power of two >= max(32, max_peaks))
};

// Shared-memory carve-up shared by host (size) and device (pointers).
struct SmemLayout {
    size_t acc, stage, carry, keys, pk, cnt, wtot, total;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline SmemLayout smem_layout(int word_rows, int stride, int hit_stage, int n_rho)
{
    SmemLayout L;
    size_t off = 0;
    L.acc = off;
    off = align_up(off + (size_t)word_rows * stride * 4, 16);
    L.stage = off;
    off = align_up(off + (size_t)hit_stage * 8, 16);
    L.carry = off;
    off = align_up(off + (size_t)2 * n_rho * 4, 16);
    L.keys = off;
    off = align_up(off + (size_t)kKeyBuf * 8, 16);
    L.pk = off;                                     // t, b, C, S per kept peak
    off = align_up(off + (size_t)4 * HOUGH_MAX_PEAKS * 4, 16);
    L.cnt = off;                                    // counts + cursors per category
    off = align_up(off + (size_t)2 * (HOUGH_MAX_PEAKS + 2) * 4, 16);
    L.wtot = off;
    off = align_up(off + 32 * 4, 16);
    L.total = off;
    return L;
}

struct WinScalars {
    unsigned long long kth;   // admit a candidate key only if key < kth
    int n_cand;               // candidates appended since the last merge
    int n_found;              // local maxima >= T in the window (all of them)
    int n_top;                // kept peaks in keys[0 .. n_top)
    unsigned int flags;       // HOUGH_WIN_* for this window
    int next_w;               // next window for this CTA
    int n_valid;              // staged (valid) hits
};

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Encoded (phi, z) of hit i, and whether it lies inside the detector box.
__device__ __forceinline__ bool load_hit(const KParams &p, long long i, int &phi, int &z)
{
    int a = __ldg(p.a + i);
    int b = __ldg(p.b + i);
    if (p.raw) {
        phi = (int)((long long)p.vane_step * (long long)a);
        z = (int)((long long)p.z_min_u + (long long)p.z_pitch_u * (long long)b + p.z_half);
    } else {
        phi = a;
        z = b;
    }
    return phi >= 0 && (long long)phi < p.phi_end && z >= p.z_min_u && (long long)z <= p.z_end;
}

__device__ __forceinline__ int rho_bin(int phi, int z, int c, int s, long long D)
{
    long long v = (long long)phi * (long long)c + (long long)z * (long long)s + D;
    return (int)(v >> kFrac);   // arithmetic shift = floor division by 2^24
}

// Stage hits [base, base + n) of the global arrays into `stage`, keeping only
// valid hits, in their original order.  Returns the number staged (uniform).
__device__ int stage_hits(const KParams &p, long long base, int n, int2 *stage, int *wtot,
                          WinScalars &ws)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int total = 0;
    bool bad = false;
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
        int i = c0 + threadIdx.x;
        int phi = 0, z = 0;
        bool ok = false;
        if (i < n) {
            ok = load_hit(p, base + i, phi, z);
            bad |= !ok;
        }
        unsigned m = __ballot_sync(0xffffffffu, ok);
        if (lane == 0)
            wtot[warp] = __popc(m);
        __syncthreads();
        int pre = 0, tot = 0;
        for (int k = 0; k < nw; ++k) {
            int v = wtot[k];
            pre += (k < warp) ? v : 0;
            tot += v;
        }
        if (ok)
            stage[total + pre + __popc(m & lanemask_lt())] = make_int2(phi, z);
        total += tot;
        __syncthreads();
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0)
        atomicOr(&ws.flags, HOUGH_WIN_HIT_OUT_OF_RANGE);
    return total;
}

// Step B on one tile: every staged hit votes once in each of the tile's rows.
template <int P>
__device__ void vote_tile(const KParams &p, uint32_t *acc, const int2 *stage, int nh, int t0,
                          WinScalars &ws)
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
        int t = t0 + k * WR + wr;
        act[k] = t < p.n_theta;
        c[k] = act[k] ? __ldg(p.C + t) : 0;
        s[k] = act[k] ? __ldg(p.S + t) : 0;
    }
    uint32_t *row = acc + (size_t)wr * p.stride;
    const long long D = p.D;
    const unsigned nr = (unsigned)p.n_rho;
    bool oor = false;
#pragma unroll 4
    for (int h = warp / G; h < nh; h += hstep) {
        int2 hv = stage[h];
#pragma unroll
        for (int k = 0; k < P; ++k) {
            if (act[k]) {
                int b = rho_bin(hv.x, hv.y, c[k], s[k], D);
                if ((unsigned)b < nr)
                    atomicAdd(row + b, 1u << (k * CW));
                else
                    oor = true;
            }
        }
    }
    if (oor)
        atomicOr(&ws.flags, HOUGH_WIN_VOTE_OUT_OF_RANGE);
}

// Value of tile-local row i (0 <= i < WR*P) at bin b.
__device__ __forceinline__ int tile_val(const uint32_t *acc, int stride, int WR, int P, int i, int b)
{
    int s = i / WR, wr = i - s * WR;
    uint32_t w = acc[(size_t)wr * stride + b];
    int cw = 32 / P;
    return P == 1 ? (int)w : (int)((w >> (s * cw)) & ((1u << cw) - 1u));
}

struct TileView {
    const uint32_t *acc;
    const int *carry0;   // row t0 - 2
    const int *carry1;   // row t0 - 1
    int t0, R, WR, P, stride, n_theta, n_rho;

    __device__ __forceinline__ int get(int t, int b) const
    {
        if (t < 0 || t >= n_theta || b < 0 || b >= n_rho)
            return 0;
        int i = t - t0;
        if (i >= 0)
            return i < R ? tile_val(acc, stride, WR, P, i, b) : 0;
        if (i == -1)
            return carry1[b];
        if (i == -2)
            return carry0[b];
        return 0;
    }
};

__device__ __forceinline__ unsigned long long make_key(int v, int t, int b)
{
    return ((unsigned long long)(0xffffffffu - (unsigned)v) << 32) |
           ((unsigned long long)t << 16) | (unsigned long long)b;
}

// Local-maximum test of Section 4/5 with the row-major tie-break, then feed.
__device__ __forceinline__ void consider(const KParams &p, const TileView &tv, int t, int b, int v,
                                         bool count, unsigned long long *cand, int cand_cap,
                                         WinScalars &ws)
{
    if (!(v > tv.get(t - 1, b - 1) && v > tv.get(t - 1, b) && v > tv.get(t - 1, b + 1) &&
          v > tv.get(t, b - 1) && v >= tv.get(t, b + 1) && v >= tv.get(t + 1, b - 1) &&
          v >= tv.get(t + 1, b) && v >= tv.get(t + 1, b + 1)))
        return;
    if (count)
        atomicAdd(&ws.n_found, 1);
    unsigned long long key = make_key(v, t, b);
    if (key < ws.kth) {
        int idx = atomicAdd(&ws.n_cand, 1);
        if (idx < cand_cap)
            cand[idx] = key;
    }
}

template <int P>
__device__ __forceinline__ bool any_ge(uint32_t w, int T)
{
    if (P == 1)
        return (int)w >= T;
    if (P == 2)
        return (int)max(w & 0xffffu, w >> 16) >= T;
    return __vcmpgeu4(w, (unsigned)T * 0x01010101u) != 0u;
}

// Scan evaluable rows [rlo, rhi) of the current view for peaks.
template <int P>
__device__ void scan_rows(const KParams &p, const TileView &tv, int rlo, int rhi, bool count,
                          unsigned long long *cand, int cand_cap, WinScalars &ws)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int T = p.T;
    // the previous tile's last row lives in the carry buffer
    int tc = tv.t0 - 1;
    if (tc >= 0 && tc >= rlo && tc < rhi) {
        for (int b = threadIdx.x; b < p.n_rho; b += blockDim.x) {
            int v = tv.carry1[b];
            if (v >= T)
                consider(p, tv, tc, b, v, count, cand, cand_cap, ws);
        }
    }
    int ilo = max(rlo - tv.t0, 0), ihi = min(rhi - tv.t0, tv.R);
    if (ilo >= ihi)
        return;
    constexpr int CW = 32 / P;
    for (int wr = warp; wr < tv.WR; wr += nw) {
        // rows of this word row that fall in [ilo, ihi)
        bool any_row = false;
#pragma unroll
        for (int s = 0; s < P; ++s) {
            int i = s * tv.WR + wr;
            any_row |= (i >= ilo && i < ihi);
        }
        if (!any_row)
            continue;
        const uint32_t *row = tv.acc + (size_t)wr * tv.stride;
        for (int b = lane; b < p.n_rho; b += 32) {
            uint32_t w = row[b];
            if (!any_ge<P>(w, T))
                continue;
#pragma unroll
            for (int s = 0; s < P; ++s) {
                int i = s * tv.WR + wr;
                int v = P == 1 ? (int)w : (int)((w >> (s * CW)) & ((1u << CW) - 1u));
                if (v >= T && i >= ilo && i < ihi)
                    consider(p, tv, tv.t0 + i, b, v, count, cand, cand_cap, ws);
            }
        }
    }
}

// Ascending bitonic sort of a[0..n), n a power of two, by the whole block.
__device__ void bitonic_sort(unsigned long long *a, int n)
{
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    unsigned long long x = a[i], y = a[ixj];
                    bool up = (i & k) == 0;
                    if ((x > y) == up) {
                        a[i] = y;
                        a[ixj] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// keys[0 .. kp) = kept list padded with kKeyMax; keys[kp .. kp + n_cand) =
// new candidates.  Sort everything, keep the best max_peaks, tighten kth.
__device__ void merge_candidates(const KParams &p, unsigned long long *keys, WinScalars &ws)
{
    __syncthreads();
    int nc = min(ws.n_cand, kKeyBuf - p.kp);
    int used = p.kp + nc;
    int n = 1;
    while (n < used)
        n <<= 1;
    for (int i = used + threadIdx.x; i < n; i += blockDim.x)
        keys[i] = kKeyMax;
    __syncthreads();
    bitonic_sort(keys, n);
    int keep = min(p.max_peaks, ws.n_top + nc);
    for (int i = p.max_peaks + threadIdx.x; i < p.kp; i += blockDim.x)
        keys[i] = kKeyMax;
    __syncthreads();
    if (threadIdx.x == 0) {
        ws.n_top = keep;
        ws.n_cand = 0;
        ws.kth = (p.max_peaks > 0 && keep == p.max_peaks) ? keys[p.max_peaks - 1] : kKeyMax;
        if (p.max_peaks == 0)
            ws.kth = 0ull;
    }
    __syncthreads();
}

template <int P>
__device__ void process_tiles(const KParams &p, long long beg, int H, uint32_t *acc, int2 *stage,
                              int *carry, unsigned long long *keys, int *wtot, WinScalars &ws,
                              long long w)
{
    const int WR = p.word_rows;
    const int R = WR * P;
    const int n_tiles = (p.n_theta + R - 1) / R;
    const bool single = H <= p.hit_stage;
    const int cand_cap = kKeyBuf - p.kp;
    unsigned long long *cand = keys + p.kp;
    int *carry0 = carry, *carry1 = carry + p.n_rho;
    const size_t acc_words4 = (size_t)WR * p.stride / 4;

    int nv = 0;
    if (single)
        nv = stage_hits(p, beg, H, stage, wtot, ws);

    for (int tile = 0; tile < n_tiles; ++tile) {
        const int t0 = tile * R;
        const bool last = tile == n_tiles - 1;
        uint4 *acc4 = reinterpret_cast<uint4 *>(acc);
        for (size_t i = threadIdx.x; i < acc_words4; i += blockDim.x)
            acc4[i] = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
        if (single) {
            vote_tile<P>(p, acc, stage, nv, t0, ws);
        } else {
            for (long long s0 = 0; s0 < H; s0 += p.hit_stage) {
                int n = (int)min((long long)p.hit_stage, (long long)H - s0);
                int ns = stage_hits(p, beg + s0, n, stage, wtot, ws);
                vote_tile<P>(p, acc, stage, ns, t0, ws);
                __syncthreads();
            }
        }
        __syncthreads();

        if (p.export_acc) {
            const int r_eff = min(R, p.n_theta - t0);
            const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            for (int i = warp; i < r_eff; i += nw) {
                int32_t *dst = p.acc + ((size_t)w * p.n_theta + (size_t)(t0 + i)) * p.n_rho;
                for (int b = lane; b < p.n_rho; b += 32)
                    dst[b] = tile_val(acc, p.stride, WR, P, i, b);
            }
        }

        TileView tv{acc, carry0, carry1, t0, R, WR, P, p.stride, p.n_theta, p.n_rho};
        const int rlo = max(t0 - 1, 0);
        const int rhi = last ? p.n_theta : t0 + R - 1;
        const int n_before = ws.n_cand;      // unmerged candidates of earlier tiles
        __syncthreads();
        scan_rows<P>(p, tv, rlo, rhi, true, cand, cand_cap, ws);
        __syncthreads();
        if (ws.n_cand > cand_cap) {
            // Rare: the buffer overflowed.  Keep the earlier tiles' entries
            // (they precede this tile's in the buffer), merge them, then rescan
            // this tile in slices small enough that their peaks always fit
            // (peaks are never 8-neighbours, so r rows hold at most
            // ceil(r/2) * ceil(n_rho/2) of them).
            __syncthreads();
            if (threadIdx.x == 0)
                ws.n_cand = n_before;
            __syncthreads();
            if (n_before > 0)
                merge_candidates(p, keys, ws);
            int per_row_pair = (p.n_rho + 1) / 2;
            int rows = max(1, 2 * (cand_cap / per_row_pair));
            for (int r0 = rlo; r0 < rhi; r0 += rows) {
                scan_rows<P>(p, tv, r0, min(r0 + rows, rhi), false, cand, cand_cap, ws);
                __syncthreads();
                if (ws.n_cand > 0)
                    merge_candidates(p, keys, ws);
            }
        } else if (ws.n_cand > 0 && (last || ws.n_cand > cand_cap / 2)) {
            merge_candidates(p, keys, ws);
        }
        if (!last) {
            for (int b = threadIdx.x; b < p.n_rho; b += blockDim.x) {
                carry0[b] = tile_val(acc, p.stride, WR, P, R - 2, b);
                carry1[b] = tile_val(acc, p.stride, WR, P, R - 1, b);
            }
        }
        __syncthreads();
    }
}

// Step D: first matching peak in order, then per-peak compaction.
__device__ void associate(const KParams &p, long long w, long long beg, int H, int n_top,
                          const unsigned long long *keys, int *pk, int *cnt, int *cursor,
                          int *cat_s, bool cat_in_smem, WinScalars &ws)
{
    int *pk_t = pk, *pk_b = pk + HOUGH_MAX_PEAKS, *pk_c = pk + 2 * HOUGH_MAX_PEAKS,
        *pk_s = pk + 3 * HOUGH_MAX_PEAKS;
    for (int i = threadIdx.x; i < n_top; i += blockDim.x) {
        unsigned long long k = keys[i];
        int t = (int)((k >> 16) & 0xffffu);
        pk_t[i] = t;
        pk_b[i] = (int)(k & 0xffffu);
        pk_c[i] = __ldg(p.C + t);
        pk_s[i] = __ldg(p.S + t);
    }
    for (int i = threadIdx.x; i < n_top + 2; i += blockDim.x)
        cnt[i] = 0;
    __syncthreads();
    const long long D = p.D;
    const int tol = p.tol;
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        int phi, z;
        bool ok = load_hit(p, beg + i, phi, z);
        int cat = n_top + 1;
        if (ok) {
            cat = n_top;
            for (int q = 0; q < n_top; ++q) {
                int d = rho_bin(phi, z, pk_c[q], pk_s[q], D) - pk_b[q];
                if (d <= tol && d >= -tol) {
                    cat = q;
                    break;
                }
            }
        }
        p.hit_track[beg + i] = cat < n_top ? cat : (cat == n_top ? -1 : -2);
        if (cat_in_smem)
            cat_s[i] = cat;
        atomicAdd(&cnt[cat], 1);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int run = 0;
        for (int base = 0; base < n_top + 2; base += 32) {
            int q = base + lane;
            int c = q < n_top + 2 ? cnt[q] : 0;
            int incl = c;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d)
                    incl += y;
            }
            int excl = run + incl - c;
            if (q < n_top + 2)
                cursor[q] = excl;
            if (q < n_top) {
                unsigned long long k = keys[q];
                hough_peak pr;
                pr.theta = (uint16_t)((k >> 16) & 0xffffu);
                pr.rho = (uint16_t)(k & 0xffffu);
                pr.votes = (int32_t)(0xffffffffu - (unsigned)(k >> 32));
                pr.n_hits = c;
                pr.hit_begin = excl;
                p.peaks[(size_t)w * p.max_peaks + q] = pr;
            }
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
        __syncwarp();
        for (int base = 0; base < H; base += 32) {
            int i = base + lane;
            bool in = i < H;
            int cat = -1;
            if (in) {
                if (cat_in_smem) {
                    cat = cat_s[i];
                } else {
                    int v = p.hit_track[beg + i];
                    cat = v >= 0 ? v : (v == -1 ? n_top : n_top + 1);
                }
            }
            unsigned m = __match_any_sync(0xffffffffu, cat);
            int leader = __ffs(m) - 1;
            int rank = __popc(m & lanemask_lt());
            int pos = 0;
            if (in && lane == leader) {
                pos = cursor[cat];
                cursor[cat] = pos + __popc(m);
            }
            pos = __shfl_sync(0xffffffffu, pos, leader);
            if (in)
                p.track_hits[beg + pos + rank] = i;
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(1024, 1) find_kernel(KParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ WinScalars ws;
    const SmemLayout L = smem_layout(p.word_rows, p.stride, p.hit_stage, p.n_rho);
    uint32_t *acc = reinterpret_cast<uint32_t *>(smem + L.acc);
    int2 *stage = reinterpret_cast<int2 *>(smem + L.stage);
    int *carry = reinterpret_cast<int *>(smem + L.carry);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(smem + L.keys);
    int *pk = reinterpret_cast<int *>(smem + L.pk);
    int *cnt = reinterpret_cast<int *>(smem + L.cnt);
    int *cursor = cnt + (HOUGH_MAX_PEAKS + 2);
    int *wtot = reinterpret_cast<int *>(smem + L.wtot);

    long long w = blockIdx.x;
    while (w < p.n_windows) {
        long long beg = p.offsets[w], end = p.offsets[w + 1];
        bool bad = !(beg >= 0 && beg <= end && end <= p.n_hits && end - beg < (1ll << 30));
        if (bad) {
            if (threadIdx.x == 0) {
                p.status[w] = HOUGH_WIN_BAD_OFFSETS;
                p.n_peaks[w] = 0;
                if (p.n_found)
                    p.n_found[w] = 0;
            }
        } else {
            const int H = (int)(end - beg);
            if (threadIdx.x == 0) {
                ws.kth = p.max_peaks > 0 ? kKeyMax : 0ull;
                ws.n_cand = 0;
                ws.n_found = 0;
                ws.n_top = 0;
                ws.flags = 0u;
            }
            for (int i = threadIdx.x; i < p.kp; i += blockDim.x)
                keys[i] = kKeyMax;
            __syncthreads();
            if (H <= 255)
                process_tiles<4>(p, beg, H, acc, stage, carry, keys, wtot, ws, w);
            else if (H <= 65535)
                process_tiles<2>(p, beg, H, acc, stage, carry, keys, wtot, ws, w);
            else
                process_tiles<1>(p, beg, H, acc, stage, carry, keys, wtot, ws, w);
            __syncthreads();
            const int n_top = ws.n_top;
            const bool cat_in_smem = H <= 2 * p.hit_stage;
            associate(p, w, beg, H, n_top, keys, pk, cnt, cursor, reinterpret_cast<int *>(stage),
                      cat_in_smem, ws);
            if (threadIdx.x == 0) {
                unsigned fl = ws.flags;
                if (ws.n_found > p.max_peaks)
                    fl |= HOUGH_WIN_PEAK_OVERFLOW;
                p.status[w] = fl;
                p.n_peaks[w] = n_top;
                if (p.n_found)
                    p.n_found[w] = ws.n_found;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0)
            ws.next_w = (int)gridDim.x + (int)atomicAdd(p.work, 1u);
        __syncthreads();
        w = ws.next_w;
    }
    // The last CTA to finish resets the scheduling counters for the next launch.
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned done = atomicAdd(p.work + 1, 1u);
        if (done == gridDim.x - 1) {
            atomicExch(p.work, 0u);
            atomicExch(p.work + 1, 0u);
            __threadfence();
        }
    }
}

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
