// hough_kernels.cuh -- device code of the track-finding path (sm_103a).
//
// One persistent kernel processes whole time windows (Section 6: one window
// per unit of work).  Per window, in one CTA:
//   1. stage: the window's hits are loaded (encoded on the fly from strip
//      addresses if asked), checked against the detector box and compacted
//      into shared memory;
//   2. for each theta tile: zero the shared accumulator tile, vote (Eq. (1)),
//      optionally export it, collect the bins >= T, test them for 3x3 local
//      maxima and feed the peaks to an exact online top-k (Section 4 /
//      Section 5 peak finding);
//   3. associate every hit with the first peak whose line it lies on and
//      compact the hits per peak (Section 5 seed finding).
//
// Accumulator tile layout.  The tile covers R = WR * P consecutive theta
// rows.  Its WR "word rows" hold P packed counters per 32-bit word: counter s
// of word (wr, b) is the count of bin b in tile row s*WR + wr.  P = 4 (8-bit)
// when the window has <= 255 hits, P = 2 (16-bit) when <= 65535, else P = 1:
// a count never exceeds the number of hits, so the packed counters are exact.
// Words are stored bank-private: word (wr, b) lives at
//     ((wr / 32) * n_rho + b) * 32 + wr % 32,
// so every word of word row wr sits in shared-memory bank wr % 32.
//
// Voting assigns lane l of a warp to word row 32*g + l and loops the warp over
// hits; each lane adds one vote per packed row.  Lane l only ever touches bank
// l, so a warp's vote atomic is always a single conflict-free wavefront,
// whatever bins the lanes hit (and no two lanes share a word, so no warp
// aggregation is needed).  The votes use reduction atomics (no return value).
// The tile is then scanned 16 bytes at a time with a SIMD-within-a-word test
// for "some counter >= T"; only the indices of the 16-byte groups that pass
// are listed, and a second pass tests the listed counters for 3x3 local
// maxima.
//
// Book-keeping never uses a shared-memory atomic that many warps hit at
// once (those serialise at tens of cycles each): every warp lists its
// candidates and its peaks into its own segment with a register counter, and
// segments are joined through a prefix over the warps.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hough.h"

namespace hk {

constexpr int kSegPk = 64;      // peak-key segment per warp; merged when past 32 entries
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
    int D;              // tables at scale 2^K: every box hit's sum fits in int32
    int K;
    int in_range;       // every valid hit votes inside [0, n_rho) in every row
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
    int word_rows;      // WR, 32, 64 or 128
    int lw;             // log2(WR)
    unsigned nrho_inv;  // ceil(2^32 / n_rho): word-column index -> row group
    int hit_stage;      // HS
    int kp;             // top-k region (power of two >= max(32, max_peaks))
    int seg_cl;         // candidate-list entries per warp
};

// Shared-memory carve-up shared by host (size) and device (pointers).
struct SmemLayout {
    size_t acc, stage, carry, keys, cl, pk, cnt, hist, vh, pre, wtot, total;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline SmemLayout smem_layout(int word_rows, int hit_stage, int n_rho,
                                                   int cl_entries, int n_warps)
{
    SmemLayout L;
    size_t off = 0;
    L.acc = off;
    off = align_up(off + (size_t)word_rows * n_rho * 4, 16);
    L.stage = off;
    off = align_up(off + (size_t)hit_stage * 8, 16);
    L.carry = off;
    off = align_up(off + (size_t)2 * n_rho * 4, 16);
    L.keys = off;                                   // kept list + one peak segment per warp
    off = align_up(off + (size_t)(HOUGH_MAX_PEAKS + n_warps * kSegPk) * 8, 16);
    L.cl = off;                                     // candidate lists, one per warp
    off = align_up(off + (size_t)cl_entries * 4, 16);
    L.pk = off;                                     // t, b, C, S per kept peak
    off = align_up(off + (size_t)4 * HOUGH_MAX_PEAKS * 4, 16);
    L.cnt = off;                                    // counts + cursors per category
    off = align_up(off + (size_t)2 * (HOUGH_MAX_PEAKS + 2) * 4, 16);
    L.hist = off;                                   // per-warp counters (WarpCounters)
    off = align_up(off + (size_t)5 * 32 * 4, 16);
    L.vh = off;                                     // per-warp peak-vote histograms
    off = align_up(off + (size_t)n_warps * 64 * 4, 16);
    L.pre = off;                                    // per-thread list prefix
    off = align_up(off + (size_t)n_warps * 32 * 4, 16);
    L.wtot = off;
    off = align_up(off + 32 * 4, 16);
    L.total = off;
    return L;
}

struct WinScalars {
    unsigned long long kth;   // a peak enters a segment only if its key < kth
    int n_top;                // kept peaks in keys[0 .. n_top)
    int n_sel;                // entries gathered for a merge
    int seg_ovf;              // a warp's candidate list overflowed in this tile
    int vk;                   // lower bound of the k-th best vote count
    int n_keep_top;           // kept-list entries with >= vk votes (merging)
    unsigned int flags;       // HOUGH_WIN_* for this window
    int next_w;               // next window for this CTA
};

// Per-warp counters kept in shared memory between phases.
struct WarpCounters {
    int *n_cl;      // candidate-list entries of the warp in this tile
    int *n_pk;      // peaks in the warp's segment since the last merge
    int *n_found;   // local maxima >= T found by the warp in this window
    int *pre_cl;    // exclusive prefix of n_cl (spreading the check over warps)
    int *pre_pk;    // exclusive prefix of n_pk (merging); separate from pre_cl
                    // because a merge can run in the middle of the check
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

// floor((phi*c + z*s + D) / 2^K): the tables' scale keeps the exact sum of
// any hit of the detector box inside int32, so 32-bit wrap-around arithmetic
// gives it exactly; the arithmetic shift is the floor division.
__device__ __forceinline__ int rho_bin(int phi, int z, int c, int s, int D, int K)
{
    const unsigned v = (unsigned)phi * (unsigned)c + (unsigned)z * (unsigned)s + (unsigned)D;
    return (int)v >> K;
}

__device__ __forceinline__ unsigned atom_add_shared(unsigned addr, unsigned v)
{
    unsigned old;
    asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(addr), "r"(v) : "memory");
    return old;
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
// A vote whose atomic returns T - 1 made its bin reach T (exactly once per
// such bin): the bin is listed in the lane's own column of the warp's list,
// seg[slot * 32 + lane], as (word index << 2) | field, cnt being the lane's
// register count (no shared counter, no warp vote).  cnt may pass L: then
// only the first L entries were stored.  FAST: the host proved that every
// valid hit votes in range, and the tile has no row past n_theta, so the
// per-vote checks are left out.
template <int P, bool FAST>
__device__ void vote_tile(const KParams &p, uint32_t *acc, const int2 *stage, int nh, int t0,
                          uint32_t *seg, int L, int &cnt, WinScalars &ws)
{
    constexpr int CW = 32 / P;
    constexpr unsigned MASK = P == 1 ? 0xffffffffu : ((1u << CW) - 1u);
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
    // bank-private column of this lane: word (wr, b) at col_word0 + 32 b
    const unsigned col_word0 = (unsigned)(g * p.n_rho) * 32u + (unsigned)lane;
    const unsigned col = (unsigned)__cvta_generic_to_shared(acc) + 4u * col_word0;
    const int D = p.D, K = p.K;
    const unsigned nr = (unsigned)p.n_rho;
    const unsigned tm1 = (unsigned)(p.T - 1);
    bool oor = false;
#pragma unroll 2
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
            const unsigned old = in ? atom_add_shared(col + (unsigned)b * 128u, 1u << (k * CW)) : 0u;
            if (in && ((old >> (k * CW)) & MASK) == tm1) {
                if (cnt < L)
                    seg[cnt * 32 + lane] = ((col_word0 + (unsigned)b * 32u) << 2) | (unsigned)k;
                ++cnt;
            }
        }
    }
    if (oor)
        atomicOr(&ws.flags, HOUGH_WIN_VOTE_OUT_OF_RANGE);
}

template <int P>
__device__ __forceinline__ int field(uint32_t w, int s)
{
    constexpr int CW = 32 / P;
    return P == 1 ? (int)w : (int)((w >> (s * CW)) & ((1u << CW) - 1u));
}

// Shared-memory index of word (wr, b) in the bank-private layout.
__device__ __forceinline__ int word_index(int wr, int b, int n_rho)
{
    return ((wr >> 5) * n_rho + b) * 32 + (wr & 31);
}

// Value of tile-local row i (0 <= i < WR*P) at bin b.
template <int P>
__device__ __forceinline__ int tile_val(const uint32_t *acc, int n_rho, int lw, int i, int b)
{
    int s = i >> lw, wr = i & ((1 << lw) - 1);
    return field<P>(acc[word_index(wr, b, n_rho)], s);
}

template <int P>
struct TileView {
    const uint32_t *acc;
    const int *carry0;   // row t0 - 2
    const int *carry1;   // row t0 - 1
    int t0, R, lw, n_theta, n_rho;

    // Count of (theta row t, rho bin b), 0 outside the accumulator.  Branch
    // free: the tile word and the carried value are both loaded (with clamped
    // indices) and the right one is selected, so that the eight loads of a
    // neighbourhood test are issued together.
    __device__ __forceinline__ int get(int t, int b) const
    {
        constexpr int CW = 32 / P;
        constexpr unsigned MASK = P == 1 ? 0xffffffffu : ((1u << CW) - 1u);
        const int i = t - t0;
        const int ic = min(max(i, 0), R - 1);
        const int bc = min(max(b, 0), n_rho - 1);
        const int sl = ic >> lw, wr = ic & ((1 << lw) - 1);
        const uint32_t w = acc[((wr >> 5) * n_rho + bc) * 32 + (wr & 31)];
        const int vt = (int)((w >> (sl * CW)) & MASK);
        const int vc = (i == -2 ? carry0 : carry1)[bc];
        const int v = i >= 0 ? vt : vc;
        const bool inside = (unsigned)t < (unsigned)n_theta && (unsigned)b < (unsigned)n_rho &&
                            i >= -2 && i < R;
        return inside ? v : 0;
    }

    // Section 4/5 peak rule: > earlier neighbours (row-major), >= later ones.
    __device__ __forceinline__ bool is_peak(int t, int b, int v) const
    {
        const int a0 = get(t - 1, b - 1), a1 = get(t - 1, b), a2 = get(t - 1, b + 1);
        const int a3 = get(t, b - 1), a4 = get(t, b + 1);
        const int a5 = get(t + 1, b - 1), a6 = get(t + 1, b), a7 = get(t + 1, b + 1);
        const int earlier = max(max(a0, a1), max(a2, a3));
        const int later = max(max(a4, a5), max(a6, a7));
        return v > earlier && v >= later;
    }
};

__device__ __forceinline__ unsigned long long make_key(int v, int t, int b)
{
    return ((unsigned long long)(0xffffffffu - (unsigned)v) << 32) |
           ((unsigned long long)t << 16) | (unsigned long long)b;
}

__device__ __forceinline__ int key_votes(unsigned long long k)
{
    return (int)(0xffffffffu - (unsigned)(k >> 32));
}

// Threshold test on a packed word.  For 8- and 16-bit fields with T at most
// half the field range, field >= T exactly when the field's top bit of
// w | ((w & low) + add) is set (add = (2^(cw-1) - T) per field; the masked
// sum cannot carry into the next field).
struct ScanTest {
    uint32_t low, add, hi;
    int T;
    bool swar;
};

template <int P>
__device__ __forceinline__ ScanTest make_test(int T)
{
    ScanTest k;
    k.T = T;
    if (P == 4) {
        k.low = 0x7f7f7f7fu;
        k.hi = 0x80808080u;
        k.swar = T <= 128;
        k.add = k.swar ? (unsigned)(128 - T) * 0x01010101u : 0u;
    } else if (P == 2) {
        k.low = 0x7fff7fffu;
        k.hi = 0x80008000u;
        k.swar = T <= 32768;
        k.add = k.swar ? (unsigned)(32768 - T) * 0x00010001u : 0u;
    } else {
        k.low = k.hi = k.add = 0u;
        k.swar = false;
    }
    return k;
}

template <int P>
__device__ __forceinline__ bool word_has(uint32_t w, const ScanTest &k)
{
    if (P == 1)
        return (int)w >= k.T;
    if (k.swar)
        return ((w | ((w & k.low) + k.add)) & k.hi) != 0u;
#pragma unroll
    for (int s = 0; s < P; ++s)
        if (field<P>(w, s) >= k.T)
            return true;
    return false;
}

template <int P>
__device__ __forceinline__ bool quad_has(const uint4 &q, const ScanTest &k)
{
    if (P != 1 && k.swar) {
        uint32_t m = (q.x | ((q.x & k.low) + k.add)) | (q.y | ((q.y & k.low) + k.add)) |
                     (q.z | ((q.z & k.low) + k.add)) | (q.w | ((q.w & k.low) + k.add));
        return (m & k.hi) != 0u;
    }
    return word_has<P>(q.x, k) || word_has<P>(q.y, k) || word_has<P>(q.z, k) ||
           word_has<P>(q.w, k);
}

__device__ __forceinline__ uint32_t quad_word(const uint4 &q, int e)
{
    return e == 0 ? q.x : (e == 1 ? q.y : (e == 2 ? q.z : q.w));
}

// Per-field flags "counter >= T" of a packed word: the top bit of each
// field of the returned word is set for the fields that pass (for P = 1 the
// word itself is the counter and bit 31 carries the flag).
template <int P>
__device__ __forceinline__ uint32_t field_flags(uint32_t w, const ScanTest &k)
{
    if (P == 1)
        return (int)w >= k.T ? 0x80000000u : 0u;
    if (k.swar)
        return (w | ((w & k.low) + k.add)) & k.hi;
    constexpr int CW = 32 / P;
    uint32_t f = 0u;
#pragma unroll
    for (int s = 0; s < P; ++s)
        if (field<P>(w, s) >= k.T)
            f |= 1u << (s * CW + CW - 1);
    return f;
}

// Add the bins >= T of the previous tile's last row (carry buffer, evaluated
// with this tile) to the lanes' columns as 0x80000000 | b; every thread takes
// every blockDim-th bin.
template <int P>
__device__ void list_carry(const KParams &p, const TileView<P> &tv, int rlo, int rhi,
                           uint32_t *seg, int L, int &cnt)
{
    const int lane = threadIdx.x & 31;
    const int tc = tv.t0 - 1;
    if (!(tc >= 0 && tc >= rlo && tc < rhi))
        return;
    for (int b = threadIdx.x; b < p.n_rho; b += blockDim.x) {
        if (tv.carry1[b] >= p.T) {
            if (cnt < L)
                seg[cnt * 32 + lane] = 0x80000000u | (unsigned)b;
            ++cnt;
        }
    }
}

// Book-keeping of the peaks a warp found in one step (all lanes call): count
// them, and append the keys below the k-th best so far to the warp's segment.
struct PeakSink {
    unsigned long long *seg;   // this warp's peak segment
    int cap;                   // its capacity
    int n;                     // entries so far
    int found;                 // peaks found in this pass
    unsigned long long kth;
    int vk;                    // lower bound of the k-th best vote count
    int *hist;                 // this warp's row of the vote histogram (null: off)
};

constexpr int kHistBins = 64;   // per-warp peak-vote histogram; last bin = ">= 63"

__device__ __forceinline__ void record_peaks(bool peak, int v, int t, int b, PeakSink &ps)
{
    const unsigned m = __ballot_sync(0xffffffffu, peak);
    if (m == 0u)
        return;
    ps.found += __popc(m);
    if (peak && ps.hist)
        atomicAdd(ps.hist + min(v, kHistBins - 1), 1);   // this warp's own row
    const unsigned long long key = make_key(v, t, b);
    const bool app = peak && key < ps.kth && v >= ps.vk;
    const unsigned ma = __ballot_sync(0xffffffffu, app);
    const int pos = ps.n + __popc(ma & lanemask_lt());
    if (app && pos < ps.cap)
        ps.seg[pos] = key;
    ps.n += __popc(ma);
}

// The value, row and bin of a listed candidate.
template <int P>
__device__ __forceinline__ void decode_entry(const KParams &p, const TileView<P> &tv, uint32_t e,
                                             int &v, int &i, int &b)
{
    constexpr int CW = 32 / P;
    constexpr unsigned MASK = P == 1 ? 0xffffffffu : ((1u << CW) - 1u);
    if (e & 0x80000000u) {
        b = (int)(e & 0xffffu);
        i = -1;
        v = tv.carry1[b];
    } else {
        const int f = (int)(e >> 2), s = (int)(e & 3u);
        const int qq = f >> 5;                                     // g * n_rho + b
        const int g = (int)__umulhi((unsigned)qq, p.nrho_inv);
        b = qq - g * p.n_rho;
        i = s * p.word_rows + g * 32 + (f & 31);
        v = (int)((tv.acc[f] >> (s * CW)) & MASK);
    }
}

// Merge every warp's peak segment into the kept list.
//  1. From the per-warp vote histograms (every peak found so far in the
//     window), vk = the largest v with at least max_peaks peaks of >= v votes:
//     no peak with fewer votes can be among the best max_peaks.
//  2. Each warp compacts its segment, in place, to the entries with >= vk votes.
//  3. The kept list's prefix with >= vk votes and the compacted segments form
//     one virtual list (placed by a prefix over the warps); an entry's place
//     is the number of smaller keys (keys are distinct), so the best max_peaks
//     are written in order to a staging area and then to keys[0 ..).
// kth is tightened and the segments are emptied.
__device__ void merge_peaks(const KParams &p, unsigned long long *keys,
                            unsigned long long *top_stage, int seg_cap, WarpCounters wc,
                            const int *hist, WinScalars &ws)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned lt = lanemask_lt();
    __syncthreads();
    if (warp == 0) {
        int vk = 0x7fffffff;
        if (p.max_peaks > 0) {
            int h0 = 0, h1 = 0;
            for (int k = 0; k < nw; ++k) {
                h0 += hist[k * kHistBins + 2 * lane];
                h1 += hist[k * kHistBins + 2 * lane + 1];
            }
            const int mine = h0 + h1;
            int suf = mine;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_down_sync(0xffffffffu, suf, d);
                if (lane + d < 32)
                    suf += y;
            }
            const int above = suf - mine;
            int best = -1;
            if (above + h1 >= p.max_peaks)
                best = 2 * lane + 1;
            else if (above + h1 + h0 >= p.max_peaks)
                best = 2 * lane;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1)
                best = max(best, __shfl_xor_sync(0xffffffffu, best, d));
            vk = max(best, 0);
        }
        vk = max(vk, ws.vk);
        int keep_top = 0;
        for (int i = lane; i < ws.n_top; i += 32)
            keep_top += key_votes(keys[i]) >= vk ? 1 : 0;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1)
            keep_top += __shfl_xor_sync(0xffffffffu, keep_top, d);
        if (lane == 0) {
            ws.vk = vk;
            ws.n_keep_top = keep_top;
        }
    }
    __syncthreads();
    {
        const int vk = ws.vk;
        unsigned long long *seg = keys + p.kp + (size_t)warp * seg_cap;
        const int c = min(wc.n_pk[warp], seg_cap);
        int nn = 0;
        for (int i0 = 0; i0 < c; i0 += 32) {
            const int i = i0 + lane;
            const unsigned long long key = i < c ? seg[i] : kKeyMax;
            const bool ok = i < c && key_votes(key) >= vk;
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            if (ok)
                seg[nn + __popc(m & lt)] = key;   // never ahead of an unread entry
            nn += __popc(m);
        }
        if (lane == 0)
            wc.n_pk[warp] = nn;
    }
    __syncthreads();
    if (warp == 0) {
        const int c = lane < nw ? wc.n_pk[lane] : 0;
        int incl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d)
                incl += y;
        }
        if (lane < nw)
            wc.pre_pk[lane] = ws.n_keep_top + incl - c;
        if (lane == 31)
            ws.n_sel = ws.n_keep_top + incl;
    }
    __syncthreads();
    const int n_top = ws.n_keep_top;
    const int m = ws.n_sel;
    const int keep = min(p.max_peaks, m);
    const unsigned long long *segs = keys + p.kp;
    for (int idx = threadIdx.x; idx < m; idx += blockDim.x) {
        unsigned long long x;
        if (idx < n_top) {
            x = keys[idx];
        } else {
            int k = 0;
            while (k + 1 < nw && wc.pre_pk[k + 1] <= idx)
                ++k;
            x = segs[(size_t)k * seg_cap + (idx - wc.pre_pk[k])];
        }
        int rank = 0;
        for (int y = 0; y < n_top; ++y)
            rank += keys[y] < x ? 1 : 0;
        for (int k = 0; k < nw; ++k) {
            const unsigned long long *sg = segs + (size_t)k * seg_cap;
            const int c = wc.n_pk[k];
#pragma unroll 4
            for (int y = 0; y < c; ++y)
                rank += sg[y] < x ? 1 : 0;
        }
        if (rank < keep)
            top_stage[rank] = x;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < p.kp; i += blockDim.x)
        keys[i] = i < keep ? top_stage[i] : kKeyMax;
    if (lane == 0)
        wc.n_pk[warp] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        ws.n_top = keep;
        ws.kth = (p.max_peaks > 0 && keep == p.max_peaks) ? keys[p.max_peaks - 1] : kKeyMax;
        if (p.max_peaks == 0)
            ws.kth = 0ull;
    }
    __syncthreads();
}

// Export mode: write the tile's rows as int32 to acc[w][t][b].  A warp takes
// 32 word rows x 8 bins: each lane reads its own word row (one bank, no
// conflict), then shuffles turn the 32 x 8 block around so that every store
// instruction writes 8 consecutive bins of 4 rows (four whole 32-byte sectors).
template <int P>
__device__ void export_tile(const KParams &p, const uint32_t *acc, int t0, int R, long long w)
{
    const int WR = p.word_rows, G = WR >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nchunks = (p.n_rho + 7) >> 3;
    int32_t *out = p.acc + (size_t)w * p.n_theta * p.n_rho;
    for (int item = warp; item < G * nchunks; item += nw) {
        const int g = item / nchunks, b0 = (item - g * nchunks) * 8;
        uint32_t v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            v[j] = (b0 + j < p.n_rho) ? acc[(g * p.n_rho + b0 + j) * 32 + lane] : 0u;
        const int j = lane & 7;
        const int b = b0 + j;
#pragma unroll 1
        for (int q = 0; q < 8; ++q) {
            const int src = 4 * q + (lane >> 3);
            uint32_t word = 0u;
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                uint32_t x = __shfl_sync(0xffffffffu, v[jj], src);
                word = (j == jj) ? x : word;
            }
            const int wr = g * 32 + src;
#pragma unroll
            for (int s = 0; s < P; ++s) {
                const int i = s * WR + wr;
                const int t = t0 + i;
                if (i < R && t < p.n_theta && b < p.n_rho)
                    out[(size_t)t * p.n_rho + b] = field<P>(word, s);
            }
        }
    }
}

// Direct test of every counter of the evaluable rows: used only when a
// tile holds more candidate bins than the lists (adversarial inputs).
template <int P>
__device__ void check_direct(const KParams &p, const TileView<P> &tv, int rlo, int rhi,
                             PeakSink &ps, unsigned long long *keys, unsigned long long *top_stage,
                             int seg_cap, WarpCounters wc, const int *vh, WinScalars &ws)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ilo = max(rlo - tv.t0, -1), ihi = min(rhi - tv.t0, tv.R);
    const int nrows = ihi - ilo;
    const long long total = (long long)nrows * p.n_rho;
    for (long long x0 = 0; x0 < total; x0 += blockDim.x) {
        const long long x = x0 + threadIdx.x;
        const int i = ilo + (int)(x / p.n_rho);
        const int b = (int)(x % p.n_rho);
        const int t = tv.t0 + i;
        const int v = x < total ? tv.get(t, b) : 0;
        const bool peak = x < total && t >= rlo && v >= p.T && tv.is_peak(t, b, v);
        record_peaks(peak, v, t, b, ps);
        if (lane == 0)
            wc.n_pk[warp] = ps.n;
        if (__syncthreads_or(lane == 0 && ps.n > ps.cap - 32)) {
            merge_peaks(p, keys, top_stage, seg_cap, wc, vh, ws);
            ps.n = 0;
            ps.kth = ws.kth;
            ps.vk = ws.vk;
        }
    }
}

template <int P>
__device__ void process_tiles(const KParams &p, long long beg, int H, uint32_t *acc, int2 *stage,
                              int *carry, unsigned long long *keys, uint32_t *cl,
                              unsigned long long *top_stage, WarpCounters wc, int *vh,
                              int *pre_thr, int *wtot, WinScalars &ws, long long w)
{
    const int WR = p.word_rows;
    const int R = WR * P;
    const int n_tiles = (p.n_theta + R - 1) / R;
    const bool single = H <= p.hit_stage;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int seg_cap = kSegPk;
    int *carry0 = carry, *carry1 = carry + p.n_rho;
    const int acc_words4 = (WR * p.n_rho) >> 2;
    uint32_t *my_cl = cl + (size_t)warp * p.seg_cl;
    (void)lane;

    int nv = 0;
    if (single)
        nv = stage_hits(p, beg, H, stage, wtot, ws);

    for (int tile = 0; tile < n_tiles; ++tile) {
        const int t0 = tile * R;
        const bool last = tile == n_tiles - 1;
        uint4 *acc4 = reinterpret_cast<uint4 *>(acc);
        for (int i = threadIdx.x; i < acc_words4; i += blockDim.x)
            acc4[i] = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
        int cnt = 0;        // this lane's candidate count (a register)
        const int L = p.seg_cl >> 5;
        const bool fast = p.in_range && t0 + R <= p.n_theta;
        if (single) {
            if (fast)
                vote_tile<P, true>(p, acc, stage, nv, t0, my_cl, L, cnt, ws);
            else
                vote_tile<P, false>(p, acc, stage, nv, t0, my_cl, L, cnt, ws);
        } else {
            for (long long s0 = 0; s0 < H; s0 += p.hit_stage) {
                int n = (int)min((long long)p.hit_stage, (long long)H - s0);
                int ns = stage_hits(p, beg + s0, n, stage, wtot, ws);
                vote_tile<P, false>(p, acc, stage, ns, t0, my_cl, L, cnt, ws);
                __syncthreads();
            }
        }
        __syncthreads();

        if (p.export_acc)
            export_tile<P>(p, acc, t0, R, w);

        TileView<P> tv{acc, carry0, carry1, t0, R, p.lw, p.n_theta, p.n_rho};
        const int rlo = max(t0 - 1, 0);
        const int rhi = last ? p.n_theta : t0 + R - 1;
        const int ihi = rhi - t0;
        list_carry<P>(p, tv, rlo, rhi, my_cl, L, cnt);
        // block-wide exclusive prefix of the lanes' counts (list overflow: any
        // count past L sends the tile to the direct test)
        {
            const int c = min(cnt, L);
            int incl = c;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d)
                    incl += y;
            }
            if (lane == 31)
                wc.n_cl[warp] = incl;
            const bool ovf = __syncthreads_or(cnt > L);
            if (warp == 0) {
                const int wt = lane < nw ? wc.n_cl[lane] : 0;
                int wi = wt;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, wi, d);
                    if (lane >= d)
                        wi += y;
                }
                if (lane < nw)
                    wc.pre_cl[lane] = wi - wt;
                if (lane == 31) {
                    ws.n_sel = wi;
                    ws.seg_ovf = ovf ? 1 : 0;
                }
            }
            __syncthreads();
            pre_thr[threadIdx.x] = wc.pre_cl[warp] + incl - c;
            __syncthreads();
        }
        PeakSink ps{keys + p.kp + (size_t)warp * seg_cap, seg_cap, wc.n_pk[warp], 0, ws.kth,
                    ws.vk, vh + warp * kHistBins};
        if (!ws.seg_ovf) {
            // one thread per listed candidate, spread over all warps
            const int total = ws.n_sel;
            for (int x0 = 0; x0 < total; x0 += blockDim.x) {
                const int x = x0 + threadIdx.x;
                bool peak = false;
                int v = 0, i = 0, b = 0;
                if (x < total) {
                    // the thread (warp, lane) whose column holds entry x
                    int u = 0;
#pragma unroll 1
                    for (int step = 512; step > 0; step >>= 1)
                        if (u + step < (int)blockDim.x && pre_thr[u + step] <= x)
                            u += step;
                    const int slot = x - pre_thr[u];
                    const uint32_t e = cl[(size_t)(u >> 5) * p.seg_cl + slot * 32 + (u & 31)];
                    decode_entry<P>(p, tv, e, v, i, b);
                    peak = i < ihi && v >= p.T && tv.is_peak(t0 + i, b, v);
                }
                record_peaks(peak, v, t0 + i, b, ps);
                if (lane == 0)
                    wc.n_pk[warp] = ps.n;
                if (__syncthreads_or(lane == 0 && ps.n > seg_cap - 32)) {
                    merge_peaks(p, keys, top_stage, seg_cap, wc, vh, ws);
                    ps.n = 0;
                    ps.kth = ws.kth;
                    ps.vk = ws.vk;
                }
            }
        } else {
            check_direct<P>(p, tv, rlo, rhi, ps, keys, top_stage, seg_cap, wc, vh, ws);
        }
        if (lane == 0) {
            wc.n_pk[warp] = ps.n;
            wc.n_found[warp] += ps.found;
        }
        // keep room for a full step of appends in every segment
        if (__syncthreads_or(lane == 0 && ps.n > seg_cap - 32))
            merge_peaks(p, keys, top_stage, seg_cap, wc, vh, ws);
        if (!last) {
            for (int b = threadIdx.x; b < p.n_rho; b += blockDim.x) {
                carry0[b] = tile_val<P>(acc, p.n_rho, p.lw, R - 2, b);
                carry1[b] = tile_val<P>(acc, p.n_rho, p.lw, R - 1, b);
            }
        }
        __syncthreads();
    }
    int pending = 0;
    for (int k = 0; k < nw; ++k)
        pending += wc.n_pk[k];
    if (pending > 0)
        merge_peaks(p, keys, top_stage, seg_cap, wc, vh, ws);
}
// Step D: first matching peak in order, then per-peak compaction.  Warp 0
// counts the categories and scatters; no other warp touches the counters.
__device__ void associate(const KParams &p, long long w, long long beg, int H, int n_top,
                          const unsigned long long *keys, int *pk, int *cnt, int *cursor,
                          int *cat_s, bool cat_in_smem)
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
    __syncthreads();
    const int D = p.D, K = p.K;
    const int tol = p.tol;
    // four lanes per hit, each testing every fourth peak; the first match is
    // the smallest matching index over the four
    const int sub = threadIdx.x & 3;
    const int per = blockDim.x >> 2;
    for (int i0 = 0; i0 < H; i0 += per) {
        const int i = i0 + (int)(threadIdx.x >> 2);
        int phi = 0, z = 0;
        const bool in = i < H;
        const bool ok = in && load_hit(p, beg + i, phi, z);
        int first = n_top;
        if (ok) {
            for (int q = sub; q < n_top; q += 4) {
                int d = rho_bin(phi, z, pk_c[q], pk_s[q], D, K) - pk_b[q];
                if (d <= tol && d >= -tol) {
                    first = q;
                    break;
                }
            }
        }
        first = min(first, __shfl_xor_sync(0xffffffffu, first, 1));
        first = min(first, __shfl_xor_sync(0xffffffffu, first, 2));
        if (in && sub == 0) {
            const int cat = ok ? first : n_top + 1;
            p.hit_track[beg + i] = cat < n_top ? cat : (cat == n_top ? -1 : -2);
            if (cat_in_smem)
                cat_s[i] = cat;
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int q = lane; q < n_top + 2; q += 32)
            cnt[q] = 0;
        __syncwarp();
        for (int base = 0; base < H; base += 32) {
            const int i = base + lane;
            int cat = -1;
            if (i < H) {
                if (cat_in_smem) {
                    cat = cat_s[i];
                } else {
                    int v = p.hit_track[beg + i];
                    cat = v >= 0 ? v : (v == -1 ? n_top : n_top + 1);
                }
            }
            const unsigned m = __match_any_sync(0xffffffffu, cat);
            if (i < H && lane == __ffs(m) - 1)
                cnt[cat] += __popc(m);
            __syncwarp();
        }
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
                pr.votes = (int32_t)key_votes(k);
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
            __syncwarp();
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(1024, 1) find_kernel(KParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ WinScalars ws;
    const int nw = blockDim.x >> 5;
    const SmemLayout L = smem_layout(p.word_rows, p.hit_stage, p.n_rho, p.seg_cl * nw, nw);
    uint32_t *acc = reinterpret_cast<uint32_t *>(smem + L.acc);
    int2 *stage = reinterpret_cast<int2 *>(smem + L.stage);
    int *carry = reinterpret_cast<int *>(smem + L.carry);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(smem + L.keys);
    uint32_t *cl = reinterpret_cast<uint32_t *>(smem + L.cl);
    int *pk = reinterpret_cast<int *>(smem + L.pk);
    unsigned long long *top_stage = reinterpret_cast<unsigned long long *>(smem + L.pk);
    int *cnt = reinterpret_cast<int *>(smem + L.cnt);
    int *cursor = cnt + (HOUGH_MAX_PEAKS + 2);
    int *wcnt = reinterpret_cast<int *>(smem + L.hist);
    WarpCounters wc{wcnt, wcnt + 32, wcnt + 64, wcnt + 96, wcnt + 128};
    int *vh = reinterpret_cast<int *>(smem + L.vh);
    int *pre_thr = reinterpret_cast<int *>(smem + L.pre);
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
                ws.n_top = 0;
                ws.seg_ovf = 0;
                ws.vk = 0;
                ws.flags = 0u;
            }
            for (int i = threadIdx.x; i < p.kp; i += blockDim.x)
                keys[i] = kKeyMax;
            if (threadIdx.x < 32) {
                wc.n_pk[threadIdx.x] = 0;
                wc.n_found[threadIdx.x] = 0;
                wc.n_cl[threadIdx.x] = 0;
            }
            for (int i = threadIdx.x; i < nw * kHistBins; i += blockDim.x)
                vh[i] = 0;
            __syncthreads();
            if (H <= 255)
                process_tiles<4>(p, beg, H, acc, stage, carry, keys, cl, top_stage, wc, vh, pre_thr, wtot, ws, w);
            else if (H <= 65535)
                process_tiles<2>(p, beg, H, acc, stage, carry, keys, cl, top_stage, wc, vh, pre_thr, wtot, ws, w);
            else
                process_tiles<1>(p, beg, H, acc, stage, carry, keys, cl, top_stage, wc, vh, pre_thr, wtot, ws, w);
            __syncthreads();
            const int n_top = ws.n_top;
            const bool cat_in_smem = H <= 2 * p.hit_stage;
            associate(p, w, beg, H, n_top, keys, pk, cnt, cursor, reinterpret_cast<int *>(stage),
                      cat_in_smem);
            if (threadIdx.x == 0) {
                int found = 0;
                for (int k = 0; k < nw; ++k)
                    found += wc.n_found[k];
                unsigned fl = ws.flags;
                if (found > p.max_peaks)
                    fl |= HOUGH_WIN_PEAK_OVERFLOW;
                p.status[w] = fl;
                p.n_peaks[w] = n_top;
                if (p.n_found)
                    p.n_found[w] = found;
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
