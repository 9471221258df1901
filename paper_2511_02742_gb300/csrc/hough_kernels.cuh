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
// of word (wr, j) is the count of bin lo + j in tile row s*WR + wr.  P = 4
// (8-bit) when the window has <= 255 hits, P = 2 (16-bit) when <= 65535, else
// P = 1: a count never exceeds the number of hits, so the packed counters are
// exact.  A tile stores only NB bins [lo, lo + NB) of each row: the bin is
// monotone in phi and in z, so the corners of the detector box bound the bins
// that any hit can reach in a row, and the host gives every tile the first
// bin lo of a window of NB bins that holds every reachable bin inside
// [0, n_rho) of its rows (NB about 0.6 n_rho for 128-row tiles over half a
// turn; NB = n_rho, lo = 0 when no table is given).  Bins outside the window
// are zero in that tile.  Words are stored bank-private: word (wr, j) lives at
//     ((wr / 32) * NB + j) * 32 + wr % 32,
// so every word of word row wr sits in shared-memory bank wr % 32.
//
// Voting assigns lane l of a warp to word row 32*g + l and loops the warp over
// hits; each lane adds one vote per packed row.  Lane l only ever touches bank
// l, so a warp's vote atomic is always a single conflict-free wavefront,
// whatever bins the lanes hit (and no two lanes share a word, so no warp
// aggregation is needed).  The vote whose atomic returns T - 1 lists its bin
// as a candidate (every bin that reaches T is listed exactly once); after the
// vote the listed bins are tested for 3x3 local maxima.
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

constexpr int kSegPk = 128;     // peak-key segment per warp; merged when past 96 entries
constexpr int kSegRoom = 32;    // appends one check step can make per warp (1 per lane)
constexpr int kMergeStage = 4 * HOUGH_MAX_PEAKS * 4 / 8;   // merge staging keys (the pk area)
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
    // the FP64 variant (HOUGH_FLAG_FP64): cos/sin of the row centres and the
    // units, for b = floor((phi/u_phi cos + z/u_z sin - rho_min) / drho)
    const double *Cd;
    const double *Sd;
    double u_phi, u_z, rho_min, drho;
    int fp64;
    int in_range;       // every valid hit votes inside [0, n_rho) in every row
    int n_theta, n_rho;
    // narrowed tiles: NB bins stored per row; the first bin of tile k of
    // counter width P at lo_tab[log2(P) * lo_stride + k] (null: lo = 0)
    int n_b;
    const int32_t *lo_tab;
    int lo_stride;
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
    unsigned nb_inv;    // ceil(2^32 / NB): word-column index -> row group
    unsigned nrho_inv;  // ceil(2^32 / n_rho), the same for full-width tiles
    int hit_stage;      // HS
    int kp;             // top-k region (power of two >= max(32, max_peaks))
    int cl_total;       // entries of the list area (the host sized shared memory with it)
    int seg_cl;         // candidate-list entries per warp
    int seg_ovf;        // of which the warp's shared overflow area
};

// Shared-memory carve-up shared by host (size) and device (pointers).
struct SmemLayout {
    size_t acc, stage, carry, keys, cl, pk, cnt, hist, vh, wtot, total;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// n_b: the bins a tile stores per row (NB).
__host__ __device__ inline SmemLayout smem_layout(int word_rows, int hit_stage, int n_b,
                                                   int cl_entries, int n_warps)
{
    SmemLayout L;
    size_t off = 0;
    L.acc = off;
    off = align_up(off + (size_t)word_rows * n_b * 4, 16);
    L.stage = off;
    off = align_up(off + (size_t)hit_stage * 8, 16);
    L.carry = off;
    off = align_up(off + (size_t)2 * n_b * 4, 16);
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
    L.wtot = off;
    off = align_up(off + 32 * 4, 16);
    L.total = off;
    return L;
}

struct WinScalars {
    unsigned long long kth;   // a peak enters a segment only if its key < kth
    int n_top;                // kept peaks in keys[0 .. n_top)
    int n_sel;                // entries gathered for a merge
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
    int *pre_pk;    // exclusive prefix of n_pk (merging)
    int *n_ovf;     // entries the warp's lanes sent to its overflow area in this tile
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
__device__ __forceinline__ int rho_bin(int phi, int z, int c, int s, int D, int K);

// The FP64 variant of the bin: Eq. (1) in double precision with the
// Section 5 binning, each operation rounded to nearest in this order (no
// fused multiply-add), so that it is reproducible: phi_deg = phi / u_phi and
// z_mm = z / u_z once per hit, then per row
// floor(((phi_deg cos + z_mm sin) - rho_min) / drho).
__device__ __forceinline__ int rho_bin64(double phi_deg, double z_mm, double c, double s,
                                         const KParams &p)
{
    const double rho = __dadd_rn(__dmul_rn(phi_deg, c), __dmul_rn(z_mm, s));
    return __double2int_rd(__ddiv_rn(__dsub_rn(rho, p.rho_min), p.drho));
}

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
__device__ inline int stage_hits(const KParams &p, long long base, int n, int2 *stage, int *wtot,
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
// register count (no shared counter, no warp vote).  A lane whose column is
// full (cnt >= L) appends to the warp's overflow area instead (list_append).  FAST: the host proved that every
// valid hit votes in range, and the tile has no row past n_theta, so the
// per-vote checks are left out.
// Per-warp candidate list: L column slots per lane (seg[slot * 32 + lane]),
// then an overflow area of p.seg_ovf entries shared by the warp's lanes
// (seg[L * 32 + j], j from the warp's counter *ovf).  Overflow is rare, so
// its shared counter is seldom contended.
struct ListOvf {
    int *count;   // the warp's overflow counter
    int cap;      // overflow-area entries
};

__device__ __forceinline__ void list_append(uint32_t *seg, int L, int &cnt, const ListOvf &ovf,
                                            uint32_t e)
{
    if (cnt < L) {
        seg[cnt * 32 + (threadIdx.x & 31)] = e;
        ++cnt;
    } else {
        const int j = atomicAdd(ovf.count, 1);
        if (j < ovf.cap)
            seg[L * 32 + j] = e;
    }
}

template <int P, bool FAST, bool F64 = false>
__device__ void vote_tile(const KParams &p, uint32_t *acc, const int2 *stage, int nh, int t0,
                          int lo, uint32_t *seg, int L, int &cnt, const ListOvf &ovf,
                          WinScalars &ws)
{
    constexpr int CW = 32 / P;
    constexpr unsigned MASK = P == 1 ? 0xffffffffu : ((1u << CW) - 1u);
    const int WR = p.word_rows, G = WR >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int g = warp % G;
    const int wr = g * 32 + lane;
    const int hstep = nw / G;
    int c[P], s[P];
    double cd[P], sd[P];
    bool act[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
        int t = t0 + k * WR + wr;
        act[k] = t < p.n_theta;
        if constexpr (F64) {
            cd[k] = act[k] ? __ldg(p.Cd + t) : 0.0;
            sd[k] = act[k] ? __ldg(p.Sd + t) : 0.0;
            c[k] = s[k] = 0;
        } else {
            c[k] = act[k] ? __ldg(p.C + t) : 0;
            s[k] = act[k] ? __ldg(p.S + t) : 0;
            cd[k] = sd[k] = 0.0;
        }
    }
    // bank-private column of this lane: word (wr, j) at col_word0 + 32 j.
    // j = b - lo comes straight from the sum with D - lo 2^K: its exact value
    // lies between 0 and the sum with D for every hit whose bin is >= lo
    // (and lo = 0 when a bin below 0 is reachable), so it fits in int32 too.
    const unsigned col_word0 = (unsigned)(g * p.n_b) * 32u + (unsigned)lane;
    const unsigned col = (unsigned)__cvta_generic_to_shared(acc) + 4u * col_word0;
    const int K = p.K;
    const int D = (int)((unsigned)p.D - ((unsigned)lo << K));
    // a valid hit's vote is inside [0, n_rho) exactly when j is inside [0, NB)
    const unsigned nr = (unsigned)p.n_b;
    const unsigned tm1 = (unsigned)(p.T - 1);
    bool oor = false;
    // Software pipelined: the next hit is loaded before this hit's atomics
    // (which the "memory" clobber keeps in program order), and all P atomics
    // are issued before any returned value is tested.
    int h = warp / G;
    int2 nxt = stage[max(min(h, nh - 1), 0)];
#pragma unroll 4
    for (; h < nh; h += hstep) {
        const int2 hv = nxt;
        nxt = stage[min(h + hstep, nh - 1)];
        int bb[P];
        bool in[P];
        unsigned old[P];
        double phd = 0.0, zmm = 0.0;
        if constexpr (F64) {
            phd = __ddiv_rn((double)hv.x, p.u_phi);
            zmm = __ddiv_rn((double)hv.y, p.u_z);
        }
#pragma unroll
        for (int k = 0; k < P; ++k) {
            if constexpr (F64)
                bb[k] = rho_bin64(phd, zmm, cd[k], sd[k], p) - lo;
            else
                bb[k] = rho_bin(hv.x, hv.y, c[k], s[k], D, K);
            in[k] = true;
            if (!FAST) {
                in[k] = act[k] && (unsigned)bb[k] < nr;
                oor |= act[k] && !in[k];
            }
        }
#pragma unroll
        for (int k = 0; k < P; ++k)
            old[k] = in[k] ? atom_add_shared(col + (unsigned)bb[k] * 128u, 1u << (k * CW)) : 0u;
        if (P == 4) {
            // four fields: one xor-and test per vote, one branch per hit
            unsigned hit = 0u;
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const unsigned mk = MASK << (k * CW), tk = tm1 << (k * CW);
                hit |= (in[k] && ((old[k] ^ tk) & mk) == 0u) ? (1u << k) : 0u;
            }
            if (hit) {
#pragma unroll
                for (int k = 0; k < P; ++k)
                    if (hit & (1u << k))
                        list_append(seg, L, cnt, ovf,
                                    ((col_word0 + (unsigned)bb[k] * 32u) << 2) | (unsigned)k);
            }
        } else {
#pragma unroll
            for (int k = 0; k < P; ++k)
                if (in[k] && ((old[k] >> (k * CW)) & MASK) == tm1)
                    list_append(seg, L, cnt, ovf,
                                ((col_word0 + (unsigned)bb[k] * 32u) << 2) | (unsigned)k);
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

template <int P>
struct TileView {
    const uint32_t *acc;
    const int *carry0;   // row t0 - 2
    const int *carry1;   // row t0 - 1
    int t0, R, lw, n_theta, n_b;
    int lo;              // first stored bin of this tile
    int lo_prev;         // first stored bin of the previous tile (the carried rows)

    // Count of (theta row t, rho bin b), 0 outside the accumulator and
    // outside the stored bins of the row's tile (no vote reaches those).
    // Branch free: the tile word and the carried value are both loaded (with
    // clamped indices) and the right one is selected, so that the eight loads
    // of a neighbourhood test are issued together.
    __device__ __forceinline__ int get(int t, int b) const
    {
        constexpr int CW = 32 / P;
        constexpr unsigned MASK = P == 1 ? 0xffffffffu : ((1u << CW) - 1u);
        const int i = t - t0;
        const int ic = min(max(i, 0), R - 1);
        const int jt = b - lo, jc = b - lo_prev;
        const int jtc = min(max(jt, 0), n_b - 1), jcc = min(max(jc, 0), n_b - 1);
        const int sl = ic >> lw, wr = ic & ((1 << lw) - 1);
        const uint32_t w = acc[((wr >> 5) * n_b + jtc) * 32 + (wr & 31)];
        const int vt = (int)((w >> (sl * CW)) & MASK);
        const int vc = (i == -2 ? carry0 : carry1)[jcc];
        const int v = i >= 0 ? vt : vc;
        const bool inside = (unsigned)t < (unsigned)n_theta && i >= -2 && i < R &&
                            (unsigned)(i >= 0 ? jt : jc) < (unsigned)n_b;
        return inside ? v : 0;
    }

    // Section 4/5 peak rule: > earlier neighbours (row-major), >= later ones.
    __device__ __forceinline__ bool is_peak(int t, int b, int v) const
    {
        const int i = t - t0, j = b - lo;
        if (i >= 1 && i + 1 < R && t + 1 < n_theta && j >= 1 && j + 1 < n_b)
            return is_peak_inside(i, j, v);
        const int jc = b - lo_prev;
        if (t0 > 0 && (i == 0 || i == -1) && t + 1 < n_theta && j >= 1 && j + 1 < n_b &&
            jc >= 1 && jc + 1 < n_b)
            return is_peak_carried(i, j, jc, v);
        const int a0 = get(t - 1, b - 1), a1 = get(t - 1, b), a2 = get(t - 1, b + 1);
        const int a3 = get(t, b - 1), a4 = get(t, b + 1);
        const int a5 = get(t + 1, b - 1), a6 = get(t + 1, b), a7 = get(t + 1, b + 1);
        const int earlier = max(max(a0, a1), max(a2, a3));
        const int later = max(max(a4, a5), max(a6, a7));
        return v > earlier && v >= later;
    }

    // The rule for tile row 0 (i = 0) and the carried row (i = -1) of a tile
    // that has a previous one, when the bin's neighbours lie in the stored
    // bins of both tiles (j in this tile, jc in the previous one): the rows
    // above come from the carried rows, the rest from the tile, with plain
    // loads.
    __device__ __forceinline__ bool is_peak_carried(int i, int j, int jc, int v) const
    {
        constexpr unsigned MASK = P == 1 ? 0xffffffffu : ((1u << (32 / P)) - 1u);
        const int *up = i == 0 ? carry1 : carry0;           // row i - 1
        const int a0 = up[jc - 1], a1 = up[jc], a2 = up[jc + 1];
        int sb, sc;
        const int wb = row_word(0, j, sb);                  // tile row 0
        const int wc = row_word(i + 1, j, sc);              // row i + 1, in the tile
        const int t3 = (int)((acc[wb - 32] >> sb) & MASK), t4 = (int)((acc[wb + 32] >> sb) & MASK);
        const int c3 = carry1[jc - 1], c4 = carry1[jc + 1];
        const int a3 = i == 0 ? t3 : c3, a4 = i == 0 ? t4 : c4;   // row i itself
        const int a5 = (int)((acc[wc - 32] >> sc) & MASK), a6 = (int)((acc[wc] >> sc) & MASK);
        const int a7 = (int)((acc[wc + 32] >> sc) & MASK);
        const int earlier = max(max(a0, a1), max(a2, a3));
        const int later = max(max(a4, a5), max(a6, a7));
        return v > earlier && v >= later;
    }

    // Word index of tile row i at stored bin j, and the shift of its field.
    __device__ __forceinline__ int row_word(int i, int j, int &sh) const
    {
        const int wr = i & ((1 << lw) - 1);
        sh = (i >> lw) * (32 / P);
        return ((wr >> 5) * n_b + j) * 32 + (wr & 31);
    }

    // The same rule for a bin whose eight neighbours all lie in the tile's
    // stored bins: three row bases, then eight plain loads (no clamping or
    // selection).  j is the stored-bin index.
    __device__ __forceinline__ bool is_peak_inside(int i, int j, int v) const
    {
        constexpr unsigned MASK = P == 1 ? 0xffffffffu : ((1u << (32 / P)) - 1u);
        int sa, sb, sc;
        const int wa = row_word(i - 1, j, sa), wb = row_word(i, j, sb), wc = row_word(i + 1, j, sc);
        const int a0 = (int)((acc[wa - 32] >> sa) & MASK), a1 = (int)((acc[wa] >> sa) & MASK);
        const int a2 = (int)((acc[wa + 32] >> sa) & MASK), a3 = (int)((acc[wb - 32] >> sb) & MASK);
        const int a4 = (int)((acc[wb + 32] >> sb) & MASK), a5 = (int)((acc[wc - 32] >> sc) & MASK);
        const int a6 = (int)((acc[wc] >> sc) & MASK), a7 = (int)((acc[wc + 32] >> sc) & MASK);
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
// with this tile) to the lanes' columns as 0x80000000 | b (b the bin, stored
// at carry1[b - lo_prev]); every thread takes every blockDim-th bin.
template <int P>
__device__ void list_carry(const KParams &p, const TileView<P> &tv, int rlo, int rhi,
                           uint32_t *seg, int L, int &cnt, const ListOvf &ovf)
{
    const int tc = tv.t0 - 1;
    if (!(tc >= 0 && tc >= rlo && tc < rhi))
        return;
    for (int j = threadIdx.x; j < p.n_b; j += blockDim.x)
        if (tv.carry1[j] >= p.T)
            list_append(seg, L, cnt, ovf, 0x80000000u | (unsigned)(j + tv.lo_prev));
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

constexpr int kHistBins = 64;
constexpr int kSerialCompact = 512;    // association: one warp compacts windows up to this size   // per-warp peak-vote histogram; last bin = ">= 63"

__device__ __forceinline__ void record_peaks(bool peak, int v, int t, int b, PeakSink &ps)
{
    const unsigned m = __ballot_sync(0xffffffffu, peak);
    if (m == 0u)
        return;
    ps.found += __popc(m);
    // vote counts below the current bound vk can never again decide it (vk
    // only rises), so only peaks with >= vk votes are counted
    if (peak && ps.hist && v >= ps.vk)
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
        v = tv.carry1[b - tv.lo_prev];
    } else {
        const int f = (int)(e >> 2), s = (int)(e & 3u);
        const int qq = f >> 5;                                     // g * NB + j
        const int g = (int)__umulhi((unsigned)qq, p.nb_inv);
        b = qq - g * p.n_b + tv.lo;
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
__device__ inline void merge_peaks(const KParams &p, unsigned long long *keys,
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
    // entry idx of the virtual list: the kept prefix, then the segments
    auto entry = [&](int idx) {
        if (idx < n_top)
            return keys[idx];
        int k = 0;
        while (k + 1 < nw && wc.pre_pk[k + 1] <= idx)
            ++k;
        return segs[(size_t)k * seg_cap + (idx - wc.pre_pk[k])];
    };
    if (m <= kMergeStage) {
        // gather the entries into one array, then rank each against all
        // (keys are distinct: its rank is its place) and write the best
        // `keep` straight into the kept list
        for (int idx = threadIdx.x; idx < m; idx += blockDim.x)
            top_stage[idx] = entry(idx);
        __syncthreads();
        for (int idx = threadIdx.x; idx < m; idx += blockDim.x) {
            const unsigned long long x = top_stage[idx];
            int r0 = 0, r1 = 0, r2 = 0, r3 = 0;
            int y = 0;
            for (; y + 4 <= m; y += 4) {
                r0 += top_stage[y] < x ? 1 : 0;
                r1 += top_stage[y + 1] < x ? 1 : 0;
                r2 += top_stage[y + 2] < x ? 1 : 0;
                r3 += top_stage[y + 3] < x ? 1 : 0;
            }
            for (; y < m; ++y)
                r0 += top_stage[y] < x ? 1 : 0;
            const int rank = r0 + r1 + r2 + r3;
            if (rank < keep)
                keys[rank] = x;
        }
        for (int i = keep + threadIdx.x; i < p.kp; i += blockDim.x)
            keys[i] = kKeyMax;
    } else {
        for (int idx = threadIdx.x; idx < m; idx += blockDim.x) {
            const unsigned long long x = entry(idx);
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
    }
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

// The P counters of four packed words as four int32 (field s of each).
template <int P>
__device__ __forceinline__ int4 fields4(const uint4 &v, int s)
{
    constexpr int CW = 32 / P;
    constexpr unsigned MASK = P == 1 ? 0xffffffffu : ((1u << CW) - 1u);
    return make_int4((int)((v.x >> (s * CW)) & MASK), (int)((v.y >> (s * CW)) & MASK),
                     (int)((v.z >> (s * CW)) & MASK), (int)((v.w >> (s * CW)) & MASK));
}

// Export mode, at the end of a tile (after the check, when the tile is not
// read again): the tile's rows written as int32 to acc[w][t][b], the carried
// rows saved and the tile zeroed, with no barrier.  Each warp takes blocks of
// 32 word rows x 32 stored bins (1024 consecutive words): it holds the block
// in registers (saving its carried words, field P-1 of word rows WR-2 and
// WR-1, when the block is in the last row group), writes it back transposed
// in place -- word row r becomes 32 consecutive words, its 16-byte chunk c
// stored at chunk c ^ (r & 7), so that the 16-byte writes and reads that
// follow take the fewest wavefronts -- then each lane reads four bins of one
// word row and writes each of its P theta rows with one 16-byte store (a warp
// store covers four whole 128-byte lines), and the warp zeroes the block.
// lo is a multiple of 4, so those stores are aligned.  Stored bins past the
// last whole block, tiles with rows past n_theta and accumulators that are
// not 16-byte aligned go out with 4-byte stores; the bins the tile does not
// store are written as zeros.
template <int P>
__device__ void export_tile_end(const KParams &p, uint32_t *acc, int *carry0, int *carry1,
                                bool save, int t0, int R, int lo, long long w)
{
    constexpr int CW = 32 / P;
    constexpr unsigned MASK = P == 1 ? 0xffffffffu : ((1u << CW) - 1u);
    const int WR = p.word_rows, G = WR >> 5, NB = p.n_b;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nblk = NB >> 5;
    int32_t *out = p.acc + (size_t)w * p.n_theta * p.n_rho;
    const bool vec = (reinterpret_cast<uintptr_t>(p.acc) & 15u) == 0u;
    const bool fast = t0 + R <= p.n_theta && vec;
    for (int item = warp; item < G * nblk; item += nw) {
        const int g = item / nblk, j0 = (item - g * nblk) * 32;
        uint32_t *blk = acc + (size_t)(g * NB + j0) * 32;
        uint32_t r[32];
#pragma unroll
        for (int j = 0; j < 32; ++j)
            r[j] = blk[j * 32 + lane];                 // word (g*32 + lane, j0 + j)
        if (save && g == G - 1 && lane >= 30) {
            int *cr = lane == 30 ? carry0 : carry1;
#pragma unroll
            for (int j = 0; j < 32; ++j)
                cr[j0 + j] = field<P>(r[j], P - 1);
        }
        __syncwarp();
#pragma unroll
        for (int c = 0; c < 8; ++c)
            *reinterpret_cast<uint4 *>(blk + lane * 32 + ((c ^ (lane & 7)) << 2)) =
                make_uint4(r[4 * c], r[4 * c + 1], r[4 * c + 2], r[4 * c + 3]);
        __syncwarp();
        if (fast) {
            // lane: word row q + (lane >> 3), bins lo + j0 + 4 (lane & 7) .. + 3
            const int rs = lane >> 3, c = lane & 7;
            int32_t *o = out + (size_t)(t0 + g * 32 + rs) * p.n_rho + lo + j0 + 4 * c;
            const size_t sstep = (size_t)WR * p.n_rho;
#pragma unroll 4
            for (int q = 0; q < 32; q += 4) {
                const int row = q + rs;
                const uint4 v = *reinterpret_cast<const uint4 *>(blk + row * 32 + ((c ^ (row & 7)) << 2));
#pragma unroll
                for (int s = 0; s < P; ++s)
                    *reinterpret_cast<int4 *>(o + (size_t)q * p.n_rho + s * sstep) = fields4<P>(v, s);
            }
        } else {
            for (int q = 0; q < 32; ++q) {
                const uint32_t v = blk[q * 32 + ((((lane >> 2) ^ (q & 7))) << 2) + (lane & 3)];
#pragma unroll
                for (int s = 0; s < P; ++s) {
                    const int i = s * WR + g * 32 + q, t = t0 + i;
                    if (i < R && t < p.n_theta)
                        out[(size_t)t * p.n_rho + lo + j0 + lane] = (int)((v >> (s * CW)) & MASK);
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int c = 0; c < 8; ++c)
            *reinterpret_cast<uint4 *>(blk + lane * 32 + 4 * c) = make_uint4(0u, 0u, 0u, 0u);
    }
    // stored bins past the last whole block: one bin of 32 word rows per warp
    // step, one lane per word row
    const int rb = nblk * 32, nr = NB - rb;
    if (nr > 0) {
        for (int x = warp; x < G * nr; x += nw) {
            const int g = x / nr, j = rb + (x - g * nr);
            const int wr = g * 32 + lane;
            {
                const size_t idx = (size_t)(g * NB + j) * 32 + lane;
                const uint32_t v = acc[idx];
                if (save && g == G - 1 && lane >= 30)
                    (lane == 30 ? carry0 : carry1)[j] = field<P>(v, P - 1);
#pragma unroll
                for (int s = 0; s < P; ++s) {
                    const int i = s * WR + wr, t = t0 + i;
                    if (i < R && t < p.n_theta)
                        out[(size_t)t * p.n_rho + lo + j] = (int)((v >> (s * CW)) & MASK);
                }
                acc[idx] = 0u;
            }
        }
    }
    // the bins the tile does not store, [0, lo) and [lo + NB, n_rho) of every
    // row: zeros, four bins per store (lo, NB and n_rho are multiples of 4)
    const int nq = (p.n_rho - NB) >> 2;
    if (nq > 0) {
        const int nrows = min(R, p.n_theta - t0);
        for (int x = threadIdx.x; x < nrows * nq; x += blockDim.x) {
            const int i = x / nq, k = x - i * nq;
            const int b = 4 * k < lo ? 4 * k : 4 * k + NB;
            int32_t *o = out + (size_t)(t0 + i) * p.n_rho + b;
            if (vec) {
                *reinterpret_cast<int4 *>(o) = make_int4(0, 0, 0, 0);
            } else {
                o[0] = 0;
                o[1] = 0;
                o[2] = 0;
                o[3] = 0;
            }
        }
    }
}

// Direct test of every counter of the evaluable rows, used when a tile holds
// more candidate bins than the lists (an overflow area overflowed).  Warp
// local, like the list test: the work items are the carried row's stored bins
// in groups of 32 (when that row is evaluated with this tile), then every word
// column (g, j) of the tile with one word row per lane (so a warp's loads hit
// 32 different banks); items are dealt to the warps in turn.  A word column
// whose 32 words hold no counter >= T (one SWAR test per word) costs one load
// and one vote; otherwise its P fields are tested one step each.  A warp
// stops while its peak segment lacks room for 32 more keys; the block barrier
// that ends the round merges the segments and the warps go on.  Every warp
// leaves through the same barrier.
template <int P>
__device__ void check_direct(const KParams &p, const TileView<P> &tv, int rlo, int rhi,
                             PeakSink &ps, unsigned long long *keys, unsigned long long *top_stage,
                             WarpCounters wc, const int *vh, WinScalars &ws)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int ilo = max(rlo - tv.t0, -1), ihi = min(rhi - tv.t0, tv.R);
    const int G = p.word_rows >> 5;
    const ScanTest k = make_test<P>(p.T);
    const int n_carry = ilo < 0 ? (p.n_b + 31) >> 5 : 0;
    const int n_items = n_carry + G * p.n_b;
    int x = warp, s0 = 0;     // this warp's next item and, in a word column, its next field
    for (;;) {
        while (x < n_items && ps.n <= kSegPk - kSegRoom) {
            if (x < n_carry) {
                const int j = x * 32 + lane;
                const int v = j < p.n_b ? tv.carry1[j] : 0;
                const int b = tv.lo_prev + j;
                const bool peak = v >= p.T && tv.is_peak(tv.t0 - 1, b, v);
                record_peaks(peak, v, tv.t0 - 1, b, ps);
                x += nw;
                continue;
            }
            const int q = x - n_carry;                          // g * NB + j
            const int g = (int)__umulhi((unsigned)q, p.nb_inv);
            const int j = q - g * p.n_b;
            const uint32_t wv = tv.acc[q * 32 + lane];
            if (s0 == 0 && __ballot_sync(0xffffffffu, word_has<P>(wv, k)) == 0u) {
                x += nw;
                continue;
            }
            const int i = s0 * p.word_rows + g * 32 + lane;
            const int v = field<P>(wv, s0);
            const int b = tv.lo + j;
            const bool peak = i < ihi && v >= p.T && tv.is_peak(tv.t0 + i, b, v);
            record_peaks(peak, v, tv.t0 + i, b, ps);
            if (++s0 == P) {
                s0 = 0;
                x += nw;
            }
        }
        if (lane == 0)
            wc.n_pk[warp] = ps.n;
        if (!__syncthreads_or(lane == 0 && x < n_items))
            break;
        merge_peaks(p, keys, top_stage, kSegPk, wc, vh, ws);
        ps.n = 0;
        ps.kth = ws.kth;
        ps.vk = ws.vk;
    }
}

// End of a tile: zero the tile after its last read and, when another tile
// follows, first save its last two rows (tile rows R-2 and R-1, field P-1 of
// word rows WR-2 and WR-1, i.e. words 30 and 31 of the 16-byte chunk
// ((G-1) NB + j) * 8 + 7) as the carried rows of the next tile (stored bin j
// of this tile at carry[j]).  The thread that saves a chunk's words is the
// one that zeroes the chunk, so no barrier separates the two.
template <int P>
__device__ void tile_end(const KParams &p, uint32_t *acc, int *carry0, int *carry1, bool save)
{
    const int G = p.word_rows >> 5;
    const int n4 = (p.word_rows * p.n_b) >> 2;
    const int c0 = 8 * (G - 1) * p.n_b;
    uint4 *acc4 = reinterpret_cast<uint4 *>(acc);
    for (int i = threadIdx.x; i < n4; i += blockDim.x) {
        if (save && i >= c0 && (i & 7) == 7) {
            const uint4 q = acc4[i];
            const int b = (i - c0) >> 3;
            carry0[b] = field<P>(q.z, P - 1);
            carry1[b] = field<P>(q.w, P - 1);
        }
        acc4[i] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// The 3x3 test of a warp's listed candidates (all lanes call).  The warp's
// entries are its lanes' column entries, level-major (entry j of every lane
// holding more than j, in lane order), then its overflow entries.  The column
// entries are first compacted in place (an entry only moves down, never over
// an unread one), so that every step gives each lane one entry: within a
// level the entries come from different lanes, whose word rows -- and so
// whose tile banks -- differ.  A step runs only while the warp's peak segment
// has room for 32 more keys; a warp that stops early asks for a merge at the
// block barrier that ends the round, and continues after it.  Returns when
// every warp is done (all warps leave through the same barrier).
template <int P>
__device__ void check_lists(const KParams &p, const TileView<P> &tv, int ihi, uint32_t *my_cl,
                            int L, int cnt, int n_ovf, PeakSink &ps, unsigned long long *keys,
                            unsigned long long *top_stage, WarpCounters wc, const int *vh,
                            WinScalars &ws)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const int cmax = __reduce_max_sync(0xffffffffu, cnt);
    int n_cmp = 0;
    for (int j = 0; j < cmax; ++j) {
        const bool has = j < cnt;
        const unsigned m = __ballot_sync(0xffffffffu, has);
        const uint32_t e = has ? my_cl[j * 32 + lane] : 0u;
        __syncwarp();
        if (has)
            my_cl[n_cmp + __popc(m & lt)] = e;
        n_cmp += __popc(m);
    }
    __syncwarp();
    const int n_ovf_w = min(n_ovf, p.seg_ovf);
    const int n_all = n_cmp + n_ovf_w;
    int y0 = 0;
    for (;;) {
        while (y0 < n_all && ps.n <= kSegPk - kSegRoom) {
            const int y = y0 + lane;
            bool peak = false;
            int v = 0, i = 0, b = 0;
            if (y < n_all) {
                const uint32_t e = my_cl[y < n_cmp ? y : L * 32 + (y - n_cmp)];
                decode_entry<P>(p, tv, e, v, i, b);
                peak = i < ihi && v >= p.T && tv.is_peak(tv.t0 + i, b, v);
            }
            record_peaks(peak, v, tv.t0 + i, b, ps);
            y0 += 32;
        }
        if (lane == 0)
            wc.n_pk[warp] = ps.n;
        if (!__syncthreads_or(lane == 0 && y0 < n_all))
            break;
        merge_peaks(p, keys, top_stage, kSegPk, wc, vh, ws);
        ps.n = 0;
        ps.kth = ws.kth;
        ps.vk = ws.vk;
    }
}

// Returns the number of valid hits left in `stage` (in their original order),
// or -1 when the window was streamed through the stage in parts.  On entry
// the tile is all zero (the kernel zeroes it before its first window, and
// every tile zeroes it again when done); so it is on return.  Per tile the
// CTA passes three block barriers in the common case: after the votes, at
// the end of the candidate check, and after the tile is saved and zeroed.
template <int P, bool F64>
__device__ int process_tiles(const KParams &p, long long beg, int H, uint32_t *acc, int2 *stage,
                              int *carry, unsigned long long *keys, uint32_t *cl,
                              unsigned long long *top_stage, WarpCounters wc, int *vh,
                              int *wtot, WinScalars &ws, long long w)
{
    const int WR = p.word_rows;
    const int R = WR * P;
    const int n_tiles = (p.n_theta + R - 1) / R;
    const bool single = H <= p.hit_stage;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int seg_cap = kSegPk;
    int *carry0 = carry, *carry1 = carry + p.n_b;
    constexpr int lgP = P == 4 ? 2 : (P == 2 ? 1 : 0);
    const int32_t *lo_row = p.lo_tab ? p.lo_tab + lgP * p.lo_stride : nullptr;
    int lo_prev = 0;
    uint32_t *my_cl = cl + (size_t)warp * p.seg_cl;
    const int L = (p.seg_cl - p.seg_ovf) >> 5;      // column slots per lane
    const ListOvf ovf{wc.n_ovf + warp, p.seg_ovf};

    int nv = 0;
    if (single)
        nv = stage_hits(p, beg, H, stage, wtot, ws);

    for (int tile = 0; tile < n_tiles; ++tile) {
        const int t0 = tile * R;
        const bool last = tile == n_tiles - 1;
        int cnt = 0;        // this lane's column entries (a register)
        const bool fast = !F64 && p.in_range && t0 + R <= p.n_theta;
        const int lo = lo_row ? __ldg(lo_row + tile) : 0;
        TileView<P> tv{acc, carry0, carry1, t0, R, p.lw, p.n_theta, p.n_b, lo, lo_prev};
        const int rlo = max(t0 - 1, 0);
        const int rhi = last ? p.n_theta : t0 + R - 1;
        const int ihi = rhi - t0;
        if (single) {
            if (fast)
                vote_tile<P, !F64, F64>(p, acc, stage, nv, t0, lo, my_cl, L, cnt, ovf, ws);
            else
                vote_tile<P, false, F64>(p, acc, stage, nv, t0, lo, my_cl, L, cnt, ovf, ws);
        } else {
            for (long long s0 = 0; s0 < H; s0 += p.hit_stage) {
                int n = (int)min((long long)p.hit_stage, (long long)H - s0);
                int ns = stage_hits(p, beg + s0, n, stage, wtot, ws);
                vote_tile<P, false, F64>(p, acc, stage, ns, t0, lo, my_cl, L, cnt, ovf, ws);
                __syncthreads();
            }
        }
        // the carried row's candidates (it is complete since the previous
        // tile) join the lists before the barrier that ends the vote
        list_carry<P>(p, tv, rlo, rhi, my_cl, L, cnt, ovf);
        __syncwarp();
        // barrier: the votes are complete.  An overflow area that overflowed
        // sends the tile to the direct test of every counter.
        const bool lost = __syncthreads_or(lane == 0 && *ovf.count > p.seg_ovf);
        PeakSink ps{keys + p.kp + (size_t)warp * seg_cap, seg_cap, wc.n_pk[warp], 0, ws.kth,
                    ws.vk, vh + warp * kHistBins};
        if (!lost)
            check_lists<P>(p, tv, ihi, my_cl, L, cnt, *ovf.count, ps, keys, top_stage, wc, vh, ws);
        else
            check_direct<P>(p, tv, rlo, rhi, ps, keys, top_stage, wc, vh, ws);
        if (lane == 0) {
            wc.n_pk[warp] = ps.n;
            wc.n_found[warp] += ps.found;
        }
        // every check step ended in a barrier, so neither the tile nor the
        // carried rows are read any more
        if (p.export_acc)
            export_tile_end<P>(p, acc, carry0, carry1, !last, t0, R, lo, w);
        else
            tile_end<P>(p, acc, carry0, carry1, !last);
        lo_prev = lo;
        if (threadIdx.x < 32)
            wc.n_ovf[threadIdx.x] = 0;
        __syncthreads();
    }
    int pending = 0;
    for (int k = 0; k < nw; ++k)
        pending += wc.n_pk[k];
    if (pending > 0)
        merge_peaks(p, keys, top_stage, seg_cap, wc, vh, ws);
    return single ? nv : -1;
}
// Step D: first matching peak in order, then the stable per-peak compaction.
// Categories: peak index q < n_top, n_top for a hit on no peak's line,
// n_top + 1 for a hit outside the detector box.  hits_s: the window's hits
// in shared memory when every one of them is valid (else NULL: read from
// global memory); cat_s: room for H categories in shared memory (else NULL:
// re-read from hit_track).  Each warp compacts its own contiguous slice of
// the hits: it counts its categories (wcat, one row per warp), a prefix over
// categories and then over warps gives every (warp, category) its first
// slot, and the warp scatters its slice in order.
template <bool F64>
__device__ void associate(const KParams &p, long long w, long long beg, int H, int n_top,
                          const unsigned long long *keys, int *pk, const int2 *hits_s,
                          int *cat_s, int *wcat, int *cat_base)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
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
    const int NC = n_top + 2;
    const bool serial = cat_s && H <= kSerialCompact;
    if (!serial)
        for (int q = threadIdx.x; q < nw * NC; q += blockDim.x)
            wcat[q] = 0;
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
        bool ok = false;
        if (in) {
            if (hits_s) {
                const int2 h = hits_s[i];
                phi = h.x;
                z = h.y;
                ok = true;
            } else {
                ok = load_hit(p, beg + i, phi, z);
            }
        }
        int first = n_top;
        if (ok) {
            double phd = 0.0, zmm = 0.0;
            if constexpr (F64) {
                phd = __ddiv_rn((double)phi, p.u_phi);
                zmm = __ddiv_rn((double)z, p.u_z);
            }
            for (int q = sub; q < n_top; q += 4) {
                int d;
                if constexpr (F64)
                    d = rho_bin64(phd, zmm, __ldg(p.Cd + pk_t[q]), __ldg(p.Sd + pk_t[q]), p) -
                        pk_b[q];
                else
                    d = rho_bin(phi, z, pk_c[q], pk_s[q], D, K) - pk_b[q];
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
            if (cat_s)
                cat_s[i] = cat;
        }
    }
    __syncthreads();
    if (cat_s && H <= kSerialCompact) {
        // one warp counts, places and scatters (categories in cat_s): no
        // per-warp table, three block barriers in all
        int *ccnt = cat_base, *cbase = cat_base + (HOUGH_MAX_PEAKS + 2);
        if (warp == 0) {
            const unsigned lt = lanemask_lt();
            for (int q = lane; q < NC; q += 32)
                ccnt[q] = 0;
            __syncwarp();
            for (int b0 = 0; b0 < H; b0 += 32) {
                const int i = b0 + lane;
                const int cat = i < H ? cat_s[i] : -1;
                const unsigned m = __match_any_sync(0xffffffffu, cat);
                if (i < H && lane == __ffs(m) - 1)
                    ccnt[cat] += __popc(m);
                __syncwarp();
            }
            int run = 0;
            for (int b0 = 0; b0 < NC; b0 += 32) {
                const int q = b0 + lane;
                const int tot = q < NC ? ccnt[q] : 0;
                int incl = tot;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, d);
                    if (lane >= d)
                        incl += y;
                }
                const int excl = run + incl - tot;
                if (q < NC)
                    cbase[q] = excl;
                if (q < n_top) {
                    const unsigned long long k = keys[q];
                    hough_peak pr;
                    pr.theta = (uint16_t)((k >> 16) & 0xffffu);
                    pr.rho = (uint16_t)(k & 0xffffu);
                    pr.votes = (int32_t)key_votes(k);
                    pr.n_hits = tot;
                    pr.hit_begin = excl;
                    p.peaks[(size_t)w * p.max_peaks + q] = pr;
                }
                run += __shfl_sync(0xffffffffu, incl, 31);
            }
            __syncwarp();
            for (int b0 = 0; b0 < H; b0 += 32) {
                const int i = b0 + lane;
                const int cat = i < H ? cat_s[i] : -1;
                const unsigned m = __match_any_sync(0xffffffffu, cat);
                const int leader = __ffs(m) - 1;
                int pos = 0;
                if (i < H && lane == leader) {
                    pos = cbase[cat];
                    cbase[cat] = pos + __popc(m);
                }
                pos = __shfl_sync(0xffffffffu, pos, leader);
                if (i < H)
                    p.track_hits[beg + pos + __popc(m & lt)] = i;
                __syncwarp();
            }
        }
        __syncthreads();
        return;
    }
    auto category = [&](int i) {
        if (cat_s)
            return cat_s[i];
        const int v = p.hit_track[beg + i];
        return v >= 0 ? v : (v == -1 ? n_top : n_top + 1);
    };
    const int chunk = (H + nw - 1) / nw;
    const int h0 = min(H, warp * chunk), h1 = min(H, h0 + chunk);
    int *mine = wcat + warp * NC;
    for (int base = h0; base < h1; base += 32) {
        const int i = base + lane;
        const int cat = i < h1 ? category(i) : -1;
        const unsigned m = __match_any_sync(0xffffffffu, cat);
        if (i < h1 && lane == __ffs(m) - 1)
            mine[cat] += __popc(m);          // leaders of distinct categories
        __syncwarp();
    }
    __syncthreads();
    if (warp == 0) {
        int run = 0;
        for (int b0 = 0; b0 < NC; b0 += 32) {
            const int q = b0 + lane;
            int tot = 0;
            if (q < NC)
                for (int k = 0; k < nw; ++k)
                    tot += wcat[k * NC + q];
            int incl = tot;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d)
                    incl += y;
            }
            const int excl = run + incl - tot;
            if (q < NC)
                cat_base[q] = excl;
            if (q < n_top) {
                const unsigned long long k = keys[q];
                hough_peak pr;
                pr.theta = (uint16_t)((k >> 16) & 0xffffu);
                pr.rho = (uint16_t)(k & 0xffffu);
                pr.votes = (int32_t)key_votes(k);
                pr.n_hits = tot;
                pr.hit_begin = excl;
                p.peaks[(size_t)w * p.max_peaks + q] = pr;
            }
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < NC; q += blockDim.x) {
        int run = cat_base[q];
        for (int k = 0; k < nw; ++k) {
            const int c = wcat[k * NC + q];
            wcat[k * NC + q] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int base = h0; base < h1; base += 32) {
        const int i = base + lane;
        const bool in = i < h1;
        const int cat = in ? category(i) : -1;
        const unsigned m = __match_any_sync(0xffffffffu, cat);
        const int leader = __ffs(m) - 1;
        const int rank = __popc(m & lanemask_lt());
        int pos = 0;
        if (in && lane == leader) {
            pos = mine[cat];
            mine[cat] = pos + __popc(m);
        }
        pos = __shfl_sync(0xffffffffu, pos, leader);
        if (in)
            p.track_hits[beg + pos + rank] = i;
        __syncwarp();
    }
    __syncthreads();
}

// The body of the find kernels.  F64: the FP64 variant of the bins
// (HOUGH_FLAG_FP64), a kernel of its own so that its registers do not weigh
// on the fixed-point kernel.
template <bool F64>
__device__ __forceinline__ void find_body(const KParams &p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ WinScalars ws;
    const int nw = blockDim.x >> 5;
    const SmemLayout L = smem_layout(p.word_rows, p.hit_stage, p.n_b, p.cl_total, nw);
    uint32_t *acc = reinterpret_cast<uint32_t *>(smem + L.acc);
    int2 *stage = reinterpret_cast<int2 *>(smem + L.stage);
    int *carry = reinterpret_cast<int *>(smem + L.carry);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(smem + L.keys);
    uint32_t *cl = reinterpret_cast<uint32_t *>(smem + L.cl);
    int *pk = reinterpret_cast<int *>(smem + L.pk);
    unsigned long long *top_stage = reinterpret_cast<unsigned long long *>(smem + L.pk);
    int *cnt = reinterpret_cast<int *>(smem + L.cnt);
    int *wcnt = reinterpret_cast<int *>(smem + L.hist);
    WarpCounters wc{wcnt, wcnt + 32, wcnt + 64, wcnt + 96, wcnt + 128};
    int *vh = reinterpret_cast<int *>(smem + L.vh);
    int *wtot = reinterpret_cast<int *>(smem + L.wtot);

    // the tile starts all zero; every tile and the association leave it so
    {
        uint4 *acc4 = reinterpret_cast<uint4 *>(acc);
        for (int i = threadIdx.x; i < (p.word_rows * p.n_b) >> 2; i += blockDim.x)
            acc4[i] = make_uint4(0u, 0u, 0u, 0u);
    }
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
                ws.vk = 0;
                ws.flags = 0u;
            }
            for (int i = threadIdx.x; i < p.kp; i += blockDim.x)
                keys[i] = kKeyMax;
            if (threadIdx.x < 32) {
                wc.n_pk[threadIdx.x] = 0;
                wc.n_found[threadIdx.x] = 0;
                wc.n_cl[threadIdx.x] = 0;
                wc.n_ovf[threadIdx.x] = 0;
            }
            for (int i = threadIdx.x; i < nw * kHistBins; i += blockDim.x)
                vh[i] = 0;
            __syncthreads();
            int nv;
            if constexpr (F64) {
                if (H <= 255)
                    nv = process_tiles<4, true>(p, beg, H, acc, stage, carry, keys, cl, top_stage, wc, vh, wtot, ws, w);
                else if (H <= 65535)
                    nv = process_tiles<2, true>(p, beg, H, acc, stage, carry, keys, cl, top_stage, wc, vh, wtot, ws, w);
                else
                    nv = process_tiles<1, true>(p, beg, H, acc, stage, carry, keys, cl, top_stage, wc, vh, wtot, ws, w);
            } else {
                if (H <= 255)
                    nv = process_tiles<4, false>(p, beg, H, acc, stage, carry, keys, cl, top_stage, wc, vh, wtot, ws, w);
                else if (H <= 65535)
                    nv = process_tiles<2, false>(p, beg, H, acc, stage, carry, keys, cl, top_stage, wc, vh, wtot, ws, w);
                else
                    nv = process_tiles<1, false>(p, beg, H, acc, stage, carry, keys, cl, top_stage, wc, vh, wtot, ws, w);
            }
            __syncthreads();
            const int n_top = ws.n_top;
            // the tile and the list area are free now: the per-warp category
            // counts go to the tile (else to the list area; the host made
            // sure one of them is large enough), the categories to the list
            // area when they fit
            int *wcat, *cat_s;
            const int need = nw * (n_top + 2);
            if (need <= p.word_rows * p.n_b) {
                wcat = reinterpret_cast<int *>(acc);
                cat_s = H <= p.cl_total ? reinterpret_cast<int *>(cl) : nullptr;
            } else {
                wcat = reinterpret_cast<int *>(cl);
                cat_s = H + need <= p.cl_total ? reinterpret_cast<int *>(cl) + need : nullptr;
            }
            if constexpr (F64)
                associate<true>(p, w, beg, H, n_top, keys, pk, nv == H ? stage : nullptr, cat_s, wcat, cnt);
            else
                associate<false>(p, w, beg, H, n_top, keys, pk, nv == H ? stage : nullptr, cat_s, wcat, cnt);
            // the category counts used the tile: leave it zero for the next window
            if (wcat == reinterpret_cast<int *>(acc) && !(cat_s && H <= kSerialCompact))
                for (int i = threadIdx.x; i < need; i += blockDim.x)
                    wcat[i] = 0;
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

// The find kernels (instances of find_body), compiled in translation units of
// their own so that they build in parallel: find_kernel (fixed point, any CTA
// size up to 1024 threads) and find_kernel_256 (fixed point, CTAs of at most
// 256 threads) in hough_find.cu, find_kernel_fp64 (HOUGH_FLAG_FP64) in
// hough_find_fp64.cu.
__global__ void find_kernel(KParams p);
__global__ void find_kernel_256(KParams p);
__global__ void find_kernel_fp64(KParams p);

}  // namespace hk
