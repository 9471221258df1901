// hough_api.cu -- host side of the C ABI declared in include/hough.h.
//
// The context owns: the fixed-point tables on the device, one scheduling
// counter pair per stream it has launched on (the persistent kernel resets
// its own pair when it ends, so no memset is needed between launches), the
// device staging buffers of hough_find_host, and the chosen launch shape.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "hough.h"
#include "hough_internal.h"
#include "hough_kernels.cuh"
#include "hough_coarse_fine.cuh"
#include "hough_iterative.cuh"
#include "hough_extend.cuh"
#include "hough_slice.cuh"
#include "hough_accumulate.cuh"
#include "hough_encode.cuh"

// The lowest and highest bin that a hit of the detector box can vote in row
// t: the bin is monotone in phi and in z, so the box's four corners bound it
// (phi in [0, 360 deg), z in [z_min, z_min + n_z_strips * pitch], the box the
// find kernel keeps hits in).
static void row_reach(const hough_geometry *g, const int32_t *C, const int32_t *S, long long D,
                      int K, int t, long long &lo, long long &hi)
{
    const long long phis[2] = {0, 360LL * g->phi_u_per_deg - 1};
    const long long zs[2] = {g->z_min_u, (long long)g->z_min_u + (long long)g->n_z_strips * g->z_pitch_u};
    lo = LLONG_MAX;
    hi = LLONG_MIN;
    for (long long ph : phis)
        for (long long z : zs) {
            const long long v = ph * C[t] + z * S[t] + D;
            const long long b = v >= 0 ? (v >> K) : -((-v + (1LL << K) - 1) >> K);
            lo = std::min(lo, b);
            hi = std::max(hi, b);
        }
}

// Whether every valid hit votes inside [0, n_rho) in every row.
static bool box_votes_in_range(const hough_geometry *g, int n_theta, int n_rho, const int32_t *C,
                               const int32_t *S, long long D, int K)
{
    for (int t = 0; t < n_theta; ++t) {
        long long lo, hi;
        row_reach(g, C, S, D, K, t, lo, hi);
        if (lo < 0 || hi >= n_rho)
            return false;
    }
    return true;
}

// Narrowed find tiles.  With WR word rows and P counters per word a tile
// covers rows [k R, (k + 1) R), R = WR P.  Per WR, NB is the widest range of
// reachable bins inside [0, n_rho) over every tile of every P, plus 3,
// rounded up to a multiple of 4 (at most n_rho), and tile k starts at
// lo = min(max(lowest reachable bin, 0), n_rho - NB) rounded down to a
// multiple of 4 (so that the export's 16-byte stores stay aligned; the 3
// spare bins cover the rounding): [lo, lo + NB) then holds every reachable
// bin of the tile's rows that lies in [0, n_rho), and lies in [0, n_rho)
// itself, so a vote is inside [0, n_rho) exactly when it is inside the
// stored bins.  When a bin below 0 is reachable, lo is 0.
// nb[WR index]; lo_all: [WR index][log2 P][tile], tiles ceil(n_theta / 32)
// apart.
static void narrow_tiles(const hough_geometry *g, int nt, int nr, const int32_t *C,
                         const int32_t *S, long long D, int K, int nb_out[3],
                         std::vector<int32_t> &lo_all)
{
    std::vector<long long> rlo(nt), rhi(nt);
    for (int t = 0; t < nt; ++t)
        row_reach(g, C, S, D, K, t, rlo[t], rhi[t]);
    const int stride = (nt + 31) / 32;
    lo_all.assign((size_t)9 * stride, 0);
    for (int wi = 0; wi < 3; ++wi) {
        const int WR = 32 << wi;
        std::vector<long long> tlo((size_t)3 * stride), thi((size_t)3 * stride);
        long long nb = 4;
        for (int lp = 0; lp < 3; ++lp) {
            const int R = WR << lp;
            for (int k = 0; k * R < nt; ++k) {
                long long lo = LLONG_MAX, hi = LLONG_MIN;
                for (int t = k * R; t < std::min(nt, (k + 1) * R); ++t) {
                    lo = std::min(lo, rlo[t]);
                    hi = std::max(hi, rhi[t]);
                }
                tlo[(size_t)lp * stride + k] = lo;
                const long long a = std::max(lo, 0LL), b = std::min(hi, (long long)nr - 1);
                if (b >= a)
                    nb = std::max(nb, b - a + 1);
            }
        }
        nb = std::min<long long>((nb + 3 + 3) & ~3LL, nr);
        nb_out[wi] = (int)nb;
        for (int lp = 0; lp < 3; ++lp)
            for (int k = 0; k * (WR << lp) < nt; ++k)
                lo_all[(size_t)(wi * 3 + lp) * stride + k] = (int32_t)(std::min(
                    std::max(tlo[(size_t)lp * stride + k], 0LL), (long long)nr - nb) & ~3LL);
    }
}

// Bins a find tile stores per row for this word-row count.
static int tile_bins(const hough_ctx *ctx, int word_rows)
{
    const int wi = word_rows == 32 ? 0 : (word_rows == 64 ? 1 : 2);
    return ctx->tile_nb[wi] > 0 ? ctx->tile_nb[wi] : ctx->n_rho;
}

// SM count and shared-memory limits of device dev.
static int device_limits(hough_ctx *ctx, int dev)
{
    int smem_optin = 0, smem_sm = 0;
    if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
            cudaSuccess)
        return HOUGH_ERR_CUDA;
    // the kernel's static shared scalars share the per-block limit
    ctx->smem_optin = (size_t)smem_optin - 128;
    ctx->smem_per_sm = (size_t)smem_sm;
    return HOUGH_OK;
}

struct hough_plan {
    hough_ctx *ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned int *counter = nullptr;
};

namespace {

// Static shared memory of the find kernel (its per-window scalars), rounded
// up; checked against the compiled kernel in prepare_find.
constexpr size_t kStaticSmemReserve = 256;

// Raise a kernel's dynamic shared-memory limit on the current device to at
// least `bytes`.  The limit belongs to the kernel, not to a context, so it is
// only ever raised, under a lock: lowering it could fail a launch that
// another context or host thread is making with more.  The limits set so far
// are kept in a fixed table (no heap allocation: the allocation-free entry
// point comes through here too).
int raise_smem_limit(const void *func, size_t bytes)
{
    struct Entry {
        int dev;
        const void *func;
        size_t bytes;
    };
    static std::mutex mu;
    static Entry table[256];
    static int n_used = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return HOUGH_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(mu);
    Entry *e = nullptr;
    for (int i = 0; i < n_used && !e; ++i)
        if (table[i].dev == dev && table[i].func == func)
            e = &table[i];
    if (e && bytes <= e->bytes)
        return HOUGH_OK;
    if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess) {
        cudaGetLastError();
        return HOUGH_ERR_CUDA;
    }
    if (!e && n_used < 256)
        e = &table[n_used++];
    if (e)
        *e = Entry{dev, func, bytes};
    return HOUGH_OK;
}

int fail(hough_ctx *ctx, int code)
{
    if (ctx && code != HOUGH_OK)
        ctx->last_error = code;
    return code;
}

long long round_half_away(double x)
{
    return x >= 0.0 ? (long long)std::floor(x + 0.5) : -(long long)std::floor(-x + 0.5);
}

bool geometry_ok(const hough_geometry *g)
{
    return g && g->n_vanes > 0 && g->n_z_strips > 0 && g->z_pitch_u > 0 && g->phi_u_per_deg > 0 &&
           g->z_u_per_mm > 0 && std::isfinite(g->rho_min) && std::isfinite(g->rho_max) &&
           g->rho_max > g->rho_min && (360LL * g->phi_u_per_deg) % g->n_vanes == 0;
}

int next_pow2(int x)
{
    int n = 1;
    while (n < x)
        n <<= 1;
    return n;
}

// Candidate-list entries: whatever shared memory the tile leaves, up to what
// lists holding every counter of the tile and of the carried row need.
// Returns -1 when fewer than max(1024, threads + 64 per warp) would fit: a
// list that overflows only sends its tile to the direct test, but every
// warp needs at least two column slots per lane and the check needs one
// gathered entry per thread.
int cl_entries_for(const hough_ctx *ctx, int word_rows, int hit_stage, int ctas, int threads)
{
    const int nw = threads / 32;
    // per CTA the SM also reserves 1 KB and holds the kernel's static shared
    // variables (kStaticSmemReserve covers them): `ctas` CTAs must fit
    const size_t budget = std::min(ctx->smem_optin,
                                   ctx->smem_per_sm / (size_t)ctas - 1024 - kStaticSmemReserve);
    const int nb = tile_bins(ctx, word_rows);
    hk::SmemLayout L0 = hk::smem_layout(word_rows, hit_stage, nb, 0, nw);
    long long room = L0.total < budget ? (long long)((budget - L0.total) / 4) : 0;
    // lists able to hold every counter of the tile and of the carried row in
    // their columns, plus the gathered-entry sixth
    const long long need = std::max<long long>(1024, threads + 64LL * nw);
    const long long worst = (4LL * word_rows * nb + nb) * 12 / 5 + threads;
    long long n = std::min(room, std::max(worst, need));
    n -= n % (4 * nw);
    if (n < need)
        return -1;
    return (int)n;
}

// Fill in defaults and check a launch shape against the device limits.
int resolve_launch(const hough_ctx *ctx, const hough_launch &in, hough_launch &out, size_t &smem)
{
    hough_launch l = in;
    // Fully default: the first of these that fits, all with 32-word-row
    // tiles: three CTAs of 256 threads per SM, two of 512 (several CTAs per
    // SM overlap one CTA's barriers with the others' votes, and small CTAs
    // wait less at each barrier), one of 1024; else one CTA of 512 threads
    // with the largest tile.
    if (l.threads == 0 && l.word_rows == 0 && l.hit_stage == 0 && l.ctas_per_sm == 0) {
        for (const hough_launch &c : {hough_launch{256, 32, 512, 3}, hough_launch{512, 32, 1024, 2},
                                      hough_launch{1024, 32, 2048, 1}})
            if (resolve_launch(ctx, c, out, smem) == HOUGH_OK)
                return HOUGH_OK;
    }
    if (l.threads == 0)
        l.threads = 512;
    if (l.hit_stage == 0)
        l.hit_stage = 2048;
    if (l.ctas_per_sm == 0)
        l.ctas_per_sm = 1;
    if (l.word_rows == 0) {
        // the largest tile that fits, as long as 16-bit tiles do not pass n_theta
        l.word_rows = 32;
        for (int wr : {128, 64}) {
            hk::SmemLayout L = hk::smem_layout(wr, l.hit_stage, tile_bins(ctx, wr), 4096,
                                               l.threads / 32);
            if ((L.total + 1024 + kStaticSmemReserve) * (size_t)l.ctas_per_sm <= ctx->smem_per_sm &&
                L.total <= ctx->smem_optin &&
                ctx->n_theta >= 2 * wr) {
                l.word_rows = wr;
                break;
            }
        }
    }
    if (!(l.threads == 256 || l.threads == 512 || l.threads == 1024))
        return HOUGH_ERR_INVALID_ARG;
    if (!(l.word_rows == 32 || l.word_rows == 64 || l.word_rows == 128))
        return HOUGH_ERR_INVALID_ARG;
    if (l.hit_stage < 256 || l.hit_stage % 256 != 0 || l.hit_stage > 16384)
        return HOUGH_ERR_INVALID_ARG;
    if (l.ctas_per_sm < 1 || l.ctas_per_sm > 4)
        return HOUGH_ERR_INVALID_ARG;
    const int cl = cl_entries_for(ctx, l.word_rows, l.hit_stage, l.ctas_per_sm, l.threads);
    if (cl < 0)
        return HOUGH_ERR_UNSUPPORTED_SHAPE;    // no room for useful candidate lists
    // association keeps one count per warp and category in the tile or in
    // the list area
    const long long cat_counts = (long long)(l.threads / 32) * (ctx->th.max_peaks + 2);
    if (cat_counts > (long long)l.word_rows * tile_bins(ctx, l.word_rows) && cat_counts > cl)
        return HOUGH_ERR_UNSUPPORTED_SHAPE;
    hk::SmemLayout L = hk::smem_layout(l.word_rows, l.hit_stage, tile_bins(ctx, l.word_rows), cl,
                                       l.threads / 32);
    if (L.total > ctx->smem_optin)
        return HOUGH_ERR_UNSUPPORTED_SHAPE;
    out = l;
    smem = L.total;
    return HOUGH_OK;
}

// The shape a find of n_windows windows and n_hits hits runs in: `base`, or,
// when the shape was left to the library (automatic) and its default is
// three 256-thread CTAs per SM, two 512-thread CTAs per SM for windows of
// more than kHeavyWindowHits hits on average.  Heavier windows list more
// candidate bins per tile than the small CTAs' shared memory holds.  Where
// the shapes cross depends on the spread of window sizes as well as the
// mean: Poisson mixes of tracks at 71 / 143 / 199 / 256 / 313 / 427 hits per
// window ran 0.71 / 0.78 / 0.83 / 0.87 / 0.99 / 1.16 times as long in three
// 256-thread CTAs as in two 512-thread ones, and a uniform mix of 1 to 40
// tracks (295 hits, with a long tail) 1.24 times.
constexpr int64_t kHeavyWindowHits = 250;

}  // namespace

hough_launch launch_for(const hough_ctx *ctx, const hough_launch &base, bool automatic,
                        int64_t n_hits, int64_t n_windows)
{
    if (!automatic || n_windows <= 0 || base.threads != 256 || base.ctas_per_sm != 3 ||
        n_hits <= kHeavyWindowHits * n_windows)
        return base;
    hough_launch l{};
    size_t smem = 0;
    if (resolve_launch(ctx, hough_launch{512, 32, 1024, 2}, l, smem) == HOUGH_OK)
        return l;
    return base;
}

namespace {

bool tracks_ok(const hough_ctx *ctx, const hough_tracks *t)
{
    if (!t || !t->n_peaks || !t->hit_track || !t->track_hits || !t->window_status)
        return false;
    if (ctx->th.max_peaks > 0 && !t->peaks)
        return false;
    if ((ctx->th.flags & HOUGH_FLAG_EXPORT_ACC) && !t->acc)
        return false;
    return true;
}

bool hits_ok(const hough_hits *h)
{
    if (!h || h->n_hits < 0)
        return false;
    bool raw = h->vane && h->strip;
    if (!raw && h->n_hits > 0 && !(h->phi_q && h->z_q))
        return false;
    return true;
}

// narrow: the find kernel's narrowed tiles (the other kernels that take these
// parameters keep full-width tiles)
hk::KParams make_params(const hough_ctx *ctx, const hough_hits *hits, const int64_t *offsets,
                        int64_t n_windows, const hough_tracks *out, unsigned int *counter,
                        const hough_launch &l, bool narrow = true)
{
    hk::KParams p{};
    const hough_geometry &g = ctx->g;
    bool raw = hits->vane && hits->strip;
    p.a = raw ? hits->vane : hits->phi_q;
    p.b = raw ? hits->strip : hits->z_q;
    p.n_hits = hits->n_hits;
    p.raw = raw ? 1 : 0;
    p.vane_step = (int)(360LL * g.phi_u_per_deg / g.n_vanes);
    p.z_min_u = g.z_min_u;
    p.z_pitch_u = g.z_pitch_u;
    p.z_half = g.z_pitch_u / 2;
    p.phi_end = 360LL * g.phi_u_per_deg;
    p.z_end = (long long)g.z_min_u + (long long)g.n_z_strips * g.z_pitch_u;
    p.offsets = reinterpret_cast<const long long *>(offsets);
    p.n_windows = n_windows;
    p.C = ctx->d_C;
    p.S = ctx->d_S;
    p.D = (int)ctx->D;
    p.K = ctx->K;
    p.in_range = ctx->in_range ? 1 : 0;
    p.fp64 = (ctx->th.flags & HOUGH_FLAG_FP64) ? 1 : 0;
    p.Cd = ctx->d_Cd;
    p.Sd = ctx->d_Sd;
    p.u_phi = (double)g.phi_u_per_deg;
    p.u_z = (double)g.z_u_per_mm;
    p.rho_min = g.rho_min;
    p.drho = (g.rho_max - g.rho_min) / (double)ctx->n_rho;
    p.n_theta = ctx->n_theta;
    p.n_rho = ctx->n_rho;
    p.T = ctx->th.vote_threshold;
    p.tol = ctx->th.assoc_tol_bins;
    p.max_peaks = ctx->th.max_peaks;
    p.export_acc = (ctx->th.flags & HOUGH_FLAG_EXPORT_ACC) ? 1 : 0;
    p.peaks = out->peaks;
    p.n_peaks = out->n_peaks;
    p.n_found = out->n_found;
    p.hit_track = out->hit_track;
    p.track_hits = out->track_hits;
    p.status = out->window_status;
    p.acc = out->acc;
    p.work = counter;
    p.word_rows = l.word_rows;
    p.lw = l.word_rows == 32 ? 5 : (l.word_rows == 64 ? 6 : 7);
    const int wi = p.lw - 5;
    p.n_b = narrow ? tile_bins(ctx, l.word_rows) : ctx->n_rho;
    p.lo_tab = narrow && ctx->d_lo ? ctx->d_lo + (size_t)wi * 3 * ctx->lo_stride : nullptr;
    p.lo_stride = ctx->lo_stride;
    p.nb_inv = (unsigned)(((1ull << 32) + (unsigned long long)p.n_b - 1) /
                          (unsigned long long)p.n_b);
    p.nrho_inv = (unsigned)(((1ull << 32) + (unsigned long long)ctx->n_rho - 1) /
                            (unsigned long long)ctx->n_rho);
    p.hit_stage = l.hit_stage;
    p.kp = std::max(32, next_pow2(std::max(1, ctx->th.max_peaks)));
    // the list area, split into per-warp lists (a multiple of 32 entries),
    // half of each being the warp's overflow area: a lane's column overflows
    // when its word row is crossed by many more lines than the average row
    const int cl = cl_entries_for(ctx, l.word_rows, l.hit_stage, l.ctas_per_sm, l.threads);
    p.cl_total = cl;
    p.seg_cl = (cl / (l.threads / 32)) & ~31;
    p.seg_ovf = (p.seg_cl / 2) & ~31;
    return p;
}

struct Prepared {
    hough_launch l;
    size_t smem;
    unsigned grid;
};

// The find kernel of a context: fixed-point bins, or the FP64 variant.
using FindKernel = void (*)(hk::KParams);
// The find kernel for this context and CTA size.
static FindKernel find_kernel_of(const hough_ctx *ctx, int threads)
{
    if (ctx->th.flags & HOUGH_FLAG_FP64)
        return hk::find_kernel_fp64;
    return threads <= 256 ? hk::find_kernel_256 : hk::find_kernel;
}

// Resolve a launch shape, raise the kernel's shared-memory limit and size the
// persistent grid (not stream operations, so this runs outside any capture).
int prepare_find(hough_ctx *ctx, int64_t n_windows, const hough_launch &req, Prepared &pr)
{
    int rc = resolve_launch(ctx, req, pr.l, pr.smem);
    if (rc != HOUGH_OK)
        return rc;
    const FindKernel fk = find_kernel_of(ctx, pr.l.threads);
    if (raise_smem_limit(reinterpret_cast<const void *>(fk), pr.smem) != HOUGH_OK)
        return HOUGH_ERR_CUDA;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, fk) != cudaSuccess || fa.sharedSizeBytes > kStaticSmemReserve)
        return HOUGH_ERR_CUDA;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fk, pr.l.threads, pr.smem) !=
            cudaSuccess ||
        occ < 1)
        return HOUGH_ERR_UNSUPPORTED_SHAPE;
    long long grid = (long long)ctx->num_sms * std::min(occ, pr.l.ctas_per_sm);
    pr.grid = (unsigned)std::max<long long>(1, std::min<long long>(grid, n_windows));
    return HOUGH_OK;
}

int enqueue_find(hough_ctx *ctx, const hough_hits *hits, const int64_t *offsets,
                 int64_t n_windows, const hough_tracks *out, cudaStream_t s,
                 unsigned int *counter, const Prepared &pr)
{
    hk::KParams p = make_params(ctx, hits, offsets, n_windows, out, counter, pr.l);
    find_kernel_of(ctx, pr.l.threads)<<<pr.grid, pr.l.threads, pr.smem, s>>>(p);
    if (cudaGetLastError() != cudaSuccess)
        return HOUGH_ERR_CUDA;
    ctx->launches += 1;
    return HOUGH_OK;
}

int launch_find(hough_ctx *ctx, const hough_hits *hits, const int64_t *offsets, int64_t n_windows,
                const hough_tracks *out, cudaStream_t s, unsigned int *counter,
                const hough_launch &req)
{
    Prepared pr{};
    int rc = prepare_find(ctx, n_windows, req, pr);
    if (rc != HOUGH_OK)
        return rc;
    return enqueue_find(ctx, hits, offsets, n_windows, out, s, counter, pr);
}

unsigned int *counter_for(hough_ctx *ctx, cudaStream_t s)
{
    auto it = ctx->counters.find(s);
    if (it != ctx->counters.end())
        return it->second;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (s && cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return nullptr;   // cannot allocate inside a capture; use a plan
    unsigned int *c = nullptr;
    if (cudaMalloc(&c, 2 * sizeof(unsigned int)) != cudaSuccess)
        return nullptr;
    if (cudaMemset(c, 0, 2 * sizeof(unsigned int)) != cudaSuccess) {
        cudaFree(c);
        return nullptr;
    }
    ctx->counters[s] = c;
    return c;
}

int check_find_args(hough_ctx *ctx, const hough_hits *hits, const int64_t *offsets,
                    int64_t n_windows, const hough_tracks *out)
{
    if (!ctx || !hits_ok(hits) || n_windows < 0 || n_windows >= (1ll << 31) - 65536 ||
        (n_windows > 0 && !offsets) || !tracks_ok(ctx, out))
        return HOUGH_ERR_INVALID_ARG;
    return HOUGH_OK;
}

}  // namespace

extern "C" {

int hough_tables(const hough_geometry *g, int n_theta, int n_rho, int32_t *C, int32_t *S,
                 int64_t *D, int32_t *K)
{
    if (!geometry_ok(g) || n_theta <= 0 || n_rho <= 0 || !C || !S || !D || !K)
        return HOUGH_ERR_INVALID_ARG;
    const double span = g->rho_max - g->rho_min;
    const double step = M_PI / (double)n_theta;
    // the four corners of the detector box (the sum is linear in phi and z)
    const long long phis[2] = {0, 360LL * g->phi_u_per_deg - 1};
    const long long zs[2] = {g->z_min_u, (long long)g->z_min_u + (long long)g->n_z_strips * g->z_pitch_u};
    for (int k = HOUGH_MAX_FRAC_BITS; k >= 8; --k) {
        const double scale = std::ldexp((double)n_rho, k) / span;
        const double cs = scale / (double)g->phi_u_per_deg;
        const double ss = scale / (double)g->z_u_per_mm;
        const long long d = round_half_away(-g->rho_min * scale);
        bool fits = d >= -(1LL << 31) && d < (1LL << 31);
        for (int t = 0; t < n_theta && fits; ++t) {
            const double th = ((double)t + 0.5) * step;
            const long long c = round_half_away(std::cos(th) * cs);
            const long long s = round_half_away(std::sin(th) * ss);
            C[t] = (int32_t)c;
            S[t] = (int32_t)s;
            for (long long ph : phis)
                for (long long z : zs) {
                    const long long v = ph * c + z * s + d;
                    if (v < -(1LL << 31) || v >= (1LL << 31))
                        fits = false;
                }
        }
        if (fits) {
            *D = d;
            *K = k;
            return HOUGH_OK;
        }
    }
    return HOUGH_ERR_UNSUPPORTED_SHAPE;
}

int hough_tile_bins(const hough_geometry *g, int n_theta, int n_rho, int word_rows, int32_t *nb,
                    int32_t *lo)
{
    if (!geometry_ok(g) || !nb || !lo || !(word_rows == 32 || word_rows == 64 || word_rows == 128))
        return HOUGH_ERR_INVALID_ARG;
    if (n_theta < 1 || n_theta > HOUGH_MAX_THETA || n_rho < 4 || n_rho > HOUGH_MAX_RHO ||
        n_rho % 4 != 0)
        return HOUGH_ERR_UNSUPPORTED_SHAPE;
    std::vector<int32_t> C(n_theta), S(n_theta), lo_all;
    int64_t D = 0;
    int32_t K = 0;
    const int rc = hough_tables(g, n_theta, n_rho, C.data(), S.data(), &D, &K);
    if (rc != HOUGH_OK)
        return rc;
    int nbs[3];
    narrow_tiles(g, n_theta, n_rho, C.data(), S.data(), D, K, nbs, lo_all);
    const int wi = word_rows == 32 ? 0 : (word_rows == 64 ? 1 : 2);
    const size_t per = (size_t)3 * ((n_theta + 31) / 32);
    *nb = nbs[wi];
    std::memcpy(lo, lo_all.data() + (size_t)wi * per, per * sizeof(int32_t));
    return HOUGH_OK;
}

int hough_create(const hough_geometry *g, int n_theta, int n_rho, const hough_thresholds *th,
                 hough_ctx **out)
{
    if (!out)
        return HOUGH_ERR_INVALID_ARG;
    *out = nullptr;
    if (!geometry_ok(g) || !th || th->vote_threshold < 1 || th->assoc_tol_bins < 0 ||
        th->max_peaks < 0)
        return HOUGH_ERR_INVALID_ARG;
    if (n_theta < 1 || n_theta > HOUGH_MAX_THETA || n_rho < 4 || n_rho > HOUGH_MAX_RHO ||
        n_rho % 4 != 0 || th->max_peaks > HOUGH_MAX_PEAKS)
        return HOUGH_ERR_UNSUPPORTED_SHAPE;
    int dev = 0, ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return HOUGH_ERR_NO_DEVICE;
    }
    if (cudaGetDevice(&dev) != cudaSuccess)
        return HOUGH_ERR_NO_DEVICE;
    hough_ctx *ctx = new (std::nothrow) hough_ctx();
    if (!ctx)
        return HOUGH_ERR_ALLOC;
    ctx->device = dev;
    ctx->g = *g;
    ctx->th = *th;
    ctx->n_theta = n_theta;
    ctx->n_rho = n_rho;
    ctx->C.resize(n_theta);
    ctx->S.resize(n_theta);
    int64_t D = 0;
    int32_t K = 0;
    int rc = hough_tables(g, n_theta, n_rho, ctx->C.data(), ctx->S.data(), &D, &K);
    if (rc != HOUGH_OK) {
        delete ctx;
        return rc;
    }
    ctx->D = D;
    ctx->K = K;
    ctx->in_range = box_votes_in_range(g, n_theta, n_rho, ctx->C.data(), ctx->S.data(), D, K);
    if (device_limits(ctx, dev) != HOUGH_OK) {
        delete ctx;
        return HOUGH_ERR_CUDA;
    }
    if (cudaMalloc(&ctx->d_C, sizeof(int32_t) * n_theta) != cudaSuccess ||
        cudaMalloc(&ctx->d_S, sizeof(int32_t) * n_theta) != cudaSuccess) {
        hough_destroy(ctx);
        return HOUGH_ERR_ALLOC;
    }
    if (cudaMemcpy(ctx->d_C, ctx->C.data(), sizeof(int32_t) * n_theta, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(ctx->d_S, ctx->S.data(), sizeof(int32_t) * n_theta, cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        hough_destroy(ctx);
        return HOUGH_ERR_CUDA;
    }
    if (!(th->flags & HOUGH_FLAG_FP64)) {
        // narrowed tiles (the FP64 variant's bins come from another formula,
        // so its tiles keep every bin)
        std::vector<int32_t> lo_all;
        narrow_tiles(&ctx->g, ctx->n_theta, ctx->n_rho, ctx->C.data(), ctx->S.data(), ctx->D,
                     ctx->K, ctx->tile_nb, lo_all);
        ctx->lo_stride = (ctx->n_theta + 31) / 32;
        if (cudaMalloc(&ctx->d_lo, sizeof(int32_t) * lo_all.size()) != cudaSuccess) {
            hough_destroy(ctx);
            return HOUGH_ERR_ALLOC;
        }
        if (cudaMemcpy(ctx->d_lo, lo_all.data(), sizeof(int32_t) * lo_all.size(),
                       cudaMemcpyHostToDevice) != cudaSuccess) {
            hough_destroy(ctx);
            return HOUGH_ERR_CUDA;
        }
    }
    if (th->flags & HOUGH_FLAG_FP64) {
        // cos and sin of the row centres theta_t = (t + 1/2) pi / n_theta
        std::vector<double> cd(n_theta), sd(n_theta);
        for (int t = 0; t < n_theta; ++t) {
            const double theta = ((double)t + 0.5) * (M_PI / (double)n_theta);
            cd[t] = cos(theta);
            sd[t] = sin(theta);
        }
        if (cudaMalloc(&ctx->d_Cd, sizeof(double) * n_theta) != cudaSuccess ||
            cudaMalloc(&ctx->d_Sd, sizeof(double) * n_theta) != cudaSuccess) {
            hough_destroy(ctx);
            return HOUGH_ERR_ALLOC;
        }
        if (cudaMemcpy(ctx->d_Cd, cd.data(), sizeof(double) * n_theta, cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(ctx->d_Sd, sd.data(), sizeof(double) * n_theta, cudaMemcpyHostToDevice) !=
                cudaSuccess) {
            hough_destroy(ctx);
            return HOUGH_ERR_CUDA;
        }
    }
    hough_launch l{};
    size_t smem = 0;
    rc = resolve_launch(ctx, hough_launch{}, l, smem);
    if (rc != HOUGH_OK) {
        hough_destroy(ctx);
        return rc;
    }
    ctx->launch = l;
    *out = ctx;
    return HOUGH_OK;
}

void hough_destroy(hough_ctx *ctx)
{
    if (!ctx)
        return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    for (auto &kv : ctx->counters)
        cudaFree(kv.second);
    cudaFree(ctx->d_C);
    cudaFree(ctx->d_S);
    cudaFree(ctx->d_Cd);
    cudaFree(ctx->d_Sd);
    cudaFree(ctx->d_lo);
    cudaFree(ctx->stage_dev);
    cudaFree(ctx->d_cf);
    for (int i = 0; i < 2; ++i) {
        if (ctx->host_streams[i])
            cudaStreamDestroy(ctx->host_streams[i]);
        if (ctx->host_events[i])
            cudaEventDestroy(ctx->host_events[i]);
    }
    cudaSetDevice(prev);
    delete ctx;
}

int hough_encode(hough_ctx *ctx, const int32_t *vane, const int32_t *strip, int64_t n,
                 int32_t *phi_q, int32_t *z_q, void *stream)
{
    if (!ctx || n < 0 || (n > 0 && (!vane || !strip || !phi_q || !z_q)))
        return fail(ctx, HOUGH_ERR_INVALID_ARG);
    if (n == 0)
        return HOUGH_OK;
    const hough_geometry &g = ctx->g;
    int blocks = (int)std::min<long long>((n + 255) / 256, (long long)ctx->num_sms * 8);
    hk::encode_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(
        vane, strip, n, (int)(360LL * g.phi_u_per_deg / g.n_vanes), g.z_min_u, g.z_pitch_u,
        g.z_pitch_u / 2, phi_q, z_q);
    if (cudaGetLastError() != cudaSuccess)
        return fail(ctx, HOUGH_ERR_CUDA);
    ctx->launches += 1;
    return HOUGH_OK;
}

int hough_find(hough_ctx *ctx, const hough_hits *hits, const int64_t *window_offsets,
               int64_t n_windows, const hough_tracks *tracks_out, void *stream)
{
    int rc = check_find_args(ctx, hits, window_offsets, n_windows, tracks_out);
    if (rc != HOUGH_OK)
        return fail(ctx, rc);
    if (n_windows == 0)
        return HOUGH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int *c = counter_for(ctx, s);
    if (!c)
        return fail(ctx, HOUGH_ERR_ALLOC);
    rc = launch_find(ctx, hits, window_offsets, n_windows, tracks_out, s, c,
                     launch_for(ctx, ctx->launch, ctx->auto_launch, hits->n_hits, n_windows));
    return fail(ctx, rc);
}

}  // extern "C"

// ---------------------------------------------------------------- no alloc
// hough_find_noalloc keeps the little global memory the find kernel needs
// beyond its inputs and outputs -- the scheduling counter pair and the
// cos/sin tables -- in this file-scope device array instead of memory from
// cudaMalloc.  Every GPU that loads the library holds it until the process
// exits, and every call on that GPU shares it.
namespace {
constexpr size_t kNoAllocCounterBytes = 256;
constexpr size_t kNoAllocBytes =
    kNoAllocCounterBytes + 2 * sizeof(int32_t) * (size_t)HOUGH_NOALLOC_MAX_THETA;
std::mutex g_noalloc_mutex;
void *g_noalloc_base[HOUGH_NOALLOC_MAX_DEVICES];   // device address of the array, per device
// host copies of the tables, written and sent under the mutex (static: the
// callers this entry point serves may run on small stacks)
int32_t g_noalloc_C[HOUGH_NOALLOC_MAX_THETA], g_noalloc_S[HOUGH_NOALLOC_MAX_THETA];
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

extern "C" {

int hough_find_noalloc(const hough_geometry *g, int n_theta, int n_rho,
                       const hough_thresholds *th, const hough_hits *hits,
                       const int64_t *window_offsets, int64_t n_windows,
                       const hough_tracks *tracks_out, void *stream)
{
    if (!geometry_ok(g) || !th || th->vote_threshold < 1 || th->assoc_tol_bins < 0 ||
        th->max_peaks < 0 || (th->flags & HOUGH_FLAG_FP64) || !hits_ok(hits) || n_windows < 0 ||
        n_windows >= (1ll << 31) - 65536 || (n_windows > 0 && !window_offsets))
        return HOUGH_ERR_INVALID_ARG;
    if (n_theta < 1 || n_theta > HOUGH_NOALLOC_MAX_THETA || n_rho < 4 || n_rho > HOUGH_MAX_RHO ||
        n_rho % 4 != 0 || th->max_peaks > HOUGH_MAX_PEAKS)
        return HOUGH_ERR_UNSUPPORTED_SHAPE;
    cudaStream_t s = (cudaStream_t)stream;
    // every call copies its tables from host memory, which a stream that is
    // capturing a graph cannot take: refuse before touching the stream
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        return HOUGH_ERR_CUDA;
    }
    if (cap != cudaStreamCaptureStatusNone)
        return HOUGH_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return HOUGH_ERR_NO_DEVICE;
    }
    if (dev < 0 || dev >= HOUGH_NOALLOC_MAX_DEVICES)
        return HOUGH_ERR_UNSUPPORTED_SHAPE;
    // set-up, once per device, with that device current: the array's name is
    // only a host-side stand-in, so ask the runtime for its device address
    std::unique_lock<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_base[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return HOUGH_ERR_CUDA;
        }
        g_noalloc_base[dev] = ptr;
    }
    unsigned char *base = static_cast<unsigned char *>(g_noalloc_base[dev]);
    // the tables in the library's static host buffers (held under the mutex
    // until the copies below have taken them), then into the device array
    int32_t *C = g_noalloc_C, *S = g_noalloc_S;
    int64_t D = 0;
    int32_t K = 0;
    int rc = hough_tables(g, n_theta, n_rho, C, S, &D, &K);
    if (rc != HOUGH_OK)
        return rc;
    hough_ctx ctx;          // a plain local description: nothing in it allocates or is freed
    ctx.device = dev;
    ctx.g = *g;
    ctx.th = *th;
    ctx.n_theta = n_theta;
    ctx.n_rho = n_rho;
    ctx.D = D;
    ctx.K = K;
    ctx.in_range = box_votes_in_range(g, n_theta, n_rho, C, S, D, K);
    if (device_limits(&ctx, dev) != HOUGH_OK)
        return HOUGH_ERR_CUDA;
    if (!tracks_ok(&ctx, tracks_out))
        return HOUGH_ERR_INVALID_ARG;
    unsigned int *counter = reinterpret_cast<unsigned int *>(base);
    ctx.d_C = reinterpret_cast<int32_t *>(base + kNoAllocCounterBytes);
    ctx.d_S = ctx.d_C + HOUGH_NOALLOC_MAX_THETA;
    hough_launch l{};
    size_t smem = 0;
    rc = resolve_launch(&ctx, hough_launch{}, l, smem);
    if (rc != HOUGH_OK)
        return rc;
    ctx.launch = l;
    // the array keeps the last call's contents: the counters must start at 0
    if (cudaMemsetAsync(counter, 0, 2 * sizeof(unsigned int), s) != cudaSuccess ||
        cudaMemcpyAsync(ctx.d_C, C, sizeof(int32_t) * n_theta, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(ctx.d_S, S, sizeof(int32_t) * n_theta, cudaMemcpyHostToDevice, s) !=
            cudaSuccess) {
        cudaGetLastError();
        return HOUGH_ERR_CUDA;
    }
    // a copy from pageable host memory has taken its source when it returns
    lock.unlock();
    if (n_windows == 0)
        return HOUGH_OK;
    return launch_find(&ctx, hits, window_offsets, n_windows, tracks_out, s, counter, l);
}

int hough_find_coarse_fine(hough_ctx *ctx, const hough_hits *hits, const int64_t *window_offsets,
                           int64_t n_windows, hough_line *lines, int32_t *hit_track,
                           void *stream)
{
    if (!ctx || !hits_ok(hits) || n_windows < 0 || (n_windows > 0 && (!window_offsets || !lines)) ||
        (hits->n_hits > 0 && !hit_track))
        return fail(ctx, HOUGH_ERR_INVALID_ARG);
    if (n_windows == 0)
        return HOUGH_OK;
    if (!ctx->d_cf) {
        // the coarse 18 x 100 and fine 180 x 1000 tables, built once
        std::vector<int32_t> tab(2 * hk::kCfCoarseT + 2 * hk::kCfFineT);
        int64_t D = 0;
        int32_t K = 0;
        int rc = hough_tables(&ctx->g, hk::kCfCoarseT, hk::kCfCoarseR, tab.data(),
                              tab.data() + hk::kCfCoarseT, &D, &K);
        if (rc != HOUGH_OK)
            return fail(ctx, rc);
        ctx->cf_D[0] = D;
        ctx->cf_K[0] = K;
        rc = hough_tables(&ctx->g, hk::kCfFineT, hk::kCfFineR, tab.data() + 2 * hk::kCfCoarseT,
                          tab.data() + 2 * hk::kCfCoarseT + hk::kCfFineT, &D, &K);
        if (rc != HOUGH_OK)
            return fail(ctx, rc);
        ctx->cf_D[1] = D;
        ctx->cf_K[1] = K;
        int32_t *d = nullptr;
        if (cudaMalloc(&d, sizeof(int32_t) * tab.size()) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, HOUGH_ERR_ALLOC);
        }
        if (cudaMemcpy(d, tab.data(), sizeof(int32_t) * tab.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
            cudaFree(d);
            return fail(ctx, HOUGH_ERR_CUDA);
        }
        ctx->d_cf = d;
    }
    const hough_geometry &g = ctx->g;
    const bool raw = hits->vane && hits->strip;
    hk::CfParams p{};
    p.a = raw ? hits->vane : hits->phi_q;
    p.b = raw ? hits->strip : hits->z_q;
    p.n_hits = hits->n_hits;
    p.raw = raw ? 1 : 0;
    p.vane_step = (int)(360LL * g.phi_u_per_deg / g.n_vanes);
    p.z_min_u = g.z_min_u;
    p.z_pitch_u = g.z_pitch_u;
    p.z_half = g.z_pitch_u / 2;
    p.phi_end = 360LL * g.phi_u_per_deg;
    p.z_end = (long long)g.z_min_u + (long long)g.n_z_strips * g.z_pitch_u;
    p.offsets = reinterpret_cast<const long long *>(window_offsets);
    p.n_windows = n_windows;
    p.Cc = ctx->d_cf;
    p.Sc = ctx->d_cf + hk::kCfCoarseT;
    p.Cf = ctx->d_cf + 2 * hk::kCfCoarseT;
    p.Sf = ctx->d_cf + 2 * hk::kCfCoarseT + hk::kCfFineT;
    p.Dc = (int)ctx->cf_D[0];
    p.Kc = ctx->cf_K[0];
    p.Df = (int)ctx->cf_D[1];
    p.Kf = ctx->cf_K[1];
    p.T = ctx->th.vote_threshold;
    p.tol = ctx->th.assoc_tol_bins;
    p.lines = lines;
    p.hit_track = hit_track;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hk::coarse_fine_kernel,
                                                      32 * hk::kCfWarps, 0) != cudaSuccess ||
        occ < 1)
        return fail(ctx, HOUGH_ERR_CUDA);
    const long long blocks = std::min<long long>((n_windows + hk::kCfWarps - 1) / hk::kCfWarps,
                                                 (long long)ctx->num_sms * occ);
    hk::coarse_fine_kernel<<<(unsigned)blocks, 32 * hk::kCfWarps, 0, (cudaStream_t)stream>>>(p);
    if (cudaGetLastError() != cudaSuccess)
        return fail(ctx, HOUGH_ERR_CUDA);
    ctx->launches += 1;
    return HOUGH_OK;
}

int hough_accumulate(hough_ctx *ctx, const hough_hits *hits, const int64_t *window_offsets,
                     int64_t n_windows, int32_t *acc, uint32_t *window_status, void *stream)
{
    if (!ctx || !hits_ok(hits) || n_windows < 0 || n_windows >= (1ll << 31) - 65536 ||
        (n_windows > 0 && (!window_offsets || !acc || !window_status)) ||
        (reinterpret_cast<uintptr_t>(acc) & 3u) != 0 || (ctx->th.flags & HOUGH_FLAG_FP64))
        return fail(ctx, HOUGH_ERR_INVALID_ARG);
    if (n_windows == 0)
        return HOUGH_OK;
    // tiles of 32 word rows and a stage of 2048 hits; 512-thread CTAs where
    // two or more fit on an SM, else one CTA of 1024 threads
    const int word_rows = 32, hit_stage = 2048;
    const size_t smem = hk::align_up((size_t)word_rows * ctx->n_rho * 4, 16) + (size_t)hit_stage * 8;
    if (ctx->acc_threads == 0) {
        // worked out once per context
        cudaFuncAttributes fa{};
        if (cudaFuncGetAttributes(&fa, hk::accumulate_kernel) != cudaSuccess)
            return fail(ctx, HOUGH_ERR_CUDA);
        if (smem + fa.sharedSizeBytes > ctx->smem_optin)
            return fail(ctx, HOUGH_ERR_UNSUPPORTED_SHAPE);
        if (raise_smem_limit(reinterpret_cast<const void *>(hk::accumulate_kernel), smem) !=
            HOUGH_OK)
            return fail(ctx, HOUGH_ERR_CUDA);
        int threads = 512, occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hk::accumulate_kernel, threads,
                                                          smem) != cudaSuccess)
            return fail(ctx, HOUGH_ERR_CUDA);
        if (occ < 2) {
            threads = 1024;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hk::accumulate_kernel,
                                                              threads, smem) != cudaSuccess)
                return fail(ctx, HOUGH_ERR_CUDA);
            if (occ < 1)
                return fail(ctx, HOUGH_ERR_UNSUPPORTED_SHAPE);
        }
        ctx->acc_threads = threads;
        ctx->acc_occ = occ;
    }
    const int threads = ctx->acc_threads, occ = ctx->acc_occ;
    hough_tracks out{};
    out.acc = acc;
    out.window_status = window_status;
    hough_launch l{threads, word_rows, hit_stage, occ};
    const hk::KParams p = make_params(ctx, hits, window_offsets, n_windows, &out, nullptr, l, false);
    const long long grid = std::min<long long>(n_windows, (long long)ctx->num_sms * occ);
    hk::accumulate_kernel<<<(unsigned)grid, threads, smem, (cudaStream_t)stream>>>(p);
    if (cudaGetLastError() != cudaSuccess)
        return fail(ctx, HOUGH_ERR_CUDA);
    ctx->launches += 1;
    return HOUGH_OK;
}

int hough_find_iterative(hough_ctx *ctx, const hough_hits *hits, const int64_t *window_offsets,
                         int64_t n_windows, int32_t max_tracks, hough_iter_track *tracks,
                         int32_t *n_tracks, int32_t *hit_track, uint32_t *window_status,
                         void *stream)
{
    if (!ctx || !hits_ok(hits) || n_windows < 0 || max_tracks < 1 ||
        max_tracks > HOUGH_MAX_PEAKS ||
        (n_windows > 0 && (!window_offsets || !tracks || !n_tracks || !window_status)) ||
        (hits->n_hits > 0 && !hit_track) || n_windows >= (1ll << 31) - 65536)
        return fail(ctx, HOUGH_ERR_INVALID_ARG);
    if (n_windows == 0)
        return HOUGH_OK;
    // 512 threads, tiles of 32 word rows beside the stage of hits and the
    // kernel's static shared variables (small tiles let more of them be
    // skipped once their count bound falls; 64 or 128 word rows were slower)
    hough_launch l{512, 32, HOUGH_ITER_MAX_HITS, 1};
    const size_t stage = (size_t)HOUGH_ITER_MAX_HITS * 12;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, hk::iterative_kernel) != cudaSuccess)
        return fail(ctx, HOUGH_ERR_CUDA);
    const size_t room = ctx->smem_optin + 128 > fa.sharedSizeBytes
                            ? ctx->smem_optin + 128 - fa.sharedSizeBytes : 0;
    // the find's narrowed tiles
    const size_t smem = (size_t)l.word_rows * tile_bins(ctx, l.word_rows) * 4 + stage;
    if (smem > room)
        return fail(ctx, HOUGH_ERR_UNSUPPORTED_SHAPE);
    if (raise_smem_limit(reinterpret_cast<const void *>(hk::iterative_kernel), smem) != HOUGH_OK)
        return fail(ctx, HOUGH_ERR_CUDA);
    hough_tracks out{};
    out.hit_track = hit_track;
    out.window_status = window_status;
    hk::IterParams q{};
    q.k = make_params(ctx, hits, window_offsets, n_windows, &out, nullptr, l);
    q.max_tracks = max_tracks;
    q.tracks = reinterpret_cast<int4 *>(tracks);
    q.n_tracks = n_tracks;
    const long long grid = std::min<long long>(n_windows, (long long)ctx->num_sms);
    hk::iterative_kernel<<<(unsigned)grid, 512, smem, (cudaStream_t)stream>>>(q);
    if (cudaGetLastError() != cudaSuccess)
        return fail(ctx, HOUGH_ERR_CUDA);
    ctx->launches += 1;
    return HOUGH_OK;
}

int hough_extend(hough_ctx *ctx, const hough_hits *hits, const int64_t *window_offsets,
                 int64_t n_windows, const hough_tracks *found, int32_t tol_z,
                 hough_extension *out, void *stream)
{
    if (!ctx || !hits_ok(hits) || n_windows < 0 || !found || !out || tol_z < 0 ||
        tol_z > HOUGH_EXT_MAX_TOL || n_windows >= (1ll << 31) - 65536 ||
        (n_windows > 0 && (!window_offsets || !found->peaks || !found->n_peaks ||
                           !out->tracks || !out->window_status)) ||
        (hits->n_hits > 0 && (!found->hit_track || !found->track_hits || !out->ext_track ||
                              !out->ext_hits)))
        return fail(ctx, HOUGH_ERR_INVALID_ARG);
    const int nv = ctx->g.n_vanes;
    if (nv < 3 || nv > HOUGH_EXT_MAX_VANES || 360LL * ctx->g.phi_u_per_deg / nv <= 0)
        return fail(ctx, HOUGH_ERR_UNSUPPORTED_SHAPE);
    if (n_windows == 0)
        return HOUGH_OK;
    hough_launch l{32, 32, 0, 1};
    hk::ExtParams q{};
    hough_tracks f = *found;
    f.window_status = nullptr;
    f.acc = nullptr;
    q.k = make_params(ctx, hits, window_offsets, n_windows, &f, nullptr, l, false);
    q.n_vanes = nv;
    q.tol_z = tol_z;
    q.ext = reinterpret_cast<int4 *>(out->tracks);
    q.ext_track = out->ext_track;
    q.ext_hits = out->ext_hits;
    q.status = out->window_status;
    // small stages for most windows (many warps per SM), then larger ones for
    // the windows above them
    const int caps[3] = {512, 1536, HOUGH_EXT_MAX_HITS};
    long long lo = -1;
    for (int pass = 0; pass < 3; ++pass) {
        const size_t smem = hk::ext_smem_bytes(caps[pass], nv);
        if (smem > ctx->smem_optin)
            return fail(ctx, HOUGH_ERR_UNSUPPORTED_SHAPE);
        if (raise_smem_limit(reinterpret_cast<const void *>(hk::extend_kernel), smem) != HOUGH_OK)
            return fail(ctx, HOUGH_ERR_CUDA);
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hk::extend_kernel, 32, smem) !=
                cudaSuccess || occ < 1)
            return fail(ctx, HOUGH_ERR_CUDA);
        q.cap = caps[pass];
        q.lo = lo;
        q.flag_large = pass == 2;
        const long long grid = std::min<long long>(n_windows, (long long)ctx->num_sms * occ);
        hk::extend_kernel<<<(unsigned)grid, 32, smem, (cudaStream_t)stream>>>(q);
        if (cudaGetLastError() != cudaSuccess)
            return fail(ctx, HOUGH_ERR_CUDA);
        ctx->launches += 1;
        lo = caps[pass];
    }
    return HOUGH_OK;
}

int hough_time_slice(hough_ctx *ctx, const int64_t *t, const int32_t *in0, const int32_t *in1,
                     int64_t n_hits, int64_t t0, int64_t step, int64_t len, int64_t n_windows,
                     int32_t *out0, int32_t *out1, int64_t *out_index, int64_t out_capacity,
                     int64_t *window_offsets, uint32_t *status, void *stream)
{
    if (!ctx || n_hits < 0 || n_windows < 0 || step <= 0 || len <= 0 || !window_offsets ||
        (n_hits > 0 && (!t || !in0 || !in1 || !out0 || !out1)))
        return fail(ctx, HOUGH_ERR_INVALID_ARG);
    if (len % step != 0 || len / step > HOUGH_SLICE_MAX_OVERLAP)
        return fail(ctx, HOUGH_ERR_UNSUPPORTED_SHAPE);
    const int m = (int)(len / step);
    if (out_capacity < 0 || (n_hits > 0 && out_capacity / m < n_hits))
        return fail(ctx, HOUGH_ERR_INVALID_ARG);
    // the window starts must stay inside int64
    const long long lim = (long long)(INT64_MAX / 4);
    if (t0 > lim || t0 < -lim || step > lim / (n_windows + m + 1))
        return fail(ctx, HOUGH_ERR_INVALID_ARG);
    cudaStream_t s = (cudaStream_t)stream;
    if (status && cudaMemsetAsync(status, 0, sizeof(uint32_t), s) != cudaSuccess)
        return fail(ctx, HOUGH_ERR_CUDA);
    hk::SliceParams q{};
    q.t = reinterpret_cast<const long long *>(t);
    q.in0 = in0;
    q.in1 = in1;
    q.n = n_hits;
    q.t0 = t0;
    q.step = step;
    q.n_windows = n_windows;
    q.cap = out_capacity;
    q.m = m;
    q.out0 = out0;
    q.out1 = out1;
    q.out_index = reinterpret_cast<long long *>(out_index);
    q.offsets = reinterpret_cast<long long *>(window_offsets);
    q.status = status;
    // blocks of consecutive windows per CTA step: the largest power of two
    // (32 to kSliceBlock) that still gives every SM eight of them
    int B = hk::kSliceBlock;
    while (B > 32 && (n_windows + 1) / B < 8LL * ctx->num_sms)
        B >>= 1;
    q.block = B;
    const long long blocks = std::min<long long>((n_windows + 1 + B - 1) / B,
                                                 (long long)ctx->num_sms * 8);
    hk::slice_kernel<<<(unsigned)std::max<long long>(blocks, 1), 256, 0, s>>>(q);
    if (cudaGetLastError() != cudaSuccess)
        return fail(ctx, HOUGH_ERR_CUDA);
    ctx->launches += 1;
    return HOUGH_OK;
}

int hough_find_host(hough_ctx *ctx, const hough_hits *hits, const int64_t *window_offsets,
                    int64_t n_windows, const hough_tracks *out, void *stream)
{
    int rc = check_find_args(ctx, hits, window_offsets, n_windows, out);
    if (rc != HOUGH_OK)
        return fail(ctx, rc);
    if (n_windows == 0)
        return HOUGH_OK;
    const long long H = hits->n_hits;
    const bool raw = hits->vane && hits->strip;
    const int mp = ctx->th.max_peaks;
    const bool exp_acc = (ctx->th.flags & HOUGH_FLAG_EXPORT_ACC) != 0;
    const size_t acc_per_w = exp_acc ? (size_t)ctx->n_theta * ctx->n_rho * 4 : 0;
    // device layout: offsets | in0 | in1 | peaks | n_peaks | n_found | hit_track | track_hits | status | acc
    auto al = [](size_t x) { return hk::align_up(x, 256); };
    size_t o_off = 0;
    size_t o_in0 = al(o_off + 8 * (size_t)(n_windows + 1));
    size_t o_in1 = al(o_in0 + 4 * (size_t)H);
    size_t o_pk = al(o_in1 + 4 * (size_t)H);
    size_t o_np = al(o_pk + sizeof(hough_peak) * (size_t)n_windows * mp);
    size_t o_nf = al(o_np + 4 * (size_t)n_windows);
    size_t o_ht = al(o_nf + 4 * (size_t)n_windows);
    size_t o_th = al(o_ht + 4 * (size_t)H);
    size_t o_st = al(o_th + 4 * (size_t)H);
    size_t o_acc = al(o_st + 4 * (size_t)n_windows);
    size_t total = al(o_acc + acc_per_w * (size_t)n_windows);
    if (total > ctx->stage_bytes) {
        cudaFree(ctx->stage_dev);
        ctx->stage_dev = nullptr;
        ctx->stage_bytes = 0;
        if (cudaMalloc(&ctx->stage_dev, total) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, HOUGH_ERR_ALLOC);
        }
        ctx->stage_bytes = total;
    }
    char *base = (char *)ctx->stage_dev;
    cudaStream_t s = (cudaStream_t)stream;
    auto cp = [](void *dst, const void *src, size_t n, cudaMemcpyKind k, cudaStream_t cs) {
        return n == 0 || cudaMemcpyAsync(dst, src, n, k, cs) == cudaSuccess;
    };
    // two internal streams alternate over chunks of windows, so that the
    // copies of one chunk overlap the kernel of another; they start after
    // the work already queued on `stream`
    for (int i = 0; i < 2; ++i) {
        if (!ctx->host_streams[i] &&
            cudaStreamCreateWithFlags(&ctx->host_streams[i], cudaStreamNonBlocking) != cudaSuccess)
            return fail(ctx, HOUGH_ERR_CUDA);
        if (!ctx->host_events[i] &&
            cudaEventCreateWithFlags(&ctx->host_events[i], cudaEventDisableTiming) != cudaSuccess)
            return fail(ctx, HOUGH_ERR_CUDA);
    }
    if (cudaEventRecord(ctx->host_events[0], s) != cudaSuccess)
        return fail(ctx, HOUGH_ERR_CUDA);
    unsigned int *ctr[2];
    for (int i = 0; i < 2; ++i) {
        ctr[i] = counter_for(ctx, ctx->host_streams[i]);
        if (!ctr[i])
            return fail(ctx, HOUGH_ERR_ALLOC);
        if (cudaStreamWaitEvent(ctx->host_streams[i], ctx->host_events[0], 0) != cudaSuccess)
            return fail(ctx, HOUGH_ERR_CUDA);
    }
    hough_hits dh{};
    dh.n_hits = H;
    if (raw) {
        dh.vane = (const int32_t *)(base + o_in0);
        dh.strip = (const int32_t *)(base + o_in1);
    } else {
        dh.phi_q = (const int32_t *)(base + o_in0);
        dh.z_q = (const int32_t *)(base + o_in1);
    }
    hough_tracks dt{};
    dt.peaks = (hough_peak *)(base + o_pk);
    dt.n_peaks = (int32_t *)(base + o_np);
    dt.n_found = (int32_t *)(base + o_nf);
    dt.hit_track = (int32_t *)(base + o_ht);
    dt.track_hits = (int32_t *)(base + o_th);
    dt.window_status = (uint32_t *)(base + o_st);
    dt.acc = exp_acc ? (int32_t *)(base + o_acc) : nullptr;
    const int32_t *in0 = raw ? hits->vane : hits->phi_q;
    const int32_t *in1 = raw ? hits->strip : hits->z_q;
    // chunk k: windows [w0, w1) read hits [offsets[w0], offsets[w1]) of the
    // whole staged arrays (offsets stay absolute), outputs land at their
    // final places; a window whose offsets are bad reads nothing
    const int64_t n_chunks = n_windows >= 8192 ? 4 : 1;
    Prepared pr{};
    rc = prepare_find(ctx, (n_windows + n_chunks - 1) / n_chunks,
                      launch_for(ctx, ctx->launch, ctx->auto_launch, hits->n_hits, n_windows), pr);
    if (rc != HOUGH_OK)
        return fail(ctx, rc);
    auto clampH = [&](int64_t v) { return std::min<int64_t>(std::max<int64_t>(v, 0), H); };
    bool ok = true;
    for (int64_t k = 0; k < n_chunks && ok; ++k) {
        const int64_t w0 = n_windows * k / n_chunks, w1 = n_windows * (k + 1) / n_chunks;
        const int64_t nw = w1 - w0;
        // hit range of the chunk (a hull of its windows' ranges, clamped)
        int64_t h0 = H, h1 = 0;
        for (int64_t w = w0; w <= w1; ++w) {
            h0 = std::min(h0, clampH(window_offsets[w]));
            h1 = std::max(h1, clampH(window_offsets[w]));
        }
        if (h1 < h0)
            h1 = h0;
        cudaStream_t cs = ctx->host_streams[k & 1];
        ok = cp(base + o_off + 8 * w0, window_offsets + w0, 8 * (size_t)(nw + 1),
                cudaMemcpyHostToDevice, cs) &&
             cp(base + o_in0 + 4 * h0, in0 + h0, 4 * (size_t)(h1 - h0), cudaMemcpyHostToDevice, cs) &&
             cp(base + o_in1 + 4 * h0, in1 + h0, 4 * (size_t)(h1 - h0), cudaMemcpyHostToDevice, cs);
        if (!ok)
            break;
        hough_tracks ct = dt;
        ct.peaks = dt.peaks + (size_t)w0 * mp;
        ct.n_peaks = dt.n_peaks + w0;
        ct.n_found = dt.n_found + w0;
        ct.window_status = dt.window_status + w0;
        if (exp_acc)
            ct.acc = dt.acc + (size_t)w0 * ctx->n_theta * ctx->n_rho;
        Prepared pk = pr;
        pk.grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(pr.grid, nw));
        rc = enqueue_find(ctx, &dh, (const int64_t *)(base + o_off) + w0, nw, &ct, cs, ctr[k & 1], pk);
        if (rc != HOUGH_OK)
            return fail(ctx, rc);
        ok = cp(out->peaks + (size_t)w0 * mp, ct.peaks, sizeof(hough_peak) * (size_t)nw * mp,
                cudaMemcpyDeviceToHost, cs) &&
             cp(out->n_peaks + w0, ct.n_peaks, 4 * (size_t)nw, cudaMemcpyDeviceToHost, cs) &&
             (!out->n_found ||
              cp(out->n_found + w0, ct.n_found, 4 * (size_t)nw, cudaMemcpyDeviceToHost, cs)) &&
             cp(out->hit_track + h0, dt.hit_track + h0, 4 * (size_t)(h1 - h0), cudaMemcpyDeviceToHost, cs) &&
             cp(out->track_hits + h0, dt.track_hits + h0, 4 * (size_t)(h1 - h0), cudaMemcpyDeviceToHost, cs) &&
             cp(out->window_status + w0, ct.window_status, 4 * (size_t)nw, cudaMemcpyDeviceToHost, cs) &&
             (!exp_acc || cp(out->acc + (size_t)w0 * ctx->n_theta * ctx->n_rho, ct.acc,
                             acc_per_w * (size_t)nw, cudaMemcpyDeviceToHost, cs));
    }
    // both internal streams finish before the call returns; `stream` then
    // waits on them too, so later work on it sees the results
    for (int i = 0; i < 2; ++i)
        if (cudaEventRecord(ctx->host_events[i], ctx->host_streams[i]) != cudaSuccess ||
            cudaStreamWaitEvent(s, ctx->host_events[i], 0) != cudaSuccess)
            ok = false;
    if (!ok) {
        cudaStreamSynchronize(ctx->host_streams[0]);
        cudaStreamSynchronize(ctx->host_streams[1]);
        return fail(ctx, HOUGH_ERR_CUDA);
    }
    if (cudaStreamSynchronize(ctx->host_streams[0]) != cudaSuccess ||
        cudaStreamSynchronize(ctx->host_streams[1]) != cudaSuccess)
        return fail(ctx, HOUGH_ERR_CUDA);
    return HOUGH_OK;
}

int hough_plan_create(hough_ctx *ctx, const hough_hits *hits, const int64_t *window_offsets,
                      int64_t n_windows, const hough_tracks *tracks_out, void *stream,
                      hough_plan **out)
{
    if (!out)
        return fail(ctx, HOUGH_ERR_INVALID_ARG);
    *out = nullptr;
    int rc = check_find_args(ctx, hits, window_offsets, n_windows, tracks_out);
    if (rc != HOUGH_OK)
        return fail(ctx, rc);
    hough_plan *plan = new (std::nothrow) hough_plan();
    if (!plan)
        return fail(ctx, HOUGH_ERR_ALLOC);
    plan->ctx = ctx;
    if (cudaMalloc(&plan->counter, 2 * sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(plan->counter, 0, 2 * sizeof(unsigned int)) != cudaSuccess) {
        hough_plan_destroy(plan);
        return fail(ctx, HOUGH_ERR_ALLOC);
    }
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
        hough_plan_destroy(plan);
        return fail(ctx, HOUGH_ERR_CUDA);
    }
    (void)stream;
    Prepared pr{};
    rc = n_windows > 0 ? prepare_find(ctx, n_windows,
                                      launch_for(ctx, ctx->launch, ctx->auto_launch,
                                                 hits->n_hits, n_windows), pr)
                       : HOUGH_OK;
    if (rc != HOUGH_OK) {
        // nothing to capture
    } else if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        rc = HOUGH_ERR_CUDA;
    } else {
        if (n_windows > 0)
            rc = enqueue_find(ctx, hits, window_offsets, n_windows, tracks_out, cap, plan->counter,
                              pr);
        if (cudaStreamEndCapture(cap, &plan->graph) != cudaSuccess && rc == HOUGH_OK)
            rc = HOUGH_ERR_CUDA;
    }
    cudaStreamDestroy(cap);
    if (rc == HOUGH_OK && cudaGraphInstantiate(&plan->exec, plan->graph, 0) != cudaSuccess)
        rc = HOUGH_ERR_CUDA;
    if (rc != HOUGH_OK) {
        cudaGetLastError();
        hough_plan_destroy(plan);
        return fail(ctx, rc);
    }
    *out = plan;
    return HOUGH_OK;
}

int hough_plan_launch(hough_plan *plan, void *stream)
{
    if (!plan || !plan->exec)
        return HOUGH_ERR_INVALID_ARG;
    if (cudaGraphLaunch(plan->exec, (cudaStream_t)stream) != cudaSuccess)
        return fail(plan->ctx, HOUGH_ERR_CUDA);
    plan->ctx->launches += 1;
    return HOUGH_OK;
}

void hough_plan_destroy(hough_plan *plan)
{
    if (!plan)
        return;
    if (plan->exec)
        cudaGraphExecDestroy(plan->exec);
    if (plan->graph)
        cudaGraphDestroy(plan->graph);
    cudaFree(plan->counter);
    delete plan;
}

int hough_get_launch(const hough_ctx *ctx, hough_launch *out)
{
    if (!ctx || !out)
        return HOUGH_ERR_INVALID_ARG;
    *out = ctx->launch;
    return HOUGH_OK;
}

int hough_set_launch(hough_ctx *ctx, const hough_launch *cfg)
{
    if (!ctx || !cfg)
        return fail(ctx, HOUGH_ERR_INVALID_ARG);
    hough_launch l{};
    size_t smem = 0;
    int rc = resolve_launch(ctx, *cfg, l, smem);
    if (rc != HOUGH_OK)
        return fail(ctx, rc);
    ctx->launch = l;
    ctx->auto_launch = cfg->threads == 0 && cfg->word_rows == 0 && cfg->hit_stage == 0 &&
                       cfg->ctas_per_sm == 0;
    return HOUGH_OK;
}

int hough_autotune(hough_ctx *ctx, const hough_hits *hits, const int64_t *window_offsets,
                   int64_t n_windows, const hough_tracks *tracks_out, void *stream, int iters,
                   hough_launch *best)
{
    int rc = check_find_args(ctx, hits, window_offsets, n_windows, tracks_out);
    if (rc != HOUGH_OK || iters < 1)
        return fail(ctx, rc != HOUGH_OK ? rc : HOUGH_ERR_INVALID_ARG);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int *c = counter_for(ctx, s);
    if (!c)
        return fail(ctx, HOUGH_ERR_ALLOC);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(ctx, HOUGH_ERR_CUDA);
    hough_launch chosen = ctx->launch;
    float best_ms = 1e30f;
    for (int threads : {256, 512, 1024})
        for (int wr : {32, 64, 128})
            for (int cps : {1, 2, 3, 4})
                for (int hs : {1024, 2048}) {
                    hough_launch req{threads, wr, hs, cps};
                    hough_launch l{};
                    size_t smem = 0;
                    if (resolve_launch(ctx, req, l, smem) != HOUGH_OK)
                        continue;
                    if (cps > 1 && smem * cps > ctx->smem_optin)
                        continue;
                    if (launch_find(ctx, hits, window_offsets, n_windows, tracks_out, s, c, l) !=
                        HOUGH_OK) {
                        cudaGetLastError();
                        continue;
                    }
                    cudaEventRecord(e0, s);
                    for (int i = 0; i < iters; ++i)
                        launch_find(ctx, hits, window_offsets, n_windows, tracks_out, s, c, l);
                    cudaEventRecord(e1, s);
                    if (cudaEventSynchronize(e1) != cudaSuccess) {
                        cudaEventDestroy(e0);
                        cudaEventDestroy(e1);
                        return fail(ctx, HOUGH_ERR_CUDA);
                    }
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < best_ms) {
                        best_ms = ms;
                        chosen = l;
                    }
                }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->launch = chosen;
    ctx->auto_launch = false;
    // leave the outputs holding the chosen shape's (identical) results
    rc = launch_find(ctx, hits, window_offsets, n_windows, tracks_out, s, c, chosen);
    if (best)
        *best = chosen;
    return fail(ctx, rc);
}

const char *hough_status_string(int status)
{
    switch (status) {
    case HOUGH_OK: return "HOUGH_OK";
    case HOUGH_ERR_INVALID_ARG: return "HOUGH_ERR_INVALID_ARG";
    case HOUGH_ERR_ALLOC: return "HOUGH_ERR_ALLOC";
    case HOUGH_ERR_CUDA: return "HOUGH_ERR_CUDA";
    case HOUGH_ERR_TIMEOUT: return "HOUGH_ERR_TIMEOUT";
    case HOUGH_ERR_UNSUPPORTED_SHAPE: return "HOUGH_ERR_UNSUPPORTED_SHAPE";
    case HOUGH_ERR_NO_DEVICE: return "HOUGH_ERR_NO_DEVICE";
    default: return "HOUGH_ERR_UNKNOWN";
    }
}

int hough_last_error(const hough_ctx *ctx) { return ctx ? ctx->last_error : HOUGH_ERR_INVALID_ARG; }

int64_t hough_launch_count(const hough_ctx *ctx) { return ctx ? (int64_t)ctx->launches : 0; }

}  // extern "C"
