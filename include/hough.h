/*
 * hough.h -- C ABI of the GB300 track-finding library (libhough).
 *
 * The library runs the data-parallel hot path of the J-PARC muon g-2/EDM
 * positron track-finder (arXiv 2511.02742) on one GPU: per time window,
 *   A. encode strip-level hits to fixed-point (phi, z)        (Section 2, Section 5)
 *   B. Hough voting rho = phi cos(theta) + z sin(theta)      (Section 4, Eq. (1))
 *      into an n_theta x n_rho accumulator over theta in [0, 180) degrees
 *      and rho in [rho_min, rho_max)                          (Section 5 binning)
 *   C. peak extraction                                       (Section 4, Section 5)
 *   D. association of the hits that lie on each peak's line  (Section 5 seeds)
 * All arithmetic is integer, so results are bit-exact and deterministic.
 *
 * Conventions
 *   - Every call returns HOUGH_OK (0) or a negative hough_status; nothing
 *     aborts.  Arguments the host can check are checked before any launch.
 *   - Pointers documented "device" must point to memory of the context's
 *     device; "host" pointers to host memory (pinned memory lets copies
 *     overlap with compute).  The caller owns every buffer it passes in; the
 *     library owns only what it allocates itself and frees it in
 *     hough_destroy / hough_plan_destroy.
 *   - Device work is asynchronous on the given stream (a cudaStream_t passed
 *     as void*; NULL = legacy default stream).  Per-window conditions found on
 *     the device are reported in tracks_out->window_status, not as return codes.
 *   - A context may be used from one host thread at a time.
 */
#ifndef HOUGH_H
#define HOUGH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Largest scale exponent of the fixed-point cos/sin tables (see hough_tables). */
#define HOUGH_MAX_FRAC_BITS 24

/* Largest accumulator sides and peak list the kernels accept. */
#define HOUGH_MAX_THETA 4096
#define HOUGH_MAX_RHO 1024
#define HOUGH_MAX_PEAKS 256

typedef enum hough_status {
    HOUGH_OK = 0,
    HOUGH_ERR_INVALID_ARG = -1,       /* NULL pointer, negative size, bad field   */
    HOUGH_ERR_ALLOC = -2,             /* device or host allocation failed         */
    HOUGH_ERR_CUDA = -3,              /* a CUDA runtime call failed               */
    HOUGH_ERR_TIMEOUT = -4,           /* a bounded device wait gave up            */
    HOUGH_ERR_UNSUPPORTED_SHAPE = -5, /* n_theta / n_rho / max_peaks out of range */
    HOUGH_ERR_NO_DEVICE = -6,         /* no usable CUDA device                    */
    HOUGH_ERR_BUSY = -7               /* a server's queue is full; retry later    */
} hough_status;

/* Per-window flags, OR-ed into tracks_out->window_status[w]. */
#define HOUGH_WIN_PEAK_OVERFLOW 1u     /* more peaks found than max_peaks; best kept     */
#define HOUGH_WIN_HIT_OUT_OF_RANGE 2u  /* a hit lies outside the detector box; ignored   */
#define HOUGH_WIN_VOTE_OUT_OF_RANGE 4u /* a valid hit's vote fell outside [0, n_rho)    */
#define HOUGH_WIN_BAD_OFFSETS 8u       /* offsets not ordered or beyond n_hits; skipped  */
#define HOUGH_WIN_TOO_LARGE 16u        /* more valid hits than the entry point stages    */

/* hough_thresholds.flags */
#define HOUGH_FLAG_EXPORT_ACC 1u /* write the full int32 accumulator (tracks_out->acc) */
/*
 * FP64 variant of the find (hough_find and its host, plan and server forms):
 * each hit's bin in a theta row comes from Eq. (1) in double precision with
 * the Section 5 binning instead of the fixed-point tables,
 *   b = floor(((phi/phi_u_per_deg) cos(theta_t) + (z/z_u_per_mm) sin(theta_t)
 *              - rho_min) / ((rho_max - rho_min) / n_rho)),
 * every operation rounded to nearest in that order (no fused multiply-add),
 * cos and sin computed on the host in double.  Everything else (peaks,
 * association, outputs) is unchanged.  It exists to check that the
 * fixed-point result agrees with the continuous one within one bin; it is
 * slower.  Not accepted by hough_find_noalloc.
 */
#define HOUGH_FLAG_FP64 2u

/*
 * Detector geometry and fixed-point units (Section 2).  Defaults for the
 * J-PARC detector: n_vanes = 40 radial vanes, n_z_strips = 2048 z strips per
 * vane at z_pitch_u = 38 units (0.19 mm) starting at z_min_u = -38912
 * (-194.56 mm), phi_u_per_deg = z_u_per_mm = 200 (1 unit = 1/200 degree or
 * 1/200 mm), rho range [-500, 500) (Section 5).
 * A hit is inside the detector box when 0 <= phi < 360 deg and
 * z_min <= z <= z_min + n_z_strips * z_pitch (in units).
 */
typedef struct hough_geometry {
    int32_t n_vanes;
    int32_t n_z_strips;
    int32_t z_pitch_u;
    int32_t z_min_u;
    int32_t phi_u_per_deg;
    int32_t z_u_per_mm;
    double rho_min;
    double rho_max;
} hough_geometry;

/*
 * Peak and association parameters (Section 4, Section 5).
 *   vote_threshold >= 1: a peak needs at least this many votes;
 *   assoc_tol_bins >= 0: a hit lies on a peak's line when its rho bin in the
 *                        peak's theta row is within this many bins;
 *   max_peaks in [0, HOUGH_MAX_PEAKS]: peaks kept per window;
 *   flags: HOUGH_FLAG_*.
 */
typedef struct hough_thresholds {
    int32_t vote_threshold;
    int32_t assoc_tol_bins;
    int32_t max_peaks;
    uint32_t flags;
} hough_thresholds;

/* One peak: theta row, rho bin, its vote count, and the slice of track_hits
 * (window-local, starting at hit_begin, n_hits long) holding its hits. */
typedef struct hough_peak {
    uint16_t theta;
    uint16_t rho;
    int32_t votes;
    int32_t n_hits;
    int32_t hit_begin;
} hough_peak;

/*
 * Hits in structure-of-arrays form, device pointers, n_hits long.  Give
 * either the encoded pair (phi_q, z_q) or the strip addresses (vane, strip);
 * when vane and strip are both non-NULL they are used and encoded on the fly
 * (phi = vane * 360/n_vanes deg, z = centre of the strip), else phi_q and z_q.
 */
typedef struct hough_hits {
    const int32_t *phi_q;
    const int32_t *z_q;
    const int32_t *vane;
    const int32_t *strip;
    int64_t n_hits;
} hough_hits;

/*
 * Outputs, caller-owned device buffers.  For n_windows windows and n_hits hits:
 *   peaks[n_windows * max_peaks]  window w's peaks at [w*max_peaks, ...+n_peaks[w]),
 *                                 sorted by votes desc, theta asc, rho asc;
 *   n_peaks[n_windows]            peaks kept;
 *   n_found[n_windows]            peaks found before truncation (may be NULL);
 *   hit_track[n_hits]             per hit: window-local peak index, -1 if on
 *                                 no peak's line, -2 if outside the detector box;
 *   track_hits[n_hits]            per window, a permutation of the window-local
 *                                 hit indices: the hits of peak 0 in increasing
 *                                 order, then peak 1, ..., then the -1 hits, then
 *                                 the -2 hits;
 *   window_status[n_windows]      HOUGH_WIN_* flags;
 *   acc                           with HOUGH_FLAG_EXPORT_ACC, int32
 *                                 [n_windows][n_theta][n_rho]; else ignored.
 * Entries past n_peaks[w] are not written.
 */
typedef struct hough_tracks {
    hough_peak *peaks;
    int32_t *n_peaks;
    int32_t *n_found;
    int32_t *hit_track;
    int32_t *track_hits;
    uint32_t *window_status;
    int32_t *acc;
} hough_tracks;

/*
 * Launch shape of the find kernel; 0 in a field means "library default".
 * All fields 0: the first shape that fits of 3 CTAs of 256 threads per SM,
 * 2 of 512 and 1 of 1024, with 32-word-row tiles (else one CTA of 512
 * threads with the largest tile that fits); when that is 3 CTAs of 256
 * threads, a batch of more than 250 hits per window on average runs in 2
 * CTAs of 512 instead (its candidate lists need the larger CTAs' shared
 * memory).  hough_get_launch returns the first choice.
 */
typedef struct hough_launch {
    int32_t threads;      /* threads per CTA: 256, 512 or 1024                     */
    int32_t word_rows;    /* word rows of the shared accumulator tile: 32, 64 or 128   */
    int32_t hit_stage;    /* hits held in shared memory per stage (multiple of 256)  */
    int32_t ctas_per_sm;  /* resident CTAs per SM (1..4); capped by occupancy       */
} hough_launch;

typedef struct hough_ctx hough_ctx;
typedef struct hough_plan hough_plan;

/*
 * Fixed-point tables of Eq. (1) with the Section 5 binning, host only (no GPU).
 * theta_t = (t + 1/2) * 180/n_theta degrees; with span = rho_max - rho_min,
 *   C[t] = round(cos(theta_t) * 2^K * n_rho / (span * phi_u_per_deg))
 *   S[t] = round(sin(theta_t) * 2^K * n_rho / (span * z_u_per_mm))
 *   D    = round(-rho_min * 2^K * n_rho / span)
 * rounding half away from zero (computed in double precision), where K is
 * the largest value <= HOUGH_MAX_FRAC_BITS for which |phi*C[t] + z*S[t] + D|
 * < 2^31 at the four corners of the detector box for every t (so the sum is
 * a 32-bit integer for every hit of the box).  A valid hit (phi, z) votes in
 * row t for the bin b = floor((phi*C[t] + z*S[t] + D) / 2^K) if 0 <= b < n_rho.
 * C and S are host arrays of n_theta entries; *D and *K receive the offset
 * and the exponent.  Errors: INVALID_ARG, UNSUPPORTED_SHAPE (no K >= 8 fits).
 */
int hough_tables(const hough_geometry *g, int n_theta, int n_rho, int32_t *C, int32_t *S,
                 int64_t *D, int32_t *K);

/*
 * The find's narrowed tiles, host only (no GPU).  The bin of Eq. (1) is
 * monotone in phi and in z, so in each theta row the bins a hit of the
 * detector box can reach lie between those of the box's four corners.  A
 * find tile with word_rows (32, 64 or 128) word rows and 2^k counters per
 * word (k = 0, 1, 2: 32-, 16-, 8-bit counters) covers theta rows
 * [i R, (i + 1) R), R = word_rows << k, and stores only the bins
 * [lo, lo + *nb) of each row: *nb is the widest range of reachable bins
 * inside [0, n_rho) over every such tile, plus 3, rounded up to a multiple
 * of 4 (at most n_rho), and lo = min(max(lowest reachable bin of the tile,
 * 0), n_rho - *nb) rounded down to a multiple of 4.  lo[k * T + i] (caller's
 * array of 3 T entries, T = ceil(n_theta / 32); entries past a width's last
 * tile are 0) receives tile i's first bin for counter width 2^k.  Contexts
 * use these for the fixed-point find (not for HOUGH_FLAG_FP64 or
 * hough_find_noalloc, whose tiles store every bin).
 * Errors: INVALID_ARG (null pointer, bad geometry or word_rows),
 * UNSUPPORTED_SHAPE (as hough_create).
 */
int hough_tile_bins(const hough_geometry *g, int n_theta, int n_rho, int word_rows, int32_t *nb,
                    int32_t *lo);

/*
 * Create a context on the current CUDA device for one accumulator shape
 * (Section 5: 180 x 1000 in the paper; any 1 <= n_theta <= HOUGH_MAX_THETA,
 * 4 <= n_rho <= HOUGH_MAX_RHO with n_rho % 4 == 0).  Copies g and th, builds
 * the tables on the device.  *out receives the context; release it with
 * hough_destroy.  Errors: INVALID_ARG, UNSUPPORTED_SHAPE, NO_DEVICE, ALLOC, CUDA.
 */
int hough_create(const hough_geometry *g, int n_theta, int n_rho, const hough_thresholds *th,
                 hough_ctx **out);

/* Release a context and everything it allocated.  NULL is a no-op.  The caller
 * must make sure no work using the context is still running. */
void hough_destroy(hough_ctx *ctx);

/*
 * Step A alone (Section 2 geometry, Section 5 phi = atan(y/x)): device arrays
 * vane[n], strip[n] -> phi_q[n], z_q[n] (device).  Addresses outside the
 * detector give values the find step rejects.  Asynchronous on stream.
 */
int hough_encode(hough_ctx *ctx, const int32_t *vane, const int32_t *strip, int64_t n,
                 int32_t *phi_q, int32_t *z_q, void *stream);

/*
 * Steps B-D for n_windows windows (Section 4, Section 5; one window per
 * independent unit of work as in Section 6).  window_offsets is a device
 * array of n_windows + 1 int64: window w owns hits [offsets[w], offsets[w+1]).
 * Offsets must be non-decreasing within [0, hits->n_hits]; a window whose own
 * pair is decreasing or out of range gets HOUGH_WIN_BAD_OFFSETS and no output
 * (no memory outside [0, n_hits) is touched).  Windows must not overlap: two
 * windows sharing a hit write the same hit_track/track_hits slots.
 * Asynchronous on stream; results are identical for every launch shape,
 * stream and batch.
 * Errors: INVALID_ARG (bad pointers/sizes), CUDA (launch failed).
 */
int hough_find(hough_ctx *ctx, const hough_hits *hits, const int64_t *window_offsets,
               int64_t n_windows, const hough_tracks *tracks_out, void *stream);

/*
 * The paper's own two-stage GPU search, one line per window (Section 6 and
 * its figure of the Hough steps: a coarse histogram of 18 theta x 100 rho
 * bins, then a 10 x 10 fine histogram around its high-likelihood zone, the
 * fine maximum giving the line; seeds are the hits on that line).  Reading:
 * coarse bins of 10 degrees x 10 rho units over the same ranges as the full
 * histogram; the coarse bin with the most entries (ties: first in row-major
 * order); the fine histogram is the 10 x 10 block of the paper's 180 x 1000
 * grid (Section 5: 1 degree x 1 unit) inside that coarse bin: fine row
 * 10*coarse_theta + i, fine rho bin 10*coarse_rho + j; its highest bin (ties
 * row-major) is the line, kept if both maxima reach vote_threshold.  Seeds:
 * the valid hits whose bin in the line's fine row is within assoc_tol_bins
 * of the line's bin.  Same fixed-point arithmetic as hough_find, with the
 * 18 x 100 and 180 x 1000 tables of hough_tables.
 *   lines[n_windows]     device, one result per window;
 *   hit_track[n_hits]    device, 0 for a seed, -1 for a hit off the line (or
 *                        a window without one), -2 outside the detector box.
 * Hits and offsets as hough_find.  Asynchronous on stream.
 * Errors: INVALID_ARG, CUDA.
 */
typedef struct hough_line {
    int32_t coarse_theta;   /* 0..17   */
    int32_t coarse_rho;     /* 0..99   */
    int32_t coarse_votes;
    int32_t fine_theta;     /* 0..179, row of the 180 x 1000 grid */
    int32_t fine_rho;       /* 0..999  */
    int32_t fine_votes;
    int32_t n_seeds;
    int32_t found;          /* 1 if the window has a line */
} hough_line;
int hough_find_coarse_fine(hough_ctx *ctx, const hough_hits *hits, const int64_t *window_offsets,
                           int64_t n_windows, hough_line *lines, int32_t *hit_track,
                           void *stream);

/*
 * Steps A-B with the histograms written out: for every window, the full
 * n_theta x n_rho accumulator of Eq. (1) with the Section 5 binning (each
 * valid hit votes once in each theta row), exactly the accumulator that
 * hough_find writes with HOUGH_FLAG_EXPORT_ACC, without steps C-D.
 *   acc[n_windows * n_theta * n_rho]  device int32, row-major per window;
 *                                     any 4-byte alignment (16-byte aligned
 *                                     is written with 16-byte stores);
 *   window_status[n_windows]          device, HOUGH_WIN_HIT_OUT_OF_RANGE,
 *                                     HOUGH_WIN_VOTE_OUT_OF_RANGE, or
 *                                     HOUGH_WIN_BAD_OFFSETS (that window's
 *                                     accumulator is not written).
 * Hits and offsets as hough_find; fixed-point contexts only (an FP64
 * context gives INVALID_ARG).  Both buffers are the caller's.  Asynchronous
 * on stream.
 * Errors: INVALID_ARG, UNSUPPORTED_SHAPE, CUDA.
 */
int hough_accumulate(hough_ctx *ctx, const hough_hits *hits, const int64_t *window_offsets,
                     int64_t n_windows, int32_t *acc, uint32_t *window_status, void *stream);

/*
 * Iterative highest-bin search (the literal reading of the paper's peak step,
 * Section 4: the bin with the highest accumulation is the most probable
 * line, Section 5: its seeds are the hits aligned with it; repeated until no
 * line is left).  Per window: vote the hits not yet assigned into the full
 * n_theta x n_rho accumulator, take its highest bin (ties: first in
 * row-major order), stop if it holds fewer than vote_threshold votes, else
 * give track k every remaining hit whose bin in that row is within
 * assoc_tol_bins of it, remove them and vote again; at most max_tracks
 * tracks (1..HOUGH_MAX_PEAKS).  Same fixed-point arithmetic as hough_find.
 *   tracks[n_windows * max_tracks]  device, per track (theta, rho, votes,
 *                                   n_hits);
 *   n_tracks[n_windows]             device, tracks found;
 *   hit_track[n_hits]               device, track index, -1 if none, -2
 *                                   outside the detector box;
 *   window_status[n_windows]        device, HOUGH_WIN_* flags; a window with
 *                                   more than HOUGH_ITER_MAX_HITS valid hits
 *                                   gets HOUGH_WIN_TOO_LARGE and no track.
 * Hits and offsets as hough_find.  Asynchronous on stream.
 * Errors: INVALID_ARG, UNSUPPORTED_SHAPE, CUDA.
 */
#define HOUGH_ITER_MAX_HITS 4096
typedef struct hough_iter_track {
    int32_t theta;
    int32_t rho;
    int32_t votes;
    int32_t n_hits;
} hough_iter_track;
int hough_find_iterative(hough_ctx *ctx, const hough_hits *hits, const int64_t *window_offsets,
                         int64_t n_windows, int32_t max_tracks, hough_iter_track *tracks,
                         int32_t *n_tracks, int32_t *hit_track, uint32_t *window_status,
                         void *stream);

/*
 * Track extension (Section 4: three RecoHits on consecutive vanes form a
 * seed, whose trajectory is extrapolated to neighbouring vanes forward and
 * backward, within the time window), run on the output of hough_find for the
 * same hits and windows.
 *
 * A hit takes part when hough_find did not reject it (hit_track != -2) and it
 * lies on a vane: phi = k * vane step with 0 <= k < n_vanes (always so for
 * strip addresses).  Vanes are neighbours modulo n_vanes.  The peaks of a
 * window are taken in their order; a hit claimed by a track is not available
 * to a later one.  For peak p:
 *   seed: among the unclaimed hits a, b, c of the peak's group (track_hits)
 *     on vanes k - 1, k, k + 1 with bend |z_a - 2 z_b + z_c| <= tol_z, the
 *     one with the smallest (bend, b, a, c), comparing window-local indices;
 *     none: the peak gives no track;
 *   forward: the parabola through the last three hits predicts
 *     z = 3 z_2 - 3 z_1 + z_0 on the next vane; the unclaimed hit of the
 *     window on that vane nearest to it within tol_z is taken (ties: the
 *     lower z, then the lower index); stop when there is none;
 *   backward: the same from the seed's first hit to lower vanes;
 *   a track holds at most n_vanes hits, one per vane.
 * All integer, so the result is exact.
 *
 * Arguments (device buffers, caller-owned; window-local indices):
 *   found          hough_find's outputs for these hits and windows: peaks,
 *                  n_peaks, hit_track and track_hits are read;
 *   tol_z          0..HOUGH_EXT_MAX_TOL, in z units (1/z_u_per_mm mm);
 *   out->tracks    [n_windows * max_peaks]: entry p of window w describes
 *                  peak p (p < n_peaks[w]): first_vane (vane of the track's
 *                  first hit in increasing-vane order, -1 none), n_hits,
 *                  hit_begin (offset in ext_hits), seed_mid (the seed's middle
 *                  hit, -1 none);
 *   out->ext_track [n_hits]: track holding the hit, -1 none;
 *   out->ext_hits  [n_hits]: per window, the hits of track 0 in increasing
 *                  vane order from its first vane, then track 1's, ..., then
 *                  every unclaimed hit in increasing index;
 *   out->window_status [n_windows]: 0, or HOUGH_WIN_TOO_LARGE for a window of
 *                  more than HOUGH_EXT_MAX_HITS hits (no track, nothing
 *                  claimed, ext_hits in index order), or HOUGH_WIN_BAD_OFFSETS
 *                  when the window's offsets are out of order or beyond
 *                  n_hits (its outputs are not written).
 * Asynchronous on stream; three launches.  Errors: INVALID_ARG (NULL
 * pointer, tol_z out of range), UNSUPPORTED_SHAPE (n_vanes outside
 * 3..HOUGH_EXT_MAX_VANES), CUDA.
 */
#define HOUGH_EXT_MAX_HITS 4096
#define HOUGH_EXT_MAX_VANES 256
#define HOUGH_EXT_MAX_TOL ((1 << 19) - 1)
typedef struct hough_ext_track {
    int32_t first_vane;
    int32_t n_hits;
    int32_t hit_begin;
    int32_t seed_mid;
} hough_ext_track;
typedef struct hough_extension {
    hough_ext_track *tracks;
    int32_t *ext_track;
    int32_t *ext_hits;
    uint32_t *window_status;
} hough_extension;
int hough_extend(hough_ctx *ctx, const hough_hits *hits, const int64_t *window_offsets,
                 int64_t n_windows, const hough_tracks *found, int32_t tol_z,
                 hough_extension *out, void *stream);

/*
 * Time slicing on the device (Section 5: the hits of a readout are divided
 * into overlapping time windows of 10 ns with a sliding step of 5 ns;
 * Section 6: each window is one unit of work).  Window k, 0 <= k < n_windows,
 * holds every hit h with
 *     t0 + k*step <= t[h] < t0 + k*step + len,
 * in input order; a hit appears once in every window that covers its time.
 *   t[n_hits]          device, int64 times (any unit), non-decreasing (a
 *                      readout in time order);
 *   in0/in1[n_hits]    device, the hits' (vane, strip) or (phi_q, z_q);
 *   len                a multiple of step, at most HOUGH_SLICE_MAX_OVERLAP
 *                      steps (the paper's windows are two steps long).
 * Writes on the device, window by window:
 *   window_offsets[n_windows + 1]   CSR offsets into the outputs;
 *   out0/out1[...]                  in0/in1 of each window's hits;
 *   out_index[...]                  the hits' input positions (may be NULL).
 * out_capacity (entries of out0/out1/out_index) must be at least
 * n_hits * (len / step), the most any input can need.  The result feeds
 * hough_find as it is: hits (out0, out1) with n_hits = out_capacity, the same
 * window_offsets and n_windows.  *status (device, may be NULL) is cleared and
 * then receives HOUGH_SLICE_UNSORTED if t decreases anywhere (the outputs are
 * then unspecified, but nothing outside the given arrays is touched).
 * Asynchronous on stream.
 * Errors: INVALID_ARG, UNSUPPORTED_SHAPE (len not a multiple of step or
 * longer than HOUGH_SLICE_MAX_OVERLAP steps), CUDA.
 */
#define HOUGH_SLICE_MAX_OVERLAP 16
#define HOUGH_SLICE_UNSORTED 1u
int hough_time_slice(hough_ctx *ctx, const int64_t *t, const int32_t *in0, const int32_t *in1,
                     int64_t n_hits, int64_t t0, int64_t step, int64_t len, int64_t n_windows,
                     int32_t *out0, int32_t *out1, int64_t *out_index, int64_t out_capacity,
                     int64_t *window_offsets, uint32_t *status, void *stream);

/*
 * hough_find on HOST buffers: the same arguments, but every pointer in hits,
 * window_offsets and tracks_out is a host pointer.  The library copies inputs
 * to device staging buffers it owns, runs the path, copies the results back
 * and synchronises before returning (the end-to-end form).  Work is split
 * into chunks of windows so that copies overlap compute.
 */
int hough_find_host(hough_ctx *ctx, const hough_hits *hits, const int64_t *window_offsets,
                    int64_t n_windows, const hough_tracks *tracks_out, void *stream);

/*
 * A plan is hough_find (optionally preceded by nothing else) captured once
 * into a CUDA graph bound to these exact device buffers: one persistent
 * kernel over all windows.  hough_plan_launch replays it on any stream.
 * The buffers must stay valid while the plan exists.  Errors as hough_find.
 */
int hough_plan_create(hough_ctx *ctx, const hough_hits *hits, const int64_t *window_offsets,
                      int64_t n_windows, const hough_tracks *tracks_out, void *stream,
                      hough_plan **out);
int hough_plan_launch(hough_plan *plan, void *stream);
void hough_plan_destroy(hough_plan *plan);

/* Read or set the launch shape used by later calls (0 fields = defaults). */
int hough_get_launch(const hough_ctx *ctx, hough_launch *out);
int hough_set_launch(hough_ctx *ctx, const hough_launch *cfg);

/*
 * Time every supported launch shape on this batch (iters runs each, CUDA
 * events on stream), keep the fastest in the context and return it in *best
 * (may be NULL).  Outputs are overwritten with the (identical) results.
 */
int hough_autotune(hough_ctx *ctx, const hough_hits *hits, const int64_t *window_offsets,
                   int64_t n_windows, const hough_tracks *tracks_out, void *stream, int iters,
                   hough_launch *best);

/*
 * hough_find without any allocation (no counterpart in the paper: it serves
 * callers, not the method).  Some callers cannot call cudaMalloc -- code that
 * runs where the device allocator is off limits (a real-time loop that must
 * not block in the allocator, a process whose device memory is handed out by
 * its host framework, a sandbox without allocation rights) -- and so cannot
 * create a context.  This entry point takes the context's arguments directly
 * and does the work of hough_find with no cudaMalloc, cudaFree or other
 * allocating call: the small global memory the kernel needs beyond the
 * caller's buffers (the scheduling counters and the cos/sin tables) lives in
 * a file-scope device array of fixed size, HOUGH_NOALLOC_SCRATCH_BYTES,
 * which every GPU that loads the library holds until the process exits.
 *   - n_theta may be at most HOUGH_NOALLOC_MAX_THETA; larger shapes get
 *     HOUGH_ERR_UNSUPPORTED_SHAPE.  Other arguments as hough_find (device
 *     pointers), with the default launch shape.
 *   - The first call on a device, with that device current, looks up the
 *     array's device address (set-up); make that first call before any stream
 *     capture.
 *   - Every call on a device shares the array and leaves its contents behind:
 *     the call clears the counters and copies the tables, computed on the
 *     host into static host buffers, on its stream before the kernel runs.
 *     Calls whose work overlaps on the GPU (other streams, other host
 *     threads) race on the array: serialise them.
 *   - Because each call copies its tables from (pageable) host memory, a
 *     stream that is capturing a graph is refused with INVALID_ARG before
 *     anything is enqueued, and the capture is left as it was.
 * Errors: INVALID_ARG, UNSUPPORTED_SHAPE, NO_DEVICE, CUDA.
 */
#define HOUGH_NOALLOC_MAX_THETA 4096
#define HOUGH_NOALLOC_MAX_DEVICES 64
#define HOUGH_NOALLOC_SCRATCH_BYTES (256 + 8 * HOUGH_NOALLOC_MAX_THETA)
int hough_find_noalloc(const hough_geometry *g, int n_theta, int n_rho,
                       const hough_thresholds *th, const hough_hits *hits,
                       const int64_t *window_offsets, int64_t n_windows,
                       const hough_tracks *tracks_out, void *stream);

/* ------------------------------------------------------------------ serving
 *
 * A request loop over one context (no counterpart in the paper, which
 * processes the windows of a recorded sample; Section 6 makes each window an
 * independent unit of work, which is what lets windows from different
 * requests share a launch).  A request is one detector time slice: a CSR
 * batch of windows in HOST memory.  A worker thread owned by the server
 *   - admits queued requests, oldest first, into a free batch slot while the
 *     slot's device memory has room for their windows and hits (admission by
 *     memory: a slot holds at most slot_windows windows and slot_hits hits);
 *   - runs each slot on its own stream: the batch's window offsets (rebased
 *     to the batch) and each request's hits are copied in, the find kernel
 *     runs once over the batch, and each request's results are copied
 *     straight into its host buffers; the request then completes.
 * With n_slots > 1, requests that arrive while earlier batches are on the
 * GPU go into the next free slot at once (continuous batching), so their
 * copies and kernels overlap with the running ones.  Device buffers and
 * pinned staging are allocated once, in hough_server_create, and stay
 * resident.  Each window's results are the same bits as hough_find gives it
 * alone: windows never interact.
 *
 * While a server exists it owns its context: make no other call on that
 * context (hough_find, hough_set_launch, ...) until hough_server_destroy.
 * Server calls may be made from any host thread.  While batches are on the
 * GPU the worker polls their completion events (yielding between polls), so
 * it keeps one host core busy; when nothing is queued or running it polls the
 * queue for 2 ms more (a sleeping thread takes tens of microseconds to wake)
 * and then sleeps.
 */
typedef struct hough_server hough_server;

typedef struct hough_server_config {
    int32_t n_slots;       /* batches in flight at once, 1..16                          */
    int32_t raw_hits;      /* 1: requests carry (vane, strip); 0: encoded (phi_q, z_q)   */
    int64_t slot_windows;  /* windows one batch can hold (>= 1)                         */
    int64_t slot_hits;     /* hits one batch can hold (>= 1)                            */
    int64_t max_queued;    /* requests waiting for a slot before submit says BUSY (>= 1) */
    hough_launch launch;   /* launch shape of the server's batches; all 0: chosen per
                              batch, one CTA of 1024 threads per SM with 32-word-row
                              tiles for batches of fewer than 2 windows per SM (the
                              lowest latency), the context's shape when the server is
                              created for larger ones (the library default, or what
                              hough_set_launch or hough_autotune on representative
                              windows chose: the highest throughput); the context's
                              own shape is restored by hough_server_destroy */
} hough_server_config;

/*
 * One time slice.  in0/in1 are vane/strip (raw_hits) or phi_q/z_q, host
 * arrays of n_hits = window_offsets[n_windows] entries; window_offsets is a
 * host array of n_windows + 1 int64 starting at 0 and non-decreasing.  out
 * holds HOST buffers laid out as for hough_find (peaks[n_windows*max_peaks],
 * n_peaks, n_found (may be NULL), hit_track[n_hits], track_hits[n_hits],
 * window_status; acc is not supported).  The copies go straight between these
 * buffers and the device, so they should be page-locked (cudaHostAlloc or
 * cudaHostRegister): pageable buffers work, but the driver then stages each
 * copy and the worker waits on it.  Unlike hough_find, the whole
 * peaks[n_windows*max_peaks] array is written (entries past n_peaks[w] hold
 * unspecified values).  Every buffer must stay valid and untouched until the
 * request completes.  arrival_ns: when the slice arrived,
 * on the hough_server_clock_ns clock (0 = at submit); latencies are measured
 * from it.
 */
typedef struct hough_request {
    const int32_t *in0;
    const int32_t *in1;
    const int64_t *window_offsets;
    int64_t n_windows;
    hough_tracks out;
    int64_t arrival_ns;
} hough_request;

typedef struct hough_request_result {
    uint64_t ticket;
    int32_t status;          /* HOUGH_OK, or the error that ended the request    */
    int32_t batch_requests;  /* requests that shared its launch                  */
    int64_t batch_windows;   /* windows in that launch                           */
    int64_t arrival_ns;      /* as submitted (or the submit time)                */
    int64_t launch_ns;       /* when its batch was handed to the GPU             */
    int64_t done_ns;         /* when its results were in its host buffers        */
    /* where its batch's time went (the batch's figures, shared by its
     * requests): packing into the slot's pinned staging (host clock), copy
     * in, the find and copy out (CUDA events on the slot's stream), and the
     * scatter of the results into the requests' buffers (host clock) */
    int64_t pack_ns, h2d_ns, kernel_ns, d2h_ns, scatter_ns;
} hough_request_result;

typedef struct hough_server_stats {
    int64_t submitted;       /* accepted requests                                */
    int64_t rejected;        /* submits answered BUSY or refused as too large    */
    int64_t completed;
    int64_t queued;          /* accepted, waiting for a slot                      */
    int64_t in_flight;       /* requests in batches on the GPU                   */
    int64_t batches;         /* launches so far                                  */
    int64_t windows;         /* windows completed                                */
    int64_t device_bytes;    /* device memory held by the slots                  */
    int64_t host_bytes;      /* pinned host staging held by the slots            */
} hough_server_stats;

/*
 * Create a server over ctx (current device = ctx's device).  Allocates every
 * slot's stream, device buffers and pinned staging, and starts the worker
 * thread.  Errors: INVALID_ARG (bad config, or ctx exports accumulators),
 * ALLOC, CUDA.
 */
int hough_server_create(hough_ctx *ctx, const hough_server_config *cfg, hough_server **out);

/*
 * Queue a request; *ticket identifies it.  Checks the request on the host
 * (pointers, offsets) and its size against one slot.  Never blocks on the
 * GPU.  Errors: INVALID_ARG, UNSUPPORTED_SHAPE (more windows or hits than a
 * slot holds), BUSY (max_queued requests already waiting).
 */
int hough_server_submit(hough_server *srv, const hough_request *req, uint64_t *ticket);

/*
 * Wait up to timeout_ms (< 0: no limit) for one ticket and take its result
 * (each result is delivered once, by wait or by poll).  Errors: INVALID_ARG
 * (unknown or already delivered ticket), TIMEOUT.
 */
int hough_server_wait(hough_server *srv, uint64_t ticket, int64_t timeout_ms,
                      hough_request_result *res);

/* Take up to cap completed results, oldest completion first; *n receives
 * how many were written.  Never blocks. */
int hough_server_poll(hough_server *srv, hough_request_result *res, int64_t cap, int64_t *n);

/* Wait up to timeout_ms (< 0: no limit) until nothing is queued or in
 * flight.  Errors: TIMEOUT. */
int hough_server_drain(hough_server *srv, int64_t timeout_ms);

int hough_server_get_stats(hough_server *srv, hough_server_stats *out);

/* Finish every accepted request, stop the worker and free the slots.  NULL
 * is a no-op.  The context stays valid. */
void hough_server_destroy(hough_server *srv);

/* The server's clock (monotonic, nanoseconds), for arrival_ns. */
int64_t hough_server_clock_ns(void);

/* Human-readable name of a hough_status value. */
const char *hough_status_string(int status);

/* The status of the last failing call on ctx (HOUGH_OK if none). */
int hough_last_error(const hough_ctx *ctx);

/* Number of kernel launches the library issued on ctx (for accounting). */
int64_t hough_launch_count(const hough_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* HOUGH_H */
