/*
 * hough_oracle.c -- plain, slow, single-threaded CPU oracle for the
 * track-finding hot path (Hough voting -> peak extraction -> association).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or constant generator
 * with the CUDA library: every step below is written out independently from
 * the paper's definitions, in the most direct form (full int32 accumulator,
 * double loops, explicit floor division, qsort).
 *
 * What it computes, per time window (Section 4 Eq. (1); Section 5):
 *   A. encoding: a RecoHit on vane k, z-strip j has phi = 9 deg * k (radial
 *      vanes, Section 2) and z at the centre of strip j, both in fixed-point
 *      units of 1/200 degree and 1/200 mm;
 *   B. Hough voting: every hit votes once in each theta row t for the rho bin
 *      b = floor((phi*C[t] + z*S[t] + D) / 2^K); votes outside [0, n_rho)
 *      are dropped and counted (Section 4 Eq. (1); Section 5 binning); the
 *      scale 2^K is the largest (K <= 24) that keeps phi*C + z*S + D within
 *      32-bit signed range for every hit of the detector box;
 *   C. peaks: every bin with count >= T that is a 3x3 local maximum under the
 *      row-major tie-break, sorted by (votes desc, theta asc, rho asc), the
 *      first max_peaks kept (Section 4 and Section 5, "the bin with the highest
 *      number of entries", generalised to pileup);
 *   D. association: each hit goes to the first peak in that order whose line
 *      it lies on within the tolerance, |b_h(t_p) - b_p| <= tol (Section 5,
 *      seed hits "that align with the straight line"); then the hits are
 *      grouped per peak.
 * and, before all of these, the time slicing of a readout into overlapping
 * windows (Section 5: 10 ns windows sliding by 5 ns; oracle_time_slice).
 * Two variants of steps C-D: the paper's coarse-to-fine search for one line
 * (oracle_coarse_fine_*) and the iterative highest-bin search
 * (oracle_iterative_*).
 * Where the paper leaves a point open (units, theta sampling, fixed-point
 * tables, threshold, tie-break, tolerance), the reading taken is stated at
 * the step that uses it.
 *
 * Parity pins: tests/test_oracle_pins.py checks this file against brute force
 * on hand-built cases, the single-line closed form, the helix closed form,
 * the FP64 continuous definition (|b_fixed - b_fp64| <= 1), conservation of
 * votes and permutation invariance; tests/test_slicing_pins.py checks the
 * time slicing against a hand-worked example and the closed-form membership.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAX_FRAC_BITS 24

/* Same field order as the library's geometry struct; declared here on its own. */
typedef struct {
    int32_t n_vanes;
    int32_t n_z_strips;
    int32_t z_pitch_u;
    int32_t z_min_u;
    int32_t phi_u_per_deg;
    int32_t z_u_per_mm;
    double rho_min;
    double rho_max;
} oracle_geometry;

typedef struct {
    int32_t vote_threshold;
    int32_t assoc_tol_bins;
    int32_t max_peaks;
    uint32_t flags;
} oracle_thresholds;

typedef struct {
    uint16_t theta;
    uint16_t rho;
    int32_t votes;
    int32_t n_hits;
    int32_t hit_begin;
} oracle_peak;

enum {
    ORACLE_FLAG_FP64 = 2u, /* thresholds.flags: bins from Eq. (1) in double precision */
};

enum {
    ORACLE_WIN_PEAK_OVERFLOW = 1u,
    ORACLE_WIN_HIT_OUT_OF_RANGE = 2u,
    ORACLE_WIN_VOTE_OUT_OF_RANGE = 4u,
};

/* ---------------------------------------------------------------- helpers */

/* Round half away from zero, on a double. */
static int64_t round_half_away(double x)
{
    if (x >= 0.0)
        return (int64_t)floor(x + 0.5);
    return -(int64_t)floor(-x + 0.5);
}

/* Floor division by a positive divisor, written out with / and %. */
static int64_t floor_div(int64_t num, int64_t den)
{
    int64_t q = num / den;
    int64_t r = num % den;
    if (r != 0 && num < 0)
        q -= 1;
    return q;
}

/* --------------------------------------------------------------- step A/B */

/*
 * Fixed-point cos/sin tables (Section 4 Eq. (1) with the Section 5 binning).
 * theta_t = (t + 1/2) * pi / n_theta (bin centres over 0..180 degrees).
 * One rho bin is (rho_max - rho_min)/n_rho; a hit's rho in bins, measured
 * from rho_min, is (phi/u_phi*cos + z/u_z*sin - rho_min) * n_rho/(rho_max - rho_min).
 * The tables hold those factors scaled by 2^K and rounded half away from zero:
 *   C[t] = round(cos(theta_t) * 2^K * n_rho / ((rho_max - rho_min) * u_phi))
 *   S[t] = round(sin(theta_t) * 2^K * n_rho / ((rho_max - rho_min) * u_z))
 *   D    = round(-rho_min * 2^K * n_rho / (rho_max - rho_min))
 * K is the largest value <= 24 for which |phi*C[t] + z*S[t] + D| < 2^31 at the
 * four corners of the detector box (phi in [0, 360 deg), z in [z_min, z_end])
 * for every t; the sum is linear in (phi, z), so the whole box then fits.
 * Returns K, or -1 on bad arguments or when no K >= 8 fits.
 */
static void tables_at(const oracle_geometry *g, int n_theta, int n_rho, int k, int32_t *C,
                      int32_t *S, int64_t *D)
{
    double two_k = ldexp(1.0, k);
    double span = g->rho_max - g->rho_min;
    double cos_scale = two_k * (double)n_rho / (span * (double)g->phi_u_per_deg);
    double sin_scale = two_k * (double)n_rho / (span * (double)g->z_u_per_mm);
    for (int t = 0; t < n_theta; ++t) {
        double theta = ((double)t + 0.5) * (M_PI / (double)n_theta);
        C[t] = (int32_t)round_half_away(cos(theta) * cos_scale);
        S[t] = (int32_t)round_half_away(sin(theta) * sin_scale);
    }
    *D = round_half_away(-g->rho_min * (two_k * (double)n_rho / span));
}

int oracle_tables(const oracle_geometry *g, int n_theta, int n_rho, int32_t *C, int32_t *S,
                  int64_t *D)
{
    if (!g || n_theta <= 0 || n_rho <= 0 || !(g->rho_max > g->rho_min))
        return -1;
    int64_t phi_corner[2] = {0, (int64_t)360 * g->phi_u_per_deg - 1};
    int64_t z_corner[2] = {g->z_min_u, (int64_t)g->z_min_u + (int64_t)g->n_z_strips * g->z_pitch_u};
    for (int k = ORACLE_MAX_FRAC_BITS; k >= 8; --k) {
        tables_at(g, n_theta, n_rho, k, C, S, D);
        int fits = 1;
        for (int t = 0; t < n_theta && fits; ++t)
            for (int i = 0; i < 2 && fits; ++i)
                for (int j = 0; j < 2 && fits; ++j) {
                    int64_t v = phi_corner[i] * C[t] + z_corner[j] * S[t] + *D;
                    if (v >= ((int64_t)1 << 31) || v < -((int64_t)1 << 31))
                        fits = 0;
                }
        if (fits)
            return k;
    }
    return -1;
}

/*
 * Step A: strip address -> fixed-point (phi, z).  Radial vanes sit every
 * 360/n_vanes degrees (Section 2), so phi is the vane angle; z is the centre
 * of the strip.  Out-of-range addresses are encoded anyway (the find step
 * rejects them).
 */
void oracle_encode(const oracle_geometry *g, const int32_t *vane, const int32_t *strip, int64_t n,
                   int32_t *phi_q, int32_t *z_q)
{
    int64_t vane_step = (int64_t)360 * g->phi_u_per_deg / g->n_vanes;
    for (int64_t i = 0; i < n; ++i) {
        phi_q[i] = (int32_t)(vane_step * (int64_t)vane[i]);
        z_q[i] = (int32_t)((int64_t)g->z_min_u + (int64_t)g->z_pitch_u * strip[i] +
                           g->z_pitch_u / 2);
    }
}

/* Whether an encoded hit lies inside the detector's coordinate box. */
static int hit_is_valid(const oracle_geometry *g, int32_t phi, int32_t z)
{
    int64_t phi_end = (int64_t)360 * g->phi_u_per_deg;
    int64_t z_end = (int64_t)g->z_min_u + (int64_t)g->n_z_strips * g->z_pitch_u;
    return phi >= 0 && (int64_t)phi < phi_end && z >= g->z_min_u && (int64_t)z <= z_end;
}

/* The rho bin of one hit in one theta row, for tables at scale 2^k. */
static int64_t rho_bin(int32_t phi, int32_t z, int32_t c, int32_t s, int64_t d, int k)
{
    int64_t value = (int64_t)phi * (int64_t)c + (int64_t)z * (int64_t)s + d;
    return floor_div(value, (int64_t)1 << k);
}

/*
 * Step B alone: fill a zeroed int32 accumulator acc[n_theta][n_rho] from the
 * valid hits; returns the number of dropped (out-of-range) votes.
 */
int64_t oracle_vote(const oracle_geometry *g, int n_theta, int n_rho, const int32_t *phi_q,
                    const int32_t *z_q, int64_t n_hits, int32_t *acc)
{
    int32_t *C = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_theta);
    int32_t *S = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_theta);
    int64_t D = 0;
    int64_t dropped = 0;
    int k = oracle_tables(g, n_theta, n_rho, C, S, &D);
    memset(acc, 0, sizeof(int32_t) * (size_t)n_theta * (size_t)n_rho);
    for (int64_t h = 0; h < n_hits; ++h) {
        if (!hit_is_valid(g, phi_q[h], z_q[h]))
            continue;
        for (int t = 0; t < n_theta; ++t) {
            int64_t b = rho_bin(phi_q[h], z_q[h], C[t], S[t], D, k);
            if (b >= 0 && b < n_rho)
                acc[(size_t)t * n_rho + (size_t)b] += 1;
            else
                dropped += 1;
        }
    }
    free(C);
    free(S);
    return dropped;
}

/* FP64 continuous variant of step B: the bin from Eq. (1) in double precision,
 * b = floor((phi_deg*cos(theta) + z_mm*sin(theta) - rho_min) / drho).  Used to
 * check that the fixed-point bins agree within one bin.  bins[h*n_theta + t]. */
static int64_t bin_fp64(const oracle_geometry *g, int n_theta, int n_rho, int32_t phi_q,
                        int32_t z_q, int t)
{
    double drho = (g->rho_max - g->rho_min) / (double)n_rho;
    double phi = (double)phi_q / (double)g->phi_u_per_deg;
    double z = (double)z_q / (double)g->z_u_per_mm;
    double theta = ((double)t + 0.5) * (M_PI / (double)n_theta);
    double rho = phi * cos(theta) + z * sin(theta);
    return (int64_t)floor((rho - g->rho_min) / drho);
}

void oracle_bins_fp64(const oracle_geometry *g, int n_theta, int n_rho, const int32_t *phi_q,
                      const int32_t *z_q, int64_t n_hits, int64_t *bins)
{
    for (int64_t h = 0; h < n_hits; ++h)
        for (int t = 0; t < n_theta; ++t)
            bins[h * n_theta + t] = bin_fp64(g, n_theta, n_rho, phi_q[h], z_q[h], t);
}

/* Fixed-point bins for every (hit, theta); same layout as oracle_bins_fp64. */
void oracle_bins_fixed(const oracle_geometry *g, int n_theta, int n_rho, const int32_t *phi_q,
                       const int32_t *z_q, int64_t n_hits, int64_t *bins)
{
    int32_t *C = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_theta);
    int32_t *S = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_theta);
    int64_t D = 0;
    int k = oracle_tables(g, n_theta, n_rho, C, S, &D);
    for (int64_t h = 0; h < n_hits; ++h)
        for (int t = 0; t < n_theta; ++t)
            bins[h * n_theta + t] = rho_bin(phi_q[h], z_q[h], C[t], S[t], D, k);
    free(C);
    free(S);
}

/* ----------------------------------------------------------------- step C */

static int32_t acc_at(const int32_t *acc, int n_theta, int n_rho, int t, int b)
{
    if (t < 0 || t >= n_theta || b < 0 || b >= n_rho)
        return 0; /* no neighbour across an edge; counts are >= 0 and peaks >= T >= 1 */
    return acc[(size_t)t * n_rho + (size_t)b];
}

typedef struct {
    int32_t votes;
    int32_t t;
    int32_t b;
} cand_t;

/* votes descending, then theta ascending, then rho ascending */
static int cand_cmp(const void *pa, const void *pb)
{
    const cand_t *a = (const cand_t *)pa;
    const cand_t *b = (const cand_t *)pb;
    if (a->votes != b->votes)
        return a->votes > b->votes ? -1 : 1;
    if (a->t != b->t)
        return a->t < b->t ? -1 : 1;
    if (a->b != b->b)
        return a->b < b->b ? -1 : 1;
    return 0;
}

/*
 * Step C on a given accumulator.  A bin (t, b) with v = acc[t][b] >= T is a
 * peak iff v is strictly greater than each of its neighbours that come earlier
 * in row-major order, (t-1, b-1), (t-1, b), (t-1, b+1), (t, b-1), and greater
 * than or equal to each later one, (t, b+1), (t+1, b-1), (t+1, b), (t+1, b+1).
 * Peaks are sorted (votes desc, t asc, b asc); the first max_peaks are kept.
 * Returns the number of peaks found (before truncation); *n_kept gets the kept
 * count.
 */
int32_t oracle_peaks(const int32_t *acc, int n_theta, int n_rho, int32_t threshold,
                     int32_t max_peaks, oracle_peak *peaks, int32_t *n_kept)
{
    size_t cap = 64, n = 0;
    cand_t *cand = (cand_t *)malloc(sizeof(cand_t) * cap);
    for (int t = 0; t < n_theta; ++t) {
        for (int b = 0; b < n_rho; ++b) {
            int32_t v = acc[(size_t)t * n_rho + (size_t)b];
            if (v < threshold)
                continue;
            int ok = v > acc_at(acc, n_theta, n_rho, t - 1, b - 1) &&
                     v > acc_at(acc, n_theta, n_rho, t - 1, b) &&
                     v > acc_at(acc, n_theta, n_rho, t - 1, b + 1) &&
                     v > acc_at(acc, n_theta, n_rho, t, b - 1) &&
                     v >= acc_at(acc, n_theta, n_rho, t, b + 1) &&
                     v >= acc_at(acc, n_theta, n_rho, t + 1, b - 1) &&
                     v >= acc_at(acc, n_theta, n_rho, t + 1, b) &&
                     v >= acc_at(acc, n_theta, n_rho, t + 1, b + 1);
            if (!ok)
                continue;
            if (n == cap) {
                cap *= 2;
                cand = (cand_t *)realloc(cand, sizeof(cand_t) * cap);
            }
            cand[n].votes = v;
            cand[n].t = t;
            cand[n].b = b;
            ++n;
        }
    }
    qsort(cand, n, sizeof(cand_t), cand_cmp);
    int32_t kept = (int32_t)(n < (size_t)max_peaks ? n : (size_t)max_peaks);
    for (int32_t i = 0; i < kept; ++i) {
        peaks[i].theta = (uint16_t)cand[i].t;
        peaks[i].rho = (uint16_t)cand[i].b;
        peaks[i].votes = cand[i].votes;
        peaks[i].n_hits = 0;
        peaks[i].hit_begin = 0;
    }
    free(cand);
    *n_kept = kept;
    return (int32_t)n;
}

/* --------------------------------------------------------------- step A-D */

/*
 * One time window through steps B-D.
 *   acc        : optional int32[n_theta*n_rho] (NULL: use a private buffer)
 *   peaks      : out, max_peaks entries
 *   hit_track  : out, per hit: peak index (0..n_kept-1), -1 unassigned,
 *                -2 rejected (outside the coordinate box)
 *   track_hits : out, a permutation of 0..n_hits-1: the hits of peak 0 in
 *                increasing index, then of peak 1, ..., then the unassigned
 *                hits, then the rejected ones.  peaks[p].hit_begin/n_hits
 *                index into it.
 * Returns 0, or -1 on bad arguments.
 */
int oracle_find_window(const oracle_geometry *g, int n_theta, int n_rho,
                       const oracle_thresholds *th, const int32_t *phi_q, const int32_t *z_q,
                       int64_t n_hits, int32_t *acc_out, int64_t *n_dropped, oracle_peak *peaks,
                       int32_t *n_peaks, int32_t *n_found, int32_t *hit_track,
                       int32_t *track_hits, uint32_t *status)
{
    if (!g || !th || n_theta <= 0 || n_rho <= 0 || th->vote_threshold < 1 ||
        th->assoc_tol_bins < 0 || th->max_peaks < 0)
        return -1;
    uint32_t st = 0;
    int32_t *acc = acc_out;
    if (!acc)
        acc = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_theta * (size_t)n_rho);

    /* B: vote (the FP64 variant takes each bin from Eq. (1) in double precision) */
    const int fp64 = (th->flags & ORACLE_FLAG_FP64) != 0;
    int64_t dropped = 0;
    if (!fp64) {
        dropped = oracle_vote(g, n_theta, n_rho, phi_q, z_q, n_hits, acc);
    } else {
        memset(acc, 0, sizeof(int32_t) * (size_t)n_theta * (size_t)n_rho);
        for (int64_t h = 0; h < n_hits; ++h) {
            if (!hit_is_valid(g, phi_q[h], z_q[h]))
                continue;
            for (int t = 0; t < n_theta; ++t) {
                int64_t b = bin_fp64(g, n_theta, n_rho, phi_q[h], z_q[h], t);
                if (b >= 0 && b < n_rho)
                    acc[(size_t)t * n_rho + (size_t)b] += 1;
                else
                    ++dropped;
            }
        }
    }
    for (int64_t h = 0; h < n_hits; ++h)
        if (!hit_is_valid(g, phi_q[h], z_q[h]))
            st |= ORACLE_WIN_HIT_OUT_OF_RANGE;
    if (dropped > 0)
        st |= ORACLE_WIN_VOTE_OUT_OF_RANGE;

    /* C: peaks */
    int32_t kept = 0;
    int32_t found = oracle_peaks(acc, n_theta, n_rho, th->vote_threshold, th->max_peaks, peaks,
                                 &kept);
    if (found > th->max_peaks)
        st |= ORACLE_WIN_PEAK_OVERFLOW;

    /* D: association, first matching peak in the sorted order */
    int32_t *C = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_theta);
    int32_t *S = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_theta);
    int64_t D = 0;
    int k = oracle_tables(g, n_theta, n_rho, C, S, &D);
    for (int64_t h = 0; h < n_hits; ++h) {
        if (!hit_is_valid(g, phi_q[h], z_q[h])) {
            hit_track[h] = -2;
            continue;
        }
        hit_track[h] = -1;
        for (int32_t p = 0; p < kept; ++p) {
            int t = peaks[p].theta;
            int64_t bh = fp64 ? bin_fp64(g, n_theta, n_rho, phi_q[h], z_q[h], t)
                              : rho_bin(phi_q[h], z_q[h], C[t], S[t], D, k);
            int64_t diff = bh - (int64_t)peaks[p].rho;
            if (diff < 0)
                diff = -diff;
            if (diff <= th->assoc_tol_bins) {
                hit_track[h] = p;
                break;
            }
        }
    }
    /* per-peak compaction, each group in increasing hit index */
    int32_t pos = 0;
    for (int32_t p = 0; p < kept; ++p) {
        peaks[p].hit_begin = pos;
        for (int64_t h = 0; h < n_hits; ++h)
            if (hit_track[h] == p)
                track_hits[pos++] = (int32_t)h;
        peaks[p].n_hits = pos - peaks[p].hit_begin;
    }
    for (int64_t h = 0; h < n_hits; ++h)
        if (hit_track[h] == -1)
            track_hits[pos++] = (int32_t)h;
    for (int64_t h = 0; h < n_hits; ++h)
        if (hit_track[h] == -2)
            track_hits[pos++] = (int32_t)h;

    free(C);
    free(S);
    if (!acc_out)
        free(acc);
    if (n_dropped)
        *n_dropped = dropped;
    *n_peaks = kept;
    if (n_found)
        *n_found = found;
    *status = st;
    return 0;
}

/*
 * A batch of windows in CSR form (window w owns hits offsets[w]..offsets[w+1]),
 * each processed independently by oracle_find_window.  Outputs use the same
 * layout as the library's: peaks[w*max_peaks + i], n_peaks[w], n_found[w],
 * hit_track[h] and track_hits[h] window-local, status[w]; acc (optional) is
 * [n_windows][n_theta][n_rho].  Returns 0, or -1 on bad arguments.
 */
int oracle_find_batch(const oracle_geometry *g, int n_theta, int n_rho,
                      const oracle_thresholds *th, const int32_t *phi_q, const int32_t *z_q,
                      const int64_t *offsets, int64_t n_windows, int32_t *acc, oracle_peak *peaks,
                      int32_t *n_peaks, int32_t *n_found, int32_t *hit_track,
                      int32_t *track_hits, uint32_t *status)
{
    for (int64_t w = 0; w < n_windows; ++w) {
        int64_t b = offsets[w], e = offsets[w + 1];
        if (b < 0 || e < b)
            return -1;
        int rc = oracle_find_window(
            g, n_theta, n_rho, th, phi_q + b, z_q + b, e - b,
            acc ? acc + (size_t)w * n_theta * n_rho : NULL, NULL,
            peaks + (size_t)w * th->max_peaks, n_peaks + w, n_found ? n_found + w : NULL,
            hit_track + b, track_hits + b, status + w);
        if (rc != 0)
            return rc;
    }
    return 0;
}

/* ------------------------------------------------------------ time slicing */

/*
 * Overlapping time windows (Section 5: the hits are divided into overlapping
 * windows of 10 ns with a sliding step of 5 ns; Section 6: one window per
 * unit of work).  Window k, 0 <= k < n_windows, holds every hit h with
 *     t0 + k*step <= t[h] < t0 + k*step + len,
 * in input order; a hit lies in every window that covers its time.  The
 * result is CSR: window k owns index[offsets[k] .. offsets[k+1]), index[j]
 * being the input position of the hit.  This is the definition written out
 * as a double loop over windows and hits (no sorting is assumed here).
 * Returns the number of entries, -1 on bad arguments, -2 when they would
 * not fit in `capacity`.
 */
int64_t oracle_time_slice(const int64_t *t, int64_t n, int64_t t0, int64_t step, int64_t len,
                          int64_t n_windows, int64_t *offsets, int64_t *index, int64_t capacity)
{
    if (n < 0 || step <= 0 || len <= 0 || n_windows < 0 || (n > 0 && !t) || !offsets)
        return -1;
    int64_t m = 0;
    for (int64_t k = 0; k < n_windows; ++k) {
        const int64_t start = t0 + k * step;
        const int64_t end = start + len;
        offsets[k] = m;
        for (int64_t h = 0; h < n; ++h) {
            if (t[h] >= start && t[h] < end) {
                if (m >= capacity)
                    return -2;
                index[m] = h;
                ++m;
            }
        }
    }
    offsets[n_windows] = m;
    return m;
}

/* ------------------------------------------------------ coarse-to-fine search */

/*
 * The paper's two-stage search for one line per window (Section 6 and the
 * figure of the Hough steps: a coarse 18 x 100 histogram, then a 10 x 10 fine
 * histogram around the high-likelihood zone, whose highest bin gives the
 * line).  Reading: the coarse histogram has 18 theta bins (10 degrees) and
 * 100 rho bins (10 units) over the same ranges as the full one; the coarse
 * bin with the most entries is taken (ties: first in row-major order); the
 * fine histogram covers that coarse bin with the 1-degree x 1-unit bins of
 * the paper's 180 x 1000 grid (Section 5): fine row tc*10 + i, fine rho bin
 * bc*10 + j, 0 <= i, j < 10.  Its highest bin (ties row-major) is the line.
 * If the coarse or the fine maximum is below T the window has no line.
 * Seeds: the valid hits whose bin in the line's row is within tol of its bin.
 */
typedef struct {
    int32_t coarse_theta, coarse_rho, coarse_votes;
    int32_t fine_theta, fine_rho, fine_votes;
    int32_t n_seeds;
    int32_t found;
} oracle_cf;

#define CF_COARSE_THETA 18
#define CF_COARSE_RHO 100
#define CF_FINE_THETA 180
#define CF_FINE_RHO 1000
#define CF_BLOCK 10

int oracle_coarse_fine_window(const oracle_geometry *g, const oracle_thresholds *th,
                              const int32_t *phi_q, const int32_t *z_q, int64_t n,
                              oracle_cf *out, int32_t *hit_track)
{
    int32_t Cc[CF_COARSE_THETA], Sc[CF_COARSE_THETA], Cf[CF_FINE_THETA], Sf[CF_FINE_THETA];
    int64_t Dc = 0, Df = 0;
    int kc = oracle_tables(g, CF_COARSE_THETA, CF_COARSE_RHO, Cc, Sc, &Dc);
    int kf = oracle_tables(g, CF_FINE_THETA, CF_FINE_RHO, Cf, Sf, &Df);
    if (kc < 0 || kf < 0 || !th || !out)
        return -1;
    int32_t coarse[CF_COARSE_THETA][CF_COARSE_RHO];
    int32_t fine[CF_BLOCK][CF_BLOCK];
    memset(coarse, 0, sizeof(coarse));
    memset(fine, 0, sizeof(fine));
    memset(out, 0, sizeof(*out));
    /* coarse histogram over every valid hit */
    for (int64_t h = 0; h < n; ++h) {
        if (!hit_is_valid(g, phi_q[h], z_q[h]))
            continue;
        for (int t = 0; t < CF_COARSE_THETA; ++t) {
            int64_t b = rho_bin(phi_q[h], z_q[h], Cc[t], Sc[t], Dc, kc);
            if (b >= 0 && b < CF_COARSE_RHO)
                coarse[t][b] += 1;
        }
    }
    int tc = 0, bc = 0;
    for (int t = 0; t < CF_COARSE_THETA; ++t)
        for (int b = 0; b < CF_COARSE_RHO; ++b)
            if (coarse[t][b] > coarse[tc][bc]) {
                tc = t;
                bc = b;
            }
    out->coarse_theta = tc;
    out->coarse_rho = bc;
    out->coarse_votes = coarse[tc][bc];
    int found = out->coarse_votes >= th->vote_threshold;
    int tf = 0, bf = 0;
    if (found) {
        /* fine histogram: the 10 x 10 bins of the 180 x 1000 grid inside the
           coarse bin */
        for (int64_t h = 0; h < n; ++h) {
            if (!hit_is_valid(g, phi_q[h], z_q[h]))
                continue;
            for (int i = 0; i < CF_BLOCK; ++i) {
                int t = tc * CF_BLOCK + i;
                int64_t b = rho_bin(phi_q[h], z_q[h], Cf[t], Sf[t], Df, kf);
                int64_t j = b - (int64_t)bc * CF_BLOCK;
                if (j >= 0 && j < CF_BLOCK)
                    fine[i][j] += 1;
            }
        }
        int bi = 0, bj = 0;
        for (int i = 0; i < CF_BLOCK; ++i)
            for (int j = 0; j < CF_BLOCK; ++j)
                if (fine[i][j] > fine[bi][bj]) {
                    bi = i;
                    bj = j;
                }
        tf = tc * CF_BLOCK + bi;
        bf = bc * CF_BLOCK + bj;
        out->fine_theta = tf;
        out->fine_rho = bf;
        out->fine_votes = fine[bi][bj];
        found = out->fine_votes >= th->vote_threshold;
    }
    out->found = found;
    for (int64_t h = 0; h < n; ++h) {
        if (!hit_is_valid(g, phi_q[h], z_q[h])) {
            hit_track[h] = -2;
            continue;
        }
        hit_track[h] = -1;
        if (found) {
            int64_t b = rho_bin(phi_q[h], z_q[h], Cf[tf], Sf[tf], Df, kf);
            if (b - bf <= th->assoc_tol_bins && bf - b <= th->assoc_tol_bins) {
                hit_track[h] = 0;
                out->n_seeds += 1;
            }
        }
    }
    return 0;
}

int oracle_coarse_fine_batch(const oracle_geometry *g, const oracle_thresholds *th,
                             const int32_t *phi_q, const int32_t *z_q, const int64_t *offsets,
                             int64_t n_windows, oracle_cf *out, int32_t *hit_track)
{
    for (int64_t w = 0; w < n_windows; ++w) {
        int64_t b = offsets[w], e = offsets[w + 1];
        if (b < 0 || e < b)
            return -1;
        int rc = oracle_coarse_fine_window(g, th, phi_q + b, z_q + b, e - b, out + w,
                                           hit_track + b);
        if (rc != 0)
            return rc;
    }
    return 0;
}

/* ------------------------------------------------------ iterative single peak */

/*
 * The literal reading of the paper's peak step (Section 4: the bin with the
 * highest accumulation is the most probable line; Section 5: the seeds are
 * the hits aligned with it), repeated until no line is left: vote the hits
 * not yet assigned into the full accumulator, take its highest bin (ties:
 * first in row-major order), stop if it holds fewer than T votes, else give
 * track k every remaining hit whose bin in that row is within tol of it,
 * remove them and vote again.  At most max_tracks tracks.
 * Per window: tracks[k] = (theta, rho, votes, n_hits), n_tracks, and per hit
 * its track index, -1 if none, -2 outside the detector box.
 */
typedef struct {
    int32_t theta, rho, votes, n_hits;
} oracle_iter_track;

int oracle_iterative_window(const oracle_geometry *g, int n_theta, int n_rho,
                            const oracle_thresholds *th, const int32_t *phi_q, const int32_t *z_q,
                            int64_t n, int max_tracks, oracle_iter_track *tracks,
                            int32_t *n_tracks, int32_t *hit_track)
{
    int32_t *C = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_theta);
    int32_t *S = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_theta);
    int32_t *acc = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_theta * (size_t)n_rho);
    int64_t D = 0;
    int k = oracle_tables(g, n_theta, n_rho, C, S, &D);
    if (k < 0 || !C || !S || !acc || max_tracks < 0) {
        free(C);
        free(S);
        free(acc);
        return -1;
    }
    for (int64_t h = 0; h < n; ++h)
        hit_track[h] = hit_is_valid(g, phi_q[h], z_q[h]) ? -1 : -2;
    int found = 0;
    while (found < max_tracks) {
        memset(acc, 0, sizeof(int32_t) * (size_t)n_theta * (size_t)n_rho);
        for (int64_t h = 0; h < n; ++h) {
            if (hit_track[h] != -1)
                continue;
            for (int t = 0; t < n_theta; ++t) {
                int64_t b = rho_bin(phi_q[h], z_q[h], C[t], S[t], D, k);
                if (b >= 0 && b < n_rho)
                    acc[(size_t)t * n_rho + b] += 1;
            }
        }
        int bt = 0, bb = 0;
        for (int t = 0; t < n_theta; ++t)
            for (int b = 0; b < n_rho; ++b)
                if (acc[(size_t)t * n_rho + b] > acc[(size_t)bt * n_rho + bb]) {
                    bt = t;
                    bb = b;
                }
        int32_t votes = acc[(size_t)bt * n_rho + bb];
        if (votes < th->vote_threshold)
            break;
        int32_t taken = 0;
        for (int64_t h = 0; h < n; ++h) {
            if (hit_track[h] != -1)
                continue;
            int64_t b = rho_bin(phi_q[h], z_q[h], C[bt], S[bt], D, k);
            if (b - bb <= th->assoc_tol_bins && bb - b <= th->assoc_tol_bins) {
                hit_track[h] = found;
                ++taken;
            }
        }
        tracks[found].theta = bt;
        tracks[found].rho = bb;
        tracks[found].votes = votes;
        tracks[found].n_hits = taken;
        ++found;
    }
    *n_tracks = found;
    free(C);
    free(S);
    free(acc);
    return 0;
}

int oracle_iterative_batch(const oracle_geometry *g, int n_theta, int n_rho,
                           const oracle_thresholds *th, const int32_t *phi_q, const int32_t *z_q,
                           const int64_t *offsets, int64_t n_windows, int max_tracks,
                           oracle_iter_track *tracks, int32_t *n_tracks, int32_t *hit_track)
{
    for (int64_t w = 0; w < n_windows; ++w) {
        int64_t b = offsets[w], e = offsets[w + 1];
        if (b < 0 || e < b)
            return -1;
        int rc = oracle_iterative_window(g, n_theta, n_rho, th, phi_q + b, z_q + b, e - b,
                                         max_tracks, tracks + (size_t)w * max_tracks,
                                         n_tracks + w, hit_track + b);
        if (rc != 0)
            return rc;
    }
    return 0;
}

/* --------------------------------------------------------- track extension */

typedef struct {
    int32_t first_vane; /* vane of the track's first hit in increasing-vane order, -1: none */
    int32_t n_hits;     /* hits of the track, one per vane (0: the peak gave no seed) */
    int32_t hit_begin;  /* where the track's hits start in ext_hits */
    int32_t seed_mid;   /* window-local index of the seed's middle hit, -1: none */
} oracle_ext_track;

static int64_t abs64(int64_t x) { return x < 0 ? -x : x; }

/*
 * Track extension of one window (Section 4: a seed of three RecoHits on
 * consecutive vanes, its trajectory extrapolated to the neighbouring vanes
 * forward and backward, confined to the time window).  Inputs are the
 * window's encoded hits and the output of steps C-D for it (peaks in the
 * canonical order with their hit groups in track_hits, hit_track per hit).
 *
 * A hit takes part if it was not rejected (hit_track != -2) and lies on a
 * vane, phi_q = k * (360 deg / n_vanes) with 0 <= k < n_vanes; its vane is k.
 * Vanes are neighbours modulo n_vanes (the vanes form a ring).  The peaks are
 * taken in their order; a hit that a track has taken ("claimed") is not
 * available to any later one.  For peak p:
 *   seed: over the unclaimed hits a, b, c of the peak's group with
 *         vane(a) = vane(b) - 1 and vane(c) = vane(b) + 1 and
 *         |z_a - 2 z_b + z_c| <= tol_z, the one with the smallest
 *         (|z_a - 2 z_b + z_c|, b, a, c), comparing hit indices; no such
 *         triplet: the peak gives no track;
 *   forward: with q0, q1, q2 the last three hits (in vane order), predict
 *         z = 3 z_q2 - 3 z_q1 + z_q0 (the parabola through them, one vane on)
 *         on vane(q2) + 1; take the unclaimed hit of the window on that vane
 *         nearest the prediction within tol_z (ties: the lower z, then the
 *         lower index); stop when there is none;
 *   backward: the same from the seed's first hit towards lower vanes;
 *   a track never holds more hits than there are vanes.
 * Outputs: ext[p] for every peak, ext_track[h] = index of the track holding
 * hit h or -1, and ext_hits: the hits of track 0 in increasing vane order
 * from its first vane, then those of track 1, ..., then every hit that no
 * track holds, in increasing index.  Returns 0, -1 on bad arguments.
 */
int oracle_extend_window(const oracle_geometry *g, const int32_t *phi_q, const int32_t *z_q,
                         int64_t n_hits, const oracle_peak *peaks, int32_t n_peaks,
                         const int32_t *hit_track, const int32_t *track_hits, int32_t tol_z,
                         oracle_ext_track *ext, int32_t *ext_track, int32_t *ext_hits)
{
    if (!g || g->n_vanes < 3 || tol_z < 0 || n_hits < 0 || n_peaks < 0)
        return -1;
    const int nv = g->n_vanes;
    const int64_t vstep = (int64_t)360 * g->phi_u_per_deg / nv;
    int32_t *vane = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_hits > 0 ? n_hits : 1));
    int64_t *line = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * nv + 4));
    for (int64_t h = 0; h < n_hits; ++h) {
        vane[h] = -1;
        ext_track[h] = -1;
        if (hit_track[h] == -2 || !hit_is_valid(g, phi_q[h], z_q[h]) || vstep <= 0)
            continue;
        if (phi_q[h] % vstep == 0 && phi_q[h] / vstep < nv)
            vane[h] = (int32_t)(phi_q[h] / vstep);
    }
    for (int32_t p = 0; p < n_peaks; ++p) {
        ext[p].first_vane = -1;
        ext[p].n_hits = 0;
        ext[p].hit_begin = 0;
        ext[p].seed_mid = -1;
        const int32_t *grp = track_hits + peaks[p].hit_begin;
        const int32_t m = peaks[p].n_hits;
        /* seed */
        int64_t bc = -1, ba = -1, bb = -1, bcc = -1;
        for (int32_t ib = 0; ib < m; ++ib) {
            int32_t b = grp[ib];
            if (vane[b] < 0 || ext_track[b] >= 0)
                continue;
            for (int32_t ia = 0; ia < m; ++ia) {
                int32_t a = grp[ia];
                if (vane[a] < 0 || ext_track[a] >= 0 || vane[a] != (vane[b] - 1 + nv) % nv)
                    continue;
                for (int32_t ic = 0; ic < m; ++ic) {
                    int32_t c = grp[ic];
                    if (vane[c] < 0 || ext_track[c] >= 0 || vane[c] != (vane[b] + 1) % nv)
                        continue;
                    int64_t curv = abs64((int64_t)z_q[a] - 2 * (int64_t)z_q[b] + z_q[c]);
                    if (curv > tol_z)
                        continue;
                    int better = bc < 0 || curv < bc ||
                                 (curv == bc && (b < bb || (b == bb && (a < ba ||
                                  (a == ba && c < bcc)))));
                    if (better) {
                        bc = curv;
                        ba = a;
                        bb = b;
                        bcc = c;
                    }
                }
            }
        }
        if (bc < 0)
            continue;
        /* line[lo..hi) holds the track in increasing vane order */
        int lo = nv + 1, hi = nv + 1;
        line[hi++] = ba;
        line[hi++] = bb;
        line[hi++] = bcc;
        ext_track[ba] = ext_track[bb] = ext_track[bcc] = p;
        /* forward */
        while (hi - lo < nv) {
            int64_t q0 = line[hi - 3], q1 = line[hi - 2], q2 = line[hi - 1];
            int tv = (vane[q2] + 1) % nv;
            int64_t pred = 3 * (int64_t)z_q[q2] - 3 * (int64_t)z_q[q1] + z_q[q0];
            int64_t best = -1, bd = 0;
            for (int64_t h = 0; h < n_hits; ++h) {
                if (vane[h] != tv || ext_track[h] >= 0)
                    continue;
                int64_t d = abs64((int64_t)z_q[h] - pred);
                if (d > tol_z)
                    continue;
                if (best < 0 || d < bd || (d == bd && z_q[h] < z_q[best]))
                    best = h, bd = d; /* equal d and z: the earlier index stays */
            }
            if (best < 0)
                break;
            ext_track[best] = p;
            line[hi++] = best;
        }
        /* backward */
        while (hi - lo < nv) {
            int64_t q0 = line[lo + 2], q1 = line[lo + 1], q2 = line[lo];
            int tv = (vane[q2] - 1 + nv) % nv;
            int64_t pred = 3 * (int64_t)z_q[q2] - 3 * (int64_t)z_q[q1] + z_q[q0];
            int64_t best = -1, bd = 0;
            for (int64_t h = 0; h < n_hits; ++h) {
                if (vane[h] != tv || ext_track[h] >= 0)
                    continue;
                int64_t d = abs64((int64_t)z_q[h] - pred);
                if (d > tol_z)
                    continue;
                if (best < 0 || d < bd || (d == bd && z_q[h] < z_q[best]))
                    best = h, bd = d;
            }
            if (best < 0)
                break;
            ext_track[best] = p;
            line[--lo] = best;
        }
        ext[p].first_vane = vane[line[lo]];
        ext[p].n_hits = hi - lo;
        ext[p].seed_mid = (int32_t)bb;
    }
    /* ext_hits: tracks in peak order, each in increasing vane order, then the rest */
    int32_t pos = 0;
    for (int32_t p = 0; p < n_peaks; ++p) {
        ext[p].hit_begin = pos;
        for (int32_t k = 0; k < ext[p].n_hits; ++k) {
            int tv = (ext[p].first_vane + k) % nv;
            for (int64_t h = 0; h < n_hits; ++h)
                if (ext_track[h] == p && vane[h] == tv)
                    ext_hits[pos++] = (int32_t)h;
        }
    }
    for (int64_t h = 0; h < n_hits; ++h)
        if (ext_track[h] < 0)
            ext_hits[pos++] = (int32_t)h;
    free(line);
    free(vane);
    return 0;
}

/* A CSR batch of windows, each through oracle_extend_window, with the layout of
 * oracle_find_batch (peaks and ext strided by max_peaks, per-hit arrays
 * window-local).  Returns 0, -1 on bad arguments. */
int oracle_extend_batch(const oracle_geometry *g, const int32_t *phi_q, const int32_t *z_q,
                        const int64_t *offsets, int64_t n_windows, const oracle_peak *peaks,
                        const int32_t *n_peaks, int32_t max_peaks, const int32_t *hit_track,
                        const int32_t *track_hits, int32_t tol_z, oracle_ext_track *ext,
                        int32_t *ext_track, int32_t *ext_hits)
{
    for (int64_t w = 0; w < n_windows; ++w) {
        int64_t b = offsets[w], e = offsets[w + 1];
        if (b < 0 || e < b || n_peaks[w] < 0 || n_peaks[w] > max_peaks)
            return -1;
        int rc = oracle_extend_window(g, phi_q + b, z_q + b, e - b,
                                      peaks + (size_t)w * max_peaks, n_peaks[w], hit_track + b,
                                      track_hits + b, tol_z, ext + (size_t)w * max_peaks,
                                      ext_track + b, ext_hits + b);
        if (rc != 0)
            return rc;
    }
    return 0;
}
