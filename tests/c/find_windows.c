/*
 * A C client of libhough: reads CSR windows of (vane, strip) hits from a file,
 * runs hough_find on the GPU and prints every window's peaks and hit
 * assignments.  No Python, no torch: the C ABI, the CUDA runtime for device
 * memory, and nothing else.
 *
 * Input file (little endian): int64 n_windows, int64 n_theta, int64 n_rho,
 * int64 offsets[n_windows + 1], int32 vane[n_hits], int32 strip[n_hits].
 * Output (text): per window "w n_peaks n_found status", then one line per
 * peak "theta rho votes n_hits hit_begin", then the window's hit_track values.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "hough.h"

#define CHECK(x)                                                              \
    do {                                                                      \
        int rc_ = (int)(x);                                                   \
        if (rc_ != 0) {                                                       \
            fprintf(stderr, "%s failed: %d\n", #x, rc_);                      \
            return 1;                                                         \
        }                                                                     \
    } while (0)

static void *dalloc(size_t n)
{
    void *p = NULL;
    if (cudaMalloc(&p, n ? n : 4) != cudaSuccess)
        return NULL;
    return p;
}

int main(int argc, char **argv)
{
    if (argc != 2)
        return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f)
        return 2;
    int64_t hdr[3];
    if (fread(hdr, 8, 3, f) != 3)
        return 2;
    const int64_t nw = hdr[0];
    const int n_theta = (int)hdr[1], n_rho = (int)hdr[2];
    int64_t *off = malloc(8 * (size_t)(nw + 1));
    if (fread(off, 8, (size_t)(nw + 1), f) != (size_t)(nw + 1))
        return 2;
    const int64_t nh = off[nw];
    int32_t *vane = malloc(4 * (size_t)nh + 4), *strip = malloc(4 * (size_t)nh + 4);
    if (fread(vane, 4, (size_t)nh, f) != (size_t)nh || fread(strip, 4, (size_t)nh, f) != (size_t)nh)
        return 2;
    fclose(f);

    hough_geometry g = {40, 2048, 38, -38912, 200, 200, -500.0, 500.0};
    hough_thresholds th = {5, 1, 64, 0};
    hough_ctx *ctx = NULL;
    CHECK(hough_create(&g, n_theta, n_rho, &th, &ctx));

    int32_t *d_vane = dalloc(4 * (size_t)nh), *d_strip = dalloc(4 * (size_t)nh);
    int64_t *d_off = dalloc(8 * (size_t)(nw + 1));
    hough_tracks t = {0};
    t.peaks = dalloc(sizeof(hough_peak) * (size_t)nw * 64);
    t.n_peaks = dalloc(4 * (size_t)nw);
    t.n_found = dalloc(4 * (size_t)nw);
    t.hit_track = dalloc(4 * (size_t)nh);
    t.track_hits = dalloc(4 * (size_t)nh);
    t.window_status = dalloc(4 * (size_t)nw);
    if (!d_vane || !d_strip || !d_off || !t.peaks || !t.n_peaks || !t.n_found || !t.hit_track ||
        !t.track_hits || !t.window_status)
        return 3;
    CHECK(cudaMemcpy(d_vane, vane, 4 * (size_t)nh, cudaMemcpyHostToDevice));
    CHECK(cudaMemcpy(d_strip, strip, 4 * (size_t)nh, cudaMemcpyHostToDevice));
    CHECK(cudaMemcpy(d_off, off, 8 * (size_t)(nw + 1), cudaMemcpyHostToDevice));

    hough_hits hits = {NULL, NULL, d_vane, d_strip, nh};
    CHECK(hough_find(ctx, &hits, d_off, nw, &t, NULL));
    CHECK(cudaDeviceSynchronize());

    hough_peak *pk = malloc(sizeof(hough_peak) * (size_t)nw * 64);
    int32_t *np = malloc(4 * (size_t)nw), *nf = malloc(4 * (size_t)nw);
    uint32_t *st = malloc(4 * (size_t)nw);
    int32_t *ht = malloc(4 * (size_t)nh + 4);
    CHECK(cudaMemcpy(pk, t.peaks, sizeof(hough_peak) * (size_t)nw * 64, cudaMemcpyDeviceToHost));
    CHECK(cudaMemcpy(np, t.n_peaks, 4 * (size_t)nw, cudaMemcpyDeviceToHost));
    CHECK(cudaMemcpy(nf, t.n_found, 4 * (size_t)nw, cudaMemcpyDeviceToHost));
    CHECK(cudaMemcpy(st, t.window_status, 4 * (size_t)nw, cudaMemcpyDeviceToHost));
    CHECK(cudaMemcpy(ht, t.hit_track, 4 * (size_t)nh, cudaMemcpyDeviceToHost));
    for (int64_t w = 0; w < nw; ++w) {
        printf("%lld %d %d %u\n", (long long)w, np[w], nf[w], st[w]);
        for (int i = 0; i < np[w]; ++i) {
            const hough_peak *p = &pk[w * 64 + i];
            printf("%u %u %d %d %d\n", p->theta, p->rho, p->votes, p->n_hits, p->hit_begin);
        }
        for (int64_t h = off[w]; h < off[w + 1]; ++h)
            printf("%d%c", ht[h], h + 1 < off[w + 1] ? ' ' : '\n');
        if (off[w] == off[w + 1])
            printf("\n");
    }
    hough_destroy(ctx);
    return 0;
}
