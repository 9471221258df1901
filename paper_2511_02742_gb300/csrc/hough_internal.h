// hough_internal.h -- the library's private view of a context, shared by
// the translation units of libhough (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <unordered_map>
#include <vector>

#include "hough.h"

struct hough_ctx {
    int device = 0;
    hough_geometry g{};
    hough_thresholds th{};
    int n_theta = 0, n_rho = 0;
    std::vector<int32_t> C, S;
    long long D = 0;
    int K = 0;
    bool in_range = false;   // every valid hit votes inside [0, n_rho) in every row
    // narrowed find tiles, per launch word-row count 32, 64, 128: the bins a
    // tile stores per row (0: all n_rho), and on the device the first stored
    // bin of every tile, [word-row count][log2 P][tile], tile rows lo_stride
    // apart (null: every tile starts at bin 0)
    int tile_nb[3] = {0, 0, 0};
    int32_t *d_lo = nullptr;
    int lo_stride = 0;
    int32_t *d_C = nullptr, *d_S = nullptr;
    double *d_Cd = nullptr, *d_Sd = nullptr;   // cos/sin of the row centres (HOUGH_FLAG_FP64)
    hough_launch launch{};
    bool auto_launch = true;   // the shape was left to the library (see launch_for)
    int num_sms = 0;
    size_t smem_optin = 0;
    size_t smem_per_sm = 0;
    std::unordered_map<cudaStream_t, unsigned int *> counters;
    int last_error = HOUGH_OK;
    std::atomic<long long> launches{0};
    // hough_find_host staging (device), grown on demand
    void *stage_dev = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t host_streams[2] = {nullptr, nullptr};
    cudaEvent_t host_events[2] = {nullptr, nullptr};
    // coarse (18 x 100) and fine (180 x 1000) tables of the two-stage search:
    // C then S of each, on the device; built on first use
    int32_t *d_cf = nullptr;
    // hough_accumulate's launch (threads per CTA, resident CTAs per SM),
    // worked out on its first call
    int acc_threads = 0, acc_occ = 0;
    int cf_K[2] = {0, 0};
    long long cf_D[2] = {0, 0};
};

// The find's launch shape for a batch (hough_api.cu): `base`, or a shape
// chosen from the batch's mean hits per window when `automatic`.
hough_launch launch_for(const hough_ctx *ctx, const hough_launch &base, bool automatic,
                        int64_t n_hits, int64_t n_windows);
