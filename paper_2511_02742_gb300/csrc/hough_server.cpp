// hough_server.cpp -- the request loop declared in the serving section of
// include/hough.h.
//
// A server owns n_slots batch slots.  Each slot has its own stream, a device
// input region (offsets | in0 | in1), a device output region (peaks | n_peaks
// | n_found | status | hit_track | track_hits) and a pinned staging area for
// the batch's window offsets, all allocated once.  One worker thread loops over:
//   retire  -- a busy slot whose completion event has fired: complete its
//              requests (their results are in their buffers already);
//   admit   -- a free slot and a non-empty queue: take requests, oldest
//              first, while the slot's window and hit capacity allows,
//              write the batch's window offsets (rebased) into the slot's
//              pinned staging, then on the slot's stream copy them and each
//              request's hits in, launch the find kernel, copy the results
//              straight into each request's buffers, and record its event.
// Windows never interact (each is its own unit of work), so packing
// requests together changes no result: a window's outputs depend only on its
// own hits, and all per-window outputs are window-local (peak indices,
// track_hits entries, hit_begin).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "hough.h"
#include "hough_internal.h"

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// How long an idle worker polls the queue before it sleeps.
constexpr int64_t kIdleSpinNs = 2'000'000;

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// Byte offsets of a batch of W windows and H hits inside a slot's regions.
struct InLayout {
    size_t off, in0, in1, total;
};
struct OutLayout {
    size_t pk, np, nf, st, ht, th, total;
};

InLayout in_layout(int64_t W, int64_t H)
{
    InLayout L;
    L.off = 0;
    L.in0 = al256(8 * (size_t)(W + 1));
    L.in1 = al256(L.in0 + 4 * (size_t)H);
    L.total = L.in1 + 4 * (size_t)H;
    return L;
}

OutLayout out_layout(int64_t W, int64_t H, int mp)
{
    OutLayout L;
    L.pk = 0;
    L.np = al256(sizeof(hough_peak) * (size_t)W * (size_t)mp);
    L.nf = al256(L.np + 4 * (size_t)W);
    L.st = al256(L.nf + 4 * (size_t)W);
    L.ht = al256(L.st + 4 * (size_t)W);
    L.th = al256(L.ht + 4 * (size_t)H);
    L.total = L.th + 4 * (size_t)H;
    return L;
}

struct Pending {
    uint64_t ticket = 0;
    hough_request req{};
    int64_t n_hits = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    cudaEvent_t t_start = nullptr, t_h2d = nullptr, t_kern = nullptr;   // timing marks
    int64_t pack_ns = 0, scatter_ns = 0;
    char *d_in = nullptr, *d_out = nullptr;   // device regions
    char *h_in = nullptr;                     // pinned staging of the batch's offsets
    bool busy = false;
    std::vector<Pending> reqs;
    std::vector<int64_t> win_base, hit_base;
    int64_t W = 0, H = 0;
    int64_t launch_ns = 0;
    int status = HOUGH_OK;
};

}  // namespace

struct hough_server {
    hough_ctx *ctx = nullptr;
    hough_server_config cfg{};
    hough_launch saved_launch{};     // the context's shape before the server
    // shapes chosen per batch when the configuration leaves the shape open:
    // the latency shape for batches of fewer than 2 windows per SM, else the
    // context's default (throughput) shape
    bool per_batch = false;
    hough_launch lat_launch{}, thr_launch{};
    bool thr_auto = false;           // thr_launch was left to the library
    bool saved_auto = false;         // the context's flag before the server
    int max_peaks = 0;
    size_t in_cap = 0, out_cap = 0, stage_cap = 0;
    std::vector<Slot> slots;

    std::mutex mu;
    std::condition_variable cv_work;   // worker: a request was queued, or stop
    std::condition_variable cv_done;   // waiters: requests completed
    std::deque<Pending> queue;
    std::unordered_set<uint64_t> live;                          // accepted, not yet delivered
    std::unordered_map<uint64_t, hough_request_result> done;    // completed, not yet delivered
    std::deque<uint64_t> done_order;                            // completion order (poll)
    uint64_t next_ticket = 1;
    int64_t in_flight = 0;
    hough_server_stats st{};
    bool stop = false;
    std::atomic<int64_t> queued{0};       // queue length, read without the lock
    std::atomic<bool> stopping{false};
    std::thread worker;
};

namespace {

// Pack the slot's requests into its input mirror and enqueue copy in, find,
// copy out and the completion event on the slot's stream.  Runs without the
// server lock (only the worker touches a busy slot).
int launch_slot(hough_server *s, Slot &sl)
{
    const int64_t t_pack = now_ns();
    const InLayout L = in_layout(sl.W, sl.H);
    const OutLayout O = out_layout(sl.W, sl.H, s->max_peaks);
    const int mp = s->max_peaks;
    int64_t *off = reinterpret_cast<int64_t *>(sl.h_in + L.off);
    for (size_t k = 0; k < sl.reqs.size(); ++k) {
        const hough_request &r = sl.reqs[k].req;
        const int64_t wb = sl.win_base[k], hb = sl.hit_base[k];
        for (int64_t j = 0; j < r.n_windows; ++j)
            off[wb + j] = hb + r.window_offsets[j];
    }
    off[sl.W] = sl.H;
    sl.pack_ns = now_ns() - t_pack;
    auto in = [&](void *dst, const void *src, size_t n) {
        return n == 0 || cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, sl.stream) ==
                             cudaSuccess;
    };
    auto out = [&](void *dst, const void *src, size_t n) {
        return n == 0 || cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, sl.stream) ==
                             cudaSuccess;
    };
    // copy in: the rebased offsets from the staging, each request's hits
    // straight from its own buffers
    bool ok = cudaEventRecord(sl.t_start, sl.stream) == cudaSuccess &&
              in(sl.d_in + L.off, sl.h_in + L.off, 8 * (size_t)(sl.W + 1));
    for (size_t k = 0; ok && k < sl.reqs.size(); ++k) {
        const hough_request &r = sl.reqs[k].req;
        const size_t hb = (size_t)sl.hit_base[k], nh = (size_t)sl.reqs[k].n_hits;
        ok = in(sl.d_in + L.in0 + 4 * hb, r.in0, 4 * nh) && in(sl.d_in + L.in1 + 4 * hb, r.in1, 4 * nh);
    }
    if (!ok || cudaEventRecord(sl.t_h2d, sl.stream) != cudaSuccess)
        return HOUGH_ERR_CUDA;
    hough_hits hits{};
    hits.n_hits = sl.H;
    const int32_t *d0 = reinterpret_cast<const int32_t *>(sl.d_in + L.in0);
    const int32_t *d1 = reinterpret_cast<const int32_t *>(sl.d_in + L.in1);
    if (s->cfg.raw_hits) {
        hits.vane = d0;
        hits.strip = d1;
    } else {
        hits.phi_q = d0;
        hits.z_q = d1;
    }
    hough_tracks t{};
    t.peaks = reinterpret_cast<hough_peak *>(sl.d_out + O.pk);
    t.n_peaks = reinterpret_cast<int32_t *>(sl.d_out + O.np);
    t.n_found = reinterpret_cast<int32_t *>(sl.d_out + O.nf);
    t.window_status = reinterpret_cast<uint32_t *>(sl.d_out + O.st);
    t.hit_track = reinterpret_cast<int32_t *>(sl.d_out + O.ht);
    t.track_hits = reinterpret_cast<int32_t *>(sl.d_out + O.th);
    if (s->per_batch)
        s->ctx->launch = sl.W >= 2 * (int64_t)s->ctx->num_sms
                             ? launch_for(s->ctx, s->thr_launch, s->thr_auto, sl.H, sl.W)
                             : s->lat_launch;
    int rc = hough_find(s->ctx, &hits, reinterpret_cast<const int64_t *>(sl.d_in + L.off), sl.W,
                        &t, sl.stream);
    if (rc != HOUGH_OK)
        return rc;
    // copy out, straight into each request's buffers
    ok = cudaEventRecord(sl.t_kern, sl.stream) == cudaSuccess;
    for (size_t k = 0; ok && k < sl.reqs.size(); ++k) {
        const hough_request &r = sl.reqs[k].req;
        const size_t wb = (size_t)sl.win_base[k], hb = (size_t)sl.hit_base[k];
        const size_t nw = (size_t)r.n_windows, nh = (size_t)sl.reqs[k].n_hits;
        ok = out(r.out.n_peaks, sl.d_out + O.np + 4 * wb, 4 * nw) &&
             out(r.out.window_status, sl.d_out + O.st + 4 * wb, 4 * nw) &&
             (!r.out.n_found || out(r.out.n_found, sl.d_out + O.nf + 4 * wb, 4 * nw)) &&
             (mp == 0 || out(r.out.peaks, sl.d_out + O.pk + sizeof(hough_peak) * wb * mp,
                             sizeof(hough_peak) * nw * mp)) &&
             out(r.out.hit_track, sl.d_out + O.ht + 4 * hb, 4 * nh) &&
             out(r.out.track_hits, sl.d_out + O.th + 4 * hb, 4 * nh);
    }
    if (!ok || cudaEventRecord(sl.done, sl.stream) != cudaSuccess)
        return HOUGH_ERR_CUDA;
    return HOUGH_OK;
}

// Complete every request of a slot (lock held) and free the slot.
void complete_slot(hough_server *s, Slot &sl, int64_t t_done)
{
    const int nreq = (int)sl.reqs.size();
    // GPU time of the batch's copy in, find and copy out, from its marks
    int64_t gpu_ns[3] = {0, 0, 0};
    if (sl.status == HOUGH_OK) {
        const cudaEvent_t ev[4] = {sl.t_start, sl.t_h2d, sl.t_kern, sl.done};
        for (int k = 0; k < 3; ++k) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[k], ev[k + 1]) == cudaSuccess)
                gpu_ns[k] = (int64_t)(ms * 1e6);
            else
                cudaGetLastError();
        }
    }
    for (const Pending &p : sl.reqs) {
        hough_request_result r{};
        r.ticket = p.ticket;
        r.status = sl.status;
        r.batch_requests = nreq;
        r.batch_windows = sl.W;
        r.arrival_ns = p.req.arrival_ns;
        r.launch_ns = sl.launch_ns;
        r.done_ns = t_done;
        r.pack_ns = sl.pack_ns;
        r.h2d_ns = gpu_ns[0];
        r.kernel_ns = gpu_ns[1];
        r.d2h_ns = gpu_ns[2];
        r.scatter_ns = sl.scatter_ns;
        s->done[p.ticket] = r;
        s->done_order.push_back(p.ticket);
    }
    s->st.completed += nreq;
    if (sl.status == HOUGH_OK)
        s->st.windows += sl.W;
    s->in_flight -= nreq;
    sl.reqs.clear();
    sl.busy = false;
    s->cv_done.notify_all();
}

void worker_loop(hough_server *s)
{
    cudaSetDevice(s->ctx->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        bool progress = false;
        // retire
        for (Slot &sl : s->slots) {
            if (!sl.busy)
                continue;
            const cudaError_t e = cudaEventQuery(sl.done);
            if (e == cudaErrorNotReady)
                continue;
            if (e != cudaSuccess) {
                cudaGetLastError();
                sl.status = HOUGH_ERR_CUDA;
            }
            sl.scatter_ns = 0;
            complete_slot(s, sl, now_ns());
            progress = true;
        }
        // admit
        for (Slot &sl : s->slots) {
            if (sl.busy || s->queue.empty())
                continue;
            sl.reqs.clear();
            sl.win_base.clear();
            sl.hit_base.clear();
            sl.W = sl.H = 0;
            sl.status = HOUGH_OK;
            while (!s->queue.empty()) {
                const Pending &p = s->queue.front();
                if (!sl.reqs.empty() && (sl.W + p.req.n_windows > s->cfg.slot_windows ||
                                         sl.H + p.n_hits > s->cfg.slot_hits))
                    break;
                sl.win_base.push_back(sl.W);
                sl.hit_base.push_back(sl.H);
                sl.W += p.req.n_windows;
                sl.H += p.n_hits;
                sl.reqs.push_back(p);
                s->queue.pop_front();
                s->queued.fetch_sub(1, std::memory_order_release);
            }
            sl.busy = true;
            s->in_flight += (int64_t)sl.reqs.size();
            s->st.batches += 1;
            lk.unlock();
            sl.launch_ns = now_ns();
            const int rc = launch_slot(s, sl);
            lk.lock();
            if (rc != HOUGH_OK) {
                cudaGetLastError();
                sl.status = rc;
                // let work already queued on the stream finish before the
                // mirrors are reused
                lk.unlock();
                cudaStreamSynchronize(sl.stream);
                cudaGetLastError();
                lk.lock();
                complete_slot(s, sl, now_ns());
            }
            progress = true;
        }
        bool any_busy = false;
        for (const Slot &sl : s->slots)
            any_busy = any_busy || sl.busy;
        if (s->stop && s->queue.empty() && !any_busy)
            break;
        if (progress)
            continue;
        if (any_busy) {
            // poll the GPU; requests queued meanwhile are admitted next pass
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        } else {
            // idle: poll the queue for a while before sleeping, since a
            // sleeping worker takes tens of microseconds to wake
            lk.unlock();
            const int64_t until = now_ns() + kIdleSpinNs;
            while (s->queued.load(std::memory_order_acquire) == 0 && !s->stopping.load() &&
                   now_ns() < until)
                std::this_thread::yield();
            lk.lock();
            s->cv_work.wait(lk, [s] { return s->stop || !s->queue.empty(); });
        }
    }
}

void free_slots(hough_server *s)
{
    for (Slot &sl : s->slots) {
        if (sl.stream)
            cudaStreamSynchronize(sl.stream);
        cudaFree(sl.d_in);
        cudaFree(sl.d_out);
        cudaFreeHost(sl.h_in);
        for (cudaEvent_t e : {sl.done, sl.t_start, sl.t_h2d, sl.t_kern})
            if (e)
                cudaEventDestroy(e);
        if (sl.stream)
            cudaStreamDestroy(sl.stream);
    }
    s->slots.clear();
    cudaGetLastError();
}

}  // namespace

extern "C" {

int64_t hough_server_clock_ns(void) { return now_ns(); }

int hough_server_create(hough_ctx *ctx, const hough_server_config *cfg, hough_server **out)
{
    if (!out)
        return HOUGH_ERR_INVALID_ARG;
    *out = nullptr;
    if (!ctx || !cfg || cfg->n_slots < 1 || cfg->n_slots > 16 || cfg->slot_windows < 1 ||
        cfg->slot_hits < 1 || cfg->max_queued < 1 || cfg->slot_windows >= (1ll << 30) ||
        cfg->slot_hits >= (1ll << 40) || (ctx->th.flags & HOUGH_FLAG_EXPORT_ACC))
        return HOUGH_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        cudaGetLastError();
        return HOUGH_ERR_CUDA;
    }
    hough_server *s = new (std::nothrow) hough_server();
    if (!s) {
        cudaSetDevice(prev);
        return HOUGH_ERR_ALLOC;
    }
    s->ctx = ctx;
    s->cfg = *cfg;
    s->max_peaks = ctx->th.max_peaks;
    // the server's launch shape: as given, else chosen per batch: one CTA of
    // 1024 threads per SM with 32-word-row tiles for small batches (they then
    // spread over every SM, and each window has the most warps), the
    // context's own shape (the library default, or what hough_set_launch or
    // hough_autotune chose for the workload) for batches of at least two
    // windows per SM
    s->saved_launch = ctx->launch;
    s->saved_auto = ctx->auto_launch;
    s->thr_auto = ctx->auto_launch;
    hough_launch want = cfg->launch;
    if (want.threads == 0 && want.word_rows == 0 && want.hit_stage == 0 && want.ctas_per_sm == 0) {
        const hough_launch lat{1024, 32, 2048, 1};
        s->thr_launch = ctx->launch;
        want = lat;
        if (hough_set_launch(ctx, &want) != HOUGH_OK)
            want = s->thr_launch;       // no room for the latency shape: one shape
        else
            s->per_batch = true;
        s->lat_launch = ctx->launch;
    }
    if (hough_set_launch(ctx, &want) != HOUGH_OK) {
        ctx->launch = s->saved_launch;
        ctx->auto_launch = s->saved_auto;
        delete s;
        cudaSetDevice(prev);
        return HOUGH_ERR_INVALID_ARG;
    }
    s->in_cap = in_layout(cfg->slot_windows, cfg->slot_hits).total;
    s->stage_cap = 8 * (size_t)(cfg->slot_windows + 1);
    s->out_cap = out_layout(cfg->slot_windows, cfg->slot_hits, s->max_peaks).total;
    s->slots.resize(cfg->n_slots);
    int rc = HOUGH_OK;
    for (Slot &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreate(&sl.done) != cudaSuccess || cudaEventCreate(&sl.t_start) != cudaSuccess ||
            cudaEventCreate(&sl.t_h2d) != cudaSuccess || cudaEventCreate(&sl.t_kern) != cudaSuccess) {
            rc = HOUGH_ERR_CUDA;
            break;
        }
        if (cudaMalloc(&sl.d_in, s->in_cap) != cudaSuccess ||
            cudaMalloc(&sl.d_out, s->out_cap) != cudaSuccess ||
            cudaHostAlloc(&sl.h_in, s->stage_cap, cudaHostAllocDefault) != cudaSuccess) {
            rc = HOUGH_ERR_ALLOC;
            break;
        }
        s->st.device_bytes += (int64_t)(s->in_cap + s->out_cap);
        s->st.host_bytes += (int64_t)s->stage_cap;
    }
    // one empty window per slot stream: the context sets up its per-stream
    // scheduling counters now, not in the middle of serving
    for (size_t k = 0; rc == HOUGH_OK && k < s->slots.size(); ++k) {
        Slot &sl = s->slots[k];
        sl.W = 1;
        sl.H = 0;
        rc = launch_slot(s, sl);
        if (rc == HOUGH_OK && cudaStreamSynchronize(sl.stream) != cudaSuccess)
            rc = HOUGH_ERR_CUDA;
        sl.W = 0;
    }
    if (rc != HOUGH_OK) {
        cudaGetLastError();
        free_slots(s);
        ctx->launch = s->saved_launch;
        ctx->auto_launch = s->saved_auto;
        delete s;
        cudaSetDevice(prev);
        return rc;
    }
    s->st.batches = 0;
    try {
        s->worker = std::thread(worker_loop, s);
    } catch (...) {
        free_slots(s);
        ctx->launch = s->saved_launch;
        ctx->auto_launch = s->saved_auto;
        delete s;
        cudaSetDevice(prev);
        return HOUGH_ERR_ALLOC;
    }
    cudaSetDevice(prev);
    *out = s;
    return HOUGH_OK;
}

int hough_server_submit(hough_server *s, const hough_request *req, uint64_t *ticket)
{
    if (!s || !req || !ticket || req->n_windows < 0 || !req->window_offsets)
        return HOUGH_ERR_INVALID_ARG;
    const int64_t nw = req->n_windows;
    const int64_t *o = req->window_offsets;
    if (o[0] != 0)
        return HOUGH_ERR_INVALID_ARG;
    for (int64_t j = 0; j < nw; ++j)
        if (o[j + 1] < o[j])
            return HOUGH_ERR_INVALID_ARG;
    const int64_t nh = o[nw];
    if (nh > 0 && (!req->in0 || !req->in1 || !req->out.hit_track || !req->out.track_hits))
        return HOUGH_ERR_INVALID_ARG;
    if (nw > 0 && (!req->out.n_peaks || !req->out.window_status ||
                   (s->max_peaks > 0 && !req->out.peaks)))
        return HOUGH_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (nw > s->cfg.slot_windows || nh > s->cfg.slot_hits) {
        s->st.rejected += 1;
        return HOUGH_ERR_UNSUPPORTED_SHAPE;
    }
    if ((int64_t)s->queue.size() >= s->cfg.max_queued) {
        s->st.rejected += 1;
        return HOUGH_ERR_BUSY;
    }
    Pending p;
    p.ticket = s->next_ticket++;
    p.req = *req;
    p.n_hits = nh;
    if (p.req.arrival_ns == 0)
        p.req.arrival_ns = now_ns();
    s->queue.push_back(p);
    s->queued.fetch_add(1, std::memory_order_release);
    s->live.insert(p.ticket);
    s->st.submitted += 1;
    *ticket = p.ticket;
    s->cv_work.notify_one();
    return HOUGH_OK;
}

int hough_server_wait(hough_server *s, uint64_t ticket, int64_t timeout_ms,
                      hough_request_result *res)
{
    if (!s)
        return HOUGH_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    if (!s->live.count(ticket))
        return HOUGH_ERR_INVALID_ARG;
    auto ready = [&] { return s->done.count(ticket) != 0; };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return HOUGH_ERR_TIMEOUT;
    if (res)
        *res = s->done[ticket];
    s->done.erase(ticket);
    s->live.erase(ticket);
    return HOUGH_OK;
}

int hough_server_poll(hough_server *s, hough_request_result *res, int64_t cap, int64_t *n)
{
    if (!s || !n || cap < 0 || (cap > 0 && !res))
        return HOUGH_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    int64_t k = 0;
    while (k < cap && !s->done_order.empty()) {
        const uint64_t t = s->done_order.front();
        s->done_order.pop_front();
        auto it = s->done.find(t);
        if (it == s->done.end())
            continue;                   // already taken by wait
        res[k++] = it->second;
        s->done.erase(it);
        s->live.erase(t);
    }
    *n = k;
    return HOUGH_OK;
}

int hough_server_drain(hough_server *s, int64_t timeout_ms)
{
    if (!s)
        return HOUGH_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto idle = [&] { return s->queue.empty() && s->in_flight == 0; };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, idle);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), idle))
        return HOUGH_ERR_TIMEOUT;
    return HOUGH_OK;
}

int hough_server_get_stats(hough_server *s, hough_server_stats *out)
{
    if (!s || !out)
        return HOUGH_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->queued = (int64_t)s->queue.size();
    out->in_flight = s->in_flight;
    return HOUGH_OK;
}

void hough_server_destroy(hough_server *s)
{
    if (!s)
        return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->stopping.store(true);
    }
    s->cv_work.notify_all();
    if (s->worker.joinable())
        s->worker.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->ctx->device);
    free_slots(s);
    s->ctx->launch = s->saved_launch;
    s->ctx->auto_launch = s->saved_auto;
    cudaSetDevice(prev);
    delete s;
}

}  // extern "C"
