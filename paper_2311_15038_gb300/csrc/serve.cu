// serve.cu -- a preview server with continuous batching (host runtime).
//
// The paper's server renders previews on request and streams the images to
// remote clients (Sec. III-C).  This runtime keeps many slicemaps resident and
// turns a stream of independent requests into device work:
//  * submit() queues a request (any view of any resident slicemap, any
//    transfer function) with its arrival time;
//  * a dispatcher thread admits requests in arrival order while their images
//    fit in the free part of a caller-provided device arena (admission by
//    memory), packs the admitted ones into batches and launches each batch as
//    one mctp_render_batch work-queue launch on one of up to 8 streams, so a
//    batch starts as soon as a stream is free while others are still on the
//    device (their work overlaps in the SMs: CTAs of the next launch start as
//    those of the previous one retire);
//  * completion is observed with events; poll() hands out finished requests
//    with their timestamps, release() returns the image memory.
// A per-view mode launches one mctp_render_views call per request instead, in
// arrival order, as the plain baseline.  No device code waits for the host.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "render_common.cuh"

namespace mctp {

int check_slicemap(const mctp_slicemap *sm);

namespace {

constexpr size_t kGranule = 256;
constexpr int kMaxInflight = 8;
constexpr int kMaxBatchViews = 4096;

size_t round_up(size_t v) { return (v + kGranule - 1) / kGranule * kGranule; }

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) in 256-byte granules with coalescing.
class Arena {
public:
    void reset(size_t begin, size_t end)
    {
        free_.clear();
        if (end > begin) free_[begin] = end - begin;
        used_ = 0;
        high_ = 0;
    }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = round_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes;
            const size_t at = it->first + bytes;
            free_.erase(it);
            if (rest) free_[at] = rest;
            used_ += bytes;
            high_ = std::max(high_, used_);
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = round_up(bytes);
        used_ -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
    size_t high_water() const { return high_; }

private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0, high_ = 0;
};

enum ReqState { kQueued, kAdmitted, kLaunched, kDone };

struct Request {
    mctp_view view;
    int32_t sm = 0, lut = 0;
    int state = kQueued;
    int status = MCTP_OK;
    bool has_img = false;  // its image memory is taken from the heap
    size_t img_off = 0, img_bytes = 0;
    double t_submit = 0, t_admit = 0, t_launch = 0, t_done = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint64_t *d_samples = nullptr;  // in the arena
    uint64_t *h_samples = nullptr;  // pinned host copy
    void *workspace = nullptr;      // in the arena, ws_bytes
    std::vector<uint64_t> tickets;
    bool busy = false;
};

}  // namespace
}  // namespace mctp

struct mctp_server {
    std::vector<mctp_slicemap> sms;
    const float *luts = nullptr;
    int32_t nluts = 0, nlut = 0;
    float alpha_stop = 0.99f;
    mctp_serve_params params{};
    uint8_t *arena = nullptr;
    size_t arena_bytes = 0, ws_bytes = 0, heap_begin = 0;
    int device = 0;

    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::unordered_map<uint64_t, mctp::Request> reqs;
    std::deque<uint64_t> queued, admitted;
    std::deque<uint64_t> finished;
    mctp::Arena heap;
    std::vector<mctp::Slot> slots;
    uint64_t samples_total = 0, launches = 0;
    int32_t fail_launches = 0;  // fault injection: launches still to fail
    std::thread worker;

    void run();
    bool launch(mctp::Slot &slot, std::vector<uint64_t> &batch);
};

using mctp::Request;
using mctp::Slot;

bool mctp_server::launch(Slot &slot, std::vector<uint64_t> &batch)
{
    // called without the lock: the batch's requests are owned by this thread
    const int n = int(batch.size());
    std::vector<mctp_view> v(n);
    std::vector<int32_t> vsm(n), vlut(n);
    std::vector<int64_t> off(n);
    {
        std::lock_guard<std::mutex> lock(mu);
        for (int i = 0; i < n; ++i) {
            const Request &r = reqs[batch[i]];
            v[i] = r.view;
            vsm[i] = r.sm;
            vlut[i] = r.lut;
            off[i] = int64_t(r.img_off / sizeof(float));
        }
    }
    int rc;
    bool inject = false;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (fail_launches > 0) {
            --fail_launches;
            inject = true;
        }
    }
    if (inject) {
        rc = MCTP_ECUDA;  // as a failed launch: nothing is enqueued
    } else if (params.mode == MCTP_SERVE_PER_VIEW) {
        rc = mctp_render_views(&sms[vsm[0]], &v[0], 1, luts + size_t(vlut[0]) * nlut * 4, nlut, alpha_stop,
                               reinterpret_cast<float *>(arena) + off[0], slot.d_samples, slot.stream);
    } else {
        rc = mctp::render_batch_impl(sms.data(), int32_t(sms.size()), v.data(), vsm.data(), vlut.data(), n, luts,
                                     nluts, nlut, alpha_stop, &params.tuning, reinterpret_cast<float *>(arena),
                                     off.data(), slot.d_samples, slot.workspace, ws_bytes, slot.stream,
                                     mctp::kBoundsIfRoom);
    }
    if (rc == MCTP_OK &&
        cudaMemcpyAsync(slot.h_samples, slot.d_samples, sizeof(uint64_t), cudaMemcpyDeviceToHost, slot.stream) !=
            cudaSuccess)
        rc = MCTP_ECUDA;
    if (rc == MCTP_OK && cudaEventRecord(slot.done, slot.stream) != cudaSuccess) rc = MCTP_ECUDA;
    const double t = mctp::now_s();
    std::lock_guard<std::mutex> lock(mu);
    for (uint64_t tk : batch) {
        Request &r = reqs[tk];
        r.t_launch = t;
        r.state = mctp::kLaunched;
        r.status = rc;
    }
    if (rc != MCTP_OK) {  // nothing in flight: finish the requests with the error
        for (uint64_t tk : batch) {
            Request &r = reqs[tk];
            r.state = mctp::kDone;
            r.t_done = t;
            finished.push_back(tk);
        }
        return false;
    }
    slot.tickets = batch;
    slot.busy = true;
    ++launches;
    return true;
}

void mctp_server::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lock(mu);
    for (;;) {
        // completions
        bool any_busy = false;
        for (Slot &s : slots) {
            if (!s.busy) continue;
            const cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaErrorNotReady) {
                any_busy = true;
                continue;
            }
            const double t = mctp::now_s();
            if (q == cudaSuccess) samples_total += *s.h_samples;
            for (uint64_t tk : s.tickets) {
                Request &r = reqs[tk];
                if (q != cudaSuccess) r.status = MCTP_ECUDA;
                r.state = mctp::kDone;
                r.t_done = t;
                finished.push_back(tk);
            }
            s.tickets.clear();
            s.busy = false;
        }
        if (stop && !any_busy) break;
        // admission in arrival order while the images fit
        while (!stop && !queued.empty()) {
            Request &r = reqs[queued.front()];
            size_t off = 0;
            if (!heap.alloc(r.img_bytes, &off)) break;
            r.img_off = off;
            r.has_img = true;
            r.state = mctp::kAdmitted;
            r.t_admit = mctp::now_s();
            admitted.push_back(queued.front());
            queued.pop_front();
        }
        // launches on free streams
        for (Slot &s : slots) {
            if (stop || admitted.empty()) break;
            if (s.busy) continue;
            const int cap = params.mode == MCTP_SERVE_PER_VIEW ? 1 : params.max_batch_views;
            std::vector<uint64_t> batch;
            while (!admitted.empty() && int(batch.size()) < cap) {
                batch.push_back(admitted.front());
                admitted.pop_front();
            }
            lock.unlock();
            launch(s, batch);
            lock.lock();
            any_busy = any_busy || s.busy;
        }
        if (any_busy) {
            lock.unlock();
            std::this_thread::yield();
            lock.lock();
        } else if (!stop && admitted.empty()) {
            // idle, or waiting for memory that only a release() can free
            cv.wait_for(lock, std::chrono::milliseconds(1));
        }
    }
}

extern "C" double mctp_now(void) { return mctp::now_s(); }

extern "C" int mctp_server_create(const mctp_slicemap *sms, int32_t nsm, const float *luts_rgba, int32_t nluts,
                                  int32_t nlut, float alpha_stop, void *arena, size_t arena_bytes,
                                  const mctp_serve_params *params, mctp_server **server)
{
    using namespace mctp;
    if (!server) return MCTP_EINVAL;
    *server = nullptr;
    if (!sms || nsm < 1 || !luts_rgba || nluts < 1 || nlut < 2 || nlut > 4096 || !params || !arena) return MCTP_EINVAL;
    if (!(alpha_stop > 0.0f && alpha_stop <= 1.0f)) return MCTP_EINVAL;
    if ((reinterpret_cast<uintptr_t>(arena) & (kGranule - 1)) || (reinterpret_cast<uintptr_t>(luts_rgba) & 15))
        return MCTP_EINVAL;
    const mctp_serve_params &p = *params;
    if (p.mode != MCTP_SERVE_BATCHED && p.mode != MCTP_SERVE_PER_VIEW) return MCTP_EINVAL;
    if (p.max_inflight < 1 || p.max_inflight > kMaxInflight || p.reserved != 0) return MCTP_EINVAL;
    if (p.mode == MCTP_SERVE_BATCHED && (p.max_batch_views < 1 || p.max_batch_views > kMaxBatchViews))
        return MCTP_EINVAL;
    for (int i = 0; i < nsm; ++i) {
        const int rc = check_slicemap(&sms[i]);
        if (rc != MCTP_OK) return rc;
        if (sms[i].dtype != sms[0].dtype) return MCTP_EUNSUPPORTED;
    }
    auto *S = new mctp_server();
    S->sms.assign(sms, sms + nsm);
    S->luts = luts_rgba;
    S->nluts = nluts;
    S->nlut = nlut;
    S->alpha_stop = alpha_stop;
    S->params = p;
    S->arena = static_cast<uint8_t *>(arena);
    S->arena_bytes = arena_bytes;
    const int nslots = p.max_inflight;
    // arena: per-stream sample counters, per-stream workspaces, then the image heap
    S->ws_bytes = p.mode == MCTP_SERVE_BATCHED ? round_up(batch_workspace_bound(sms, nsm, p.max_batch_views)) : 0;
    const size_t counters = round_up(size_t(nslots) * kGranule);
    S->heap_begin = counters + size_t(nslots) * S->ws_bytes;
    if (S->heap_begin >= arena_bytes) {
        delete S;
        return MCTP_ESIZE;
    }
    S->heap.reset(S->heap_begin, arena_bytes & ~(kGranule - 1));
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        return MCTP_ECUDA;
    }
    S->slots.resize(size_t(nslots));
    int rc = MCTP_OK;
    for (int i = 0; i < nslots && rc == MCTP_OK; ++i) {
        Slot &s = S->slots[size_t(i)];
        s.d_samples = reinterpret_cast<uint64_t *>(S->arena + size_t(i) * kGranule);
        s.workspace = S->arena + counters + size_t(i) * S->ws_bytes;
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaHostAlloc(reinterpret_cast<void **>(&s.h_samples), sizeof(uint64_t), cudaHostAllocDefault) !=
                cudaSuccess)
            rc = MCTP_ECUDA;
    }
    if (rc != MCTP_OK) {
        mctp_server_destroy(S);
        return rc;
    }
    S->worker = std::thread([S] { S->run(); });
    *server = S;
    return MCTP_OK;
}

extern "C" int mctp_server_submit(mctp_server *S, const mctp_view *view, int32_t slicemap, int32_t lut,
                                  uint64_t *ticket)
{
    using namespace mctp;
    if (!S || !view || !ticket) return MCTP_EINVAL;
    if (slicemap < 0 || slicemap >= int32_t(S->sms.size()) || lut < 0 || lut >= S->nluts) return MCTP_EINVAL;
    const mctp_slicemap &sm = S->sms[size_t(slicemap)];
    int rc = render::check_view(*view, sm.nlevels);
    if (rc != MCTP_OK) return rc;
    if (!render::level_fits_32bit(&sm, view->level)) return MCTP_ESIZE;
    const size_t img = size_t(view->width) * size_t(view->height) * 4 * sizeof(float);
    if (round_up(img) > S->arena_bytes - S->heap_begin) return MCTP_ESIZE;  // could never be admitted
    Request r;
    r.view = *view;
    r.sm = slicemap;
    r.lut = lut;
    r.img_bytes = img;
    r.t_submit = now_s();
    {
        std::lock_guard<std::mutex> lock(S->mu);
        const uint64_t tk = S->next_ticket++;
        S->reqs.emplace(tk, r);
        S->queued.push_back(tk);
        *ticket = tk;
    }
    S->cv.notify_one();
    return MCTP_OK;
}

extern "C" int mctp_server_poll(mctp_server *S, mctp_serve_result *results, int32_t max_results, int32_t *count)
{
    if (!S || !count || max_results < 0 || (max_results > 0 && !results)) return MCTP_EINVAL;
    std::lock_guard<std::mutex> lock(S->mu);
    int n = 0;
    while (n < max_results && !S->finished.empty()) {
        const uint64_t tk = S->finished.front();
        S->finished.pop_front();
        const Request &r = S->reqs[tk];
        mctp_serve_result &o = results[n++];
        o.ticket = tk;
        o.status = r.status;
        o.reserved = 0;
        o.image = r.has_img ? reinterpret_cast<float *>(S->arena + r.img_off) : nullptr;
        o.t_submit = r.t_submit;
        o.t_admit = r.t_admit;
        o.t_launch = r.t_launch;
        o.t_done = r.t_done;
    }
    *count = n;
    return MCTP_OK;
}

extern "C" int mctp_server_release(mctp_server *S, uint64_t ticket)
{
    if (!S) return MCTP_EINVAL;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end() || it->second.state != mctp::kDone) return MCTP_EINVAL;
        if (it->second.has_img) S->heap.release(it->second.img_off, it->second.img_bytes);
        S->reqs.erase(it);
    }
    S->cv.notify_one();
    return MCTP_OK;
}

extern "C" int mctp_server_cancel(mctp_server *S, uint64_t ticket)
{
    if (!S) return MCTP_EINVAL;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return MCTP_EINVAL;
        Request &r = it->second;
        std::deque<uint64_t> *q = r.state == mctp::kQueued ? &S->queued
                                  : r.state == mctp::kAdmitted ? &S->admitted : nullptr;
        if (!q) return MCTP_EINVAL;  // launched or finished: too late
        auto at = std::find(q->begin(), q->end(), ticket);
        if (at == q->end()) return MCTP_EINVAL;  // being launched by the server thread right now
        q->erase(at);
        if (r.has_img) {
            S->heap.release(r.img_off, r.img_bytes);
            r.has_img = false;
        }
        r.state = mctp::kDone;
        r.status = MCTP_ECANCELED;
        r.t_done = mctp::now_s();
        S->finished.push_back(ticket);
    }
    S->cv.notify_one();
    return MCTP_OK;
}

extern "C" int mctp_server_inject_launch_failures(mctp_server *S, int32_t n)
{
    if (!S || n < 0) return MCTP_EINVAL;
    std::lock_guard<std::mutex> lock(S->mu);
    S->fail_launches = n;
    return MCTP_OK;
}

extern "C" int mctp_server_stats(mctp_server *S, uint64_t *samples, uint64_t *launches, uint64_t *arena_high_water)
{
    if (!S) return MCTP_EINVAL;
    std::lock_guard<std::mutex> lock(S->mu);
    if (samples) *samples = S->samples_total;
    if (launches) *launches = S->launches;
    if (arena_high_water) *arena_high_water = S->heap.high_water();
    return MCTP_OK;
}

extern "C" int mctp_server_destroy(mctp_server *S)
{
    if (!S) return MCTP_EINVAL;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
    }
    S->cv.notify_one();
    if (S->worker.joinable()) S->worker.join();
    for (Slot &s : S->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.h_samples) cudaFreeHost(s.h_samples);
    }
    delete S;
    return MCTP_OK;
}
