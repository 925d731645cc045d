// hc_serve.cu -- the request loop: continuous batching of linear-layer
// requests over resident weights, admission by a device-memory budget.
//
// Threads: callers submit / wait / release from any host thread; one
// scheduler thread admits and launches batches; one completion thread
// retires them.  All shared state is guarded by hc_server::mu.
#include <algorithm>
#include <cstring>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hc_internal.h"

using namespace hc;
using Clock = std::chrono::steady_clock;

namespace {

constexpr size_t kPoolAlign = 256;

// first-fit allocator over one device range, coalescing on free
class Pool {
  public:
    void init(size_t bytes)
    {
        size_ = bytes;
        free_.clear();
        if (bytes) free_[0] = bytes;
    }
    size_t size() const { return size_; }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = round(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes, at = it->first + bytes;
            free_.erase(it);
            if (rest) free_[at] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = round(bytes);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    static size_t round(size_t b) { return (b + kPoolAlign - 1) / kPoolAlign * kPoolAlign; }

  private:
    size_t size_ = 0;
    std::map<size_t, size_t> free_;  // offset -> length
};

struct Layer {
    const hc_ctx *ctx;
    const hc_weights *w;
    size_t in_words, out_words;  // [I][2][L][N], [O][2][L][N]
    uint64_t products;
    bool blocked;
};

enum ReqState { RQ_QUEUED = 0, RQ_ADMITTED = 1, RQ_LAUNCHED = 2, RQ_DONE = 3 };

struct Request {
    uint32_t layer;
    const uint64_t *h_in;
    uint64_t *h_out;
    size_t off_a = 0, bytes_a = 0;  // input + NTT scratch
    size_t off_o = 0, bytes_o = 0;  // output
    bool has_a = false, has_o = false;
    int state = RQ_QUEUED;
    hc_status status = HC_OK;
    uint32_t batch_size = 0;
    Clock::time_point t_submit, t_launch, t_done;
};

struct Batch {
    std::vector<uint64_t> tickets;
    int slot;
    hc_status status;
};

constexpr int kDegrees = 3;  // ring degrees 2^12, 2^13, 2^14: one stream class each

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct hc_server {
    uint32_t magic;
    int device;
    hc_server_config cfg;
    void *d_pool = nullptr;
    Pool pool;
    std::vector<Layer> layers;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done, cv_complete;
    std::unordered_map<uint64_t, Request> reqs;
    std::deque<uint64_t> queued, admitted;
    std::vector<Batch *> inflight;
    // per stream slot: one stream per ring degree (smaller degrees at higher CUDA
    // stream priority unless HC_SERVER_EQUAL_PRIORITY), their per-limb side
    // streams, the batch's completion event, the device word its bounded waits
    // report timeouts into and its pinned host copy, and fused-form counters
    std::vector<cudaStream_t> streams;   // [slot * kDegrees + logN - 12]
    std::vector<hc::SidePool> sides;     // same index
    std::vector<cudaEvent_t> events;
    int *d_err = nullptr;                // [max_inflight]
    int *h_err = nullptr;                // [max_inflight], pinned
    std::vector<uint32_t *> ctrs;        // per stream slot: fused-form counters
    size_t ctr_words = 1u << 18;
    std::vector<bool> slot_busy;
    uint64_t next_ticket = 1;
    bool stopping = false, sched_exited = false, joined = false;
    hc_server_stats st{};
    std::thread sched, compl_;
};

namespace {

inline bool server_ok(const hc_server *s) { return s && s->magic == kMagicServer; }

uint64_t *pool_ptr(hc_server *s, size_t off) { return (uint64_t *)((char *)s->d_pool + off); }

// reserve a request's buffers; false if the pool cannot hold them now
bool try_admit(hc_server *s, Request &r)
{
    size_t a = 0, o = 0;
    if (!s->pool.alloc(r.bytes_a, &a)) return false;
    if (!s->pool.alloc(r.bytes_o, &o)) {
        s->pool.release(a, r.bytes_a);
        return false;
    }
    r.off_a = a;
    r.off_o = o;
    r.has_a = r.has_o = true;
    s->st.bytes_in_use += Pool::round(r.bytes_a) + Pool::round(r.bytes_o);
    if (s->st.bytes_in_use > s->st.peak_bytes_in_use) s->st.peak_bytes_in_use = s->st.bytes_in_use;
    return true;
}

void free_a(hc_server *s, Request &r)
{
    if (!r.has_a) return;
    s->pool.release(r.off_a, r.bytes_a);
    s->st.bytes_in_use -= Pool::round(r.bytes_a);
    r.has_a = false;
}

void free_o(hc_server *s, Request &r)
{
    if (!r.has_o) return;
    s->pool.release(r.off_o, r.bytes_o);
    s->st.bytes_in_use -= Pool::round(r.bytes_o);
    r.has_o = false;
}

// enqueue one batch (all of one ring degree) on its slot's stream for that
// degree, then the batch's timeout word to the host (called without the lock held)
hc_status enqueue_batch(hc_server *s, const std::vector<ConvJob> &jobs, const std::vector<const uint64_t *> &h_in,
                        const std::vector<uint64_t *> &h_out, const std::vector<size_t> &in_bytes,
                        const std::vector<size_t> &out_bytes, int slot, cudaStream_t st)
{
    const size_t k = (size_t)slot * kDegrees + (jobs[0].ctx->logN - 12);
    LaunchScope scope(s->d_err + slot, &s->sides[k]);
    for (size_t i = 0; i < jobs.size(); ++i)
        HC_CUDA_TRY(cudaMemcpyAsync((void *)jobs[i].in, h_in[i], in_bytes[i], cudaMemcpyHostToDevice, st));
    hc_status rc = launch_conv_jobs(jobs.data(), jobs.size(), st, s->ctrs[slot], s->ctr_words);
    if (rc != HC_OK) return rc;
    if (s->cfg.selftest_wait_limit) {  // one wait that nothing completes: the batch must report a timeout
        rc = launch_wait_selftest(jobs[0].ctx, s->cfg.selftest_wait_limit, st);
        if (rc != HC_OK) return rc;
    }
    for (size_t i = 0; i < jobs.size(); ++i)
        if (h_out[i])
            HC_CUDA_TRY(cudaMemcpyAsync(h_out[i], jobs[i].out, out_bytes[i], cudaMemcpyDeviceToHost, st));
    HC_CUDA_TRY(cudaMemcpyAsync(s->h_err + slot, s->d_err + slot, sizeof(int), cudaMemcpyDeviceToHost, st));
    HC_CUDA_TRY(cudaMemsetAsync(s->d_err + slot, 0, sizeof(int), st));
    return HC_OK;
}

void scheduler_main(hc_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        while (!s->queued.empty()) {  // admission in arrival order
            Request &r = s->reqs[s->queued.front()];
            if (!try_admit(s, r)) break;
            r.state = RQ_ADMITTED;
            s->admitted.push_back(s->queued.front());
            s->queued.pop_front();
        }
        int slot = -1;
        for (size_t i = 0; i < s->slot_busy.size(); ++i)
            if (!s->slot_busy[i]) {
                slot = (int)i;
                break;
            }
        if (!s->admitted.empty() && slot >= 0) {
            Batch *b = new Batch();
            b->slot = slot;
            s->slot_busy[slot] = true;
            std::vector<ConvJob> jobs;
            std::vector<const uint64_t *> h_in;
            std::vector<uint64_t *> h_out;
            std::vector<size_t> in_bytes, out_bytes;
            const Clock::time_point now = Clock::now();
            // the batch: the oldest admitted request and the admitted requests of its
            // ring degree after it, in arrival order (the others keep their place)
            const uint32_t logN = s->layers[s->reqs[s->admitted.front()].layer].ctx->logN;
            for (auto it = s->admitted.begin(); it != s->admitted.end() && b->tickets.size() < s->cfg.max_batch;) {
                if (s->layers[s->reqs[*it].layer].ctx->logN != logN) {
                    ++it;
                    continue;
                }
                const uint64_t t = *it;
                it = s->admitted.erase(it);
                Request &r = s->reqs[t];
                const Layer &ly = s->layers[r.layer];
                r.state = RQ_LAUNCHED;
                r.t_launch = now;
                b->tickets.push_back(t);
                uint64_t *a = pool_ptr(s, r.off_a);
                jobs.push_back(ConvJob{ly.ctx, ly.w, a, pool_ptr(s, r.off_o), a + ly.in_words, ly.blocked});
                h_in.push_back(r.h_in);
                h_out.push_back(r.h_out);
                in_bytes.push_back(ly.in_words * sizeof(uint64_t));
                out_bytes.push_back(ly.out_words * sizeof(uint64_t));
            }
            for (uint64_t t : b->tickets) s->reqs[t].batch_size = (uint32_t)b->tickets.size();
            if (b->tickets.size() > s->st.max_batch_seen) s->st.max_batch_seen = (uint32_t)b->tickets.size();
            ++s->st.batches;
            lk.unlock();
            cudaStream_t st = s->streams[(size_t)slot * kDegrees + (logN - 12)];
            b->status = enqueue_batch(s, jobs, h_in, h_out, in_bytes, out_bytes, slot, st);
            cudaError_t e = cudaEventRecord(s->events[slot], st);
            if (e != cudaSuccess && b->status == HC_OK) b->status = cuda_error(e, "cudaEventRecord");
            lk.lock();
            s->inflight.push_back(b);
            s->cv_complete.notify_one();
            continue;
        }
        if (s->stopping && s->queued.empty() && s->admitted.empty()) break;
        if (s->stopping && s->admitted.empty() && s->inflight.empty()) {
            // shutting down with requests that wait for memory only a release could free: fail them
            const Clock::time_point now = Clock::now();
            for (uint64_t t : s->queued) {
                Request &r = s->reqs[t];
                r.state = RQ_DONE;
                r.status = HC_ERR_BUDGET;
                r.t_launch = r.t_done = now;
                ++s->st.completed;
            }
            s->queued.clear();
            s->cv_done.notify_all();
            continue;
        }
        s->cv_sched.wait(lk);
    }
    s->sched_exited = true;
    s->cv_complete.notify_one();
}

void completion_main(hc_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        if (s->inflight.empty()) {
            if (s->sched_exited) return;
            s->cv_complete.wait(lk);
            continue;
        }
        std::vector<Batch *> snap = s->inflight;
        lk.unlock();
        std::vector<Batch *> ready;
        for (Batch *b : snap) {
            const cudaError_t e = cudaEventQuery(s->events[b->slot]);
            if (e == cudaErrorNotReady) continue;
            if (e != cudaSuccess && b->status == HC_OK) b->status = cuda_error(e, "batch execution");
            if (e == cudaSuccess && s->h_err[b->slot]) {  // a bounded device wait ran out: results unspecified
                if (b->status == HC_OK) b->status = HC_ERR_TIMEOUT;
                s->h_err[b->slot] = 0;
            }
            ready.push_back(b);
        }
        const Clock::time_point now = Clock::now();
        if (ready.empty()) std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
        for (Batch *b : ready) {
            for (uint64_t t : b->tickets) {
                Request &r = s->reqs[t];
                r.state = RQ_DONE;
                r.status = b->status;
                r.t_done = now;
                free_a(s, r);
                if (r.h_out || b->status != HC_OK) free_o(s, r);
                ++s->st.completed;
                if (b->status == HC_OK) s->st.products += s->layers[r.layer].products;
            }
            s->slot_busy[b->slot] = false;
            s->inflight.erase(std::find(s->inflight.begin(), s->inflight.end(), b));
            delete b;
        }
        if (!ready.empty()) {
            s->cv_done.notify_all();
            s->cv_sched.notify_one();
        }
    }
}

void fill_info(const Request &r, hc_request_info *info)
{
    if (!info) return;
    info->status = r.status;
    info->batch_size = r.batch_size;
    info->queue_ms = ms_between(r.t_submit, r.t_launch);
    info->latency_ms = ms_between(r.t_submit, r.t_done);
}

}  // namespace

namespace hc {
void server_destroy(hc_server *s)
{
    hc_server_shutdown(s);
    DeviceGuard g(s->device);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    for (auto &sp : s->sides) {
        for (cudaStream_t st : sp.st) cudaStreamDestroy(st);
        for (cudaEvent_t e : sp.ev) cudaEventDestroy(e);
    }
    for (cudaEvent_t e : s->events) cudaEventDestroy(e);
    dev_free_persistent(s->d_err);
    if (s->h_err) cudaFreeHost(s->h_err);
    for (uint32_t *c : s->ctrs) dev_free_persistent(c);
    dev_free_persistent(s->d_pool);
    s->magic = kMagicDead;
    delete s;
}
}  // namespace hc

extern "C" {

hc_status hc_server_create(const hc_server_config *cfg, hc_server **out)
{
    if (!out) return set_error(HC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    hc_server_config c{};
    if (cfg) c = *cfg;
    if (c.budget_bytes == 0) c.budget_bytes = (size_t)32 << 30;
    if (c.max_batch == 0) c.max_batch = 64;
    if (c.max_inflight == 0) c.max_inflight = 4;
    if (c.selftest_wait_limit > (1u << 20)) return set_error(HC_ERR_INVALID_ARG, "selftest_wait_limit <= 2^20");
    if (c.max_batch > 4096 || c.max_inflight > 16)
        return set_error(HC_ERR_INVALID_ARG, "max_batch <= 4096 and max_inflight <= 16");
    int dev = 0;
    HC_CUDA_TRY(cudaGetDevice(&dev));
    hc_server *s = new (std::nothrow) hc_server();
    if (!s) return set_error(HC_ERR_OOM, "host allocation failed");
    s->magic = kMagicServer;
    s->device = dev;
    s->cfg = c;
    s->joined = true;  // nothing to join until the threads start
    s->d_pool = dev_alloc_persistent(c.budget_bytes);
    if (!s->d_pool) {
        hc::server_destroy(s);
        return set_error(HC_ERR_OOM, "cannot reserve a %zu-byte pool", c.budget_bytes);
    }
    s->pool.init(c.budget_bytes);
    s->st.pool_bytes = c.budget_bytes;
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        least = greatest = 0;
    }
    s->d_err = (int *)dev_alloc_persistent(c.max_inflight * sizeof(int));
    cudaError_t e0 = s->d_err ? cudaMemset(s->d_err, 0, c.max_inflight * sizeof(int)) : cudaErrorMemoryAllocation;
    if (e0 == cudaSuccess) e0 = cudaHostAlloc((void **)&s->h_err, c.max_inflight * sizeof(int), cudaHostAllocDefault);
    if (e0 != cudaSuccess) {
        s->h_err = nullptr;
        hc::server_destroy(s);
        return cuda_error(e0, "server error words");
    }
    memset(s->h_err, 0, c.max_inflight * sizeof(int));
    s->sides.resize((size_t)c.max_inflight * kDegrees);
    for (uint32_t i = 0; i < c.max_inflight; ++i) {
        cudaError_t e = cudaSuccess;
        for (int d = 0; d < kDegrees && e == cudaSuccess; ++d) {
            // ring degree 2^(12+d): smaller rings (shorter requests) at higher priority
            int prio = least - (kDegrees - 1 - d);
            if (prio < greatest) prio = greatest;
            if (c.flags & HC_SERVER_EQUAL_PRIORITY) prio = least;
            cudaStream_t st = nullptr;
            e = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio);
            if (e == cudaSuccess) s->streams.push_back(st);
            s->sides[(size_t)i * kDegrees + d].priority = prio;
        }
        cudaEvent_t ev = nullptr;
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) s->events.push_back(ev);
        uint32_t *ctr = e == cudaSuccess ? (uint32_t *)dev_alloc_persistent(s->ctr_words * sizeof(uint32_t)) : nullptr;
        if (ctr) s->ctrs.push_back(ctr);
        if (e == cudaSuccess && !ctr) e = cudaErrorMemoryAllocation;
        if (e != cudaSuccess) {
            hc::server_destroy(s);
            return cuda_error(e, "server stream/event creation");
        }
    }
    s->slot_busy.assign(c.max_inflight, false);
    try {
        s->joined = false;
        s->sched = std::thread(scheduler_main, s);
        s->compl_ = std::thread(completion_main, s);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stopping = true;
            s->sched_exited = !s->sched.joinable();
        }
        s->cv_sched.notify_all();
        s->cv_complete.notify_all();
        if (s->sched.joinable()) s->sched.join();
        if (s->compl_.joinable()) s->compl_.join();
        s->joined = true;
        hc::server_destroy(s);
        return set_error(HC_ERR_OOM, "cannot start server threads");
    }
    *out = s;
    return HC_OK;
}

hc_status hc_server_add_layer(hc_server *s, const hc_ctx *ctx, const hc_weights *w, uint32_t *layer_id)
{
    if (!server_ok(s) || !layer_id) return set_error(HC_ERR_INVALID_ARG, "invalid server or layer_id");
    if (!ctx || ctx->magic != kMagicCtx || !w || w->magic != kMagicWeights || w->ctx != ctx)
        return set_error(HC_ERR_INVALID_ARG, "invalid context or weights");
    if (ctx->device != s->device) return set_error(HC_ERR_INVALID_ARG, "context on another device");
    if (w->mode != HC_WEIGHTS_NTT_OFFLINE)
        return set_error(HC_ERR_UNSUPPORTED, "the server needs NTT-preprocessed (offline) weights");
    Layer ly;
    ly.ctx = ctx;
    ly.w = w;
    ly.in_words = (size_t)w->I * 2 * ctx->L * ctx->N;
    ly.out_words = (size_t)w->O * 2 * ctx->L * ctx->N;
    ly.products = (uint64_t)w->Mp * w->G * w->B;
    ly.blocked = conv_job_blocked(ctx, w);
    std::lock_guard<std::mutex> lk(s->mu);
    *layer_id = (uint32_t)s->layers.size();
    s->layers.push_back(ly);
    return HC_OK;
}

hc_status hc_server_submit(hc_server *s, uint32_t layer_id, const uint64_t *h_ct_in, uint64_t *h_ct_out,
                           uint64_t *ticket)
{
    if (!server_ok(s) || !ticket || !h_ct_in) return set_error(HC_ERR_INVALID_ARG, "invalid server, ticket or input");
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stopping) return set_error(HC_ERR_INVALID_ARG, "server is shutting down");
    if (layer_id >= s->layers.size()) return set_error(HC_ERR_INVALID_ARG, "unknown layer %u", layer_id);
    const Layer &ly = s->layers[layer_id];
    Request r;
    r.layer = layer_id;
    r.h_in = h_ct_in;
    r.h_out = h_ct_out;
    r.bytes_a = 2 * ly.in_words * sizeof(uint64_t);
    r.bytes_o = ly.out_words * sizeof(uint64_t);
    if (Pool::round(r.bytes_a) + Pool::round(r.bytes_o) > s->pool.size()) {
        ++s->st.refused;
        return set_error(HC_ERR_BUDGET, "request needs %zu bytes, pool holds %zu",
                         Pool::round(r.bytes_a) + Pool::round(r.bytes_o), s->pool.size());
    }
    r.t_submit = Clock::now();
    const uint64_t t = s->next_ticket++;
    s->reqs.emplace(t, r);
    s->queued.push_back(t);
    ++s->st.submitted;
    *ticket = t;
    lk.unlock();
    s->cv_sched.notify_one();
    return HC_OK;
}

hc_status hc_server_wait(hc_server *s, uint64_t ticket, double timeout_s, hc_request_info *info)
{
    if (!server_ok(s)) return set_error(HC_ERR_INVALID_ARG, "invalid server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(HC_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    auto done = [&] { return it->second.state == RQ_DONE; };
    if (timeout_s < 0) {
        s->cv_done.wait(lk, done);
    } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) {
        return set_error(HC_ERR_TIMEOUT, "request %llu not done", (unsigned long long)ticket);
    }
    fill_info(it->second, info);
    return HC_OK;
}

hc_status hc_server_poll(hc_server *s, uint64_t ticket, int *done, hc_request_info *info)
{
    if (!server_ok(s) || !done) return set_error(HC_ERR_INVALID_ARG, "invalid server or done");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(HC_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    *done = it->second.state == RQ_DONE;
    if (*done) fill_info(it->second, info);
    return HC_OK;
}

hc_status hc_server_result(hc_server *s, uint64_t ticket, const uint64_t **d_ct_out)
{
    if (!server_ok(s) || !d_ct_out) return set_error(HC_ERR_INVALID_ARG, "invalid server or output");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end() || it->second.state != RQ_DONE || !it->second.has_o)
        return set_error(HC_ERR_INVALID_ARG, "ticket %llu has no device result", (unsigned long long)ticket);
    *d_ct_out = pool_ptr(s, it->second.off_o);
    return HC_OK;
}

hc_status hc_server_fetch(hc_server *s, uint64_t ticket, uint64_t *h_ct_out)
{
    if (!server_ok(s) || !h_ct_out) return set_error(HC_ERR_INVALID_ARG, "invalid server or output");
    const uint64_t *src = nullptr;
    size_t bytes = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end() || it->second.state != RQ_DONE || !it->second.has_o)
            return set_error(HC_ERR_INVALID_ARG, "ticket %llu has no device result", (unsigned long long)ticket);
        src = pool_ptr(s, it->second.off_o);
        bytes = s->layers[it->second.layer].out_words * sizeof(uint64_t);
    }
    DeviceGuard g(s->device);
    HC_CUDA_TRY(cudaMemcpy(h_ct_out, src, bytes, cudaMemcpyDeviceToHost));
    return HC_OK;
}

hc_status hc_server_release(hc_server *s, uint64_t ticket)
{
    if (!server_ok(s)) return set_error(HC_ERR_INVALID_ARG, "invalid server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end() || it->second.state != RQ_DONE)
            return set_error(HC_ERR_INVALID_ARG, "ticket %llu unknown or not done", (unsigned long long)ticket);
        free_o(s, it->second);
        s->reqs.erase(it);
    }
    s->cv_sched.notify_one();
    return HC_OK;
}

hc_status hc_server_stats_get(hc_server *s, hc_server_stats *out)
{
    if (!server_ok(s) || !out) return set_error(HC_ERR_INVALID_ARG, "invalid server or output");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    return HC_OK;
}

hc_status hc_server_shutdown(hc_server *s)
{
    if (!server_ok(s)) return set_error(HC_ERR_INVALID_ARG, "invalid server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->joined) return HC_OK;
        s->stopping = true;
    }
    s->cv_sched.notify_all();
    if (s->sched.joinable()) s->sched.join();
    s->cv_complete.notify_all();
    if (s->compl_.joinable()) s->compl_.join();
    std::lock_guard<std::mutex> lk(s->mu);
    s->joined = true;
    return HC_OK;
}

}  // extern "C"
