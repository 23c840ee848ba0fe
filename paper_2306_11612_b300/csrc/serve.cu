// Serving loop of include/dvl_serve.h: resident data sets, per-data-set
// request queues, memory- and slot-based admission, continuous batching
// through dvl_update_batch on one stream per data set.  Host code only; the
// GPU work is the batched kernels (batch.cu, bins.cu).
//
// One scheduler thread owns every context.  A batch's alpha tables and
// results live in pinned buffers of its data set; after the batch and the
// copies of its bins are queued on the data set's stream, an event follows
// them.  While batches are in flight the scheduler polls those events
// (no thread hand-off between the device finishing and the results being
// handed out) and keeps launching; with nothing in flight it polls the queues
// for a short while before it sleeps, and a waiting caller likewise polls its
// request's flag for a short while before it sleeps.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/dvl.h"
#include "../../include/dvl_serve.h"
#include "dvl_internal.h"

using namespace dvl;

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

uint32_t pow2_ceil(uint32_t k)
{
    uint32_t b = 1;
    while (b < k) b <<= 1;
    return b;
}

struct Request {
    uint64_t id = 0;
    uint32_t ds = 0, W = 0;
    std::vector<float> alpha;           // M x T
    double t_submit = 0, t_done = 0;
    bool done = false;
    std::atomic<bool> ready{false};     // done, readable without the lock (set after `done`)
    int status = DVL_OK;
    std::vector<float> mean, mn, mx, y;  // M x W
    std::vector<double> sum;
    std::vector<uint32_t> count;        // W
};

template <typename T>
struct Pinned {                          // grow-only pinned host buffer
    T* p = nullptr;
    size_t cap = 0;
    cudaError_t reserve(size_t n)
    {
        if (n <= cap) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&p), n * sizeof(T), cudaHostAllocDefault);
        if (e == cudaSuccess) cap = n;
        return e;
    }
    ~Pinned()
    {
        if (p) cudaFreeHost(p);
    }
};

struct Dataset {
    dvl_ctx* ctx = nullptr;
    uint64_t n = 0;
    uint32_t M = 0;
    uint64_t resident = 0;               // estimated bytes of data and tables
    uint64_t bytes_per_tf = 0;           // estimated batch-buffer bytes per TF slot
    uint32_t cap_tf = 0;                 // TF slots the context's batch buffers hold
    std::deque<Request*> queue;
    // batch on the GPU
    bool busy = false;
    cudaEvent_t done_ev = nullptr;       // after the batch's result copies, on its stream
    std::vector<Request*> batch;
    uint32_t K = 0;
    Pinned<float> h_alpha, r_mean, r_mn, r_mx, r_y;
    Pinned<double> r_sum;
    Pinned<uint32_t> r_count;
    std::vector<uint32_t> pair_tf, pair_w;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;   // the batch's kernels: before and after, on its stream
    Pinned<unsigned long long> r_stamps;        // device clock at its first kernel's start, last kernel's end
};

// One finished batch on the device timeline: its data set, real requests,
// the events around its kernels and the device-clock stamps of their run.
struct Span {
    uint32_t ds, k;
    cudaEvent_t ev0, ev1;
    unsigned long long ns0, ns1;
};

constexpr size_t MAX_SPANS = 1u << 20;

}  // namespace

struct dvl_server {
    int device = 0;
    dvl_server_config cfg{};
    std::vector<std::unique_ptr<Dataset>> ds;
    std::unordered_map<uint64_t, Request*> reqs;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::thread th;
    bool stop = false;
    uint64_t next_id = 1;
    std::atomic<uint64_t> queued_total{0};   // requests ever queued (the scheduler polls it without the lock)
    uint64_t mem_used = 0;
    int inflight = 0;
    std::string last_error;
    // statistics
    std::vector<double> lat;
    uint64_t submitted = 0, completed = 0, failed = 0, batches = 0, batch_reqs = 0, cells = 0;
    uint32_t max_batch_seen = 0;
    double t_first = 0, t_last = 0;
    // device timeline of the finished batches (events are recycled through `free_ev`)
    std::vector<Span> spans;
    std::vector<cudaEvent_t> free_ev;
};

namespace {

int sfail(dvl_server* s, int code, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int sfail(dvl_server* s, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    s->last_error = buf;
    return code;
}

// Estimated device bytes of one resident data set: input and sorted fields,
// levels, order and sort scratch, the value tables (prefix sums within and
// over blocks of steps, per-step and in-block min/max, the blocks' sparse
// table), the per-cell TF entries with their level row and the single-update
// scan state.
uint64_t resident_bytes(uint64_t n, uint32_t M)
{
    const uint64_t pad = (n + PAD - 1) / PAD * PAD;
    const uint64_t steps = (n + STEP - 1) / STEP, tiles = (n + TILE - 1) / TILE, chunks = tiles * WARPS;
    const uint64_t blocks = (steps + VT_BLOCK - 1) / VT_BLOCK;
    const uint64_t tables = (uint64_t)M * ((steps + 1) * 16 + (blocks + 1) * 16 + steps * 3 * 8 +
                                           (uint64_t)value_table_levels(blocks) * blocks * 8 +
                                           value_table_segments(blocks) * 16);
    return pad * (9ull * M + 2) + n * (4 + 8 + 8 + 4) + tables + tiles * 8 + chunks * 8 + chunks * STEPS * 8;
}

// Estimated batch-buffer bytes per TF slot (one pair of width W per slot).
uint64_t per_tf_bytes(uint64_t n, uint32_t M, uint32_t T, uint32_t W)
{
    const uint64_t tiles = (n + TILE - 1) / TILE, chunks = tiles * WARPS;
    return sizeof(UpdateConsts) + (uint64_t)M * T * 4 + tiles * 8 + chunks * 8 + chunks * STEPS * 8 +
           (uint64_t)M * W * (8 + 4 * 4) + (uint64_t)W * 4 + (uint64_t)(W + 1) * (8 + 1 + 2ull * M * 24) +
           sizeof(PairDesc);
}

void finish_request(dvl_server* s, Request* r, int status, double t)
{
    r->status = status;
    r->done = true;
    r->ready.store(true, std::memory_order_release);
    r->t_done = t;
    if (status == DVL_OK) {
        ++s->completed;
        s->lat.push_back((t - r->t_submit) * 1e3);
        s->cells += s->ds[r->ds]->n;
        s->t_last = std::max(s->t_last, t);
    } else {
        ++s->failed;
    }
}

// Hands a finished batch's results to its requests (lock held; no CUDA
// calls: rc is the data set's dvl_sync status, taken without the lock).
void complete_batch(dvl_server* s, Dataset* d, int rc)
{
    const double t = now_s();
    uint64_t bin_off = 0, cnt_off = 0;
    for (size_t i = 0; i < d->batch.size(); ++i) {
        Request* r = d->batch[i];
        const uint64_t MW = (uint64_t)d->M * r->W;
        if (rc == DVL_OK) {
            r->mean.assign(d->r_mean.p + bin_off, d->r_mean.p + bin_off + MW);
            r->mn.assign(d->r_mn.p + bin_off, d->r_mn.p + bin_off + MW);
            r->mx.assign(d->r_mx.p + bin_off, d->r_mx.p + bin_off + MW);
            r->y.assign(d->r_y.p + bin_off, d->r_y.p + bin_off + MW);
            r->sum.assign(d->r_sum.p + bin_off, d->r_sum.p + bin_off + MW);
            r->count.assign(d->r_count.p + cnt_off, d->r_count.p + cnt_off + r->W);
        }
        finish_request(s, r, rc, t);
        bin_off += MW;
        cnt_off += r->W;
    }
    if (d->ev0 && d->ev1) {
        if (rc == DVL_OK && s->spans.size() < MAX_SPANS) {
            uint32_t idx = 0;
            for (size_t i = 0; i < s->ds.size(); ++i)
                if (s->ds[i].get() == d) idx = (uint32_t)i;
            s->spans.push_back(Span{idx, (uint32_t)d->batch.size(), d->ev0, d->ev1, d->r_stamps.p[0],
                                    d->r_stamps.p[1]});
        } else {
            s->free_ev.push_back(d->ev0);
            s->free_ev.push_back(d->ev1);
        }
        d->ev0 = d->ev1 = nullptr;
    }
    d->batch.clear();
    d->busy = false;
    --s->inflight;
    s->cv_done.notify_all();
}

// Launches the next batch of data set d if admission allows (lock held on
// entry and exit; released around the library calls).
bool launch_batch(dvl_server* s, Dataset* d, std::unique_lock<std::mutex>& lk)
{
    const uint32_t queued = (uint32_t)d->queue.size();
    const uint32_t k = dvl_serve_admit(queued, s->cfg.max_batch, d->cap_tf, d->bytes_per_tf, s->mem_used,
                                       s->cfg.mem_budget);
    if (k == 0) {
        // not even one TF slot fits, and device memory held by the server is
        // never released before destroy: the head request can never run
        Request* r = d->queue.front();
        d->queue.pop_front();
        finish_request(s, r, DVL_ERR_NOMEM, now_s());
        s->cv_done.notify_all();
        return false;
    }
    const uint32_t K = dvl_serve_bucket(k, s->cfg.max_batch);
    if (K > d->cap_tf) {
        s->mem_used += (uint64_t)(K - d->cap_tf) * d->bytes_per_tf;
        d->cap_tf = K;
    }
    d->batch.assign(d->queue.begin(), d->queue.begin() + k);
    d->queue.erase(d->queue.begin(), d->queue.begin() + k);
    d->busy = true;
    d->K = K;
    ++s->inflight;
    ++s->batches;
    s->batch_reqs += k;
    s->max_batch_seen = std::max(s->max_batch_seen, k);
    const uint32_t M = d->M, T = s->cfg.n_entries;
    // one pair per slot (padding slots repeat the first request's tables and
    // have width 1)
    uint64_t nb = 0, nc = 0;
    d->pair_tf.resize(K);
    d->pair_w.resize(K);
    for (uint32_t i = 0; i < K; ++i) {
        d->pair_tf[i] = i;
        d->pair_w[i] = i < k ? d->batch[i]->W : 1u;
        nb += (uint64_t)M * d->pair_w[i];
        nc += d->pair_w[i];
    }
    dvl_params prm = s->cfg.params;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    for (int i = 0; i < 2 && !s->free_ev.empty(); ++i) {
        ev[i] = s->free_ev.back();
        s->free_ev.pop_back();
    }
    // No CUDA call while the lock is held: pinned allocation, the library
    // calls and the stream callback may all wait on device work whose host
    // callbacks take the lock.  The batch's requests stay alive (not done)
    // and the data set's buffers belong to this thread until it is finished.
    lk.unlock();
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2; ++i)
        if (!ev[i] && cudaEventCreate(&ev[i]) != cudaSuccess) {
            cudaGetLastError();
            ev[i] = nullptr;
        }
    cudaStream_t st = static_cast<cudaStream_t>(dvl_stream(d->ctx));
    const bool timed = ev[0] && ev[1] && cudaEventRecord(ev[0], st) == cudaSuccess;
    if (e == cudaSuccess) e = d->h_alpha.reserve((size_t)K * M * T);
    if (e == cudaSuccess) e = d->r_mean.reserve(nb);
    if (e == cudaSuccess) e = d->r_mn.reserve(nb);
    if (e == cudaSuccess) e = d->r_mx.reserve(nb);
    if (e == cudaSuccess) e = d->r_y.reserve(nb);
    if (e == cudaSuccess) e = d->r_sum.reserve(nb);
    if (e == cudaSuccess) e = d->r_count.reserve(nc);
    if (e == cudaSuccess) e = d->r_stamps.reserve(2);
    for (uint32_t i = 0; i < K && e == cudaSuccess; ++i)
        std::memcpy(d->h_alpha.p + (size_t)i * M * T, d->batch[i < k ? i : 0]->alpha.data(), (size_t)M * T * 4);
    int rc = e == cudaSuccess ? DVL_OK : DVL_ERR_NOMEM;
    if (rc == DVL_OK)
        rc = dvl_update_batch(d->ctx, d->h_alpha.p, K, T, DVL_MEM_HOST, nullptr, &prm, d->pair_tf.data(),
                              d->pair_w.data(), K);
    const bool timed1 = timed && rc == DVL_OK && cudaEventRecord(ev[1], st) == cudaSuccess;
    if (rc == DVL_OK) {
        dvl_bins out{d->r_mean.p, d->r_mn.p, d->r_mx.p, d->r_y.p, d->r_sum.p, d->r_count.p, DVL_MEM_HOST};
        rc = dvl_read_batch_all_async(d->ctx, &out);
    }
    if (rc == DVL_OK && cudaMemcpyAsync(d->r_stamps.p, batch_stamps(d->ctx), 2 * sizeof(unsigned long long),
                                        cudaMemcpyDeviceToHost, st) != cudaSuccess) {
        cudaGetLastError();
        rc = DVL_ERR_CUDA;
    }
    if (rc == DVL_OK) {
        if (!d->done_ev && cudaEventCreateWithFlags(&d->done_ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            d->done_ev = nullptr;
            rc = DVL_ERR_CUDA;
        } else if (cudaEventRecord(d->done_ev, st) != cudaSuccess) {
            cudaGetLastError();
            rc = DVL_ERR_CUDA;
        }
    }
    lk.lock();
    if (timed1 && rc == DVL_OK) {
        d->ev0 = ev[0];
        d->ev1 = ev[1];
    } else {
        for (cudaEvent_t x : ev)
            if (x) s->free_ev.push_back(x);
    }
    if (rc != DVL_OK) {
        const double t = now_s();
        for (Request* r : d->batch) finish_request(s, r, rc, t);
        d->batch.clear();
        d->busy = false;
        --s->inflight;
        s->cv_done.notify_all();
    }
    return true;
}

constexpr double SPIN_IDLE_S = 300e-6;     // the scheduler polls empty queues this long before it sleeps
constexpr double SPIN_WAIT_S = 2e-3;       // a caller polls its request this long before it sleeps

// A batch is finished when its completion event has passed (or the event
// reports an error, which dvl_sync then returns).  CUDA call: lock not held.
bool batch_finished(Dataset* d)
{
    const cudaError_t e = cudaEventQuery(d->done_ev);
    if (e == cudaErrorNotReady) {
        if (cudaPeekAtLastError() == cudaErrorNotReady) cudaGetLastError();
        return false;
    }
    return true;
}

void scheduler(dvl_server* s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    double idle_since = now_s();
    std::vector<Dataset*> busy, done;
    std::vector<int> rc;
    while (true) {
        // finished batches: poll the in-flight batches' events, sync (device-
        // side errors) and hand out the results; CUDA calls without the lock
        busy.clear();
        for (auto& dp : s->ds)
            if (dp->busy && dp->done_ev) busy.push_back(dp.get());
        if (!busy.empty()) {
            done.clear();
            lk.unlock();
            for (Dataset* d : busy)
                if (batch_finished(d)) done.push_back(d);
            rc.assign(done.size(), DVL_OK);
            for (size_t i = 0; i < done.size(); ++i) rc[i] = dvl_sync(done[i]->ctx);
            lk.lock();
            for (size_t i = 0; i < done.size(); ++i) complete_batch(s, done[i], rc[i]);
            if (!done.empty()) idle_since = now_s();
        }
        if (s->stop && s->inflight == 0) break;
        bool launched = false;
        if (!s->stop)
            for (size_t i = 0; i < s->ds.size(); ++i) {       // by index: add_dataset may grow ds
                if (s->inflight >= (int)s->cfg.max_inflight) break;
                Dataset* d = s->ds[i].get();
                if (!d->busy && !d->queue.empty()) launched |= launch_batch(s, d, lk);
            }
        if (launched) {
            idle_since = now_s();
            continue;
        }
        if (s->inflight > 0 || now_s() - idle_since < SPIN_IDLE_S) {
            // batches in flight, or a closed-loop caller about to submit its
            // next request: poll without the lock (so that submitting and
            // waiting threads are not held up) until a batch's event passes,
            // a request is queued or the idle window ends
            const uint64_t q0 = s->queued_total.load(std::memory_order_acquire);
            busy.clear();
            for (auto& dp : s->ds)
                if (dp->busy && dp->done_ev) busy.push_back(dp.get());
            const bool idle = s->inflight == 0;
            lk.unlock();
            while (true) {
                if (s->queued_total.load(std::memory_order_acquire) != q0) break;
                bool any = false;
                for (Dataset* d : busy)
                    if (batch_finished(d)) any = true;
                if (any) break;
                if (idle && now_s() - idle_since >= SPIN_IDLE_S) break;
                const double t = now_s();
                while (now_s() - t < 2e-6) std::this_thread::yield();   // ~2 us between polls
            }
            lk.lock();
            continue;
        }
        s->cv_sched.wait(lk, [&] {
            if (s->stop) return true;
            for (auto& dp : s->ds)
                if (!dp->busy && !dp->queue.empty()) return true;
            return false;
        });
        idle_since = now_s();
    }
    // requests never launched fail
    const double t = now_s();
    for (auto& dp : s->ds)
        for (Request* r : dp->queue) finish_request(s, r, DVL_ERR_STATE, t);
    for (auto& dp : s->ds) dp->queue.clear();
    s->cv_done.notify_all();
}

}  // namespace

extern "C" {

uint32_t dvl_serve_bucket(uint32_t k, uint32_t max_batch)
{
    if (k == 0 || max_batch == 0) return 0;
    const uint32_t b = pow2_ceil(k);
    return b < max_batch ? b : max_batch;
}

uint32_t dvl_serve_admit(uint32_t queued, uint32_t max_batch, uint32_t cap_tf, uint64_t bytes_per_tf,
                         uint64_t mem_used, uint64_t mem_budget)
{
    const uint32_t want = queued < max_batch ? queued : max_batch;
    if (want == 0) return 0;
    uint32_t b = dvl_serve_bucket(want, max_batch);
    while (b >= 1) {
        const uint64_t grow = b > cap_tf ? (uint64_t)(b - cap_tf) * bytes_per_tf : 0;
        if (mem_used <= mem_budget && grow <= mem_budget - mem_used) return want < b ? want : b;
        if (b == 1) break;
        uint32_t lower = 1;                      // next power of two below b
        while (lower * 2 < b) lower *= 2;
        b = lower;
    }
    return 0;
}

int dvl_server_create(dvl_server** out, int device, const dvl_server_config* cfg)
{
    if (!out || !cfg) return DVL_ERR_ARG;
    *out = nullptr;
    if (cfg->max_batch < 1 || cfg->max_batch > DVL_MAX_BATCH_TF || cfg->max_inflight < 1 || cfg->n_entries < 2 ||
        cfg->n_entries > DVL_MAX_TF_ENTRIES || cfg->max_width < 1 || cfg->max_width > DVL_MAX_WIDTH ||
        cfg->params.vmax_mode != DVL_VMAX_APPROX || cfg->params.want_alpha)
        return DVL_ERR_ARG;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
        cudaGetLastError();
        return DVL_ERR_CUDA;
    }
    if (device < 0 || device >= count) return DVL_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return DVL_ERR_CUDA;
    auto* s = new (std::nothrow) dvl_server;
    if (!s) return DVL_ERR_NOMEM;
    s->device = device;
    s->cfg = *cfg;
    if (s->cfg.mem_budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            delete s;
            return DVL_ERR_CUDA;
        }
        s->cfg.mem_budget = (uint64_t)(0.9 * (double)fr);
    }
    s->th = std::thread(scheduler, s);
    *out = s;
    return DVL_OK;
}

void dvl_server_destroy(dvl_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv_sched.notify_all();
    if (s->th.joinable()) s->th.join();
    for (auto& kv : s->reqs) delete kv.second;
    for (auto& dp : s->ds) {
        if (dp->done_ev) cudaEventDestroy(dp->done_ev);
        dvl_destroy(dp->ctx);
    }
    for (const Span& sp : s->spans) {
        cudaEventDestroy(sp.ev0);
        cudaEventDestroy(sp.ev1);
    }
    for (cudaEvent_t x : s->free_ev) cudaEventDestroy(x);
    delete s;
}

int dvl_server_add_dataset(dvl_server* s, uint64_t n, const int32_t* lower, const uint8_t* level, uint32_t M,
                           const float* const* fields, int sfc, uint32_t* id)
{
    if (!s || !id) return DVL_ERR_ARG;
    if (M < 1 || M > DVL_MAX_FIELDS) return sfail(s, DVL_ERR_ARG, "n_fields must be in [1, %d]", DVL_MAX_FIELDS);
    const uint64_t res = resident_bytes(n, M);
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->mem_used + res > s->cfg.mem_budget)
            return sfail(s, DVL_ERR_NOMEM, "data set needs ~%llu bytes, %llu of %llu in use",
                         (unsigned long long)res, (unsigned long long)s->mem_used,
                         (unsigned long long)s->cfg.mem_budget);
        s->mem_used += res;                     // reserved while loading
    }
    auto d = std::make_unique<Dataset>();
    d->n = n;
    d->M = M;
    d->resident = res;
    d->bytes_per_tf = per_tf_bytes(n, M, s->cfg.n_entries, s->cfg.max_width);
    int rc = dvl_create(&d->ctx, s->device, nullptr);            // own stream
    if (rc == DVL_OK) rc = dvl_load_amr(d->ctx, n, lower, level, M, fields, DVL_MEM_HOST);
    if (rc == DVL_OK) rc = dvl_build_order(d->ctx, sfc);
    if (rc == DVL_OK) rc = dvl_sync(d->ctx);
    if (rc != DVL_OK) {
        std::string msg = d->ctx ? dvl_last_error(d->ctx) : "dvl_create failed";
        if (d->ctx) dvl_destroy(d->ctx);
        std::lock_guard<std::mutex> g(s->mu);
        s->mem_used -= res;
        return sfail(s, rc, "%s", msg.c_str());
    }
    std::lock_guard<std::mutex> g(s->mu);
    *id = (uint32_t)s->ds.size();
    s->ds.push_back(std::move(d));
    return DVL_OK;
}

int dvl_server_submit(dvl_server* s, uint32_t dataset, const float* alpha, uint32_t width, uint64_t* id)
{
    if (!s || !id) return DVL_ERR_ARG;
    if (!alpha) return sfail(s, DVL_ERR_ARG, "alpha is NULL");
    if (width < 1 || width > s->cfg.max_width) return sfail(s, DVL_ERR_ARG, "width must be in [1, %u]", s->cfg.max_width);
    auto* r = new (std::nothrow) Request;
    if (!r) return DVL_ERR_NOMEM;
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->stop) {
            delete r;
            return sfail(s, DVL_ERR_STATE, "server is stopping");
        }
        if (dataset >= s->ds.size()) {
            delete r;
            return sfail(s, DVL_ERR_ARG, "data set %u does not exist", dataset);
        }
        const size_t nt = (size_t)s->ds[dataset]->M * s->cfg.n_entries;
        for (size_t i = 0; i < nt; ++i)
            if (!(alpha[i] >= 0.0f && alpha[i] <= 1.0f)) {
                delete r;
                return sfail(s, DVL_ERR_ARG, "alpha[%zu] outside [0, 1]", i);
            }
        r->alpha.assign(alpha, alpha + nt);
        r->id = s->next_id++;
        r->ds = dataset;
        r->W = width;
        r->t_submit = now_s();
        if (s->submitted == 0 || s->t_first == 0) s->t_first = r->t_submit;
        ++s->submitted;
        s->reqs[r->id] = r;
        s->ds[dataset]->queue.push_back(r);
        s->queued_total.fetch_add(1, std::memory_order_release);
        *id = r->id;
    }
    s->cv_sched.notify_one();
    return DVL_OK;
}

int dvl_server_wait(dvl_server* s, uint64_t id, double timeout_s, const dvl_bins* out)
{
    if (!s) return DVL_ERR_ARG;
    if (out && out->mem_kind != DVL_MEM_HOST) return sfail(s, DVL_ERR_ARG, "results go to host memory");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, DVL_ERR_ARG, "unknown request %llu", (unsigned long long)id);
    Request* r = it->second;
    auto ready = [&] { return r->done; };
    if (!r->done) {
        // poll the request's flag for a short while without the lock, then sleep
        lk.unlock();
        const double t0 = now_s(), spin = timeout_s < 0 ? SPIN_WAIT_S : std::min(SPIN_WAIT_S, timeout_s);
        while (!r->ready.load(std::memory_order_acquire) && now_s() - t0 < spin) std::this_thread::yield();
        lk.lock();
        if (timeout_s >= 0) timeout_s = std::max(0.0, timeout_s - (now_s() - t0));
    }
    if (timeout_s < 0) {
        s->cv_done.wait(lk, ready);
    } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
        return sfail(s, DVL_ERR_TIMEOUT, "request %llu not finished", (unsigned long long)id);
    }
    const int status = r->status;
    if (status == DVL_OK && out) {
        const size_t MW = r->mean.size(), W = r->count.size();
        if (out->mean) std::memcpy(out->mean, r->mean.data(), MW * 4);
        if (out->min) std::memcpy(out->min, r->mn.data(), MW * 4);
        if (out->max) std::memcpy(out->max, r->mx.data(), MW * 4);
        if (out->y) std::memcpy(out->y, r->y.data(), MW * 4);
        if (out->sum) std::memcpy(out->sum, r->sum.data(), MW * 8);
        if (out->count) std::memcpy(out->count, r->count.data(), W * 4);
    }
    s->reqs.erase(it);
    delete r;
    if (status != DVL_OK) return sfail(s, status, "request %llu failed", (unsigned long long)id);
    return DVL_OK;
}

int dvl_server_warmup(dvl_server* s)
{
    if (!s) return DVL_ERR_ARG;
    uint32_t n_ds;
    {
        std::lock_guard<std::mutex> g(s->mu);
        n_ds = (uint32_t)s->ds.size();
    }
    // one request batch per bucket and data set, through the normal queues
    for (uint32_t b = 1;; b = b * 2 < s->cfg.max_batch ? b * 2 : s->cfg.max_batch) {
        std::vector<uint64_t> ids;
        for (uint32_t d = 0; d < n_ds; ++d) {
            // queue b requests at once: they form one batch of bucket b
            std::lock_guard<std::mutex> g(s->mu);
            const size_t nt = (size_t)s->ds[d]->M * s->cfg.n_entries;
            std::vector<float> alpha(nt);
            for (size_t i = 0; i < nt; ++i) alpha[i] = (float)((i * 37) % 101) / 100.0f;
            for (uint32_t i = 0; i < b; ++i) {
                auto* r = new Request;
                r->alpha = alpha;
                r->id = s->next_id++;
                r->ds = d;
                r->W = s->cfg.max_width;
                r->t_submit = now_s();
                s->reqs[r->id] = r;
                s->ds[d]->queue.push_back(r);
                s->queued_total.fetch_add(1, std::memory_order_release);
                ids.push_back(r->id);
            }
        }
        s->cv_sched.notify_one();
        int rc = DVL_OK;
        for (uint64_t id : ids) {
            const int r = dvl_server_wait(s, id, 600.0, nullptr);
            if (r != DVL_OK && rc == DVL_OK) rc = r;
        }
        if (rc != DVL_OK) return rc;
        if (b >= s->cfg.max_batch) break;
    }
    return dvl_server_reset_stats(s);
}

int dvl_server_get_stats(dvl_server* s, dvl_server_stats* out)
{
    if (!s || !out) return DVL_ERR_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    dvl_server_stats st{};
    st.submitted = s->submitted;
    st.completed = s->completed;
    st.failed = s->failed;
    st.batches = s->batches;
    st.mean_batch = s->batches ? (double)s->batch_reqs / (double)s->batches : 0.0;
    if (!s->lat.empty()) {
        std::vector<double> v = s->lat;
        std::sort(v.begin(), v.end());
        auto q = [&](double f) { return v[(size_t)std::min<double>((double)v.size() - 1, std::floor(f * (double)v.size()))]; };
        st.p50_ms = q(0.50);
        st.p99_ms = q(0.99);
        st.max_ms = v.back();
        double acc = 0;
        for (double x : v) acc += x;
        st.mean_ms = acc / (double)v.size();
    }
    st.cells_per_s = s->t_last > s->t_first ? (double)s->cells / (s->t_last - s->t_first) : 0.0;
    st.mem_used = s->mem_used;
    st.mem_budget = s->cfg.mem_budget;
    for (auto& dp : s->ds) st.slot_bytes = std::max(st.slot_bytes, dp->bytes_per_tf);
    st.n_datasets = (uint32_t)s->ds.size();
    st.max_batch_seen = s->max_batch_seen;
    *out = st;
    return DVL_OK;
}

int dvl_server_reset_stats(dvl_server* s)
{
    if (!s) return DVL_ERR_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    s->lat.clear();
    s->submitted = s->completed = s->failed = s->batches = s->batch_reqs = s->cells = 0;
    s->max_batch_seen = 0;
    s->t_first = s->t_last = 0;
    for (const Span& sp : s->spans) {
        s->free_ev.push_back(sp.ev0);
        s->free_ev.push_back(sp.ev1);
    }
    s->spans.clear();
    return DVL_OK;
}

int dvl_server_timeline(dvl_server* s, dvl_batch_span* out, uint32_t cap, uint32_t* n)
{
    if (!s || !n || (cap && !out)) return DVL_ERR_ARG;
    std::vector<Span> sp;
    {
        std::lock_guard<std::mutex> g(s->mu);
        sp = s->spans;
    }
    *n = (uint32_t)sp.size();
    if (sp.empty() || cap == 0) return DVL_OK;
    cudaSetDevice(s->device);
    // times relative to the first span's start event, then shifted so that
    // the earliest start is 0
    std::vector<double> t0(sp.size()), t1(sp.size());
    double first = 0.0;
    unsigned long long ns_first = ~0ull;
    for (const Span& x : sp) ns_first = std::min(ns_first, x.ns0);
    for (size_t i = 0; i < sp.size(); ++i) {
        float a = 0.f, b = 0.f;
        if (cudaEventElapsedTime(&a, sp[0].ev0, sp[i].ev0) != cudaSuccess ||
            cudaEventElapsedTime(&b, sp[0].ev0, sp[i].ev1) != cudaSuccess) {
            cudaGetLastError();
            return sfail(s, DVL_ERR_CUDA, "batch events not readable");
        }
        t0[i] = a;
        t1[i] = b;
        first = std::min(first, (double)a);
    }
    const uint32_t k = std::min<uint32_t>(cap, (uint32_t)sp.size());
    for (uint32_t i = 0; i < k; ++i)
        out[i] = dvl_batch_span{sp[i].ds, sp[i].k, t0[i] - first, t1[i] - first,
                                (double)(sp[i].ns0 - ns_first) * 1e-6,
                                sp[i].ns1 >= sp[i].ns0 ? (double)(sp[i].ns1 - ns_first) * 1e-6 : -1.0};
    return DVL_OK;
}

const char* dvl_server_last_error(dvl_server* s) { return s ? s->last_error.c_str() : ""; }

}  // extern "C"
