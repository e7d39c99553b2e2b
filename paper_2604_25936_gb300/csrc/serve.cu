// Serving engine: continuous batching of SAND queries over resident models.
//
// Requests (host points in, host SDF out) queue per model.  A scheduler thread
// keeps up to n_streams batches in flight: whenever a stream is free it takes
// the model whose oldest request waited longest, packs that model's queued
// requests in arrival order into one batch while the batch fits both the point
// limit and the free device memory, and launches it on the stream: one
// host-to-device copy per request into a contiguous point buffer, one SAND query
// over the whole batch, one device-to-host copy per request.  Requests that
// arrive while other batches run join the next batch as soon as a stream and
// memory free up (admission by memory: every batch holds
// 16 + workspace bytes per point of a pre-allocated device arena, so the loop
// never calls cudaMalloc).  A completion thread polls the batches' events,
// releases their memory and wakes the waiting clients; each request records its
// submit-to-complete latency.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace sand {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id;
    int model;
    const float *h_points;
    int64_t n;
    float *h_out;
    Clock::time_point t_submit, t_done;
    sand_status status = SAND_OK;
    bool done = false;
};

// First-fit allocator over one device arena (offsets 256-byte aligned).
class Arena {
  public:
    bool init(size_t bytes) {
        if (cudaMalloc(&base_, bytes) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        size_ = bytes;
        free_[0] = bytes;
        return true;
    }
    void release_all() {
        cudaFree(base_);
        base_ = nullptr;
    }
    // returns offset or SIZE_MAX
    size_t alloc(size_t bytes) {
        bytes = align_up(bytes, 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used_ += bytes;
                return off;
            }
        }
        return SIZE_MAX;
    }
    void free(size_t off, size_t bytes) {
        bytes = align_up(bytes, 256);
        used_ -= bytes;
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
    char *ptr(size_t off) const { return static_cast<char *>(base_) + off; }
    size_t size() const { return size_; }
    size_t used() const { return used_; }

  private:
    void *base_ = nullptr;
    size_t size_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;
};

struct Batch {
    int model = -1;
    std::vector<Request *> reqs;
    int64_t points = 0;
    size_t off = 0, bytes = 0;
    cudaEvent_t start = nullptr, done = nullptr;  // around the batch's copies and query on its stream
    bool launched = false;  // set (under the server mutex) once every copy, the query and the event are enqueued
};

}  // namespace sand

struct sand_server_s {
    std::vector<sand_model> models;
    std::vector<int32_t> precision;  // per model
    sand_server_opts opts{};
    int device = 0;
    std::vector<cudaStream_t> streams;
    std::vector<sand::Batch *> in_flight;  // one slot per stream (nullptr = free)
    sand::Arena arena;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::deque<sand::Request *>> queues;
    std::map<uint64_t, sand::Request *> requests;
    std::vector<double> latencies_ms;
    uint64_t next_id = 1;
    int64_t points_done = 0, batches_done = 0, requests_done = 0;
    double batch_ms_sum = 0.0;  // sum over completed batches of their time on the device (start to done event)
    sand::Clock::time_point t_first, t_last;
    bool any = false, stop = false;
    std::thread scheduler, completer;
    sand_status fault = SAND_OK;
};

namespace sand {

static size_t batch_bytes(int64_t n) { return align_up((size_t)n * 12, 256) + align_up((size_t)n * 4, 256) + ws_layout(n).total; }

static void launch_batch(sand_server_s *S, int slot, Batch *b) {
    cudaStream_t st = S->streams[slot];
    char *base = S->arena.ptr(b->off);
    float *d_pts = reinterpret_cast<float *>(base);
    float *d_out = reinterpret_cast<float *>(base + align_up((size_t)b->points * 12, 256));
    void *ws = base + align_up((size_t)b->points * 12, 256) + align_up((size_t)b->points * 4, 256);
    sand_status st_q = SAND_OK;
    int64_t o = 0;
    cudaEventRecord(b->start, st);
    for (Request *r : b->reqs) {
        if (cudaMemcpyAsync(d_pts + 3 * o, r->h_points, (size_t)r->n * 12, cudaMemcpyHostToDevice, st) != cudaSuccess)
            st_q = SAND_ECUDA;
        o += r->n;
    }
    sand_query_opts qo{};
    qo.precision = S->precision[b->model];
    qo.d_workspace = ws;
    qo.workspace_bytes = ws_layout(b->points).total;
    if (st_q == SAND_OK) st_q = sand_query_sdf(S->models[b->model], d_pts, b->points, d_out, &qo, st);
    o = 0;
    for (Request *r : b->reqs) {
        if (st_q == SAND_OK &&
            cudaMemcpyAsync(r->h_out, d_out + o, (size_t)r->n * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            st_q = SAND_ECUDA;
        o += r->n;
    }
    if (st_q != SAND_OK)
        for (Request *r : b->reqs) r->status = st_q;
    cudaEventRecord(b->done, st);
}

static void scheduler_loop(sand_server_s *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        // find a free stream and the model whose oldest request has waited longest
        int slot = -1;
        for (size_t i = 0; i < S->in_flight.size(); ++i)
            if (!S->in_flight[i]) { slot = (int)i; break; }
        int model = -1;
        Clock::time_point oldest = Clock::time_point::max();
        for (size_t m = 0; m < S->queues.size(); ++m)
            if (!S->queues[m].empty() && S->queues[m].front()->t_submit < oldest) {
                oldest = S->queues[m].front()->t_submit;
                model = (int)m;
            }
        if (S->stop && model < 0) return;
        if (slot < 0 || model < 0) {
            S->cv_work.wait(lk);
            continue;
        }
        // pack this model's requests in arrival order while they fit the limits
        auto &q = S->queues[model];
        Batch *b = new Batch();
        b->model = model;
        while (!q.empty()) {
            Request *r = q.front();
            const int64_t np = b->points + r->n;
            if (!b->reqs.empty() && np > S->opts.max_batch_points) break;
            const size_t need = batch_bytes(np);
            if (need > S->arena.size()) {
                if (b->reqs.empty()) {  // can never fit: fail it
                    q.pop_front();
                    r->status = SAND_ENOMEM;
                    r->done = true;
                    r->t_done = Clock::now();
                    continue;
                }
                break;
            }
            if (S->arena.size() - S->arena.used() < need) break;  // check again with the allocator below
            b->reqs.push_back(r);
            b->points = np;
            q.pop_front();
        }
        if (b->reqs.empty()) {  // nothing fits the free memory yet (or only failed requests): wait
            delete b;
            S->cv_done.notify_all();
            if (!q.empty()) S->cv_work.wait(lk);
            continue;
        }
        b->bytes = batch_bytes(b->points);
        b->off = S->arena.alloc(b->bytes);
        if (b->off == SIZE_MAX) {  // fragmented or full: put the requests back and wait for memory
            for (auto it = b->reqs.rbegin(); it != b->reqs.rend(); ++it) q.push_front(*it);
            delete b;
            S->cv_work.wait(lk);
            continue;
        }
        S->in_flight[slot] = b;  // occupies the stream; polled only once launched (an unrecorded event reads as complete)
        cudaEventCreate(&b->start);
        cudaEventCreate(&b->done);
        lk.unlock();
        launch_batch(S, slot, b);
        lk.lock();
        b->launched = true;
        S->cv_work.notify_all();  // wake the completion poller
    }
}

static void completion_loop(sand_server_s *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        bool busy = false;
        for (size_t i = 0; i < S->in_flight.size(); ++i) {
            Batch *b = S->in_flight[i];
            if (!b) continue;
            busy = true;
            if (!b->launched) continue;
            const cudaError_t e = cudaEventQuery(b->done);
            if (e == cudaErrorNotReady) continue;
            const auto now = Clock::now();
            for (Request *r : b->reqs) {
                if (e != cudaSuccess && r->status == SAND_OK) r->status = SAND_ECUDA;
                r->t_done = now;
                r->done = true;
                S->latencies_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
                S->requests_done++;
            }
            S->points_done += b->points;
            S->batches_done++;
            S->t_last = now;
            float ms = 0.f;
            if (e == cudaSuccess && cudaEventElapsedTime(&ms, b->start, b->done) == cudaSuccess) S->batch_ms_sum += ms;
            S->arena.free(b->off, b->bytes);
            cudaEventDestroy(b->start);
            cudaEventDestroy(b->done);
            delete b;
            S->in_flight[i] = nullptr;
            S->cv_done.notify_all();
            S->cv_work.notify_all();
        }
        if (S->stop && !busy) {
            bool queued = false;
            for (auto &q : S->queues) queued |= !q.empty();
            if (!queued) return;
        }
        if (!busy) {
            S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        } else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(50));
            lk.lock();
        }
    }
}

}  // namespace sand

using namespace sand;

extern "C" {

sand_status sand_server_create(const sand_model *models, int n_models, const sand_server_opts *opts, sand_server *out) {
    if (!models || n_models < 1 || !out) {
        set_error("need at least one model and an output handle");
        return SAND_EINVAL;
    }
    *out = nullptr;
    for (int i = 0; i < n_models; ++i)
        if (!models[i]) {
            set_error("model %d is NULL", i);
            return SAND_EINVAL;
        }
    auto *S = new sand_server_s();
    S->models.assign(models, models + n_models);
    if (opts) S->opts = *opts;
    if (S->opts.n_streams <= 0) S->opts.n_streams = 3;
    if (S->opts.n_streams > 16) S->opts.n_streams = 16;
    if (S->opts.mem_budget == 0) S->opts.mem_budget = (size_t)1 << 30;
    if (S->opts.max_batch_points <= 0) S->opts.max_batch_points = (int64_t)1 << 22;
    S->device = model_device(models[0]);
    for (int i = 1; i < n_models; ++i)
        if (model_device(models[i]) != S->device) {
            delete S;
            set_error("all models of a server must live on one device");
            return SAND_EINVAL;
        }
    S->precision.assign(n_models, S->opts.precision);
    if (S->opts.model_precision)
        for (int i = 0; i < n_models; ++i) S->precision[i] = S->opts.model_precision[i];
    S->opts.model_precision = nullptr;  // copied; the caller's array need not outlive this call
    // a model keeps the packed weights of one tensor-core precision: one handle served in two
    // would repack (free and allocate) inside the serving loop
    for (int i = 0; i < n_models; ++i)
        for (int j = i + 1; j < n_models; ++j)
            if (models[i] == models[j] && S->precision[i] != S->precision[j] && S->precision[i] != SAND_FP32_SIMT &&
                S->precision[j] != SAND_FP32_SIMT) {
                delete S;
                set_error("models %d and %d are one handle with two tensor-core precisions (%d, %d)", i, j,
                          S->precision[i], S->precision[j]);
                return SAND_EINVAL;
            }
    for (int i = 0; i < n_models; ++i) {  // pack tensor-core weights now: the serving loop allocates nothing
        sand_status st = model_prepare(models[i], S->precision[i]);
        if (st) {
            delete S;
            return st;
        }
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    if (!S->arena.init(S->opts.mem_budget)) {
        if (prev >= 0) cudaSetDevice(prev);
        delete S;
        set_error("cannot reserve a %zu-byte device arena", S->opts.mem_budget);
        return SAND_ENOMEM;
    }
    S->streams.resize(S->opts.n_streams);
    for (auto &st : S->streams) cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    S->in_flight.assign(S->opts.n_streams, nullptr);
    S->queues.resize(n_models);
    if (prev >= 0) cudaSetDevice(prev);
    S->scheduler = std::thread(scheduler_loop, S);
    S->completer = std::thread(completion_loop, S);
    *out = S;
    return SAND_OK;
}

sand_status sand_server_submit(sand_server S, int model, const float *h_points, int64_t n, float *h_out,
                               uint64_t *ticket) {
    if (!S || !ticket) { set_error("NULL server or ticket"); return SAND_EINVAL; }
    if (model < 0 || model >= (int)S->models.size()) { set_error("model index %d out of range", model); return SAND_EINVAL; }
    if (n < 0 || (n > 0 && (!h_points || !h_out))) { set_error("bad request buffers"); return SAND_EINVAL; }
    auto *r = new Request();
    r->model = model;
    r->h_points = h_points;
    r->n = n;
    r->h_out = h_out;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) { delete r; set_error("server is shutting down"); return SAND_EINVAL; }
        r->id = S->next_id++;
        *ticket = r->id;
        S->requests[r->id] = r;
        if (!S->any) { S->t_first = r->t_submit; S->any = true; }
        if (n == 0) {
            r->done = true;
            r->t_done = r->t_submit;
        } else {
            S->queues[model].push_back(r);
        }
    }
    S->cv_work.notify_all();
    return SAND_OK;
}

sand_status sand_server_wait(sand_server S, uint64_t ticket, double timeout_s, double *latency_ms) {
    if (!S) { set_error("NULL server"); return SAND_EINVAL; }
    if (!(timeout_s >= 0.0)) { set_error("timeout_s must be a number >= 0"); return SAND_EINVAL; }
    if (timeout_s > 1e7) timeout_s = 1e7;  // about 116 days: keeps the deadline arithmetic finite
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->requests.find(ticket);
    if (it == S->requests.end()) { set_error("unknown ticket %llu", (unsigned long long)ticket); return SAND_EINVAL; }
    Request *r = it->second;
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    while (!r->done) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !r->done) {
            set_error("request %llu still running after %.3f s", (unsigned long long)ticket, timeout_s);
            return SAND_ETIMEOUT;
        }
    }
    const sand_status st = r->status;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    S->requests.erase(it);
    delete r;
    if (st != SAND_OK) set_error("request failed with status %d", (int)st);
    return st;
}

sand_status sand_server_stats(sand_server S, sand_server_report *out) {
    if (!S || !out) { set_error("NULL argument"); return SAND_EINVAL; }
    std::lock_guard<std::mutex> lk(S->mu);
    std::vector<double> v = S->latencies_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) { return v.empty() ? 0.0 : v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
    out->requests = S->requests_done;
    out->batches = S->batches_done;
    out->points = S->points_done;
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = v.empty() ? 0.0 : v.back();
    const double span = S->any ? std::chrono::duration<double>(S->t_last - S->t_first).count() : 0.0;
    out->queries_per_s = span > 0 ? S->points_done / span : 0.0;
    out->arena_bytes = S->arena.size();
    out->span_ms = span * 1e3;
    out->batch_ms_sum = S->batch_ms_sum;
    return SAND_OK;
}

sand_status sand_server_destroy(sand_server S) {
    if (!S) return SAND_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->scheduler.joinable()) S->scheduler.join();
    if (S->completer.joinable()) S->completer.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    for (auto &st : S->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    S->arena.release_all();
    if (prev >= 0) cudaSetDevice(prev);
    for (auto &kv : S->requests) delete kv.second;
    delete S;
    return SAND_OK;
}

}  // extern "C"
