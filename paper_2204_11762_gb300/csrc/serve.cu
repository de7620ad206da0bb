// Serving: continuous batching of render requests over resident models.
//
// mfadvr_submit validates a request and queues it; a serving thread admits
// queued requests while the frame-buffer budget (bytes of output images in
// flight) and the limits on batch size and batches in flight allow, packs
// them into one batched launch per degree and storage type (the persistent
// kernel of render_kernels.cu, whose warps take ray tiles of every image of
// the batch from one queue), records that launch sequence as a CUDA graph
// per group signature and stream (later batches update and replay it), and
// marks the requests done when the batch's event completes.  Requests that
// arrive while batches run are admitted as budget and slots free up, and
// their batch runs on another stream, overlapping the ones in flight.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "ctx.h"
#include "mfa_internal.h"
#include "mfadvr.h"

namespace mfadvr {
namespace api {

namespace {

int64_t now_us()
{
    return std::chrono::duration_cast<std::chrono::microseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

constexpr int kMaxFlights = 8;
constexpr unsigned kSlots = 2 * kMaxFlights;  // job tables
constexpr unsigned kCounters = 64 * kMaxFlights;

}  // namespace

struct Server {
    struct Request {
        uint64_t id;
        RenderJob job;
        size_t bytes;
    };
    struct Ticket {
        int state = 0;  // 0 queued, 1 on the GPU, 2 done
        mfadvr_status status = MFADVR_OK;
        int64_t t_submit = 0, t_done = 0;
    };
    struct Flight {
        std::vector<uint64_t> ids;
        size_t bytes = 0;
        cudaEvent_t done = nullptr;
        unsigned slot = 0;
        mfadvr_serve_trace_record rec{};
    };
    using Signature = std::vector<std::tuple<int, int, int, int, int>>;

    mfadvr_ctx *ctx = nullptr;
    int device = 0;
    size_t budget = 0, in_use = 0;
    int max_batch = 64, max_flights = 2;

    std::thread thread;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stopping = false;
    std::deque<Request> pending;
    std::unordered_map<uint64_t, Ticket> tickets;
    std::deque<Flight> flights;
    uint64_t next_id = 1;
    unsigned next_flight = 0;

    cudaStream_t streams[kMaxFlights] = {};
    RenderJob *h_jobs = nullptr, *d_jobs = nullptr;  // kSlots job tables
    unsigned next_slot = 0;
    int *counters = nullptr;
    unsigned next_counter = 0;
    std::map<std::pair<Signature, int>, cudaGraphExec_t> graphs;
    std::atomic<uint64_t> launches{0}, graph_updates{0}, graph_instantiations{0};
    // the last kTrace batches, oldest first once the ring wraps
    static constexpr size_t kTrace = 4096;
    std::vector<mfadvr_serve_trace_record> trace;
    size_t trace_next = 0;
    int64_t t_origin = 0;

    // Packs `batch` into the next job-table slot and launches it on stream k
    // through the graph of its group signature.  Called without the lock.
    cudaError_t launch(const std::vector<Request> &batch, int k, unsigned slot, cudaEvent_t ev, int *ngroups)
    {
        TraceRange trace("mfadvr_serve_batch");
        cudaError_t e = cudaSuccess;
        RenderJob *hj = h_jobs + static_cast<size_t>(slot) * MFADVR_MAX_BATCH;
        RenderJob *dj = d_jobs + static_cast<size_t>(slot) * MFADVR_MAX_BATCH;
        std::vector<RenderJob> src(batch.size());
        for (size_t i = 0; i < batch.size(); ++i) src[i] = batch[i].job;
        std::vector<BatchGroup> groups = pack_jobs(src.data(), static_cast<int>(src.size()), hj);
        Signature sig;
        for (const BatchGroup &g : groups) sig.emplace_back(g.p, g.dtype, g.grad, g.nu, g.rat);
        *ngroups = static_cast<int>(groups.size());

        cudaStream_t s = streams[k];
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        cudaError_t body = cudaMemcpyAsync(dj, hj, sizeof(RenderJob) * batch.size(), cudaMemcpyHostToDevice, s);
        for (const BatchGroup &g : groups) {
            if (body != cudaSuccess) break;
            int *counter = counters + (next_counter++ % kCounters);
            body = launch_render_batch(g.p, g.dtype, g.grad, g.nu, g.rat, dj + g.first, g.count, g.tiles, 0, counter,
                                       nullptr, s);
        }
        e = cudaStreamEndCapture(s, &graph);
        if (body != cudaSuccess) e = body;
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return e;
        }
        auto key = std::make_pair(sig, k);
        auto it = graphs.find(key);
        if (it != graphs.end()) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(it->second, graph, &info) == cudaSuccess) {
                ++graph_updates;
            } else {
                cudaGetLastError();
                cudaGraphExecDestroy(it->second);
                graphs.erase(it);
                it = graphs.end();
            }
        }
        if (it == graphs.end()) {
            cudaGraphExec_t exec = nullptr;
            e = cudaGraphInstantiate(&exec, graph, 0);
            if (e != cudaSuccess) {
                cudaGraphDestroy(graph);
                return e;
            }
            it = graphs.emplace(key, exec).first;
            ++graph_instantiations;
        }
        cudaGraphDestroy(graph);
        e = cudaGraphLaunch(it->second, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev, s);
        ++launches;
        return e;
    }

    void run()
    {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            // completions (batches on different streams may finish out of order)
            for (auto it = flights.begin(); it != flights.end();) {
                const cudaError_t q = cudaEventQuery(it->done);
                if (q == cudaErrorNotReady) {
                    ++it;
                    continue;
                }
                const int64_t t = now_us();
                for (uint64_t id : it->ids) {
                    Ticket &tk = tickets[id];
                    tk.state = 2;
                    tk.t_done = t;
                    if (q != cudaSuccess) tk.status = MFADVR_ECUDA;
                }
                if (q != cudaSuccess) cudaGetLastError();
                in_use -= it->bytes;
                it->rec.t_done_us = t - t_origin;
                if (trace.size() < kTrace) trace.push_back(it->rec);
                else trace[trace_next % kTrace] = it->rec;
                ++trace_next;
                cudaEventDestroy(it->done);
                it = flights.erase(it);
                cv_done.notify_all();
            }
            // admission: first in, first out, within the budget
            if (!pending.empty() && static_cast<int>(flights.size()) < max_flights) {
                std::vector<Request> batch;
                size_t bytes = 0;
                while (!pending.empty() && static_cast<int>(batch.size()) < max_batch) {
                    const Request &r = pending.front();
                    const bool fits = in_use + bytes + r.bytes <= budget;
                    if (!fits && !(batch.empty() && flights.empty())) break;  // an idle server takes one anyway
                    bytes += r.bytes;
                    batch.push_back(r);
                    pending.pop_front();
                }
                if (!batch.empty()) {
                    Flight f;
                    f.bytes = bytes;
                    f.rec.t_admit_us = now_us() - t_origin;
                    f.rec.jobs = static_cast<int32_t>(batch.size());
                    f.rec.queued_after = static_cast<int32_t>(pending.size());
                    f.rec.oldest_submit_us = tickets[batch.front().id].t_submit - t_origin;
                    for (const Request &r : batch) {
                        f.ids.push_back(r.id);
                        tickets[r.id].state = 1;
                    }
                    in_use += bytes;
                    const int k = static_cast<int>(next_flight++ % static_cast<unsigned>(max_flights));
                    cudaError_t e = cudaEventCreateWithFlags(&f.done, cudaEventDisableTiming);
                    f.rec.stream = k;
                    // a job-table slot no batch in flight reads (kSlots > kMaxFlights)
                    bool busy[kSlots] = {};
                    for (const Flight &o : flights) busy[o.slot] = true;
                    while (busy[next_slot % kSlots]) ++next_slot;
                    f.slot = next_slot++ % kSlots;
                    lk.unlock();
                    int groups = 0;
                    if (e == cudaSuccess) e = launch(batch, k, f.slot, f.done, &groups);
                    lk.lock();
                    f.rec.groups = groups;
                    f.rec.t_launched_us = now_us() - t_origin;
                    if (e != cudaSuccess) {
                        cudaGetLastError();
                        const int64_t t = now_us();
                        for (uint64_t id : f.ids) {
                            Ticket &tk = tickets[id];
                            tk.state = 2;
                            tk.status = MFADVR_ECUDA;
                            tk.t_done = t;
                        }
                        in_use -= bytes;
                        if (f.done) cudaEventDestroy(f.done);
                        cv_done.notify_all();
                    } else {
                        flights.push_back(f);
                    }
                    continue;
                }
            }
            if (stopping && pending.empty() && flights.empty()) break;
            if (!flights.empty())
                cv_work.wait_for(lk, std::chrono::microseconds(50));
            else
                cv_work.wait(lk, [&] { return stopping || !pending.empty(); });
        }
    }
};

void stop_server(mfadvr_ctx *ctx)
{
    Server *sv = ctx ? ctx->server : nullptr;
    if (!sv) return;
    {
        std::lock_guard<std::mutex> g(sv->mu);
        sv->stopping = true;
    }
    sv->cv_work.notify_all();
    if (sv->thread.joinable()) sv->thread.join();
    DeviceGuard dg(sv->device);
    for (auto &kv : sv->graphs) cudaGraphExecDestroy(kv.second);
    for (auto &s : sv->streams)
        if (s) cudaStreamDestroy(s);
    if (sv->d_jobs) cudaFree(sv->d_jobs);
    if (sv->h_jobs) cudaFreeHost(sv->h_jobs);
    if (sv->counters) cudaFree(sv->counters);
    delete sv;
    ctx->server = nullptr;
}

}  // namespace api
}  // namespace mfadvr

using namespace mfadvr;
using namespace mfadvr::api;

extern "C" {

mfadvr_status mfadvr_serve_start(mfadvr_ctx *ctx, const mfadvr_serve_config *cfg)
{
    if (!ctx) return fail(nullptr, MFADVR_EINVAL, "ctx must not be NULL");
    if (ctx->server) return fail(ctx, MFADVR_EBUSY, "the serving loop already runs");
    mfadvr_serve_config c = cfg ? *cfg : mfadvr_serve_config{0, 0, 0};
    if (c.max_batch < 0 || c.max_batch > MFADVR_MAX_BATCH || c.max_in_flight < 0 || c.max_in_flight > kMaxFlights)
        return fail(ctx, MFADVR_EINVAL, "max_batch must be in 0..%d and max_in_flight in 0..%d", MFADVR_MAX_BATCH,
                    kMaxFlights);
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "cudaSetDevice");
    Server *sv = new (std::nothrow) Server();
    if (!sv) return fail(ctx, MFADVR_ENOMEM, "out of host memory");
    sv->ctx = ctx;
    sv->device = ctx->device;
    sv->budget = c.frame_budget_bytes ? c.frame_budget_bytes : (size_t(1) << 30);
    sv->max_batch = c.max_batch ? c.max_batch : 64;
    sv->max_flights = c.max_in_flight ? c.max_in_flight : 2;
    const size_t table = sizeof(RenderJob) * MFADVR_MAX_BATCH * kSlots;
    cudaError_t e = cudaMalloc(&sv->d_jobs, table);
    if (e == cudaSuccess) e = cudaMallocHost(&sv->h_jobs, table);
    if (e == cudaSuccess) e = cudaMalloc(&sv->counters, sizeof(int) * kCounters);
    for (int k = 0; e == cudaSuccess && k < kMaxFlights; ++k)
        e = cudaStreamCreateWithFlags(&sv->streams[k], cudaStreamNonBlocking);
    ctx->server = sv;
    if (e != cudaSuccess) {
        stop_server(ctx);
        return cuda_fail(ctx, e, "serving-loop setup");
    }
    sv->t_origin = now_us();
    sv->trace.reserve(Server::kTrace);
    sv->thread = std::thread([sv] { sv->run(); });
    return MFADVR_OK;
}

mfadvr_status mfadvr_serve_stop(mfadvr_ctx *ctx)
{
    if (!ctx) return fail(nullptr, MFADVR_EINVAL, "ctx must not be NULL");
    if (!ctx->server) return fail(ctx, MFADVR_EINVAL, "the serving loop is not running");
    stop_server(ctx);
    return MFADVR_OK;
}

mfadvr_status mfadvr_submit(mfadvr_ctx *ctx, const mfadvr_render_job *job, uint64_t *ticket)
{
    if (!ctx) return fail(nullptr, MFADVR_EINVAL, "ctx must not be NULL");
    Server *sv = ctx->server;
    if (!sv) return fail(ctx, MFADVR_EINVAL, "the serving loop is not running");
    if (!job || !ticket) return fail(ctx, MFADVR_EINVAL, "job and ticket must not be NULL");
    Server::Request r;
    {
        DeviceGuard g(ctx->device);
        if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "cudaSetDevice");
        if (mfadvr_status st = make_job(ctx, *job, 0, &r.job)) return st;
    }
    const size_t px = static_cast<size_t>(job->params.width) * job->params.height;
    r.bytes = px * 16 + (job->nsamples_dev ? px * 4 : 0);
    {
        std::lock_guard<std::mutex> g(sv->mu);
        if (sv->stopping) return fail(ctx, MFADVR_EBUSY, "the serving loop is stopping");
        r.id = sv->next_id++;
        Server::Ticket t;
        t.t_submit = now_us();
        sv->tickets[r.id] = t;
        sv->pending.push_back(r);
        *ticket = r.id;
    }
    sv->cv_work.notify_one();
    return MFADVR_OK;
}

mfadvr_status mfadvr_wait(mfadvr_ctx *ctx, uint64_t ticket, int64_t timeout_us, int64_t *latency_us)
{
    if (!ctx) return fail(nullptr, MFADVR_EINVAL, "ctx must not be NULL");
    Server *sv = ctx->server;
    if (!sv) return fail(ctx, MFADVR_EINVAL, "the serving loop is not running");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return fail(ctx, MFADVR_ENOTFOUND, "no ticket %llu", (unsigned long long)ticket);
    auto done = [&] { return sv->tickets[ticket].state == 2; };
    if (timeout_us < 0) sv->cv_done.wait(lk, done);
    else if (!sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done))
        return fail(ctx, MFADVR_ETIMEOUT, "ticket %llu not done", (unsigned long long)ticket);
    const Server::Ticket t = sv->tickets[ticket];
    sv->tickets.erase(ticket);
    if (latency_us) *latency_us = t.t_done - t.t_submit;
    if (t.status != MFADVR_OK) return fail(ctx, t.status, "ticket %llu failed on the GPU", (unsigned long long)ticket);
    return MFADVR_OK;
}

mfadvr_status mfadvr_serve_stats(mfadvr_ctx *ctx, uint64_t *launches, uint64_t *graph_updates,
                                 uint64_t *graph_instantiations)
{
    if (!ctx) return fail(nullptr, MFADVR_EINVAL, "ctx must not be NULL");
    Server *sv = ctx->server;
    if (!sv) return fail(ctx, MFADVR_EINVAL, "the serving loop is not running");
    if (launches) *launches = sv->launches.load();
    if (graph_updates) *graph_updates = sv->graph_updates.load();
    if (graph_instantiations) *graph_instantiations = sv->graph_instantiations.load();
    return MFADVR_OK;
}



mfadvr_status mfadvr_serve_trace(mfadvr_ctx *ctx, mfadvr_serve_trace_record *records, int32_t capacity,
                                 int32_t *count)
{
    if (!ctx) return fail(nullptr, MFADVR_EINVAL, "ctx must not be NULL");
    Server *sv = ctx->server;
    if (!sv) return fail(ctx, MFADVR_EINVAL, "the serving loop is not running");
    if (!count || capacity < 0 || (capacity > 0 && !records))
        return fail(ctx, MFADVR_EINVAL, "count must not be NULL and records must hold capacity entries");
    std::lock_guard<std::mutex> g(sv->mu);
    const size_t n = sv->trace.size();
    const size_t take = std::min(n, static_cast<size_t>(capacity));
    // oldest first: when the ring has wrapped, it starts at trace_next % kTrace
    const size_t start = (sv->trace_next > Server::kTrace) ? sv->trace_next % Server::kTrace : 0;
    for (size_t i = 0; i < take; ++i) records[i] = sv->trace[(start + (n - take) + i) % n];
    *count = static_cast<int32_t>(take);
    return MFADVR_OK;
}

}  // extern "C"
