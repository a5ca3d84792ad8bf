// A serving loop over many filters (C ABI in include/gpufilter.h): requests
// arrive as host batches and wait in their filter's FIFO; the scheduler of
// gf_sched.h admits them continuously. Any idle worker (a host thread with
// its own CUDA stream and pinned bounce buffers) takes the oldest waiting
// request of a filter that has nothing in flight, merged with the requests
// right behind it when their results provably do not change (queries,
// counts, GQF removes), as soon as its staging fits in the device pool.
// Batches of different filters overlap on the device; one filter's batches
// run one after another in submission order, so each request's results are
// the same alone and in the mix.
//
// Per batch: host keys of each merged request -> device pool (pageable ones
// through pinned staging), one filter operation over all of them, results of
// each request -> its host buffer.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "gf_internal.cuh"
#include "gf_sched.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Pending {
    filter_request r;
    Clock::time_point t_submit;
};

struct Done {
    int rc;
    double latency_s;
};

struct Worker {
    std::thread th;
    cudaStream_t stream = nullptr;
    uint64_t *h_keys = nullptr;  // pinned bounce buffers for pageable host memory
    void *h_out = nullptr;
};

}  // namespace

struct filter_server {
    std::vector<filter_t *> filters;
    std::vector<Worker> workers;
    uint64_t max_keys = 0;
    int device = 0;
    char *d_pool = nullptr;  // device staging pool shared by all batches
    gfsched::Scheduler *sched = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::unordered_map<uint64_t, Pending> pending;  // submitted, not yet run
    std::unordered_map<uint64_t, Done> done;
    std::unordered_set<uint64_t> outstanding;  // submitted, not yet collected by a wait
    uint64_t next_ticket = 1;
    bool stop = false;
    filter_server_stats stats{};
};

namespace {

// page-locked host memory can be copied to and from the device directly
static bool page_locked(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

static int run_batch(filter_server *S, Worker &W, const gfsched::Batch &b, const std::vector<filter_request> &rq)
{
    filter_t *f = S->filters[b.filter];
    uint64_t *d_keys = reinterpret_cast<uint64_t *>(S->d_pool + b.offset);
    char *d_out = S->d_pool + b.offset + ((b.n * 8 + 255) & ~255ull);
    const uint64_t rb = gfsched::result_bytes(b.op);
    // keys of every request, back to back (pageable ones through the pinned buffer)
    uint64_t at = 0;
    for (const filter_request &r : rq) {
        if (r.n) {
            const uint64_t *src = r.host_keys;
            if (!page_locked(src)) {
                std::memcpy(W.h_keys + at, src, r.n * 8);
                src = W.h_keys + at;
            }
            GF_CUDA(cudaMemcpyAsync(d_keys + at, src, r.n * 8, cudaMemcpyHostToDevice, W.stream));
        }
        at += r.n;
    }
    int rc = FILTER_OK;
    if (b.n) {
        switch (b.op) {
        case FILTER_OP_INSERT:
            rc = filter_insert(f, d_keys, b.n, reinterpret_cast<uint8_t *>(d_out), W.stream);
            break;
        case FILTER_OP_QUERY:
            rc = filter_query(f, d_keys, b.n, reinterpret_cast<uint8_t *>(d_out), W.stream);
            break;
        case FILTER_OP_REMOVE:
            rc = filter_remove(f, d_keys, b.n, reinterpret_cast<uint8_t *>(d_out), W.stream);
            break;
        case FILTER_OP_COUNT:
            rc = filter_count(f, d_keys, b.n, reinterpret_cast<uint64_t *>(d_out), W.stream);
            break;
        default:
            rc = FILTER_ERR_ARG;
        }
    }
    if (rc != FILTER_OK) {
        cudaStreamSynchronize(W.stream);
        return rc;
    }
    // each request's results to its own buffer
    at = 0;
    std::vector<std::pair<uint64_t, const filter_request *>> bounce;
    for (const filter_request &r : rq) {
        if (r.n && r.host_out) {
            if (page_locked(r.host_out)) {
                GF_CUDA(cudaMemcpyAsync(r.host_out, d_out + at * rb, r.n * rb, cudaMemcpyDeviceToHost, W.stream));
            } else {
                GF_CUDA(cudaMemcpyAsync(static_cast<char *>(W.h_out) + at * rb, d_out + at * rb, r.n * rb,
                                        cudaMemcpyDeviceToHost, W.stream));
                bounce.emplace_back(at, &r);
            }
        }
        at += r.n;
    }
    GF_CUDA(cudaStreamSynchronize(W.stream));
    for (auto &x : bounce)
        std::memcpy(x.second->host_out, static_cast<char *>(W.h_out) + x.first * rb, x.second->n * rb);
    return FILTER_OK;
}

static void worker_main(filter_server *S, size_t wi)
{
    Worker &W = S->workers[wi];
    cudaSetDevice(S->device);
    for (;;) {
        gfsched::Batch b;
        std::vector<filter_request> rq;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            bool got = false;
            S->cv_work.wait(lk, [&] {
                got = S->sched->next(b);
                return got || (S->stop && S->sched->waiting() == 0);
            });
            if (!got) return;  // stop requested and nothing left
            for (const gfsched::Req &q : b.reqs) rq.push_back(S->pending[q.ticket].r);
            S->stats.batches++;
            S->stats.requests += b.reqs.size();
            if (b.reqs.size() > 1) S->stats.merged_requests += b.reqs.size();
            const uint64_t run = S->sched->running();
            if (run > S->stats.max_concurrent) S->stats.max_concurrent = run;
            const uint64_t used = S->sched->pool_size() - S->sched->pool_available();
            if (used > S->stats.pool_peak_bytes) S->stats.pool_peak_bytes = used;
        }
        const int rc = run_batch(S, W, b, rq);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->sched->finish(b);
            const Clock::time_point now = Clock::now();
            for (const gfsched::Req &q : b.reqs) {
                const Pending &p = S->pending[q.ticket];
                S->done[q.ticket] = Done{rc, std::chrono::duration<double>(now - p.t_submit).count()};
                S->pending.erase(q.ticket);
            }
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();  // staging and the filter are free again
    }
}

static void free_server(filter_server *S)
{
    for (Worker &W : S->workers) {
        if (W.stream) cudaStreamDestroy(W.stream);
        if (W.h_keys) cudaFreeHost(W.h_keys);
        if (W.h_out) cudaFreeHost(W.h_out);
    }
    gf::dev_free(S->d_pool);
    delete S->sched;
    delete S;
}

}  // namespace

extern "C" {

int filter_server_create(filter_t *const *filters, uint32_t n_filters, uint32_t n_workers, uint64_t max_keys,
                         filter_server_t **out)
{
    if (!filters || !out || n_filters == 0 || n_workers == 0 || n_workers > 64 || max_keys == 0) return FILTER_ERR_ARG;
    *out = nullptr;
    std::vector<bool> merge_removes(n_filters);
    std::vector<uint64_t> max_merge(n_filters);
    for (uint32_t i = 0; i < n_filters; i++) {
        if (!filters[i]) return FILTER_ERR_ARG;
        merge_removes[i] = filters[i]->cfg.kind == FILTER_GQF;
        max_merge[i] = filters[i]->cfg.max_batch < max_keys ? filters[i]->cfg.max_batch : max_keys;
        if (max_merge[i] == 0) max_merge[i] = 1;
    }
    // the staging pool: room for every worker's largest batch when the free
    // device memory allows, else as many largest batches as fit (at least one)
    const uint64_t one = gfsched::staging_bytes(FILTER_OP_COUNT, max_keys);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return FILTER_ERR_CUDA;
    }
    const uint64_t usable = free_b > (64ull << 20) ? free_b - (64ull << 20) : 0;  // keep 64 MiB for the runtime
    uint64_t pool = one * n_workers;
    if (pool > usable) pool = usable / one * one;
    if (pool < one) return FILTER_ERR_OOM;
    filter_server *S = new (std::nothrow) filter_server();
    if (!S) return FILTER_ERR_OOM;
    S->filters.assign(filters, filters + n_filters);
    S->max_keys = max_keys;
    cudaGetDevice(&S->device);
    S->sched = new (std::nothrow) gfsched::Scheduler(merge_removes, max_merge, pool);
    if (!S->sched || gf::dev_malloc(reinterpret_cast<void **>(&S->d_pool), pool) != cudaSuccess) {
        cudaGetLastError();
        S->d_pool = nullptr;
        free_server(S);
        return FILTER_ERR_OOM;
    }
    S->stats.pool_bytes = pool;
    S->workers.resize(n_workers);
    for (Worker &W : S->workers) {
        if (cudaStreamCreateWithFlags(&W.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMallocHost(&W.h_keys, max_keys * 8) != cudaSuccess ||
            cudaMallocHost(&W.h_out, max_keys * 8) != cudaSuccess) {
            cudaGetLastError();
            free_server(S);
            return FILTER_ERR_OOM;
        }
    }
    for (size_t i = 0; i < S->workers.size(); i++) S->workers[i].th = std::thread(worker_main, S, i);
    *out = S;
    return FILTER_OK;
}

int filter_server_submit(filter_server_t *s, const filter_request *req, uint64_t *ticket)
{
    if (!s || !req || !ticket || req->filter >= s->filters.size() || req->n > s->max_keys ||
        (req->n && !req->host_keys) || req->op > FILTER_OP_COUNT)
        return FILTER_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return FILTER_ERR_ARG;
        const uint64_t t = s->next_ticket;
        if (!s->sched->submit(t, req->filter, req->op, req->n)) return FILTER_ERR_ARG;
        s->next_ticket++;
        s->pending[t] = Pending{*req, Clock::now()};
        s->outstanding.insert(t);
        *ticket = t;
    }
    s->cv_work.notify_one();
    return FILTER_OK;
}

int filter_server_wait(filter_server_t *s, uint64_t ticket, int *op_rc, double *latency_s)
{
    if (!s || ticket == 0) return FILTER_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    if (!s->outstanding.count(ticket)) return FILTER_ERR_ARG;  // unknown or already collected
    s->cv_done.wait(lk, [&] { return s->done.count(ticket) != 0; });
    const Done d = s->done[ticket];
    s->done.erase(ticket);
    s->outstanding.erase(ticket);
    if (op_rc) *op_rc = d.rc;
    if (latency_s) *latency_s = d.latency_s;
    return FILTER_OK;
}

int filter_server_get_stats(filter_server_t *s, filter_server_stats *out)
{
    if (!s || !out) return FILTER_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    return FILTER_OK;
}

int filter_server_destroy(filter_server_t *s)
{
    if (!s) return FILTER_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (Worker &W : s->workers)
        if (W.th.joinable()) W.th.join();
    free_server(s);
    return FILTER_OK;
}

}  // extern "C"
