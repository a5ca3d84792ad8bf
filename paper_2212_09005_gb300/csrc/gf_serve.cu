// A serving loop over many filters (C ABI in include/gpufilter.h): requests
// arrive as host batches, wait in their filter's FIFO, are admitted when a
// worker with device staging is free, and run on that worker's CUDA stream.
//
// Every filter is bound to one worker (filter i -> worker i mod W), and a
// worker takes its requests in submission order, so each filter sees its
// batches in exactly the order they were submitted, whatever else is in
// flight: a batch's results are the same alone and in the mix. Workers run
// concurrently on their own streams and pinned staging buffers; a worker
// handles one request at a time (host keys -> pinned staging -> device, the
// filter operation, results -> pinned staging -> caller's buffer); page-locked
// caller buffers skip the staging copies.
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

#include "gf_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t ticket;
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
    std::deque<Req> q;
    uint64_t *d_keys = nullptr;  // device staging: keys
    void *d_out = nullptr;       // device staging: results (8 bytes per key)
    uint64_t *h_keys = nullptr;  // pinned staging
    void *h_out = nullptr;
};

}  // namespace

struct filter_server {
    std::vector<filter_t *> filters;
    std::vector<Worker> workers;
    uint64_t max_keys = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::unordered_map<uint64_t, Done> done;
    std::unordered_set<uint64_t> outstanding;  // submitted, not yet collected by a wait
    uint64_t next_ticket = 1;
    uint64_t in_flight = 0;
    bool stop = false;
};

namespace {

static int out_bytes(uint32_t op) { return op == FILTER_OP_COUNT ? 8 : 1; }

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

static int run_one(filter_server *S, Worker &W, const filter_request &r)
{
    filter_t *f = S->filters[r.filter];
    const uint64_t n = r.n;
    const size_t ob = (size_t)out_bytes(r.op) * n;
    if (n) {
        const uint64_t *src = r.host_keys;
        if (!page_locked(src)) {  // pageable: through the worker's pinned staging
            std::memcpy(W.h_keys, src, n * 8);
            src = W.h_keys;
        }
        GF_CUDA(cudaMemcpyAsync(W.d_keys, src, n * 8, cudaMemcpyHostToDevice, W.stream));
    }
    int rc;
    switch (r.op) {
    case FILTER_OP_INSERT:
        rc = filter_insert(f, W.d_keys, n, static_cast<uint8_t *>(W.d_out), W.stream);
        break;
    case FILTER_OP_QUERY:
        rc = filter_query(f, W.d_keys, n, static_cast<uint8_t *>(W.d_out), W.stream);
        break;
    case FILTER_OP_REMOVE:
        rc = filter_remove(f, W.d_keys, n, static_cast<uint8_t *>(W.d_out), W.stream);
        break;
    case FILTER_OP_COUNT:
        rc = filter_count(f, W.d_keys, n, static_cast<uint64_t *>(W.d_out), W.stream);
        break;
    default:
        rc = FILTER_ERR_ARG;
    }
    if (rc != FILTER_OK) return rc;
    const bool direct = n && r.host_out && page_locked(r.host_out);
    if (n && r.host_out)
        GF_CUDA(cudaMemcpyAsync(direct ? r.host_out : W.h_out, W.d_out, ob, cudaMemcpyDeviceToHost, W.stream));
    GF_CUDA(cudaStreamSynchronize(W.stream));
    if (n && r.host_out && !direct) std::memcpy(r.host_out, W.h_out, ob);
    return FILTER_OK;
}

static void worker_main(filter_server *S, size_t wi)
{
    Worker &W = S->workers[wi];
    cudaSetDevice(S->device);
    for (;;) {
        Req q;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !W.q.empty(); });
            if (W.q.empty()) return;  // stop requested and nothing left
            q = W.q.front();
            W.q.pop_front();
        }
        const int rc = run_one(S, W, q.r);
        const double lat = std::chrono::duration<double>(Clock::now() - q.t_submit).count();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->done[q.ticket] = Done{rc, lat};
            S->in_flight--;
        }
        S->cv_done.notify_all();
    }
}

static void free_workers(filter_server *S)
{
    for (Worker &W : S->workers) {
        if (W.stream) cudaStreamDestroy(W.stream);
        if (W.d_keys) cudaFree(W.d_keys);
        if (W.d_out) cudaFree(W.d_out);
        if (W.h_keys) cudaFreeHost(W.h_keys);
        if (W.h_out) cudaFreeHost(W.h_out);
    }
}

}  // namespace

extern "C" {

int filter_server_create(filter_t *const *filters, uint32_t n_filters, uint32_t n_workers, uint64_t max_keys,
                         filter_server_t **out)
{
    if (!filters || !out || n_filters == 0 || n_workers == 0 || n_workers > 64 || max_keys == 0) return FILTER_ERR_ARG;
    *out = nullptr;
    for (uint32_t i = 0; i < n_filters; i++)
        if (!filters[i]) return FILTER_ERR_ARG;
    filter_server *S = new (std::nothrow) filter_server();
    if (!S) return FILTER_ERR_OOM;
    S->filters.assign(filters, filters + n_filters);
    S->max_keys = max_keys;
    cudaGetDevice(&S->device);
    // admission by free device memory: every worker's staging must fit
    size_t free_b = 0, total_b = 0;
    const uint64_t per_worker = max_keys * 16;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess || per_worker * n_workers > free_b) {
        cudaGetLastError();
        delete S;
        return FILTER_ERR_OOM;
    }
    S->workers.resize(n_workers);
    int rc = FILTER_OK;
    for (Worker &W : S->workers) {
        if (cudaStreamCreateWithFlags(&W.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMalloc(&W.d_keys, max_keys * 8) != cudaSuccess || cudaMalloc(&W.d_out, max_keys * 8) != cudaSuccess ||
            cudaMallocHost(&W.h_keys, max_keys * 8) != cudaSuccess ||
            cudaMallocHost(&W.h_out, max_keys * 8) != cudaSuccess) {
            cudaGetLastError();
            rc = FILTER_ERR_OOM;
            break;
        }
    }
    if (rc != FILTER_OK) {
        free_workers(S);
        delete S;
        return rc;
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
    Req q;
    q.r = *req;
    q.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return FILTER_ERR_ARG;
        q.ticket = s->next_ticket++;
        s->outstanding.insert(q.ticket);
        s->workers[req->filter % s->workers.size()].q.push_back(q);
        s->in_flight++;
    }
    s->cv_work.notify_all();
    *ticket = q.ticket;
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
    free_workers(s);
    delete s;
    return FILTER_OK;
}

}  // extern "C"
