// Host-side driver for the serving loop's scheduler (gf_sched.h), for the
// CPU tests: the admission budget is a plain number of bytes here, so a test
// can make memory scarce at will and watch what gets admitted.
#include "gf_sched.h"

using gfsched::Batch;
using gfsched::Scheduler;

struct Shim {
    Scheduler *s;
};

extern "C" {

void *sched_new(uint32_t n_filters, const uint8_t *merge_removes, const uint64_t *max_merge, uint64_t pool_bytes,
                uint32_t max_skips)
{
    std::vector<bool> mr(n_filters);
    std::vector<uint64_t> mm(n_filters);
    for (uint32_t i = 0; i < n_filters; i++) {
        mr[i] = merge_removes[i] != 0;
        mm[i] = max_merge[i];
    }
    return new Scheduler(mr, mm, pool_bytes, max_skips);
}

void sched_free(void *h) { delete static_cast<Scheduler *>(h); }

int sched_submit(void *h, uint64_t ticket, uint32_t filter, uint32_t op, uint64_t n)
{
    return static_cast<Scheduler *>(h)->submit(ticket, filter, op, n) ? 1 : 0;
}

// out: [filter, op, n, offset, bytes, n_reqs, tickets...]; returns 0 if no batch can start
int sched_next(void *h, uint64_t *out, uint32_t cap)
{
    Batch b;
    if (!static_cast<Scheduler *>(h)->next(b)) return 0;
    out[0] = b.filter;
    out[1] = b.op;
    out[2] = b.n;
    out[3] = b.offset;
    out[4] = b.bytes;
    out[5] = b.reqs.size();
    for (size_t k = 0; k < b.reqs.size() && 6 + k < cap; k++) out[6 + k] = b.reqs[k].ticket;
    return 1;
}

void sched_finish(void *h, uint32_t filter, uint32_t op, uint64_t n, uint64_t offset, uint64_t bytes)
{
    Batch b;
    b.filter = filter;
    b.op = op;
    b.n = n;
    b.offset = offset;
    b.bytes = bytes;
    static_cast<Scheduler *>(h)->finish(b);
}

uint64_t sched_pool_available(void *h) { return static_cast<Scheduler *>(h)->pool_available(); }
uint64_t sched_waiting(void *h) { return static_cast<Scheduler *>(h)->waiting(); }
uint64_t sched_staging_bytes(uint32_t op, uint64_t n) { return gfsched::staging_bytes(op, n); }
}
