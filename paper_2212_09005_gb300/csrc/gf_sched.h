// Admission and batching policy of the serving loop, in plain C++ (no CUDA),
// so that it can be exercised on a host without a GPU.
//
// Requests wait in one FIFO per filter. A filter has at most one batch in
// flight, so its requests are applied in submission order whatever else runs
// beside them. Any idle worker may take the oldest waiting request of any
// filter that is not in flight (continuous batching: a request that arrives
// while others are on the GPU starts as soon as a worker, its filter and
// staging memory are free). The batch it takes is that request plus the
// requests queued right behind it on the same filter whose merged result is
// provably the same as running them one after the other:
//   - queries and counts (read only: the table does not change in between);
//   - removes from a GQF (its table is a function of the stored multiset, and
//     the keys of the earlier request come first in the merged batch, so the
//     copies that are not found are the same ones).
// TCF inserts and removes, and GQF inserts (whose kept prefix on overflow
// depends on the batch), always run alone.
//
// Admission by device memory: each batch reserves its staging (8 bytes per
// key and the result bytes) in a fixed pool, first fit. A batch that does not
// fit waits until running batches release their space; a request larger than
// the whole pool is refused at submission. To keep a large request from
// waiting for ever behind a stream of small ones, once the oldest waiting
// batch has been passed over `max_skips` times nothing else is admitted until
// it fits.
#pragma once

#include <algorithm>
#include <cstdint>
#include <deque>
#include <iterator>
#include <map>
#include <vector>

namespace gfsched {

enum Op : uint32_t { OP_INSERT = 0, OP_QUERY = 1, OP_REMOVE = 2, OP_COUNT = 3 };

struct Req {
    uint64_t ticket;
    uint32_t filter, op;
    uint64_t n;
    uint64_t seq;  // arrival order
};

struct Batch {
    uint32_t filter = 0, op = 0;
    uint64_t n = 0;            // keys over all merged requests
    uint64_t offset = 0;       // staging reservation in the pool
    uint64_t bytes = 0;
    std::vector<Req> reqs;     // in submission order
};

inline uint64_t result_bytes(uint32_t op) { return op == OP_COUNT ? 8 : 1; }
inline uint64_t staging_bytes(uint32_t op, uint64_t n)
{
    // keys + results, each rounded to 256 bytes so that every piece stays aligned
    return ((n * 8 + 255) & ~255ull) + ((n * result_bytes(op) + 255) & ~255ull);
}

// first-fit allocator over [0, size)
class Pool {
   public:
    explicit Pool(uint64_t size) : size_(size) { free_[0] = size; }
    uint64_t size() const { return size_; }
    uint64_t available() const
    {
        uint64_t a = 0;
        for (auto &kv : free_) a += kv.second;
        return a;
    }
    bool alloc(uint64_t bytes, uint64_t &off)
    {
        if (bytes == 0) bytes = 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                off = it->first;
                const uint64_t rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t bytes)
    {
        if (bytes == 0) bytes = 256;
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

   private:
    uint64_t size_;
    std::map<uint64_t, uint64_t> free_;  // offset -> bytes
};

class Scheduler {
   public:
    // merge_removes[f]: removes on filter f may be merged (GQF);
    // max_merge[f]: the largest merged batch of filter f (its scratch bound)
    Scheduler(const std::vector<bool> &merge_removes, const std::vector<uint64_t> &max_merge, uint64_t pool_bytes,
              uint32_t max_skips = 8)
        : merge_removes_(merge_removes),
          max_merge_(max_merge),
          q_(merge_removes.size()),
          busy_(merge_removes.size(), false),
          pool_(pool_bytes),
          max_skips_(max_skips)
    {
    }

    // false: the request can never be admitted (more staging than the pool)
    bool submit(uint64_t ticket, uint32_t filter, uint32_t op, uint64_t n)
    {
        if (filter >= q_.size() || staging_bytes(op, n) > pool_.size()) return false;
        q_[filter].push_back(Req{ticket, filter, op, n, seq_++});
        waiting_++;
        return true;
    }

    // The next batch to run, if one can start now.
    bool next(Batch &b)
    {
        // waiting filters, oldest head first
        std::vector<std::pair<uint64_t, uint32_t>> heads;
        for (uint32_t f = 0; f < q_.size(); f++)
            if (!busy_[f] && !q_[f].empty()) heads.emplace_back(q_[f].front().seq, f);
        if (heads.empty()) return false;
        std::sort(heads.begin(), heads.end());
        int best = -1;
        for (size_t h = 0; h < heads.size() && best < 0; h++) {
            const uint32_t f = heads[h].second;
            // the merged batch, else the head request alone
            for (int merge = 1; merge >= 0 && best < 0; merge--) {
                Batch c = form(f, merge != 0);
                if (pool_.alloc(c.bytes, c.offset)) {
                    best = (int)f;
                    b = c;
                }
                if (c.reqs.size() == 1) break;
            }
            // the oldest head does not fit: count the pass-over, and once it
            // has waited long enough, admit nothing ahead of it
            if (best < 0 && h == 0) {
                if (q_[f].front().seq != starving_seq_) {
                    starving_seq_ = q_[f].front().seq;
                    skips_ = 0;
                }
                if (skips_ >= max_skips_) return false;
            }
        }
        if (best < 0) return false;
        if (heads[0].second != (uint32_t)best && heads[0].first == starving_seq_) skips_++;
        for (size_t k = 0; k < b.reqs.size(); k++) q_[best].pop_front();
        busy_[best] = true;
        waiting_ -= b.reqs.size();
        running_++;
        return true;
    }

    void finish(const Batch &b)
    {
        pool_.release(b.offset, b.bytes);
        busy_[b.filter] = false;
        running_--;
    }

    uint64_t waiting() const { return waiting_; }
    uint64_t running() const { return running_; }
    uint64_t pool_available() const { return pool_.available(); }
    uint64_t pool_size() const { return pool_.size(); }

   private:
    bool mergeable(uint32_t f, uint32_t op) const
    {
        return op == OP_QUERY || op == OP_COUNT || (op == OP_REMOVE && merge_removes_[f]);
    }

    // the head request of filter f and (merge) the mergeable requests right
    // behind it, up to max_merge[f] keys in all
    Batch form(uint32_t f, bool merge) const
    {
        Batch b;
        b.filter = f;
        const Req &h = q_[f].front();
        b.op = h.op;
        b.reqs.push_back(h);
        b.n = h.n;
        if (merge && mergeable(f, h.op)) {
            for (size_t k = 1; k < q_[f].size(); k++) {
                const Req &r = q_[f][k];
                if (r.op != h.op || b.n + r.n > max_merge_[f] || staging_bytes(h.op, b.n + r.n) > pool_.size())
                    break;
                b.reqs.push_back(r);
                b.n += r.n;
            }
        }
        b.bytes = staging_bytes(b.op, b.n);
        return b;
    }

    std::vector<bool> merge_removes_;
    std::vector<uint64_t> max_merge_;
    std::vector<std::deque<Req>> q_;
    std::vector<bool> busy_;
    Pool pool_;
    uint32_t max_skips_;
    uint64_t seq_ = 0, waiting_ = 0, running_ = 0;
    uint64_t starving_seq_ = ~0ull;
    uint32_t skips_ = 0;
};

}  // namespace gfsched
