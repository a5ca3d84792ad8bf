// Internal declarations shared by the gpufilter CUDA sources.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/gpufilter.h"
#include "../../include/gpufilter_hash.cuh"

namespace gf {

// ---------------------------------------------------------------------------
// Error plumbing
// ---------------------------------------------------------------------------
#define GF_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) {                        \
            gf::set_last_cuda_error(e_, #call, __LINE__); \
            return FILTER_ERR_CUDA;                     \
        }                                               \
    } while (0)

void set_last_cuda_error(cudaError_t e, const char *what, int line);

// Device status word bits (sticky, atomically OR-ed by kernels).
static constexpr unsigned long long ST_FULL = 1ull << FILTER_ERR_FULL;
static constexpr unsigned long long ST_TIMEOUT = 1ull << FILTER_ERR_TIMEOUT;
static constexpr unsigned long long ST_INTERNAL = 1ull << FILTER_ERR_INTERNAL;

// Iteration cap for every spin-wait in the library's kernels. A wait that
// reaches it records ST_TIMEOUT and returns; it never traps.
static constexpr uint32_t SPIN_LIMIT = 1u << 24;

// Shared device counters of one filter: [0] status word, [1] failed keys,
// [2..] per-call scratch counters.
struct DevCounters {
    unsigned long long status;
    unsigned long long failed;
    unsigned long long backing;
    unsigned long long overflow;  // GQF merge: 1 if a run would pass the tail
    unsigned int pend[8];         // TCF: pending-list lengths per phase
    unsigned int tile_ctr[4];     // dynamic tile counters
    long long gqf_end;            // GQF merge: end of the last run (dry runs)
    unsigned int touched[4];      // TCF sparse phases: touched destinations (cursor must follow)
    unsigned int cursor[4];       // TCF sparse phases: records placed so far
    unsigned long long wflag;     // GQF counted insert: 1 if some count was 0
};
static_assert(offsetof(DevCounters, cursor) == offsetof(DevCounters, touched) + sizeof(DevCounters::touched),
              "touched and cursor are cleared together");

// ---------------------------------------------------------------------------
// Hashing (paper Sec. 5.1 fingerprint h; Sec. 4 block/tag hash). Bijective:
// xor-shifts by s >= p/2 and products with odd constants mod 2^p.
// ---------------------------------------------------------------------------
// mix64, PHash, fold_p, fingerprint, tcf_g, tcf_key_parts, tcf_bucket:
// include/gpufilter_hash.cuh (shared with the device-side API)

struct TcfGeom {
    uint64_t nb;      // blocks (power of two)
    uint64_t nbk;     // backing buckets
    uint64_t seed;
    uint32_t f, B;    // slot bits, slots per block
    uint32_t bbytes = 32;  // bytes per block (whole 32-byte sectors)
    uint32_t tsc;     // shortcut threshold 3B/4
    uint32_t tmask;   // the tag: f - vbits bits
    uint32_t vbits = 0;  // value bits below the tag in each slot
    uint32_t vmask = 0;  // (1 << vbits) - 1
};

// a block geometry other than one 32-byte sector of 8- or 16-bit slots
__host__ __device__ __forceinline__ bool tcf_custom(const TcfGeom &G) { return G.f == 12 || G.B * G.f != 256; }

// t is the key's slot with value 0: the tag shifted above the value bits
struct KeyInfo {
    uint64_t b1, b2;
    uint32_t t;
};

__host__ __device__ __forceinline__ KeyInfo tcf_keyinfo(uint64_t key, const TcfGeom &G)
{
    KeyInfo k;
    uint32_t t;
    tcf_key_parts(key, G.seed, G.nb, G.tmask, k.b1, k.b2, t);
    k.t = t << G.vbits;
    return k;
}

__host__ __device__ __forceinline__ uint64_t tcf_entry(const KeyInfo &k, uint32_t f)
{
    uint64_t lo = k.b1 < k.b2 ? k.b1 : k.b2;
    return (lo << f) | k.t;
}

// the bucket of an entry that may carry a value: chosen by the tag part only
__host__ __device__ __forceinline__ uint64_t tcf_bucket_of(uint64_t e, const TcfGeom &G)
{
    return tcf_bucket(e & ~(uint64_t)G.vmask, G.nbk);
}

// ---------------------------------------------------------------------------
// One-dimensional bulk copies between global and shared memory (the TMA's
// cp.async.bulk, sm_90 and later), completed through an mbarrier. Addresses
// 16-byte aligned, sizes a multiple of 16 bytes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one arrival that also announces `bytes` of copies completing on the barrier
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// the phase with this parity completed, or false after `limit` tries
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst_smem)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void bulk_store(void *dst, const void *src_smem, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src_smem)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// the shared-memory sources of this thread's bulk stores have been read
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// this thread's bulk stores are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// this thread's shared-memory writes become visible to the bulk copies
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Filter groups: member m of a group call owns keys [off[m], off[m + 1]).
// ---------------------------------------------------------------------------
// The member holding key i: the largest m with off[m] <= i (so empty members
// are skipped). off has n + 1 entries.
__device__ __forceinline__ uint32_t member_of(const uint64_t *off, uint32_t n, uint64_t i)
{
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Keys of a group call are split into one contiguous chunk per CTA, visited
// in steps of blockDim.x, so a thread finds its member once by binary search
// and then only steps forward.
struct MemberCursor {
    uint64_t i, end;
    uint32_t m;
    __device__ __forceinline__ MemberCursor(const uint64_t *off, uint32_t n, uint64_t n_keys)
    {
        const uint64_t per = (((n_keys + gridDim.x - 1) / gridDim.x) + 31) & ~31ull;  // warp-aligned chunks
        const uint64_t c0 = per * blockIdx.x;
        end = c0 + per < n_keys ? c0 + per : n_keys;
        i = c0 + threadIdx.x;
        m = i < end ? member_of(off, n, i) : 0;
    }
    __device__ __forceinline__ bool valid() const { return i < end; }
    __device__ __forceinline__ void next(const uint64_t *off)
    {
        i += blockDim.x;
        if (i < end)
            while (__ldg(off + m + 1) <= i) m++;
    }
};

// geometry of one TCF group member
struct TcfMember {
    uint64_t nb, nbk, seed;
    uint64_t block0, bucket0;  // its first block and bucket in the group's arrays
};

// the keys of a TCF group call, hashed for their members, as separate arrays
// so that each phase reads only what it needs (bt null: keys not prepared)
struct TcfPrep {
    uint64_t *bt;       // b1 << 32 | tag, b1 group-wide
    uint32_t *b2;       // group-wide
    uint32_t *bucket;   // group-wide backing bucket
    uint64_t *e;        // backing entry (member-local block index << f | tag)
    const uint8_t *vals = nullptr;  // single filters with values: the batch's values
};

// ---------------------------------------------------------------------------
// Scratch arena: one cudaMalloc per filter, carved into aligned pieces.
// ---------------------------------------------------------------------------
struct Arena {
    char *base = nullptr;
    size_t size = 0, used = 0;
    template <class T>
    T *take(size_t count)
    {
        size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base + used);
        used += bytes;
        return p;
    }
};

// ---------------------------------------------------------------------------
// Generic device primitives (gf_prims.cu)
// ---------------------------------------------------------------------------
// In-place-safe exclusive scan of n uint32 (out may equal in). Needs
// scan_tmp_words(n) words of temporary state. Values must sum below 2^32.
size_t scan_tmp_words(uint64_t n);
void exclusive_scan_u32(const uint32_t *in, uint32_t *out, uint64_t n, uint64_t *tmp,
                        DevCounters *ctr, cudaStream_t st);

// Run-length encoding of a sorted array: uniq[g] / start[g] for each run g,
// start[m] = n and *m_out = m (the number of runs); run_of[i] (optional) =
// the run of element i. tmp: scan_tmp_words(n) words.
void rle_sorted_u64(const uint64_t *keys, uint64_t n, uint64_t *uniq, uint32_t *start, uint32_t *run_of,
                    uint32_t *m_out, uint64_t *tmp, DevCounters *ctr, cudaStream_t st);

// LSD radix sort of 64-bit keys on bits [0, bits), optional 32-bit values.
// Result lands in keys_out / vals_out. `tmp` holds radix_tmp_words(n) words.
size_t radix_tmp_words(uint64_t n);
// first_hist_done: tmp already holds the first pass's per-tile histogram
// (from fingerprint_for_sort)
void radix_sort_u64(const uint64_t *keys_in, uint64_t *keys_out, uint64_t *keys_alt,
                    const uint32_t *vals_in, uint32_t *vals_out, uint32_t *vals_alt,
                    uint64_t n, uint32_t bits, uint32_t *tmp, uint64_t *scan_tmp,
                    DevCounters *ctr, cudaStream_t st, bool first_hist_done = false);
// fp[i] = fingerprint(keys[i], H) (idx[i] = i when idx is set), with the
// per-tile histogram of the lowest digit that radix_sort_u64(.., bits, tmp)
// takes for its first pass
void fingerprint_for_sort(const uint64_t *keys, uint64_t n, const PHash &H, uint64_t *fp, uint32_t *idx,
                          uint32_t bits, uint32_t *tmp, cudaStream_t st);

// Kernel tracing: a TraceScope around a launch records CUDA events before and
// after it when tracing is on. Launches whose work is only known on the device
// (the sparse phases) open the scope with dev_units and pass units() to the
// kernel, which adds its work units there (a null pointer when not tracing).
extern bool g_trace_on;
int trace_open(const char *name, uint64_t units, cudaStream_t st, bool dev_units);
void trace_close(int slot, cudaStream_t st);
unsigned long long *trace_units(int slot);
struct TraceScope {
    int slot;
    cudaStream_t st;
    TraceScope(const char *name, uint64_t units, cudaStream_t s, bool dev_units = false) : slot(-1), st(s)
    {
        if (g_trace_on) slot = trace_open(name, units, s, dev_units);
    }
    unsigned long long *units() const { return slot >= 0 ? trace_units(slot) : nullptr; }
    ~TraceScope()
    {
        if (slot >= 0) trace_close(slot, st);
    }
};

// Device allocations of the library go through these, so that a test can
// make the n-th one fail as if the device were full (filter_debug_fail_alloc)
// and count the allocations still held (filter_debug_live_allocations).
cudaError_t dev_malloc(void **p, size_t bytes);
cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st);
void dev_free(void *p);
void dev_free_async(void *p, cudaStream_t st);
long long live_allocations();
void fail_allocation(uint32_t nth);
// runs the look-back wait against a predecessor that never publishes, with
// `limit` loads at most; the timeout lands in ctr->status (tmp: 2 words)
void debug_wait_timeout(uint64_t *tmp, DevCounters *ctr, uint32_t limit, cudaStream_t st);

// grid size helper: a multiple of the SM count
int grid_for(uint64_t work, int threads, int per_sm = 8);
int sm_count();

}  // namespace gf

// ---------------------------------------------------------------------------
// The filter object
// ---------------------------------------------------------------------------
struct TcfState {
    gf::TcfGeom G;
    uint32_t mode;
    uint8_t *blocks;   // nb * 32
    uint64_t *bk;      // nbk * 8
    uint8_t *fill;     // nb (bulk mode)
    // scratch
    uint32_t *cnt;     // max(nb, nbk) + 1, kept zero between phases
    uint32_t *off;     // max(nb, nbk) + 1
    uint64_t *rec;     // max_batch
    uint32_t *pend0;   // max_batch
    uint64_t *pend1;   // max_batch
    uint32_t *pend2;   // max_batch
    // sparse phases: destinations touched per CTA chunk, then the dense list
    // of touched destinations with their record segments
    uint32_t *tlist;   // max_batch
    uint32_t *tcount;  // one per CTA of a phase launch
    uint32_t *dlist;   // max_batch
    uint64_t *seg;     // max_batch: start << 32 | count
    // tiled phases: per-tile counts and cursors, and a second pending list
    uint32_t *tcur;    // 2 * ceil(nb / 32) + 264
    uint64_t *pb;      // max_batch
    uint32_t *pbi;     // max_batch
};

struct GqfState {
    uint32_t q, r, p;
    uint64_t N, S, nslots, nblk, ntiles;
    gf::PHash H;
    uint8_t *meta[2];  // nblk * 32
    uint8_t *rem[2];   // nslots * r/8
    int cur;           // which buffer holds the table
    uint32_t *locks;   // point updates: a lock word per 8192 quotients, 128 bytes apart
    uint64_t nlocks;
    bool merge_only;   // inserts always merge into the other buffer (no in-place path)
    // scratch
    uint64_t *fp_a, *fp_b, *fp_c;  // max_batch
    uint32_t *idx_a, *idx_b, *idx_c;
    uint64_t *ufp;     // unique fingerprints
    uint32_t *ustart;  // group start in the sorted batch (+1 sentinel)
    uint32_t *flags;   // max_batch + 1
    uint32_t *removed; // per group: copies removed (delete) / accepted flag
    unsigned long long *tile_state;  // ntiles * 4 (look-back)
    uint32_t *tile_lo;               // ntiles + 1: first group of each tile
    uint32_t *radix_tmp;
};

struct filter {
    filter_config cfg{};
    filter_tuning tune{};
    gf::Arena arena;
    void *table_mem = nullptr;
    size_t table_bytes_alloc = 0;
    gf::DevCounters *ctr = nullptr;
    uint64_t *scan_tmp = nullptr;
    TcfState tcf;
    GqfState gqf;
    int device = 0;
};

// A group of filters of one kind sharing one allocation and one set of
// launches per call. members[m] is a host-side view of member m whose table
// pointers point into the group's arrays and whose scratch is the group's.
struct filter_group {
    filter_tuning tune{};
    uint32_t kind = 0, n = 0;
    uint32_t bits = 0;          // TCF f / GQF r, shared by all members
    uint64_t max_total = 0;
    gf::Arena arena;
    gf::DevCounters *ctr = nullptr;   // group-wide (TCF counters; GQF overflow list length)
    gf::DevCounters *mctr = nullptr;  // GQF: one per member
    uint64_t *scan_tmp = nullptr;
    filter *members = nullptr;
    int device = 0;
    // TCF: concatenated blocks, buckets and fill bytes; G.nb / G.nbk are the totals
    TcfState tcf;
    gf::TcfMember *d_tmem = nullptr;
    gf::TcfPrep prep{nullptr, nullptr, nullptr, nullptr};
    // GQF: meta[b] / rem[b] are the concatenated regions of all members
    GqfState gqf;
    uint64_t tiles = 0;               // total merge tiles
    uint32_t pbits = 0, mbits = 0;    // sort key = member << pbits | fingerprint
    void *d_margs = nullptr;          // merge arguments [cur][del][member]
    void *d_gmem = nullptr;           // per-member hash and table descriptors
    uint32_t *d_tile_member = nullptr;
    uint32_t *d_ovf = nullptr;        // members that overflowed in the last insert
    uint64_t *d_mblk0 = nullptr;      // GQF: each member's first 64-slot block (n + 1 entries)
    int cur = 0;
};

namespace gf {
// tuning values with the defaults filled in; false if one is out of range
bool tuning_valid(const filter_tuning &t);
// TCF bulk calls: the tiled path for this table and batch?
bool tcf_tiled(const filter_tuning &t, uint64_t nb, uint64_t n);
bool tcf_geom_supported(uint32_t f, uint32_t B);
uint32_t tcf_tile_target(const filter_tuning &t);
uint64_t gqf_region_groups(const filter_tuning &t);
int tcf_group_setup(filter_group *G, const filter_config *cfgs, uint64_t &bytes, bool plan_only);
int tcf_group_clear(filter_group *G, cudaStream_t st);
int tcf_group_op(filter_group *G, int op, const uint64_t *off, const uint64_t *keys, uint64_t n, uint8_t *out,
                 cudaStream_t st);
int gqf_group_setup(filter_group *G, const filter_config *cfgs, uint64_t &bytes, bool plan_only);
int gqf_group_clear(filter_group *G, cudaStream_t st);
int gqf_group_insert(filter_group *G, const uint64_t *off, const uint64_t *keys, uint64_t n, uint8_t *status,
                     cudaStream_t st);
int gqf_group_remove(filter_group *G, const uint64_t *off, const uint64_t *keys, uint64_t n, uint8_t *status,
                     cudaStream_t st);
int gqf_group_count(filter_group *G, const uint64_t *off, const uint64_t *keys, uint64_t n, uint64_t *counts,
                    uint8_t *found, cudaStream_t st);
// Insert (del = 0) or remove (del = 1) without any host synchronisation: the
// merge goes to the spare buffer and every member whose merge fit is copied
// back, so the current buffer never changes; a member whose insert does not
// fit keeps its table and its keys get FILTER_KEY_FULL.
int gqf_group_update_async(filter_group *G, const uint64_t *off, const uint64_t *keys, uint64_t n, uint8_t *status,
                           int del, cudaStream_t st);
enum GroupOp : int { GROUP_INSERT = 0, GROUP_REMOVE = 1, GROUP_QUERY = 2 };

int tcf_setup(filter *F, uint64_t &table_bytes, uint64_t &scratch_bytes, bool plan_only);
int tcf_clear(filter *F, cudaStream_t st);
int tcf_insert(filter *F, const uint64_t *keys, const uint8_t *vals, uint64_t n, uint8_t *status, cudaStream_t st);
int tcf_query(filter *F, const uint64_t *keys, uint64_t n, uint8_t *found, bool values, cudaStream_t st);
int tcf_remove(filter *F, const uint64_t *keys, uint64_t n, uint8_t *status, cudaStream_t st);
uint64_t tcf_image_bytes(const filter *F);
int tcf_copy_image(filter *F, void *host, bool to_host, cudaStream_t st);

int gqf_setup(filter *F, uint64_t &table_bytes, uint64_t &scratch_bytes, bool plan_only);
uint64_t gqf_tile_lo_words(const GqfState &Q);
int gqf_clear(filter *F, cudaStream_t st);
int gqf_insert(filter *F, const uint64_t *keys, const uint32_t *counts, uint64_t n, uint8_t *status,
               cudaStream_t st);
int gqf_remove(filter *F, const uint64_t *keys, uint64_t n, uint8_t *status, cudaStream_t st);
int gqf_point_update(filter *F, const uint64_t *keys, uint64_t n, int remove, uint8_t *status, cudaStream_t st);
int gqf_count(filter *F, const uint64_t *keys, uint64_t n, uint64_t *counts, uint8_t *found,
              cudaStream_t st);
uint64_t gqf_image_bytes(const filter *F);
int gqf_copy_image(filter *F, void *host, bool to_host, cudaStream_t st);
int gqf_enumerate(filter *F, uint64_t *fps, uint64_t *counts, uint64_t cap, uint64_t *n_out, cudaStream_t st);
int gqf_unhash(filter *F, const uint64_t *fps, uint64_t n, uint64_t *keys, cudaStream_t st);
}  // namespace gf
