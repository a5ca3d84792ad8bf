// Generic device primitives: exclusive scan (single pass, decoupled
// look-back) and LSD radix sort of 64-bit keys with optional 32-bit values.
// The GQF sorts fingerprints before inserting them (paper Sec. 5.3, "Sorting
// hashes"); the TCF groups batches by block with the scan.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "gf_internal.cuh"

namespace gf {

static int g_sm_count = 0;

int sm_count()
{
    if (g_sm_count == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            g_sm_count <= 0)
            g_sm_count = 152;
    }
    return g_sm_count;
}

// 0: no injected failure; k > 0: the k-th allocation from now fails
static std::atomic<uint32_t> g_fail_nth{0};
static std::atomic<long long> g_live_allocs{0};

static bool injected_failure()
{
    uint32_t k = g_fail_nth.load();
    while (k != 0) {
        if (g_fail_nth.compare_exchange_weak(k, k - 1)) return k == 1;
    }
    return false;
}

cudaError_t dev_malloc(void **p, size_t bytes)
{
    *p = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) g_live_allocs++;
    else *p = nullptr;
    return e;
}

cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st)
{
    *p = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e == cudaSuccess) g_live_allocs++;
    else *p = nullptr;
    return e;
}

void dev_free(void *p)
{
    if (!p) return;
    cudaFree(p);
    g_live_allocs--;
}

void dev_free_async(void *p, cudaStream_t st)
{
    if (!p) return;
    cudaFreeAsync(p, st);
    g_live_allocs--;
}

long long live_allocations() { return g_live_allocs.load(); }
void fail_allocation(uint32_t nth) { g_fail_nth.store(nth); }

int grid_for(uint64_t work, int threads, int per_sm)
{
    uint64_t want = (work + threads - 1) / threads;
    uint64_t cap = (uint64_t)sm_count() * per_sm;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    return (int)want;
}

// ---------------------------------------------------------------------------
// Exclusive scan. Tiles of SCAN_T threads x SCAN_I items; tile order taken
// from an atomic counter so that every tile's predecessors are running or
// done. State word per tile: (flag << 32) | value, flag 1 = tile aggregate,
// 2 = inclusive prefix.
// ---------------------------------------------------------------------------
static constexpr int SCAN_T = 256;
static constexpr int SCAN_I = 16;
static constexpr uint64_t SCAN_TILE = SCAN_T * SCAN_I;
static_assert(SCAN_TILE <= 65536, "positions inside a tile fit 16 bits");

size_t scan_tmp_words(uint64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 2; }

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long *p)
{
    return *(const volatile unsigned long long *)p;
}

// Warp 0 of tile `tile`: publish the tile's total, look back over 32
// predecessors at a time for the exclusive prefix, publish the inclusive one.
// All 32 lanes call it and get the prefix. A wait that reaches SPIN_LIMIT
// records ST_TIMEOUT and gives up (prefix then incomplete).
__device__ uint32_t lookback_prefix(unsigned long long *st, uint64_t tile, uint32_t total,
                                    unsigned long long *status, uint32_t limit = SPIN_LIMIT)
{
    const int lane = threadIdx.x & 31;
    uint32_t prefix = 0;
    if (tile == 0) {
        if (lane == 0) atomicExch(&st[0], (2ull << 32) | total);
        return 0;
    }
    if (lane == 0) atomicExch(&st[tile], (1ull << 32) | total);
    int64_t jtop = (int64_t)tile - 1;
    uint32_t spins = 0;
    while (true) {
        const int64_t j = jtop - lane;
        unsigned long long w2 = 2ull << 32;  // before tile 0: inclusive prefix 0
        if (j >= 0) {
            w2 = ld_volatile(&st[j]);
            while ((w2 >> 32) == 0 && ++spins <= limit) w2 = ld_volatile(&st[j]);
        }
        const uint32_t flag = (uint32_t)(w2 >> 32);
        if (__ballot_sync(0xffffffffu, flag == 0)) {
            if (lane == 0) atomicOr(status, ST_TIMEOUT);
            break;
        }
        const unsigned incl_mask = __ballot_sync(0xffffffffu, flag == 2);
        const int L = incl_mask ? __ffs(incl_mask) - 1 : 31;
        uint32_t part = (lane <= L) ? (uint32_t)w2 : 0u;
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        prefix += part;
        if (incl_mask) break;
        jtop -= 32;
    }
    if (lane == 0) atomicExch(&st[tile], (2ull << 32) | (uint32_t)(prefix + total));
    return prefix;
}

__global__ void __launch_bounds__(SCAN_T) scan_kernel(const uint32_t *in, uint32_t *out, uint64_t n,
                                                      unsigned long long *tmp,
                                                      unsigned long long *status)
{
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_warp[SCAN_T / 32];
    __shared__ uint32_t s_prefix;
    if (threadIdx.x == 0) s_tile = (uint32_t)atomicAdd(&tmp[0], 1ull);
    __syncthreads();
    const uint64_t tile = s_tile;
    unsigned long long *st = tmp + 1;
    const uint64_t base = tile * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_I;
    uint32_t v[SCAN_I];
    if (base + SCAN_I <= n) {
        const uint4 *p = reinterpret_cast<const uint4 *>(in + base);
#pragma unroll
        for (int k = 0; k < SCAN_I / 4; k++) {
            uint4 q = p[k];
            v[4 * k] = q.x;
            v[4 * k + 1] = q.y;
            v[4 * k + 2] = q.z;
            v[4 * k + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < SCAN_I; k++) v[k] = (base + k < n) ? in[base + k] : 0u;
    }
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_I; k++) {
        uint32_t x = v[k];
        v[k] = sum;
        sum += x;
    }
    // block-wide exclusive scan of the thread sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < SCAN_T / 32 ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < SCAN_T / 32) s_warp[lane] = wi - w;
        // tile total sits in lane 7
        const uint32_t total = __shfl_sync(0xffffffffu, wi, SCAN_T / 32 - 1);
        const uint32_t prefix = lookback_prefix(st, tile, total, status);
        if (lane == 0) s_prefix = prefix;
    }
    __syncthreads();
    const uint32_t add = s_prefix + s_warp[warp] + (incl - sum);
    if (base + SCAN_I <= n) {
        uint4 *p = reinterpret_cast<uint4 *>(out + base);
#pragma unroll
        for (int k = 0; k < SCAN_I / 4; k++)
            p[k] = make_uint4(v[4 * k] + add, v[4 * k + 1] + add, v[4 * k + 2] + add, v[4 * k + 3] + add);
    } else {
#pragma unroll
        for (int k = 0; k < SCAN_I; k++)
            if (base + k < n) out[base + k] = v[k] + add;
    }
}

// A look-back whose predecessor never publishes: tile 1 of a two-tile state
// array whose tile 0 stays empty. The wait gives up after `limit` loads and
// records ST_TIMEOUT in `status` (the self-test of the bounded waits).
__global__ void debug_lookback_kernel(unsigned long long *st, unsigned long long *status, uint32_t limit)
{
    lookback_prefix(st, 1, 1, status, limit);
}

void debug_wait_timeout(uint64_t *tmp, DevCounters *ctr, uint32_t limit, cudaStream_t st)
{
    cudaMemsetAsync(tmp, 0, 2 * sizeof(uint64_t), st);
    debug_lookback_kernel<<<1, 32, 0, st>>>((unsigned long long *)tmp, &ctr->status, limit);
}

void exclusive_scan_u32(const uint32_t *in, uint32_t *out, uint64_t n, uint64_t *tmp,
                        DevCounters *ctr, cudaStream_t st)
{
    if (n == 0) return;
    uint64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    cudaMemsetAsync(tmp, 0, (tiles + 1) * sizeof(uint64_t), st);
    TraceScope ts_("scan_kernel", n, st);
    scan_kernel<<<(unsigned)tiles, SCAN_T, 0, st>>>(in, out, n, (unsigned long long *)tmp,
                                                   &ctr->status);
}

// ---------------------------------------------------------------------------
// Run-length encoding of a sorted array in one pass: each run's first key and
// start, the number of runs, and optionally each element's run index. Run
// starts are counted per tile and ranked by the same decoupled look-back as
// the scan.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SCAN_T) rle_kernel(const uint64_t *__restrict__ keys, uint64_t n,
                                                     uint64_t *__restrict__ uniq, uint32_t *__restrict__ start,
                                                     uint32_t *__restrict__ run_of, uint32_t *m_out,
                                                     unsigned long long *tmp, unsigned long long *status)
{
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_warp[SCAN_T / 32];
    __shared__ uint32_t s_prefix, s_total;
    __shared__ uint64_t s_key[SCAN_TILE];  // the tile's groups in order: first key,
    __shared__ uint16_t s_pos[SCAN_TILE];  // and start within the tile
    if (threadIdx.x == 0) s_tile = (uint32_t)atomicAdd(&tmp[0], 1ull);
    __syncthreads();
    const uint64_t tile = s_tile;
    const uint64_t base = tile * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_I;
    uint64_t k[SCAN_I];
    if (base + SCAN_I <= n) {
        const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(keys + base);
#pragma unroll
        for (int q = 0; q < SCAN_I / 2; q++) {
            const ulonglong2 v = __ldcs(p + q);
            k[2 * q] = v.x;
            k[2 * q + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < SCAN_I; q++) k[q] = (base + q < n) ? keys[base + q] : 0ull;
    }
    uint64_t prev = (base > 0 && base - 1 < n) ? keys[base - 1] : ~k[0];
    uint32_t starts = 0;  // bit q: element base + q starts a run
#pragma unroll
    for (int q = 0; q < SCAN_I; q++) {
        if (base + q < n && k[q] != prev) starts |= 1u << q;
        prev = k[q];
    }
    const uint32_t sum = __popc(starts);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < SCAN_T / 32 ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < SCAN_T / 32) s_warp[lane] = wi - w;
        const uint32_t total = __shfl_sync(0xffffffffu, wi, SCAN_T / 32 - 1);
        const uint32_t prefix = lookback_prefix(tmp + 1, tile, total, status);
        if (lane == 0) {
            s_prefix = prefix;
            s_total = total;
        }
    }
    __syncthreads();
    // groups are staged in shared memory in order, then written as whole lines
    uint32_t lg = s_warp[warp] + (incl - sum);  // the tile's runs started before this thread's elements
    const uint32_t g0 = s_prefix;
    uint32_t rv[SCAN_I];
#pragma unroll
    for (int q = 0; q < SCAN_I; q++) {
        if ((starts >> q) & 1u) {
            s_key[lg] = k[q];
            s_pos[lg] = (uint16_t)(threadIdx.x * SCAN_I + q);
            lg++;
        }
        rv[q] = g0 + lg - 1;
        if (base + q == n - 1) {
            *m_out = g0 + lg;
            start[g0 + lg] = (uint32_t)n;
        }
    }
    __syncthreads();
    const uint32_t tot = s_total;
    for (uint32_t x = threadIdx.x; x < tot; x += SCAN_T) {
        uniq[g0 + x] = s_key[x];
        start[g0 + x] = (uint32_t)(tile * SCAN_TILE) + s_pos[x];
    }
    if (run_of) {
        if (base + SCAN_I <= n) {
            uint4 *p = reinterpret_cast<uint4 *>(run_of + base);
#pragma unroll
            for (int q = 0; q < SCAN_I / 4; q++) p[q] = make_uint4(rv[4 * q], rv[4 * q + 1], rv[4 * q + 2], rv[4 * q + 3]);
        } else {
#pragma unroll
            for (int q = 0; q < SCAN_I; q++)
                if (base + q < n) run_of[base + q] = rv[q];
        }
    }
}

void rle_sorted_u64(const uint64_t *keys, uint64_t n, uint64_t *uniq, uint32_t *start, uint32_t *run_of,
                    uint32_t *m_out, uint64_t *tmp, DevCounters *ctr, cudaStream_t st)
{
    if (n == 0) {
        cudaMemsetAsync(m_out, 0, 4, st);
        cudaMemsetAsync(start, 0, 4, st);
        return;
    }
    const uint64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    cudaMemsetAsync(tmp, 0, (tiles + 1) * sizeof(uint64_t), st);
    TraceScope ts_("rle_kernel", n, st);
    rle_kernel<<<(unsigned)tiles, SCAN_T, 0, st>>>(keys, n, uniq, start, run_of, m_out, (unsigned long long *)tmp,
                                                  &ctr->status);
}

// ---------------------------------------------------------------------------
// LSD radix sort with digits of up to 9 bits (the fewest passes that cover the
// key bits, e.g. 4 x 9 bits for 36-bit fingerprints). Per pass: per-tile digit
// histograms, one exclusive scan over the digit-major count matrix, then a
// stable scatter that ranks each tile's keys with warp match and stages them
// in shared memory so that the global writes are runs of consecutive
// addresses.
// ---------------------------------------------------------------------------
static constexpr int RS_T = 256;
static constexpr int RS_I = 16;
static constexpr int RS_TILE = RS_T * RS_I;
static constexpr int RS_WARPS = RS_T / 32;
static constexpr int RS_MAXB = 512;  // buckets of the widest digit
static_assert(RS_MAXB == 2 * RS_T, "the scatter's scan gives each thread two digits");
static_assert(RS_TILE < (1 << 16), "tile positions fit the 16-bit counters");

size_t radix_tmp_words(uint64_t n)
{
    uint64_t tiles = (n + RS_TILE - 1) / RS_TILE;
    return tiles * RS_MAXB + 1;
}

// Per-tile digit counts. Each warp counts into its own shared histogram
// with plain shared atomics (equal digits inside one warp serialise on one
// address, which is cheaper than ranking them), then the warps' counts are
// summed per digit.
__global__ void __launch_bounds__(RS_T) rs_hist(const uint64_t *__restrict__ keys, uint64_t n, uint32_t shift,
                                                uint32_t nb, uint32_t *counts, uint64_t ntiles)
{
    __shared__ uint32_t h[RS_WARPS][RS_MAXB];
    for (int i = threadIdx.x; i < RS_WARPS * RS_MAXB; i += RS_T) (&h[0][0])[i] = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    const uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
    uint64_t k[RS_I];
#pragma unroll
    for (int r = 0; r < RS_I; r++) {
        uint64_t i = base + (uint64_t)r * RS_T + threadIdx.x;
        k[r] = (i < n) ? __ldcs(keys + i) : 0;
    }
#pragma unroll
    for (int r = 0; r < RS_I; r++) {
        uint64_t i = base + (uint64_t)r * RS_T + threadIdx.x;
        if (i < n) atomicAdd(&h[warp][(uint32_t)(k[r] >> shift) & (nb - 1)], 1u);
    }
    __syncthreads();
    for (uint32_t d = threadIdx.x; d < nb; d += RS_T) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) c += h[w][d];
        counts[(uint64_t)d * ntiles + blockIdx.x] = c;
    }
}

// The same first-pass histogram fused with the fingerprinting that feeds
// the sort: keys are hashed (H), the fingerprints written (with their batch
// indices when wanted) and counted by their lowest digit, so that the sort's
// first pass needs no histogram pass of its own.
__global__ void __launch_bounds__(RS_T) rs_fp_hist(const uint64_t *__restrict__ keys, uint64_t n, PHash H,
                                                   uint64_t *__restrict__ fp, uint32_t *__restrict__ idx, uint32_t nb,
                                                   uint32_t *counts, uint64_t ntiles)
{
    __shared__ uint32_t h[RS_WARPS][RS_MAXB];
    for (int i = threadIdx.x; i < RS_WARPS * RS_MAXB; i += RS_T) (&h[0][0])[i] = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    const uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
    uint64_t k[RS_I];
#pragma unroll
    for (int r = 0; r < RS_I; r++) {
        uint64_t i = base + (uint64_t)r * RS_T + threadIdx.x;
        k[r] = (i < n) ? __ldcs(keys + i) : 0;
    }
#pragma unroll
    for (int r = 0; r < RS_I; r++) {
        uint64_t i = base + (uint64_t)r * RS_T + threadIdx.x;
        if (i < n) {
            const uint64_t f = fingerprint(k[r], H);
            fp[i] = f;
            if (idx) idx[i] = (uint32_t)i;
            atomicAdd(&h[warp][(uint32_t)f & (nb - 1)], 1u);
        }
    }
    __syncthreads();
    for (uint32_t d = threadIdx.x; d < nb; d += RS_T) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) c += h[w][d];
        counts[(uint64_t)d * ntiles + blockIdx.x] = c;
    }
}

// Scatter of one pass. Keys are ranked inside each warp: a round's lanes
// with equal digits are found with one ballot per digit bit (DB > 0: the
// digit width is a compile-time constant and the lanes that differ are
// accumulated with one ballot and one logic operation per bit), or with
// match_any when the round is a single run of one digit (long runs of equal
// keys, which the earlier passes of a skewed key set produce); a per-warp
// 16-bit counter per digit carries the rank across the warp's 16 rounds. A
// scan in shared memory, two digits per thread on packed counter pairs, turns
// the counters into one tile position per (warp, digit), the keys are staged
// in digit order, and the copy-out writes runs of consecutive addresses,
// taking each key's global position from its digit's offset. Shared memory
// and registers are sized for 3 CTAs per SM (2 with values).
//
// STABLE = false (the first pass of a sort without values): the order of keys
// with equal digits does not matter, because keys that agree in every sorted
// bit are identical (the callers sort fingerprints with nothing above the
// sorted bits) and the later passes are stable. Each key then takes its rank
// with one shared-memory atomic on its (warp, digit) counter instead of the
// ballots.
template <bool VALS, int DB, bool STABLE = true>
__global__ void __launch_bounds__(RS_T, VALS ? 2 : 3) rs_scatter(const uint64_t *__restrict__ kin,
                                                                 uint64_t *__restrict__ kout,
                                                                 const uint32_t *__restrict__ vin,
                                                                 uint32_t *__restrict__ vout, uint64_t n,
                                                                 uint32_t shift, uint32_t nb,
                                                                 const uint32_t *__restrict__ offs, uint64_t ntiles)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *skeys = reinterpret_cast<uint64_t *>(smem);              // [RS_TILE] keys in digit order
    uint32_t *svals = reinterpret_cast<uint32_t *>(skeys + RS_TILE);   // [RS_TILE] values (VALS)
    uint32_t *gdelta = svals + (VALS ? RS_TILE : 0);                   // [RS_MAXB] global start - tile start
    uint16_t *wcnt = reinterpret_cast<uint16_t *>(gdelta + RS_MAXB);    // [RS_WARPS][RS_MAXB]
    __shared__ uint32_t s_w[RS_WARPS];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RS_MAXB / 8; i += RS_T) reinterpret_cast<uint4 *>(wcnt)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();

    const uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
    const unsigned lt = (1u << lane) - 1u;
    uint64_t key[RS_I];
    uint32_t val[RS_I];
    uint16_t rank[RS_I];
    // all loads first, so that the tile's 16 keys per thread are in flight together
#pragma unroll
    for (int r = 0; r < RS_I; r++) {
        uint64_t i = base + (uint64_t)warp * (RS_I * 32) + r * 32 + lane;
        bool ok = i < n;
        key[r] = ok ? __ldcs(kin + i) : 0;
        if (VALS) val[r] = ok ? __ldcs(vin + i) : 0;
    }
#pragma unroll
    for (int r = 0; r < RS_I && !STABLE; r++) {
        const uint64_t i = base + (uint64_t)warp * (RS_I * 32) + r * 32 + lane;
        const bool ok = i < n;
        const uint32_t d = ok ? ((uint32_t)(key[r] >> shift) & (nb - 1)) : 0xffffu;
        const uint32_t dprev = __shfl_up_sync(0xffffffffu, d, 1);
        uint32_t *w32 = reinterpret_cast<uint32_t *>(wcnt) + warp * (RS_MAXB / 2) + (d >> 1);
        const uint32_t sh = (d & 1u) * 16u;  // the counters are 16-bit halves of 32-bit words; no half carries
        if (__ballot_sync(0xffffffffu, lane == 0 || d != dprev) == 1u) {
            // one run of one digit (skewed keys; a round is all valid or all
            // past the end, whose digit differs): lane order, one update by lane 0
            uint32_t b = 0;
            if (lane == 0 && ok) b = atomicAdd(w32, 32u << sh) >> sh;
            b = __shfl_sync(0xffffffffu, b, 0) & 0xffffu;
            rank[r] = (uint16_t)(b + lane);
        } else if (ok) {
            rank[r] = (uint16_t)(atomicAdd(w32, 1u << sh) >> sh);
        }
    }
#pragma unroll
    for (int r = 0; r < RS_I && STABLE; r++) {
        uint64_t i = base + (uint64_t)warp * (RS_I * 32) + r * 32 + lane;
        bool ok = i < n;
        uint32_t d = ok ? ((uint32_t)(key[r] >> shift) & (nb - 1)) : 0xffffu;
        unsigned peers;
        const uint32_t dprev = __shfl_up_sync(0xffffffffu, d, 1);
        if (__ballot_sync(0xffffffffu, lane == 0 || d != dprev) == 1u) {
            peers = __match_any_sync(0xffffffffu, d);  // one run: the cheap case of match_any
        } else if (DB > 0) {
            // digit width known at compile time: accumulate the lanes that
            // differ in validity or in any digit bit, one ballot per bit
            const uint32_t sok = ok ? ~0u : 0u;
            uint32_t x = __ballot_sync(0xffffffffu, ok) ^ sok;
#pragma unroll
            for (int bit = 0; bit < DB; bit++) {
                const uint32_t sb = (uint32_t)((int32_t)(d << (31 - bit)) >> 31);
                x |= __ballot_sync(0xffffffffu, sb != 0u) ^ sb;
            }
            peers = ~x;
        } else {
            peers = __ballot_sync(0xffffffffu, ok);
            if (!ok) peers = ~peers;
            for (uint32_t bit = 0; (1u << bit) < nb; bit++) {
                const unsigned m = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
                peers &= ((d >> bit) & 1u) ? m : ~m;
            }
        }
        uint32_t b = ok ? wcnt[warp * RS_MAXB + d] : 0;
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) wcnt[warp * RS_MAXB + d] = (uint16_t)(b + __popc(peers));
        __syncwarp();
        rank[r] = (uint16_t)(b + __popc(peers & lt));
    }
    __syncthreads();
    {
        // thread t owns digits 2t and 2t + 1, whose per-warp counters share one
        // 32-bit word (counts stay below 2^16, so the halves add without carry):
        // tile totals, an exclusive scan of them in digit order, then every
        // (warp, digit) counter becomes that warp's first tile position
        uint32_t *wc32 = reinterpret_cast<uint32_t *>(wcnt);
        uint32_t acc = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) acc += wc32[w * (RS_MAXB / 2) + threadIdx.x];
        const uint32_t t0 = acc & 0xffffu, t1 = acc >> 16;
        const uint32_t pair = t0 + t1;
        uint32_t incl = pair;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        uint32_t wpre = 0;
        for (int w = 0; w < warp; w++) wpre += s_w[w];
        const uint32_t st0 = wpre + incl - pair, st1 = st0 + t0;
        uint32_t run = st0 | (st1 << 16);
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) {
            const uint32_t c = wc32[w * (RS_MAXB / 2) + threadIdx.x];
            wc32[w * (RS_MAXB / 2) + threadIdx.x] = run;
            run += c;
        }
        const uint32_t d0 = 2 * threadIdx.x;
        if (d0 < nb) gdelta[d0] = offs[(uint64_t)d0 * ntiles + blockIdx.x] - st0;
        if (d0 + 1 < nb) gdelta[d0 + 1] = offs[(uint64_t)(d0 + 1) * ntiles + blockIdx.x] - st1;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_I; r++) {
        uint64_t i = base + (uint64_t)warp * (RS_I * 32) + r * 32 + lane;
        if (i < n) {
            uint32_t d = (uint32_t)(key[r] >> shift) & (nb - 1);
            uint32_t pos = (uint32_t)wcnt[warp * RS_MAXB + d] + rank[r];
            skeys[pos] = key[r];
            if (VALS) svals[pos] = val[r];
        }
    }
    __syncthreads();
    const uint32_t cnt = (uint32_t)((n - base) < (uint64_t)RS_TILE ? (n - base) : RS_TILE);
#pragma unroll
    for (int r = 0; r < RS_I; r++) {
        const uint32_t k = r * RS_T + threadIdx.x;
        if (k < cnt) {
            const uint64_t kk = skeys[k];
            const uint32_t g = gdelta[(uint32_t)(kk >> shift) & (nb - 1)] + k;
            __stcs(kout + g, kk);
            if (VALS) __stcs(vout + g, svals[k]);
        }
    }
}

template <bool VALS>
static constexpr size_t rs_smem()
{
    return RS_TILE * 8 + (VALS ? RS_TILE * 4 : 0) + RS_MAXB * 4 + RS_WARPS * RS_MAXB * 2;
}

// the scatter specialised for the common digit widths (36-bit fingerprints:
// 9 bits; 40-bit group keys: 8 bits), else the generic loop
template <bool VALS>
static void launch_scatter(uint32_t db, uint64_t ntiles, const uint64_t *ks, uint64_t *kd, const uint32_t *vs,
                           uint32_t *vd, uint64_t n, uint32_t shift, uint32_t nb, const uint32_t *offs,
                           cudaStream_t st, bool stable)
{
    const unsigned g = (unsigned)ntiles;
    const size_t sm = rs_smem<VALS>();
    if (!VALS && !stable) {
        rs_scatter<false, 0, false><<<g, RS_T, sm, st>>>(ks, kd, vs, vd, n, shift, nb, offs, ntiles);
        return;
    }
    if (db == 9) rs_scatter<VALS, 9><<<g, RS_T, sm, st>>>(ks, kd, vs, vd, n, shift, nb, offs, ntiles);
    else if (db == 8) rs_scatter<VALS, 8><<<g, RS_T, sm, st>>>(ks, kd, vs, vd, n, shift, nb, offs, ntiles);
    else rs_scatter<VALS, 0><<<g, RS_T, sm, st>>>(ks, kd, vs, vd, n, shift, nb, offs, ntiles);
}

static uint32_t first_digit_bits(uint32_t bits)
{
    const uint32_t npass = (bits + 8) / 9;
    return npass ? bits / npass + (bits % npass ? 1u : 0u) : 0u;
}

void fingerprint_for_sort(const uint64_t *keys, uint64_t n, const PHash &H, uint64_t *fp, uint32_t *idx,
                          uint32_t bits, uint32_t *tmp, cudaStream_t st)
{
    if (n == 0) return;
    const uint32_t db = first_digit_bits(bits);
    const uint64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    TraceScope ts_("rs_fp_hist", n, st);
    rs_fp_hist<<<(unsigned)ntiles, RS_T, 0, st>>>(keys, n, H, fp, idx, 1u << db, tmp, ntiles);
}

void radix_sort_u64(const uint64_t *keys_in, uint64_t *keys_out, uint64_t *keys_alt,
                    const uint32_t *vals_in, uint32_t *vals_out, uint32_t *vals_alt, uint64_t n,
                    uint32_t bits, uint32_t *tmp, uint64_t *scan_tmp, DevCounters *ctr,
                    cudaStream_t st, bool first_hist_done)
{
    if (n == 0) return;
    static bool attr_done = false;
    if (!attr_done) {
        cudaFuncSetAttribute(rs_scatter<true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs_smem<true>());
        cudaFuncSetAttribute(rs_scatter<false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs_smem<false>());
        cudaFuncSetAttribute(rs_scatter<true, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs_smem<true>());
        cudaFuncSetAttribute(rs_scatter<false, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs_smem<false>());
        cudaFuncSetAttribute(rs_scatter<true, 9>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs_smem<true>());
        cudaFuncSetAttribute(rs_scatter<false, 9>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs_smem<false>());
        cudaFuncSetAttribute(rs_scatter<false, 0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)rs_smem<false>());
        attr_done = true;
    }
    const bool vals = vals_in != nullptr;
    const uint32_t npass = (bits + 8) / 9;  // digits of at most 9 bits
    if (npass == 0) {
        cudaMemcpyAsync(keys_out, keys_in, n * 8, cudaMemcpyDeviceToDevice, st);
        if (vals) cudaMemcpyAsync(vals_out, vals_in, n * 4, cudaMemcpyDeviceToDevice, st);
        return;
    }
    const uint64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    const uint64_t *ksrc = keys_in;
    const uint32_t *vsrc = vals_in;
    uint32_t shift = 0;
    for (uint32_t p = 0; p < npass; p++) {
        // split the bits as evenly as possible: the first passes take the extra bit
        const uint32_t db = bits / npass + (p < bits % npass ? 1u : 0u);
        const uint32_t nb = 1u << db;
        bool to_out = ((npass - 1 - p) % 2) == 0;
        uint64_t *kdst = to_out ? keys_out : keys_alt;
        uint32_t *vdst = to_out ? vals_out : vals_alt;
        if (p > 0 || !first_hist_done) {
            TraceScope ts_("rs_hist", n, st);
            rs_hist<<<(unsigned)ntiles, RS_T, 0, st>>>(ksrc, n, shift, nb, tmp, ntiles);
        }
        exclusive_scan_u32(tmp, tmp, ntiles * nb, scan_tmp, ctr, st);
        TraceScope ts_(vals ? "rs_scatter_kv" : "rs_scatter", n, st);
        if (vals)
            launch_scatter<true>(db, ntiles, ksrc, kdst, vsrc, vdst, n, shift, nb, tmp, st, true);
        else
            launch_scatter<false>(db, ntiles, ksrc, kdst, nullptr, nullptr, n, shift, nb, tmp, st, p > 0);
        ksrc = kdst;
        vsrc = vdst;
        shift += db;
    }
}

// ---------------------------------------------------------------------------
// Random-access calibration: the memory pattern of a filter query (a key
// read, `spk` random 32-byte sectors of a table, one result byte) without
// any filter arithmetic. Its throughput is the random-gather roofline at a
// given table footprint.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) gather32_kernel(const uint4 *__restrict__ table, uint64_t nsect,
                                                       const uint64_t *__restrict__ keys, uint64_t n, uint32_t spk,
                                                       uint8_t *__restrict__ out)
{
    for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i < n; i += (uint64_t)gridDim.x * 256) {
        uint64_t h = mix64(__ldg(keys + i));
        uint32_t acc = 0;
        for (uint32_t k = 0; k < spk; k++) {
            const uint64_t sct = (h & 0xffffffffull) * nsect >> 32;  // sector index in [0, nsect)
            const uint4 a = __ldg(table + 2 * sct), b = __ldg(table + 2 * sct + 1);
            acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w;
            h = mix64(h + k + 1);
        }
        out[i] = (uint8_t)acc;
    }
}

// ---------------------------------------------------------------------------
// Kernel tracing
// ---------------------------------------------------------------------------
bool g_trace_on = false;

struct TraceRec {
    const char *name;
    uint64_t units;
    cudaEvent_t a, b;
    int dev_slot;  // >= 0: the units are the device counter g_units_dev[dev_slot]
};
static std::vector<TraceRec> g_trace;
static std::vector<cudaEvent_t> g_event_pool;
static std::mutex g_trace_mu;
static constexpr int TRACE_DEV_SLOTS = 1 << 16;
static unsigned long long *g_units_dev = nullptr;  // zeroed on enable and reset
static int g_units_used = 0;

static cudaEvent_t pool_event()
{
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

int trace_open(const char *name, uint64_t units, cudaStream_t st, bool dev_units)
{
    std::lock_guard<std::mutex> g(g_trace_mu);
    if (g_trace.size() >= (1u << 20)) return -1;
    TraceRec r{name, units, pool_event(), pool_event(), -1};
    if (dev_units && g_units_dev && g_units_used < TRACE_DEV_SLOTS) r.dev_slot = g_units_used++;
    cudaEventRecord(r.a, st);
    g_trace.push_back(r);
    return (int)g_trace.size() - 1;
}

unsigned long long *trace_units(int slot)
{
    std::lock_guard<std::mutex> g(g_trace_mu);
    if (slot < 0 || slot >= (int)g_trace.size() || g_trace[slot].dev_slot < 0) return nullptr;
    return g_units_dev + g_trace[slot].dev_slot;
}

void trace_close(int slot, cudaStream_t st)
{
    std::lock_guard<std::mutex> g(g_trace_mu);
    if (slot >= 0 && slot < (int)g_trace.size()) cudaEventRecord(g_trace[slot].b, st);
}

static void trace_clear_locked()
{
    for (auto &r : g_trace) {
        g_event_pool.push_back(r.a);
        g_event_pool.push_back(r.b);
    }
    g_trace.clear();
    if (g_units_dev && g_units_used) cudaMemset(g_units_dev, 0, sizeof(unsigned long long) * g_units_used);
    g_units_used = 0;
}

static char g_last_err[256];

void set_last_cuda_error(cudaError_t e, const char *what, int line)
{
    snprintf(g_last_err, sizeof(g_last_err), "%s (line %d): %s", what, line, cudaGetErrorString(e));
}

const char *last_cuda_error() { return g_last_err[0] ? g_last_err : "CUDA runtime error"; }

}  // namespace gf

extern "C" {

int filter_trace_enable(int on)
{
    if (on) {
        std::lock_guard<std::mutex> g(gf::g_trace_mu);
        if (!gf::g_units_dev) {
            void *p = nullptr;
            if (gf::dev_malloc(&p, sizeof(unsigned long long) * gf::TRACE_DEV_SLOTS) != cudaSuccess) {
                cudaGetLastError();
                return FILTER_ERR_OOM;
            }
            if (cudaMemset(p, 0, sizeof(unsigned long long) * gf::TRACE_DEV_SLOTS) != cudaSuccess) {
                gf::dev_free(p);
                return FILTER_ERR_CUDA;
            }
            gf::g_units_dev = static_cast<unsigned long long *>(p);
            gf::g_units_used = 0;
        }
    }
    gf::g_trace_on = on != 0;
    return FILTER_OK;
}

int filter_trace_reset(void)
{
    std::lock_guard<std::mutex> g(gf::g_trace_mu);
    for (auto &r : gf::g_trace) cudaEventSynchronize(r.b);
    gf::trace_clear_locked();
    return FILTER_OK;
}

int filter_trace_summary(uint32_t cap, filter_trace_entry *out, uint32_t *n_kernels)
{
    std::lock_guard<std::mutex> g(gf::g_trace_mu);
    std::vector<filter_trace_entry> acc;
    std::vector<unsigned long long> dev_units(gf::g_units_used);
    for (auto &r : gf::g_trace)
        if (cudaEventSynchronize(r.b) != cudaSuccess) return FILTER_ERR_CUDA;
    if (gf::g_units_used &&
        cudaMemcpy(dev_units.data(), gf::g_units_dev, sizeof(unsigned long long) * gf::g_units_used,
                   cudaMemcpyDeviceToHost) != cudaSuccess)
        return FILTER_ERR_CUDA;
    for (auto &r : gf::g_trace) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return FILTER_ERR_CUDA;
        filter_trace_entry *e = nullptr;
        for (auto &x : acc)
            if (std::strncmp(x.name, r.name, sizeof(x.name)) == 0) e = &x;
        if (!e) {
            filter_trace_entry z;
            std::memset(&z, 0, sizeof(z));
            std::strncpy(z.name, r.name, sizeof(z.name) - 1);
            acc.push_back(z);
            e = &acc.back();
        }
        e->launches++;
        e->units += r.dev_slot >= 0 ? dev_units[r.dev_slot] : r.units;
        e->ms += ms;
    }
    if (n_kernels) *n_kernels = (uint32_t)acc.size();
    for (uint32_t i = 0; i < cap && i < acc.size(); i++) out[i] = acc[i];
    return FILTER_OK;
}

}  // extern "C"

namespace gf {

}  // namespace gf

extern "C" int filter_calibrate_gather(const void *d_table, uint64_t table_bytes, const uint64_t *d_keys, uint64_t n,
                                       uint32_t sectors_per_key, uint8_t *d_out, void *stream)
{
    const uint64_t nsect = table_bytes / 32;
    if (!d_table || nsect == 0 || nsect > 0xffffffffull || (n && (!d_keys || !d_out)) ||
        (reinterpret_cast<uintptr_t>(d_table) & 15u))
        return FILTER_ERR_ARG;
    if (n == 0) return FILTER_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    {
        gf::TraceScope ts_("gather32_kernel", n, st);
        gf::gather32_kernel<<<gf::grid_for(n, 256, 16), 256, 0, st>>>(static_cast<const uint4 *>(d_table), nsect, d_keys,
                                                                      n, sectors_per_key, d_out);
    }
    GF_CUDA(cudaGetLastError());
    return FILTER_OK;
}

