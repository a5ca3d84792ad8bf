// Two-choice filter (TCF), paper Sec. 4, for sm_103a.
//
// Table: nb blocks of 32 bytes (one DRAM sector), B = 256 / f tags each, plus a
// backing table of nbk buckets of 8 uint64 entries (Sec. 4.1, "Backing table").
//
// Query (Sec. 4): probe both candidate blocks with two 16-byte loads each and a
// SIMD compare (__vcmpeq2 / __vcmpeq4), then the backing bucket (L2-resident)
// if the tag was in neither block.
//
// Bulk insert, deterministic mode (Sec. 4.1 shortcut + Sec. 4 two choices +
// Sec. 4.1 backing table + Sec. 4.2 sorted blocks). Each block phase groups
// its candidates by tile of consecutive blocks (one or two coalesced counting
// passes), then one CTA per tile sorts them by block in shared memory and one
// thread per block takes the k smallest (tag, batch index) candidates that
// fit, merges them into its sorted block, and emits the rest to the next
// phase:
//   A shortcut into b1 while fill + j < 3B/4, B the less-full block under the
//   post-A fills, C the other block, D the backing bucket (few candidates:
//   a counting sort over the touched buckets only).
// Blocks keep a fill byte array beside them so that the two-choice decision
// reads 1 byte from L2 instead of a 32-byte sector from HBM.
//
// Point mode (Alg. 1): one thread per key; the tag goes into the first EMPTY
// or TOMBSTONE slot by an atomic compare-and-swap, retried a bounded number of
// times; deletes swap the tag for TOMBSTONE.
//
// Values (Sec. 1 and Sec. 4: small values stored with the items): with v
// value bits a slot holds the (f - v)-bit tag above the value. The phases
// carry whole slots; g and the bucket use the tag alone; matching masks the
// value bits; a value query answers the smallest value stored with the key's
// fingerprint in its blocks and backing bucket.
#include <type_traits>
#include <vector>

#include "gf_internal.cuh"
#include "gf_packed.cuh"

namespace gf {

static constexpr int TPB = 256;
static constexpr uint32_t BK_W = 8;  // backing bucket entries
static constexpr int MAXSEL = 32;    // largest B

// ---------------------------------------------------------------------------
// 32-byte block in registers
// ---------------------------------------------------------------------------
template <int F>
struct Blk {
    static constexpr int B = 256 / F;
    uint32_t w[8];

    __device__ __forceinline__ void load(const uint8_t *blocks, uint64_t b)
    {
        const uint4 *p = reinterpret_cast<const uint4 *>(blocks + b * 32);
        uint4 lo = p[0], hi = p[1];
        w[0] = lo.x; w[1] = lo.y; w[2] = lo.z; w[3] = lo.w;
        w[4] = hi.x; w[5] = hi.y; w[6] = hi.z; w[7] = hi.w;
    }
    __device__ __forceinline__ void load_ro(const uint8_t *blocks, uint64_t b)
    {
        const uint4 *p = reinterpret_cast<const uint4 *>(blocks + b * 32);
        uint4 lo = __ldg(p), hi = __ldg(p + 1);
        w[0] = lo.x; w[1] = lo.y; w[2] = lo.z; w[3] = lo.w;
        w[4] = hi.x; w[5] = hi.y; w[6] = hi.z; w[7] = hi.w;
    }
    __device__ __forceinline__ void load_l2(const uint8_t *blocks, uint64_t b)
    {
        const uint4 *p = reinterpret_cast<const uint4 *>(blocks + b * 32);
        uint4 lo = __ldcg(p), hi = __ldcg(p + 1);
        w[0] = lo.x; w[1] = lo.y; w[2] = lo.z; w[3] = lo.w;
        w[4] = hi.x; w[5] = hi.y; w[6] = hi.z; w[7] = hi.w;
    }
    __device__ __forceinline__ void store(uint8_t *blocks, uint64_t b) const
    {
        uint4 *p = reinterpret_cast<uint4 *>(blocks + b * 32);
        p[0] = make_uint4(w[0], w[1], w[2], w[3]);
        p[1] = make_uint4(w[4], w[5], w[6], w[7]);
    }
    __device__ __forceinline__ uint32_t tag(int s) const
    {
        if (F == 16) return (w[s >> 1] >> ((s & 1) * 16)) & 0xffffu;
        return (w[s >> 2] >> ((s & 3) * 8)) & 0xffu;
    }
    // the tag part of every lane of a word (all ones without values)
    static __device__ __forceinline__ uint32_t lane_mask(uint32_t vmask)
    {
        return F == 16 ? (0xffffu & ~vmask) * 0x00010001u : (0xffu & ~vmask) * 0x01010101u;
    }
    // some slot holds tag t (t: the slot with value 0; lm from lane_mask)
    __device__ __forceinline__ bool has(uint32_t t, uint32_t lm) const
    {
        uint32_t m = 0;
        if (F == 16) {
            uint32_t tt = t | (t << 16);
#pragma unroll
            for (int k = 0; k < 8; k++) m |= __vcmpeq2(w[k] & lm, tt);
        } else {
            uint32_t tt = t * 0x01010101u;
#pragma unroll
            for (int k = 0; k < 8; k++) m |= __vcmpeq4(w[k] & lm, tt);
        }
        return m != 0;
    }
    // smallest value stored with tag t, or the lane maximum when none is
    __device__ __forceinline__ uint32_t min_value(uint32_t t, uint32_t lm) const
    {
        uint32_t b = 0xffffffffu;
        if (F == 16) {
            const uint32_t tt = t | (t << 16);
#pragma unroll
            for (int k = 0; k < 8; k++) b = __vminu2(b, (w[k] & ~lm) | ~__vcmpeq2(w[k] & lm, tt));
            return min(b & 0xffffu, b >> 16);
        } else {
            const uint32_t tt = t * 0x01010101u;
#pragma unroll
            for (int k = 0; k < 8; k++) b = __vminu4(b, (w[k] & ~lm) | ~__vcmpeq4(w[k] & lm, tt));
            b = __vminu4(b, b >> 16);
            return min(b & 0xffu, (b >> 8) & 0xffu);
        }
    }
    // tags >= 2 (neither EMPTY nor TOMBSTONE)
    __device__ __forceinline__ int live() const
    {
        int c = 0;
        if (F == 16) {
#pragma unroll
            for (int k = 0; k < 8; k++) c += __popc(__vcmpgeu2(w[k], 0x00020002u));
            return c >> 4;
        } else {
#pragma unroll
            for (int k = 0; k < 8; k++) c += __popc(__vcmpgeu4(w[k], 0x02020202u));
            return c >> 3;
        }
    }
    __device__ __forceinline__ int nonzero() const
    {
        int c = 0;
        if (F == 16) {
#pragma unroll
            for (int k = 0; k < 8; k++) c += __popc(__vcmpne2(w[k], 0u));
            return c >> 4;
        } else {
#pragma unroll
            for (int k = 0; k < 8; k++) c += __popc(__vcmpne4(w[k], 0u));
            return c >> 3;
        }
    }
    // bit s set where slot s holds tag t
    __device__ __forceinline__ uint32_t eq_slots(uint32_t t, uint32_t lm) const
    {
        uint32_t sm = 0;
        if (F == 16) {
            const uint32_t tt = t | (t << 16);
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const uint32_t m = __vcmpeq2(w[k] & lm, tt);
                sm |= ((m & 1u) | ((m >> 15) & 2u)) << (2 * k);
            }
        } else {
            const uint32_t tt = t * 0x01010101u;
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const uint32_t m = __vcmpeq4(w[k] & lm, tt);
                sm |= ((m & 1u) | ((m >> 7) & 2u) | ((m >> 14) & 4u) | ((m >> 21) & 8u)) << (4 * k);
            }
        }
        return sm;
    }
    // bits of word k below bit position bp of the 256-bit block
    static __device__ __forceinline__ uint32_t low_bits(int k, int bp)
    {
        const int lo = bp - 32 * k;
        return lo >= 32 ? 0xffffffffu : (lo <= 0 ? 0u : ((1u << lo) - 1u));
    }
    // slot pos is removed: slots above it move down by one, the last becomes EMPTY
    __device__ __forceinline__ void delete_at(int pos)
    {
        const int bp = pos * F;
        uint32_t nw[8];
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const uint32_t sh = k < 7 ? __funnelshift_r(w[k], w[k + 1], F) : (w[7] >> F);
            const uint32_t lo = low_bits(k, bp);
            nw[k] = (w[k] & lo) | (sh & ~lo);
        }
#pragma unroll
        for (int k = 0; k < 8; k++) w[k] = nw[k];
    }
    // Merge k new tags (the high words of r[0 .. k), ascending) into the f0
    // sorted tags of the block (f0 + k <= B, k <= 8) with a bitonic merge on
    // packed lanes: empty lanes become the largest tag value, the new tags go
    // descending into the top lanes, and log2(B) half-cleaner stages of SIMD
    // min / max sort the lanes ascending; lanes from f0 + k on are cleared.
    // Equal tags are indistinguishable, so the result equals the stable merge.
    __device__ __forceinline__ void merge_new(uint32_t f0, uint32_t k, const uint64_t (&r)[8])
    {
#pragma unroll
        for (int q = 0; q < 8; q++) w[q] |= ~low_bits(q, (int)(f0 * F));
#pragma unroll
        for (int m = 0; m < 8; m++) {
            if (m < (int)k) {
                constexpr int LPW = 32 / F;  // lanes per word
                const int L = B - 1 - m;
                const int sh = (L % LPW) * F;
                const uint32_t lane_mask = (F == 16 ? 0xffffu : 0xffu) << sh;
                w[L / LPW] = (w[L / LPW] & ~lane_mask) | ((uint32_t)(r[m] >> 32) << sh);
            }
        }
        // word-level half-cleaners: distances of 4, 2 and 1 words
#pragma unroll
        for (int dw = 4; dw >= 1; dw >>= 1) {
#pragma unroll
            for (int q = 0; q < 8; q++) {
                if ((q & dw) == 0) {
                    const uint32_t a = w[q], c = w[q + dw];
                    w[q] = F == 16 ? __vminu2(a, c) : __vminu4(a, c);
                    w[q + dw] = F == 16 ? __vmaxu2(a, c) : __vmaxu4(a, c);
                }
            }
        }
        // lane-level half-cleaners inside each word
#pragma unroll
        for (int q = 0; q < 8; q++) {
            uint32_t x = w[q];
            if (F == 8) {  // lanes two apart: swap the 16-bit halves
                const uint32_t y = __byte_perm(x, 0u, 0x1032u);
                x = __byte_perm(__vminu4(x, y), __vmaxu4(x, y), 0x7610u);
            }
            if (F == 16) {  // lanes one apart: the two halves
                const uint32_t y = __byte_perm(x, 0u, 0x1032u);
                x = __byte_perm(__vminu2(x, y), __vmaxu2(x, y), 0x7610u);
            } else {        // lanes one apart: bytes 0/1 and 2/3
                const uint32_t y = __byte_perm(x, 0u, 0x2301u);
                x = __byte_perm(__vminu4(x, y), __vmaxu4(x, y), 0x7250u);
            }
            w[q] = x;
        }
#pragma unroll
        for (int q = 0; q < 8; q++) w[q] &= low_bits(q, (int)((f0 + k) * F));
    }
    // pack B tags (ascending, zero padded) from an array
    __device__ __forceinline__ void pack(const uint32_t *t)
    {
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if (F == 16) w[k] = (t[2 * k] & 0xffffu) | (t[2 * k + 1] << 16);
            else w[k] = (t[4 * k] & 0xffu) | ((t[4 * k + 1] & 0xffu) << 8) | ((t[4 * k + 2] & 0xffu) << 16) |
                        (t[4 * k + 3] << 24);
        }
    }
};

// sort up to 8 records held in registers (absent ones are ~0 and sort last):
// a 19-comparator network of depth 6, or 5 comparators for the first 4
// when no lane of the warp has more; callers index the array only in
// unrolled loops, which keeps it in registers
__device__ __forceinline__ void cswap(uint64_t &a, uint64_t &b)
{
    const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
    a = lo;
    b = hi;
}
__device__ __forceinline__ void sort4(uint64_t (&r)[8])
{
    cswap(r[0], r[1]); cswap(r[2], r[3]);
    cswap(r[0], r[2]); cswap(r[1], r[3]);
    cswap(r[1], r[2]);
}
__device__ __forceinline__ void sort8(uint64_t (&r)[8])
{
    cswap(r[0], r[2]); cswap(r[1], r[3]); cswap(r[4], r[6]); cswap(r[5], r[7]);
    cswap(r[0], r[4]); cswap(r[1], r[5]); cswap(r[2], r[6]); cswap(r[3], r[7]);
    cswap(r[0], r[1]); cswap(r[2], r[3]); cswap(r[4], r[5]); cswap(r[6], r[7]);
    cswap(r[2], r[4]); cswap(r[3], r[5]);
    cswap(r[1], r[4]); cswap(r[3], r[6]);
    cswap(r[1], r[2]); cswap(r[3], r[4]); cswap(r[5], r[6]);
}
__device__ __forceinline__ void sort_small(uint64_t (&r)[8], uint32_t cnt)
{
    const uint32_t wmax = __reduce_max_sync(__activemask(), cnt);
    if (wmax > 4) sort8(r);
    else if (wmax > 1) sort4(r);
}

// keep the `have` smallest values seen so far in a[0..have), ascending, at most k
__device__ __forceinline__ int topk_push(uint64_t *a, int have, int k, uint64_t v)
{
    if (have == k) {
        if (k == 0 || v >= a[k - 1]) return have;
        have--;
    }
    int j = have;
    while (j > 0 && a[j - 1] > v) {
        a[j] = a[j - 1];
        j--;
    }
    a[j] = v;
    return have + 1;
}

// ---------------------------------------------------------------------------
// Query (both modes)
// ---------------------------------------------------------------------------
// VAL: answer the smallest value stored with the key's fingerprint in its two
// blocks and its backing bucket, 0xFF when there is none; else 1 / 0.
template <int F, bool VAL>
__global__ void __launch_bounds__(TPB) tcf_query_kernel(const uint64_t *__restrict__ keys, uint64_t n,
                                                        TcfGeom G, const uint8_t *__restrict__ blocks,
                                                        const uint64_t *__restrict__ bk,
                                                        const DevCounters *ctr,
                                                        uint8_t *__restrict__ out)
{
    const bool backing = ctr->backing != 0;
    const uint32_t lm = Blk<F>::lane_mask(G.vmask);
    const uint64_t em = ~(uint64_t)G.vmask;
    for (uint64_t i = blockIdx.x * (uint64_t)TPB + threadIdx.x; i < n; i += (uint64_t)gridDim.x * TPB) {
        KeyInfo k = tcf_keyinfo(__ldcs(keys + i), G);  // keys and answers stream past the L2
        Blk<F> x, y;
        x.load_ro(blocks, k.b1);
        y.load_ro(blocks, k.b2);
        if (VAL) {
            uint32_t best = min(x.min_value(k.t, lm), y.min_value(k.t, lm));
            if (backing) {
                const uint64_t e = tcf_entry(k, G.f);
                const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(bk + tcf_bucket_of(e, G) * BK_W);
#pragma unroll
                for (int s = 0; s < 4; s++) {
                    const ulonglong2 v = __ldg(p + s);
                    if ((v.x & em) == e) best = min(best, (uint32_t)v.x & G.vmask);
                    if ((v.y & em) == e) best = min(best, (uint32_t)v.y & G.vmask);
                }
            }
            __stcs(out + i, (uint8_t)(best <= G.vmask ? best : 0xffu));
            continue;
        }
        bool hit = x.has(k.t, lm) || y.has(k.t, lm);
        if (!hit && backing) {
            uint64_t e = tcf_entry(k, G.f);
            const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(bk + tcf_bucket_of(e, G) * BK_W);
#pragma unroll
            for (int s = 0; s < 4; s++) {
                ulonglong2 v = __ldg(p + s);
                hit |= ((v.x & em) == e) | ((v.y & em) == e);
            }
        }
        __stcs(out + i, (uint8_t)(hit ? 1 : 0));
    }
}

// ---------------------------------------------------------------------------
// Counting-sort grouping kernels
// ---------------------------------------------------------------------------
// source of a phase's candidate list
enum Src : int { SRC_KEYS = 0, SRC_PEND_U32 = 1, SRC_PEND_U64 = 2 };
// how a candidate picks its destination
enum Dst : int { DST_B1 = 0, DST_TARGET = 1, DST_ALT = 2, DST_B2 = 3, DST_BUCKET = 4 };

// Key i of the call: hashed here, or (group calls) read from the prepared
// keys, whose block indices already address the group's concatenated arrays;
// b2 is read only by the destinations that need it.
template <int DST>
__device__ __forceinline__ KeyInfo key_at(const uint64_t *keys, const TcfPrep &P, uint64_t i, const TcfGeom &G)
{
    if (P.bt) {
        const uint64_t v = P.bt[i];
        KeyInfo k;
        k.b1 = v >> 32;
        k.t = (uint32_t)v;
        k.b2 = (DST == DST_TARGET || DST == DST_B2) ? P.b2[i] : 0;
        return k;
    }
    KeyInfo k = tcf_keyinfo(keys[i], G);
    if (P.vals) k.t |= P.vals[i] & G.vmask;
    return k;
}

__device__ __forceinline__ uint64_t dest_of(int dst, const KeyInfo &k, uint64_t pend_word, const TcfGeom &G,
                                            const uint8_t *fill, const TcfPrep &P, uint64_t i)
{
    switch (dst) {
    case DST_B1: return k.b1;
    case DST_B2: return k.b2;
    case DST_TARGET: return fill[k.b1] <= fill[k.b2] ? k.b1 : k.b2;
    case DST_ALT: return pend_word >> 32;
    default: return P.bt ? (uint64_t)P.bucket[i] : tcf_bucket_of(tcf_entry(k, G.f), G);
    }
}

// Traced launches whose work is only known on the device record it here
// (units is null when tracing is off)
__device__ __forceinline__ void note_units(unsigned long long *units, uint64_t v)
{
    if (units && blockIdx.x == 0 && threadIdx.x == 0) *units = v;
}

// A CTA's share of a sparse phase's candidates: one contiguous, warp-aligned
// chunk (the touched destinations it finds are listed from the chunk's start)
__device__ __forceinline__ void cta_chunk(uint64_t n, uint64_t &c0, uint64_t &c1)
{
    const uint64_t per = (((n + gridDim.x - 1) / gridDim.x) + 31) & ~31ull;
    c0 = per * blockIdx.x;
    if (c0 > n) c0 = n;
    c1 = c0 + per < n ? c0 + per : n;
}

// Dense phases count every candidate per destination; sparse phases (few
// candidates, as in the later phases) also list each destination the first
// time it is hit, per CTA chunk, in tlist[c0 ..] with the count in tcount.
template <int SRC, int DST, bool SPARSE>
__global__ void __launch_bounds__(TPB) tcf_group_hist(const uint64_t *__restrict__ keys, const TcfPrep prep,
                                                      uint64_t n_keys, const void *pend, const unsigned *npend,
                                                      TcfGeom G, const uint8_t *fill, uint32_t *cnt,
                                                      uint32_t *tlist, uint32_t *tcount, unsigned long long *units)
{
    const uint64_t n = (SRC == SRC_KEYS) ? n_keys : (uint64_t)*npend;
    note_units(units, n);
    __shared__ unsigned s_n;
    uint64_t c0 = 0, c1 = n, step = (uint64_t)gridDim.x * TPB, j = blockIdx.x * (uint64_t)TPB + threadIdx.x;
    if (SPARSE) {
        if (threadIdx.x == 0) s_n = 0;
        __syncthreads();
        cta_chunk(n, c0, c1);
        step = TPB;
        j = c0 + threadIdx.x;
    }
    for (; j < c1; j += step) {
        uint64_t pw = 0, i = j;
        if (SRC == SRC_PEND_U32) i = static_cast<const uint32_t *>(pend)[j];
        if (SRC == SRC_PEND_U64) {
            pw = static_cast<const uint64_t *>(pend)[j];
            i = pw & 0xffffffffu;
        }
        KeyInfo k = key_at<DST>(keys, prep, i, G);
        const uint64_t d = dest_of(DST, k, pw, G, fill, prep, i);
        if (SPARSE) {
            if (atomicAdd(&cnt[d], 1u) == 0u) tlist[c0 + atomicAdd(&s_n, 1u)] = (uint32_t)d;
        } else {
            atomicAdd(&cnt[d], 1u);  // no result used: a reduction the L2 applies without a reply
        }
    }
    if (SPARSE) {
        __syncthreads();
        if (threadIdx.x == 0) tcount[blockIdx.x] = s_n;
    }
}

// Sparse phases: every touched destination gets a contiguous segment of the
// record array (CTA-wide scan of the counts, one atomic per 256 destinations)
// and an entry in the dense touched list. Same grid as the histogram.
__global__ void __launch_bounds__(TPB) tcf_alloc(const unsigned *npend, uint64_t n_keys,
                                                 const uint32_t *__restrict__ tlist,
                                                 const uint32_t *__restrict__ tcount, const uint32_t *cnt,
                                                 uint32_t *off, uint32_t *dlist, uint64_t *seg, unsigned *cursor,
                                                 unsigned *nlist, unsigned long long *units)
{
    __shared__ uint32_t s_w[TPB / 32];
    __shared__ uint32_t s_base, s_lbase;
    const uint64_t n = npend ? (uint64_t)*npend : n_keys;
    uint64_t c0, c1;
    cta_chunk(n, c0, c1);
    const uint32_t m = tcount[blockIdx.x];
    if (units && threadIdx.x == 0 && m) atomicAdd(units, (unsigned long long)m);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t j0 = 0; j0 < m; j0 += TPB) {
        const uint32_t j = j0 + threadIdx.x;
        const uint32_t d = j < m ? tlist[c0 + j] : 0u;
        const uint32_t c = j < m ? cnt[d] : 0u;
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        uint32_t pre = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < TPB / 32; w++) {
            if (w < warp) pre += s_w[w];
            tot += s_w[w];
        }
        if (threadIdx.x == 0) {
            s_base = atomicAdd(cursor, tot);
            s_lbase = atomicAdd(nlist, m - j0 < (uint32_t)TPB ? m - j0 : (uint32_t)TPB);
        }
        __syncthreads();
        if (j < m) {
            const uint32_t start = s_base + pre + incl - c;
            off[d] = start;
            dlist[s_lbase + threadIdx.x] = d;
            seg[s_lbase + threadIdx.x] = ((uint64_t)start << 32) | c;
        }
        __syncthreads();
    }
}

// rec = (tag << 32) | batch index, or the backing entry with the index in recI
template <int SRC, int DST>
__global__ void __launch_bounds__(TPB) tcf_group_scatter(const uint64_t *__restrict__ keys, const TcfPrep prep,
                                                         uint64_t n_keys, const void *pend, const unsigned *npend,
                                                         TcfGeom G,
                                                         const uint8_t *fill, uint32_t *cnt,
                                                         const uint32_t *__restrict__ off, uint64_t *rec,
                                                         uint32_t *recI, unsigned long long *units)
{
    const uint64_t n = (SRC == SRC_KEYS) ? n_keys : (uint64_t)*npend;
    note_units(units, n);
    for (uint64_t j = blockIdx.x * (uint64_t)TPB + threadIdx.x; j < n; j += (uint64_t)gridDim.x * TPB) {
        uint64_t pw = 0, i = j;
        if (SRC == SRC_PEND_U32) i = static_cast<const uint32_t *>(pend)[j];
        if (SRC == SRC_PEND_U64) {
            pw = static_cast<const uint64_t *>(pend)[j];
            i = pw & 0xffffffffu;
        }
        KeyInfo k = key_at<DST>(keys, prep, i, G);
        uint64_t d = dest_of(DST, k, pw, G, fill, prep, i);
        uint32_t pos = off[d] + atomicSub(&cnt[d], 1u) - 1u;
        if (DST == DST_BUCKET) {
            rec[pos] = prep.bt ? prep.e[i] : tcf_entry(k, G.f);
            recI[pos] = (uint32_t)i;
        } else {
            rec[pos] = ((uint64_t)k.t << 32) | i;
        }
    }
}

// ---------------------------------------------------------------------------
// Bulk insert: per-block acceptance
// ---------------------------------------------------------------------------
// phase 0 (A): cap = 3B/4, rejects -> pend_u32; phase 1 (B): cap = B, rejects
// -> pend_u64 (alt block << 32 | index); phase 2 (C): cap = B, rejects -> pend_u32
// The blocks of a phase: every block with the scanned offsets (dense phases),
// or only the touched ones with their segments (sparse phases, dlist set).
struct PhaseDst {
    const uint32_t *off;     // dense: nb + 1 scanned offsets
    const uint32_t *dlist;   // sparse: touched destinations
    const uint64_t *seg;     // sparse: start << 32 | count
    const unsigned *nlist;   // sparse: number of touched destinations
};

__device__ __forceinline__ uint64_t phase_count(const PhaseDst &P, uint64_t dense_n)
{
    return P.dlist ? (uint64_t)*P.nlist : dense_n;
}

// destination j of the phase with its record range [s, e)
__device__ __forceinline__ uint64_t phase_dst(const PhaseDst &P, uint64_t j, uint32_t &s, uint32_t &e)
{
    if (P.dlist) {
        const uint64_t sg = P.seg[j];
        s = (uint32_t)(sg >> 32);
        e = s + (uint32_t)sg;
        return P.dlist[j];
    }
    s = P.off[j];
    e = P.off[j + 1];
    return j;
}

// A warp reserves room for all its lanes' entries of a pending list with one
// atomic; lane l's entries start at the returned position. Every lane of the
// warp must call it.
__device__ __forceinline__ uint32_t warp_reserve(unsigned *counter, uint32_t mine)
{
    const int lane = threadIdx.x & 31;
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    uint32_t base = 0;
    if (lane == 31 && total) base = atomicAdd(counter, total);
    base = __shfl_sync(0xffffffffu, base, 31);
    return base + incl - mine;
}

// Candidates that a per-block step passes on, collected per warp in shared
// memory and written out with one reservation on the list's counter per
// full buffer, instead of one returning atomic per warp and iteration. The
// order of a pending list is free: every later phase orders its candidates
// by (tag, batch index) itself. Exactly one of o32 / o64 is set; `n` is the
// same in every lane, and every lane of the warp calls reserve and flush.
static constexpr uint32_t SINK_CAP = 256;  // entries per warp

struct RejSink {
    uint64_t *buf;
    uint32_t n;
    uint32_t *o32;
    uint64_t *o64;
    unsigned *ctr;

    __device__ __forceinline__ void flush()
    {
        const int lane = threadIdx.x & 31;
        __syncwarp();
        uint32_t base = 0;
        if (lane == 0 && n) base = atomicAdd(ctr, n);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (uint32_t q = lane; q < n; q += 32) {
            if (o64) o64[base + q] = buf[q];
            else o32[base + q] = (uint32_t)buf[q];
        }
        __syncwarp();
        n = 0;
    }
    // this lane's first position for `mine` entries; `direct` when the warp's
    // entries exceed a buffer and go straight to the list
    __device__ __forceinline__ uint32_t reserve(uint32_t mine, bool &direct)
    {
        const int lane = threadIdx.x & 31;
        uint32_t incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        if (n + total > SINK_CAP) flush();
        if (total > SINK_CAP) {
            uint32_t base = 0;
            if (lane == 31) base = atomicAdd(ctr, total);
            base = __shfl_sync(0xffffffffu, base, 31);
            direct = true;
            return base + incl - mine;
        }
        direct = false;
        const uint32_t pos = n + incl - mine;
        n += total;
        return pos;
    }
    __device__ __forceinline__ void put(bool direct, uint32_t &slot, uint64_t v)
    {
        if (!direct) buf[slot] = v;
        else if (o64) o64[slot] = v;
        else o32[slot] = (uint32_t)v;
        slot++;
    }
};

// The grid-stride loops of the per-block kernels step whole warps, so that
// every lane reaches the sink's reserve in every iteration and its flush
// after the last one.
template <int F>
__global__ void __launch_bounds__(TPB) tcf_block_insert(TcfGeom G, uint8_t *blocks, uint8_t *fill, PhaseDst P,
                                                        const uint64_t *__restrict__ rec, int phase,
                                                        uint32_t cap, uint32_t *pend32, uint64_t *pend64,
                                                        unsigned *npend, const TcfPrep prep,
                                                        unsigned long long *units)
{
    constexpr int B = Blk<F>::B;
    __shared__ uint64_t s_sink[TPB / 32][SINK_CAP];
    RejSink sink{s_sink[threadIdx.x >> 5], 0u, phase == 1 ? nullptr : pend32, phase == 1 ? pend64 : nullptr, npend};
    const uint64_t nd = phase_count(P, G.nb);
    if (P.dlist) note_units(units, nd);  // units: blocks with candidates
    const uint64_t stride = (uint64_t)gridDim.x * TPB;
    for (uint64_t j0 = blockIdx.x * (uint64_t)TPB + (threadIdx.x & ~31u); j0 < nd; j0 += stride) {
        const uint64_t j = j0 + (threadIdx.x & 31);
        uint32_t s = 0, e = 0, k = 0, f0 = 0;
        uint64_t b = 0, thr = 0;  // records <= thr are accepted
        if (j < nd) {
            b = phase_dst(P, j, s, e);
            f0 = fill[b];  // dense phases: b = j, so this load goes out with the offsets'
        }
        if (units && !P.dlist) {
            const unsigned t = __ballot_sync(0xffffffffu, s != e);
            if ((threadIdx.x & 31) == 0 && t) atomicAdd(units, (unsigned long long)__popc(t));
        }
        if (j < nd) {
            if (s != e) {
                const uint32_t cnt = e - s;
                k = cap > f0 ? min(cnt, cap - f0) : 0u;
                if (k > 0 && cnt <= 8) {
                    // few candidates: all loads in flight at once, a sorting
                    // network in registers, a bitonic merge into the block
                    Blk<F> blk;
                    blk.load(blocks, b);
                    uint64_t r8[8];
#pragma unroll
                    for (int q = 0; q < 8; q++) r8[q] = q < (int)cnt ? rec[s + q] : ~0ull;
                    sort_small(r8, cnt);
#pragma unroll
                    for (int q = 0; q < 8; q++)
                        if (q == (int)k - 1) thr = r8[q];
                    blk.merge_new(f0, k, r8);
                    blk.store(blocks, b);
                    fill[b] = (uint8_t)(f0 + k);
                } else if (k > 0) {
                    Blk<F> blk;
                    blk.load(blocks, b);
                    uint64_t a[MAXSEL];
                    int have = 0;
                    for (uint32_t q = s; q < e; q++) have = topk_push(a, have, (int)k, rec[q]);
                    thr = a[k - 1];
                    uint32_t t_out[B];
                    int ia = 0, ib = 0;
#pragma unroll
                    for (int p = 0; p < B; p++) {
                        uint32_t ta = (ia < (int)f0) ? blk.tag(ia) : 0xffffffffu;
                        uint32_t tb = (ib < (int)k) ? (uint32_t)(a[ib] >> 32) : 0xffffffffu;
                        if (ta == 0xffffffffu && tb == 0xffffffffu) {
                            t_out[p] = 0;
                        } else if (ta <= tb) {
                            t_out[p] = ta;
                            ia++;
                        } else {
                            t_out[p] = tb;
                            ib++;
                        }
                    }
                    blk.pack(t_out);
                    blk.store(blocks, b);
                    fill[b] = (uint8_t)(f0 + k);
                }
            }
        }
        const uint32_t nrej = (e - s) - k;
        bool direct;
        uint32_t slot = sink.reserve(nrej, direct);
        if (nrej == 0) continue;
        for (uint32_t q = s; q < e; q++) {
            const uint64_t r = rec[q];
            if (k > 0 && r <= thr) continue;
            const uint32_t i = (uint32_t)r;
            if (phase == 1) {
                // the other block of the pair: b1 + b2 - b
                uint64_t alt = prep.bt ? (prep.bt[i] >> 32) + prep.b2[i] - b
                                       : b ^ tcf_g((uint32_t)(r >> 32) >> G.vbits, G.nb);
                sink.put(direct, slot, (alt << 32) | i);
            } else {
                sink.put(direct, slot, i);
            }
        }
    }
    sink.flush();
}

// backing buckets: candidates (entry in rec, index in recI) taken in (entry,
// index) order while there is room; the rest are FULL
__global__ void __launch_bounds__(TPB) tcf_bucket_insert(TcfGeom G, uint64_t *bk, PhaseDst P,
                                                         const uint64_t *__restrict__ rec,
                                                         const uint32_t *__restrict__ recI, uint8_t *status,
                                                         DevCounters *ctr, unsigned long long *units)
{
    const uint64_t nd = phase_count(P, G.nbk);
    note_units(units, nd);  // units: buckets with candidates
    for (uint64_t j = blockIdx.x * (uint64_t)TPB + threadIdx.x; j < nd; j += (uint64_t)gridDim.x * TPB) {
        uint32_t s, e;
        const uint64_t q = phase_dst(P, j, s, e);
        if (s == e) continue;
        uint64_t cur[BK_W];
        int used = 0;
        for (int j = 0; j < (int)BK_W; j++) {
            cur[j] = bk[q * BK_W + j];
            used += cur[j] != 0;
        }
        const uint32_t cnt = e - s;
        const uint32_t k = min(cnt, BK_W - (uint32_t)used);
        // select the k smallest (entry, index) pairs by repeated minimum
        uint64_t pe = 0;
        uint32_t pi = 0;
        bool have_prev = false;
        uint64_t acc_e[BK_W];
        for (uint32_t m = 0; m < k; m++) {
            uint64_t be = ~0ull;
            uint32_t bi = 0xffffffffu;
            for (uint32_t j = s; j < e; j++) {
                uint64_t ee = rec[j];
                uint32_t ii = recI[j];
                bool after = !have_prev || ee > pe || (ee == pe && ii > pi);
                bool better = ee < be || (ee == be && ii < bi);
                if (after && better) {
                    be = ee;
                    bi = ii;
                }
            }
            acc_e[m] = be;
            pe = be;
            pi = bi;
            have_prev = true;
        }
        // merge accepted (ascending) into the bucket's sorted entries
        uint64_t outv[BK_W];
        int ia = 0, ib = 0;
        for (int p = 0; p < (int)BK_W; p++) {
            uint64_t va = ia < used ? cur[ia] : ~0ull;
            uint64_t vb = ib < (int)k ? acc_e[ib] : ~0ull;
            if (va == ~0ull && vb == ~0ull) outv[p] = 0;
            else if (va <= vb) { outv[p] = va; ia++; }
            else { outv[p] = vb; ib++; }
        }
        for (int j = 0; j < (int)BK_W; j++) bk[q * BK_W + j] = outv[j];
        if (k > 0) atomicAdd(&ctr->backing, (unsigned long long)k);
        if (k < cnt) {
            // rejected: every pair after the k-th accepted one
            for (uint32_t j = s; j < e; j++) {
                uint64_t ee = rec[j];
                uint32_t ii = recI[j];
                bool acc = k > 0 && (ee < pe || (ee == pe && ii <= pi));
                if (!acc) {
                    if (status) status[ii] = FILTER_KEY_FULL;
                    atomicAdd(&ctr->failed, 1ull);
                }
            }
            atomicOr(&ctr->status, ST_FULL);
        }
    }
}

// ---------------------------------------------------------------------------
// Bulk delete: per-block matching. For each tag present c times in the block,
// the c smallest (tag, index) candidates with that tag remove one copy each.
// ---------------------------------------------------------------------------
template <int F>
__global__ void __launch_bounds__(TPB) tcf_block_remove(TcfGeom G, uint8_t *blocks, uint8_t *fill, PhaseDst P,
                                                        const uint64_t *__restrict__ rec, uint32_t *pend32,
                                                        unsigned *npend, unsigned long long *units)
{
    constexpr int B = Blk<F>::B;
    __shared__ uint64_t s_sink[TPB / 32][SINK_CAP];
    RejSink sink{s_sink[threadIdx.x >> 5], 0u, pend32, nullptr, npend};
    const uint64_t nd = phase_count(P, G.nb);
    if (P.dlist) note_units(units, nd);  // units: blocks with candidates
    const uint32_t lm = Blk<F>::lane_mask(G.vmask);
    const uint64_t stride = (uint64_t)gridDim.x * TPB;
    for (uint64_t j0 = blockIdx.x * (uint64_t)TPB + (threadIdx.x & ~31u); j0 < nd; j0 += stride) {
        const uint64_t j = j0 + (threadIdx.x & 31);
        uint32_t s = 0, e = 0, nunm = 0, unm = 0;
        bool fast = false;
        uint64_t r8[8];  // fast path: the candidates, sorted
        // general path: per distinct stored tag, its first slot, the copies,
        // the candidates that matched and the largest matched record
        uint32_t dt[B], dp[B], dc[B], used[B];
        uint64_t thr[B];
        int ndt = 0;
        uint64_t b = 0;
        uint32_t f0 = 0;
        if (j < nd) {
            b = phase_dst(P, j, s, e);
            f0 = fill[b];  // dense phases: b = j, so this load goes out with the offsets'
        }
        if (units && !P.dlist) {
            const unsigned t = __ballot_sync(0xffffffffu, s != e);
            if ((threadIdx.x & 31) == 0 && t) atomicAdd(units, (unsigned long long)__popc(t));
        }
        if (j < nd) {
            if (s != e) {
                Blk<F> blk;
                blk.load(blocks, b);
                int removed = 0;
                if (e - s <= 8) {
                    // few candidates: sort them in registers; each takes the
                    // first remaining copy of its tag, so the block stays sorted
                    fast = true;
                    const uint32_t c = e - s;
#pragma unroll
                    for (int q = 0; q < 8; q++) r8[q] = (uint32_t)q < c ? rec[s + q] : ~0ull;
                    sort_small(r8, c);
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        if ((uint32_t)q < c) {
                            const uint32_t sm = blk.eq_slots((uint32_t)(r8[q] >> 32), lm);
                            if (sm) {
                                blk.delete_at(__ffs(sm) - 1);
                                removed++;
                            } else {
                                unm |= 1u << q;
                                nunm++;
                            }
                        }
                    }
                    if (removed) {
                        blk.store(blocks, b);
                        fill[b] = (uint8_t)(f0 - removed);
                    }
                } else {
                    uint32_t tags[B];
#pragma unroll
                    for (int p = 0; p < B; p++) tags[p] = blk.tag(p);
                    // copies of a tag are adjacent (sorted by tag, then value)
                    for (int p = 0; p < (int)f0; p++) {
                        const uint32_t mt = tags[p] & ~G.vmask;
                        if (ndt > 0 && dt[ndt - 1] == mt) {
                            dc[ndt - 1]++;
                        } else {
                            dt[ndt] = mt;
                            dp[ndt] = (uint32_t)p;
                            dc[ndt] = 1;
                            ndt++;
                        }
                    }
                    for (int d = 0; d < ndt; d++) {
                        uint64_t a[MAXSEL];
                        int have = 0;
                        uint64_t lo = (uint64_t)dt[d] << 32, hi = lo | 0xffffffffull;
                        for (uint32_t q = s; q < e; q++) {
                            uint64_t r = rec[q];
                            if (r >= lo && r <= hi) have = topk_push(a, have, (int)dc[d], r);
                        }
                        used[d] = (uint32_t)have;
                        thr[d] = have ? a[have - 1] : 0;
                    }
                    // rebuild the block without the removed copies (the
                    // smallest values of each tag)
                    uint32_t t_out[B];
                    int o = 0;
                    for (int d = 0; d < ndt; d++) {
                        for (uint32_t c = used[d]; c < dc[d]; c++) t_out[o++] = tags[dp[d] + c];
                        removed += (int)used[d];
                    }
                    for (int p = o; p < B; p++) t_out[p] = 0;
                    if (removed) {
                        blk.pack(t_out);
                        blk.store(blocks, b);
                        fill[b] = (uint8_t)(f0 - removed);
                    }
                    nunm = (e - s) - (uint32_t)removed;
                }
            }
        }
        // unmatched candidates go on
        bool direct;
        uint32_t slot = sink.reserve(nunm, direct);
        if (nunm == 0) continue;
        if (fast) {
#pragma unroll
            for (int q = 0; q < 8; q++)
                if ((unm >> q) & 1u) sink.put(direct, slot, (uint32_t)r8[q]);
        } else {
            for (uint32_t q = s; q < e; q++) {
                const uint64_t r = rec[q];
                const uint32_t t = (uint32_t)(r >> 32);
                bool matched = false;
                for (int d = 0; d < ndt; d++)
                    if (dt[d] == t && used[d] > 0 && r <= thr[d]) matched = true;
                if (!matched) sink.put(direct, slot, (uint32_t)r);
            }
        }
    }
    sink.flush();
}

// ---------------------------------------------------------------------------
// Bulk delete of the backing buckets: per stored entry, the smallest batch
// indices among the candidates with that entry remove one copy each.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TPB) tcf_bucket_remove(TcfGeom G, uint64_t *bk, PhaseDst P,
                                                         const uint64_t *__restrict__ rec,
                                                         const uint32_t *__restrict__ recI, uint8_t *status,
                                                         DevCounters *ctr, unsigned long long *units)
{
    const uint64_t nd = phase_count(P, G.nbk);
    note_units(units, nd);  // units: buckets with candidates
    for (uint64_t j = blockIdx.x * (uint64_t)TPB + threadIdx.x; j < nd; j += (uint64_t)gridDim.x * TPB) {
        uint32_t s, e;
        const uint64_t q = phase_dst(P, j, s, e);
        if (s == e) continue;
        // distinct stored entries without their values (the bucket is sorted,
        // so copies are adjacent) with their first position and copy counts
        uint64_t cur[BK_W], dv[BK_W];
        uint32_t dp[BK_W], dc[BK_W], used[BK_W], thr[BK_W];
        int nd = 0;
        for (int j = 0; j < (int)BK_W; j++) {
            const uint64_t v = bk[q * BK_W + j];
            cur[j] = v;
            if (!v) continue;
            const uint64_t mv = v & ~(uint64_t)G.vmask;
            if (nd > 0 && dv[nd - 1] == mv) {
                dc[nd - 1]++;
            } else {
                dv[nd] = mv;
                dp[nd] = (uint32_t)j;
                dc[nd] = 1;
                nd++;
            }
        }
        // for each stored entry, the dc smallest candidate indices with that entry match
        for (int d = 0; d < nd; d++) {
            uint64_t a[BK_W];
            int have = 0;
            for (uint32_t j = s; j < e; j++)
                if (rec[j] == dv[d]) have = topk_push(a, have, (int)dc[d], (uint64_t)recI[j]);
            used[d] = (uint32_t)have;
            thr[d] = have ? (uint32_t)a[have - 1] : 0u;
        }
        int removed = 0;
        uint64_t outv[BK_W];
        int o = 0;
        for (int d = 0; d < nd; d++) {
            removed += (int)used[d];
            for (uint32_t c = used[d]; c < dc[d]; c++) outv[o++] = cur[dp[d] + c];
        }
        for (int j = o; j < (int)BK_W; j++) outv[j] = 0;
        if (removed) {
            for (int j = 0; j < (int)BK_W; j++) bk[q * BK_W + j] = outv[j];
            atomicAdd(&ctr->backing, (unsigned long long)(-(long long)removed));
        }
        for (uint32_t j = s; j < e; j++) {
            uint64_t v = rec[j];
            uint32_t ii = recI[j];
            bool matched = false;
            for (int d = 0; d < nd; d++)
                if (dv[d] == v && used[d] > 0 && ii <= thr[d]) matched = true;
            if (!matched && status) status[ii] = FILTER_KEY_NOT_FOUND;
        }
    }
}

// ---------------------------------------------------------------------------
// Tiled bulk phases. A phase groups its candidates by destination block in
// two steps that keep every global write coalesced: a partition by tile (TB
// consecutive blocks) in one or two counting passes, each staging a chunk of
// candidates in shared memory in bin order before writing it out, then one
// CTA per tile that sorts the tile's candidates by block in shared memory and
// runs the per-block step (accept into the sorted block, or remove) with the
// block loaded and stored by consecutive threads. A candidate record is
// (dest << 16 | slot, batch index); inside a tile it becomes the per-block
// record (slot << 32 | index) that the per-block steps take in (slot, index)
// order. The partition passes write to L2-sized runs instead of scattering 8
// bytes per key over a batch-sized array, which is what keeps large batches
// (2^24 keys into 2^24 blocks) off the DRAM read-modify-write path.
// ---------------------------------------------------------------------------
static constexpr int TT_TPB = 256;      // threads of the partition and tile kernels
static constexpr int TT_CH = 2048;      // items per partition chunk (8 per thread)
static constexpr int TT_BINS = 512;     // shared-memory bins of a partition chunk
static constexpr uint32_t TT_CAP = 2048;  // candidates a tile stages in shared memory (8 per thread)
static constexpr uint32_t TT_TB_MAX = 2048;
static constexpr uint64_t TT_LEFT = 1ull << 63;  // stage entry: the candidate is left for the next phase

// words of the tile counters a filter needs: counts (nt + 1), high-bin
// cursors (nh) and tile cursors (nt), at the smallest tile size
static uint64_t tt_counter_words(uint64_t nb) { return 2 * ((nb + 31) / 32) + 256 + 8; }

// tile geometry of one call: tiles of 2^tb_log blocks; lo > 0: two passes,
// the first by tile >> lo (nh bins), the second by tile
struct TtGeom {
    uint64_t nb, nt, nh;
    uint32_t tb_log, lo;
};

// where a phase's candidates come from: the call's keys (hashed here, or the
// prepared keys of a group call), or a pending list (rec, idx) of n_dev items
struct TtSrc {
    const uint64_t *keys;
    const uint64_t *rec;
    const uint32_t *idx;
    const unsigned *n_dev;  // pending lists: their length on the device
    uint64_t n;             // keys: their number; pending lists: an upper bound
};

enum TtSrcKind : int { TT_KEYS = 0, TT_PEND = 1 };
enum TtRule : int { TT_SAME = 0, TT_TARGET = 1 };              // dest: the record's block, or the less full
enum TtNext : int { TT_NX_SAME = 0, TT_NX_OTHER = 1, TT_NX_IDX = 2 };  // what a reject becomes

__device__ __forceinline__ uint64_t tt_count(const TtSrc &s) { return s.n_dev ? (uint64_t)*s.n_dev : s.n; }

// the other block of the pair of candidate (b, slot, idx): b1 ^ b2 = g(tag)
// for a single filter; group calls read the prepared pair
__device__ __forceinline__ uint64_t tt_other(uint64_t b, uint32_t slot, uint32_t i, const TcfGeom &G,
                                            const TcfPrep &P)
{
    if (P.bt) return (P.bt[i] >> 32) + P.b2[i] - b;
    return b ^ tcf_g(slot >> G.vbits, G.nb);
}

// candidate j of a phase as (dest << 16 | slot, index)
template <int SRC, int RULE>
__device__ __forceinline__ void tt_item(const TtSrc &s, uint64_t j, const TcfGeom &G, const TcfPrep &P,
                                        const uint8_t *fill, uint64_t &rec, uint32_t &idx)
{
    if (SRC == TT_KEYS) {
        idx = (uint32_t)j;
        if (P.bt) {
            const uint64_t v = P.bt[j];
            rec = ((v >> 32) << 16) | (uint32_t)(v & 0xffffu);
        } else {
            KeyInfo k = tcf_keyinfo(s.keys[j], G);
            if (P.vals) k.t |= P.vals[j] & G.vmask;
            rec = (k.b1 << 16) | k.t;
        }
        return;
    }
    rec = s.rec[j];
    idx = s.idx[j];
    if (RULE == TT_TARGET) {
        const uint64_t b1 = rec >> 16;
        const uint32_t slot = (uint32_t)(rec & 0xffffu);
        const uint64_t b2 = tt_other(b1, slot, idx, G, P);
        const uint64_t d = fill[b1] <= fill[b2] ? b1 : b2;
        rec = (d << 16) | slot;
    }
}

// Counter words of a phase: cnt[nt + 1] | hcur[nh] | tcur[nt] | done.
struct TtCtr {
    uint32_t *cnt, *hcur, *tcur, *done;
};

__device__ __forceinline__ TtCtr tt_ctr(uint32_t *base, const TtGeom &tg)
{
    TtCtr c;
    c.cnt = base;
    c.hcur = base + tg.nt + 1;
    c.tcur = c.hcur + tg.nh;
    c.done = c.tcur + tg.nt;
    return c;
}

// Per-tile candidate counts, from a shared histogram when the tiles fit in
// it. The last CTA to finish turns them into the tiles' offsets toff[0 ..
// nt] (toff[nt] = all candidates) and clears the counts and `done`; `reset`
// (first phase of a call) also clears the call's pending-list lengths and
// bucket-phase cursors. Every counter word is zero between phases (the tile
// kernel clears the partition cursors), whatever tile geometry a call uses.
template <int SRC, int RULE>
__global__ void __launch_bounds__(TT_TPB) tt_hist(const TtSrc s, TcfGeom G, TcfPrep P, const uint8_t *fill,
                                                  TtGeom tg, uint32_t *ctr_words, uint32_t *toff,
                                                  DevCounters *reset, unsigned long long *units)
{
    extern __shared__ uint32_t s_h[];
    __shared__ uint32_t s_wsum[TT_TPB / 32];
    __shared__ bool s_last;
    const TtCtr C = tt_ctr(ctr_words, tg);
    const uint64_t n = tt_count(s);
    note_units(units, n);
    if (n == 0) return;  // an empty phase: the later kernels of the phase see n = 0 and do nothing
    // a shared histogram pays off when each CTA has enough items for its bins
    const bool shared = tg.nt <= 8192 && n * 8 >= (uint64_t)gridDim.x * tg.nt;
    if (shared) {
        for (uint32_t t = threadIdx.x; t < tg.nt; t += TT_TPB) s_h[t] = 0;
        __syncthreads();
    }
    for (uint64_t j = blockIdx.x * (uint64_t)TT_TPB + threadIdx.x; j < n; j += (uint64_t)gridDim.x * TT_TPB) {
        uint64_t rec;
        uint32_t idx;
        tt_item<SRC, RULE>(s, j, G, P, fill, rec, idx);
        const uint32_t t = (uint32_t)((rec >> 16) >> tg.tb_log);
        if (shared) atomicAdd(&s_h[t], 1u);
        else atomicAdd(&C.cnt[t], 1u);
    }
    if (shared) {
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < tg.nt; t += TT_TPB)
            if (s_h[t]) atomicAdd(&C.cnt[t], s_h[t]);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(C.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the last CTA: exclusive scan of cnt[0 .. nt] into toff, in chunks of
    // 16 counts per thread with a running carry
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr uint32_t PER = 16;
    uint32_t carry = 0;
    for (uint64_t c0 = 0; c0 <= tg.nt; c0 += (uint64_t)TT_TPB * PER) {
        const uint64_t b0 = c0 + (uint64_t)threadIdx.x * PER;
        uint32_t v[PER], sum = 0;
#pragma unroll
        for (uint32_t k = 0; k < PER; k++) {
            v[k] = (b0 + k <= tg.nt) ? __ldcg(C.cnt + b0 + k) : 0u;
            sum += v[k];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        uint32_t run = carry + incl - sum, tot = 0;
        for (int w = 0; w < TT_TPB / 32; w++) {
            if (w < warp) run += s_wsum[w];
            tot += s_wsum[w];
        }
#pragma unroll
        for (uint32_t k = 0; k < PER; k++) {
            if (b0 + k <= tg.nt) toff[b0 + k] = run;
            run += v[k];
        }
        carry += tot;
        __syncthreads();
    }
    // clear the counts for the next phase (the partition cursors are
    // cleared by the tile kernel, after the passes that use them)
    for (uint64_t k = threadIdx.x; k <= tg.nt; k += TT_TPB) ctr_words[k] = 0;
    if (reset && threadIdx.x == 0) {
        for (int k = 0; k < 8; k++) reset->pend[k] = 0;
        for (int k = 0; k < 4; k++) reset->touched[k] = reset->cursor[k] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) *C.done = 0;
}

// One partition pass. PASS 0: the only pass, bins are tiles; PASS 1: bins are
// tile >> lo, each bin's region the span of its tiles; PASS 2: the pass-1
// output, bins are tiles relative to the chunk's first high bin (a chunk that
// reaches past TT_BINS of them places the rest by global atomics). toff: the
// tiles' scanned offsets; hcur / tcur: the running cursors of the high bins
// and of the tiles (zero at the start of the phase).
template <int SRC, int RULE, int PASS>
__global__ void __launch_bounds__(TT_TPB, 4) tt_part(const TtSrc s, TcfGeom G, TcfPrep P, const uint8_t *fill,
                                                  TtGeom tg, const uint32_t *__restrict__ toff, uint32_t *ctr_words,
                                                  uint64_t *__restrict__ orec, uint32_t *__restrict__ oidx,
                                                  unsigned long long *units)
{
    const TtCtr C = tt_ctr(ctr_words, tg);
    uint32_t *hcur = C.hcur, *tcur = C.tcur;
    __shared__ uint32_t s_cnt[TT_BINS], s_start[TT_BINS], s_base[TT_BINS];
    __shared__ uint64_t s_rec[TT_CH];
    __shared__ uint32_t s_idx[TT_CH];
    __shared__ uint16_t s_bin[TT_CH];
    __shared__ uint32_t s_wsum[TT_TPB / 32];
    __shared__ uint64_t s_tbase;
    constexpr int IPT = TT_CH / TT_TPB;
    const uint64_t n = tt_count(s);
    note_units(units, n);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint64_t c0 = (uint64_t)blockIdx.x * TT_CH; c0 < n; c0 += (uint64_t)gridDim.x * TT_CH) {
        for (int b = threadIdx.x; b < TT_BINS; b += TT_TPB) s_cnt[b] = 0;
        if (PASS == 2 && threadIdx.x == 0) s_tbase = ((s.rec[c0] >> 16) >> (tg.tb_log + tg.lo)) << tg.lo;
        __syncthreads();
        uint64_t rec[IPT];
        uint32_t idx[IPT], rank[IPT];
        uint32_t bin[IPT];
#pragma unroll
        for (int q = 0; q < IPT; q++) {
            const uint64_t j = c0 + threadIdx.x + (uint64_t)q * TT_TPB;
            bin[q] = 0xffffffffu;
            if (j < n) {
                tt_item<SRC, RULE>(s, j, G, P, fill, rec[q], idx[q]);
                const uint64_t t = (rec[q] >> 16) >> tg.tb_log;
                const uint64_t b = PASS == 1 ? (t >> tg.lo) : (PASS == 2 ? t - s_tbase : t);
                if (b < TT_BINS && t < tg.nt) {
                    bin[q] = (uint32_t)b;
                    rank[q] = atomicAdd(&s_cnt[b], 1u);
                } else if (PASS == 2 && t < tg.nt) {  // a tile far past the chunk's first high bin
                    const uint32_t pos = toff[t] + atomicAdd(&tcur[t], 1u);
                    if (pos < toff[tg.nt]) {
                        orec[pos] = rec[q];
                        oidx[pos] = idx[q];
                    }
                }
            }
        }
        __syncthreads();
        // bin starts inside the chunk (exclusive scan, 2 bins per thread) and
        // each bin's global base, one atomic per non-empty bin
        {
            const uint32_t a = s_cnt[2 * threadIdx.x], b = s_cnt[2 * threadIdx.x + 1];
            uint32_t incl = a + b;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) s_wsum[warp] = incl;
            __syncthreads();
            uint32_t pre = 0;
            for (int w = 0; w < warp; w++) pre += s_wsum[w];
            const uint32_t ex = pre + incl - a - b;
            s_start[2 * threadIdx.x] = ex;
            s_start[2 * threadIdx.x + 1] = ex + a;
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const uint32_t bb = 2 * threadIdx.x + k, c = k ? b : a;
                if (!c) continue;
                if (PASS == 1) {
                    s_base[bb] = toff[(uint64_t)bb << tg.lo] + atomicAdd(&hcur[bb], c);
                } else {
                    const uint64_t t = PASS == 2 ? s_tbase + bb : bb;
                    s_base[bb] = toff[t] + atomicAdd(&tcur[t], c);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < IPT; q++) {
            if (bin[q] != 0xffffffffu) {
                const uint32_t p = s_start[bin[q]] + rank[q];
                s_rec[p] = rec[q];
                s_idx[p] = idx[q];
                s_bin[p] = (uint16_t)bin[q];
            }
        }
        __syncthreads();
        const uint32_t total = s_start[TT_BINS - 1] + s_cnt[TT_BINS - 1];
        const uint32_t lim = toff[tg.nt];
        for (uint32_t p = threadIdx.x; p < total; p += TT_TPB) {
            const uint32_t b = s_bin[p];
            const uint32_t pos = s_base[b] + (p - s_start[b]);
            if (pos < lim) {  // positions past the counted total would mean counts that disagree
                orec[pos] = s_rec[p];
                oidx[pos] = s_idx[p];
            }
        }
        __syncthreads();
    }
}

// block-wide exclusive scan of v[0 .. m) in place, v[m] = the total; m <= TT_TB_MAX
__device__ __forceinline__ void tt_block_scan(uint32_t *v, uint32_t m, uint32_t *s_wsum)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // chunks of TT_TPB entries in order, one entry per thread, with a carry
    uint32_t carry = 0;
    for (uint32_t k0 = 0; k0 <= m; k0 += TT_TPB) {
        const uint32_t i = k0 + threadIdx.x;
        const uint32_t x = i < m ? v[i] : 0u;
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        uint32_t pre = carry, tot = 0;
        for (int w = 0; w < TT_TPB / 32; w++) {
            if (w < warp) pre += s_wsum[w];
            tot += s_wsum[w];
        }
        if (i <= m) v[i] = pre + incl - x;
        carry += tot;
        __syncthreads();
    }
}

// Per-block steps with more than 8 candidates (rare: hot blocks), kept out
// of line so that the common path stays light on registers. Insert: the k
// smallest candidates join the sorted block (f0 tags); remove: for each
// stored tag present d times, the d smallest candidates with that tag take
// one copy each. Left candidates get `mark` in place. Return the new fill.
template <int F>
__device__ __noinline__ uint32_t tt_insert_many(uint8_t *blocks, uint64_t b, uint32_t f0, uint32_t k, uint64_t *cand,
                                                uint32_t c, uint64_t mark)
{
    constexpr int B = Blk<F>::B;
    Blk<F> blk;
    blk.load(blocks, b);
    uint64_t a[MAXSEL];
    int have = 0;
    for (uint32_t q = 0; q < c; q++) have = topk_push(a, have, (int)k, cand[q]);
    const uint64_t thr = a[k - 1];
    uint32_t t_out[B];
    int ia = 0, ib = 0;
#pragma unroll
    for (int p = 0; p < B; p++) {
        const uint32_t ta = (ia < (int)f0) ? blk.tag(ia) : 0xffffffffu;
        const uint32_t tb = (ib < (int)k) ? (uint32_t)(a[ib] >> 32) : 0xffffffffu;
        if (ta == 0xffffffffu && tb == 0xffffffffu) {
            t_out[p] = 0;
        } else if (ta <= tb) {
            t_out[p] = ta;
            ia++;
        } else {
            t_out[p] = tb;
            ib++;
        }
    }
    blk.pack(t_out);
    blk.store(blocks, b);
    for (uint32_t q = 0; q < c; q++)
        if (cand[q] > thr) cand[q] |= mark;
    return f0 + k;
}

template <int F>
__device__ __noinline__ uint32_t tt_remove_many(uint8_t *blocks, uint64_t b, uint32_t f0, uint64_t *cand, uint32_t c,
                                                uint32_t vmask, uint64_t mark)
{
    constexpr int B = Blk<F>::B;
    Blk<F> blk;
    blk.load(blocks, b);
    uint32_t tags[B], dt[B], dp[B], dc[B], used[B];
    uint64_t dthr[B];
    int ndt = 0, removed = 0;
#pragma unroll
    for (int p = 0; p < B; p++) tags[p] = blk.tag(p);
    for (int p = 0; p < (int)f0; p++) {
        const uint32_t mt = tags[p] & ~vmask;
        if (ndt > 0 && dt[ndt - 1] == mt) {
            dc[ndt - 1]++;
        } else {
            dt[ndt] = mt;
            dp[ndt] = (uint32_t)p;
            dc[ndt] = 1;
            ndt++;
        }
    }
    for (int d = 0; d < ndt; d++) {
        uint64_t a[MAXSEL];
        int have = 0;
        const uint64_t lo = (uint64_t)dt[d] << 32, hi = lo | 0xffffffffull;
        for (uint32_t q = 0; q < c; q++) {
            const uint64_t r = cand[q];
            if (r >= lo && r <= hi) have = topk_push(a, have, (int)dc[d], r);
        }
        used[d] = (uint32_t)have;
        dthr[d] = have ? a[have - 1] : 0;
    }
    uint32_t t_out[B];
    int o = 0;
    for (int d = 0; d < ndt; d++) {
        for (uint32_t q = used[d]; q < dc[d]; q++) t_out[o++] = tags[dp[d] + q];
        removed += (int)used[d];
    }
    for (int p = o; p < B; p++) t_out[p] = 0;
    for (uint32_t q = 0; q < c; q++) {
        const uint64_t r = cand[q];
        const uint32_t t = (uint32_t)(r >> 32);
        bool matched = false;
        for (int d = 0; d < ndt; d++)
            if (dt[d] == t && used[d] > 0 && r <= dthr[d]) matched = true;
        if (!matched) cand[q] = r | mark;
    }
    if (removed) {
        blk.pack(t_out);
        blk.store(blocks, b);
    }
    return f0 - (uint32_t)removed;
}

// The per-block step of one block: candidates cand[0 .. c) (slot << 32 |
// index, any order), the block's fill f0. Insert: the k smallest that fit
// under `cap` join the sorted block. Remove: each candidate removes one copy
// of its tag, smallest first. Candidates that are left get TT_LEFT | lb << 48
// in place. Returns the new fill.
template <int F, int OP>
__device__ __forceinline__ uint32_t tt_block_step(uint8_t *blocks, uint64_t b, uint32_t lb, uint32_t f0, uint32_t cap,
                                                  uint64_t *cand, uint32_t c, uint32_t lm, uint32_t vmask,
                                                  uint64_t &bytes)
{
    const uint64_t mark = TT_LEFT | ((uint64_t)lb << 48);
    if (OP == 0) {
        const uint32_t k = cap > f0 ? min(c, cap - f0) : 0u;
        if (k == 0) {
            for (uint32_t q = 0; q < c; q++) cand[q] |= mark;
            return f0;
        }
        bytes += 66;
        if (c > 8) return tt_insert_many<F>(blocks, b, f0, k, cand, c, mark);
        Blk<F> blk;
        blk.load(blocks, b);
        uint64_t r8[8];
#pragma unroll
        for (int q = 0; q < 8; q++) r8[q] = q < (int)c ? cand[q] : ~0ull;
        sort_small(r8, c);
        blk.merge_new(f0, k, r8);
        blk.store(blocks, b);
#pragma unroll
        for (int q = 0; q < 8; q++)
            if (q < (int)c) cand[q] = q < (int)k ? r8[q] : (r8[q] | mark);
        return f0 + k;
    }
    bytes += 32;
    if (c > 8) {
        const uint32_t f1 = tt_remove_many<F>(blocks, b, f0, cand, c, vmask, mark);
        if (f1 != f0) bytes += 34;
        return f1;
    }
    Blk<F> blk;
    blk.load(blocks, b);
    int removed = 0;
    uint64_t r8[8];
#pragma unroll
    for (int q = 0; q < 8; q++) r8[q] = (uint32_t)q < c ? cand[q] : ~0ull;
    sort_small(r8, c);
#pragma unroll
    for (int q = 0; q < 8; q++) {
        if ((uint32_t)q < c) {
            const uint32_t sm = blk.eq_slots((uint32_t)(r8[q] >> 32), lm);
            if (sm) {
                blk.delete_at(__ffs(sm) - 1);
                removed++;
                cand[q] = r8[q];
            } else {
                cand[q] = r8[q] | mark;
            }
        }
    }
    if (removed) {
        blk.store(blocks, b);
        bytes += 34;
    }
    return f0 - (uint32_t)removed;
}

// One CTA per tile (looping over tiles): the tile's candidates are counted
// per block with their rank (shared atomics, the records held in registers),
// placed in block order in shared memory (a tile with more than TT_CAP of
// them is staged in the spare record buffer `gstage` at the same offsets and
// read twice), each block with candidates takes its step, and the candidates
// left are written out with one reservation per tile. A dense tile (at least
// one candidate per TT_DENSE blocks) moves its blocks into shared memory with
// one bulk copy, issued before the staging so that the two overlap, and back
// with one bulk store; a sparse one reads and writes only the blocks it
// touches. What a candidate left becomes (NEXT): the same block's record
// (phase A rejects: phase B finds their target), the other block's record
// (phase B rejects, remove misses in b1), or its batch index (for the
// backing-bucket phase). n_dev: the phase's candidate count when it comes from
// a pending list (the kernel returns at once for an empty phase). units:
// algorithmic bytes (12 per candidate read and per candidate left, 32 per
// block read, 32 per block written, 2 per fill read and written).
static constexpr uint32_t TT_DENSE = 4;

template <int F, int OP, int NEXT>
__global__ void __launch_bounds__(TT_TPB, 4) tt_tile(TcfGeom G, TcfPrep P, uint8_t *blocks, uint8_t *fill, TtGeom tg,
                                                  const uint32_t *__restrict__ toff, const uint64_t *__restrict__ rec,
                                                  const uint32_t *__restrict__ ridx, uint64_t *gstage, uint32_t cap,
                                                  uint64_t *orec, uint32_t *oidx, unsigned *nout, uint64_t out_cap,
                                                  const unsigned *n_dev, uint32_t *ctr_words,
                                                  unsigned long long *status, unsigned long long *units)
{
    constexpr uint32_t RPT = TT_CAP / TT_TPB;
    if (n_dev && *n_dev == 0) return;  // an empty phase: nothing was counted or placed
    extern __shared__ __align__(128) uint64_t s_mem[];
    const uint32_t TB = 1u << tg.tb_log;
    uint8_t *s_blocks = reinterpret_cast<uint8_t *>(s_mem);                     // TB x 32 bytes
    uint64_t *s_stage = s_mem + TB * 4;                                         // TT_CAP entries
    uint32_t *s_start = reinterpret_cast<uint32_t *>(s_stage + TT_CAP);         // TB + 1
    uint8_t *s_fill = reinterpret_cast<uint8_t *>(s_start + TB + 1);            // TB
    __shared__ uint32_t s_wsum[TT_TPB / 32];
    __shared__ uint32_t s_base;
    __shared__ unsigned long long s_bytes;
    __shared__ __align__(8) uint64_t s_bar;
    {
        // the partition passes of this phase are done with their cursors
        const TtCtr C = tt_ctr(ctr_words, tg);
        const uint64_t w = tg.nh + tg.nt;
        for (uint64_t k = blockIdx.x * (uint64_t)TT_TPB + threadIdx.x; k < w; k += (uint64_t)gridDim.x * TT_TPB)
            C.hcur[k] = 0;
    }
    if (threadIdx.x == 0) mbar_init(&s_bar, 1);
    __syncthreads();
    uint32_t parity = 0;
    bool stores_pending = false;  // thread 0: a bulk store may still read s_blocks
    const uint32_t lm = Blk<F>::lane_mask(G.vmask);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint64_t T = blockIdx.x; T < tg.nt; T += gridDim.x) {
        const uint32_t s = toff[T], e = toff[T + 1];
        if (s == e) continue;
        const uint64_t b0 = T << tg.tb_log;
        const uint32_t nblk = (uint32_t)min((uint64_t)TB, tg.nb - b0);
        const uint32_t cnt = e - s;
        const bool in_smem = cnt <= TT_CAP;
        const bool dense = (uint64_t)cnt * TT_DENSE >= nblk;
        uint64_t *stage = in_smem ? s_stage : gstage + s;
        if (dense && threadIdx.x == 0) {
            if (stores_pending) bulk_wait_read();  // the previous tile's store has read s_blocks
            stores_pending = false;
            mbar_arrive_expect(&s_bar, nblk * 32);
            bulk_load(s_blocks, blocks + b0 * 32, nblk * 32, &s_bar);
        }
        for (uint32_t k = threadIdx.x; k <= nblk; k += TT_TPB) s_start[k] = 0;
        if (dense)
            for (uint32_t k = threadIdx.x; k < nblk; k += TT_TPB) s_fill[k] = fill[b0 + k];
        if (threadIdx.x == 0) s_bytes = 0;
        __syncthreads();
        uint64_t rv[RPT];
        uint32_t rank[RPT];
        if (in_smem) {
#pragma unroll
            for (uint32_t q = 0; q < RPT; q++) {
                const uint32_t r = s + threadIdx.x + q * TT_TPB;
                rank[q] = 0xffffffffu;
                if (r < e) {
                    const uint64_t v = rec[r];
                    const uint64_t lb = (v >> 16) - b0;
                    if (lb >= nblk) {  // a record outside its tile: report, never index with it
                        atomicOr(status, ST_INTERNAL);
                        continue;
                    }
                    rank[q] = atomicAdd(&s_start[lb], 1u);
                    rv[q] = (lb << 48) | ((v & 0xffffu) << 32) | ridx[r];
                }
            }
        } else {
            for (uint32_t r = s + threadIdx.x; r < e; r += TT_TPB) {
                const uint64_t lb = (rec[r] >> 16) - b0;
                if (lb < nblk) atomicAdd(&s_start[lb], 1u);
                else atomicOr(status, ST_INTERNAL);
            }
        }
        __syncthreads();
        tt_block_scan(s_start, nblk, s_wsum);
        if (in_smem) {
#pragma unroll
            for (uint32_t q = 0; q < RPT; q++) {
                const uint32_t r = s + threadIdx.x + q * TT_TPB;
                if (r < e && rank[q] != 0xffffffffu) {
                    const uint32_t lb = (uint32_t)(rv[q] >> 48);
                    const uint32_t p = s_start[lb] + rank[q];
                    if (p < cnt) stage[p] = rv[q] & 0x0000ffffffffffffull;
                    else atomicOr(status, ST_INTERNAL);
                }
            }
        } else {
            // ranks come from a second pass: the counts above turned into
            // starts, then advanced per placed candidate and restored
            for (uint32_t r = s + threadIdx.x; r < e; r += TT_TPB) {
                const uint64_t v = rec[r];
                const uint64_t lb = (v >> 16) - b0;
                if (lb >= nblk) continue;
                const uint32_t p = atomicAdd(&s_start[lb], 1u);
                if (p < cnt) stage[p] = ((v & 0xffffu) << 32) | ridx[r];
                else atomicOr(status, ST_INTERNAL);
            }
            __syncthreads();
            // s_start[lb] now holds the end of block lb, the start of lb + 1
            constexpr uint32_t PB = TT_TB_MAX / TT_TPB;
            uint32_t prev[PB];
#pragma unroll
            for (uint32_t j = 0; j < PB; j++) {
                const uint32_t k = threadIdx.x + j * TT_TPB;
                prev[j] = (k < nblk && k > 0) ? s_start[k - 1] : 0u;
            }
            __syncthreads();
#pragma unroll
            for (uint32_t j = 0; j < PB; j++) {
                const uint32_t k = threadIdx.x + j * TT_TPB;
                if (k < nblk) s_start[k] = prev[j];
            }
        }
        if (dense) {
            // the tile's blocks have arrived (a bounded wait: give up on the
            // whole kernel, reporting a timeout, rather than spin for ever)
            const bool ok = mbar_wait_bounded(&s_bar, parity, SPIN_LIMIT);
            parity ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
                break;
            }
        } else {
            __syncthreads();
        }
        // each block with candidates takes its step
        uint8_t *blk_base = dense ? s_blocks : blocks;
        uint64_t bytes = 0;
        for (uint32_t k = threadIdx.x; k < nblk; k += TT_TPB) {
            const uint32_t c = s_start[k + 1] - s_start[k];
            if (!c) continue;
            const uint64_t b = b0 + k;
            const uint32_t f0 = dense ? s_fill[k] : fill[b];
            if (s_start[k + 1] > cnt || s_start[k + 1] < s_start[k] || f0 > (uint32_t)Blk<F>::B) {
                atomicOr(status, ST_INTERNAL);
                continue;
            }
            bytes += 12ull * c + 2;
            const uint32_t f1 = tt_block_step<F, OP>(blk_base, dense ? k : b, k, f0, cap, stage + s_start[k], c, lm,
                                                     G.vmask, bytes);
            if (f1 != f0) fill[b] = (uint8_t)f1;
        }
        if (dense) {
            fence_async_shared();  // the block writes above, before the bulk store reads them
            __syncthreads();
            if (threadIdx.x == 0) {
                bulk_store(blocks + b0 * 32, s_blocks, nblk * 32);
                stores_pending = true;
            }
        } else {
            __syncthreads();
        }
        // the candidates left, written out in stage order with one reservation
        for (uint32_t c0 = 0; c0 < cnt; c0 += TT_CAP) {
            const uint32_t i0 = c0 + threadIdx.x * RPT;
            uint32_t mine = 0;
#pragma unroll
            for (uint32_t q = 0; q < RPT; q++)
                if (i0 + q < cnt && (stage[i0 + q] & TT_LEFT)) mine++;
            uint32_t incl = mine;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) s_wsum[warp] = incl;
            __syncthreads();
            uint32_t pre = 0, tot = 0;
            for (int w = 0; w < TT_TPB / 32; w++) {
                if (w < warp) pre += s_wsum[w];
                tot += s_wsum[w];
            }
            if (threadIdx.x == 0 && tot) s_base = atomicAdd(nout, tot);
            __syncthreads();
            uint32_t pos = s_base + pre + incl - mine;
            if (mine) {
#pragma unroll
                for (uint32_t q = 0; q < RPT; q++) {
                    if (i0 + q >= cnt) break;
                    const uint64_t v = stage[i0 + q];
                    if (!(v & TT_LEFT)) continue;
                    const uint32_t sl = (uint32_t)(v >> 32) & 0xffffu, i = (uint32_t)v;
                    if (pos >= out_cap) {  // more left than the pending list holds
                        atomicOr(status, ST_INTERNAL);
                        break;
                    }
                    if (NEXT == TT_NX_IDX) {
                        oidx[pos++] = i;
                    } else {
                        const uint64_t b = b0 + ((v >> 48) & 0x7fffu);
                        const uint64_t d = NEXT == TT_NX_OTHER ? tt_other(b, sl, i, G, P) : b;
                        orec[pos] = (d << 16) | sl;
                        oidx[pos++] = i;
                    }
                }
            }
            bytes += 12ull * mine;
            __syncthreads();
        }
        if (units && bytes) atomicAdd(&s_bytes, bytes);
        __syncthreads();
        if (units && threadIdx.x == 0 && s_bytes) atomicAdd(units, s_bytes);
    }
    if (threadIdx.x == 0 && stores_pending) bulk_wait_all();
}

// ---------------------------------------------------------------------------
// Point mode (Alg. 1)
// ---------------------------------------------------------------------------
template <int F>
__device__ bool point_put(uint8_t *blocks, uint64_t b, uint32_t t, DevCounters *ctr)
{
    constexpr int B = Blk<F>::B;
    for (int attempt = 0; attempt < 4 * B; attempt++) {
        Blk<F> blk;
        blk.load_l2(blocks, b);
        int s = -1;
#pragma unroll
        for (int p = 0; p < B; p++)
            if (s < 0 && blk.tag(p) < 2) s = p;
        if (s < 0) return false;
        uint32_t seen = blk.tag(s);
        if (F == 16) {
            unsigned short *slot = reinterpret_cast<unsigned short *>(blocks + b * 32) + s;
            if (atomicCAS(slot, (unsigned short)seen, (unsigned short)t) == (unsigned short)seen) return true;
        } else {
            unsigned int *word = reinterpret_cast<unsigned int *>(blocks + b * 32) + (s >> 2);
            unsigned sh = (s & 3) * 8;
            unsigned int cur = blk.w[s >> 2];
            unsigned int want = (cur & ~(0xffu << sh)) | (t << sh);
            if (atomicCAS(word, cur, want) == cur) return true;
        }
    }
    atomicOr(&ctr->status, ST_TIMEOUT);
    return false;
}

template <int F>
__device__ bool point_take(uint8_t *blocks, uint64_t b, uint32_t t, uint32_t vmask, DevCounters *ctr)
{
    constexpr int B = Blk<F>::B;
    for (int attempt = 0; attempt < 4 * B; attempt++) {
        Blk<F> blk;
        blk.load_l2(blocks, b);
        int s = -1;
#pragma unroll
        for (int p = 0; p < B; p++)
            if (s < 0 && (blk.tag(p) & ~vmask) == t) s = p;
        if (s < 0) return false;
        if (F == 16) {
            unsigned short *slot = reinterpret_cast<unsigned short *>(blocks + b * 32) + s;
            const unsigned short seen = (unsigned short)blk.tag(s);
            if (atomicCAS(slot, seen, (unsigned short)1) == seen) return true;
        } else {
            unsigned int *word = reinterpret_cast<unsigned int *>(blocks + b * 32) + (s >> 2);
            unsigned sh = (s & 3) * 8;
            unsigned int cur = blk.w[s >> 2];
            unsigned int want = (cur & ~(0xffu << sh)) | (1u << sh);
            if (atomicCAS(word, cur, want) == cur) return true;
        }
    }
    atomicOr(&ctr->status, ST_TIMEOUT);
    return false;
}

template <int F>
__global__ void __launch_bounds__(TPB) tcf_point_insert(const uint64_t *__restrict__ keys,
                                                        const uint8_t *__restrict__ vals, uint64_t n, TcfGeom G,
                                                        uint8_t *blocks, uint64_t *bk, uint8_t *status,
                                                        DevCounters *ctr)
{
    for (uint64_t i = blockIdx.x * (uint64_t)TPB + threadIdx.x; i < n; i += (uint64_t)gridDim.x * TPB) {
        KeyInfo k = tcf_keyinfo(keys[i], G);
        if (vals) k.t |= vals[i] & G.vmask;
        Blk<F> x;
        x.load_l2(blocks, k.b1);
        int f1 = x.live();
        bool done = false;
        if (f1 < (int)G.tsc) done = point_put<F>(blocks, k.b1, k.t, ctr);  // shortcut (Sec. 4.1)
        if (!done) {
            Blk<F> y;
            y.load_l2(blocks, k.b2);
            x.load_l2(blocks, k.b1);
            uint64_t first = x.live() <= y.live() ? k.b1 : k.b2;
            done = point_put<F>(blocks, first, k.t, ctr) ||
                   point_put<F>(blocks, first == k.b1 ? k.b2 : k.b1, k.t, ctr);
        }
        if (!done) {
            uint64_t e = tcf_entry(k, G.f);
            unsigned long long *p =
                reinterpret_cast<unsigned long long *>(bk + tcf_bucket_of(e, G) * BK_W);
            for (int s = 0; s < (int)BK_W && !done; s++)
                if (atomicCAS(p + s, 0ull, (unsigned long long)e) == 0ull) done = true;
            if (done) atomicAdd(&ctr->backing, 1ull);
        }
        if (!done) {
            if (status) status[i] = FILTER_KEY_FULL;
            atomicAdd(&ctr->failed, 1ull);
            atomicOr(&ctr->status, ST_FULL);
        } else if (status) {
            status[i] = FILTER_KEY_OK;
        }
    }
}

template <int F>
__global__ void __launch_bounds__(TPB) tcf_point_remove(const uint64_t *__restrict__ keys, uint64_t n, TcfGeom G,
                                                        uint8_t *blocks, uint64_t *bk, uint8_t *status,
                                                        DevCounters *ctr)
{
    for (uint64_t i = blockIdx.x * (uint64_t)TPB + threadIdx.x; i < n; i += (uint64_t)gridDim.x * TPB) {
        KeyInfo k = tcf_keyinfo(keys[i], G);
        bool done = point_take<F>(blocks, k.b1, k.t, G.vmask, ctr) || point_take<F>(blocks, k.b2, k.t, G.vmask, ctr);
        if (!done) {
            const uint64_t e = tcf_entry(k, G.f), em = ~(uint64_t)G.vmask;
            unsigned long long *p =
                reinterpret_cast<unsigned long long *>(bk + tcf_bucket_of(e, G) * BK_W);
            for (int s = 0; s < (int)BK_W && !done; s++) {
                const unsigned long long v = __ldcg(p + s);
                if ((v & em) == e && atomicCAS(p + s, v, 0ull) == v) done = true;
            }
            if (done) atomicAdd(&ctr->backing, (unsigned long long)-1ll);
        }
        if (status) status[i] = done ? FILTER_KEY_OK : FILTER_KEY_NOT_FOUND;
    }
}

// fill bytes and backing count from the table image (after import)
template <int F>
__global__ void tcf_refill(TcfGeom G, const uint8_t *blocks, uint8_t *fill)
{
    for (uint64_t b = blockIdx.x * (uint64_t)TPB + threadIdx.x; b < G.nb; b += (uint64_t)gridDim.x * TPB) {
        Blk<F> x;
        x.load(blocks, b);
        fill[b] = (uint8_t)x.nonzero();
    }
}

__global__ void tcf_count_backing(TcfGeom G, const uint64_t *bk, DevCounters *ctr)
{
    unsigned long long c = 0;
    for (uint64_t j = blockIdx.x * (uint64_t)TPB + threadIdx.x; j < G.nbk * BK_W; j += (uint64_t)gridDim.x * TPB)
        c += bk[j] != 0;
    if (c) atomicAdd(&ctr->backing, c);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
int tcf_setup(filter *F, uint64_t &table_bytes, uint64_t &scratch_bytes, bool plan_only)
{
    const filter_config &c = F->cfg;
    if (c.tag_bits != 8 && c.tag_bits != 12 && c.tag_bits != 16) return FILTER_ERR_ARG;
    if (c.value_bits > c.tag_bits / 2 || c.value_bits > 7) return FILTER_ERR_ARG;
    if (c.mode != FILTER_MODE_BULK && c.mode != FILTER_MODE_POINT) return FILTER_ERR_ARG;
    const uint32_t B = c.block_slots ? c.block_slots : 256 / c.tag_bits;
    TcfState &T = F->tcf;
    T.G.f = c.tag_bits;
    T.G.B = B;
    if (tcf_custom(T.G) && (!tcf_geom_supported(c.tag_bits, B) || c.mode != FILTER_MODE_BULK || c.value_bits))
        return FILTER_ERR_ARG;
    // nb: the largest power of two with nb B <= 2^log2_slots
    uint32_t lb = 0;
    while ((1ull << lb) < B) lb++;  // ceil(log2 B)
    if (c.log2_slots < lb + 1 || c.log2_slots > lb + 32) return FILTER_ERR_ARG;
    T.mode = c.mode;
    T.G.bbytes = (c.tag_bits * B + 255) / 256 * 32;
    T.G.tsc = 3 * B / 4;
    T.G.tmask = (1u << (c.tag_bits - c.value_bits)) - 1u;
    T.G.vbits = c.value_bits;
    T.G.vmask = (1u << c.value_bits) - 1u;
    T.G.nb = 1ull << (c.log2_slots - lb);
    T.G.seed = c.hash_seed;
    const uint64_t N = T.G.nb * B;
    uint64_t cap = (N + 99) / 100;
    T.G.nbk = (cap + BK_W - 1) / BK_W;
    if (T.G.nbk < 8) T.G.nbk = 8;
    const uint64_t M = c.max_batch ? c.max_batch : 1;
    if (M > 0xffffffffull) return FILTER_ERR_ARG;
    const uint64_t groups = (T.G.nb > T.G.nbk ? T.G.nb : T.G.nbk) + 1;
    // every buffer is listed once: the same list sizes the arena (plan) and
    // carves it (allocation); the table comes first
    uint64_t bytes = 0;
    Arena &A = F->arena;
    auto piece = [&](auto *&ptr, uint64_t count) {
        using T_ = typename std::remove_reference<decltype(*ptr)>::type;
        const uint64_t b = (count * sizeof(T_) + 255) & ~255ull;
        bytes += b;
        if (!plan_only) ptr = A.take<T_>(count);
    };
    piece(T.blocks, T.G.nb * T.G.bbytes);
    piece(T.bk, T.G.nbk * BK_W);
    piece(T.fill, T.G.nb);
    table_bytes = bytes;
    piece(T.cnt, groups);
    piece(T.off, groups);
    piece(T.rec, M);
    piece(T.pend0, M);
    piece(T.pend1, M);
    piece(T.pend2, M);
    piece(T.tlist, M);
    piece(T.tcount, (uint64_t)sm_count() * 8);
    piece(T.dlist, M);
    piece(T.seg, M);
    piece(T.tcur, tt_counter_words(T.G.nb));
    piece(T.pb, M);
    piece(T.pbi, M);
    piece(F->scan_tmp, scan_tmp_words(groups));
    scratch_bytes = bytes - table_bytes;
    return FILTER_OK;
}

int tcf_clear(filter *F, cudaStream_t st)
{
    TcfState &T = F->tcf;
    const uint64_t groups = (T.G.nb > T.G.nbk ? T.G.nb : T.G.nbk) + 1;
    GF_CUDA(cudaMemsetAsync(T.blocks, 0, T.G.nb * T.G.bbytes, st));
    GF_CUDA(cudaMemsetAsync(T.bk, 0, T.G.nbk * BK_W * 8, st));
    GF_CUDA(cudaMemsetAsync(T.fill, 0, T.G.nb, st));
    GF_CUDA(cudaMemsetAsync(T.cnt, 0, groups * 4, st));
    GF_CUDA(cudaMemsetAsync(T.tcur, 0, tt_counter_words(T.G.nb) * 4, st));
    GF_CUDA(cudaMemsetAsync(F->ctr, 0, sizeof(DevCounters), st));
    return FILTER_OK;
}

// Everything one bulk call touches: a filter's own table, or for a group the
// concatenated arrays of all members (G.nb and G.nbk are then the totals)
// with the keys prepared per member.
struct TcfBulk {
    TcfGeom G;
    uint8_t *blocks;
    uint64_t *bk;
    uint8_t *fill;
    uint32_t *cnt, *off;
    uint64_t *rec;
    uint32_t *pend0;
    uint64_t *pend1;
    uint32_t *pend2;
    uint32_t *tlist, *tcount, *dlist;
    uint64_t *seg;
    uint64_t max_n;  // entries of every per-key scratch list (max_batch)
    uint32_t tile_target;  // tiled path: expected candidates per tile
    uint32_t *tcur;  // tiled phases: tile counts and cursors
    uint64_t *pb;    // tiled phases: the second pending list
    uint32_t *pbi;
    uint64_t *scan_tmp;
    DevCounters *ctr;
    TcfPrep prep;
};

static TcfBulk bulk_of(const TcfState &T, uint64_t *scan_tmp, DevCounters *ctr, const TcfPrep &prep, uint64_t max_n,
                       const filter_tuning &tune)
{
    TcfBulk W;
    W.max_n = max_n;
    W.tile_target = tcf_tile_target(tune);
    W.G = T.G;
    W.blocks = T.blocks;
    W.bk = T.bk;
    W.fill = T.fill;
    W.cnt = T.cnt;
    W.off = T.off;
    W.rec = T.rec;
    W.pend0 = T.pend0;
    W.pend1 = T.pend1;
    W.pend2 = T.pend2;
    W.tlist = T.tlist;
    W.tcount = T.tcount;
    W.dlist = T.dlist;
    W.seg = T.seg;
    W.tcur = T.tcur;
    W.pb = T.pb;
    W.pbi = T.pbi;
    W.scan_tmp = scan_tmp;
    W.ctr = ctr;
    W.prep = prep;
    return W;
}

// CTAs of the grouping launches of a phase (the same for histogram and
// segment allocation, whose chunks must agree)
static int group_grid(uint64_t n) { return grid_for(n, TPB, 8); }

// Groups one phase's candidates by destination. The first phase of a call
// (all keys, most blocks hit) is dense: per-destination counts, an exclusive
// scan over all destinations, then the scatter. Later phases see few
// candidates and are sparse: only the touched destinations get a segment and
// a list entry (slot: the phase's counters), so their per-destination kernel
// visits those alone. `recI` (bucket phases) receives the batch indices.
template <int SRC, int DST>
static PhaseDst group_phase(const TcfBulk &T, const uint64_t *keys, uint64_t n, const void *pend,
                            const unsigned *npend, int slot, uint32_t *recI, cudaStream_t st)
{
    const TcfGeom G = T.G;
    const int gk = group_grid(n);
    constexpr bool SPARSE = SRC != SRC_KEYS;
    const uint64_t ndst = (DST == DST_BUCKET ? G.nbk : G.nb);
    PhaseDst P{nullptr, nullptr, nullptr, nullptr};
    {
        gf::TraceScope ts_(SPARSE ? "tcf_group_hist_sparse" : "tcf_group_hist", n, st, SPARSE);
        tcf_group_hist<SRC, DST, SPARSE><<<gk, TPB, 0, st>>>(keys, T.prep, n, pend, npend, G, T.fill, T.cnt, T.tlist,
                                                             T.tcount, ts_.units());
    }
    if (SPARSE) {
        gf::TraceScope ts_("tcf_alloc", 0, st, true);
        tcf_alloc<<<gk, TPB, 0, st>>>(npend, n, T.tlist, T.tcount, T.cnt, T.off, T.dlist, T.seg, &T.ctr->cursor[slot],
                                      &T.ctr->touched[slot], ts_.units());
        P.dlist = T.dlist;
        P.seg = T.seg;
        P.nlist = &T.ctr->touched[slot];
    } else {
        exclusive_scan_u32(T.cnt, T.off, ndst + 1, T.scan_tmp, T.ctr, st);
        P.off = T.off;
    }
    {
        gf::TraceScope ts_(SPARSE ? "tcf_group_scatter_sparse" : "tcf_group_scatter", n, st, SPARSE);
        tcf_group_scatter<SRC, DST><<<gk, TPB, 0, st>>>(keys, T.prep, n, pend, npend, G, T.fill, T.cnt, T.off, T.rec,
                                                        recI, ts_.units());
    }
    return P;
}

// per-destination grid: dense phases visit every destination, sparse ones at
// most one per candidate
static int dst_grid(const PhaseDst &P, uint64_t n, uint64_t ndst)
{
    return grid_for(P.dlist ? (n < ndst ? n : ndst) : ndst, TPB, 8);
}

// ---------------------------------------------------------------------------
// Other block geometries (Sec. 4.1: blocks sized up to a cache line and
// beyond; Sec. 4.2: the bulk TCF's 128-slot blocks; Sec. 4: 12-bit tags that
// straddle word boundaries). A block is B slots of F bits packed
// little-endian into whole 32-byte sectors (gf_packed.cuh); the phases and
// their grouping are the ones above, only the per-block steps and the query
// read and write packed slots. One thread per block, as in the 32-byte path;
// the per-block candidate and tag lists live in local memory.
// ---------------------------------------------------------------------------
template <int F, int B>
struct GBlk : Packed<F, B> {
    using Packed<F, B>::w;
    static constexpr int WORDS = Packed<F, B>::WORDS;
    static constexpr int BYTES = WORDS * 4;
    static_assert(BYTES % 32 == 0, "whole sectors");

    __device__ __forceinline__ void load(const uint8_t *blocks, uint64_t b, bool ro)
    {
        const uint4 *p = reinterpret_cast<const uint4 *>(blocks + b * BYTES);
#pragma unroll
        for (int k = 0; k < WORDS / 4; k++) {
            const uint4 v = ro ? __ldg(p + k) : p[k];
            w[4 * k] = v.x;
            w[4 * k + 1] = v.y;
            w[4 * k + 2] = v.z;
            w[4 * k + 3] = v.w;
        }
    }
    __device__ __forceinline__ void store(uint8_t *blocks, uint64_t b) const
    {
        uint4 *p = reinterpret_cast<uint4 *>(blocks + b * BYTES);
#pragma unroll
        for (int k = 0; k < WORDS / 4; k++) p[k] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
    }
    // some slot holds tag t (t >= 2; the bits past the last slot are 0)
    __device__ __forceinline__ bool has(uint32_t t) const
    {
        if constexpr (F == 16 || F == 8) {
            const uint32_t tt = F == 16 ? (t | (t << 16)) : t * 0x01010101u;
            uint32_t m = 0;
#pragma unroll
            for (int k = 0; k < WORDS; k++) m |= F == 16 ? __vcmpeq2(w[k], tt) : __vcmpeq4(w[k], tt);
            return m != 0;
        } else {
            for (int s = 0; s < B; s++)
                if (this->get(s) == t) return true;
            return false;
        }
    }
};

template <int F, int B>
__global__ void __launch_bounds__(TPB) tcf_gblock_insert(TcfGeom G, uint8_t *blocks, uint8_t *fill, PhaseDst P,
                                                         const uint64_t *__restrict__ rec, int phase, uint32_t cap,
                                                         uint32_t *pend32, uint64_t *pend64, unsigned *npend,
                                                         unsigned long long *units)
{
    const uint64_t nd = phase_count(P, G.nb);
    if (P.dlist) note_units(units, nd);  // units: blocks with candidates
    const uint64_t stride = (uint64_t)gridDim.x * TPB;
    for (uint64_t j0 = blockIdx.x * (uint64_t)TPB + (threadIdx.x & ~31u); j0 < nd; j0 += stride) {
        const uint64_t j = j0 + (threadIdx.x & 31);
        uint32_t s = 0, e = 0, k = 0;
        uint64_t b = 0, thr = 0;  // records <= thr are accepted
        if (j < nd) {
            b = phase_dst(P, j, s, e);
            if (s != e) {
                const uint32_t f0 = fill[b];
                k = cap > f0 ? min(e - s, cap - f0) : 0u;
                if (k > 0) {
                    // the k smallest (tag, index) candidates, merged into the sorted block
                    uint64_t a[B];
                    int have = 0;
                    for (uint32_t q = s; q < e; q++) have = topk_push(a, have, (int)k, rec[q]);
                    thr = a[k - 1];
                    uint32_t nv[B];
                    for (uint32_t q = 0; q < k; q++) nv[q] = (uint32_t)(a[q] >> 32);
                    GBlk<F, B> blk;
                    blk.load(blocks, b, false);
                    blk.merge_sorted((int)f0, nv, (int)k);
                    blk.store(blocks, b);
                    fill[b] = (uint8_t)(f0 + k);
                }
            }
        }
        const uint32_t nrej = (e - s) - k;
        uint32_t slot = warp_reserve(npend, nrej);
        if (nrej == 0) continue;
        for (uint32_t q = s; q < e; q++) {
            const uint64_t r = rec[q];
            if (k > 0 && r <= thr) continue;
            const uint32_t i = (uint32_t)r;
            if (phase == 1) pend64[slot++] = ((b ^ tcf_g((uint32_t)(r >> 32), G.nb)) << 32) | i;  // the other block
            else pend32[slot++] = i;
        }
    }
}

// per distinct stored tag, the smallest candidates with that tag remove one copy each
template <int F, int B>
__global__ void __launch_bounds__(TPB) tcf_gblock_remove(TcfGeom G, uint8_t *blocks, uint8_t *fill, PhaseDst P,
                                                         const uint64_t *__restrict__ rec, uint32_t *pend32,
                                                         unsigned *npend, unsigned long long *units)
{
    const uint64_t nd = phase_count(P, G.nb);
    if (P.dlist) note_units(units, nd);
    const uint64_t stride = (uint64_t)gridDim.x * TPB;
    for (uint64_t j0 = blockIdx.x * (uint64_t)TPB + (threadIdx.x & ~31u); j0 < nd; j0 += stride) {
        const uint64_t j = j0 + (threadIdx.x & 31);
        uint32_t s = 0, e = 0, removed = 0;
        uint32_t dt[B], dc[B], used[B];
        uint64_t thr[B];
        int ndt = 0;
        if (j < nd) {
            const uint64_t b = phase_dst(P, j, s, e);
            if (s != e) {
                const uint32_t f0 = fill[b];
                GBlk<F, B> blk;
                blk.load(blocks, b, false);
                for (int p = 0; p < (int)f0; p++) {  // copies of a tag are adjacent
                    const uint32_t t = blk.get(p);
                    if (ndt > 0 && dt[ndt - 1] == t) {
                        dc[ndt - 1]++;
                    } else {
                        dt[ndt] = t;
                        dc[ndt] = 1;
                        ndt++;
                    }
                }
                for (int d = 0; d < ndt; d++) {
                    uint64_t a[B];
                    int have = 0;
                    const uint64_t lo = (uint64_t)dt[d] << 32, hi = lo | 0xffffffffull;
                    for (uint32_t q = s; q < e; q++) {
                        const uint64_t r = rec[q];
                        if (r >= lo && r <= hi) have = topk_push(a, have, (int)dc[d], r);
                    }
                    used[d] = (uint32_t)have;
                    thr[d] = have ? a[have - 1] : 0;
                    removed += (uint32_t)have;
                }
                if (removed) {
                    GBlk<F, B> out;
                    out.clear();
                    int o = 0;
                    for (int d = 0; d < ndt; d++)
                        for (uint32_t c = used[d]; c < dc[d]; c++) out.set(o++, dt[d]);
                    out.store(blocks, b);
                    fill[b] = (uint8_t)(f0 - removed);
                }
            }
        }
        const uint32_t nunm = (e - s) - removed;  // unmatched candidates go on
        uint32_t slot = warp_reserve(npend, nunm);
        if (nunm == 0) continue;
        for (uint32_t q = s; q < e; q++) {
            const uint64_t r = rec[q];
            const uint32_t t = (uint32_t)(r >> 32);
            bool matched = false;
            for (int d = 0; d < ndt; d++)
                if (dt[d] == t && used[d] > 0 && r <= thr[d]) matched = true;
            if (!matched) pend32[slot++] = (uint32_t)r;
        }
    }
}

template <int F, int B>
__global__ void __launch_bounds__(TPB) tcf_gquery_kernel(const uint64_t *__restrict__ keys, uint64_t n, TcfGeom G,
                                                         const uint8_t *__restrict__ blocks,
                                                         const uint64_t *__restrict__ bk, const DevCounters *ctr,
                                                         uint8_t *__restrict__ out)
{
    const bool backing = ctr->backing != 0;
    for (uint64_t i = blockIdx.x * (uint64_t)TPB + threadIdx.x; i < n; i += (uint64_t)gridDim.x * TPB) {
        const KeyInfo k = tcf_keyinfo(__ldcs(keys + i), G);
        GBlk<F, B> x;
        x.load(blocks, k.b1, true);
        bool hit = x.has(k.t);
        if (!hit) {
            x.load(blocks, k.b2, true);
            hit = x.has(k.t);
        }
        if (!hit && backing) {
            const uint64_t e = tcf_entry(k, G.f);
            const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(bk + tcf_bucket_of(e, G) * BK_W);
#pragma unroll
            for (int s = 0; s < 4; s++) {
                const ulonglong2 v = __ldg(p + s);
                hit |= (v.x == e) | (v.y == e);
            }
        }
        __stcs(out + i, (uint8_t)(hit ? 1 : 0));
    }
}

// The per-block counting-sort path: each phase groups its candidates by
// destination block (counts, scan, scatter) and one thread per block takes
// its step. Its scratch (a counter and an offset per block, a record per
// candidate) stays in the L2 for moderate tables and batches.
template <int F, int GB = 0>  // GB: slots of a packed block of another geometry
static void tcf_bulk_insert(const TcfBulk &T, const uint64_t *keys, uint64_t n, uint8_t *status, cudaStream_t st)
{
    const TcfGeom G = T.G;
    DevCounters *ctr = T.ctr;
    unsigned *np = ctr->pend;
    cudaMemsetAsync(np, 0, sizeof(ctr->pend), st);
    cudaMemsetAsync(ctr->touched, 0, sizeof(ctr->touched) + sizeof(ctr->cursor), st);  // adjacent fields
    // A: shortcut into b1
    PhaseDst P = group_phase<SRC_KEYS, DST_B1>(T, keys, n, nullptr, nullptr, 0, nullptr, st);
    {
        gf::TraceScope ts_("tcf_block_insert", 0, st, true);
        if constexpr (GB == 0)
            tcf_block_insert<F><<<dst_grid(P, n, G.nb), TPB, 0, st>>>(G, T.blocks, T.fill, P, T.rec, 0, G.tsc, T.pend0,
                                                                       nullptr, &np[0], T.prep, ts_.units());
        else
            tcf_gblock_insert<F, GB><<<dst_grid(P, n, G.nb), TPB, 0, st>>>(G, T.blocks, T.fill, P, T.rec, 0, G.tsc,
                                                                           T.pend0, nullptr, &np[0], ts_.units());
    }
    // B: the less full of b1, b2 under the post-A fills
    P = group_phase<SRC_PEND_U32, DST_TARGET>(T, keys, n, T.pend0, &np[0], 1, nullptr, st);
    {
        gf::TraceScope ts_("tcf_block_insert_sparse", 0, st, true);
        if constexpr (GB == 0)
            tcf_block_insert<F><<<dst_grid(P, n, G.nb), TPB, 0, st>>>(G, T.blocks, T.fill, P, T.rec, 1, G.B, nullptr,
                                                                       T.pend1, &np[1], T.prep, ts_.units());
        else
            tcf_gblock_insert<F, GB><<<dst_grid(P, n, G.nb), TPB, 0, st>>>(G, T.blocks, T.fill, P, T.rec, 1, G.B,
                                                                           nullptr, T.pend1, &np[1], ts_.units());
    }
    // C: the other block
    P = group_phase<SRC_PEND_U64, DST_ALT>(T, keys, n, T.pend1, &np[1], 2, nullptr, st);
    {
        gf::TraceScope ts_("tcf_block_insert_sparse", 0, st, true);
        if constexpr (GB == 0)
            tcf_block_insert<F><<<dst_grid(P, n, G.nb), TPB, 0, st>>>(G, T.blocks, T.fill, P, T.rec, 2, G.B, T.pend2,
                                                                       nullptr, &np[2], T.prep, ts_.units());
        else
            tcf_gblock_insert<F, GB><<<dst_grid(P, n, G.nb), TPB, 0, st>>>(G, T.blocks, T.fill, P, T.rec, 2, G.B,
                                                                           T.pend2, nullptr, &np[2], ts_.units());
    }
    // D: backing buckets
    P = group_phase<SRC_PEND_U32, DST_BUCKET>(T, keys, n, T.pend2, &np[2], 3, T.pend0, st);
    {
        gf::TraceScope ts_("tcf_bucket_insert", 0, st, true);
        tcf_bucket_insert<<<dst_grid(P, n, G.nbk), TPB, 0, st>>>(G, T.bk, P, T.rec, T.pend0, status, ctr, ts_.units());
    }
}

template <int F, int GB = 0>
static void tcf_bulk_remove(const TcfBulk &T, const uint64_t *keys, uint64_t n, uint8_t *status, cudaStream_t st)
{
    const TcfGeom G = T.G;
    DevCounters *ctr = T.ctr;
    unsigned *np = ctr->pend;
    cudaMemsetAsync(np, 0, sizeof(ctr->pend), st);
    cudaMemsetAsync(ctr->touched, 0, sizeof(ctr->touched) + sizeof(ctr->cursor), st);  // adjacent fields
    // 1: primary block
    PhaseDst P = group_phase<SRC_KEYS, DST_B1>(T, keys, n, nullptr, nullptr, 0, nullptr, st);
    {
        gf::TraceScope ts_("tcf_block_remove", 0, st, true);
        if constexpr (GB == 0)
            tcf_block_remove<F><<<dst_grid(P, n, G.nb), TPB, 0, st>>>(G, T.blocks, T.fill, P, T.rec, T.pend0, &np[0],
                                                                       ts_.units());
        else
            tcf_gblock_remove<F, GB><<<dst_grid(P, n, G.nb), TPB, 0, st>>>(G, T.blocks, T.fill, P, T.rec, T.pend0,
                                                                           &np[0], ts_.units());
    }
    // 2: secondary block
    P = group_phase<SRC_PEND_U32, DST_B2>(T, keys, n, T.pend0, &np[0], 1, nullptr, st);
    {
        gf::TraceScope ts_("tcf_block_remove_sparse", 0, st, true);
        if constexpr (GB == 0)
            tcf_block_remove<F><<<dst_grid(P, n, G.nb), TPB, 0, st>>>(G, T.blocks, T.fill, P, T.rec, T.pend2, &np[2],
                                                                       ts_.units());
        else
            tcf_gblock_remove<F, GB><<<dst_grid(P, n, G.nb), TPB, 0, st>>>(G, T.blocks, T.fill, P, T.rec, T.pend2,
                                                                           &np[2], ts_.units());
    }
    // 3: backing bucket; what is left is not found
    P = group_phase<SRC_PEND_U32, DST_BUCKET>(T, keys, n, T.pend2, &np[2], 2, T.pend0, st);
    {
        gf::TraceScope ts_("tcf_bucket_remove", 0, st, true);
        tcf_bucket_remove<<<dst_grid(P, n, G.nbk), TPB, 0, st>>>(G, T.bk, P, T.rec, T.pend0, status, ctr, ts_.units());
    }
}


// the packed geometries (f, B) that have kernels
#define GF_TCF_GEOMS(X) X(16, 8) X(16, 32) X(16, 64) X(16, 128) X(12, 21) X(8, 64)

bool tcf_geom_supported(uint32_t f, uint32_t B)
{
#define GF_GEOM_IS(FF, BB) \
    if (f == FF && B == BB) return true;
    GF_TCF_GEOMS(GF_GEOM_IS)
#undef GF_GEOM_IS
    return false;
}

static void tcf_custom_bulk(const TcfBulk &W, const uint64_t *keys, uint64_t n, uint8_t *status, bool del,
                            cudaStream_t st)
{
#define GF_GEOM_BULK(FF, BB)                                      \
    if (W.G.f == FF && W.G.B == BB) {                             \
        if (del) tcf_bulk_remove<FF, BB>(W, keys, n, status, st); \
        else tcf_bulk_insert<FF, BB>(W, keys, n, status, st);     \
        return;                                                   \
    }
    GF_TCF_GEOMS(GF_GEOM_BULK)
#undef GF_GEOM_BULK
}

// ---------------------------------------------------------------------------
// Tiled phases: host side
// ---------------------------------------------------------------------------
// Tiles of TB blocks, TB the largest power of two in [32, TT_TB_MAX] that
// keeps a tile's expected candidates (n keys spread over nb blocks) at or
// below `target` (at most half of TT_CAP, so that a tile's records fit its
// shared-memory stage with room for the spread); partitioned in one pass up
// to 256 tiles and in two above (at most 256 high bins).
static TtGeom tt_geom(uint64_t nb, uint64_t n, uint32_t target)
{
    TtGeom g;
    g.nb = nb;
    uint32_t tl = 5;
    while ((1u << (tl + 1)) <= TT_TB_MAX && (n << (tl + 1)) <= (uint64_t)target * nb) tl++;
    g.tb_log = tl;
    g.nt = (nb + (1ull << tl) - 1) >> tl;
    uint32_t lg = 0;
    while ((1ull << lg) < g.nt) lg++;
    g.lo = g.nt <= 256 ? 0 : ((lg + 1) / 2 > lg - 8 ? (lg + 1) / 2 : lg - 8);
    g.nh = g.lo ? (g.nt + (1ull << g.lo) - 1) >> g.lo : g.nt;
    return g;
}

template <int F, int OP, int NEXT>
static void tt_tile_launch(const TcfBulk &T, const TtGeom &tg, const unsigned *n_dev, const uint64_t *rec,
                           const uint32_t *ridx, uint64_t *gstage, uint32_t cap, uint64_t *orec, uint32_t *oidx,
                           unsigned *nout, const char *name, cudaStream_t st)
{
    const size_t TB = (size_t)1 << tg.tb_log;
    const size_t smem = TB * 32 + TT_CAP * 8 + (TB + 1) * 4 + TB;
    cudaFuncSetAttribute(tt_tile<F, OP, NEXT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(TT_TB_MAX * 32 + TT_CAP * 8 + (TT_TB_MAX + 1) * 4 + TT_TB_MAX));
    const uint64_t grid = tg.nt < (uint64_t)sm_count() * 8 ? tg.nt : (uint64_t)sm_count() * 8;
    gf::TraceScope ts_(name, 0, st, true);
    tt_tile<F, OP, NEXT><<<(unsigned)grid, TT_TPB, smem, st>>>(T.G, T.prep, T.blocks, T.fill, tg, T.off, rec, ridx,
                                                               gstage, cap, orec, oidx, nout, T.max_n, n_dev, T.tcur,
                                                               &T.ctr->status, ts_.units());
}

// group one phase's candidates by tile: counts (their last CTA scans them
// into T.off and clears the counters), then one or two partition passes;
// returns the buffers holding the grouped records (and the spare pair,
// which the tile kernel may use for a hot tile)
template <int SRC, int RULE>
static void tt_group(const TcfBulk &T, const TtGeom &tg, const TtSrc &src, DevCounters *reset, const uint64_t **grec,
                     const uint32_t **gidx, uint64_t **spare, cudaStream_t st)
{
    const bool keys = SRC == TT_KEYS;
    const int ghist = grid_for(src.n, TT_TPB * 16, 4);
    {
        gf::TraceScope ts_(keys ? "tcf_tile_hist" : "tcf_tile_hist_pend", keys ? src.n : 0, st, !keys);
        tt_hist<SRC, RULE><<<ghist, TT_TPB, tg.nt <= 8192 ? tg.nt * 4 : 0, st>>>(src, T.G, T.prep, T.fill, tg, T.tcur,
                                                                                T.off, reset, ts_.units());
    }
    const int gpart = grid_for((src.n + TT_CH - 1) / TT_CH * TT_TPB, TT_TPB, 6);
    if (tg.lo == 0) {
        gf::TraceScope ts_(keys ? "tcf_tile_part" : "tcf_tile_part_pend", keys ? src.n : 0, st, !keys);
        tt_part<SRC, RULE, 0><<<gpart, TT_TPB, 0, st>>>(src, T.G, T.prep, T.fill, tg, T.off, T.tcur, T.rec, T.tlist,
                                                        ts_.units());
        *grec = T.rec;
        *gidx = T.tlist;
        *spare = T.seg;
        return;
    }
    {
        gf::TraceScope ts_(keys ? "tcf_tile_part" : "tcf_tile_part_pend", keys ? src.n : 0, st, !keys);
        tt_part<SRC, RULE, 1><<<gpart, TT_TPB, 0, st>>>(src, T.G, T.prep, T.fill, tg, T.off, T.tcur, T.rec, T.tlist,
                                                        ts_.units());
    }
    TtSrc s2{nullptr, T.rec, T.tlist, src.n_dev, src.n};
    {
        gf::TraceScope ts_("tcf_tile_part2", 0, st, true);
        tt_part<TT_PEND, TT_SAME, 2><<<gpart, TT_TPB, 0, st>>>(s2, T.G, T.prep, T.fill, tg, T.off, T.tcur, T.seg,
                                                               T.dlist, ts_.units());
    }
    *grec = T.seg;
    *gidx = T.dlist;
    *spare = T.rec;
}

template <int F>
static void tcf_tiled_insert(const TcfBulk &T, const uint64_t *keys, uint64_t n, uint8_t *status, cudaStream_t st)
{
    const TcfGeom G = T.G;
    DevCounters *ctr = T.ctr;
    unsigned *np = ctr->pend;
    const TtGeom tg = tt_geom(G.nb, n, T.tile_target);
    const uint64_t *gr;
    const uint32_t *gi;
    uint64_t *sp;
    // A: shortcut into b1 while fill < 3B/4; rejects keep b1 (the counts'
    // last CTA also clears the call's pending-list lengths)
    tt_group<TT_KEYS, TT_SAME>(T, tg, TtSrc{keys, nullptr, nullptr, nullptr, n}, ctr, &gr, &gi, &sp, st);
    tt_tile_launch<F, 0, TT_NX_SAME>(T, tg, nullptr, gr, gi, sp, G.tsc, T.pend1, T.pend0, &np[0], "tcf_tile_insert", st);
    // B: the less full of b1, b2 under the post-A fills; rejects go to the other block
    tt_group<TT_PEND, TT_TARGET>(T, tg, TtSrc{nullptr, T.pend1, T.pend0, &np[0], n}, nullptr, &gr, &gi, &sp, st);
    tt_tile_launch<F, 0, TT_NX_OTHER>(T, tg, &np[0], gr, gi, sp, G.B, T.pb, T.pbi, &np[1], "tcf_tile_insert", st);
    // C: the other block; rejects go to the backing buckets by index
    tt_group<TT_PEND, TT_SAME>(T, tg, TtSrc{nullptr, T.pb, T.pbi, &np[1], n}, nullptr, &gr, &gi, &sp, st);
    tt_tile_launch<F, 0, TT_NX_IDX>(T, tg, &np[1], gr, gi, sp, G.B, nullptr, T.pend2, &np[2], "tcf_tile_insert", st);
    // D: backing buckets
    PhaseDst P = group_phase<SRC_PEND_U32, DST_BUCKET>(T, keys, n, T.pend2, &np[2], 3, T.pend0, st);
    {
        gf::TraceScope ts_("tcf_bucket_insert", 0, st, true);
        tcf_bucket_insert<<<dst_grid(P, n, G.nbk), TPB, 0, st>>>(G, T.bk, P, T.rec, T.pend0, status, ctr, ts_.units());
    }
}

template <int F>
static void tcf_tiled_remove(const TcfBulk &T, const uint64_t *keys, uint64_t n, uint8_t *status, cudaStream_t st)
{
    const TcfGeom G = T.G;
    DevCounters *ctr = T.ctr;
    unsigned *np = ctr->pend;
    const TtGeom tg = tt_geom(G.nb, n, T.tile_target);
    const uint64_t *gr;
    const uint32_t *gi;
    uint64_t *sp;
    // 1: primary block; misses go on to the secondary block
    tt_group<TT_KEYS, TT_SAME>(T, tg, TtSrc{keys, nullptr, nullptr, nullptr, n}, ctr, &gr, &gi, &sp, st);
    tt_tile_launch<F, 1, TT_NX_OTHER>(T, tg, nullptr, gr, gi, sp, 0, T.pend1, T.pend0, &np[0], "tcf_tile_remove", st);
    // 2: secondary block; misses go to the backing buckets by index
    tt_group<TT_PEND, TT_SAME>(T, tg, TtSrc{nullptr, T.pend1, T.pend0, &np[0], n}, nullptr, &gr, &gi, &sp, st);
    tt_tile_launch<F, 1, TT_NX_IDX>(T, tg, &np[0], gr, gi, sp, 0, nullptr, T.pend2, &np[2], "tcf_tile_remove", st);
    // 3: backing bucket; what is left is not found
    PhaseDst P = group_phase<SRC_PEND_U32, DST_BUCKET>(T, keys, n, T.pend2, &np[2], 2, T.pend0, st);
    {
        gf::TraceScope ts_("tcf_bucket_remove", 0, st, true);
        tcf_bucket_remove<<<dst_grid(P, n, G.nbk), TPB, 0, st>>>(G, T.bk, P, T.rec, T.pend0, status, ctr,
                                                                 ts_.units());
    }
}

int tcf_insert(filter *F, const uint64_t *keys, const uint8_t *vals, uint64_t n, uint8_t *status, cudaStream_t st)
{
    if (n == 0) return FILTER_OK;
    if (status) GF_CUDA(cudaMemsetAsync(status, 0, n, st));
    TcfState &T = F->tcf;
    if (T.mode == FILTER_MODE_POINT) {
        const int g = grid_for(n, TPB, 16);
        {
            gf::TraceScope ts_("tcf_point_insert", n, st);
            if (T.G.f == 16) tcf_point_insert<16><<<g, TPB, 0, st>>>(keys, vals, n, T.G, T.blocks, T.bk, status, F->ctr);
            else tcf_point_insert<8><<<g, TPB, 0, st>>>(keys, vals, n, T.G, T.blocks, T.bk, status, F->ctr);
        }
    } else {
        const TcfBulk W = bulk_of(T, F->scan_tmp, F->ctr, TcfPrep{nullptr, nullptr, nullptr, nullptr, vals}, F->cfg.max_batch,
                                   F->tune);
        const bool tiled = !tcf_custom(T.G) && tcf_tiled(F->tune, T.G.nb, n);
        if (tcf_custom(T.G)) tcf_custom_bulk(W, keys, n, status, false, st);
        else if (T.G.f == 16) tiled ? tcf_tiled_insert<16>(W, keys, n, status, st) : tcf_bulk_insert<16>(W, keys, n, status, st);
        else tiled ? tcf_tiled_insert<8>(W, keys, n, status, st) : tcf_bulk_insert<8>(W, keys, n, status, st);
    }
    GF_CUDA(cudaGetLastError());
    return FILTER_OK;
}

int tcf_remove(filter *F, const uint64_t *keys, uint64_t n, uint8_t *status, cudaStream_t st)
{
    if (n == 0) return FILTER_OK;
    if (status) GF_CUDA(cudaMemsetAsync(status, 0, n, st));
    TcfState &T = F->tcf;
    if (T.mode == FILTER_MODE_POINT) {
        const int g = grid_for(n, TPB, 16);
        {
            gf::TraceScope ts_("tcf_point_remove", n, st);
            if (T.G.f == 16) tcf_point_remove<16><<<g, TPB, 0, st>>>(keys, n, T.G, T.blocks, T.bk, status, F->ctr);
            else tcf_point_remove<8><<<g, TPB, 0, st>>>(keys, n, T.G, T.blocks, T.bk, status, F->ctr);
        }
    } else {
        const TcfBulk W = bulk_of(T, F->scan_tmp, F->ctr, TcfPrep{nullptr, nullptr, nullptr, nullptr}, F->cfg.max_batch, F->tune);
        const bool tiled = !tcf_custom(T.G) && tcf_tiled(F->tune, T.G.nb, n);
        if (tcf_custom(T.G)) tcf_custom_bulk(W, keys, n, status, true, st);
        else if (T.G.f == 16) tiled ? tcf_tiled_remove<16>(W, keys, n, status, st) : tcf_bulk_remove<16>(W, keys, n, status, st);
        else tiled ? tcf_tiled_remove<8>(W, keys, n, status, st) : tcf_bulk_remove<8>(W, keys, n, status, st);
    }
    GF_CUDA(cudaGetLastError());
    return FILTER_OK;
}

int tcf_query(filter *F, const uint64_t *keys, uint64_t n, uint8_t *found, bool values, cudaStream_t st)
{
    if (n == 0) return FILTER_OK;
    TcfState &T = F->tcf;
    const int g = grid_for(n, TPB, 16);
    if (values) {
        gf::TraceScope ts_("tcf_query_values_kernel", n, st);
        if (T.G.f == 16) tcf_query_kernel<16, true><<<g, TPB, 0, st>>>(keys, n, T.G, T.blocks, T.bk, F->ctr, found);
        else tcf_query_kernel<8, true><<<g, TPB, 0, st>>>(keys, n, T.G, T.blocks, T.bk, F->ctr, found);
    } else if (tcf_custom(T.G)) {
        gf::TraceScope ts_("tcf_gquery_kernel", n, st);
#define GF_GEOM_QUERY(FF, BB)                                                                                   \
    if (T.G.f == FF && T.G.B == BB) tcf_gquery_kernel<FF, BB><<<g, TPB, 0, st>>>(keys, n, T.G, T.blocks, T.bk, \
                                                                                F->ctr, found);
        GF_TCF_GEOMS(GF_GEOM_QUERY)
#undef GF_GEOM_QUERY
    } else {
        gf::TraceScope ts_("tcf_query_kernel", n, st);
        if (T.G.f == 16) tcf_query_kernel<16, false><<<g, TPB, 0, st>>>(keys, n, T.G, T.blocks, T.bk, F->ctr, found);
        else tcf_query_kernel<8, false><<<g, TPB, 0, st>>>(keys, n, T.G, T.blocks, T.bk, F->ctr, found);
    }
    GF_CUDA(cudaGetLastError());
    return FILTER_OK;
}

uint64_t tcf_image_bytes(const filter *F) { return F->tcf.G.nb * F->tcf.G.bbytes + F->tcf.G.nbk * BK_W * 8; }

int tcf_copy_image(filter *F, void *host, bool to_host, cudaStream_t st)
{
    TcfState &T = F->tcf;
    char *h = static_cast<char *>(host);
    const uint64_t nbB = T.G.nb * T.G.bbytes, bkB = T.G.nbk * BK_W * 8;
    if (to_host) {
        GF_CUDA(cudaMemcpyAsync(h, T.blocks, nbB, cudaMemcpyDeviceToHost, st));
        GF_CUDA(cudaMemcpyAsync(h + nbB, T.bk, bkB, cudaMemcpyDeviceToHost, st));
    } else {
        GF_CUDA(cudaMemcpyAsync(T.blocks, h, nbB, cudaMemcpyHostToDevice, st));
        GF_CUDA(cudaMemcpyAsync(T.bk, h + nbB, bkB, cudaMemcpyHostToDevice, st));
        const int g = grid_for(T.G.nb, TPB, 8);
        {
            gf::TraceScope ts_("tcf_refill", T.G.nb, st);
            if (T.G.f == 16) tcf_refill<16><<<g, TPB, 0, st>>>(T.G, T.blocks, T.fill);
            else tcf_refill<8><<<g, TPB, 0, st>>>(T.G, T.blocks, T.fill);
        }
        GF_CUDA(cudaMemsetAsync(&F->ctr->backing, 0, 8, st));
        {
            gf::TraceScope ts_("tcf_count_backing", T.G.nbk * BK_W, st);
            tcf_count_backing<<<grid_for(T.G.nbk * BK_W, TPB, 4), TPB, 0, st>>>(T.G, T.bk, F->ctr);
        }
    }
    GF_CUDA(cudaStreamSynchronize(st));
    return FILTER_OK;
}

// ---------------------------------------------------------------------------
// Filter groups: every member's keys in one set of launches. A member's keys
// are hashed with its own geometry, then every phase runs over the
// concatenated blocks and buckets of all members. Candidates of one block
// all belong to its member and keep their batch order, so each member ends
// up exactly as a standalone filter given the same keys.
// ---------------------------------------------------------------------------
__device__ __forceinline__ TcfGeom member_geom(const TcfMember &M, uint32_t f)
{
    TcfGeom G;
    G.nb = M.nb;
    G.nbk = M.nbk;
    G.seed = M.seed;
    G.f = f;
    G.B = 256 / f;
    G.tsc = 3 * G.B / 4;
    G.tmask = (1u << f) - 1u;
    return G;
}

__global__ void __launch_bounds__(TPB) tcf_group_prep(const uint64_t *__restrict__ keys, uint64_t n,
                                                      const uint64_t *__restrict__ off, uint32_t nmem,
                                                      const TcfMember *__restrict__ mem, uint32_t f, TcfPrep out)
{
    MemberCursor c(off, nmem, n);
    uint32_t cm = 0xffffffffu;
    TcfMember M;
    TcfGeom G;
    for (; c.valid(); c.next(off)) {
        if (c.m != cm) {
            cm = c.m;
            M = mem[cm];
            G = member_geom(M, f);
        }
        const KeyInfo k = tcf_keyinfo(__ldcs(keys + c.i), G);
        const uint64_t e = tcf_entry(k, f);
        out.bt[c.i] = ((M.block0 + k.b1) << 32) | k.t;
        out.b2[c.i] = (uint32_t)(M.block0 + k.b2);
        out.bucket[c.i] = (uint32_t)(M.bucket0 + tcf_bucket(e, M.nbk));
        out.e[c.i] = e;
    }
}

template <int F>
__global__ void __launch_bounds__(TPB) tcf_group_query_kernel(const uint64_t *__restrict__ keys, uint64_t n,
                                                              const uint64_t *__restrict__ off, uint32_t nmem,
                                                              const TcfMember *__restrict__ mem,
                                                              const uint8_t *__restrict__ blocks,
                                                              const uint64_t *__restrict__ bk,
                                                              const DevCounters *ctr, uint8_t *__restrict__ out)
{
    const bool backing = ctr->backing != 0;
    MemberCursor c(off, nmem, n);
    uint32_t cm = 0xffffffffu;
    TcfMember M;
    TcfGeom G;
    for (; c.valid(); c.next(off)) {
        if (c.m != cm) {
            cm = c.m;
            M = mem[cm];
            G = member_geom(M, F);
        }
        const KeyInfo k = tcf_keyinfo(__ldcs(keys + c.i), G);
        Blk<F> x, y;
        x.load_ro(blocks, M.block0 + k.b1);
        y.load_ro(blocks, M.block0 + k.b2);
        bool hit = x.has(k.t, 0xffffffffu) || y.has(k.t, 0xffffffffu);  // group members carry no values
        if (!hit && backing) {
            const uint64_t e = tcf_entry(k, F);
            const ulonglong2 *p =
                reinterpret_cast<const ulonglong2 *>(bk + (M.bucket0 + tcf_bucket(e, M.nbk)) * BK_W);
#pragma unroll
            for (int s = 0; s < 4; s++) {
                ulonglong2 v = __ldg(p + s);
                hit |= (v.x == e) | (v.y == e);
            }
        }
        __stcs(out + c.i, (uint8_t)(hit ? 1 : 0));
    }
}

int tcf_group_setup(filter_group *GR, const filter_config *cfgs, uint64_t &bytes_out, bool plan_only)
{
    const uint32_t n = GR->n;
    const uint32_t f = cfgs[0].tag_bits;
    const uint64_t M = GR->max_total ? GR->max_total : 1;
    if (M > 0xffffffffull) return FILTER_ERR_ARG;
    std::vector<TcfMember> tm(n);
    uint64_t nb_tot = 0, nbk_tot = 0;
    for (uint32_t m = 0; m < n; m++) {
        const filter_config &c = cfgs[m];
        if (c.kind != FILTER_TCF || c.tag_bits != f || c.mode != FILTER_MODE_BULK || c.value_bits || c.block_slots ||
            (f != 8 && f != 16))
            return FILTER_ERR_ARG;  // members: 32-byte blocks of 8- or 16-bit tags
        filter V;
        V.cfg = c;
        V.cfg.max_batch = M;
        uint64_t tb = 0, sb = 0;
        int rc = tcf_setup(&V, tb, sb, true);  // geometry only
        if (rc != FILTER_OK) return rc;
        tm[m].nb = V.tcf.G.nb;
        tm[m].nbk = V.tcf.G.nbk;
        tm[m].seed = V.tcf.G.seed;
        tm[m].block0 = nb_tot;
        tm[m].bucket0 = nbk_tot;
        nb_tot += V.tcf.G.nb;
        nbk_tot += V.tcf.G.nbk;
    }
    if (nb_tot > 0xffffffffull || nbk_tot > 0xffffffffull) return FILTER_ERR_ARG;  // 32-bit indices
    TcfState &T = GR->tcf;
    T.mode = FILTER_MODE_BULK;
    T.G.f = f;
    T.G.B = 256 / f;
    T.G.tsc = 3 * T.G.B / 4;
    T.G.tmask = (1u << f) - 1u;
    T.G.nb = nb_tot;
    T.G.nbk = nbk_tot;
    T.G.seed = 0;
    const uint64_t groups = (nb_tot > nbk_tot ? nb_tot : nbk_tot) + 1;
    uint64_t bytes = 0;
    Arena &A = GR->arena;
    auto piece = [&](auto *&ptr, uint64_t count) {
        using T_ = typename std::remove_reference<decltype(*ptr)>::type;
        bytes += (count * sizeof(T_) + 255) & ~255ull;
        if (!plan_only) ptr = A.take<T_>(count);
    };
    piece(T.blocks, nb_tot * 32);
    piece(T.bk, nbk_tot * BK_W);
    piece(T.fill, nb_tot);
    piece(T.cnt, groups);
    piece(T.off, groups);
    piece(T.rec, M);
    piece(T.pend0, M);
    piece(T.pend1, M);
    piece(T.pend2, M);
    piece(T.tlist, M);
    piece(T.tcount, (uint64_t)sm_count() * 8);
    piece(T.dlist, M);
    piece(T.seg, M);
    piece(T.tcur, tt_counter_words(nb_tot));
    piece(T.pb, M);
    piece(T.pbi, M);
    piece(GR->prep.bt, M);
    piece(GR->prep.b2, M);
    piece(GR->prep.bucket, M);
    piece(GR->prep.e, M);
    piece(GR->d_tmem, (uint64_t)n);
    piece(GR->scan_tmp, scan_tmp_words(groups));
    bytes_out = bytes;
    if (plan_only) return FILTER_OK;
    if (!T.blocks || !T.bk || !T.fill || !T.cnt || !T.off || !T.rec || !T.pend0 || !T.pend1 || !T.pend2 ||
        !T.tlist || !T.tcount || !T.dlist || !T.seg || !T.tcur || !T.pb || !T.pbi || !GR->prep.bt || !GR->prep.b2 || !GR->prep.bucket ||
        !GR->prep.e || !GR->d_tmem || !GR->scan_tmp)
        return FILTER_ERR_INTERNAL;
    GF_CUDA(cudaMemcpy(GR->d_tmem, tm.data(), n * sizeof(TcfMember), cudaMemcpyHostToDevice));
    // host views of the members: their slices of the group's arrays
    for (uint32_t m = 0; m < n; m++) {
        filter &V = GR->members[m];
        V.cfg = cfgs[m];
        V.cfg.max_batch = M;
        uint64_t tb = 0, sb = 0;
        tcf_setup(&V, tb, sb, true);
        TcfState &S = V.tcf;
        S.blocks = T.blocks + tm[m].block0 * 32;
        S.bk = T.bk + tm[m].bucket0 * BK_W;
        S.fill = T.fill + tm[m].block0;
        S.cnt = T.cnt;
        S.off = T.off;
        S.rec = T.rec;
        S.pend0 = T.pend0;
        S.pend1 = T.pend1;
        S.pend2 = T.pend2;
        S.tlist = T.tlist;
        S.tcount = T.tcount;
        S.dlist = T.dlist;
        S.seg = T.seg;
        S.tcur = T.tcur;
        S.pb = T.pb;
        S.pbi = T.pbi;
        V.ctr = GR->ctr;
        V.scan_tmp = GR->scan_tmp;
        V.arena.base = GR->arena.base;  // marks the view valid; the group owns the memory
        V.device = GR->device;
    }
    return FILTER_OK;
}

int tcf_group_clear(filter_group *GR, cudaStream_t st)
{
    TcfState &T = GR->tcf;
    const uint64_t groups = (T.G.nb > T.G.nbk ? T.G.nb : T.G.nbk) + 1;
    GF_CUDA(cudaMemsetAsync(T.blocks, 0, T.G.nb * T.G.bbytes, st));
    GF_CUDA(cudaMemsetAsync(T.bk, 0, T.G.nbk * BK_W * 8, st));
    GF_CUDA(cudaMemsetAsync(T.fill, 0, T.G.nb, st));
    GF_CUDA(cudaMemsetAsync(T.cnt, 0, groups * 4, st));
    GF_CUDA(cudaMemsetAsync(T.tcur, 0, tt_counter_words(T.G.nb) * 4, st));
    GF_CUDA(cudaMemsetAsync(GR->ctr, 0, sizeof(DevCounters), st));
    return FILTER_OK;
}

int tcf_group_op(filter_group *GR, int op, const uint64_t *off, const uint64_t *keys, uint64_t n, uint8_t *out,
                 cudaStream_t st)
{
    if (n == 0) return FILTER_OK;
    TcfState &T = GR->tcf;
    if (op == GROUP_QUERY) {
        const int g = grid_for(n, TPB, 16);
        gf::TraceScope ts_("tcf_group_query_kernel", n, st);
        if (T.G.f == 16)
            tcf_group_query_kernel<16><<<g, TPB, 0, st>>>(keys, n, off, GR->n, GR->d_tmem, T.blocks, T.bk, GR->ctr, out);
        else
            tcf_group_query_kernel<8><<<g, TPB, 0, st>>>(keys, n, off, GR->n, GR->d_tmem, T.blocks, T.bk, GR->ctr, out);
        GF_CUDA(cudaGetLastError());
        return FILTER_OK;
    }
    if (out) GF_CUDA(cudaMemsetAsync(out, 0, n, st));
    {
        gf::TraceScope ts_("tcf_group_prep", n, st);
        tcf_group_prep<<<grid_for(n, TPB, 8), TPB, 0, st>>>(keys, n, off, GR->n, GR->d_tmem, T.G.f, GR->prep);
    }
    const TcfBulk W = bulk_of(T, GR->scan_tmp, GR->ctr, GR->prep, GR->max_total, GR->tune);
    const bool tiled = tcf_tiled(GR->tune, T.G.nb, n);
    if (op == GROUP_INSERT) {
        if (T.G.f == 16) tiled ? tcf_tiled_insert<16>(W, nullptr, n, out, st) : tcf_bulk_insert<16>(W, nullptr, n, out, st);
        else tiled ? tcf_tiled_insert<8>(W, nullptr, n, out, st) : tcf_bulk_insert<8>(W, nullptr, n, out, st);
    } else {
        if (T.G.f == 16) tiled ? tcf_tiled_remove<16>(W, nullptr, n, out, st) : tcf_bulk_remove<16>(W, nullptr, n, out, st);
        else tiled ? tcf_tiled_remove<8>(W, nullptr, n, out, st) : tcf_bulk_remove<8>(W, nullptr, n, out, st);
    }
    GF_CUDA(cudaGetLastError());
    return FILTER_OK;
}

}  // namespace gf
