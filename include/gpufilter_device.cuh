/*
 * gpufilter_device.cuh - device-side point operations on filters built by the
 * library, callable from the caller's own CUDA kernels (header only).
 *
 * The paper's filters are also used from inside GPU applications, one key
 * per thread, next to the bulk API (Sec. 4: point operations; Sec. 6). This
 * header lets a kernel written elsewhere query a TCF or count a key in a GQF
 * that the C ABI built and filled, and insert into or remove from a point-mode
 * TCF:
 *
 *   host:    filter_device_view v;  filter_get_device_view(f, &v);
 *            pass v by value to the kernel
 *   device:  bool hit  = gf_device_tcf_contains(v, key);
 *            uint32_t x = gf_device_tcf_value(v, key);     (TCF with values)
 *            uint64_t c = gf_device_gqf_count(v, key);
 *            int st = gf_device_tcf_insert(v, key[, value]); (point-mode TCF only)
 *            int st = gf_device_tcf_remove(v, key);          (point-mode TCF only)
 *            int st = gf_device_gqf_insert(v, key);          (GQF, Sec. 5.2 locks)
 *            int st = gf_device_gqf_remove(v, key);
 *
 * A view describes the table as it is when filter_get_device_view returns;
 * it must be taken again after any insert, remove, clear or import through
 * the C ABI (a GQF update switches between two table buffers). Queries and
 * counts read only. Point-mode TCF inserts and removes may run concurrently
 * with each other and with queries from any number of threads (one atomic
 * compare-and-swap per slot, Alg. 1), but not with the library's own calls on
 * the filter. GQF point inserts and removes may run concurrently with each
 * other (region locks, gpufilter_gqf_ops.cuh, shared with the library's
 * in-place bulk updates); they update the current table buffer in place, so
 * the view stays valid, but they must not overlap counts or the library's
 * own calls on the filter. The hashing is the library's own
 * (gpufilter_hash.cuh); the TCF block access and point-mode updates are
 * restated here for one key per thread, and GPU tests check them against the
 * C ABI.
 */
#pragma once

#include <stdint.h>

#include "gpufilter.h"
#include "gpufilter_gqf_ops.cuh"
#include "gpufilter_hash.cuh"

namespace gf_device {

using gf::mix64;

// The GQF fingerprint (include/gpufilter_hash.cuh, the library's own)
__device__ __forceinline__ uint64_t gqf_fingerprint(uint64_t key, uint32_t p, uint64_t seed)
{
    return gf::fingerprint(key, gf::phash_of(p, seed));
}

// the tag part of every f-bit lane of a word (a TCF with v value bits keeps
// the value in the low v bits of each slot)
__device__ __forceinline__ uint32_t tcf_lane_mask(uint32_t f, uint32_t vbits)
{
    const uint32_t vm = (1u << vbits) - 1u;
    return f == 16 ? (0xffffu & ~vm) * 0x00010001u : (0xffu & ~vm) * 0x01010101u;
}

// does the 32-byte block hold tag t (f = 8 or 16 bits per slot; t is the
// slot with value 0, lm from tcf_lane_mask)?
__device__ __forceinline__ bool tcf_block_has(const uint8_t *blocks, uint64_t b, uint32_t t, uint32_t f,
                                              uint32_t lm)
{
    // L2 loads: coherent with device-side updates made by other threads
    const uint4 *p = reinterpret_cast<const uint4 *>(blocks + b * 32);
    const uint4 lo = __ldcg(p), hi = __ldcg(p + 1);
    const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
    uint32_t m = 0;
    if (f == 16) {
        const uint32_t tt = t | (t << 16);
#pragma unroll
        for (int k = 0; k < 8; k++) m |= __vcmpeq2(w[k] & lm, tt);
    } else {
        const uint32_t tt = t * 0x01010101u;
#pragma unroll
        for (int k = 0; k < 8; k++) m |= __vcmpeq4(w[k] & lm, tt);
    }
    return m != 0;
}

// smallest value part among the slots of block b that hold tag t, or 0xff /
// 0xffff (more than any value) when none does
__device__ __forceinline__ uint32_t tcf_block_min_value(const uint8_t *blocks, uint64_t b, uint32_t t, uint32_t f,
                                                        uint32_t lm)
{
    const uint4 *p = reinterpret_cast<const uint4 *>(blocks + b * 32);
    const uint4 lo = __ldcg(p), hi = __ldcg(p + 1);
    const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
    uint32_t m = 0xffffffffu;
    if (f == 16) {
        const uint32_t tt = t | (t << 16);
#pragma unroll
        for (int k = 0; k < 8; k++) m = __vminu2(m, (w[k] & ~lm) | ~__vcmpeq2(w[k] & lm, tt));
        return min(m & 0xffffu, m >> 16);
    }
    const uint32_t tt = t * 0x01010101u;
#pragma unroll
    for (int k = 0; k < 8; k++) m = __vminu4(m, (w[k] & ~lm) | ~__vcmpeq4(w[k] & lm, tt));
    m = __vminu4(m, m >> 16);
    return min(m & 0xffu, (m >> 8) & 0xffu);
}

template <int R>
__device__ __forceinline__ uint32_t gqf_slot(const uint8_t *rem, uint64_t i)
{
    if (R == 8) return rem[i];
    return reinterpret_cast<const uint16_t *>(rem)[i];
}

// Count of fingerprint fp: the quotient's home block gives the offset of the
// first run end at or after it; the run of quotient x ends at the d-th run
// end from there, where d counts the occupied quotients of the block up to x;
// it starts one past the previous run end (or at x). Inside the run, groups
// are [rem] or [rem, rem, n, n base-2^R digits of count - 2], ascending.
template <int R>
__device__ uint64_t gqf_count_fp(uint64_t fp, const uint8_t *meta, const uint8_t *rem, uint64_t nblk)
{
    // metadata record of block j: occupieds u64, runends u64, offset u32, 12 bytes unused
    auto occ_of = [&](uint64_t j) { return __ldg(reinterpret_cast<const unsigned long long *>(meta + 32 * j)); };
    auto rend_of = [&](uint64_t j) { return __ldg(reinterpret_cast<const unsigned long long *>(meta + 32 * j + 8)); };
    auto off_of = [&](uint64_t j) { return __ldg(reinterpret_cast<const unsigned int *>(meta + 32 * j + 16)); };
    const uint64_t x = fp >> R;
    const uint32_t v = (uint32_t)(fp & ((1ull << R) - 1ull));
    const uint64_t j = x >> 6;
    if (j >= nblk) return 0;
    const unsigned long long occ = occ_of(j);
    if (!((occ >> (x & 63)) & 1ull)) return 0;
    const long long base = (long long)(64 * j) + (long long)off_of(j);
    const unsigned sh = (unsigned)(x & 63);
    const unsigned long long upto = (sh == 63) ? ~0ull : ((1ull << (sh + 1)) - 1ull);
    int d = __popcll(occ & upto & ~1ull);
    long long end = base;
    if (d > 0) {
        long long w = base >> 6;
        const unsigned bsh = (unsigned)(base & 63);
        unsigned long long bits = (bsh == 63) ? 0ull : (rend_of((uint64_t)w) & (~0ull << (bsh + 1)));
        while (true) {
            const int pc = __popcll(bits);
            if (pc >= d) {
                for (int k = 1; k < d; k++) bits &= bits - 1;
                end = 64 * w + __ffsll((long long)bits) - 1;
                break;
            }
            d -= pc;
            if (++w >= (long long)nblk) return 0;
            bits = rend_of((uint64_t)w);
        }
    }
    long long start = (long long)x;
    for (long long p = end - 1; p >= (long long)x;) {
        const long long w = p >> 6;
        unsigned long long bits = rend_of((uint64_t)w);
        const unsigned pb = (unsigned)(p & 63);
        bits &= (pb == 63) ? ~0ull : ((1ull << (pb + 1)) - 1ull);
        if (64 * w < (long long)x) bits &= ~0ull << (x & 63);
        if (bits) {
            start = 64 * w + 63 - __clzll((long long)bits) + 1;
            break;
        }
        p = 64 * w - 1;
    }
    for (long long q = start; q <= end;) {
        const uint32_t s = gqf_slot<R>(rem, (uint64_t)q);
        uint64_t c = 1;
        long long step = 1;
        if (q + 2 <= end && gqf_slot<R>(rem, (uint64_t)(q + 1)) == s) {
            uint32_t nd = gqf_slot<R>(rem, (uint64_t)(q + 2));
            if (q + 2 + (long long)nd > end) nd = (uint32_t)(end - q - 2);
            uint64_t acc = 0;
            for (uint32_t k = 0; k < nd; k++) acc = (acc << R) | gqf_slot<R>(rem, (uint64_t)(q + 3 + k));
            c = acc + 2;
            step = 3 + nd;
        }
        if (s == v) return c;
        if (s > v) return 0;
        q += step;
    }
    return 0;
}

}  // namespace gf_device

// Is key in the TCF (a false positive with the filter's rate, never a false
// negative for an inserted key)? Tag t and block pair (b1, b2 = b1 xor g(t))
// from one 64-bit hash; the backing bucket is read only when some key was
// stored there.
namespace gf_device {

// the key's block pair and its slot with value 0: the (f - v)-bit tag from
// bits 44.. of the hash, shifted above the v value bits; g uses the tag alone
__device__ __forceinline__ void tcf_key(const filter_device_view &v, uint64_t key, uint64_t &b1, uint64_t &b2,
                                        uint32_t &t)
{
    uint32_t tag;
    gf::tcf_key_parts(key, v.seed, v.n_blocks, (1u << (v.tag_bits - v.value_bits)) - 1u, b1, b2, tag);
    t = tag << v.value_bits;
}

// the key's backing bucket (chosen by the entry without its value bits)
__device__ __forceinline__ uint64_t *tcf_bucket_ptr(const filter_device_view &v, uint64_t e)
{
    return static_cast<uint64_t *>(v.aux) + gf::tcf_bucket(e, v.n_aux) * 8;
}

}  // namespace gf_device

// Is key in the TCF (a false positive with the filter's rate, never a false
// negative for an inserted key)? Tag t and block pair (b1, b2 = b1 xor g(t))
// from one 64-bit hash; the backing bucket is read only when some key was
// stored there.
__device__ __forceinline__ bool gf_device_tcf_contains(const filter_device_view &v, uint64_t key)
{
    using namespace gf_device;
    uint64_t b1, b2;
    uint32_t t;
    tcf_key(v, key, b1, b2, t);
    const uint32_t lm = tcf_lane_mask(v.tag_bits, v.value_bits);
    const uint8_t *blocks = static_cast<const uint8_t *>(v.table);
    if (tcf_block_has(blocks, b1, t, v.tag_bits, lm) || tcf_block_has(blocks, b2, t, v.tag_bits, lm)) return true;
    if (!v.counters || *(volatile unsigned long long *)(v.counters + 2) == 0) return false;
    const uint64_t e = ((b1 < b2 ? b1 : b2) << v.tag_bits) | t;
    const uint64_t em = ~((1ull << v.value_bits) - 1ull);
    const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(tcf_bucket_ptr(v, e));
#pragma unroll
    for (int s = 0; s < 4; s++) {
        const ulonglong2 w = __ldcg(p + s);
        if ((w.x & em) == e || (w.y & em) == e) return true;
    }
    return false;
}

// TCF with values: the smallest value stored with the key's fingerprint (in
// b1, b2 or its backing bucket), 0xFF when there is none. The same answer as
// filter_query_values.
__device__ __forceinline__ uint32_t gf_device_tcf_value(const filter_device_view &v, uint64_t key)
{
    using namespace gf_device;
    uint64_t b1, b2;
    uint32_t t;
    tcf_key(v, key, b1, b2, t);
    const uint32_t lm = tcf_lane_mask(v.tag_bits, v.value_bits), vm = (1u << v.value_bits) - 1u;
    const uint8_t *blocks = static_cast<const uint8_t *>(v.table);
    uint32_t best = min(tcf_block_min_value(blocks, b1, t, v.tag_bits, lm),
                        tcf_block_min_value(blocks, b2, t, v.tag_bits, lm));
    if (v.counters && *(volatile unsigned long long *)(v.counters + 2) != 0) {
        const uint64_t e = ((b1 < b2 ? b1 : b2) << v.tag_bits) | t;
        const uint64_t em = ~(uint64_t)vm;
        const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(tcf_bucket_ptr(v, e));
#pragma unroll
        for (int s = 0; s < 4; s++) {
            const ulonglong2 w = __ldcg(p + s);
            if ((w.x & em) == e) best = min(best, (uint32_t)w.x & vm);
            if ((w.y & em) == e) best = min(best, (uint32_t)w.y & vm);
        }
    }
    return best <= vm ? best : 0xffu;
}

namespace gf_device {

__device__ __forceinline__ uint32_t tcf_tag_at(const uint8_t *blocks, uint64_t b, int s, uint32_t f)
{
    const volatile uint8_t *p = blocks + b * 32;
    if (f == 16) return (uint32_t)p[2 * s] | ((uint32_t)p[2 * s + 1] << 8);
    return p[s];
}

// tags of block b that are neither EMPTY (0) nor TOMBSTONE (1)
__device__ __forceinline__ int tcf_live(const uint8_t *blocks, uint64_t b, uint32_t f)
{
    int c = 0;
    for (int s = 0; s < (int)(256 / f); s++) c += tcf_tag_at(blocks, b, s, f) >= 2;
    return c;
}

// put slot t into the first EMPTY or TOMBSTONE slot of block b (a bounded
// number of compare-and-swap attempts; false when the block is full)
__device__ __forceinline__ bool tcf_put(uint8_t *blocks, uint64_t b, uint32_t t, uint32_t f,
                                        unsigned long long *counters)
{
    const int B = (int)(256 / f);
    for (int attempt = 0; attempt < 4 * B; attempt++) {
        int s = -1;
        uint32_t seen = 0;
        for (int p = 0; p < B && s < 0; p++) {
            const uint32_t x = tcf_tag_at(blocks, b, p, f);
            if (x < 2) {
                s = p;
                seen = x;
            }
        }
        if (s < 0) return false;
        unsigned int *word = reinterpret_cast<unsigned int *>(blocks + b * 32) + ((s * f) >> 5);
        const unsigned sh = (unsigned)((s * f) & 31);
        const unsigned int lane = (f == 16 ? 0xffffu : 0xffu) << sh;
        const unsigned int cur = *(volatile unsigned int *)word;
        if (((cur & lane) >> sh) != seen) continue;  // changed since it was read
        if (atomicCAS(word, cur, (cur & ~lane) | (t << sh)) == cur) return true;
    }
    atomicOr(counters, 1ull << FILTER_ERR_TIMEOUT);
    return false;
}

// replace one copy of tag t (whatever its value: vm is the value part) in
// block b by TOMBSTONE
__device__ __forceinline__ bool tcf_take(uint8_t *blocks, uint64_t b, uint32_t t, uint32_t vm, uint32_t f,
                                         unsigned long long *counters)
{
    const int B = (int)(256 / f);
    for (int attempt = 0; attempt < 4 * B; attempt++) {
        int s = -1;
        uint32_t seen = 0;
        for (int p = 0; p < B && s < 0; p++) {
            const uint32_t x = tcf_tag_at(blocks, b, p, f);
            if ((x & ~vm) == t) {
                s = p;
                seen = x;
            }
        }
        if (s < 0) return false;
        unsigned int *word = reinterpret_cast<unsigned int *>(blocks + b * 32) + ((s * f) >> 5);
        const unsigned sh = (unsigned)((s * f) & 31);
        const unsigned int lane = (f == 16 ? 0xffffu : 0xffu) << sh;
        const unsigned int cur = *(volatile unsigned int *)word;
        if (((cur & lane) >> sh) != seen) continue;  // changed since it was read
        if (atomicCAS(word, cur, (cur & ~lane) | (1u << sh)) == cur) return true;
    }
    atomicOr(counters, 1ull << FILTER_ERR_TIMEOUT);
    return false;
}

}  // namespace gf_device

// Point-mode TCF insert (Alg. 1): into b1 while it holds fewer than 3B/4
// live tags (the shortcut), else into the block with fewer live tags, then
// the other, then an empty entry of the backing bucket. FILTER_KEY_OK, or
// FILTER_KEY_FULL (also counted in the filter's counters); FILTER_KEY_FULL
// without counting for a view that is not a point-mode TCF. A TCF with
// values stores the low value_bits of `value` with the tag.
__device__ __forceinline__ int gf_device_tcf_insert(const filter_device_view &v, uint64_t key, uint32_t value = 0)
{
    using namespace gf_device;
    if (v.kind != FILTER_TCF || v.mode != FILTER_MODE_POINT) return FILTER_KEY_FULL;
    uint64_t b1, b2;
    uint32_t t;
    tcf_key(v, key, b1, b2, t);
    t |= value & ((1u << v.value_bits) - 1u);
    const uint32_t f = v.tag_bits;
    uint8_t *blocks = static_cast<uint8_t *>(v.table);
    bool done = false;
    if (tcf_live(blocks, b1, f) < (int)(3 * (256 / f) / 4)) done = tcf_put(blocks, b1, t, f, v.counters);
    if (!done) {
        const uint64_t first = tcf_live(blocks, b1, f) <= tcf_live(blocks, b2, f) ? b1 : b2;
        done = tcf_put(blocks, first, t, f, v.counters) || tcf_put(blocks, first == b1 ? b2 : b1, t, f, v.counters);
    }
    if (!done) {
        const uint64_t e = ((b1 < b2 ? b1 : b2) << f) | t;
        unsigned long long *p = reinterpret_cast<unsigned long long *>(
            tcf_bucket_ptr(v, e & ~((1ull << v.value_bits) - 1ull)));
        for (int s = 0; s < 8 && !done; s++)
            if (atomicCAS(p + s, 0ull, (unsigned long long)e) == 0ull) done = true;
        if (done) atomicAdd(v.counters + 2, 1ull);
    }
    if (done) return FILTER_KEY_OK;
    atomicAdd(v.counters + 1, 1ull);
    atomicOr(v.counters, 1ull << FILTER_ERR_FULL);
    return FILTER_KEY_FULL;
}

// Point-mode TCF remove: one copy of the key's tag in b1, else b2, becomes
// TOMBSTONE (the first slot holding the tag, whatever its value), else its
// entry leaves the backing bucket. FILTER_KEY_OK or FILTER_KEY_NOT_FOUND
// (also for a view that is not a point-mode TCF).
__device__ __forceinline__ int gf_device_tcf_remove(const filter_device_view &v, uint64_t key)
{
    using namespace gf_device;
    if (v.kind != FILTER_TCF || v.mode != FILTER_MODE_POINT) return FILTER_KEY_NOT_FOUND;
    uint64_t b1, b2;
    uint32_t t;
    tcf_key(v, key, b1, b2, t);
    const uint32_t f = v.tag_bits, vm = (1u << v.value_bits) - 1u;
    uint8_t *blocks = static_cast<uint8_t *>(v.table);
    bool done = tcf_take(blocks, b1, t, vm, f, v.counters) || tcf_take(blocks, b2, t, vm, f, v.counters);
    if (!done) {
        const uint64_t e = ((b1 < b2 ? b1 : b2) << f) | t;
        unsigned long long *p = reinterpret_cast<unsigned long long *>(tcf_bucket_ptr(v, e));
        for (int s = 0; s < 8 && !done; s++) {
            const unsigned long long x = __ldcg(p + s);
            if ((x & ~(unsigned long long)vm) == e && atomicCAS(p + s, x, 0ull) == x) done = true;
        }
        if (done) atomicAdd(v.counters + 2, ~0ull);
    }
    return done ? FILTER_KEY_OK : FILTER_KEY_NOT_FOUND;
}

// How many copies of key the GQF counts (0 if absent; at least the true
// count, exactly it when distinct keys have distinct fingerprints).
__device__ __forceinline__ uint64_t gf_device_gqf_count(const filter_device_view &v, uint64_t key)
{
    using namespace gf_device;
    const uint32_t r = v.tag_bits;
    const uint64_t fp = gqf_fingerprint(key, v.q + r, v.seed);
    const uint8_t *meta = static_cast<const uint8_t *>(v.table);
    const uint8_t *rem = static_cast<const uint8_t *>(v.aux);
    return r == 8 ? gqf_count_fp<8>(fp, meta, rem, v.n_blocks) : gqf_count_fp<16>(fp, meta, rem, v.n_blocks);
}

// GQF point insert of one copy of key (Sec. 5.2): FILTER_KEY_OK;
// FILTER_KEY_FULL when the shift it needs would leave the two lock regions
// or the table (counted in the filter's counters, nothing changed); or 3
// when a lock wait gave up (the status word records FILTER_ERR_TIMEOUT,
// nothing changed; the caller may retry).
__device__ __forceinline__ int gf_device_gqf_insert(const filter_device_view &v, uint64_t key)
{
    using namespace gf_device;
    const uint32_t r = v.tag_bits;
    const uint64_t fp = gqf_fingerprint(key, v.q + r, v.seed);
    const gf::GView g{static_cast<gf::Meta *>(v.table), static_cast<uint8_t *>(v.aux), 1ll << v.q,
                      (long long)v.n_aux, (long long)v.n_blocks};
    const int rc = gf::gqf_warp_turns([&] {
        return r == 8 ? gf::gqf_point_insert<8>(g, v.locks, fp, 1, v.counters)
                      : gf::gqf_point_insert<16>(g, v.locks, fp, 1, v.counters);
    });
    if (rc == FILTER_KEY_FULL) {
        atomicOr(v.counters, 1ull << FILTER_ERR_FULL);
        atomicAdd(v.counters + 1, 1ull);
    } else if (rc == gf::GQF_POINT_BUSY) {
        atomicOr(v.counters, 1ull << FILTER_ERR_TIMEOUT);
    }
    return rc;
}

// GQF point remove of one copy of key: FILTER_KEY_OK, FILTER_KEY_NOT_FOUND,
// or 3 as for the insert (a lock wait gave up, or the key's cluster runs past
// the two lock regions; nothing changed).
__device__ __forceinline__ int gf_device_gqf_remove(const filter_device_view &v, uint64_t key)
{
    using namespace gf_device;
    const uint32_t r = v.tag_bits;
    const uint64_t fp = gqf_fingerprint(key, v.q + r, v.seed);
    const gf::GView g{static_cast<gf::Meta *>(v.table), static_cast<uint8_t *>(v.aux), 1ll << v.q,
                      (long long)v.n_aux, (long long)v.n_blocks};
    const int rc = gf::gqf_warp_turns([&] {
        return r == 8 ? gf::gqf_point_remove<8>(g, v.locks, fp, v.counters)
                      : gf::gqf_point_remove<16>(g, v.locks, fp, v.counters);
    });
    if (rc == gf::GQF_POINT_BUSY) atomicOr(v.counters, 1ull << FILTER_ERR_TIMEOUT);
    return rc;
}
