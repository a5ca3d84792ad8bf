// Counting quotient filter (GQF) table layout and in-place updates (paper
// Sec. 5 and the cited CQF): shared by the CUDA library (its even-odd region
// phases, Sec. 5.3) and the device-side point API of gpufilter_device.cuh
// (the locked point GQF, Sec. 5.2).
//
// Table: per 64-slot block a 32-byte record {occupieds, runends, offset}
// and an array of r-bit remainders. The run of quotient x holds its groups in
// ascending remainder order: [rem] for one copy, [rem, rem, n, n base-2^r
// digits of count - 2] for more; it starts at max(x, end of the previous run
// + 1) and ends at a set runend bit.
//
// The gv_* functions read and write one table through a GView. An update that
// starts at quotient x reads nothing below x's region start r0 and writes
// nothing outside [x, the slot its shift stops at]: callers keep threads that
// update the same stretch of slots apart (even-odd regions, or locks on two
// consecutive regions).
#pragma once

#include <stdint.h>

#include "gpufilter.h"

namespace gf {

static constexpr unsigned long long GQF_ST_INTERNAL = 1ull << FILTER_ERR_INTERNAL;

struct Meta {
    unsigned long long occ, rend;
    unsigned int off, pad0;
    unsigned long long pad1;
};
static_assert(sizeof(Meta) == 32, "metadata record is 32 bytes");

__host__ __device__ __forceinline__ uint32_t ndig(uint64_t v, uint32_t r)
{
    uint32_t n = 0;
    while (v) {
        n++;
        v = (r >= 64) ? 0 : (v >> r);
    }
    return n;
}
__host__ __device__ __forceinline__ uint32_t enc_len(uint64_t c, uint32_t r) { return c == 1 ? 1u : 3u + ndig(c - 2, r); }

template <int R>
__device__ __forceinline__ uint32_t rd_slot(const uint8_t *rem, uint64_t i)
{
    if (R == 8) return rem[i];
    return reinterpret_cast<const uint16_t *>(rem)[i];
}
template <int R>
__device__ __forceinline__ void wr_slot(uint8_t *rem, uint64_t i, uint32_t v)
{
    if (R == 8) rem[i] = (uint8_t)v;
    else reinterpret_cast<uint16_t *>(rem)[i] = (uint16_t)v;
}

struct GView {
    Meta *meta;
    uint8_t *rem;
    long long N, nslots, nblk;
};

__device__ __forceinline__ bool gv_occ(const GView &g, long long y) { return (g.meta[y >> 6].occ >> (y & 63)) & 1ull; }
__device__ __forceinline__ void gv_rend_put(const GView &g, long long i, bool v)
{
    unsigned long long &w = g.meta[i >> 6].rend;
    if (v) w |= 1ull << (i & 63);
    else w &= ~(1ull << (i & 63));
}

// first runend at or after slot i, or -1
__device__ long long gv_next_runend(const GView &g, long long i)
{
    long long w = i >> 6;
    if (i < 0 || w >= g.nblk) return -1;
    unsigned long long bits = g.meta[w].rend & (~0ull << (i & 63));
    while (!bits) {
        if (++w >= g.nblk) return -1;
        bits = g.meta[w].rend;
    }
    return 64 * w + __ffsll((long long)bits) - 1;
}

// last runend in [lo, hi], or -1
__device__ long long gv_prev_runend(const GView &g, long long hi, long long lo)
{
    if (hi < lo) return -1;
    long long w = hi >> 6;
    const unsigned hb = (unsigned)(hi & 63);
    unsigned long long bits = g.meta[w].rend & (hb == 63 ? ~0ull : ((1ull << (hb + 1)) - 1ull));
    while (true) {
        if (64 * w <= lo) bits &= ~0ull << (lo - 64 * w);
        if (bits) return 64 * w + 63 - __clzll((long long)bits);
        if (64 * w <= lo) return -1;
        bits = g.meta[--w].rend;
    }
}

// smallest occupied quotient in (y, lim], or -1
__device__ long long gv_next_occ(const GView &g, long long y, long long lim)
{
    if (lim >= g.N) lim = g.N - 1;
    const long long z = y + 1;
    if (z > lim) return -1;
    long long w = z >> 6;
    unsigned long long bits = g.meta[w].occ & (~0ull << (z & 63));
    while (true) {
        if (bits) {
            long long q = 64 * w + __ffsll((long long)bits) - 1;
            return q <= lim ? q : -1;
        }
        if (64 * (w + 1) > lim) return -1;
        bits = g.meta[++w].occ;
    }
}

// end of the run of an occupied quotient y: offset of its block, then select
__device__ long long gv_runend_of(const GView &g, long long y)
{
    const long long j = y >> 6;
    const long long base = 64 * j + (long long)g.meta[j].off;
    const unsigned k = (unsigned)(y & 63);
    const unsigned long long upto = (k == 63) ? ~0ull : ((1ull << (k + 1)) - 1ull);
    int d = __popcll(g.meta[j].occ & upto & ~1ull);
    if (d == 0) return base;
    long long w = base >> 6;
    const unsigned bsh = (unsigned)(base & 63);
    unsigned long long bits = (bsh == 63) ? 0ull : (g.meta[w].rend & (~0ull << (bsh + 1)));
    while (true) {
        int pc = __popcll(bits);
        if (pc >= d) {
            for (int t = 1; t < d; t++) bits &= bits - 1;
            return 64 * w + __ffsll((long long)bits) - 1;
        }
        d -= pc;
        if (++w >= g.nblk) return -1;
        bits = g.meta[w].rend;
    }
}

// offsets of the blocks j with 64j in [y, ylim) whose largest occupied
// quotient <= 64j is y, given y's new and old run ends
__device__ __forceinline__ void gv_fix_offsets(const GView &g, long long y, long long ylim, long long new_end,
                                               long long old_end)
{
    long long jlo = (y + 63) >> 6;
    long long hi = ylim - 1 < old_end ? ylim - 1 : old_end;
    if (hi < 0) return;
    long long jhi = hi >> 6;
    if (jhi >= g.nblk) jhi = g.nblk - 1;
    for (long long j = jlo; j <= jhi; j++) {
        long long o = new_end - 64 * j;
        g.meta[j].off = (unsigned)(o > 0 ? o : 0);
    }
}

// remove min(c, d) copies of fingerprint fp; returns the number removed
template <int R>
__device__ uint64_t gv_delete(const GView &g, uint64_t fp, uint64_t d, unsigned long long *status)
{
    const long long x = (long long)(fp >> R);
    const uint32_t v = (uint32_t)(fp & ((1ull << R) - 1ull));
    if (x >= g.N || !gv_occ(g, x)) return 0;
    const long long e = gv_runend_of(g, x);
    if (e < 0) {
        atomicOr(status, GQF_ST_INTERNAL);
        return 0;
    }
    const long long pr = gv_prev_runend(g, e - 1, x);
    const long long s = pr >= 0 ? pr + 1 : x;
    long long gpos = -1;
    uint32_t glen = 0;
    uint64_t c = 0;
    for (long long p = s; p <= e;) {
        const uint32_t val = rd_slot<R>(g.rem, (uint64_t)p);
        uint64_t cc = 1;
        uint32_t len = 1;
        if (p + 2 <= e && rd_slot<R>(g.rem, (uint64_t)(p + 1)) == val) {
            uint32_t nd = rd_slot<R>(g.rem, (uint64_t)(p + 2));
            if (p + 2 + (long long)nd > e) nd = (uint32_t)(e - p - 2);
            uint64_t acc = 0;
            for (uint32_t t = 0; t < nd; t++) acc = (acc << R) | rd_slot<R>(g.rem, (uint64_t)(p + 3 + t));
            cc = acc + 2;
            len = 3 + nd;
        }
        if (val == v) {
            gpos = p;
            glen = len;
            c = cc;
            break;
        }
        if (val > v) break;
        p += len;
    }
    if (gpos < 0) return 0;
    const uint64_t rm = c < d ? c : d;
    const uint64_t c2 = c - rm;
    const uint32_t nlen = c2 ? enc_len(c2, R) : 0u;
    if (c2) {
        long long q = gpos;
        wr_slot<R>(g.rem, (uint64_t)q++, v);
        if (c2 > 1) {
            const uint64_t xx = c2 - 2;
            const uint32_t nd = ndig(xx, R);
            wr_slot<R>(g.rem, (uint64_t)q++, v);
            wr_slot<R>(g.rem, (uint64_t)q++, nd);
            for (uint32_t t = 0; t < nd; t++)
                wr_slot<R>(g.rem, (uint64_t)q++, (uint32_t)((xx >> (R * (nd - 1 - t))) & ((1u << R) - 1u)));
        }
    }
    const long long delta = (long long)glen - (long long)nlen;
    if (delta == 0) return rm;
    // the rest of run x moves left by delta
    for (long long q = gpos + glen; q <= e; q++) wr_slot<R>(g.rem, (uint64_t)(q - delta), rd_slot<R>(g.rem, (uint64_t)q));
    const bool empty = (e - s + 1) == delta;
    for (long long q = e - delta + 1; q <= e; q++) wr_slot<R>(g.rem, (uint64_t)q, 0u);  // vacated by run x
    gv_rend_put(g, e, false);
    long long new_prev_end;
    if (!empty) {
        gv_rend_put(g, e - delta, true);
        new_prev_end = e - delta;
    } else {
        g.meta[x >> 6].occ &= ~(1ull << (x & 63));
        new_prev_end = (s > x) ? s - 1 : x - 1;  // the run before x (any end < x when s == x)
    }
    long long old_prev_end = e;
    long long y = x, y_new = new_prev_end, y_old = e;
    // following runs of the cluster move to max(home, previous end + 1)
    while (true) {
        const long long yn = gv_next_occ(g, y, old_prev_end + 1);
        gv_fix_offsets(g, y, yn >= 0 ? yn : (1ll << 62), y_new, y_old);
        if (yn < 0) break;
        const long long os = yn > old_prev_end + 1 ? yn : old_prev_end + 1;
        const long long ns = yn > new_prev_end + 1 ? yn : new_prev_end + 1;
        if (ns == os) break;
        const long long oe = gv_next_runend(g, os);
        if (oe < 0) {
            atomicOr(status, GQF_ST_INTERNAL);
            break;
        }
        const long long len = oe - os + 1;
        for (long long q = 0; q < len; q++) wr_slot<R>(g.rem, (uint64_t)(ns + q), rd_slot<R>(g.rem, (uint64_t)(os + q)));
        for (long long q = (ns + len > os ? ns + len : os); q <= oe; q++) wr_slot<R>(g.rem, (uint64_t)q, 0u);  // vacated
        gv_rend_put(g, oe, false);
        gv_rend_put(g, ns + len - 1, true);
        old_prev_end = oe;
        new_prev_end = ns + len - 1;
        y = yn;
        y_new = new_prev_end;
        y_old = oe;
    }
    return rm;
}

// ---------------------------------------------------------------------------
// In-place bulk insert over even-odd regions (the paper's Sec. 5.3 scheme):
// one thread per region inserts the region's groups in ascending order, each
// by rewriting its run and moving the following runs of the cluster right
// (the mirror of the delete above; the result is the same canonical layout
// as the merge). A read-only pre-check bounds, per region, how far the
// region's inserts can push data: the Delta-th empty slot after its last
// group, Delta being the exact number of slots the region adds. When every
// region's bound ends before the region after next (and before the end of
// the table), two threads of a phase never touch the same slots or words,
// and every value a thread reads outside its own region belongs to a region
// that is idle in that phase.
// ---------------------------------------------------------------------------
// largest occupied quotient in [lo, x), or -1
__device__ long long gv_prev_occ_from(const GView &g, long long x, long long lo)
{
    long long z = x - 1;
    if (z < lo) return -1;
    long long w = z >> 6;
    unsigned long long bits = g.meta[w].occ & (((z & 63) == 63) ? ~0ull : ((1ull << ((z & 63) + 1)) - 1ull));
    while (true) {
        if (64 * w < lo) bits &= ~0ull << (lo - 64 * w);
        if (bits) return 64 * w + 63 - __clzll((long long)bits);
        if (64 * w <= lo) return -1;
        bits = g.meta[--w].occ;
    }
}

// End of the run of the largest occupied quotient < x, for x in the region
// starting at r0, from the region's own metadata (-1: it ends before r0).
// A run that reaches into the region from the left is known from the offset
// of the region's first block, which the region alone may change.
__device__ long long gv_prev_end_in(const GView &g, long long x, long long r0)
{
    const long long y = gv_prev_occ_from(g, x, r0);
    if (y >= 0) return gv_runend_of(g, y);
    const long long b0 = r0 >> 6;
    if (gv_occ(g, r0)) {
        // x == r0 and r0 has a run: the chain before it ends just before it starts
        const long long e = gv_runend_of(g, r0);
        const long long pr = gv_prev_runend(g, e - 1, r0);
        return pr >= 0 ? pr : -1;
    }
    const long long off = (long long)g.meta[b0].off;
    if (off > 0) return r0 + off;
    if ((g.meta[b0].rend & 1ull) != 0) return r0;
    return -1;
}

// one group (value v, count c) of R-bit slots at position pos
template <int R>
__device__ __forceinline__ void gv_put_group(const GView &g, long long pos, uint32_t v, uint64_t c)
{
    wr_slot<R>(g.rem, (uint64_t)pos++, v);
    if (c == 1) return;
    const uint64_t xx = c - 2;
    const uint32_t nd = ndig(xx, R);
    wr_slot<R>(g.rem, (uint64_t)pos++, v);
    wr_slot<R>(g.rem, (uint64_t)pos++, nd);
    for (uint32_t t = 0; t < nd; t++)
        wr_slot<R>(g.rem, (uint64_t)pos++, (uint32_t)((xx >> (R * (nd - 1 - t))) & ((1u << R) - 1u)));
}

// the group of run [p, e] starting at p: value, count, encoded length
template <int R>
__device__ __forceinline__ uint32_t gv_group_at(const GView &g, long long p, long long e, uint32_t &val, uint64_t &cc)
{
    val = rd_slot<R>(g.rem, (uint64_t)p);
    cc = 1;
    if (p + 2 <= e && rd_slot<R>(g.rem, (uint64_t)(p + 1)) == val) {
        uint32_t nd = rd_slot<R>(g.rem, (uint64_t)(p + 2));
        if (p + 2 + (long long)nd > e) nd = (uint32_t)(e - p - 2);
        uint64_t acc = 0;
        for (uint32_t t = 0; t < nd; t++) acc = (acc << R) | rd_slot<R>(g.rem, (uint64_t)(p + 3 + t));
        cc = acc + 2;
        return 3 + nd;
    }
    return 1;
}

// Where group (x, v) goes: run start s, old run end e (s - 1 when x has no
// run), insertion point p, and the old count and length of v's group (0 when
// v is new). False on an inconsistent table.
template <int R>
__device__ bool gv_locate(const GView &g, long long x, uint32_t v, long long r0, long long &s, long long &e,
                          long long &p, uint64_t &c_old, uint32_t &ol)
{
    c_old = 0;
    ol = 0;
    if (gv_occ(g, x)) {
        e = gv_runend_of(g, x);
        if (e < 0) return false;
        const long long pr = gv_prev_runend(g, e - 1, x);
        s = pr >= 0 ? pr + 1 : x;
        p = s;
        while (p <= e) {
            uint32_t val;
            uint64_t cc;
            const uint32_t len = gv_group_at<R>(g, p, e, val, cc);
            if (val == v) {
                c_old = cc;
                ol = len;
                break;
            }
            if (val > v) break;
            p += len;
        }
    } else {
        const long long pe = gv_prev_end_in(g, x, r0);
        s = x > pe + 1 ? x : pe + 1;
        e = s - 1;
        p = s;
    }
    return true;
}

// add c copies of fingerprint fp; false on an inconsistent table
template <int R>
__device__ bool gv_insert(const GView &g, uint64_t fp, uint64_t c, long long r0)
{
    const long long x = (long long)(fp >> R);
    const uint32_t v = (uint32_t)(fp & ((1ull << R) - 1ull));
    const bool had = gv_occ(g, x);
    long long s, e, p;
    uint64_t c_old;
    uint32_t ol;
    if (!gv_locate<R>(g, x, v, r0, s, e, p, c_old, ol)) return false;
    const uint64_t cn = c_old + c;
    const uint32_t nl = enc_len(cn, R);
    const long long delta = (long long)nl - (long long)ol;
    if (delta == 0) {
        gv_put_group<R>(g, p, v, cn);
        return true;
    }
    // the following runs of the cluster move to max(home, previous end + 1);
    // find the last one that moves (all runs between x and it move)
    long long old_prev_end = e, new_prev_end = e + delta, y = x;
    long long cy = -1, cos = 0, coe = 0, cns = 0;
    while (true) {
        const long long yn = gv_next_occ(g, y, new_prev_end + 1);
        if (yn < 0) break;
        const long long os = yn > old_prev_end + 1 ? yn : old_prev_end + 1;
        const long long ns = yn > new_prev_end + 1 ? yn : new_prev_end + 1;
        if (ns == os) break;
        const long long oe = gv_next_runend(g, os);
        if (oe < 0) return false;
        cy = yn;
        cos = os;
        coe = oe;
        cns = ns;
        old_prev_end = oe;
        new_prev_end = ns + (oe - os);
        y = yn;
    }
    if (new_prev_end >= g.nslots) return false;
    // move them, last first: each moves right and lands right after the one
    // before it, so the one before is found from the untouched bits below
    long long ny = -1, first_moved = -1;
    while (cy >= 0) {
        const long long len = coe - cos + 1, ne = cns + len - 1;
        for (long long q = len - 1; q >= 0; q--)
            wr_slot<R>(g.rem, (uint64_t)(cns + q), rd_slot<R>(g.rem, (uint64_t)(cos + q)));
        gv_rend_put(g, coe, false);
        gv_rend_put(g, ne, true);
        const long long yl = ny >= 0 ? ny : gv_next_occ(g, cy, ne);
        gv_fix_offsets(g, cy, yl >= 0 ? yl : (1ll << 62), ne, ne);
        first_moved = cy;
        const long long py = gv_prev_occ_from(g, cy, x + 1);
        if (py < 0) break;
        const long long poe = gv_prev_runend(g, cos - 1, x);       // its old end
        if (poe < py) return false;
        const long long ppr = gv_prev_runend(g, poe - 1, x);       // the end of the run before it, if >= x
        const long long pst = py > ppr + 1 ? py : ppr + 1;
        const long long pns = cns - (poe - pst + 1);
        if (pns <= pst) return false;
        ny = cy;
        cy = py;
        cos = pst;
        coe = poe;
        cns = pns;
    }
    // the run of x: its tail after the group moves right, the group is written
    for (long long q = e; q >= p + (long long)ol; q--)
        wr_slot<R>(g.rem, (uint64_t)(q + delta), rd_slot<R>(g.rem, (uint64_t)q));
    gv_put_group<R>(g, p, v, cn);
    if (had) gv_rend_put(g, e, false);
    gv_rend_put(g, e + delta, true);
    if (!had) g.meta[x >> 6].occ |= 1ull << (x & 63);
    const long long ylim0 = first_moved >= 0 ? first_moved : gv_next_occ(g, x, e + delta);
    gv_fix_offsets(g, x, ylim0 >= 0 ? ylim0 : (1ll << 62), e + delta, e + delta);
    return true;
}

// Where data pushed right by `need` slots from quotient x stops: the need-th
// empty slot at or after the chain that covers x (-1 when it would pass
// `limit`). r0: the start of x's region.
__device__ long long gv_push_end(const GView &g, long long x, long long need, long long r0, long long limit)
{
    long long pos = x;
    long long E = gv_prev_end_in(g, x + 1, r0);  // end of the run of the largest occupied quotient <= x
    if (E >= pos) {
        long long y = pos;
        while (true) {
            const long long yn = gv_next_occ(g, y, E + 1);
            if (yn < 0) break;
            E = gv_next_runend(g, E + 1);
            if (E < 0 || E > limit) return -1;
            y = yn;
        }
        pos = E + 1;
    }
    while (need > 0) {
        if (pos > limit) return -1;
        const long long yn = gv_next_occ(g, pos - 1, limit);
        const long long gap = (yn < 0 ? limit + 1 : yn) - pos;  // empty slots before the next run
        if (gap >= need) return pos + need - 1;
        if (yn < 0) return -1;
        need -= gap;
        E = gv_runend_of(g, yn);
        long long y = yn;
        while (E >= 0 && E <= limit) {
            const long long y2 = gv_next_occ(g, y, E + 1);
            if (y2 < 0) break;
            E = gv_next_runend(g, E + 1);
            y = y2;
        }
        if (E < 0 || E > limit) return -1;
        pos = E + 1;
    }
    return pos - 1;
}

// ---------------------------------------------------------------------------
// Point updates, the locked point GQF (Sec. 5.2): one thread applies one key.
// The table is cut into lock regions of 8192 quotients; an update of quotient
// x takes the lock of x's region and then of the next one (always in that
// order, so no wait can close a cycle), each a 32-bit word alone in its
// 128-byte line, with a bounded number of attempts. Two threads that hold
// locks at the same time are then at least two regions apart, as the
// threads of one even-odd phase are, and an update that stays below the
// start of the region after next never meets another one. The insert checks
// that its shift stops there, the delete that x's cluster ends there;
// otherwise nothing changes and the key is reported FULL (insert) or BUSY.
// Clusters stay far shorter than a region while the home slots are at most
// about 95 % used (the bound the paper cites); past that, updates near the
// end of a region start to report FULL / BUSY although the tail has room.
// ---------------------------------------------------------------------------
static constexpr long long GQF_LOCK_REGION = 8192;  // quotients per lock region
static constexpr int GQF_LOCK_STRIDE = 32;          // 32-bit words from one lock to the next (128 bytes)
static constexpr uint32_t GQF_LOCK_TRIES = 1u << 20;
static constexpr int GQF_POINT_BUSY = 3;            // a lock wait gave up, or the cluster is too long

// Test and test-and-set: waiters read the word (no atomic traffic on a held
// lock) and try the compare-and-swap only when it reads free, backing off
// exponentially; the wait gives up after GQF_LOCK_TRIES reads.
__device__ __forceinline__ bool gqf_lock_take(uint32_t *l)
{
    uint32_t ns = 64;
    const uint32_t zero = 0, one = 1;
    for (uint32_t t = 0; t < GQF_LOCK_TRIES; t++) {
        uint32_t cur;
        asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(cur) : "l"(l) : "memory");
        if (cur == 0) {
            uint32_t old;
            asm volatile("atom.acquire.gpu.global.cas.b32 %0, [%1], %2, %3;"
                         : "=r"(old)
                         : "l"(l), "r"(zero), "r"(one)
                         : "memory");
            if (old == 0) return true;
        }
        __nanosleep(ns + (threadIdx.x & 31) * 8);  // staggered, so that waiters do not retry together
        if (ns < 4096) ns <<= 1;
    }
    return false;
}

__device__ __forceinline__ void gqf_lock_give(uint32_t *l)
{
    const uint32_t zero = 0;
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(l), "r"(zero) : "memory");
}

// locks of x's region and the next; the slots the update may touch end at *limit
__device__ __forceinline__ bool gqf_lock_pair(const GView &g, uint32_t *locks, long long x, long long &r0,
                                              long long &limit, uint32_t *&l0, uint32_t *&l1)
{
    const long long reg = x / GQF_LOCK_REGION;
    const long long nreg = (g.N + GQF_LOCK_REGION - 1) / GQF_LOCK_REGION;
    l0 = locks + reg * GQF_LOCK_STRIDE;
    l1 = reg + 1 < nreg ? locks + (reg + 1) * GQF_LOCK_STRIDE : nullptr;
    r0 = reg * GQF_LOCK_REGION;
    limit = reg + 2 < nreg ? (reg + 2) * GQF_LOCK_REGION - 2 : g.nslots - 1;
    if (!gqf_lock_take(l0)) return false;
    if (l1 && !gqf_lock_take(l1)) {
        gqf_lock_give(l0);
        return false;
    }
    return true;
}

__device__ __forceinline__ void gqf_unlock_pair(uint32_t *l0, uint32_t *l1)
{
    if (l1) gqf_lock_give(l1);
    gqf_lock_give(l0);
}

// The lanes of a warp that call together take their turns one after another
// (lowest lane first): a lane that waits for a lock sleeps, and a sleeping
// lane would hold up a lane of its own warp that holds a lock. f(lane) runs
// the lane's update; returns its result.
template <class Fn>
__device__ __forceinline__ int gqf_warp_turns(Fn f)
{
    const unsigned active = __activemask();
    const unsigned me = 1u << (threadIdx.x & 31);
    int rc = 0;
    for (unsigned todo = active; todo; todo &= todo - 1) {
        if ((todo & (0u - todo)) == me) rc = f();
        __syncwarp(active);
    }
    return rc;
}

// c copies of fingerprint fp: FILTER_KEY_OK, FILTER_KEY_FULL (no room before
// the region after next, or past the table) or GQF_POINT_BUSY
template <int R>
__device__ int gqf_point_insert(const GView &g, uint32_t *locks, uint64_t fp, uint64_t c,
                                unsigned long long *status)
{
    const long long x = (long long)(fp >> R);
    const uint32_t v = (uint32_t)(fp & ((1ull << R) - 1ull));
    long long r0, limit;
    uint32_t *l0, *l1;
    if (x >= g.N || !gqf_lock_pair(g, locks, x, r0, limit, l0, l1)) return GQF_POINT_BUSY;
    int rc = FILTER_KEY_FULL;
    long long s, e, p;
    uint64_t c_old;
    uint32_t ol;
    if (gv_locate<R>(g, x, v, r0, s, e, p, c_old, ol)) {
        const long long need = (long long)enc_len(c_old + c, R) - (long long)ol;
        if (need <= 0 || gv_push_end(g, x, need, r0, limit) >= 0) {
            if (gv_insert<R>(g, fp, c, r0)) rc = FILTER_KEY_OK;
            else atomicOr(status, GQF_ST_INTERNAL);
        }
    }
    gqf_unlock_pair(l0, l1);
    return rc;
}

// one copy of fingerprint fp: FILTER_KEY_OK, FILTER_KEY_NOT_FOUND or
// GQF_POINT_BUSY (also when x's cluster runs past the region after next)
template <int R>
__device__ int gqf_point_remove(const GView &g, uint32_t *locks, uint64_t fp, unsigned long long *status)
{
    const long long x = (long long)(fp >> R);
    long long r0, limit;
    uint32_t *l0, *l1;
    if (x >= g.N || !gqf_lock_pair(g, locks, x, r0, limit, l0, l1)) return GQF_POINT_BUSY;
    int rc = FILTER_KEY_NOT_FOUND;  // (no run: nothing stored)
    if (gv_occ(g, x)) {
        // the run of x ends at or after x: where the cluster from x ends
        const long long ce = gv_push_end(g, x, 0, r0, limit);
        rc = ce >= x && ce <= limit ? (gv_delete<R>(g, fp, 1, status) ? FILTER_KEY_OK : FILTER_KEY_NOT_FOUND)
                                    : GQF_POINT_BUSY;
    }
    gqf_unlock_pair(l0, l1);
    return rc;
}

}  // namespace gf
