// Counting quotient filter (GQF), paper Sec. 5, for sm_103a.
//
// Table (double-buffered): per 64-slot block a 32-byte metadata record
// {occupieds, runends, offset}, and an array of r-bit remainders.
//
// Bulk insert / delete (Sec. 5.3-5.4, Sec. 6.4): fingerprints are computed,
// radix-sorted and reduced to <fingerprint, count> groups (the paper's
// map-reduce for skewed inputs). The groups are then merged into the table in
// ONE pass over quotient tiles of TQ quotients instead of the paper's
// even-odd region phases: a run of quotient x with encoded length L ends at
// e_x = max(x + L - 1, e_prev + L), so run placement is a prefix scan under
// the operator (A1, B1) . (A2, B2) = (max(A2, A1 + B2), B1 + B2). Each CTA
// decodes the old runs of its tile (located through the offset of its first
// block and select over runends), merges them with the tile's new groups,
// computes the run lengths, takes its incoming end from the preceding tiles
// by decoupled look-back, and writes its runs, runends, occupieds and
// offsets into the other buffer. Every slot of the new buffer is written by
// exactly one tile.
//
// Small batches (at most one group per 32 slots) are inserted in place over
// even-odd regions instead (Sec. 5.3), and small deletes likewise (Sec. 6.4).
//
// Counted insert (values through the counters, as in the CQF the paper
// follows): each key brings a count; the counts ride through the sort (or are
// gathered through its index array when statuses are wanted), are scanned,
// and the merge and the in-place inserts read each group's count from that
// prefix instead of from the group's number of keys.
//
// Count / query (Sec. 5.1 via the cited CQF): offset of the home block,
// rank over occupieds, select over runends, then a scan of the run.
#include <type_traits>
#include <vector>

#include "gf_internal.cuh"
#include "../../include/gpufilter_gqf_ops.cuh"

namespace gf {

static constexpr int MT = 256;          // merge threads per CTA
static constexpr int QPT = 8;           // quotients per thread
static constexpr int TQ = MT * QPT;     // quotients per tile
static constexpr int TBLK = TQ / 64;    // blocks per tile
static constexpr int OLDBUF = 3072;     // staged old slots
static constexpr int GSMALL = 640;      // staged new groups of a tile that has old runs
static constexpr int MIXCAP = 512;      // listed quotients whose run has old and new groups
static constexpr int OUTBUF = 3072;     // staged new slots
static constexpr int MERGE_CTAS = 5;    // resident merge CTAs per SM
static constexpr int RWORDS = OUTBUF / 64 + 2;
static constexpr long long NEG_INF = -(1ll << 60);


// ---------------------------------------------------------------------------
// The merge kernel
// ---------------------------------------------------------------------------
struct MergeArgs {
    const Meta *meta_old;
    const uint8_t *rem_old;
    Meta *meta_new;
    uint8_t *rem_new;
    const uint64_t *ufp;
    const uint32_t *ustart;
    const uint32_t *pm;      // number of groups (device)
    const uint32_t *tlo;     // first group of each tile (ntiles + 1 entries)
    uint64_t m_limit;        // use groups [0, min(m, m_limit))
    uint32_t *removed;       // delete: copies removed per group
    unsigned long long *ts;  // look-back state: [0] tile counter, then one status word per tile
    DevCounters *ctr;
    uint64_t N, nslots, nblk, ntiles;
    uint64_t fmask;          // fingerprint bits of a sorted value (a group keeps its member index above them)
    uint64_t tile0;          // group merge: global index of the filter's first tile
    uint32_t r;
    int del, dry;
};

__device__ __forceinline__ void agg_combine(long long &A, long long &Bs, long long A2, long long B2)
{
    // (A, Bs) then (A2, B2)
    long long a = A + B2;
    A = a > A2 ? a : A2;
    Bs += B2;
}

template <int R>
struct SlotIO {
    using T = typename std::conditional<R == 8, uint8_t, uint16_t>::type;
};


template <int R>
struct MergeSmem {
    unsigned long long occ[TBLK];
    unsigned int kpre[MT + 1];      // old runs before each thread's 8 quotients
    unsigned int Lq[TQ];            // new run length per quotient
    unsigned int qfirst[TQ];        // first new group of each quotient (or ~0)
    int qstart[TQ];                 // new run start relative to Q0
    // oend, old and gsm are adjacent: a tile without old runs stages its new
    // groups over all three
    int oend[TQ];                   // old run ends relative to Q0
    typename SlotIO<R>::T old[OLDBUF];
    unsigned int gsm[GSMALL];       // new groups, packed (qoff << 21 | rem << 5 | min(count, 31))
    typename SlotIO<R>::T out[OUTBUF];
    unsigned long long rend[RWORDS];
    unsigned short mix[MIXCAP];     // quotients (from Q0) with mixed runs, merged by all threads
    unsigned char newocc[MT];
    long long wA[MT / 32], wB[MT / 32];
    long long prev_end_old, os0, ein, w0, w1, tileP;
    unsigned long long glo, ghi;
    unsigned int tile, kold, oldlen, err, gcap, nmix;
};

// staged groups: GSMALL of them, or (no old runs) as many as fill oend, old and gsm
template <int R>
__host__ __device__ constexpr unsigned gbig()
{
    return (unsigned)((sizeof(int) * TQ + sizeof(typename SlotIO<R>::T) * OLDBUF) / 4 + GSMALL);
}
static_assert(offsetof(MergeSmem<8>, old) == offsetof(MergeSmem<8>, oend) + 4 * TQ &&
                  offsetof(MergeSmem<8>, gsm) == offsetof(MergeSmem<8>, old) + OLDBUF &&
                  offsetof(MergeSmem<16>, old) == offsetof(MergeSmem<16>, oend) + 4 * TQ &&
                  offsetof(MergeSmem<16>, gsm) == offsetof(MergeSmem<16>, old) + 2 * OLDBUF,
              "the group stage spans oend, old and gsm without gaps");

template <int R>
__device__ __forceinline__ const unsigned *gstage(const MergeSmem<R> &S)
{
    return S.gcap > GSMALL ? reinterpret_cast<const unsigned *>(S.oend) : S.gsm;
}

static_assert(offsetof(MergeSmem<8>, out) % 4 == 0 && offsetof(MergeSmem<16>, out) % 4 == 0 &&
                  OUTBUF % 4 == 0,
              "the staged output is cleared in 32-bit words");

// a new group's quotient offset from Q0, remainder and batch count, from its
// sorted value f and its start and end in the batch
template <int R>
__device__ __forceinline__ void decode_group(const MergeArgs &a, long long Q0, uint64_t fv, uint32_t s0, uint32_t s1,
                                             uint32_t &qoff, uint32_t &rem, uint64_t &cnt)
{
    const uint64_t f = fv & a.fmask;
    qoff = (uint32_t)((long long)(f >> R) - Q0);
    rem = (uint32_t)(f & ((1ull << R) - 1ull));
    cnt = s1 - s0;
}

static constexpr int GB = 4;  // groups a thread loads before using them

// new group g: quotient offset from Q0, remainder and batch count (from the
// tile's stage when it holds g)
template <int R>
__device__ __forceinline__ void new_group(const MergeSmem<R> &S, const MergeArgs &a, long long Q0, uint32_t g,
                                          uint32_t &qoff, uint32_t &rem, uint64_t &cnt)
{
    const uint64_t i = (uint64_t)g - S.glo;
    if (i < S.gcap) {
        const unsigned e = gstage<R>(S)[i];
        qoff = e >> 21;
        rem = (e >> 5) & 0xffffu;
        cnt = e & 31u;
        if (cnt == 31u) cnt = a.ustart[g + 1] - a.ustart[g];
        return;
    }
    const uint64_t f = a.ufp[g] & a.fmask;
    qoff = (uint32_t)((long long)(f >> R) - Q0);
    rem = (uint32_t)(f & ((1ull << R) - 1ull));
    cnt = a.ustart[g + 1] - a.ustart[g];
}

// old slot reader: staged when inside the staged window
template <int R>
__device__ __forceinline__ uint32_t old_at(const MergeSmem<R> &S, const MergeArgs &a, long long p)
{
    long long d = p - S.os0;
    if (d >= 0 && d < (long long)S.oldlen) return S.old[d];
    if (p < 0 || p >= (long long)a.nslots) return 0u;
    return rd_slot<R>(a.rem_old, (uint64_t)p);
}

// sequential reader of the groups of one old run [p, e]
struct OldRun {
    long long p, e;
};

template <int R>
__device__ __forceinline__ bool old_next(const MergeSmem<R> &S, const MergeArgs &a, OldRun &o, uint32_t &v,
                                         uint64_t &c)
{
    if (o.p > o.e) return false;
    v = old_at<R>(S, a, o.p);
    if (o.p + 2 <= o.e && old_at<R>(S, a, o.p + 1) == v) {
        uint32_t nd = old_at<R>(S, a, o.p + 2);
        if (o.p + 2 + (long long)nd > o.e) nd = (uint32_t)(o.e - o.p - 2);  // malformed: stay in the run
        uint64_t acc = 0;
        for (uint32_t d = 0; d < nd; d++) acc = (acc << R) | old_at<R>(S, a, o.p + 3 + d);
        c = acc + 2;
        o.p += 3 + nd;
    } else {
        c = 1;
        o.p += 1;
    }
    return true;
}

// emit one group's encoding at position pos (staged or global)
template <int R>
__device__ __forceinline__ void put_slot(MergeSmem<R> &S, const MergeArgs &a, long long pos, uint32_t v)
{
    long long d = pos - S.w0;
    if (d >= 0 && d < OUTBUF) S.out[d] = (typename SlotIO<R>::T)v;
    else if (pos < (long long)a.nslots) wr_slot<R>(a.rem_new, (uint64_t)pos, v);
}

template <int R>
__device__ __forceinline__ long long put_group(MergeSmem<R> &S, const MergeArgs &a, long long pos, uint32_t v,
                                               uint64_t c)
{
    put_slot<R>(S, a, pos++, v);
    if (c == 1) return pos;
    uint64_t x = c - 2;
    uint32_t nd = ndig(x, R);
    put_slot<R>(S, a, pos++, v);
    put_slot<R>(S, a, pos++, nd);
    for (uint32_t d = 0; d < nd; d++) put_slot<R>(S, a, pos++, (uint32_t)((x >> (R * (nd - 1 - d))) & ((1u << R) - 1u)));
    return pos;
}

// Merge the old groups of one run with the new groups [g, gend) of quotient y.
// WRITE = false: return the encoded length (and record removals);
// WRITE = true: write the run starting at `pos`.
template <int R, bool WRITE>
__device__ __forceinline__ uint32_t merge_run(MergeSmem<R> &S, const MergeArgs &a, OldRun o, bool has_old,
                                              uint32_t g, uint32_t gend, long long pos, long long Q0)
{
    uint32_t len = 0;
    uint32_t qoff_unused;
    uint32_t ov = 0, nv = 0;
    uint64_t oc = 0, nc = 0;
    bool ho = has_old && old_next<R>(S, a, o, ov, oc);
    bool hn = g < gend;
    if (hn) new_group<R>(S, a, Q0, g, qoff_unused, nv, nc);
    while (ho || hn) {
        uint32_t v;
        uint64_t c;
        if (ho && (!hn || ov < nv)) {
            v = ov;
            c = oc;
            ho = old_next<R>(S, a, o, ov, oc);
        } else {
            v = nv;
            if (ho && ov == nv) {
                if (a.del) {
                    uint64_t rm = oc < nc ? oc : nc;
                    c = oc - rm;
                    if (!WRITE && a.removed) a.removed[g] = (uint32_t)rm;
                } else {
                    c = oc + nc;
                }
                ho = old_next<R>(S, a, o, ov, oc);
            } else {
                if (a.del) {
                    c = 0;
                    if (!WRITE && a.removed) a.removed[g] = 0;
                } else {
                    c = nc;
                }
            }
            g++;
            hn = g < gend;
            if (hn) new_group<R>(S, a, Q0, g, qoff_unused, nv, nc);
        }
        if (c == 0) continue;
        if (WRITE) pos = put_group<R>(S, a, pos, v, c);
        else len += enc_len(c, R);
    }
    return len;
}

// The run of tile quotient y that has both old and new groups: its encoded
// length (WRITE = false) or its slots written from `start` (WRITE = true).
template <int R, bool WRITE>
__device__ __forceinline__ uint32_t mixed_run(MergeSmem<R> &S, const MergeArgs &a, long long Q0, int y,
                                              long long start)
{
    const unsigned byte = (unsigned)(S.occ[y >> 6] >> ((y & 56))) & 0xffu;
    const unsigned k = S.kpre[y >> 3] + __popc(byte & ((1u << (y & 7)) - 1u));
    const long long pe = (k == 0) ? S.prev_end_old : (Q0 + S.oend[k - 1]);
    OldRun o;
    o.e = Q0 + S.oend[k];
    o.p = (Q0 + y) > pe + 1 ? (Q0 + y) : pe + 1;
    const uint32_t gf = S.qfirst[y];
    uint32_t ge = gf;
    while (ge < S.ghi) {
        uint32_t qo, rm;
        uint64_t cn;
        new_group<R>(S, a, Q0, ge, qo, rm, cn);
        if ((int)qo != y) break;
        ge++;
    }
    return merge_run<R, WRITE>(S, a, o, true, gf, ge, start, Q0);
}

__device__ __forceinline__ unsigned long long ld_vol(const unsigned long long *p)
{
    return *(const volatile unsigned long long *)p;
}

// One tile of one filter. `tile` is the filter's own tile index; S.err is 0.
template <int R>
__device__ __forceinline__ void merge_tile(const MergeArgs &a, MergeSmem<R> &S, const uint64_t tile)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long Q0 = (long long)tile * TQ;
    const uint64_t j0 = tile * TBLK;
    const long long slot_end = min((long long)a.nslots, Q0 + TQ);

    // 1. old occupieds of the tile; 4a. its new group range (precomputed by
    // successor search), loaded alongside
    if (tid < TBLK) S.occ[tid] = (j0 + tid < a.nblk) ? a.meta_old[j0 + tid].occ : 0ull;
    if (tid == TBLK) {
        S.glo = a.tlo[tile];
        S.ghi = a.tlo[tile + 1];
    }
    __syncthreads();
    const uint32_t mybyte = (uint32_t)(S.occ[tid >> 3] >> ((tid & 7) * 8)) & 0xffu;

    // 2. old run index prefix per thread
    {
        uint32_t c = __popc(mybyte), incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        __shared__ unsigned int wsum[MT / 32];
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t pre = 0;
        for (int w = 0; w < warp; w++) pre += wsum[w];
        S.kpre[tid] = pre + incl - c;
        if (tid == MT - 1) {
            S.kpre[MT] = pre + incl;
            S.kold = pre + incl;
        }
    }
    __syncthreads();
    const uint32_t kold = S.kold;
    // the group stage (read by later phases, after further barriers)
    const uint32_t gcap = kold == 0 ? gbig<R>() : GSMALL;
    if (tid == 0) S.gcap = gcap;
    unsigned *gst = kold == 0 ? reinterpret_cast<unsigned *>(S.oend) : S.gsm;

    // 3. old run ends: select over runends after the offset of block j0, the
    // whole CTA at once (each thread takes 16 bits of one of 64 words a round)
    __shared__ unsigned int selw[MT / 32];
    if (kold > 0) {
        const long long base = Q0 + (long long)a.meta_old[j0].off;
        const bool q0occ = (S.occ[0] & 1ull) != 0;
        const long long sp = q0occ ? base : base + 1;
        const unsigned quarter = tid & 3;
        uint32_t found = 0;
        for (long long w0 = sp >> 6; found < kold; w0 += MT / 4) {
            const long long ww = w0 + (tid >> 2);
            unsigned long long bits = (ww < (long long)a.nblk) ? a.meta_old[ww].rend : 0ull;
            if (ww == (sp >> 6)) bits &= (~0ull) << (sp & 63);
            uint32_t b16 = (uint32_t)(bits >> (16 * quarter)) & 0xffffu;
            const uint32_t c = __popc(b16);
            uint32_t incl = c;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) selw[warp] = incl;
            __syncthreads();
            uint32_t pre = 0, tot = 0;
#pragma unroll
            for (int v = 0; v < MT / 32; v++) {
                const uint32_t x = selw[v];
                pre += v < warp ? x : 0u;
                tot += x;
            }
            uint32_t idx = found + pre + incl - c;
            while (b16 && idx < kold) {
                const int b = __ffs(b16) - 1;
                S.oend[idx] = (int)(ww * 64 + 16 * quarter + b - Q0);
                b16 &= b16 - 1;
                idx++;
            }
            found += tot;
            __syncthreads();  // selw is rewritten by the next round
            if (found < kold && w0 + MT / 4 >= (long long)a.nblk) {  // the same decision in every thread
                if (tid == 0) S.err = 1;
                break;
            }
        }
        // end of the run before the tile's first run
        if (tid == 0) {
            long long pe;
            if (q0occ) {
                // last runend in [Q0, base - 1]; Q0 is a multiple of 64
                pe = Q0 - 1;
                for (long long p = base - 1; p >= Q0;) {
                    long long w = p >> 6;
                    unsigned pb = (unsigned)(p & 63);
                    unsigned long long bits = a.meta_old[w].rend & (pb == 63 ? ~0ull : ((1ull << (pb + 1)) - 1ull));
                    if (bits) {
                        pe = 64 * w + 63 - __clzll((long long)bits);
                        break;
                    }
                    p = 64 * w - 1;
                }
            } else {
                pe = base;
            }
            S.prev_end_old = pe;
        }
    }
    // 4b. per-quotient new-group index and (insert) summed encoded lengths
    const unsigned NONE = 0xffffffffu;
    for (int y = tid; y < TQ; y += MT) {
        S.Lq[y] = 0;
        S.qfirst[y] = NONE;
    }
    __syncthreads();
    const bool old_ok = S.err == 0;
    for (uint64_t g0 = S.glo + tid; g0 < S.ghi; g0 += GB * MT) {
        // the loads of GB groups first, so that they are in flight together
        uint64_t fv[GB];
        uint32_t s0[GB], s1[GB];
#pragma unroll
        for (int u = 0; u < GB; u++) {
            const uint64_t g = g0 + (uint64_t)u * MT;
            if (g < S.ghi) {
                fv[u] = a.ufp[g];
                s0[u] = a.ustart[g];
                s1[u] = a.ustart[g + 1];
            }
        }
#pragma unroll
        for (int u = 0; u < GB; u++) {
            const uint64_t g = g0 + (uint64_t)u * MT;
            if (g < S.ghi) {
                uint32_t qo, rm;
                uint64_t cn;
                decode_group<R>(a, Q0, fv[u], s0[u], s1[u], qo, rm, cn);
                if (g - S.glo < gcap) gst[g - S.glo] = (qo << 21) | (rm << 5) | (unsigned)(cn < 31 ? cn : 31);
                atomicMin(&S.qfirst[qo], (unsigned)g);
                if (!a.del) {
                    atomicAdd(&S.Lq[qo], enc_len(cn, R));
                } else if (a.removed) {
                    const bool ho = old_ok && ((S.occ[qo >> 6] >> (qo & 63)) & 1ull);
                    if (!ho) a.removed[g] = 0;  // nothing stored to delete
                }
            }
        }
    }
    // 5 and 6 concern old runs only: a tile without any (kold is the same for
    // every thread) goes straight to the placement
    if (kold == 0) {
        if (tid == 0) {
            S.os0 = 0;
            S.oldlen = 0;
        }
    } else {
    if (tid == 0) {
        // 5. staged window of the old runs
        S.nmix = 0;
        if (kold > 0 && S.err == 0) {
            long long yfirst = -1;
            for (int w = 0; w < TBLK && yfirst < 0; w++)
                if (S.occ[w]) yfirst = Q0 + 64 * w + __ffsll((long long)S.occ[w]) - 1;
            long long os0 = yfirst > S.prev_end_old + 1 ? yfirst : S.prev_end_old + 1;
            long long oe = Q0 + S.oend[kold - 1];
            S.os0 = os0;
            long long len = oe - os0 + 1;
            S.oldlen = (unsigned)(len < OLDBUF ? len : OLDBUF);
        } else {
            S.os0 = 0;
            S.oldlen = 0;
        }
    }
    __syncthreads();
    {
        constexpr int OPT = (OLDBUF + MT - 1) / MT;
        const unsigned len = S.oldlen;
        const long long os0 = S.os0;
        uint32_t v[OPT];
#pragma unroll
        for (int u = 0; u < OPT; u++) {
            const unsigned p = tid + u * MT;
            if (p < len) v[u] = rd_slot<R>(a.rem_old, (uint64_t)(os0 + p));
        }
#pragma unroll
        for (int u = 0; u < OPT; u++) {
            const unsigned p = tid + u * MT;
            if (p < len) S.old[p] = (typename SlotIO<R>::T)v[u];
        }
    }
    __syncthreads();

    // 6. run length of every quotient: copy length for old-only runs, the summed
    // encodings for new-only runs, a full merge where both exist
    for (int y = tid; y < TQ; y += MT) {
        const bool ho = old_ok && ((S.occ[y >> 6] >> (y & 63)) & 1ull);
        const unsigned gf = S.qfirst[y];
        const bool hn = gf != NONE;
        if (!ho && !hn) continue;
        if (!ho) {
            if (a.del) S.Lq[y] = 0;
            continue;
        }
        const unsigned byte = (unsigned)(S.occ[y >> 6] >> ((y & 56))) & 0xffu;
        const unsigned k = S.kpre[y >> 3] + __popc(byte & ((1u << (y & 7)) - 1u));
        const long long pe = (k == 0) ? S.prev_end_old : (Q0 + S.oend[k - 1]);
        OldRun o;
        o.e = Q0 + S.oend[k];
        o.p = (Q0 + y) > pe + 1 ? (Q0 + y) : pe + 1;
        if (!hn) {
            S.Lq[y] = (unsigned)(o.e - o.p + 1);
        } else {
            // mixed runs are few and long to merge: listed, so that whole
            // warps take them together below (inline once the list is full)
            const unsigned slot = atomicAdd(&S.nmix, 1u);
            if (slot < MIXCAP) S.mix[slot] = (unsigned short)y;
            else S.Lq[y] = mixed_run<R, false>(S, a, Q0, y, 0);
        }
    }
    __syncthreads();
    {
        const unsigned nm = S.nmix < MIXCAP ? S.nmix : MIXCAP;
        for (unsigned i = tid; i < nm; i += MT) {
            const int y = S.mix[i];
            S.Lq[y] = mixed_run<R, false>(S, a, Q0, y, 0);
        }
    }
    }  // kold > 0
    __syncthreads();

    // 7. placement: thread tid owns quotients 8 tid .. 8 tid + 7
    const long long ybase = Q0 + (long long)tid * QPT;
    long long tA = NEG_INF, tB = 0;
#pragma unroll
    for (int c = 0; c < QPT; c++) {
        const unsigned L = S.Lq[tid * QPT + c];
        if (L) agg_combine(tA, tB, ybase + c + L - 1, L);
    }
    long long iA = tA, iB = tB;  // inclusive
    for (int o = 1; o < 32; o <<= 1) {
        long long pA = __shfl_up_sync(0xffffffffu, iA, o);
        long long pB = __shfl_up_sync(0xffffffffu, iB, o);
        if (lane >= o) {
            long long A = pA, Bs = pB;
            agg_combine(A, Bs, iA, iB);
            iA = A;
            iB = Bs;
        }
    }
    if (lane == 31) {
        S.wA[warp] = iA;
        S.wB[warp] = iB;
    }
    long long xA = __shfl_up_sync(0xffffffffu, iA, 1), xB = __shfl_up_sync(0xffffffffu, iB, 1);
    if (lane == 0) {
        xA = NEG_INF;
        xB = 0;
    }
    __syncthreads();
    {
        long long pA = NEG_INF, pB = 0;
        for (int w = 0; w < warp; w++) agg_combine(pA, pB, S.wA[w], S.wB[w]);
        agg_combine(pA, pB, xA, xB);
        xA = pA;
        xB = pB;
    }
    // 8. decoupled look-back over tiles, CTA-wide: MT predecessors per round.
    // One status word per tile: bits 62-63 flag (1 aggregate, 2 inclusive end);
    // aggregate payload (A - Q0 + 1) << 31 | B, with 0 in the A field for a tile
    // without runs; inclusive payload P + 1. A tile whose aggregate does not fit
    // publishes only its inclusive end.
    {
        const unsigned full = 0xffffffffu;
        __shared__ long long lbA[MT / 32], lbB[MT / 32], lbP;
        __shared__ int lb_incl;
        __shared__ unsigned lb_timeout;
        long long TA = NEG_INF, TB = 0;
        for (int w = 0; w < MT / 32; w++) agg_combine(TA, TB, S.wA[w], S.wB[w]);
        unsigned long long *st = a.ts + 1;
        const long long arel = (TA == NEG_INF) ? 0 : TA - Q0 + 1;
        const bool packable = TB < (1ll << 31) && arel >= 0 && arel < (1ll << 31);
        if (tid == 0) {
            lb_timeout = 0;
            if (tile > 0 && packable)
                atomicExch(&st[tile], (1ull << 62) | ((unsigned long long)arel << 31) | (unsigned long long)TB);
        }
        long long ein = -1;
        if (tile > 0) {
            long long gA = NEG_INF, gB = 0;  // composition of the newer tiles of earlier rounds
            long long jtop = (long long)tile - 1;
            while (true) {
                const long long j = jtop - tid;
                unsigned long long wd = 2ull << 62;  // before tile 0: inclusive end -1
                if (j >= 0) {
                    wd = ld_vol(&st[j]);
                    uint32_t spins = 0, ns = 32;
                    while ((wd >> 62) == 0) {
                        if (++spins > (SPIN_LIMIT >> 2)) {
                            lb_timeout = 1;
                            break;
                        }
                        __nanosleep(ns);
                        if (ns < 512) ns <<= 1;
                        wd = ld_vol(&st[j]);
                    }
                }
                const unsigned flag = (unsigned)(wd >> 62);
                if (tid == 0) lb_incl = MT;
                __syncthreads();
                if (flag == 2) atomicMin(&lb_incl, tid);
                __syncthreads();
                const int Lc = lb_incl;
                long long A = NEG_INF, Bv = 0;
                if (tid < Lc && flag == 1) {
                    const unsigned long long ar = (wd >> 31) & 0x7fffffffull;
                    Bv = (long long)(wd & 0x7fffffffull);
                    A = ar ? (long long)ar - 1 + j * TQ : NEG_INF;
                }
                // ordered composition, thread tid + 1 being the older tile
                for (int o = 1; o < 32; o <<= 1) {
                    long long oA = __shfl_down_sync(full, A, o), oB = __shfl_down_sync(full, Bv, o);
                    if (lane + o < 32) {
                        agg_combine(oA, oB, A, Bv);
                        A = oA;
                        Bv = oB;
                    }
                }
                if (lane == 0) {
                    lbA[warp] = A;
                    lbB[warp] = Bv;
                }
                if (tid == Lc) lbP = (long long)(wd & ((1ull << 62) - 1ull)) - 1;
                __syncthreads();
                long long WA = NEG_INF, WB = 0;
                for (int w = MT / 32 - 1; w >= 0; w--) agg_combine(WA, WB, lbA[w], lbB[w]);
                agg_combine(WA, WB, gA, gB);
                if (lb_timeout) {
                    if (tid == 0) atomicOr(&a.ctr->status, ST_TIMEOUT);
                    break;
                }
                if (Lc < MT) {
                    long long v = lbP + WB;
                    ein = v > WA ? v : WA;
                    break;
                }
                gA = WA;
                gB = WB;
                jtop -= MT;
            }
        }
        if (tid == 0) {
            long long v = ein + TB;
            long long P = v > TA ? v : TA;
            atomicExch(&st[tile], (2ull << 62) | (unsigned long long)(P + 1));
            S.ein = ein;
            S.tileP = P;
            atomicMax(&a.ctr->gqf_end, P);
            if (P >= (long long)a.nslots) atomicExch(&a.ctr->overflow, 1ull);
            long long w0 = Q0 > ein + 1 ? Q0 : ein + 1;
            long long w1 = slot_end > P + 1 ? slot_end : P + 1;
            if (w1 > (long long)a.nslots) w1 = (long long)a.nslots;
            if (w0 > w1) w0 = w1;
            S.w0 = w0;
            S.w1 = w1;
        }
    }
    __syncthreads();
    if (S.err) atomicOr(&a.ctr->status, ST_INTERNAL);
    if (a.dry) return;

    // 9. starts, runends, occupieds and offsets (thread tid: its 8 quotients)
    const long long w0 = S.w0, w1 = S.w1;
    const long long staged = (w1 - w0) < OUTBUF ? (w1 - w0) : OUTBUF;
    for (int p = tid; p < OUTBUF * (int)sizeof(S.out[0]) / 4; p += MT) reinterpret_cast<uint32_t *>(S.out)[p] = 0u;
    for (int p = tid; p < RWORDS; p += MT) S.rend[p] = 0ull;
    for (long long p = w0 + OUTBUF + tid; p < w1; p += MT) wr_slot<R>(a.rem_new, (uint64_t)p, 0u);
    __syncthreads();
    const long long wbase = w0 >> 6;
    long long e;
    {
        long long v = S.ein + xB;
        e = v > xA ? v : xA;
    }
    const long long e_thread_in = e;
    // runend bits go to the staged words when inside the staged window,
    // else straight to the new metadata
    auto flush_rend = [&](long long w, unsigned long long bits) {
        if (!bits) return;
        const long long wi = w - wbase;
        if ((64 * w + 63) - w0 < OUTBUF && wi >= 0 && wi < RWORDS) atomicOr(&S.rend[wi], bits);
        else atomicOr(&a.meta_new[w].rend, bits);
    };
    long long rw = -1;
    unsigned long long rbits = 0;
    uint32_t newbyte = 0;
    long long first_end = -1;
#pragma unroll
    for (int c = 0; c < QPT; c++) {
        const unsigned L = S.Lq[tid * QPT + c];
        if (!L) continue;
        const long long y = ybase + c;
        const long long start = y > e + 1 ? y : e + 1;
        const long long end = start + L - 1;
        S.qstart[tid * QPT + c] = (int)(start - Q0);
        if (end < (long long)a.nslots) {
            // a thread's run ends increase: OR them into one word at a time
            if ((end >> 6) != rw) {
                flush_rend(rw, rbits);
                rw = end >> 6;
                rbits = 0;
            }
            rbits |= 1ull << (end & 63);
        }
        e = end;
        newbyte |= 1u << c;
        if (c == 0) first_end = end;
    }
    flush_rend(rw, rbits);
    S.newocc[tid] = (unsigned char)newbyte;
    if ((tid & 7) == 0) {
        const uint64_t j = j0 + (tid >> 3);
        if (j < a.nblk) {
            const long long ref = (newbyte & 1u) ? first_end : e_thread_in;
            const long long o = ref - 64 * (long long)j;
            a.meta_new[j].off = (unsigned)(o > 0 ? o : 0);
        }
    }
    __syncthreads();

    // 10. write the runs: old-only runs are copied, mixed runs merged, and the
    // groups of new-only runs encoded by one thread each
    const bool listed = kold > 0 && S.nmix <= MIXCAP;  // every mixed run is in the list
    // old-only runs are copied by whole warps: a warp's 32 quotients lay
    // their runs end to end (a scan of their lengths) and every lane copies
    // every 32nd slot of the concatenation
    for (int y = tid; kold > 0 && y < TQ; y += MT) {  // (y - tid is the same for the whole CTA)
        const unsigned L = S.Lq[y];
        const bool ho = L && old_ok && ((S.occ[y >> 6] >> (y & 63)) & 1ull);
        const unsigned gf = S.qfirst[y];
        const long long start = Q0 + S.qstart[y];
        unsigned cl = 0;  // slots this lane's quotient copies
        long long op = 0;
        if (ho && gf == NONE) {
            const unsigned byte = (unsigned)(S.occ[y >> 6] >> ((y & 56))) & 0xffu;
            const unsigned k = S.kpre[y >> 3] + __popc(byte & ((1u << (y & 7)) - 1u));
            const long long pe = (k == 0) ? S.prev_end_old : (Q0 + S.oend[k - 1]);
            op = (Q0 + y) > pe + 1 ? (Q0 + y) : pe + 1;
            cl = L;
        } else if (ho && !listed) {
            mixed_run<R, true>(S, a, Q0, y, start);
        }
        unsigned incl = cl;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const unsigned excl = incl - cl;
        const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
        for (unsigned b0 = 0; b0 < total; b0 += 32) {
            const unsigned i = b0 + lane;
            // the last lane whose run starts at or before slot i of the concatenation
            int j = 0;
#pragma unroll
            for (int step = 16; step; step >>= 1) {
                const unsigned e = __shfl_sync(0xffffffffu, excl, (j + step) & 31);
                if (j + step < 32 && e <= i) j += step;
            }
            const unsigned ej = __shfl_sync(0xffffffffu, excl, j);
            const long long sj = __shfl_sync(0xffffffffu, op, j);
            const long long dj = __shfl_sync(0xffffffffu, start, j);
            if (i < total) put_slot<R>(S, a, dj + (i - ej), old_at<R>(S, a, sj + (i - ej)));
        }
    }
    if (listed) {
        for (unsigned i = tid; i < S.nmix; i += MT) {
            const int y = S.mix[i];
            if (S.Lq[y]) mixed_run<R, true>(S, a, Q0, y, Q0 + S.qstart[y]);
        }
    }
    if (!a.del) {
        // groups of new-only runs, one thread each, from the stage where it
        // holds them
        for (uint64_t g = S.glo + tid; g < S.ghi; g += MT) {
            uint32_t qo, rm;
            uint64_t cn;
            new_group<R>(S, a, Q0, (uint32_t)g, qo, rm, cn);
            const bool ho = old_ok && ((S.occ[qo >> 6] >> (qo & 63)) & 1ull);
            if (ho) continue;  // written by the merge above
            long long pos = Q0 + S.qstart[qo];
            for (uint32_t h = S.qfirst[qo]; h < (uint32_t)g; h++) {
                uint32_t q2, r2;
                uint64_t c2;
                new_group<R>(S, a, Q0, h, q2, r2, c2);
                pos += enc_len(c2, R);
            }
            put_group<R>(S, a, pos, rm, cn);
        }
    }
    __syncthreads();
    // flush staged remainders and runend words
    for (long long p = tid; p < staged; p += MT) wr_slot<R>(a.rem_new, (uint64_t)(w0 + p), S.out[p]);
    for (int p = tid; p < RWORDS; p += MT)
        if (S.rend[p]) atomicOr(&a.meta_new[wbase + p].rend, S.rend[p]);
    if (tid < TBLK && j0 + tid < a.nblk) {
        unsigned long long w = 0;
        for (int b = 0; b < 8; b++) w |= (unsigned long long)S.newocc[tid * 8 + b] << (8 * b);
        a.meta_new[j0 + tid].occ = w;
    }
}

// Tiles are taken from a counter in launch order, so every tile a look-back
// waits on has already been scheduled.
// Traced launches record their algorithmic bytes on the device: the old
// table read and the new one written (r / 8 + 1 / 2 bytes per slot each) and
// 12 bytes (fingerprint and start) per group read.
template <int R>
__device__ __forceinline__ void merge_units(unsigned long long *units, uint64_t slots, uint64_t groups)
{
    *units = (unsigned long long)(slots * (2 * R / 8 + 1) + 12 * groups);
}

template <int R>
__global__ void __launch_bounds__(MT, MERGE_CTAS) gqf_merge_kernel(MergeArgs a, unsigned long long *units)
{
    __shared__ MergeSmem<R> S;
    if (threadIdx.x == 0) {
        S.tile = (unsigned)atomicAdd(&a.ts[0], 1ull);
        S.err = 0;
        if (units && S.tile == 0) {
            const uint64_t m = *a.pm;
            merge_units<R>(units, a.nslots, m < a.m_limit ? m : a.m_limit);
        }
    }
    __syncthreads();
    merge_tile<R>(a, S, S.tile);
}

// Group merge: the tiles of all member filters, concatenated. tab[m] holds
// member m's arguments with `ts` and `tlo` already offset to its first tile,
// so the look-back of a member's tile stops at that member's first tile.
template <int R>
__global__ void __launch_bounds__(MT, MERGE_CTAS) gqf_merge_group_kernel(const MergeArgs *__restrict__ tab,
                                                             const uint32_t *__restrict__ tile_member,
                                                             unsigned long long *tctr, uint64_t slots,
                                                             const uint32_t *pm, unsigned long long *units)
{
    __shared__ MergeSmem<R> S;
    __shared__ MergeArgs A;
    if (threadIdx.x == 0) {
        S.tile = (unsigned)atomicAdd(tctr, 1ull);
        S.err = 0;
        if (units && S.tile == 0) merge_units<R>(units, slots, *pm);
    }
    __syncthreads();
    static_assert(sizeof(MergeArgs) % 8 == 0, "MergeArgs copies as 64-bit words");
    {
        const unsigned long long *src = reinterpret_cast<const unsigned long long *>(tab + tile_member[S.tile]);
        unsigned long long *dst = reinterpret_cast<unsigned long long *>(&A);
        for (int w = threadIdx.x; w < (int)(sizeof(MergeArgs) / 8); w += MT) dst[w] = src[w];
    }
    __syncthreads();
    merge_tile<R>(A, S, S.tile - A.tile0);
}

// first group of every tile: successor search of the tile's first fingerprint
// in the sorted groups (paper Sec. 5.3, "the starts of buffers are set using
// successor search")
__global__ void gqf_tile_ranges(const uint64_t *__restrict__ ufp, const uint32_t *pm, uint64_t m_limit,
                                uint64_t N, uint32_t r, uint64_t ntiles, uint32_t *tlo)
{
    const uint64_t m = min((uint64_t)*pm, m_limit);
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t <= ntiles;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t q0 = t * TQ;
        const uint64_t key = q0 >= N ? (N << r) : (q0 << r);
        uint64_t lo = 0, hi = m;
        while (lo < hi) {
            uint64_t mid = (lo + hi) >> 1;
            if (ufp[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        tlo[t] = (uint32_t)lo;
    }
}

// ---------------------------------------------------------------------------
// In-place bulk delete, the paper's even-odd regions (Sec. 6.4 with Sec. 5.3):
// removing copies from a run only shifts the rest of its cluster left, never
// past a home slot, so a delete is local to its cluster. One thread per
// region of RQ quotients applies the region's groups largest first; even
// regions run first, then odd ones. A read-only pre-check measures how far
// past its home slot every affected cluster reaches; RQ is then the smallest
// power of two >= RQ_MIN covering that reach, so that every cluster touched
// from region r ends before region r + 2 and two threads of a phase never
// touch the same slots or metadata words. Reaches above RQ_MAX (long
// clusters at high load) take the merge instead.
// ---------------------------------------------------------------------------
static constexpr long long RQ_MIN = 256;     // quotients per delete region, smallest (a multiple of 64)
static constexpr long long RQ_MAX = 1 << 16;
// In-place batches are worth it only while each region thread has few groups
// to apply one after another; past that the merge, whose cost does not grow
// with the batch, is faster. The limit on the mean groups per region is a
// tuning knob (gqf_region_groups, 8 by default).


// read-only: per region, the slots its groups add, and whether the data they
// push stays before the region after next (two slots of margin) and before
// the table's end
template <int R>
__global__ void gqf_insert_precheck(GView g, const uint64_t *__restrict__ ufp, const uint32_t *__restrict__ ustart,
                                    const uint32_t *__restrict__ rlo, uint64_t nreg, uint64_t rq,
                                    unsigned long long *bad)
{
    for (uint64_t reg = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; reg < nreg;
         reg += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t k0 = rlo[reg], k1 = rlo[reg + 1];
        if (k0 == k1) continue;
        const long long r0 = (long long)(reg * rq);
        long long limit = (long long)((reg + 2) * rq) - 2;
        if (limit > g.nslots - 1) limit = g.nslots - 1;
        long long need = 0;
        for (uint32_t k = k0; k < k1; k++) {
            const uint64_t fp = ufp[k];
            long long s, e, p;
            uint64_t c_old;
            uint32_t ol;
            if (!gv_locate<R>(g, (long long)(fp >> R), (uint32_t)(fp & ((1ull << R) - 1ull)), r0, s, e, p, c_old, ol)) {
                atomicExch(bad, 1ull);
                return;
            }
            need += (long long)enc_len(c_old + (uint64_t)(ustart[k + 1] - ustart[k]), R) - (long long)ol;
        }
        // the data all of them push stops, at the latest, where the data pushed
        // from the last one stops
        if (gv_push_end(g, (long long)(ufp[k1 - 1] >> R), need, r0, limit) < 0) atomicExch(bad, 1ull);
    }
}

template <int R>
__global__ void gqf_insert_phase(GView g, const uint64_t *__restrict__ ufp, const uint32_t *__restrict__ ustart,
                                 const uint32_t *__restrict__ rlo, uint64_t nreg, uint64_t rq, int phase,
                                 unsigned long long *status)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t reg = 2 * i + (uint64_t)phase;
        if (reg >= nreg) return;
        const long long r0 = (long long)(reg * rq);
        for (uint32_t k = rlo[reg]; k < rlo[reg + 1]; k++)
            if (!gv_insert<R>(g, ufp[k], ustart[k + 1] - ustart[k], r0)) atomicOr(status, ST_INTERNAL);
    }
}

// first group of every delete region (successor search)
__global__ void gqf_region_ranges(const uint64_t *__restrict__ ufp, const uint32_t *pm, uint64_t N, uint32_t r,
                                  uint64_t rq, uint64_t nreg, uint32_t *rlo)
{
    const uint64_t m = *pm;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t <= nreg;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t q0 = t * rq;
        const uint64_t key = q0 >= N ? (N << r) : (q0 << r);
        uint64_t lo = 0, hi = m;
        while (lo < hi) {
            uint64_t mid = (lo + hi) >> 1;
            if (ufp[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        rlo[t] = (uint32_t)lo;
    }
}

// read-only: the largest reach (cluster tail end - home slot + 1) over the
// groups to delete, capped just above RQ_MAX
template <int R>
__global__ void gqf_delete_precheck(GView g, const uint64_t *__restrict__ ufp, const uint32_t *pm,
                                    unsigned long long *reach)
{
    const uint64_t m = *pm;
    unsigned long long mine = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
        const long long x = (long long)(ufp[i] >> R);
        if (x >= g.N || !gv_occ(g, x)) continue;
        long long prev = gv_runend_of(g, x), y = x;
        while (prev >= 0 && prev - x < RQ_MAX) {
            const long long yn = gv_next_occ(g, y, prev + 1);
            if (yn < 0) break;
            prev = gv_next_runend(g, prev + 1);
            y = yn;
        }
        const unsigned long long r = prev < 0 ? (unsigned long long)RQ_MAX + 1 : (unsigned long long)(prev - x + 1);
        mine = r > mine ? r : mine;
    }
    if (mine) atomicMax(reach, mine);
}

template <int R>
__global__ void gqf_delete_phase(GView g, const uint64_t *__restrict__ ufp, const uint32_t *__restrict__ ustart,
                                 const uint32_t *__restrict__ rlo, uint64_t nreg, int phase, uint32_t *removed,
                                 unsigned long long *status)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t reg = 2 * i + (uint64_t)phase;
        if (reg >= nreg) return;
        for (uint32_t k = rlo[reg + 1]; k > rlo[reg]; k--) {
            const uint32_t gi = k - 1;
            const uint64_t rmv = gv_delete<R>(g, ufp[gi], ustart[gi + 1] - ustart[gi], status);
            if (removed) removed[gi] = (uint32_t)rmv;
        }
    }
}

// ---------------------------------------------------------------------------
// Counted insert: each key stands for its count of copies
// ---------------------------------------------------------------------------
// ws[j] = count of sorted element j: counts[sidx[j]], or counts[j] when the
// sort carried the counts (sidx null); the 64-bit total and whether some
// count was 0 go to *total and *zero
__global__ void __launch_bounds__(256) gqf_counts_sorted(const uint32_t *__restrict__ counts,
                                                         const uint32_t *__restrict__ sidx, uint64_t n,
                                                         uint32_t *__restrict__ ws, unsigned long long *total,
                                                         unsigned long long *zero)
{
    unsigned long long sum = 0;
    bool z = false;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = sidx ? counts[sidx[j]] : counts[j];
        ws[j] = c;
        sum += c;
        z |= c == 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    const bool anyz = __any_sync(0xffffffffu, z);
    if ((threadIdx.x & 31) == 0) {
        if (sum) atomicAdd(total, sum);
        if (anyz) atomicOr(zero, 1ull);
    }
}

// cstart[g] = copies in the groups before g (g = 0 .. m), from the exclusive
// scan of the per-element counts and their total (below 2^32, checked on the
// host): the group counts the merge and the in-place insert read
__global__ void __launch_bounds__(256) gqf_group_counts(const uint32_t *__restrict__ scanned,
                                                        const uint32_t *__restrict__ ustart, const uint32_t *pm,
                                                        const unsigned long long *total,
                                                        uint32_t *__restrict__ cstart)
{
    const uint64_t m = *pm;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g <= m; g += (uint64_t)gridDim.x * blockDim.x)
        cstart[g] = g < m ? scanned[ustart[g]] : (uint32_t)*total;
}

// ---------------------------------------------------------------------------
// per-key status after a batch
// ---------------------------------------------------------------------------
// run_of[i] = group of sorted element i
__global__ void gqf_status_kernel(uint64_t n, const uint32_t *__restrict__ run_of, const uint32_t *__restrict__ ustart,
                                  const uint32_t *__restrict__ sidx, const uint32_t *__restrict__ removed,
                                  uint64_t m_keep, int del, uint8_t *status)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t g = run_of[i];
        uint8_t s;
        if (del) s = (i - ustart[g]) < removed[g] ? FILTER_KEY_OK : FILTER_KEY_NOT_FOUND;
        else s = (g < m_keep) ? FILTER_KEY_OK : FILTER_KEY_FULL;
        status[sidx[i]] = s;
    }
}

// keys of the groups past the kept prefix were rejected
__global__ void gqf_account_full(DevCounters *ctr, const uint32_t *ustart, uint64_t m_keep, uint64_t n)
{
    uint64_t kept = m_keep ? ustart[m_keep] : 0;
    if (kept < n) {
        atomicAdd(&ctr->failed, (unsigned long long)(n - kept));
        atomicOr(&ctr->status, ST_FULL);
    }
}

// ---------------------------------------------------------------------------
// count / query
// ---------------------------------------------------------------------------
// stored count of fingerprint fp (0 if absent)
// The run of occupied quotient x: it ends at the d-th run end from the
// offset of x's block, d counting the block's occupied quotients up to x
// (bit 0 excluded, which the offset itself covers); it starts one past the
// previous run end, or at x. False if the run ends could not be found.
__device__ __forceinline__ bool locate_run(uint64_t x, const Meta *__restrict__ meta, uint64_t nblk, long long &start,
                                           long long &end)
{
    const uint64_t j = x >> 6;
    const unsigned long long occ = __ldg(&meta[j].occ);
    const long long base = (long long)(64 * j) + (long long)__ldg(&meta[j].off);
    const unsigned sh = (unsigned)(x & 63);
    const unsigned long long upto = (sh == 63) ? ~0ull : ((1ull << (sh + 1)) - 1ull);
    int d = __popcll(occ & upto & ~1ull);
    end = base;
    if (d > 0) {
        long long w = base >> 6;
        unsigned bsh = (unsigned)(base & 63);
        unsigned long long bits = (bsh == 63) ? 0ull : (__ldg(&meta[w].rend) & (~0ull << (bsh + 1)));
        while (true) {
            int pc = __popcll(bits);
            if (pc >= d) {
                for (int k = 1; k < d; k++) bits &= bits - 1;
                end = 64 * w + __ffsll((long long)bits) - 1;
                break;
            }
            d -= pc;
            if (++w >= (long long)nblk) return false;
            bits = __ldg(&meta[w].rend);
        }
    }
    // start: one past the last runend in [x, end - 1], else x
    start = (long long)x;
    long long p = end - 1;
    while (p >= (long long)x) {
        long long w = p >> 6;
        unsigned long long bits = __ldg(&meta[w].rend);
        unsigned pb = (unsigned)(p & 63);
        bits &= (pb == 63) ? ~0ull : ((1ull << (pb + 1)) - 1ull);
        if (64 * w < (long long)x) bits &= ~0ull << (x & 63);
        if (bits) {
            start = 64 * w + 63 - __clzll((long long)bits) + 1;
            break;
        }
        p = 64 * w - 1;
    }
    return true;
}

// the group at slot q of a run ending at `end`: remainder, count, slots used
template <int R>
__device__ __forceinline__ uint32_t group_at(const uint8_t *__restrict__ rem, long long q, long long end,
                                             uint64_t &cnt, uint32_t &len)
{
    const uint32_t s = rd_slot<R>(rem, (uint64_t)q);
    cnt = 1;
    len = 1;
    if (q + 2 <= end && rd_slot<R>(rem, (uint64_t)(q + 1)) == s) {
        uint32_t nd = rd_slot<R>(rem, (uint64_t)(q + 2));
        if (q + 2 + (long long)nd > end) nd = (uint32_t)(end - q - 2);
        uint64_t acc = 0;
        for (uint32_t dd = 0; dd < nd; dd++) acc = (acc << R) | rd_slot<R>(rem, (uint64_t)(q + 3 + dd));
        cnt = acc + 2;
        len = 3 + nd;
    }
    return s;
}

template <int R>
__device__ __forceinline__ uint64_t count_fp(const uint64_t fp, const Meta *__restrict__ meta,
                                             const uint8_t *__restrict__ rem, const uint64_t nblk)
{
    const uint64_t x = fp >> R;
    const uint32_t v = (uint32_t)(fp & ((1ull << R) - 1ull));
    const unsigned long long occ = __ldg(&meta[x >> 6].occ);
    if (!((occ >> (x & 63)) & 1ull)) return 0;
    long long start, end;
    if (!locate_run(x, meta, nblk, start, end)) return 0;
    for (long long q = start; q <= end;) {
        uint64_t cc;
        uint32_t len;
        const uint32_t s = group_at<R>(rem, q, end, cc, len);
        if (s == v) return cc;
        if (s > v) return 0;
        q += len;
    }
    return 0;
}

// Enumeration: one thread per 64-slot block walks the runs of its occupied
// quotients in order and their groups in remainder order, so the groups come
// out in fingerprint order. COUNT pass: groups per block; WRITE pass: the
// groups at their scanned positions (those below cap).
template <int R, bool WRITE>
__global__ void gqf_enum_kernel(const Meta *__restrict__ meta, const uint8_t *__restrict__ rem, uint64_t nblk,
                                uint64_t N, uint32_t *per_block, uint64_t *fps, uint64_t *counts, uint64_t cap)
{
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < nblk; j += (uint64_t)gridDim.x * blockDim.x) {
        unsigned long long occ = __ldg(&meta[j].occ);
        uint64_t k = WRITE ? per_block[j] : 0;
        while (occ) {
            const uint64_t x = 64 * j + (uint64_t)(__ffsll((long long)occ) - 1);
            occ &= occ - 1;
            if (x >= N) break;
            long long start, end;
            if (!locate_run(x, meta, nblk, start, end)) break;
            for (long long q = start; q <= end;) {
                uint64_t cc;
                uint32_t len;
                const uint32_t s = group_at<R>(rem, q, end, cc, len);
                if (WRITE && k < cap) {
                    fps[k] = (x << R) | s;
                    counts[k] = cc;
                }
                k++;
                q += len;
            }
        }
        if (!WRITE) per_block[j] = (uint32_t)k;
    }
}

template <int R>
__global__ void __launch_bounds__(256) gqf_count_kernel(const uint64_t *__restrict__ keys, uint64_t n, PHash H,
                                                        const Meta *__restrict__ meta,
                                                        const uint8_t *__restrict__ rem, uint64_t nblk,
                                                        uint64_t *counts, uint8_t *found)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        // keys and answers stream past the L2, which keeps the table
        const uint64_t c = count_fp<R>(fingerprint(__ldcs(keys + i), H), meta, rem, nblk);
        if (counts) __stcs(reinterpret_cast<unsigned long long *>(counts + i), (unsigned long long)c);
        if (found) __stcs(found + i, (uint8_t)(c ? 1 : 0));
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static uint64_t tail_slots(uint32_t q)
{
    uint64_t N = 1ull << q;
    uint64_t s = ((1072ull * q + 63) / 64) * 64;
    if (s > N) s = N;
    if (s < 64) s = 64;
    return s;
}

// entries of the range array: one per merge tile or per smallest region, plus one
uint64_t gqf_tile_lo_words(const GqfState &Q)
{
    const uint64_t nreg = (Q.N + RQ_MIN - 1) / RQ_MIN;
    return (Q.ntiles > nreg ? Q.ntiles : nreg) + 1;
}

int gqf_setup(filter *F, uint64_t &table_bytes, uint64_t &scratch_bytes, bool plan_only)
{
    const filter_config &c = F->cfg;
    if ((c.tag_bits != 8 && c.tag_bits != 16) || c.block_slots) return FILTER_ERR_ARG;
    if (c.value_bits != 0) return FILTER_ERR_ARG;  // values ride on the counters
    if (c.log2_slots < 6 || c.log2_slots > 36 || c.log2_slots + c.tag_bits > 64) return FILTER_ERR_ARG;
    GqfState &Q = F->gqf;
    Q.q = c.log2_slots;
    Q.r = c.tag_bits;
    Q.p = Q.q + Q.r;
    Q.N = 1ull << Q.q;
    Q.S = tail_slots(Q.q);
    Q.nslots = Q.N + Q.S;
    Q.nblk = Q.nslots / 64;
    Q.ntiles = (Q.nblk + TBLK - 1) / TBLK;
    Q.H = phash_of(Q.p, c.hash_seed);
    const uint64_t M = c.max_batch ? c.max_batch : 1;
    if (M >= (1ull << 30)) return FILTER_ERR_ARG;  // 30-bit counts in the sort and group arrays
    const uint64_t metaB = Q.nblk * 32, remB = Q.nslots * (Q.r / 8);
    // every buffer is listed once: the same list sizes the arena (plan) and
    // carves it (allocation)
    uint64_t bytes = 0;
    Arena &A = F->arena;
    auto piece = [&](auto *&ptr, uint64_t count) {
        using T = typename std::remove_reference<decltype(*ptr)>::type;
        const uint64_t b = (count * sizeof(T) + 255) & ~255ull;
        bytes += b;
        if (!plan_only) ptr = A.take<T>(count);
    };
    for (int b = 0; b < 2; b++) {
        piece(Q.meta[b], metaB);
        piece(Q.rem[b], remB);
    }
    Q.nlocks = (Q.N + GQF_LOCK_REGION - 1) / GQF_LOCK_REGION;
    piece(Q.locks, Q.nlocks * GQF_LOCK_STRIDE);
    table_bytes = bytes;
    uint64_t scan_n = radix_tmp_words(M);
    if (M + 1 > scan_n) scan_n = M + 1;
    piece(Q.fp_a, M);
    
    piece(Q.fp_b, M);
    piece(Q.fp_c, M);
    piece(Q.ufp, M);
    piece(Q.idx_a, M);
    piece(Q.idx_b, M);
    piece(Q.idx_c, M);
    piece(Q.ustart, M + 1);
    piece(Q.flags, M + 1);
    piece(Q.removed, M);
    piece(Q.tile_state, Q.ntiles * 4 + 2);
    piece(Q.tile_lo, gqf_tile_lo_words(Q));
    piece(Q.radix_tmp, radix_tmp_words(M));
    piece(F->scan_tmp, scan_tmp_words(scan_n));
    scratch_bytes = bytes - table_bytes;
    Q.cur = 0;
    Q.merge_only = false;
    return FILTER_OK;
}

int gqf_clear(filter *F, cudaStream_t st)
{
    GqfState &Q = F->gqf;
    for (int b = 0; b < 2; b++) {
        GF_CUDA(cudaMemsetAsync(Q.meta[b], 0, Q.nblk * 32, st));
        GF_CUDA(cudaMemsetAsync(Q.rem[b], 0, Q.nslots * (Q.r / 8), st));
    }
    Q.cur = 0;
    GF_CUDA(cudaMemsetAsync(Q.locks, 0, Q.nlocks * GQF_LOCK_STRIDE * 4, st));
    GF_CUDA(cudaMemsetAsync(F->ctr, 0, sizeof(DevCounters), st));
    return FILTER_OK;
}

// sort + reduce: leaves groups in ufp / ustart, group count in flags[n]. The
// sort carries the batch indices (need_idx: statuses) or a caller's per-key
// values (vals, without statuses); either ends in idx_b in sorted order.
static void gqf_prepare(filter *F, const uint64_t *keys, uint64_t n, bool need_idx, cudaStream_t st,
                        uint32_t **sorted_idx, const uint32_t *vals = nullptr)
{
    GqfState &Q = F->gqf;
    fingerprint_for_sort(keys, n, Q.H, Q.fp_a, need_idx ? Q.idx_a : nullptr, Q.p, Q.radix_tmp, st);
    radix_sort_u64(Q.fp_a, Q.fp_b, Q.fp_c, need_idx ? Q.idx_a : vals, Q.idx_b, Q.idx_c, n, Q.p, Q.radix_tmp,
                   F->scan_tmp, F->ctr, st, true);
    // groups: flags[n] = their number; flags[i] = the group of sorted element i (statuses only)
    rle_sorted_u64(Q.fp_b, n, Q.ufp, Q.ustart, need_idx ? Q.flags : nullptr, Q.flags + n, F->scan_tmp, F->ctr, st);
    *sorted_idx = Q.idx_b;
}

// cstart: group g adds (or removes) cstart[g + 1] - cstart[g] copies
static int gqf_merge(filter *F, const uint32_t *cstart, uint64_t n, uint64_t m_limit, int del, int dry,
                     cudaStream_t st)
{
    GqfState &Q = F->gqf;
    const int nb = Q.cur ^ 1;
    MergeArgs a;
    a.meta_old = reinterpret_cast<const Meta *>(Q.meta[Q.cur]);
    a.rem_old = Q.rem[Q.cur];
    a.meta_new = reinterpret_cast<Meta *>(Q.meta[nb]);
    a.rem_new = Q.rem[nb];
    a.ufp = Q.ufp;
    a.ustart = cstart;
    a.pm = Q.flags + n;
    a.tlo = Q.tile_lo;
    a.m_limit = m_limit;
    a.removed = del ? Q.removed : nullptr;
    a.ts = Q.tile_state;
    a.ctr = F->ctr;
    a.N = Q.N;
    a.nslots = Q.nslots;
    a.nblk = Q.nblk;
    a.ntiles = Q.ntiles;
    a.fmask = ~0ull;
    a.tile0 = 0;
    a.r = Q.r;
    a.del = del;
    a.dry = dry;
    GF_CUDA(cudaMemsetAsync(Q.tile_state, 0, (Q.ntiles * 4 + 2) * 8, st));
    GF_CUDA(cudaMemsetAsync(&F->ctr->overflow, 0, 8, st));
    GF_CUDA(cudaMemsetAsync(&F->ctr->gqf_end, 0xff, 8, st));  // -1
    if (!dry) GF_CUDA(cudaMemsetAsync(Q.meta[nb], 0, Q.nblk * 32, st));
    {
        gf::TraceScope ts_("gqf_tile_ranges", Q.ntiles + 1, st);
        gqf_tile_ranges<<<grid_for(Q.ntiles + 1, 256, 4), 256, 0, st>>>(Q.ufp, Q.flags + n, m_limit, Q.N, Q.r,
                                                                       Q.ntiles, Q.tile_lo);
    }
    {
        gf::TraceScope ts_("gqf_merge_kernel", 0, st, true);
        if (Q.r == 8) gqf_merge_kernel<8><<<(unsigned)Q.ntiles, MT, 0, st>>>(a, ts_.units());
        else gqf_merge_kernel<16><<<(unsigned)Q.ntiles, MT, 0, st>>>(a, ts_.units());
    }
    GF_CUDA(cudaGetLastError());
    return FILTER_OK;
}

template <class T>
static int read_dev(const T *d, T *h, cudaStream_t st)
{
    GF_CUDA(cudaMemcpyAsync(h, d, sizeof(T), cudaMemcpyDeviceToHost, st));
    GF_CUDA(cudaStreamSynchronize(st));
    return FILTER_OK;
}

// Small batches go in place over even-odd regions; `done` is false when the
// pre-check found, at every region size tried, a region whose inserts could
// reach the region after next (or the table's end).
static int gqf_insert_in_place(filter *F, const uint32_t *cstart, uint64_t n, uint32_t m, cudaStream_t st,
                               bool &done)
{
    GqfState &Q = F->gqf;
    done = false;
    GView g{reinterpret_cast<Meta *>(Q.meta[Q.cur]), Q.rem[Q.cur], (long long)Q.N, (long long)Q.nslots,
            (long long)Q.nblk};
    int rc = FILTER_OK;
    // a few region sizes, growing fourfold; dense batches go to the merge
    for (uint64_t rq = RQ_MIN; rq <= (uint64_t)RQ_MAX / 4 && (uint64_t)m * rq <= gqf_region_groups(F->tune) * Q.N; rq <<= 2) {
        const uint64_t nreg = (Q.N + rq - 1) / rq;
        {
            gf::TraceScope ts_("gqf_region_ranges", nreg + 1, st);
            gqf_region_ranges<<<grid_for(nreg + 1, 256, 4), 256, 0, st>>>(Q.ufp, Q.flags + n, Q.N, Q.r, rq, nreg,
                                                                         Q.tile_lo);
        }
        GF_CUDA(cudaMemsetAsync(&F->ctr->overflow, 0, 8, st));
        {
            gf::TraceScope ts_("gqf_insert_precheck", nreg, st);
            if (Q.r == 8)
                gqf_insert_precheck<8><<<grid_for(nreg, 128, 8), 128, 0, st>>>(g, Q.ufp, cstart, Q.tile_lo, nreg, rq,
                                                                               &F->ctr->overflow);
            else
                gqf_insert_precheck<16><<<grid_for(nreg, 128, 8), 128, 0, st>>>(g, Q.ufp, cstart, Q.tile_lo, nreg, rq,
                                                                                &F->ctr->overflow);
        }
        unsigned long long bad = 0;
        if ((rc = read_dev(&F->ctr->overflow, &bad, st))) return rc;
        if (bad) continue;
        const uint64_t half = (nreg + 1) / 2;
        for (int ph = 0; ph < 2; ph++) {
            gf::TraceScope ts_("gqf_insert_phase", half, st);
            if (Q.r == 8)
                gqf_insert_phase<8><<<grid_for(half, 128, 8), 128, 0, st>>>(g, Q.ufp, cstart, Q.tile_lo, nreg, rq, ph,
                                                                            &F->ctr->status);
            else
                gqf_insert_phase<16><<<grid_for(half, 128, 8), 128, 0, st>>>(g, Q.ufp, cstart, Q.tile_lo, nreg, rq,
                                                                             ph, &F->ctr->status);
        }
        GF_CUDA(cudaGetLastError());
        done = true;
        return FILTER_OK;
    }
    return FILTER_OK;
}

int gqf_insert(filter *F, const uint64_t *keys, const uint32_t *counts, uint64_t n, uint8_t *status,
               cudaStream_t st)
{
    if (n == 0) return FILTER_OK;
    GqfState &Q = F->gqf;
    uint32_t *sidx = nullptr;
    // counts without statuses ride through the sort in place of the indices
    const bool carry = counts != nullptr && status == nullptr;
    gqf_prepare(F, keys, n, status != nullptr, st, &sidx, carry ? counts : nullptr);
    int rc;
    // the copies each group adds: its keys, or the sum of their counts
    const uint32_t *cstart = Q.ustart;
    if (counts) {
        // fp_a and fp_c (2 words per key each) are free once the sort is done
        uint32_t *ws = reinterpret_cast<uint32_t *>(Q.fp_c), *cs = reinterpret_cast<uint32_t *>(Q.fp_a);
        GF_CUDA(cudaMemsetAsync(&F->ctr->overflow, 0, 8, st));
        GF_CUDA(cudaMemsetAsync(&F->ctr->wflag, 0, 8, st));
        {
            gf::TraceScope ts_(carry ? "gqf_counts_sorted" : "gqf_counts_gather", n, st);
            gqf_counts_sorted<<<grid_for(n, 256, 8), 256, 0, st>>>(carry ? Q.idx_b : counts, carry ? nullptr : sidx,
                                                                   n, ws, &F->ctr->overflow, &F->ctr->wflag);
        }
        unsigned long long total = 0, zero = 0;
        if ((rc = read_dev(&F->ctr->overflow, &total, st))) return rc;
        if ((rc = read_dev(&F->ctr->wflag, &zero, st))) return rc;
        if (zero || total >= (1ull << 32)) return FILTER_ERR_ARG;  // nothing was written
        exclusive_scan_u32(ws, ws, n, F->scan_tmp, F->ctr, st);
        {
            gf::TraceScope ts_("gqf_group_counts", n, st);
            gqf_group_counts<<<grid_for(n + 1, 256, 8), 256, 0, st>>>(ws, Q.ustart, Q.flags + n, &F->ctr->overflow,
                                                                      cs);
        }
        GF_CUDA(cudaGetLastError());
        cstart = cs;
    }
    // small batches: in place, region by region; larger ones: the merge
    {
        uint32_t m = 0;
        if ((rc = read_dev(Q.flags + n, &m, st))) return rc;
        if ((uint64_t)m * RQ_MIN <= gqf_region_groups(F->tune) * Q.N && !Q.merge_only) {
            bool done = false;
            if ((rc = gqf_insert_in_place(F, cstart, n, m, st, done))) return rc;
            if (done) {
                if (status) {
                    gf::TraceScope ts_("gqf_status_kernel", n, st);
                    gqf_status_kernel<<<grid_for(n, 256, 8), 256, 0, st>>>(n, Q.flags, Q.ustart, sidx, Q.removed,
                                                                          ~0ull, 0, status);
                }
                GF_CUDA(cudaGetLastError());
                return FILTER_OK;
            }
        }
    }
    rc = gqf_merge(F, cstart, n, ~0ull, 0, 0, st);
    if (rc) return rc;
    unsigned long long ovf = 0;
    if ((rc = read_dev(&F->ctr->overflow, &ovf, st))) return rc;
    uint64_t m_keep = ~0ull;
    if (ovf) {
        // keep the longest prefix of the sorted groups that fits (dry runs)
        uint32_t m = 0;
        if ((rc = read_dev(Q.flags + n, &m, st))) return rc;
        uint64_t lo = 0, hi = m;  // lo fits, hi does not
        while (hi - lo > 1) {
            uint64_t mid = (lo + hi) / 2;
            if ((rc = gqf_merge(F, cstart, n, mid, 0, 1, st))) return rc;
            unsigned long long o2 = 0;
            if ((rc = read_dev(&F->ctr->overflow, &o2, st))) return rc;
            if (o2) hi = mid;
            else lo = mid;
        }
        m_keep = lo;
        if ((rc = gqf_merge(F, cstart, n, m_keep, 0, 0, st))) return rc;
        {
            gf::TraceScope ts_("gqf_account_full", 1, st);
            gqf_account_full<<<1, 1, 0, st>>>(F->ctr, Q.ustart, m_keep, n);
        }
        GF_CUDA(cudaGetLastError());
    }
    Q.cur ^= 1;
    if (status) {
        {
            gf::TraceScope ts_("gqf_status_kernel", n, st);
            gqf_status_kernel<<<grid_for(n, 256, 8), 256, 0, st>>>(n, Q.flags, Q.ustart, sidx, Q.removed, m_keep, 0,
                                                                  status);
        }
        GF_CUDA(cudaGetLastError());
    }
    return FILTER_OK;
}

int gqf_remove(filter *F, const uint64_t *keys, uint64_t n, uint8_t *status, cudaStream_t st)
{
    if (n == 0) return FILTER_OK;
    GqfState &Q = F->gqf;
    uint32_t *sidx = nullptr;
    gqf_prepare(F, keys, n, status != nullptr, st, &sidx);
    int rc = FILTER_OK;
    // small batches: in place, cluster by cluster; large ones: full merge
    uint32_t m = 0;
    if ((rc = read_dev(Q.flags + n, &m, st))) return rc;
    bool done = false;
    if ((uint64_t)m * RQ_MIN <= gqf_region_groups(F->tune) * Q.N) {
        GView g{reinterpret_cast<Meta *>(Q.meta[Q.cur]), Q.rem[Q.cur], (long long)Q.N, (long long)Q.nslots,
                (long long)Q.nblk};
        GF_CUDA(cudaMemsetAsync(&F->ctr->overflow, 0, 8, st));
        {
            gf::TraceScope ts_("gqf_delete_precheck", m, st);
            if (Q.r == 8) gqf_delete_precheck<8><<<grid_for(m, 256, 8), 256, 0, st>>>(g, Q.ufp, Q.flags + n, &F->ctr->overflow);
            else gqf_delete_precheck<16><<<grid_for(m, 256, 8), 256, 0, st>>>(g, Q.ufp, Q.flags + n, &F->ctr->overflow);
        }
        unsigned long long reach = 0;
        if ((rc = read_dev(&F->ctr->overflow, &reach, st))) return rc;
        uint64_t rq = RQ_MIN;
        while ((unsigned long long)rq < reach) rq <<= 1;
        if (rq <= (uint64_t)RQ_MAX && (uint64_t)m * rq <= gqf_region_groups(F->tune) * Q.N) {
            const uint64_t nreg = (Q.N + rq - 1) / rq;
            {
                gf::TraceScope ts_("gqf_region_ranges", nreg + 1, st);
                gqf_region_ranges<<<grid_for(nreg + 1, 256, 4), 256, 0, st>>>(Q.ufp, Q.flags + n, Q.N, Q.r, rq, nreg,
                                                                             Q.tile_lo);
            }
            const uint64_t half = (nreg + 1) / 2;
            for (int ph = 0; ph < 2; ph++) {
                gf::TraceScope ts_("gqf_delete_phase", half, st);
                if (Q.r == 8)
                    gqf_delete_phase<8><<<grid_for(half, 128, 8), 128, 0, st>>>(g, Q.ufp, Q.ustart, Q.tile_lo, nreg, ph,
                                                                                status ? Q.removed : nullptr, &F->ctr->status);
                else
                    gqf_delete_phase<16><<<grid_for(half, 128, 8), 128, 0, st>>>(g, Q.ufp, Q.ustart, Q.tile_lo, nreg, ph,
                                                                                 status ? Q.removed : nullptr, &F->ctr->status);
            }
            GF_CUDA(cudaGetLastError());
            done = true;
        }
    }
    if (!done) {
        if ((rc = gqf_merge(F, Q.ustart, n, ~0ull, 1, 0, st))) return rc;
        Q.cur ^= 1;
    }
    if (status) {
        {
            gf::TraceScope ts_("gqf_status_kernel", n, st);
            gqf_status_kernel<<<grid_for(n, 256, 8), 256, 0, st>>>(n, Q.flags, Q.ustart, sidx, Q.removed, 0, 1, status);
        }
        GF_CUDA(cudaGetLastError());
    }
    return FILTER_OK;
}

int gqf_count(filter *F, const uint64_t *keys, uint64_t n, uint64_t *counts, uint8_t *found, cudaStream_t st)
{
    if (n == 0) return FILTER_OK;
    GqfState &Q = F->gqf;
    const int g = grid_for(n, 256, 16);
    const Meta *meta = reinterpret_cast<const Meta *>(Q.meta[Q.cur]);
    {
        gf::TraceScope ts_("gqf_count_kernel", n, st);
        if (Q.r == 8) gqf_count_kernel<8><<<g, 256, 0, st>>>(keys, n, Q.H, meta, Q.rem[Q.cur], Q.nblk, counts, found);
        else gqf_count_kernel<16><<<g, 256, 0, st>>>(keys, n, Q.H, meta, Q.rem[Q.cur], Q.nblk, counts, found);
    }
    GF_CUDA(cudaGetLastError());
    return FILTER_OK;
}

// Point updates through the C ABI (Sec. 5.2's point insertion API): one
// thread per key, the locked in-place update of the current buffer
// (include/gpufilter_gqf_ops.cuh). Nothing is sorted and nothing synchronises
// the host, so a call can be captured in a CUDA graph; keys of one call are
// applied in no particular order (the table, a function of the stored
// multiset, does not depend on it).
template <int R>
__global__ void __launch_bounds__(256) gqf_point_kernel(const uint64_t *__restrict__ keys, uint64_t n, PHash H,
                                                        GView g, uint32_t *locks, int remove, uint8_t *status,
                                                        DevCounters *ctr)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t fp = fingerprint(__ldcs(keys + i), H);
        const int rc = gqf_warp_turns([&] {
            return remove ? gqf_point_remove<R>(g, locks, fp, &ctr->status)
                          : gqf_point_insert<R>(g, locks, fp, 1, &ctr->status);
        });
        if (rc == GQF_POINT_BUSY) atomicOr(&ctr->status, ST_TIMEOUT);
        if (rc == FILTER_KEY_FULL) {
            atomicOr(&ctr->status, ST_FULL);
            atomicAdd(&ctr->failed, 1ull);
        }
        if (status) status[i] = (uint8_t)rc;
    }
}

int gqf_point_update(filter *F, const uint64_t *keys, uint64_t n, int remove, uint8_t *status, cudaStream_t st)
{
    if (n == 0) return FILTER_OK;
    GqfState &Q = F->gqf;
    const GView g{reinterpret_cast<Meta *>(Q.meta[Q.cur]), Q.rem[Q.cur], (long long)Q.N, (long long)Q.nslots,
                  (long long)Q.nblk};
    const int grid = grid_for(n, 256, 8);
    gf::TraceScope ts_(remove ? "gqf_point_remove" : "gqf_point_insert", n, st);
    if (Q.r == 8) gqf_point_kernel<8><<<grid, 256, 0, st>>>(keys, n, Q.H, g, Q.locks, remove, status, F->ctr);
    else gqf_point_kernel<16><<<grid, 256, 0, st>>>(keys, n, Q.H, g, Q.locks, remove, status, F->ctr);
    GF_CUDA(cudaGetLastError());
    return FILTER_OK;
}

// The fingerprint is invertible on p bits (Sec. 5.1): every xor-shift by
// s >= p/2 is its own inverse and every product by an odd constant is undone
// by the constant's inverse mod 2^p. A key below 2^p folds to itself, so it
// is recovered exactly from its fingerprint.
__global__ void gqf_unhash_kernel(const uint64_t *__restrict__ fps, uint64_t n, PHash H, uint64_t inv1, uint64_t inv2,
                                  uint64_t *keys)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t x = fps[i] & H.mask;
        x ^= x >> H.s;
        x = (x * inv2) & H.mask;
        x ^= x >> H.s;
        x = (x * inv1) & H.mask;
        x ^= x >> H.s;
        keys[i] = x ^ H.seed;
    }
}

static uint64_t inverse_odd(uint64_t c)
{
    uint64_t v = c;  // Newton: each step doubles the correct low bits
    for (int k = 0; k < 6; k++) v *= 2 - c * v;
    return v;
}

int gqf_unhash(filter *F, const uint64_t *fps, uint64_t n, uint64_t *keys, cudaStream_t st)
{
    if (n == 0) return FILTER_OK;
    GqfState &Q = F->gqf;
    {
        gf::TraceScope ts_("gqf_unhash_kernel", n, st);
        gqf_unhash_kernel<<<grid_for(n, 256, 8), 256, 0, st>>>(fps, n, Q.H, inverse_odd(0xff51afd7ed558ccdull),
                                                                 inverse_odd(0xc4ceb9fe1a85ec53ull), keys);
    }
    GF_CUDA(cudaGetLastError());
    return FILTER_OK;
}

int gqf_enumerate(filter *F, uint64_t *fps, uint64_t *counts, uint64_t cap, uint64_t *n_out, cudaStream_t st)
{
    GqfState &Q = F->gqf;
    const Meta *meta = reinterpret_cast<const Meta *>(Q.meta[Q.cur]);
    // per-block group counts and their scan: stream-ordered scratch for the call
    uint32_t *per = nullptr;
    uint64_t *stmp = nullptr;
    if (dev_malloc_async(reinterpret_cast<void **>(&per), (Q.nblk + 1) * sizeof(uint32_t), st) != cudaSuccess ||
        dev_malloc_async(reinterpret_cast<void **>(&stmp), scan_tmp_words(Q.nblk + 1) * sizeof(uint64_t), st) !=
            cudaSuccess) {
        cudaGetLastError();
        dev_free_async(per, st);
        return FILTER_ERR_OOM;
    }
    const int g = grid_for(Q.nblk, 256, 8);
    {
        gf::TraceScope ts_("gqf_enum_kernel", Q.nblk, st);
        if (Q.r == 8) gqf_enum_kernel<8, false><<<g, 256, 0, st>>>(meta, Q.rem[Q.cur], Q.nblk, Q.N, per, nullptr, nullptr, 0);
        else gqf_enum_kernel<16, false><<<g, 256, 0, st>>>(meta, Q.rem[Q.cur], Q.nblk, Q.N, per, nullptr, nullptr, 0);
    }
    cudaMemsetAsync(per + Q.nblk, 0, 4, st);
    exclusive_scan_u32(per, per, Q.nblk + 1, stmp, F->ctr, st);
    uint32_t total = 0;
    cudaMemcpyAsync(&total, per + Q.nblk, 4, cudaMemcpyDeviceToHost, st);
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && cap && fps && counts) {
        gf::TraceScope ts_("gqf_enum_kernel", Q.nblk, st);
        if (Q.r == 8) gqf_enum_kernel<8, true><<<g, 256, 0, st>>>(meta, Q.rem[Q.cur], Q.nblk, Q.N, per, fps, counts, cap);
        else gqf_enum_kernel<16, true><<<g, 256, 0, st>>>(meta, Q.rem[Q.cur], Q.nblk, Q.N, per, fps, counts, cap);
    }
    dev_free_async(stmp, st);
    dev_free_async(per, st);
    GF_CUDA(e);
    GF_CUDA(cudaGetLastError());
    *n_out = total;
    return FILTER_OK;
}

uint64_t gqf_image_bytes(const filter *F) { return F->gqf.nblk * 32 + F->gqf.nslots * (F->gqf.r / 8); }

int gqf_copy_image(filter *F, void *host, bool to_host, cudaStream_t st)
{
    GqfState &Q = F->gqf;
    char *h = static_cast<char *>(host);
    const uint64_t metaB = Q.nblk * 32, remB = Q.nslots * (Q.r / 8);
    if (to_host) {
        GF_CUDA(cudaMemcpyAsync(h, Q.meta[Q.cur], metaB, cudaMemcpyDeviceToHost, st));
        GF_CUDA(cudaMemcpyAsync(h + metaB, Q.rem[Q.cur], remB, cudaMemcpyDeviceToHost, st));
    } else {
        GF_CUDA(cudaMemcpyAsync(Q.meta[Q.cur], h, metaB, cudaMemcpyHostToDevice, st));
        GF_CUDA(cudaMemcpyAsync(Q.rem[Q.cur], h + metaB, remB, cudaMemcpyHostToDevice, st));
    }
    GF_CUDA(cudaStreamSynchronize(st));
    return FILTER_OK;
}

// ---------------------------------------------------------------------------
// Filter groups: one sort, one reduction and one merge launch for the keys of
// every member. Sort keys are member << pbits | fingerprint, so each member's
// groups are contiguous and in fingerprint order; the merge runs over the
// concatenated tiles of all members, each tile with its member's arguments,
// and a member's first tile starts from an empty prefix. Each member thus
// ends up exactly as a standalone filter given the same keys.
// ---------------------------------------------------------------------------
struct GqfMemberDev {
    PHash H;
    uint64_t N, nblk, tile0;
    const Meta *meta[2];
    const uint8_t *rem[2];
};

__global__ void gqf_group_fp_kernel(const uint64_t *__restrict__ keys, uint64_t n, const uint64_t *__restrict__ off,
                                    uint32_t nmem, const GqfMemberDev *__restrict__ gm, uint32_t pbits, uint64_t *fp,
                                    uint32_t *idx)
{
    MemberCursor c(off, nmem, n);
    uint32_t cm = 0xffffffffu;
    PHash H;
    for (; c.valid(); c.next(off)) {
        if (c.m != cm) {
            cm = c.m;
            H = gm[cm].H;
        }
        fp[c.i] = ((uint64_t)cm << pbits) | fingerprint(__ldg(keys + c.i), H);
        if (idx) idx[c.i] = (uint32_t)c.i;
    }
}

// first group of every tile of every member (successor search, as for one filter)
__global__ void gqf_group_tile_ranges(const uint64_t *__restrict__ ufp, const uint32_t *pm,
                                      const uint32_t *__restrict__ tile_member, const GqfMemberDev *__restrict__ gm,
                                      uint32_t pbits, uint32_t r, uint64_t tiles, uint32_t *tlo)
{
    const uint64_t m = *pm;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t <= tiles;
         t += (uint64_t)gridDim.x * blockDim.x) {
        if (t == tiles) {
            tlo[t] = (uint32_t)m;
            continue;
        }
        const uint32_t mb = tile_member[t];
        const uint64_t q0 = (t - gm[mb].tile0) * TQ, N = gm[mb].N;
        // a sum, not an or: N << r = 2^p may reach the member bits
        const uint64_t key = ((uint64_t)mb << pbits) + ((q0 >= N ? N : q0) << r);
        uint64_t lo = 0, hi = m;
        while (lo < hi) {
            uint64_t mid = (lo + hi) >> 1;
            if (ufp[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        tlo[t] = (uint32_t)lo;
    }
}

__global__ void gqf_group_reset(DevCounters *mctr, uint32_t n)
{
    for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
        mctr[m].overflow = 0;
        mctr[m].gqf_end = -1;
    }
}

// members whose merge passed the end of their table
__global__ void gqf_group_overflow(const DevCounters *mctr, uint32_t n, DevCounters *gctr, uint32_t *list)
{
    for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x)
        if (mctr[m].overflow) list[atomicAdd(&gctr->pend[0], 1u)] = m;
}

// Asynchronous group updates: copy every block of a member whose merge fit
// from the spare buffer back to the current one (a member that overflowed
// keeps its current, old table).
template <int R>
__global__ void gqf_group_commit(const uint64_t *__restrict__ mblk0, uint32_t nmem, const DevCounters *mctr,
                                 const uint8_t *__restrict__ meta_src, const uint8_t *__restrict__ rem_src,
                                 uint8_t *meta_dst, uint8_t *rem_dst, uint64_t nblk)
{
    constexpr int RW = 64 * R / 8 / 16;  // 16-byte words of one block's remainders
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < nblk; b += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = nmem;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(mblk0 + mid) <= b) lo = mid;
            else hi = mid;
        }
        if (mctr[lo].overflow) continue;
        const uint4 *ms = reinterpret_cast<const uint4 *>(meta_src + b * 32);
        uint4 *md = reinterpret_cast<uint4 *>(meta_dst + b * 32);
        md[0] = ms[0];
        md[1] = ms[1];
        const uint4 *rs = reinterpret_cast<const uint4 *>(rem_src + b * 64 * (R / 8));
        uint4 *rd = reinterpret_cast<uint4 *>(rem_dst + b * 64 * (R / 8));
#pragma unroll
        for (int w = 0; w < RW; w++) rd[w] = rs[w];
    }
}

// the keys of members whose insert did not fit: FULL, counted per member
__global__ void gqf_group_reject(const uint64_t *__restrict__ off, uint32_t nmem, uint64_t n, DevCounters *mctr,
                                 uint8_t *status)
{
    MemberCursor c(off, nmem, n);
    for (; c.valid(); c.next(off)) {
        if (!mctr[c.m].overflow) continue;
        if (status) status[c.i] = FILTER_KEY_FULL;
        atomicAdd(&mctr[c.m].failed, 1ull);
        atomicOr(&mctr[c.m].status, ST_FULL);
    }
}

template <int R>
__global__ void __launch_bounds__(256) gqf_group_count_kernel(const uint64_t *__restrict__ keys, uint64_t n,
                                                              const uint64_t *__restrict__ off, uint32_t nmem,
                                                              const GqfMemberDev *__restrict__ gm, int cur,
                                                              uint64_t *counts, uint8_t *found)
{
    MemberCursor c(off, nmem, n);
    uint32_t cm = 0xffffffffu;
    PHash H;
    const Meta *meta = nullptr;
    const uint8_t *rem = nullptr;
    uint64_t nblk = 0;
    for (; c.valid(); c.next(off)) {
        if (c.m != cm) {
            cm = c.m;
            H = gm[cm].H;
            meta = gm[cm].meta[cur];
            rem = gm[cm].rem[cur];
            nblk = gm[cm].nblk;
        }
        const uint64_t cnt = count_fp<R>(fingerprint(__ldcs(keys + c.i), H), meta, rem, nblk);
        if (counts) __stcs(reinterpret_cast<unsigned long long *>(counts + c.i), (unsigned long long)cnt);
        if (found) __stcs(found + c.i, (uint8_t)(cnt ? 1 : 0));
    }
}

int gqf_group_setup(filter_group *GR, const filter_config *cfgs, uint64_t &bytes_out, bool plan_only)
{
    const uint32_t n = GR->n, r = cfgs[0].tag_bits;
    const uint64_t M = GR->max_total ? GR->max_total : 1;
    if (M >= (1ull << 30)) return FILTER_ERR_ARG;
    std::vector<filter> V(n);
    std::vector<uint64_t> meta_off(n), rem_off(n), tile0(n);
    uint64_t nblk_tot = 0, nslots_tot = 0, tiles = 0, ts_words = 2, tlo_words = 1;
    uint32_t pbits = 0;
    for (uint32_t m = 0; m < n; m++) {
        if (cfgs[m].kind != FILTER_GQF || cfgs[m].tag_bits != r || cfgs[m].block_slots) return FILTER_ERR_ARG;
        V[m].cfg = cfgs[m];
        V[m].cfg.max_batch = M;
        uint64_t tb = 0, sb = 0;
        int rc = gqf_setup(&V[m], tb, sb, true);  // geometry only
        if (rc != FILTER_OK) return rc;
        const GqfState &Q = V[m].gqf;
        meta_off[m] = nblk_tot;
        rem_off[m] = nslots_tot;
        tile0[m] = tiles;
        nblk_tot += Q.nblk;
        nslots_tot += Q.nslots;
        tiles += Q.ntiles;
        if (Q.p > pbits) pbits = Q.p;
        if (Q.ntiles * 4 + 2 > ts_words) ts_words = Q.ntiles * 4 + 2;
        if (gqf_tile_lo_words(Q) > tlo_words) tlo_words = gqf_tile_lo_words(Q);
    }
    uint32_t mbits = 1;
    while (mbits < 32 && (1ull << mbits) < n) mbits++;
    if (pbits + mbits > 64 || tiles >= (1ull << 32)) return FILTER_ERR_ARG;
    if (tiles + 2 > ts_words) ts_words = tiles + 2;
    if (tiles + 1 > tlo_words) tlo_words = tiles + 1;
    GR->tiles = tiles;
    GR->pbits = pbits;
    GR->mbits = mbits;
    GqfState &Q = GR->gqf;
    Q.r = r;
    Q.nblk = nblk_tot;
    Q.nslots = nslots_tot;
    Q.ntiles = tiles;
    uint64_t scan_n = radix_tmp_words(M);
    if (M + 1 > scan_n) scan_n = M + 1;
    uint64_t bytes = 0;
    Arena &A = GR->arena;
    auto piece = [&](auto *&ptr, uint64_t count) {
        using T_ = typename std::remove_reference<decltype(*ptr)>::type;
        bytes += (count * sizeof(T_) + 255) & ~255ull;
        if (!plan_only) ptr = A.take<T_>(count);
    };
    for (int b = 0; b < 2; b++) {
        piece(Q.meta[b], nblk_tot * 32);
        piece(Q.rem[b], nslots_tot * (r / 8));
    }
    piece(Q.fp_a, M);
    piece(Q.fp_b, M);
    piece(Q.fp_c, M);
    piece(Q.ufp, M);
    piece(Q.idx_a, M);
    piece(Q.idx_b, M);
    piece(Q.idx_c, M);
    piece(Q.ustart, M + 1);
    piece(Q.flags, M + 1);
    piece(Q.removed, M);
    piece(Q.tile_state, ts_words);
    piece(Q.tile_lo, tlo_words);
    piece(Q.radix_tmp, radix_tmp_words(M));
    piece(GR->scan_tmp, scan_tmp_words(scan_n));
    piece(GR->mctr, (uint64_t)n);
    piece(GR->d_tile_member, tiles);
    piece(GR->d_ovf, (uint64_t)n);
    piece(GR->d_mblk0, (uint64_t)n + 1);
    {
        MergeArgs *ma = nullptr;
        GqfMemberDev *gd = nullptr;
        piece(ma, 4ull * n);
        piece(gd, (uint64_t)n);
        GR->d_margs = ma;
        GR->d_gmem = gd;
    }
    bytes_out = bytes;
    if (plan_only) return FILTER_OK;
    if (!Q.meta[1] || !Q.rem[1] || !Q.radix_tmp || !GR->scan_tmp || !GR->mctr || !GR->d_tile_member || !GR->d_ovf ||
        !GR->d_margs || !GR->d_gmem || !GR->d_mblk0)
        return FILTER_ERR_INTERNAL;
    Q.cur = 0;
    GR->cur = 0;
    // member views, merge arguments [cur][del][member], hash and table descriptors
    std::vector<MergeArgs> margs(4ull * n);
    std::vector<GqfMemberDev> gmem(n);
    std::vector<uint32_t> tmem(tiles);
    for (uint32_t m = 0; m < n; m++) {
        filter &F = GR->members[m];
        F.cfg = V[m].cfg;
        F.gqf = V[m].gqf;
        GqfState &S = F.gqf;
        S.merge_only = true;  // a member redone alone must land in the other buffer, like the group
        for (int b = 0; b < 2; b++) {
            S.meta[b] = Q.meta[b] + meta_off[m] * 32;
            S.rem[b] = Q.rem[b] + rem_off[m] * (r / 8);
        }
        S.cur = 0;
        S.fp_a = Q.fp_a;
        S.fp_b = Q.fp_b;
        S.fp_c = Q.fp_c;
        S.ufp = Q.ufp;
        S.idx_a = Q.idx_a;
        S.idx_b = Q.idx_b;
        S.idx_c = Q.idx_c;
        S.ustart = Q.ustart;
        S.flags = Q.flags;
        S.removed = Q.removed;
        S.tile_state = Q.tile_state;
        S.tile_lo = Q.tile_lo;
        S.radix_tmp = Q.radix_tmp;
        F.ctr = GR->mctr + m;
        F.scan_tmp = GR->scan_tmp;
        F.arena.base = GR->arena.base;  // marks the view valid; the group owns the memory
        F.device = GR->device;
        gmem[m].H = S.H;
        gmem[m].N = S.N;
        gmem[m].nblk = S.nblk;
        gmem[m].tile0 = tile0[m];
        for (int b = 0; b < 2; b++) {
            gmem[m].meta[b] = reinterpret_cast<const Meta *>(S.meta[b]);
            gmem[m].rem[b] = S.rem[b];
        }
        for (uint64_t t = 0; t < S.ntiles; t++) tmem[tile0[m] + t] = m;
        for (int cur = 0; cur < 2; cur++)
            for (int del = 0; del < 2; del++) {
                MergeArgs &a = margs[(uint64_t)(cur * 2 + del) * n + m];
                a.meta_old = reinterpret_cast<const Meta *>(S.meta[cur]);
                a.rem_old = S.rem[cur];
                a.meta_new = reinterpret_cast<Meta *>(S.meta[cur ^ 1]);
                a.rem_new = S.rem[cur ^ 1];
                a.ufp = Q.ufp;
                a.ustart = Q.ustart;
                a.pm = nullptr;
                a.tlo = Q.tile_lo + tile0[m];
                a.m_limit = ~0ull;
                a.removed = del ? Q.removed : nullptr;
                a.ts = Q.tile_state + tile0[m];
                a.ctr = GR->mctr + m;
                a.N = S.N;
                a.nslots = S.nslots;
                a.nblk = S.nblk;
                a.ntiles = S.ntiles;
                a.fmask = S.H.mask;
                a.tile0 = tile0[m];
                a.r = r;
                a.del = del;
                a.dry = 0;
            }
    }
    GF_CUDA(cudaMemcpy(GR->d_margs, margs.data(), margs.size() * sizeof(MergeArgs), cudaMemcpyHostToDevice));
    {
        std::vector<uint64_t> mb(meta_off);
        mb.push_back(nblk_tot);
        GF_CUDA(cudaMemcpy(GR->d_mblk0, mb.data(), mb.size() * 8, cudaMemcpyHostToDevice));
    }
    GF_CUDA(cudaMemcpy(GR->d_gmem, gmem.data(), gmem.size() * sizeof(GqfMemberDev), cudaMemcpyHostToDevice));
    if (tiles) GF_CUDA(cudaMemcpy(GR->d_tile_member, tmem.data(), tiles * 4, cudaMemcpyHostToDevice));
    return FILTER_OK;
}

static void group_set_cur(filter_group *GR, int cur)
{
    GR->cur = cur;
    GR->gqf.cur = cur;
    for (uint32_t m = 0; m < GR->n; m++) GR->members[m].gqf.cur = cur;
}

int gqf_group_clear(filter_group *GR, cudaStream_t st)
{
    GqfState &Q = GR->gqf;
    for (int b = 0; b < 2; b++) {
        GF_CUDA(cudaMemsetAsync(Q.meta[b], 0, Q.nblk * 32, st));
        GF_CUDA(cudaMemsetAsync(Q.rem[b], 0, Q.nslots * (Q.r / 8), st));
    }
    GF_CUDA(cudaMemsetAsync(GR->mctr, 0, GR->n * sizeof(DevCounters), st));
    GF_CUDA(cudaMemsetAsync(GR->ctr, 0, sizeof(DevCounters), st));
    group_set_cur(GR, 0);
    return FILTER_OK;
}

// fingerprints, sort, reduction to groups (count of groups in flags[n])
static void group_prepare(filter_group *GR, const uint64_t *off, const uint64_t *keys, uint64_t n, bool need_idx,
                          cudaStream_t st)
{
    GqfState &Q = GR->gqf;
    const int g = grid_for(n, 256, 8);
    {
        gf::TraceScope ts_("gqf_group_fp_kernel", n, st);
        gqf_group_fp_kernel<<<g, 256, 0, st>>>(keys, n, off, GR->n, static_cast<const GqfMemberDev *>(GR->d_gmem),
                                               GR->pbits, Q.fp_a, need_idx ? Q.idx_a : nullptr);
    }
    radix_sort_u64(Q.fp_a, Q.fp_b, Q.fp_c, need_idx ? Q.idx_a : nullptr, Q.idx_b, Q.idx_c, n, GR->pbits + GR->mbits,
                   Q.radix_tmp, GR->scan_tmp, GR->ctr, st);
    rle_sorted_u64(Q.fp_b, n, Q.ufp, Q.ustart, need_idx ? Q.flags : nullptr, Q.flags + n, GR->scan_tmp, GR->ctr, st);
}

static int group_merge(filter_group *GR, uint64_t n, int del, cudaStream_t st)
{
    GqfState &Q = GR->gqf;
    const int nb = GR->cur ^ 1;
    GF_CUDA(cudaMemsetAsync(Q.tile_state, 0, (GR->tiles + 2) * 8, st));
    GF_CUDA(cudaMemsetAsync(Q.meta[nb], 0, Q.nblk * 32, st));
    {
        gf::TraceScope ts_("gqf_group_reset", GR->n, st);
        gqf_group_reset<<<grid_for(GR->n, 256, 1), 256, 0, st>>>(GR->mctr, GR->n);
    }
    {
        gf::TraceScope ts_("gqf_group_tile_ranges", GR->tiles + 1, st);
        gqf_group_tile_ranges<<<grid_for(GR->tiles + 1, 256, 4), 256, 0, st>>>(
            Q.ufp, Q.flags + n, GR->d_tile_member, static_cast<const GqfMemberDev *>(GR->d_gmem), GR->pbits, Q.r,
            GR->tiles, Q.tile_lo);
    }
    const MergeArgs *tab = static_cast<const MergeArgs *>(GR->d_margs) + (uint64_t)(GR->cur * 2 + del) * GR->n;
    {
        gf::TraceScope ts_("gqf_merge_group_kernel", 0, st, true);
        if (Q.r == 8)
            gqf_merge_group_kernel<8><<<(unsigned)GR->tiles, MT, 0, st>>>(tab, GR->d_tile_member, Q.tile_state,
                                                                          Q.nslots, Q.flags + n, ts_.units());
        else
            gqf_merge_group_kernel<16><<<(unsigned)GR->tiles, MT, 0, st>>>(tab, GR->d_tile_member, Q.tile_state,
                                                                           Q.nslots, Q.flags + n, ts_.units());
    }
    GF_CUDA(cudaGetLastError());
    return FILTER_OK;
}

int gqf_group_insert(filter_group *GR, const uint64_t *off, const uint64_t *keys, uint64_t n, uint8_t *status,
                     cudaStream_t st)
{
    if (n == 0) return FILTER_OK;
    GqfState &Q = GR->gqf;
    group_prepare(GR, off, keys, n, status != nullptr, st);
    int rc = group_merge(GR, n, 0, st);
    if (rc) return rc;
    if (status) {
        gf::TraceScope ts_("gqf_status_kernel", n, st);
        gqf_status_kernel<<<grid_for(n, 256, 8), 256, 0, st>>>(n, Q.flags, Q.ustart, Q.idx_b, Q.removed, ~0ull, 0,
                                                              status);
    }
    GF_CUDA(cudaMemsetAsync(&GR->ctr->pend[0], 0, 4, st));
    {
        gf::TraceScope ts_("gqf_group_overflow", GR->n, st);
        gqf_group_overflow<<<grid_for(GR->n, 256, 1), 256, 0, st>>>(GR->mctr, GR->n, GR->ctr, GR->d_ovf);
    }
    GF_CUDA(cudaGetLastError());
    unsigned novf = 0;
    if ((rc = read_dev(&GR->ctr->pend[0], &novf, st))) return rc;
    if (novf) {
        // members that do not fit: redo them alone from their old table, which
        // keeps the longest prefix of their sorted groups that fits
        std::vector<uint32_t> list(novf);
        GF_CUDA(cudaMemcpyAsync(list.data(), GR->d_ovf, novf * 4, cudaMemcpyDeviceToHost, st));
        GF_CUDA(cudaStreamSynchronize(st));
        for (uint32_t m : list) {
            uint64_t o[2];
            GF_CUDA(cudaMemcpyAsync(o, off + m, 16, cudaMemcpyDeviceToHost, st));
            GF_CUDA(cudaStreamSynchronize(st));
            filter &F = GR->members[m];
            F.gqf.cur = GR->cur;
            if ((rc = gqf_insert(&F, keys + o[0], nullptr, o[1] - o[0], status ? status + o[0] : nullptr, st))) return rc;
        }
    }
    group_set_cur(GR, GR->cur ^ 1);
    return FILTER_OK;
}

int gqf_group_remove(filter_group *GR, const uint64_t *off, const uint64_t *keys, uint64_t n, uint8_t *status,
                     cudaStream_t st)
{
    if (n == 0) return FILTER_OK;
    GqfState &Q = GR->gqf;
    group_prepare(GR, off, keys, n, status != nullptr, st);
    int rc = group_merge(GR, n, 1, st);
    if (rc) return rc;
    if (status) {
        gf::TraceScope ts_("gqf_status_kernel", n, st);
        gqf_status_kernel<<<grid_for(n, 256, 8), 256, 0, st>>>(n, Q.flags, Q.ustart, Q.idx_b, Q.removed, 0, 1, status);
    }
    GF_CUDA(cudaGetLastError());
    group_set_cur(GR, GR->cur ^ 1);
    return FILTER_OK;
}

int gqf_group_count(filter_group *GR, const uint64_t *off, const uint64_t *keys, uint64_t n, uint64_t *counts,
                    uint8_t *found, cudaStream_t st)
{
    if (n == 0) return FILTER_OK;
    const int g = grid_for(n, 256, 16);
    const GqfMemberDev *gm = static_cast<const GqfMemberDev *>(GR->d_gmem);
    {
        gf::TraceScope ts_("gqf_group_count_kernel", n, st);
        if (GR->gqf.r == 8) gqf_group_count_kernel<8><<<g, 256, 0, st>>>(keys, n, off, GR->n, gm, GR->cur, counts, found);
        else gqf_group_count_kernel<16><<<g, 256, 0, st>>>(keys, n, off, GR->n, gm, GR->cur, counts, found);
    }
    GF_CUDA(cudaGetLastError());
    return FILTER_OK;
}

int gqf_group_update_async(filter_group *GR, const uint64_t *off, const uint64_t *keys, uint64_t n, uint8_t *status,
                           int del, cudaStream_t st)
{
    if (n == 0) return FILTER_OK;
    GqfState &Q = GR->gqf;
    group_prepare(GR, off, keys, n, status != nullptr, st);
    int rc = group_merge(GR, n, del, st);
    if (rc) return rc;
    if (status) {
        gf::TraceScope ts_("gqf_status_kernel", n, st);
        gqf_status_kernel<<<grid_for(n, 256, 8), 256, 0, st>>>(n, Q.flags, Q.ustart, Q.idx_b, Q.removed,
                                                              del ? 0 : ~0ull, del, status);
    }
    const int nb = GR->cur ^ 1;
    {
        gf::TraceScope ts_("gqf_group_commit", Q.nblk, st);
        if (Q.r == 8)
            gqf_group_commit<8><<<grid_for(Q.nblk, 256, 8), 256, 0, st>>>(GR->d_mblk0, GR->n, GR->mctr, Q.meta[nb],
                                                                         Q.rem[nb], Q.meta[GR->cur], Q.rem[GR->cur],
                                                                         Q.nblk);
        else
            gqf_group_commit<16><<<grid_for(Q.nblk, 256, 8), 256, 0, st>>>(GR->d_mblk0, GR->n, GR->mctr, Q.meta[nb],
                                                                          Q.rem[nb], Q.meta[GR->cur], Q.rem[GR->cur],
                                                                          Q.nblk);
    }
    if (!del) {
        gf::TraceScope ts_("gqf_group_reject", n, st);
        gqf_group_reject<<<grid_for(n, 256, 8), 256, 0, st>>>(off, GR->n, n, GR->mctr, status);
    }
    GF_CUDA(cudaGetLastError());
    return FILTER_OK;
}

}  // namespace gf
