/*
 * Oracle counting quotient filter (GQF). TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Specification (paper Sec. 5; the readings taken where it is silent, or
 * where it defers to the CQF paper it cites, are marked R):
 *
 *  Fingerprint. p = q + r bits; fp = mix_p(fold_p(key) ^ (seed mod 2^p)).
 *  Quotient x = fp >> r (R: "first q bits" = the high bits), remainder
 *  fp mod 2^r (Sec. 5.1). r is 8 or 16, so a slot is one machine word.
 *
 *  Slots. N = 2^q home slots plus a tail of S slots, no wrap-around (R).
 *  S = min(N, roundup64(1072 q)), at least 64: twice the longest-cluster bound
 *  ln(2^q) / (a - ln a - 1) of Sec. 5.2 at load a = 0.95, i.e. 2 q ln 2 /
 *  0.0012933 ~ 1072 q, as an integer rule.
 *
 *  Runs (Sec. 5.1). All remainders of quotient x form the run of x; runs are
 *  stored in quotient order, the run of x starting at max(x, end of the
 *  previous run + 1); a cluster is a maximal stretch of runs with no gap.
 *  Inside a run each distinct remainder v with count c is stored once, in
 *  ascending order of v, encoded as (R, the counter encoding is not given
 *  in the paper):
 *      c = 1 :  [v]
 *      c >= 2:  [v, v, n, d1 .. dn]   n = number of base-2^r digits of c - 2
 *                                     (0 when c = 2), most significant first.
 *  A reader that meets v followed by v knows a counter follows.
 *
 *  Metadata per 64-slot block j (R: the layout of the cited CQF, written out):
 *  occupieds (bit i: quotient 64j + i has a run), runends (bit i: slot 64j + i
 *  ends a run), offset = max(0, end of the run of q* - 64j) where q* is the
 *  largest occupied quotient <= 64j (0 when there is none). Free slots hold 0.
 *
 *  Byte image: per block 32 bytes {occupieds u64, runends u64, offset u32,
 *  12 zero bytes}, all blocks first, then the remainders (r/8 bytes each,
 *  little-endian).
 *
 *  Bulk insert (Sec. 5.3, 5.4): fingerprints are sorted and reduced to
 *  <fp, count> groups, which are inserted in ascending order by shifting the
 *  following runs right. If a group does not fit before the end of the tail,
 *  it and every later group of the batch are rejected (status 1), which keeps
 *  the longest prefix of the sorted batch that fits (R).
 *
 *  Counted insert (values through the counters: Sec. 2 notes that the CQF
 *  associates values with items by using its counters): key i comes with
 *  c_i >= 1 and counts as c_i copies, so a group's count is the sum of the
 *  c_i of its keys. Everything else is the bulk insert above.
 *
 *  Bulk delete (Sec. 6.4): groups are removed in descending order ("larger
 *  items first"), shifting the following runs left but never before their
 *  home slot. A group of d deletes of a fingerprint with count c removes
 *  min(c, d) copies; the keys of the group are taken in batch order and the
 *  last d - min(c, d) of them get status 2 (not found) (R).
 *
 *  Count (Sec. 5.1, via the cited CQF): locate the run of x from the offset
 *  of block x / 64 and rank / select over occupieds and runends, then parse
 *  the run.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

struct or_gqf {
    unsigned q, r, p;
    uint64_t N, S, nslots, nblk, seed, rmask;
    uint64_t *occ, *rend;
    uint32_t *off;
    uint16_t *rem;
    uint64_t maxg, maxs; /* scratch sizes: distinct remainders per run, slots per run */
    uint64_t *sv, *sc;
    uint16_t *ss;
};

uint64_t or_gqf_tail_slots(unsigned q)
{
    uint64_t N = 1ULL << q;
    uint64_t s = ((1072ULL * q + 63) / 64) * 64;
    if (s > N) s = N;
    if (s < 64) s = 64;
    return s;
}

or_gqf *or_gqf_new(unsigned q, unsigned r, uint64_t seed)
{
    if ((r != 8 && r != 16) || q < 6 || q + r > 64 || q > 40) return NULL;
    or_gqf *G = (or_gqf *)calloc(1, sizeof(or_gqf));
    G->q = q;
    G->r = r;
    G->p = q + r;
    G->N = 1ULL << q;
    G->S = or_gqf_tail_slots(q);
    G->nslots = G->N + G->S;
    G->nblk = G->nslots / 64;
    G->seed = seed;
    G->rmask = (1ULL << r) - 1ULL;
    G->occ = calloc(G->nblk, 8);
    G->rend = calloc(G->nblk, 8);
    G->off = calloc(G->nblk, 4);
    G->rem = calloc(G->nslots, 2);
    G->maxg = 1ULL << r;
    G->maxs = G->maxg * (3 + 64 / r) + 16;
    G->sv = malloc(G->maxg * 8);
    G->sc = malloc(G->maxg * 8);
    G->ss = malloc(G->maxs * 2);
    if (!G->occ || !G->rend || !G->off || !G->rem || !G->sv || !G->sc || !G->ss) {
        or_gqf_free(G);
        return NULL;
    }
    return G;
}

void or_gqf_free(or_gqf *G)
{
    if (!G) return;
    free(G->occ);
    free(G->rend);
    free(G->off);
    free(G->rem);
    free(G->sv);
    free(G->sc);
    free(G->ss);
    free(G);
}

void or_gqf_geometry(const or_gqf *G, uint64_t *o)
{
    o[0] = G->N;
    o[1] = G->S;
    o[2] = G->nslots;
    o[3] = G->nblk;
    o[4] = G->p;
}

static uint64_t fp_of(const or_gqf *G, uint64_t key)
{
    uint64_t m = G->p >= 64 ? ~0ULL : ((1ULL << G->p) - 1ULL);
    return or_mix_p(or_fold_p(key, G->p) ^ (G->seed & m), G->p);
}

void or_gqf_fingerprints(const or_gqf *G, const uint64_t *keys, uint64_t n, uint64_t *fp)
{
    for (uint64_t i = 0; i < n; i++) fp[i] = fp_of(G, keys[i]);
}

/* ---- bit helpers ---- */
static int occ_get(const or_gqf *G, int64_t x) { return (int)((G->occ[x >> 6] >> (x & 63)) & 1); }
static void occ_put(or_gqf *G, int64_t x, int v)
{
    if (v) G->occ[x >> 6] |= 1ULL << (x & 63);
    else G->occ[x >> 6] &= ~(1ULL << (x & 63));
}
static int rend_get(const or_gqf *G, int64_t i) { return (int)((G->rend[i >> 6] >> (i & 63)) & 1); }
static void rend_put(or_gqf *G, int64_t i, int v)
{
    if (v) G->rend[i >> 6] |= 1ULL << (i & 63);
    else G->rend[i >> 6] &= ~(1ULL << (i & 63));
}

/* first runend at or after slot i, or -1 */
static int64_t next_runend(const or_gqf *G, int64_t i)
{
    for (; i < (int64_t)G->nslots; i++)
        if (rend_get(G, i)) return i;
    return -1;
}

/* largest occupied quotient < x, or -1 (word-at-a-time scan) */
static int64_t prev_occ(const or_gqf *G, int64_t x)
{
    if (x <= 0) return -1;
    int64_t y = x - 1, w = y >> 6;
    unsigned k = (unsigned)(y & 63);
    uint64_t word = G->occ[w] & (k == 63 ? ~0ULL : ((1ULL << (k + 1)) - 1ULL));
    for (;;) {
        if (word) return 64 * w + 63 - __builtin_clzll(word);
        if (w == 0) return -1;
        word = G->occ[--w];
    }
}

/* smallest occupied quotient in (x, lim], or -1 */
static int64_t next_occ_upto(const or_gqf *G, int64_t x, int64_t lim)
{
    if (lim >= (int64_t)G->N) lim = (int64_t)G->N - 1;
    int64_t y = x + 1;
    if (y > lim) return -1;
    int64_t w = y >> 6;
    uint64_t word = G->occ[w] & (~0ULL << (y & 63));
    for (;;) {
        if (word) {
            int64_t z = 64 * w + __builtin_ctzll(word);
            return z <= lim ? z : -1;
        }
        if (64 * (w + 1) > lim) return -1;
        word = G->occ[++w];
    }
}

/* End of the run of an occupied quotient y, found the CQF way: the offset of
   block j = y / 64 gives the end of the run of q* (or a point <= 64j when it
   was clipped); the run of y is the d-th run ending after that point, where d
   counts the occupied quotients in (64j, y]. */
static int64_t runend_of(const or_gqf *G, int64_t y)
{
    int64_t j = y >> 6;
    int64_t base = 64 * j + (int64_t)G->off[j];
    unsigned k = (unsigned)(y & 63);
    uint64_t upto = (k == 63) ? ~0ULL : ((1ULL << (k + 1)) - 1ULL);
    int d = __builtin_popcountll(G->occ[j] & upto & ~1ULL);
    if (d == 0) return base;
    int64_t pos = base;
    while (d > 0) {
        pos++;
        if (rend_get(G, pos)) d--;
    }
    return pos;
}

/* end of the run before quotient x (the run of the largest occupied < x), or -1 */
static int64_t prev_end(const or_gqf *G, int64_t x)
{
    int64_t y = prev_occ(G, x);
    return y < 0 ? -1 : runend_of(G, y);
}

static int64_t imax(int64_t a, int64_t b) { return a > b ? a : b; }

/* ---- counter encoding ---- */
static unsigned ndigits(uint64_t v, unsigned r)
{
    unsigned n = 0;
    while (v) {
        n++;
        v >>= r;
    }
    return n;
}

static unsigned enc_put(uint16_t *dst, uint64_t v, uint64_t c, unsigned r)
{
    dst[0] = (uint16_t)v;
    if (c == 1) return 1;
    uint64_t x = c - 2;
    unsigned n = ndigits(x, r);
    dst[1] = (uint16_t)v;
    dst[2] = (uint16_t)n;
    for (unsigned d = 0; d < n; d++)
        dst[3 + d] = (uint16_t)((x >> (r * (n - 1 - d))) & ((1ULL << r) - 1ULL));
    return 3 + n;
}

/* parse slots [s, e] into (remainder, count) pairs; returns the number */
static uint64_t parse_run(const or_gqf *G, int64_t s, int64_t e, uint64_t *v, uint64_t *c)
{
    uint64_t k = 0;
    int64_t i = s;
    while (i <= e) {
        uint64_t x = G->rem[i];
        if (i + 2 <= e && G->rem[i + 1] == x) {
            unsigned n = G->rem[i + 2];
            uint64_t val = 0;
            for (unsigned d = 0; d < n; d++) val = (val << G->r) | G->rem[i + 3 + d];
            v[k] = x;
            c[k] = val + 2;
            i += 3 + n;
        } else {
            v[k] = x;
            c[k] = 1;
            i += 1;
        }
        k++;
    }
    return k;
}

/* offset of block j from its definition, given correct offsets for the
   blocks before j */
static void recompute_offset(or_gqf *G, int64_t j)
{
    int64_t Q = 64 * j;
    int64_t y = (Q < (int64_t)G->N && occ_get(G, Q)) ? Q : prev_occ(G, Q < (int64_t)G->N ? Q : (int64_t)G->N);
    if (y < 0) {
        G->off[j] = 0;
        return;
    }
    int64_t e;
    if (y < Q) {
        e = runend_of(G, y);
    } else {
        int64_t s = imax(Q, prev_end(G, Q) + 1);
        e = next_runend(G, s);
    }
    G->off[j] = (uint32_t)imax(0, e - Q);
}

/* run record used while re-placing the runs that follow a change */
typedef struct {
    int64_t y, os, oe, ns;
    uint16_t *slots;
} moved_t;

/*
 * Replace the content of the run of quotient x by new_slots[0 .. nlen) (nlen
 * may be 0: the run disappears) and re-place every following run at
 * max(home, previous end + 1) until a run stays where it was. Returns 1, and
 * changes nothing, when a slot would land past the tail.
 */
static int replace_run(or_gqf *G, int64_t x, const uint16_t *new_slots, int64_t nlen)
{
    int had = occ_get(G, x);
    int64_t pe = prev_end(G, x);
    int64_t s = imax(x, pe + 1);
    int64_t e = had ? runend_of(G, x) : s - 1;
    int64_t old_prev_end = had ? e : pe;
    int64_t new_prev_end = nlen > 0 ? s + nlen - 1 : pe;

    size_t cap = 16, nm = 0;
    moved_t *mv = malloc(cap * sizeof(moved_t));
    int64_t y = x;
    for (;;) {
        y = next_occ_upto(G, y, imax(old_prev_end, new_prev_end) + 1);
        if (y < 0) break;
        int64_t os = imax(y, old_prev_end + 1);
        int64_t oe = next_runend(G, os);
        int64_t ns = imax(y, new_prev_end + 1);
        if (ns == os) break;
        if (nm == cap) {
            cap *= 2;
            mv = realloc(mv, cap * sizeof(moved_t));
        }
        int64_t len = oe - os + 1;
        mv[nm].y = y;
        mv[nm].os = os;
        mv[nm].oe = oe;
        mv[nm].ns = ns;
        mv[nm].slots = malloc((size_t)len * 2);
        memcpy(mv[nm].slots, &G->rem[os], (size_t)len * 2);
        nm++;
        old_prev_end = oe;
        new_prev_end = ns + len - 1;
    }
    int64_t last_new = new_prev_end, old_hi = old_prev_end;
    int overflow = last_new >= (int64_t)G->nslots;
    if (!overflow) {
        for (int64_t i = s; i <= old_hi; i++) {
            G->rem[i] = 0;
            rend_put(G, i, 0);
        }
        if (nlen > 0) {
            memcpy(&G->rem[s], new_slots, (size_t)nlen * 2);
            rend_put(G, s + nlen - 1, 1);
        }
        occ_put(G, x, nlen > 0);
        for (size_t k = 0; k < nm; k++) {
            int64_t len = mv[k].oe - mv[k].os + 1;
            memcpy(&G->rem[mv[k].ns], mv[k].slots, (size_t)len * 2);
            rend_put(G, mv[k].ns + len - 1, 1);
        }
        int64_t hi = imax(old_hi, last_new);
        int64_t jlast = (hi >> 6) + 1;
        if (jlast > (int64_t)G->nblk - 1) jlast = (int64_t)G->nblk - 1;
        for (int64_t j = x >> 6; j <= jlast; j++) recompute_offset(G, j);
    }
    for (size_t k = 0; k < nm; k++) free(mv[k].slots);
    free(mv);
    return overflow;
}

/* read the groups of quotient x (empty when unoccupied) */
static uint64_t groups_of(const or_gqf *G, int64_t x, uint64_t *v, uint64_t *c)
{
    if (!occ_get(G, x)) return 0;
    int64_t s = imax(x, prev_end(G, x) + 1);
    int64_t e = runend_of(G, x);
    return parse_run(G, s, e, v, c);
}

static int64_t encode_groups(const or_gqf *G, const uint64_t *v, const uint64_t *c, uint64_t k,
                             uint16_t *out)
{
    int64_t len = 0;
    for (uint64_t i = 0; i < k; i++) len += enc_put(out + len, v[i], c[i], G->r);
    return len;
}

static int insert_group(or_gqf *G, uint64_t fp, uint64_t cnt)
{
    int64_t x = (int64_t)(fp >> G->r);
    uint64_t v0 = fp & G->rmask;
    uint64_t *v = G->sv, *c = G->sc;
    uint16_t *slots = G->ss;
    uint64_t k = groups_of(G, x, v, c);
    uint64_t pos = 0;
    while (pos < k && v[pos] < v0) pos++;
    if (pos < k && v[pos] == v0) {
        c[pos] += cnt;
    } else {
        memmove(&v[pos + 1], &v[pos], (k - pos) * 8);
        memmove(&c[pos + 1], &c[pos], (k - pos) * 8);
        v[pos] = v0;
        c[pos] = cnt;
        k++;
    }
    int64_t len = encode_groups(G, v, c, k, slots);
    return replace_run(G, x, slots, len);
}

static uint64_t delete_group(or_gqf *G, uint64_t fp, uint64_t d)
{
    int64_t x = (int64_t)(fp >> G->r);
    uint64_t v0 = fp & G->rmask;
    if (!occ_get(G, x)) return 0;
    uint64_t *v = G->sv, *c = G->sc;
    uint16_t *slots = G->ss;
    uint64_t k = groups_of(G, x, v, c);
    uint64_t pos = 0, removed = 0;
    while (pos < k && v[pos] < v0) pos++;
    if (pos < k && v[pos] == v0) {
        removed = c[pos] < d ? c[pos] : d;
        c[pos] -= removed;
        if (c[pos] == 0) {
            memmove(&v[pos], &v[pos + 1], (k - pos - 1) * 8);
            memmove(&c[pos], &c[pos + 1], (k - pos - 1) * 8);
            k--;
        }
        int64_t len = encode_groups(G, v, c, k, slots);
        replace_run(G, x, slots, len);
    }
    return removed;
}

uint64_t or_gqf_insert_groups(or_gqf *G, const uint64_t *fps, const uint64_t *cnts, uint64_t m)
{
    for (uint64_t i = 0; i < m; i++)
        if (insert_group(G, fps[i], cnts[i])) return i;
    return m;
}

typedef struct {
    uint64_t fp, i;
} pair_t;

static int pair_cmp(const void *a, const void *b)
{
    const pair_t *x = (const pair_t *)a, *y = (const pair_t *)b;
    if (x->fp != y->fp) return x->fp < y->fp ? -1 : 1;
    return (x->i > y->i) - (x->i < y->i);
}

void or_gqf_insert(or_gqf *G, const uint64_t *keys, uint64_t n, uint8_t *status)
{
    or_gqf_insert_counts(G, keys, NULL, n, status);
}

void or_gqf_insert_counts(or_gqf *G, const uint64_t *keys, const uint32_t *counts, uint64_t n, uint8_t *status)
{
    if (n == 0) return;
    pair_t *P = malloc(n * sizeof(pair_t));
    for (uint64_t i = 0; i < n; i++) P[i] = (pair_t){fp_of(G, keys[i]), i};
    qsort(P, n, sizeof(pair_t), pair_cmp);
    int overflowed = 0;
    for (uint64_t s = 0; s < n;) {
        uint64_t e = s;
        while (e < n && P[e].fp == P[s].fp) e++;
        uint64_t c = e - s;
        if (counts) {
            c = 0;
            for (uint64_t k = s; k < e; k++) c += counts[P[k].i];
        }
        if (!overflowed && insert_group(G, P[s].fp, c)) overflowed = 1;
        if (status)
            for (uint64_t k = s; k < e; k++) status[P[k].i] = overflowed ? 1 : 0;
        s = e;
    }
    free(P);
}

void or_gqf_remove(or_gqf *G, const uint64_t *keys, uint64_t n, uint8_t *status)
{
    if (n == 0) return;
    pair_t *P = malloc(n * sizeof(pair_t));
    for (uint64_t i = 0; i < n; i++) P[i] = (pair_t){fp_of(G, keys[i]), i};
    qsort(P, n, sizeof(pair_t), pair_cmp);
    for (uint64_t e = n; e > 0;) {
        uint64_t s = e - 1;
        while (s > 0 && P[s - 1].fp == P[e - 1].fp) s--;
        uint64_t removed = delete_group(G, P[s].fp, e - s);
        if (status)
            for (uint64_t k = s; k < e; k++) status[P[k].i] = (k - s) < removed ? 0 : 2;
        e = s;
    }
    free(P);
}

uint64_t or_gqf_count_fp(const or_gqf *G, uint64_t fp)
{
    int64_t x = (int64_t)(fp >> G->r);
    uint64_t v0 = fp & G->rmask;
    if (!occ_get(G, x)) return 0;
    int64_t s = imax(x, prev_end(G, x) + 1);
    int64_t e = runend_of(G, x);
    /* walk the run without materialising it */
    int64_t i = s;
    while (i <= e) {
        uint64_t val = G->rem[i], c = 1;
        int64_t step = 1;
        if (i + 2 <= e && G->rem[i + 1] == val) {
            unsigned nd = G->rem[i + 2];
            uint64_t acc = 0;
            for (unsigned d = 0; d < nd; d++) acc = (acc << G->r) | G->rem[i + 3 + d];
            c = acc + 2;
            step = 3 + nd;
        }
        if (val == v0) return c;
        if (val > v0) return 0;
        i += step;
    }
    return 0;
}

void or_gqf_count(const or_gqf *G, const uint64_t *keys, uint64_t n, uint64_t *counts)
{
    for (uint64_t i = 0; i < n; i++) counts[i] = or_gqf_count_fp(G, fp_of(G, keys[i]));
}

/* every stored group, by the plain definition: the k-th occupied quotient
   owns the k-th run, which starts at max(quotient, previous end + 1) */
uint64_t or_gqf_groups(const or_gqf *G, uint64_t *fps, uint64_t *cnts, uint64_t cap)
{
    uint64_t *v = malloc(G->maxg * 8), *c = malloc(G->maxg * 8);
    uint64_t total = 0;
    int64_t prev = -1, pos = 0;
    for (int64_t x = 0; x < (int64_t)G->N; x++) {
        if (!occ_get(G, x)) continue;
        int64_t s = imax(x, prev + 1);
        while (pos < (int64_t)G->nslots && (pos < s || !rend_get(G, pos))) pos++;
        int64_t e = pos;
        uint64_t k = parse_run(G, s, e, v, c);
        for (uint64_t i = 0; i < k; i++) {
            if (total < cap) {
                fps[total] = ((uint64_t)x << G->r) | v[i];
                cnts[total] = c[i];
            }
            total++;
        }
        prev = e;
        pos = e + 1;
    }
    free(v);
    free(c);
    return total;
}

uint64_t or_gqf_max_cluster(const or_gqf *G)
{
    uint64_t best = 0, cur = 0;
    int64_t prev = -1, pos = 0, cstart = -1;
    for (int64_t x = 0; x < (int64_t)G->N; x++) {
        if (!occ_get(G, x)) continue;
        int64_t s = imax(x, prev + 1);
        while (pos < (int64_t)G->nslots && (pos < s || !rend_get(G, pos))) pos++;
        if (s > prev + 1 || cstart < 0) cstart = s;
        cur = (uint64_t)(pos - cstart + 1);
        if (cur > best) best = cur;
        prev = pos;
        pos++;
    }
    return best;
}

uint64_t or_gqf_export_size(const or_gqf *G) { return G->nblk * 32 + G->nslots * (G->r / 8); }

static void put64(uint8_t *b, uint64_t v)
{
    for (int i = 0; i < 8; i++) b[i] = (uint8_t)(v >> (8 * i));
}

static void export_arrays(uint64_t nblk, uint64_t nslots, unsigned r, const uint64_t *occ,
                          const uint64_t *rend, const uint32_t *off, const uint16_t *rem,
                          uint8_t *buf)
{
    memset(buf, 0, nblk * 32);
    for (uint64_t j = 0; j < nblk; j++) {
        put64(buf + 32 * j, occ[j]);
        put64(buf + 32 * j + 8, rend[j]);
        for (int i = 0; i < 4; i++) buf[32 * j + 16 + i] = (uint8_t)(off[j] >> (8 * i));
    }
    uint8_t *rb = buf + nblk * 32;
    for (uint64_t i = 0; i < nslots; i++) {
        if (r == 8) {
            rb[i] = (uint8_t)rem[i];
        } else {
            rb[2 * i] = (uint8_t)(rem[i] & 0xff);
            rb[2 * i + 1] = (uint8_t)(rem[i] >> 8);
        }
    }
}

void or_gqf_export(const or_gqf *G, uint8_t *buf)
{
    export_arrays(G->nblk, G->nslots, G->r, G->occ, G->rend, G->off, G->rem, buf);
}

/*
 * Canonical builder, written from the definition alone (no shifting): walk
 * the sorted groups quotient by quotient, place each run at max(x, previous
 * end + 1), then give block j the offset of the last run whose quotient is
 * <= 64j.
 */
int or_gqf_build(unsigned q, unsigned r, const uint64_t *fps, const uint64_t *cnts, uint64_t m,
                 uint8_t *buf)
{
    uint64_t N = 1ULL << q, S = or_gqf_tail_slots(q), ns = N + S, nblk = ns / 64;
    uint64_t *occ = calloc(nblk, 8), *rend = calloc(nblk, 8);
    uint32_t *off = calloc(nblk, 4);
    uint16_t *rem = calloc(ns, 2);
    int64_t *rq = malloc((m + 1) * 8), *re = malloc((m + 1) * 8);
    uint64_t nruns = 0;
    int64_t prev = -1;
    int bad = 0;
    for (uint64_t i = 0; i < m && !bad;) {
        uint64_t x = fps[i] >> r;
        uint64_t j = i;
        int64_t len = 0;
        while (j < m && (fps[j] >> r) == x) {
            len += cnts[j] == 1 ? 1 : 3 + ndigits(cnts[j] - 2, r);
            j++;
        }
        int64_t start = imax((int64_t)x, prev + 1), end = start + len - 1;
        if (end >= (int64_t)ns) {
            bad = 1;
            break;
        }
        int64_t at = start;
        for (uint64_t k = i; k < j; k++) {
            uint64_t v = fps[k] & ((1ULL << r) - 1ULL), c = cnts[k];
            rem[at++] = (uint16_t)v;
            if (c >= 2) {
                uint64_t val = c - 2;
                unsigned n = ndigits(val, r);
                rem[at++] = (uint16_t)v;
                rem[at++] = (uint16_t)n;
                for (unsigned d = 0; d < n; d++)
                    rem[at++] = (uint16_t)((val >> (r * (n - 1 - d))) & ((1ULL << r) - 1ULL));
            }
        }
        occ[x >> 6] |= 1ULL << (x & 63);
        rend[end >> 6] |= 1ULL << (end & 63);
        rq[nruns] = (int64_t)x;
        re[nruns] = end;
        nruns++;
        prev = end;
        i = j;
    }
    if (!bad) {
        uint64_t k = 0;
        int64_t last_end = -1;
        int have = 0;
        for (uint64_t j = 0; j < nblk; j++) {
            int64_t Q = (int64_t)(64 * j);
            while (k < nruns && rq[k] <= Q) {
                last_end = re[k];
                have = 1;
                k++;
            }
            off[j] = have ? (uint32_t)imax(0, last_end - Q) : 0;
        }
        export_arrays(nblk, ns, r, occ, rend, off, rem, buf);
    }
    free(occ);
    free(rend);
    free(off);
    free(rem);
    free(rq);
    free(re);
    return bad;
}
