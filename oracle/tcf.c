/*
 * Oracle two-choice filter (TCF). TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Specification (paper Sec. 4; the readings taken where it is silent are
 * marked R):
 *
 *  Table. nb = N / B blocks of B tags of f bits; one block is 32 bytes, so
 *  B = 16 for f = 16 and B = 32 for f = 8 (Sec. 4.1 bounds a block by a cache
 *  line; R: one 32-byte sector). Tag 0 is EMPTY, tag 1 is TOMBSTONE (Alg. 1).
 *
 *  Key -> (b1, tag, b2). h = mix64(key ^ seed); b1 = h mod nb (nb a power of
 *  two); tag = bits 44.. of h, f bits wide, with 0 and 1 moved to 2 and 3;
 *  b2 = b1 xor g(tag), g(tag) = mix64(tag) mod nb, or 1 when that is 0.
 *  (Sec. 4 picks two blocks "via a pair of unique hashes"; R: partial-key
 *  pairing, so a fingerprint is the unordered pair {b1, b2} plus the tag and
 *  a query answer is the membership of that fingerprint.)
 *
 *  Deterministic bulk insert of one batch (Sec. 4.1 shortcut, Sec. 4
 *  power-of-two-choice, Sec. 4.1 backing table, Sec. 4.2 sorted blocks;
 *  R: the phase order below makes the table a function of the batch).
 *  Candidates of a block are always taken in (tag, batch index) order.
 *   A  shortcut: block b takes its j-th candidate with b1 = b iff
 *      fill(b) + j < 3B/4.
 *   B  two-choice: every other key targets b1 if fillA(b1) <= fillA(b2),
 *      else b2 (fillA = fills after A); block b takes its j-th candidate iff
 *      fillA(b) + j < B.
 *   C  other block: every key rejected in B targets its other block; block b
 *      takes its j-th candidate iff fillB(b) + j < B.
 *   D  backing table: entry e = (min(b1, b2) << f) | tag lands in bucket
 *      ((mix64(e) >> 32) * nbk) >> 32 of nbk buckets of W = 8 entries,
 *      nbk = max(8, ceil(ceil(N / 100) / 8)) (Sec. 4.1 sizes it to 1/100 of
 *      the table; R: sorted buckets instead of double hashing). Bucket k takes
 *      its j-th candidate, in (e, batch index) order, iff fill(k) + j < W.
 *      The rest are rejected: status 1 (full).
 *   Afterwards every block holds its tags in ascending order followed by
 *   EMPTY, and every bucket its entries ascending followed by 0.
 *
 *  Query: tag in block b1, or in block b2, or e in its bucket.
 *
 *  Other geometries (Sec. 4.1 bounds the point TCF's block by a 128-byte
 *  cache line; Sec. 4.2 gives the bulk TCF 128-slot blocks of 16 bits; the
 *  design study varies the block size and stores 12-bit tags, which then
 *  straddle word boundaries). nb = 2^k blocks of B slots of f bits, f in
 *  {8, 12, 16}, 4 <= B and f B <= 2048 bits. A block occupies the smallest
 *  multiple of 32 bytes that holds its slots; slot s sits at bit f s of the
 *  block, little-endian, and the bits past the last slot are 0. N = nb B,
 *  the backing table is sized from N as above, and everything else is the
 *  same, with the shortcut at fill + j < floor(3B/4).
 *
 *  Values (Sec. 1 and Sec. 4 list associating small values with items as a
 *  TCF feature; R: the layout below). With v value bits (v <= f / 2, and
 *  v <= 7 so that 0xFF stays free to answer "absent"), a slot of f bits
 *  holds the (f - v)-bit tag in its high bits and the value in its low bits,
 *  so that tag 0 and 1 still never occur and a slot is EMPTY or TOMBSTONE only
 *  when it is 0 or 1. The tag is bits 44.. of h, f - v bits wide; g and the
 *  bucket of an entry depend on the tag and the blocks only (the value bits
 *  are cleared before the bucket hash), so a key's placement never depends on
 *  its value. Candidates of a block are taken in (slot, batch index) order,
 *  slot = tag << v | value, and blocks and buckets stay sorted by slot.
 *  Matching (query, delete) compares the tag part only. A value query answers
 *  the smallest value among all stored copies of the key's fingerprint
 *  (blocks b1, b2 and its backing bucket), or 0xFF when there is none; a
 *  delete removes the first copy in b1, else in b2, else in the bucket, which
 *  in a sorted block or bucket is the one with the smallest value.
 *
 *  Deterministic bulk delete (Sec. 6.4 deletes one copy; R: phases as insert):
 *   1  block b1 removes one copy of the tag for each of its candidates, in
 *      (tag, batch index) order, while a copy is left;
 *   2  the keys still unmatched try b2 the same way;
 *   3  then the backing bucket;
 *   4  the rest get status 2 (not found). Blocks and buckets are recompacted.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

#define BK_W 8u

struct or_tcf {
    unsigned f, B, tsc;
    unsigned bbytes; /* bytes per block in the image */
    unsigned vb;     /* value bits in each slot */
    uint64_t vmask;  /* the value part of a slot or entry */
    uint64_t nb, nbk, seed;
    uint16_t *tags; /* nb * B */
    uint64_t *bk;   /* nbk * BK_W */
};

typedef struct {
    uint64_t g, k, i;
} rec_t;

static int rec_cmp(const void *a, const void *b)
{
    const rec_t *x = (const rec_t *)a, *y = (const rec_t *)b;
    if (x->g != y->g) return x->g < y->g ? -1 : 1;
    if (x->k != y->k) return x->k < y->k ? -1 : 1;
    if (x->i != y->i) return x->i < y->i ? -1 : 1;
    return 0;
}

static int u16_cmp(const void *a, const void *b)
{
    uint16_t x = *(const uint16_t *)a, y = *(const uint16_t *)b;
    return (x > y) - (x < y);
}

static int u64_cmp(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

or_tcf *or_tcf_new(unsigned log2_slots, unsigned tag_bits, uint64_t seed)
{
    return or_tcf_new_values(log2_slots, tag_bits, 0, seed);
}

or_tcf *or_tcf_new_values(unsigned log2_slots, unsigned tag_bits, unsigned value_bits, uint64_t seed)
{
    if (tag_bits != 8 && tag_bits != 16) return NULL;
    unsigned B = 256u / tag_bits;
    unsigned lb = (B == 16) ? 4 : 5;
    if (log2_slots < lb + 1 || log2_slots > 40) return NULL;
    return or_tcf_new_geom(log2_slots - lb, tag_bits, B, value_bits, seed);
}

or_tcf *or_tcf_new_geom(unsigned log2_blocks, unsigned tag_bits, unsigned block_slots, unsigned value_bits,
                        uint64_t seed)
{
    if (tag_bits != 8 && tag_bits != 12 && tag_bits != 16) return NULL;
    if (value_bits > tag_bits / 2 || value_bits > 7) return NULL; /* 0xFF answers "absent" */
    unsigned B = block_slots;
    if (B < 4 || tag_bits * B > 2048 || log2_blocks < 1 || log2_blocks > 34) return NULL;
    or_tcf *T = (or_tcf *)calloc(1, sizeof(or_tcf));
    T->f = tag_bits;
    T->vb = value_bits;
    T->vmask = (1ULL << value_bits) - 1ULL;
    T->B = B;
    T->tsc = 3 * B / 4;
    T->bbytes = (tag_bits * B + 255) / 256 * 32;
    T->nb = 1ULL << log2_blocks;
    T->seed = seed;
    uint64_t N = T->nb * B;
    uint64_t cap = (N + 99) / 100;
    T->nbk = (cap + BK_W - 1) / BK_W;
    if (T->nbk < 8) T->nbk = 8;
    T->tags = (uint16_t *)calloc(T->nb * B, sizeof(uint16_t));
    T->bk = (uint64_t *)calloc(T->nbk * BK_W, sizeof(uint64_t));
    if (!T->tags || !T->bk) {
        or_tcf_free(T);
        return NULL;
    }
    return T;
}

void or_tcf_free(or_tcf *T)
{
    if (!T) return;
    free(T->tags);
    free(T->bk);
    free(T);
}

void or_tcf_geometry(const or_tcf *T, uint64_t *o)
{
    o[0] = T->nb;
    o[1] = T->B;
    o[2] = T->f;
    o[3] = T->tsc;
    o[4] = T->nbk;
    o[5] = BK_W;
    o[6] = T->vb;
    o[7] = T->bbytes;
}

static void keyinfo1(const or_tcf *T, uint64_t key, uint64_t *b1, uint64_t *b2, uint32_t *t)
{
    uint64_t h = or_mix64(key ^ T->seed);
    uint64_t tag = (h >> 44) & ((1ULL << (T->f - T->vb)) - 1ULL);
    if (tag < 2) tag += 2;
    uint64_t g = or_mix64(tag) & (T->nb - 1);
    if (g == 0) g = 1;
    *b1 = h & (T->nb - 1);
    *b2 = *b1 ^ g;
    *t = (uint32_t)(tag << T->vb); /* the slot with value 0 */
}

void or_tcf_keyinfo(const or_tcf *T, const uint64_t *keys, uint64_t n, uint64_t *b1,
                    uint64_t *b2, uint32_t *tag)
{
    for (uint64_t i = 0; i < n; i++) keyinfo1(T, keys[i], &b1[i], &b2[i], &tag[i]);
}

static uint64_t entry_of(const or_tcf *T, uint64_t b1, uint64_t b2, uint32_t t)
{
    uint64_t lo = b1 < b2 ? b1 : b2;
    return (lo << T->f) | t;
}

static uint64_t bucket_of(const or_tcf *T, uint64_t e)
{
    e &= ~T->vmask;
    return ((or_mix64(e) >> 32) * T->nbk) >> 32;
}

/* slot or entry x holds tag (or entry) t, whatever its value */
static int same_tag(const or_tcf *T, uint64_t x, uint64_t t)
{
    return x != 0 && (x & ~T->vmask) == t;
}

static unsigned block_fill(const or_tcf *T, uint64_t b)
{
    unsigned c = 0;
    for (unsigned s = 0; s < T->B; s++) c += T->tags[b * T->B + s] != 0;
    return c;
}

static void block_put(or_tcf *T, uint64_t b, uint32_t t)
{
    for (unsigned s = 0; s < T->B; s++) {
        if (T->tags[b * T->B + s] == 0) {
            T->tags[b * T->B + s] = (uint16_t)t;
            return;
        }
    }
    abort(); /* callers check the fill first */
}

static int block_has(const or_tcf *T, uint64_t b, uint32_t t)
{
    for (unsigned s = 0; s < T->B; s++)
        if (same_tag(T, T->tags[b * T->B + s], t)) return 1;
    return 0;
}

/* smallest value stored with tag t in block b, folded into *best */
static void block_min_value(const or_tcf *T, uint64_t b, uint32_t t, unsigned *best)
{
    for (unsigned s = 0; s < T->B; s++) {
        uint64_t x = T->tags[b * T->B + s];
        if (same_tag(T, x, t) && (x & T->vmask) < *best) *best = (unsigned)(x & T->vmask);
    }
}

static int block_take(or_tcf *T, uint64_t b, uint32_t t)
{
    for (unsigned s = 0; s < T->B; s++) {
        if (same_tag(T, T->tags[b * T->B + s], t)) {
            T->tags[b * T->B + s] = 0;
            return 1;
        }
    }
    return 0;
}

/* ascending tags, EMPTY padding */
static void block_canon(or_tcf *T, uint64_t b)
{
    uint16_t v[256];
    unsigned c = 0;
    for (unsigned s = 0; s < T->B; s++)
        if (T->tags[b * T->B + s]) v[c++] = T->tags[b * T->B + s];
    qsort(v, c, sizeof(uint16_t), u16_cmp);
    for (unsigned s = 0; s < T->B; s++) T->tags[b * T->B + s] = s < c ? v[s] : 0;
}

static unsigned bucket_fill(const or_tcf *T, uint64_t k)
{
    unsigned c = 0;
    for (unsigned s = 0; s < BK_W; s++) c += T->bk[k * BK_W + s] != 0;
    return c;
}

static void bucket_canon(or_tcf *T, uint64_t k)
{
    uint64_t v[BK_W];
    unsigned c = 0;
    for (unsigned s = 0; s < BK_W; s++)
        if (T->bk[k * BK_W + s]) v[c++] = T->bk[k * BK_W + s];
    qsort(v, c, sizeof(uint64_t), u64_cmp);
    for (unsigned s = 0; s < BK_W; s++) T->bk[k * BK_W + s] = s < c ? v[s] : 0;
}

void or_tcf_insert(or_tcf *T, const uint64_t *keys, uint64_t n, uint8_t *status, uint8_t *phase,
                   uint64_t *where)
{
    or_tcf_insert_values(T, keys, NULL, n, status, phase, where);
}

void or_tcf_insert_values(or_tcf *T, const uint64_t *keys, const uint8_t *values, uint64_t n, uint8_t *status,
                          uint8_t *phase, uint64_t *where)
{
    if (n == 0) return;
    uint64_t *b1 = malloc(n * 8), *b2 = malloc(n * 8);
    uint32_t *t = malloc(n * 4);
    uint64_t *tgt = malloc(n * 8);
    rec_t *R = malloc(n * sizeof(rec_t));
    uint64_t *pend = malloc(n * 8);
    or_tcf_keyinfo(T, keys, n, b1, b2, t);
    if (values)
        for (uint64_t i = 0; i < n; i++) t[i] |= (uint32_t)(values[i] & T->vmask);
    if (status) memset(status, 0, n);

    /* Phase A: shortcut into b1 while fill(b1) + j < 3B/4 */
    for (uint64_t i = 0; i < n; i++) R[i] = (rec_t){b1[i], t[i], i};
    qsort(R, n, sizeof(rec_t), rec_cmp);
    uint64_t m = 0;
    for (uint64_t s = 0; s < n;) {
        uint64_t e = s, g = R[s].g;
        while (e < n && R[e].g == g) e++;
        unsigned fill0 = block_fill(T, g);
        for (uint64_t j = 0; j < e - s; j++) {
            uint64_t i = R[s + j].i;
            if (fill0 + j < T->tsc) {
                block_put(T, g, t[i]);
                if (phase) phase[i] = 0;
                if (where) where[i] = g;
            } else {
                pend[m++] = i;
            }
        }
        s = e;
    }

    /* Phase B: target the less full block under the post-A fills (tie: b1) */
    for (uint64_t k = 0; k < m; k++) {
        uint64_t i = pend[k];
        tgt[i] = block_fill(T, b1[i]) <= block_fill(T, b2[i]) ? b1[i] : b2[i];
        R[k] = (rec_t){tgt[i], t[i], i};
    }
    qsort(R, m, sizeof(rec_t), rec_cmp);
    uint64_t m2 = 0;
    for (uint64_t s = 0; s < m;) {
        uint64_t e = s, g = R[s].g;
        while (e < m && R[e].g == g) e++;
        unsigned fill0 = block_fill(T, g);
        for (uint64_t j = 0; j < e - s; j++) {
            uint64_t i = R[s + j].i;
            if (fill0 + j < T->B) {
                block_put(T, g, t[i]);
                if (phase) phase[i] = 1;
                if (where) where[i] = g;
            } else {
                pend[m2++] = i;
            }
        }
        s = e;
    }

    /* Phase C: the keys rejected in B try their other block */
    for (uint64_t k = 0; k < m2; k++) {
        uint64_t i = pend[k];
        uint64_t alt = (tgt[i] == b1[i]) ? b2[i] : b1[i];
        R[k] = (rec_t){alt, t[i], i};
    }
    qsort(R, m2, sizeof(rec_t), rec_cmp);
    uint64_t m3 = 0;
    for (uint64_t s = 0; s < m2;) {
        uint64_t e = s, g = R[s].g;
        while (e < m2 && R[e].g == g) e++;
        unsigned fill0 = block_fill(T, g);
        for (uint64_t j = 0; j < e - s; j++) {
            uint64_t i = R[s + j].i;
            if (fill0 + j < T->B) {
                block_put(T, g, t[i]);
                if (phase) phase[i] = 2;
                if (where) where[i] = g;
            } else {
                pend[m3++] = i;
            }
        }
        s = e;
    }

    /* Phase D: backing table */
    for (uint64_t k = 0; k < m3; k++) {
        uint64_t i = pend[k];
        uint64_t e = entry_of(T, b1[i], b2[i], t[i]);
        R[k] = (rec_t){bucket_of(T, e), e, i};
    }
    qsort(R, m3, sizeof(rec_t), rec_cmp);
    for (uint64_t s = 0; s < m3;) {
        uint64_t e = s, g = R[s].g;
        while (e < m3 && R[e].g == g) e++;
        unsigned fill0 = bucket_fill(T, g);
        for (uint64_t j = 0; j < e - s; j++) {
            uint64_t i = R[s + j].i;
            if (fill0 + j < BK_W) {
                T->bk[g * BK_W + fill0 + j] = R[s + j].k;
                if (phase) phase[i] = 3;
                if (where) where[i] = g;
            } else {
                if (status) status[i] = 1;
                if (phase) phase[i] = 4;
                if (where) where[i] = ~0ULL;
            }
        }
        bucket_canon(T, g);
        s = e;
    }

    for (uint64_t i = 0; i < n; i++) {
        block_canon(T, b1[i]);
        block_canon(T, b2[i]);
    }
    free(b1);
    free(b2);
    free(t);
    free(tgt);
    free(R);
    free(pend);
}

void or_tcf_query(const or_tcf *T, const uint64_t *keys, uint64_t n, uint8_t *found)
{
    for (uint64_t i = 0; i < n; i++) {
        uint64_t b1, b2;
        uint32_t t;
        keyinfo1(T, keys[i], &b1, &b2, &t);
        int hit = block_has(T, b1, t) || block_has(T, b2, t);
        if (!hit) {
            uint64_t e = entry_of(T, b1, b2, t), k = bucket_of(T, e);
            for (unsigned s = 0; s < BK_W; s++)
                if (same_tag(T, T->bk[k * BK_W + s], e)) hit = 1;
        }
        found[i] = (uint8_t)hit;
    }
}

void or_tcf_query_values(const or_tcf *T, const uint64_t *keys, uint64_t n, uint8_t *values)
{
    for (uint64_t i = 0; i < n; i++) {
        uint64_t b1, b2;
        uint32_t t;
        keyinfo1(T, keys[i], &b1, &b2, &t);
        unsigned best = 0x100;
        block_min_value(T, b1, t, &best);
        block_min_value(T, b2, t, &best);
        uint64_t e = entry_of(T, b1, b2, t), k = bucket_of(T, e);
        for (unsigned s = 0; s < BK_W; s++) {
            uint64_t x = T->bk[k * BK_W + s];
            if (same_tag(T, x, e) && (x & T->vmask) < best) best = (unsigned)(x & T->vmask);
        }
        values[i] = best == 0x100 ? 0xFF : (uint8_t)best;
    }
}

void or_tcf_remove(or_tcf *T, const uint64_t *keys, uint64_t n, uint8_t *status)
{
    if (n == 0) return;
    uint64_t *b1 = malloc(n * 8), *b2 = malloc(n * 8);
    uint32_t *t = malloc(n * 4);
    rec_t *R = malloc(n * sizeof(rec_t));
    uint64_t *pend = malloc(n * 8);
    or_tcf_keyinfo(T, keys, n, b1, b2, t);
    if (status) memset(status, 0, n);

    /* Phase 1: primary block */
    for (uint64_t i = 0; i < n; i++) R[i] = (rec_t){b1[i], t[i], i};
    qsort(R, n, sizeof(rec_t), rec_cmp);
    uint64_t m = 0;
    for (uint64_t k = 0; k < n; k++)
        if (!block_take(T, R[k].g, t[R[k].i])) pend[m++] = R[k].i;

    /* Phase 2: secondary block */
    for (uint64_t k = 0; k < m; k++) R[k] = (rec_t){b2[pend[k]], t[pend[k]], pend[k]};
    qsort(R, m, sizeof(rec_t), rec_cmp);
    uint64_t m2 = 0;
    for (uint64_t k = 0; k < m; k++)
        if (!block_take(T, R[k].g, t[R[k].i])) pend[m2++] = R[k].i;

    /* Phase 3: backing bucket; Phase 4: not found */
    for (uint64_t k = 0; k < m2; k++) {
        uint64_t i = pend[k];
        uint64_t e = entry_of(T, b1[i], b2[i], t[i]);
        R[k] = (rec_t){bucket_of(T, e), e, i};
    }
    qsort(R, m2, sizeof(rec_t), rec_cmp);
    for (uint64_t k = 0; k < m2; k++) {
        uint64_t g = R[k].g;
        int done = 0;
        for (unsigned s = 0; s < BK_W && !done; s++) {
            if (same_tag(T, T->bk[g * BK_W + s], R[k].k)) {
                T->bk[g * BK_W + s] = 0;
                done = 1;
            }
        }
        if (!done && status) status[R[k].i] = 2;
        bucket_canon(T, g);
    }
    for (uint64_t i = 0; i < n; i++) {
        block_canon(T, b1[i]);
        block_canon(T, b2[i]);
    }
    free(b1);
    free(b2);
    free(t);
    free(R);
    free(pend);
}

uint64_t or_tcf_export_size(const or_tcf *T)
{
    return T->nb * (uint64_t)T->bbytes + T->nbk * BK_W * 8ULL;
}

/* Byte image of the device table: the blocks (slot s at bit f s of its
   block, little-endian, bbytes per block, unused bits 0) followed by the
   backing buckets (8 little-endian uint64 entries each). */
void or_tcf_export(const or_tcf *T, uint8_t *buf)
{
    uint64_t o = T->nb * (uint64_t)T->bbytes;
    memset(buf, 0, o);
    for (uint64_t b = 0; b < T->nb; b++) {
        uint8_t *blk = buf + b * T->bbytes;
        for (unsigned s = 0; s < T->B; s++) {
            uint32_t v = T->tags[b * T->B + s];
            for (unsigned k = 0; k < T->f; k++) {
                unsigned bit = s * T->f + k;
                if ((v >> k) & 1u) blk[bit >> 3] |= (uint8_t)(1u << (bit & 7));
            }
        }
    }
    for (uint64_t i = 0; i < T->nbk * BK_W; i++) {
        uint64_t v = T->bk[i];
        for (int b = 0; b < 8; b++) buf[o++] = (uint8_t)(v >> (8 * b));
    }
}

uint64_t or_tcf_backing_count(const or_tcf *T)
{
    uint64_t c = 0;
    for (uint64_t i = 0; i < T->nbk * BK_W; i++) c += T->bk[i] != 0;
    return c;
}

uint64_t or_tcf_stored_count(const or_tcf *T)
{
    uint64_t c = 0;
    for (uint64_t i = 0; i < T->nb * T->B; i++) c += T->tags[i] != 0;
    return c + or_tcf_backing_count(T);
}
