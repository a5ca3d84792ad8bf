/*
 * Oracle hashing. TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper hashes items to p-bit fingerprints, h : U -> {0 .. 2^p - 1}
 * (Sec. 5.1), and feeds its benchmarks pre-hashed 64-bit items (Sec. 6), but
 * it never names h. Reading taken here: h is invertible, so a fingerprint
 * identifies its key whenever the universe has at most 2^p keys.
 *
 *   mix64(x)  = x ^= x>>33; x *= C1; x ^= x>>33; x *= C2; x ^= x>>33
 *               (the 64-bit Murmur3 finaliser shape; C1, C2 odd)
 *   mix_p(x)  = the same rounds with every product taken mod 2^p and shift
 *               s = ceil(p/2), which makes each xor-shift an involution
 *   fold_p(x) = xor of the successive p-bit chunks of x (identity on x < 2^p)
 *
 * Each step is a bijection: an xor-shift by s >= p/2 is its own inverse and
 * multiplication by an odd constant is inverted by its inverse mod 2^p.
 */
#include "oracle.h"

static const uint64_t C1 = 0xff51afd7ed558ccdULL;
static const uint64_t C2 = 0xc4ceb9fe1a85ec53ULL;

static uint64_t mask_p(unsigned p) { return p >= 64 ? ~0ULL : ((1ULL << p) - 1ULL); }

/* inverse of an odd a mod 2^64 by Newton's iteration y <- y(2 - a y) */
static uint64_t odd_inverse(uint64_t a)
{
    uint64_t y = a;
    for (int i = 0; i < 6; i++) y *= 2ULL - a * y;
    return y;
}

uint64_t or_mix64(uint64_t x)
{
    x ^= x >> 33;
    x *= C1;
    x ^= x >> 33;
    x *= C2;
    x ^= x >> 33;
    return x;
}

uint64_t or_unmix64(uint64_t x)
{
    x ^= x >> 33;
    x *= odd_inverse(C2);
    x ^= x >> 33;
    x *= odd_inverse(C1);
    x ^= x >> 33;
    return x;
}

uint64_t or_mix_p(uint64_t x, unsigned p)
{
    const uint64_t m = mask_p(p);
    const unsigned s = (p + 1) / 2;
    x &= m;
    x ^= x >> s;
    x = (x * C1) & m;
    x ^= x >> s;
    x = (x * C2) & m;
    x ^= x >> s;
    return x;
}

uint64_t or_unmix_p(uint64_t x, unsigned p)
{
    const uint64_t m = mask_p(p);
    const unsigned s = (p + 1) / 2;
    x &= m;
    x ^= x >> s;
    x = (x * odd_inverse(C2)) & m;
    x ^= x >> s;
    x = (x * odd_inverse(C1)) & m;
    x ^= x >> s;
    return x;
}

uint64_t or_fold_p(uint64_t x, unsigned p)
{
    if (p >= 64) return x;
    const uint64_t m = mask_p(p);
    uint64_t r = 0;
    while (x) {
        r ^= x & m;
        x >>= p;
    }
    return r;
}

void or_mix64_many(const uint64_t *in, uint64_t *out, uint64_t n)
{
    for (uint64_t i = 0; i < n; i++) out[i] = or_mix64(in[i]);
}

void or_mix_p_many(const uint64_t *in, uint64_t *out, uint64_t n, unsigned p)
{
    for (uint64_t i = 0; i < n; i++) out[i] = or_mix_p(in[i], p);
}
