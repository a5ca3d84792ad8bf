// Key hashing of the two filters (paper Sec. 4 block pair and tag, Sec. 5.1
// fingerprint h), shared by the CUDA library and the device-side API of
// gpufilter_device.cuh so that the two cannot drift apart. Host and device.
//
// mix64 is the Murmur3 64-bit finaliser shape (xor-shifts and odd-constant
// products, a bijection of 64-bit words). The GQF fingerprint of a key is
// the key folded to p bits (xor of its p-bit chunks), xored with the seed,
// then the same rounds mod 2^p with shifts by ceil(p / 2): a bijection of
// p-bit words, so a fingerprint can be inverted back to the folded key.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define GF_HASH_FN __host__ __device__ __forceinline__
#else
#define GF_HASH_FN inline
#endif

namespace gf {

GF_HASH_FN uint64_t mix64(uint64_t x)
{
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

struct PHash {
    uint64_t mask;  // 2^p - 1
    uint64_t seed;  // seed mod 2^p
    uint32_t p, s;  // width and shift ceil(p/2)
};

GF_HASH_FN PHash phash_of(uint32_t p, uint64_t seed)
{
    PHash H;
    H.p = p;
    H.s = (p + 1) / 2;
    H.mask = p >= 64 ? ~0ull : ((1ull << p) - 1ull);
    H.seed = seed & H.mask;
    return H;
}

GF_HASH_FN uint64_t fold_p(uint64_t x, const PHash &H)
{
    if (H.p >= 64) return x;
    uint64_t r = 0;
    while (x) {
        r ^= x & H.mask;
        x >>= H.p;
    }
    return r;
}

GF_HASH_FN uint64_t fingerprint(uint64_t key, const PHash &H)
{
    uint64_t x = fold_p(key, H) ^ H.seed;
    x ^= x >> H.s;
    x = (x * 0xff51afd7ed558ccdull) & H.mask;
    x ^= x >> H.s;
    x = (x * 0xc4ceb9fe1a85ec53ull) & H.mask;
    x ^= x >> H.s;
    return x;
}

// TCF: the second block of a pair, b2 = b1 xor g(tag) (never b1 itself)
GF_HASH_FN uint64_t tcf_g(uint32_t t, uint64_t nb)
{
    uint64_t g = mix64((uint64_t)t) & (nb - 1);
    return g ? g : 1;
}

// TCF: block pair and tag of a key (tmask: the tag bits; tags 0 and 1, EMPTY
// and TOMBSTONE, move to 2 and 3)
GF_HASH_FN void tcf_key_parts(uint64_t key, uint64_t seed, uint64_t nb, uint32_t tmask, uint64_t &b1, uint64_t &b2,
                              uint32_t &tag)
{
    const uint64_t h = mix64(key ^ seed);
    uint32_t t = (uint32_t)((h >> 44) & tmask);
    if (t < 2) t += 2;
    tag = t;
    b1 = h & (nb - 1);
    b2 = b1 ^ tcf_g(t, nb);
}

// TCF: the backing bucket of an entry (min(b1, b2) << f | tag) among nbk
GF_HASH_FN uint64_t tcf_bucket(uint64_t e, uint64_t nbk) { return ((mix64(e) >> 32) * nbk) >> 32; }

}  // namespace gf
