// TCF blocks of B slots of F bits packed into 32-bit words (paper Sec. 4.1
// block sizes up to a cache line, the 128-slot blocks of the bulk TCF in
// Sec. 4.2, and 12-bit tags, which Sec. 4 notes no longer fit one atomic
// word each). Slot s occupies bits F*s .. F*s + F - 1 of the block,
// little-endian across the words; the bits past the last slot stay 0; a
// block takes whole 32-byte sectors. Slot 0 is EMPTY; a bulk block keeps its
// live slots sorted ascending, followed by EMPTY.
//
// Host and device: the same functions build and check blocks on the CPU.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define GF_HD __host__ __device__ __forceinline__
#else
#define GF_HD inline
#endif

namespace gf {

template <int F, int B>
struct Packed {
    static_assert(F == 8 || F == 12 || F == 16, "slot width");
    static_assert(B >= 4 && F * B <= 2048, "block size");
    static constexpr int WORDS = (F * B + 255) / 256 * 8;
    static constexpr uint32_t MASK = (1u << F) - 1u;
    uint32_t w[WORDS];

    GF_HD void clear()
    {
        for (int k = 0; k < WORDS; k++) w[k] = 0;
    }
    GF_HD uint32_t get(int s) const
    {
        const int bit = F * s, k = bit >> 5, o = bit & 31;
        uint64_t x = w[k];
        if (o + F > 32) x |= (uint64_t)w[k + 1] << 32;  // the slot straddles two words
        return (uint32_t)(x >> o) & MASK;
    }
    GF_HD void set(int s, uint32_t v)
    {
        const int bit = F * s, k = bit >> 5, o = bit & 31;
        const uint64_t m = (uint64_t)MASK << o, x = (uint64_t)(v & MASK) << o;
        w[k] = (w[k] & ~(uint32_t)m) | (uint32_t)x;
        if (o + F > 32) w[k + 1] = (w[k + 1] & ~(uint32_t)(m >> 32)) | (uint32_t)(x >> 32);
    }
    // slots that are not EMPTY
    GF_HD int fill() const
    {
        int c = 0;
        for (int s = 0; s < B; s++) c += get(s) != 0;
        return c;
    }
    // first slot whose tag part (tmask) equals t, or -1
    GF_HD int find(uint32_t t, uint32_t tmask) const
    {
        for (int s = 0; s < B; s++)
            if ((get(s) & tmask) == t) return s;
        return -1;
    }
    // smallest value part (~tmask) among the slots holding tag t, or MASK + 1
    GF_HD uint32_t min_value(uint32_t t, uint32_t tmask) const
    {
        uint32_t best = MASK + 1u;
        for (int s = 0; s < B; s++) {
            const uint32_t x = get(s);
            if ((x & tmask) == t && (x & ~tmask) < best) best = x & ~tmask;
        }
        return best;
    }
    // a sorted block with f0 live slots takes k more, given ascending in nv;
    // f0 + k <= B. The result is sorted with EMPTY after it.
    GF_HD void merge_sorted(int f0, const uint32_t *nv, int k)
    {
        int a = f0 - 1, b = k - 1;
        for (int o = f0 + k - 1; o >= 0; o--) {  // from the top, so no slot is read after it is written
            const bool take_new = a < 0 || (b >= 0 && nv[b] >= get(a));
            if (take_new) set(o, nv[b--]);
            else set(o, get(a--));
        }
    }
    // remove slot s of a block with f0 live slots, moving the later ones down
    GF_HD void delete_at(int s, int f0)
    {
        for (int p = s; p + 1 < f0; p++) set(p, get(p + 1));
        set(f0 - 1, 0);
    }
};

}  // namespace gf
