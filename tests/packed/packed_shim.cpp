// Host-side driver for the packed TCF block functions (gf_packed.cuh), for
// the CPU tests: one operation per call on a block given as 32-bit words.
#include "gf_packed.cuh"

using gf::Packed;

template <int F, int B>
static int run(int op, uint32_t *w, int a, int b, const uint32_t *nv, uint32_t *out)
{
    Packed<F, B> p;
    for (int k = 0; k < Packed<F, B>::WORDS; k++) p.w[k] = w[k];
    switch (op) {
    case 0: out[0] = p.get(a); break;
    case 1: p.set(a, (uint32_t)b); break;
    case 2: out[0] = (uint32_t)p.fill(); break;
    case 3: out[0] = (uint32_t)p.find(nv[0], nv[1]); break;
    case 4: p.merge_sorted(a, nv, b); break;
    case 5: p.delete_at(a, b); break;
    case 6: out[0] = p.min_value(nv[0], nv[1]); break;
    default: return -1;
    }
    for (int k = 0; k < Packed<F, B>::WORDS; k++) w[k] = p.w[k];
    return Packed<F, B>::WORDS;
}

extern "C" int packed_op(int f, int B, int op, uint32_t *w, int a, int b, const uint32_t *nv, uint32_t *out)
{
#define GF_CASE(F_, B_) \
    if (f == F_ && B == B_) return run<F_, B_>(op, w, a, b, nv, out);
    GF_CASE(16, 16)
    GF_CASE(8, 32)
    GF_CASE(12, 21)
    GF_CASE(12, 42)
    GF_CASE(16, 8)
    GF_CASE(16, 64)
    GF_CASE(16, 128)
    GF_CASE(8, 64)
#undef GF_CASE
    return -1;
}
