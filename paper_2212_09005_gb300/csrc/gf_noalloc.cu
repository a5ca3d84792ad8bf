// GQF bulk insert that allocates nothing: its scratch is a file-scope static
// device array, and the caller passes the table images in and out.
//
// Who needs it: callers that must not call cudaMalloc, e.g. a process whose
// device memory is owned by its own allocator or a fixed arena reserved at
// start-up (a cudaMalloc there would fail on a full device or fragment the
// arena), or a latency-critical path that cannot afford cudaMalloc's implicit
// device synchronisation.
#include <cstring>
#include <mutex>

#include "gf_internal.cuh"

namespace gf {

// Capacity limits of the static scratch.
static constexpr uint64_t NOALLOC_MAX_KEYS = FILTER_NOALLOC_MAX_KEYS;
static constexpr uint32_t NOALLOC_MAX_Q = FILTER_NOALLOC_MAX_Q;
static constexpr size_t NOALLOC_SCRATCH_BYTES = 4u << 20;

// The scratch. Every GPU that loads the library holds this array until the
// process exits. In host code its name is only a host-side stand-in: the
// kernels get the device address looked up by cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[64];

// Device address of the scratch on the current device, looked up once per
// device with that device current.
static int noalloc_scratch(void **out)
{
    int dev = 0;
    GF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return FILTER_ERR_ARG;
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        GF_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return FILTER_OK;
}

}  // namespace gf

extern "C" int filter_gqf_insert_noalloc(uint32_t q, uint32_t r, uint64_t hash_seed, const void *d_table_in,
                                         void *d_table_out, const uint64_t *d_keys, uint64_t n,
                                         uint8_t *d_status, void *stream)
{
    using namespace gf;
    if (q > NOALLOC_MAX_Q || n > NOALLOC_MAX_KEYS || !d_table_in || !d_table_out || (n && !d_keys))
        return FILTER_ERR_ARG;
    filter F;  // host-side description only; nothing is allocated
    F.cfg = filter_config{};
    F.cfg.kind = FILTER_GQF;
    F.cfg.log2_slots = q;
    F.cfg.tag_bits = r;
    F.cfg.mode = 0;
    F.cfg.hash_seed = hash_seed;
    F.cfg.max_batch = NOALLOC_MAX_KEYS;
    uint64_t table_bytes = 0, scratch_bytes = 0;
    int rc = gqf_setup(&F, table_bytes, scratch_bytes, true);
    if (rc != FILTER_OK) return rc;
    GqfState &Q = F.gqf;
    const uint64_t metaB = Q.nblk * 32;
    const char *tin = static_cast<const char *>(d_table_in);
    char *tout = static_cast<char *>(d_table_out);
    const uint64_t imageB = gqf_image_bytes(&F);
    if ((tin < tout + imageB) && (tout < tin + imageB)) return FILTER_ERR_ARG;  // must not overlap

    void *base = nullptr;
    if ((rc = noalloc_scratch(&base)) != FILTER_OK) return rc;
    Arena A;
    A.base = static_cast<char *>(base);
    A.size = NOALLOC_SCRATCH_BYTES;
    const uint64_t M = NOALLOC_MAX_KEYS;
    Q.meta[0] = reinterpret_cast<uint8_t *>(const_cast<char *>(tin));
    Q.rem[0] = reinterpret_cast<uint8_t *>(const_cast<char *>(tin)) + metaB;
    Q.meta[1] = reinterpret_cast<uint8_t *>(tout);
    Q.rem[1] = reinterpret_cast<uint8_t *>(tout) + metaB;
    Q.cur = 0;
    Q.merge_only = true;  // the input image is read only: the result goes to the output image
    F.ctr = A.take<DevCounters>(1);
    Q.fp_a = A.take<uint64_t>(M);
    Q.fp_b = A.take<uint64_t>(M);
    Q.fp_c = A.take<uint64_t>(M);
    Q.ufp = A.take<uint64_t>(M);
    Q.idx_a = A.take<uint32_t>(M);
    Q.idx_b = A.take<uint32_t>(M);
    Q.idx_c = A.take<uint32_t>(M);
    Q.ustart = A.take<uint32_t>(M + 1);
    Q.flags = A.take<uint32_t>(M + 1);
    Q.removed = A.take<uint32_t>(M);
    Q.tile_state = A.take<unsigned long long>(Q.ntiles * 4 + 2);
    Q.tile_lo = A.take<uint32_t>(gqf_tile_lo_words(Q));
    Q.radix_tmp = A.take<uint32_t>(radix_tmp_words(M));
    uint64_t scan_n = radix_tmp_words(M);
    if (M + 1 > scan_n) scan_n = M + 1;
    F.scan_tmp = A.take<uint64_t>(scan_tmp_words(scan_n));
    if (A.used > A.size) return FILTER_ERR_INTERNAL;
    F.arena.base = A.base;  // marks the description valid; never freed

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the scratch keeps the previous call's contents: reset the counters
    GF_CUDA(cudaMemsetAsync(F.ctr, 0, sizeof(DevCounters), st));
    if (n == 0) {
        GF_CUDA(cudaMemcpyAsync(tout, tin, imageB, cudaMemcpyDeviceToDevice, st));
        rc = FILTER_OK;
    } else {
        rc = gqf_insert(&F, d_keys, nullptr, n, d_status, st);
    }
    F.arena.base = nullptr;  // the host description goes out of scope; nothing to free
    return rc;
}
