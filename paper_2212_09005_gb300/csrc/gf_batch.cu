// The batched work list (C ABI in include/gpufilter.h): one call applies a
// list of (group, member, operation, device key range) items to a TCF group
// and a GQF group. The list lives in host memory, so that every launch is
// sized when it is enqueued; the items' keys and results are device buffers.
// Nothing synchronises the host: a sequence of calls can be captured in one
// CUDA graph and replayed.
//
// Per group the operations run as classes, in this order: inserts, removes,
// queries, counts. A class gathers its items' keys into one member-ordered
// array (a member's items in list order), runs one group call over it, and
// scatters the results back to the items. The descriptors of a call (member
// offsets, item placements) travel inside the parameters of small upload
// kernels (up to 32 KB each), which write them to one device buffer ahead of
// the call's other launches. A launch keeps its parameters by value, so the
// host may build the next call's descriptors at once, and a captured graph
// carries its own copy; calls and replays on one stream run in order and
// can share that buffer.
#include <cstring>
#include <new>
#include <vector>

#include "gf_internal.cuh"

namespace {

// 16-byte words of descriptors one upload kernel carries (the parameter
// space of a launch holds 32,764 bytes; this leaves room for the others)
constexpr uint32_t UPLOAD_WORDS = 2040;

struct UploadChunk {
    uint4 w[UPLOAD_WORDS];
};

struct ItemDesc {
    const uint64_t *src;  // the item's keys
    void *out;            // its results, or null
    uint64_t n;
    uint64_t dst;  // position of its first key in the class's member-ordered array
    uint64_t at;   // position of its first key in the class's list-ordered numbering
};

}  // namespace

struct filter_batch {
    filter_group *g[2] = {nullptr, nullptr};  // TCF, GQF
    uint64_t max_keys = 0;
    uint32_t max_items = 0;
    uint64_t *d_keys = nullptr;  // gathered keys of one class
    uint8_t *d_out = nullptr;    // its results (8 bytes per key)
    char *d_desc = nullptr;      // descriptors of the current call
    std::vector<uint4> h_desc;   // their host image (built per call)
    size_t desc_bytes = 0;
    int device = 0;
};

namespace {

__global__ void batch_upload(const __grid_constant__ UploadChunk c, uint32_t words, uint4 *dst)
{
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) dst[i] = c.w[i];
}

// key j of a class (list order) goes to its member-ordered place
__global__ void batch_gather(const ItemDesc *__restrict__ items, uint32_t ni, uint64_t total, uint64_t *keys)
{
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < total; j += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = ni;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (items[mid].at <= j) lo = mid;
            else hi = mid;
        }
        const ItemDesc &d = items[lo];
        const uint64_t p = j - d.at;
        keys[d.dst + p] = d.src[p];
    }
}

// results back to the items (rb bytes per result)
__global__ void batch_scatter(const ItemDesc *__restrict__ items, uint32_t ni, uint64_t total, const uint8_t *res,
                              uint32_t rb)
{
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < total; j += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = ni;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (items[mid].at <= j) lo = mid;
            else hi = mid;
        }
        const ItemDesc &d = items[lo];
        if (!d.out) continue;
        const uint64_t p = j - d.at;
        if (rb == 8) static_cast<uint64_t *>(d.out)[p] = reinterpret_cast<const uint64_t *>(res)[d.dst + p];
        else static_cast<uint8_t *>(d.out)[p] = res[d.dst + p];
    }
}

static void batch_free(filter_batch *B)
{
    if (!B) return;
    gf::dev_free(B->d_keys);
    gf::dev_free(B->d_out);
    gf::dev_free(B->d_desc);
    delete B;
}

}  // namespace

extern "C" {

int filter_batch_create(filter_group_t *tcf, filter_group_t *gqf, uint64_t max_keys, uint32_t max_items,
                        filter_batch_t **out)
{
    if (!out || (!tcf && !gqf) || max_keys == 0 || max_items == 0) return FILTER_ERR_ARG;
    if ((tcf && tcf->kind != FILTER_TCF) || (gqf && gqf->kind != FILTER_GQF)) return FILTER_ERR_ARG;
    *out = nullptr;
    filter_batch *B = new (std::nothrow) filter_batch();
    if (!B) return FILTER_ERR_OOM;
    B->g[0] = tcf;
    B->g[1] = gqf;
    B->max_keys = max_keys;
    B->max_items = max_items;
    cudaGetDevice(&B->device);
    uint64_t nm = 0;
    for (int g = 0; g < 2; g++)
        if (B->g[g] && B->g[g]->n > nm) nm = B->g[g]->n;
    // one call: at most 8 classes of member offsets, and one descriptor per item
    B->desc_bytes = (8 * (((nm + 1) * 8 + 255) & ~255ull) + (uint64_t)max_items * sizeof(ItemDesc) + 8 * 256 + 255) &
                    ~(size_t)255;
    try {
        B->h_desc.resize(B->desc_bytes / 16);
    } catch (...) {
        batch_free(B);
        return FILTER_ERR_OOM;
    }
    if (gf::dev_malloc(reinterpret_cast<void **>(&B->d_keys), max_keys * 8) != cudaSuccess ||
        gf::dev_malloc(reinterpret_cast<void **>(&B->d_out), max_keys * 8) != cudaSuccess ||
        gf::dev_malloc(reinterpret_cast<void **>(&B->d_desc), B->desc_bytes) != cudaSuccess) {
        cudaGetLastError();
        batch_free(B);
        return FILTER_ERR_OOM;
    }
    *out = B;
    return FILTER_OK;
}

int filter_batch_destroy(filter_batch_t *b)
{
    if (!b) return FILTER_OK;
    const int rc = cudaDeviceSynchronize() == cudaSuccess ? FILTER_OK : FILTER_ERR_CUDA;
    batch_free(b);
    return rc;
}

int filter_batch_run(filter_batch_t *B, const filter_work *items, uint32_t n_items, void *stream)
{
    if (!B || (n_items && !items) || n_items > B->max_items) return FILTER_ERR_ARG;
    // validate every item and the class totals before anything is enqueued
    uint64_t tot[2][4] = {{0}};
    for (uint32_t i = 0; i < n_items; i++) {
        const filter_work &w = items[i];
        if (w.group > 1 || !B->g[w.group] || w.member >= B->g[w.group]->n || w.op > FILTER_OP_COUNT ||
            (w.n && !w.d_keys))
            return FILTER_ERR_ARG;
        if (w.op == FILTER_OP_COUNT && w.group == 0) return FILTER_ERR_UNSUPPORTED;
        tot[w.group][w.op] += w.n;
    }
    for (int g = 0; g < 2; g++)
        for (int op = 0; op < 4; op++) {
            if (tot[g][op] == 0) continue;  // (only a configured group has items)
            if (tot[g][op] > B->max_keys) return FILTER_ERR_ARG;
            if ((op == FILTER_OP_INSERT || op == FILTER_OP_REMOVE) && tot[g][op] > B->g[g]->max_total)
                return FILTER_ERR_ARG;
        }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // descriptors of every class, built on the host first
    struct Class {
        int g;
        uint32_t op, ni;
        uint64_t n;
        size_t off_at, desc_at;  // byte offsets in the descriptor buffer
        bool want_out;
    };
    Class cls[8];
    int ncls = 0;
    char *h = reinterpret_cast<char *>(B->h_desc.data());
    size_t used = 0;
    static const uint32_t order[4] = {FILTER_OP_INSERT, FILTER_OP_REMOVE, FILTER_OP_QUERY, FILTER_OP_COUNT};
    std::vector<uint64_t> cursor;
    for (int g = 0; g < 2; g++) {
        filter_group *G = B->g[g];
        if (!G) continue;
        for (uint32_t op : order) {
            if (tot[g][op] == 0) continue;
            Class &c = cls[ncls++];
            c.g = g;
            c.op = op;
            c.want_out = false;
            const uint32_t nm = G->n;
            c.off_at = used;
            uint64_t *h_off = reinterpret_cast<uint64_t *>(h + used);
            used += (((size_t)nm + 1) * 8 + 255) & ~(size_t)255;
            c.desc_at = used;
            ItemDesc *h_item = reinterpret_cast<ItemDesc *>(h + used);
            // member offsets of the class, then each item's place
            std::memset(h_off, 0, ((size_t)nm + 1) * 8);
            for (uint32_t i = 0; i < n_items; i++)
                if (items[i].group == (uint32_t)g && items[i].op == op && items[i].n) h_off[items[i].member + 1] += items[i].n;
            for (uint32_t m = 0; m < nm; m++) h_off[m + 1] += h_off[m];
            cursor.assign(h_off, h_off + nm);
            uint64_t at = 0;
            uint32_t k = 0;
            for (uint32_t i = 0; i < n_items; i++) {
                const filter_work &w = items[i];
                if (w.group != (uint32_t)g || w.op != op || !w.n) continue;
                h_item[k++] = ItemDesc{w.d_keys, w.d_out, w.n, cursor[w.member], at};
                c.want_out |= w.d_out != nullptr;
                cursor[w.member] += w.n;
                at += w.n;
            }
            c.ni = k;
            c.n = at;
            used += ((size_t)k * sizeof(ItemDesc) + 255) & ~(size_t)255;
        }
    }
    // to the device, inside the parameters of the upload launches
    {
        const uint32_t words = (uint32_t)(used / 16);
        gf::TraceScope ts_("batch_upload", words, st);
        for (uint32_t w0 = 0; w0 < words; w0 += UPLOAD_WORDS) {
            const uint32_t nw = words - w0 < UPLOAD_WORDS ? words - w0 : UPLOAD_WORDS;
            UploadChunk chunk;
            std::memcpy(chunk.w, B->h_desc.data() + w0, (size_t)nw * 16);
            batch_upload<<<1, 256, 0, st>>>(chunk, nw, reinterpret_cast<uint4 *>(B->d_desc) + w0);
        }
        GF_CUDA(cudaGetLastError());
    }
    for (int ci = 0; ci < ncls; ci++) {
        const Class &c = cls[ci];
        filter_group *G = B->g[c.g];
        const uint64_t *d_off = reinterpret_cast<const uint64_t *>(B->d_desc + c.off_at);
        const ItemDesc *d_item = reinterpret_cast<const ItemDesc *>(B->d_desc + c.desc_at);
        const uint64_t n = c.n;
        {
            gf::TraceScope ts_("batch_gather", n, st);
            batch_gather<<<gf::grid_for(n, 256, 8), 256, 0, st>>>(d_item, c.ni, n, B->d_keys);
        }
        uint8_t *res = c.want_out ? B->d_out : nullptr;
        int rc;
        if (c.g == 0) {
            const int gop = c.op == FILTER_OP_INSERT ? gf::GROUP_INSERT
                                                     : (c.op == FILTER_OP_REMOVE ? gf::GROUP_REMOVE : gf::GROUP_QUERY);
            if (gop == gf::GROUP_QUERY && !res) res = B->d_out;  // a query always needs somewhere to answer
            rc = gf::tcf_group_op(G, gop, d_off, B->d_keys, n, res, st);
        } else if (c.op == FILTER_OP_INSERT || c.op == FILTER_OP_REMOVE) {
            rc = gf::gqf_group_update_async(G, d_off, B->d_keys, n, res, c.op == FILTER_OP_REMOVE, st);
        } else if (c.op == FILTER_OP_QUERY) {
            rc = gf::gqf_group_count(G, d_off, B->d_keys, n, nullptr, B->d_out, st);
        } else {
            rc = gf::gqf_group_count(G, d_off, B->d_keys, n, reinterpret_cast<uint64_t *>(B->d_out), nullptr, st);
        }
        if (rc != FILTER_OK) return rc;
        if (c.want_out) {
            gf::TraceScope ts_("batch_scatter", n, st);
            batch_scatter<<<gf::grid_for(n, 256, 8), 256, 0, st>>>(d_item, c.ni, n, B->d_out,
                                                                   c.op == FILTER_OP_COUNT ? 8u : 1u);
        }
        GF_CUDA(cudaGetLastError());
    }
    return FILTER_OK;
}

}  // extern "C"
