// The filter-group part of the C ABI (include/gpufilter.h): argument checks,
// the single allocation of a group, and dispatch to the TCF and GQF group
// paths. Exports of a member go through its host-side view, which points
// into the group's arrays, so the image format is the standalone filter's.
#include <cstring>
#include <new>

#include "gf_internal.cuh"

static cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

static bool valid(const filter_group_t *g) { return g != nullptr && g->arena.base != nullptr && g->members; }

static void group_free(filter_group *G)
{
    if (!G) return;
    gf::dev_free(G->arena.base);
    delete[] G->members;
    delete G;
}

extern "C" {

int filter_group_set_tuning(filter_group_t *g, const filter_tuning *t)
{
    if (!valid(g) || !t || !gf::tuning_valid(*t)) return FILTER_ERR_ARG;
    g->tune = *t;
    for (uint32_t m = 0; m < g->n; m++) g->members[m].tune = *t;
    return FILTER_OK;
}

int filter_group_create(const filter_config *cfgs, uint32_t n_filters, uint64_t max_total, void *stream,
                        filter_group_t **out)
{
    if (!cfgs || !out || n_filters == 0) return FILTER_ERR_ARG;
    *out = nullptr;
    const uint32_t kind = cfgs[0].kind;
    if (kind != FILTER_TCF && kind != FILTER_GQF) return FILTER_ERR_ARG;
    filter_group *G = new (std::nothrow) filter_group();
    if (!G) return FILTER_ERR_OOM;
    G->kind = kind;
    G->n = n_filters;
    G->bits = cfgs[0].tag_bits;
    G->max_total = max_total ? max_total : 1;
    uint64_t bytes = 0;
    int rc = kind == FILTER_TCF ? gf::tcf_group_setup(G, cfgs, bytes, true) : gf::gqf_group_setup(G, cfgs, bytes, true);
    if (rc != FILTER_OK) {
        group_free(G);
        return rc;
    }
    G->members = new (std::nothrow) filter[n_filters];
    if (!G->members) {
        group_free(G);
        return FILTER_ERR_OOM;
    }
    const size_t total = bytes + 512 + (64u << 10);
    cudaGetDevice(&G->device);
    if (gf::dev_malloc(reinterpret_cast<void **>(&G->arena.base), total) != cudaSuccess) {
        cudaGetLastError();
        G->arena.base = nullptr;
        group_free(G);
        return FILTER_ERR_OOM;
    }
    G->arena.size = total;
    G->ctr = G->arena.take<gf::DevCounters>(1);
    rc = kind == FILTER_TCF ? gf::tcf_group_setup(G, cfgs, bytes, false) : gf::gqf_group_setup(G, cfgs, bytes, false);
    if (rc == FILTER_OK && G->arena.used > G->arena.size) rc = FILTER_ERR_INTERNAL;
    if (rc == FILTER_OK)
        rc = kind == FILTER_TCF ? gf::tcf_group_clear(G, as_stream(stream)) : gf::gqf_group_clear(G, as_stream(stream));
    if (rc == FILTER_OK && cudaStreamSynchronize(as_stream(stream)) != cudaSuccess) rc = FILTER_ERR_CUDA;
    if (rc != FILTER_OK) {
        group_free(G);
        return rc;
    }
    *out = G;
    return FILTER_OK;
}

int filter_group_destroy(filter_group_t *g)
{
    if (!g) return FILTER_OK;
    int rc = FILTER_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) rc = FILTER_ERR_CUDA;
    group_free(g);
    return rc;
}

int filter_group_clear(filter_group_t *g, void *stream)
{
    if (!valid(g)) return FILTER_ERR_ARG;
    return g->kind == FILTER_TCF ? gf::tcf_group_clear(g, as_stream(stream)) : gf::gqf_group_clear(g, as_stream(stream));
}

static bool keys_ok(const filter_group_t *g, const uint64_t *d_offsets, const uint64_t *d_keys, uint64_t n_total)
{
    return valid(g) && d_offsets && (n_total == 0 || d_keys);
}

int filter_group_insert(filter_group_t *g, const uint64_t *d_offsets, const uint64_t *d_keys, uint64_t n_total,
                        uint8_t *d_status, void *stream)
{
    if (!keys_ok(g, d_offsets, d_keys, n_total) || n_total > g->max_total) return FILTER_ERR_ARG;
    if (g->kind == FILTER_TCF)
        return gf::tcf_group_op(g, gf::GROUP_INSERT, d_offsets, d_keys, n_total, d_status, as_stream(stream));
    return gf::gqf_group_insert(g, d_offsets, d_keys, n_total, d_status, as_stream(stream));
}

int filter_group_remove(filter_group_t *g, const uint64_t *d_offsets, const uint64_t *d_keys, uint64_t n_total,
                        uint8_t *d_status, void *stream)
{
    if (!keys_ok(g, d_offsets, d_keys, n_total) || n_total > g->max_total) return FILTER_ERR_ARG;
    if (g->kind == FILTER_TCF)
        return gf::tcf_group_op(g, gf::GROUP_REMOVE, d_offsets, d_keys, n_total, d_status, as_stream(stream));
    return gf::gqf_group_remove(g, d_offsets, d_keys, n_total, d_status, as_stream(stream));
}

int filter_group_query(filter_group_t *g, const uint64_t *d_offsets, const uint64_t *d_keys, uint64_t n_total,
                       uint8_t *d_found, void *stream)
{
    if (!keys_ok(g, d_offsets, d_keys, n_total) || (n_total && !d_found)) return FILTER_ERR_ARG;
    if (g->kind == FILTER_TCF)
        return gf::tcf_group_op(g, gf::GROUP_QUERY, d_offsets, d_keys, n_total, d_found, as_stream(stream));
    return gf::gqf_group_count(g, d_offsets, d_keys, n_total, nullptr, d_found, as_stream(stream));
}

int filter_group_count(filter_group_t *g, const uint64_t *d_offsets, const uint64_t *d_keys, uint64_t n_total,
                       uint64_t *d_counts, void *stream)
{
    if (!keys_ok(g, d_offsets, d_keys, n_total) || (n_total && !d_counts)) return FILTER_ERR_ARG;
    if (g->kind != FILTER_GQF) return FILTER_ERR_UNSUPPORTED;
    return gf::gqf_group_count(g, d_offsets, d_keys, n_total, d_counts, nullptr, as_stream(stream));
}

int filter_group_get_stats(filter_group_t *g, uint32_t member, void *stream, filter_stats *out)
{
    if (!valid(g) || !out || member >= g->n) return FILTER_ERR_ARG;
    filter &F = g->members[member];
    gf::DevCounters c;
    if (cudaMemcpyAsync(&c, F.ctr, sizeof(c), cudaMemcpyDeviceToHost, as_stream(stream)) != cudaSuccess ||
        cudaStreamSynchronize(as_stream(stream)) != cudaSuccess)
        return FILTER_ERR_CUDA;
    std::memset(out, 0, sizeof(*out));
    out->status_word = c.status;
    out->failed_keys = c.failed;
    out->backing_used = g->kind == FILTER_TCF ? c.backing : 0;
    out->table_bytes = g->kind == FILTER_TCF ? gf::tcf_image_bytes(&F) : gf::gqf_image_bytes(&F);
    out->device_bytes = g->arena.size;
    out->nslots = g->kind == FILTER_TCF ? F.tcf.G.nb * F.tcf.G.B : F.gqf.nslots;
    return FILTER_OK;
}

int filter_group_export_size(filter_group_t *g, uint32_t member, uint64_t *nbytes)
{
    if (!valid(g) || !nbytes || member >= g->n) return FILTER_ERR_ARG;
    filter &F = g->members[member];
    *nbytes = g->kind == FILTER_TCF ? gf::tcf_image_bytes(&F) : gf::gqf_image_bytes(&F);
    return FILTER_OK;
}

int filter_group_export(filter_group_t *g, uint32_t member, void *host_buf, uint64_t nbytes, void *stream)
{
    uint64_t want = 0;
    if (!host_buf || filter_group_export_size(g, member, &want) != FILTER_OK || nbytes != want) return FILTER_ERR_ARG;
    filter &F = g->members[member];
    return g->kind == FILTER_TCF ? gf::tcf_copy_image(&F, host_buf, true, as_stream(stream))
                                 : gf::gqf_copy_image(&F, host_buf, true, as_stream(stream));
}

}  // extern "C"
