// The C ABI of include/gpufilter.h: argument checks, allocation, dispatch.
#include <cstring>
#include <new>

#include "gf_internal.cuh"

namespace gf {
const char *last_cuda_error();
}

static cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

static bool valid(const filter_t *f) { return f != nullptr && f->arena.base != nullptr; }

// every device buffer of the filter got an address
static bool pointers_set(const filter *F)
{
    if (!F->ctr || !F->scan_tmp) return false;
    if (F->cfg.kind == FILTER_TCF) {
        const TcfState &T = F->tcf;
        return T.blocks && T.bk && T.fill && T.cnt && T.off && T.rec && T.pend0 && T.pend1 && T.pend2 && T.tlist &&
               T.tcount && T.dlist && T.seg;
    }
    const GqfState &Q = F->gqf;
    return Q.meta[0] && Q.meta[1] && Q.rem[0] && Q.rem[1] && Q.fp_a && Q.fp_b && Q.fp_c && Q.ufp && Q.idx_a &&
           Q.idx_b && Q.idx_c && Q.ustart && Q.flags && Q.removed && Q.tile_state && Q.tile_lo && Q.radix_tmp;
}

namespace gf {

bool tuning_valid(const filter_tuning &t)
{
    if (t.tcf_path > FILTER_TCF_PATH_TILED) return false;
    if (t.tcf_tile_target && (t.tcf_tile_target < 128 || t.tcf_tile_target > 1024)) return false;
    if (t.gqf_region_groups > 256) return false;
    return true;
}

bool tcf_tiled(const filter_tuning &t, uint64_t nb, uint64_t n)
{
    if (t.tcf_path == FILTER_TCF_PATH_BLOCK) return false;
    if (t.tcf_path == FILTER_TCF_PATH_TILED) return true;
    const uint64_t m = t.tcf_tiled_min_blocks ? t.tcf_tiled_min_blocks : (1ull << 23);
    return nb >= m && n >= m;
}

uint32_t tcf_tile_target(const filter_tuning &t) { return t.tcf_tile_target ? t.tcf_tile_target : 1024u; }
uint64_t gqf_region_groups(const filter_tuning &t) { return t.gqf_region_groups ? t.gqf_region_groups : 8u; }

}  // namespace gf

extern "C" {

int filter_set_tuning(filter_t *f, const filter_tuning *t)
{
    if (!valid(f) || !t || !gf::tuning_valid(*t)) return FILTER_ERR_ARG;
    f->tune = *t;
    return FILTER_OK;
}

int filter_get_tuning(filter_t *f, filter_tuning *out)
{
    if (!valid(f) || !out) return FILTER_ERR_ARG;
    *out = f->tune;
    return FILTER_OK;
}

int filter_gqf_point_update(filter_t *f, const uint64_t *d_keys, uint64_t n, int remove, uint8_t *d_status,
                            void *stream)
{
    if (!valid(f) || n > f->cfg.max_batch || (n && !d_keys) || (remove != 0 && remove != 1)) return FILTER_ERR_ARG;
    if (f->cfg.kind != FILTER_GQF) return FILTER_ERR_UNSUPPORTED;
    if (d_status && n) GF_CUDA(cudaMemsetAsync(d_status, 0, n, as_stream(stream)));
    return gf::gqf_point_update(f, d_keys, n, remove, d_status, as_stream(stream));
}

int filter_create(const filter_config *cfg, void *stream, filter_t **out)
{
    if (!cfg || !out) return FILTER_ERR_ARG;
    *out = nullptr;
    filter *F = new (std::nothrow) filter();
    if (!F) return FILTER_ERR_OOM;
    F->cfg = *cfg;
    if (F->cfg.max_batch == 0) F->cfg.max_batch = 1;
    uint64_t tb = 0, sb = 0;
    int rc;
    if (cfg->kind == FILTER_TCF) rc = gf::tcf_setup(F, tb, sb, true);
    else if (cfg->kind == FILTER_GQF) rc = gf::gqf_setup(F, tb, sb, true);
    else rc = FILTER_ERR_ARG;
    if (rc != FILTER_OK) {
        delete F;
        return rc;
    }
    const size_t total = tb + sb + (64u << 10);
    cudaGetDevice(&F->device);
    if (gf::dev_malloc(reinterpret_cast<void **>(&F->arena.base), total) != cudaSuccess) {
        cudaGetLastError();
        delete F;
        return FILTER_ERR_OOM;
    }
    F->arena.size = total;
    if (gf::dev_malloc(reinterpret_cast<void **>(&F->ctr), sizeof(gf::DevCounters)) != cudaSuccess) {
        cudaGetLastError();
        gf::dev_free(F->arena.base);
        delete F;
        return FILTER_ERR_OOM;
    }
    if (cfg->kind == FILTER_TCF) rc = gf::tcf_setup(F, tb, sb, false);
    else rc = gf::gqf_setup(F, tb, sb, false);
    if (rc == FILTER_OK && F->arena.used > F->arena.size) rc = FILTER_ERR_INTERNAL;
    if (rc == FILTER_OK && !pointers_set(F)) rc = FILTER_ERR_INTERNAL;
    if (rc == FILTER_OK) rc = (cfg->kind == FILTER_TCF) ? gf::tcf_clear(F, as_stream(stream)) : gf::gqf_clear(F, as_stream(stream));
    if (rc != FILTER_OK) {
        gf::dev_free(F->ctr);
        gf::dev_free(F->arena.base);
        delete F;
        return rc;
    }
    *out = F;
    return FILTER_OK;
}

int filter_destroy(filter_t *f)
{
    if (!f) return FILTER_OK;
    int rc = FILTER_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) rc = FILTER_ERR_CUDA;
    gf::dev_free(f->ctr);
    gf::dev_free(f->arena.base);
    f->arena.base = nullptr;
    delete f;
    return rc;
}

int filter_clear(filter_t *f, void *stream)
{
    if (!valid(f)) return FILTER_ERR_ARG;
    return f->cfg.kind == FILTER_TCF ? gf::tcf_clear(f, as_stream(stream)) : gf::gqf_clear(f, as_stream(stream));
}

int filter_insert(filter_t *f, const uint64_t *d_keys, uint64_t n, uint8_t *d_status, void *stream)
{
    if (!valid(f) || n > f->cfg.max_batch || (n && !d_keys)) return FILTER_ERR_ARG;
    return f->cfg.kind == FILTER_TCF ? gf::tcf_insert(f, d_keys, nullptr, n, d_status, as_stream(stream))
                                     : gf::gqf_insert(f, d_keys, nullptr, n, d_status, as_stream(stream));
}

int filter_insert_counts(filter_t *f, const uint64_t *d_keys, const uint32_t *d_counts, uint64_t n,
                         uint8_t *d_status, void *stream)
{
    if (!valid(f) || n > f->cfg.max_batch || (n && (!d_keys || !d_counts))) return FILTER_ERR_ARG;
    if (f->cfg.kind != FILTER_GQF) return FILTER_ERR_UNSUPPORTED;
    return gf::gqf_insert(f, d_keys, d_counts, n, d_status, as_stream(stream));
}

int filter_insert_values(filter_t *f, const uint64_t *d_keys, const uint8_t *d_values, uint64_t n,
                         uint8_t *d_status, void *stream)
{
    if (!valid(f) || n > f->cfg.max_batch || (n && (!d_keys || !d_values))) return FILTER_ERR_ARG;
    if (f->cfg.kind != FILTER_TCF || f->cfg.value_bits == 0) return FILTER_ERR_UNSUPPORTED;
    return gf::tcf_insert(f, d_keys, d_values, n, d_status, as_stream(stream));
}

int filter_query(filter_t *f, const uint64_t *d_keys, uint64_t n, uint8_t *d_found, void *stream)
{
    if (!valid(f) || (n && (!d_keys || !d_found))) return FILTER_ERR_ARG;
    return f->cfg.kind == FILTER_TCF ? gf::tcf_query(f, d_keys, n, d_found, false, as_stream(stream))
                                     : gf::gqf_count(f, d_keys, n, nullptr, d_found, as_stream(stream));
}

int filter_query_values(filter_t *f, const uint64_t *d_keys, uint64_t n, uint8_t *d_values, void *stream)
{
    if (!valid(f) || (n && (!d_keys || !d_values))) return FILTER_ERR_ARG;
    if (f->cfg.kind != FILTER_TCF || f->cfg.value_bits == 0) return FILTER_ERR_UNSUPPORTED;
    return gf::tcf_query(f, d_keys, n, d_values, true, as_stream(stream));
}

int filter_remove(filter_t *f, const uint64_t *d_keys, uint64_t n, uint8_t *d_status, void *stream)
{
    if (!valid(f) || n > f->cfg.max_batch || (n && !d_keys)) return FILTER_ERR_ARG;
    return f->cfg.kind == FILTER_TCF ? gf::tcf_remove(f, d_keys, n, d_status, as_stream(stream))
                                     : gf::gqf_remove(f, d_keys, n, d_status, as_stream(stream));
}

int filter_count(filter_t *f, const uint64_t *d_keys, uint64_t n, uint64_t *d_counts, void *stream)
{
    if (!valid(f) || (n && (!d_keys || !d_counts))) return FILTER_ERR_ARG;
    if (f->cfg.kind != FILTER_GQF) return FILTER_ERR_UNSUPPORTED;
    return gf::gqf_count(f, d_keys, n, d_counts, nullptr, as_stream(stream));
}

int filter_get_stats(filter_t *f, void *stream, filter_stats *out)
{
    if (!valid(f) || !out) return FILTER_ERR_ARG;
    gf::DevCounters c;
    if (cudaMemcpyAsync(&c, f->ctr, sizeof(c), cudaMemcpyDeviceToHost, as_stream(stream)) != cudaSuccess ||
        cudaStreamSynchronize(as_stream(stream)) != cudaSuccess)
        return FILTER_ERR_CUDA;
    std::memset(out, 0, sizeof(*out));
    out->status_word = c.status;
    out->failed_keys = c.failed;
    out->backing_used = f->cfg.kind == FILTER_TCF ? c.backing : 0;
    out->table_bytes = f->cfg.kind == FILTER_TCF ? gf::tcf_image_bytes(f) : gf::gqf_image_bytes(f);
    out->device_bytes = f->arena.size + sizeof(gf::DevCounters);
    out->nslots = f->cfg.kind == FILTER_TCF ? f->tcf.G.nb * f->tcf.G.B : f->gqf.nslots;
    return FILTER_OK;
}

int filter_get_device_view(filter_t *f, filter_device_view *out)
{
    if (!valid(f) || !out) return FILTER_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    static_assert(offsetof(gf::DevCounters, status) == 0 && offsetof(gf::DevCounters, failed) == 8 &&
                      offsetof(gf::DevCounters, backing) == 16,
                  "the device view exposes the first three counters");
    if (f->cfg.kind == FILTER_TCF && gf::tcf_custom(f->tcf.G)) return FILTER_ERR_UNSUPPORTED;  // 32-byte blocks only
    out->kind = f->cfg.kind;
    out->tag_bits = f->cfg.tag_bits;
    out->seed = f->cfg.hash_seed;
    out->counters = &f->ctr->status;
    if (f->cfg.kind == FILTER_TCF) {
        const TcfState &T = f->tcf;
        out->mode = T.mode;
        out->value_bits = T.G.vbits;
        out->table = T.blocks;
        out->aux = T.bk;
        out->n_blocks = T.G.nb;
        out->n_aux = T.G.nbk;
    } else {
        const GqfState &Q = f->gqf;
        out->q = Q.q;
        out->table = Q.meta[Q.cur];
        out->aux = Q.rem[Q.cur];
        out->n_blocks = Q.nblk;
        out->n_aux = Q.nslots;
        out->locks = Q.locks;
    }
    return FILTER_OK;
}

int filter_gqf_enumerate(filter_t *f, uint64_t *d_fingerprints, uint64_t *d_counts, uint64_t cap,
                         uint64_t *n_groups, void *stream)
{
    if (!valid(f) || !n_groups || f->cfg.kind != FILTER_GQF || (cap && (!d_fingerprints || !d_counts)))
        return FILTER_ERR_ARG;
    return gf::gqf_enumerate(f, d_fingerprints, d_counts, cap, n_groups, as_stream(stream));
}

int filter_gqf_keys_of(filter_t *f, const uint64_t *d_fingerprints, uint64_t n, uint64_t *d_keys, void *stream)
{
    if (!valid(f) || f->cfg.kind != FILTER_GQF || (n && (!d_fingerprints || !d_keys))) return FILTER_ERR_ARG;
    return gf::gqf_unhash(f, d_fingerprints, n, d_keys, as_stream(stream));
}

int filter_export_size(filter_t *f, uint64_t *nbytes)
{
    if (!valid(f) || !nbytes) return FILTER_ERR_ARG;
    *nbytes = f->cfg.kind == FILTER_TCF ? gf::tcf_image_bytes(f) : gf::gqf_image_bytes(f);
    return FILTER_OK;
}

int filter_export(filter_t *f, void *host_buf, uint64_t nbytes, void *stream)
{
    uint64_t want = 0;
    if (!valid(f) || !host_buf || filter_export_size(f, &want) != FILTER_OK || nbytes != want) return FILTER_ERR_ARG;
    return f->cfg.kind == FILTER_TCF ? gf::tcf_copy_image(f, host_buf, true, as_stream(stream))
                                     : gf::gqf_copy_image(f, host_buf, true, as_stream(stream));
}

int filter_import(filter_t *f, const void *host_buf, uint64_t nbytes, void *stream)
{
    uint64_t want = 0;
    if (!valid(f) || !host_buf || filter_export_size(f, &want) != FILTER_OK || nbytes != want) return FILTER_ERR_ARG;
    void *h = const_cast<void *>(host_buf);
    return f->cfg.kind == FILTER_TCF ? gf::tcf_copy_image(f, h, false, as_stream(stream))
                                     : gf::gqf_copy_image(f, h, false, as_stream(stream));
}

const char *filter_error_string(int code)
{
    switch (code) {
    case FILTER_OK: return "ok";
    case FILTER_ERR_ARG: return "invalid argument";
    case FILTER_ERR_OOM: return "device allocation failed";
    case FILTER_ERR_UNSUPPORTED: return "operation not supported by this filter kind";
    case FILTER_ERR_FULL: return "filter full";
    case FILTER_ERR_TIMEOUT: return "bounded device wait gave up";
    case FILTER_ERR_CUDA: return gf::last_cuda_error();
    case FILTER_ERR_INTERNAL: return "internal consistency check failed";
    default: return "unknown error";
    }
}

int filter_debug_fail_alloc(uint32_t nth)
{
    gf::fail_allocation(nth);
    return FILTER_OK;
}

int filter_debug_live_allocations(uint64_t *n)
{
    if (!n) return FILTER_ERR_ARG;
    const long long v = gf::live_allocations();
    *n = v > 0 ? (uint64_t)v : 0;
    return FILTER_OK;
}

int filter_debug_wait_timeout(filter_t *f, uint32_t spin_limit, void *stream)
{
    if (!valid(f) || spin_limit == 0) return FILTER_ERR_ARG;
    gf::debug_wait_timeout(f->scan_tmp, f->ctr, spin_limit, as_stream(stream));
    GF_CUDA(cudaGetLastError());
    return FILTER_OK;
}

}  // extern "C"
