/*
 * gpufilter: GPU two-choice filter (TCF) and counting quotient filter (GQF)
 * for NVIDIA GB300 (sm_103a), after "High-Performance Filters for GPUs"
 * (Pandey et al., arXiv 2212.09005).
 *
 * C ABI. Every pointer argument named d_* is a device pointer; host_* is host
 * memory. Streams are cudaStream_t values passed as void* (NULL = the legacy
 * default stream). All calls except filter_create, filter_destroy,
 * filter_get_stats, filter_export, filter_import and filter_gqf_enumerate
 * are asynchronous (filter_get_device_view does not touch the device): they
 * enqueue kernels on the stream and return; the caller's buffers must stay
 * valid until the stream reaches the call. Exceptions: GQF inserts and
 * removes synchronise the stream to read the number of distinct fingerprints
 * (which picks the in-place or the merge path) and, after a merge, whether
 * the table overflowed. Calls on one filter must be ordered (same stream, or
 * externally synchronised); different filters are independent.
 *
 * Errors are returned synchronously for bad arguments, allocation failure
 * and unsupported operations. Conditions found on the device (a full table,
 * a bounded wait that gave up) are recorded in a sticky status word read by
 * filter_get_stats, and per key in the optional status arrays.
 *
 * Fingerprints and layouts
 *   TCF (paper Sec. 4): h = mix64(key ^ seed), block b1 = h mod nb, tag =
 *   bits 44.. of h (f bits, 0 and 1 moved to 2 and 3), b2 = b1 xor g(tag).
 *   nb = 2^log2_slots / B blocks of 32 bytes (B = 256 / f tags; other block
 *   geometries: see filter_config.block_slots). Backing
 *   table: nbk buckets of 8 uint64 entries (min(b1,b2) << f | tag), nbk =
 *   max(8, ceil(ceil(N/100) / 8)) (Sec. 4.1, "backing table"). With
 *   value_bits v > 0 the tag is f - v bits wide and each slot holds
 *   tag << v | value; g and the bucket (hashed with the value bits cleared)
 *   depend on the tag alone.
 *   GQF (paper Sec. 5): p = q + r, fp = mix_p(fold_p(key) ^ seed mod 2^p),
 *   quotient = fp >> r, remainder = fp mod 2^r. N = 2^q home slots plus a
 *   tail of S = max(64, min(N, roundup64(1072 q))) slots. Per 64-slot block a
 *   32-byte metadata record {occupieds u64, runends u64, offset u32, 12 zero
 *   bytes}; remainders r/8 bytes each. Counts use the encoding
 *   [v] (count 1) or [v, v, n, n base-2^r digits of count - 2].
 */
#ifndef GPUFILTER_H
#define GPUFILTER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define FILTER_OK 0
#define FILTER_ERR_ARG 1          /* null pointer, bad geometry, n > max_batch */
#define FILTER_ERR_OOM 2          /* device allocation failed */
#define FILTER_ERR_UNSUPPORTED 3  /* operation not defined for this filter kind */
#define FILTER_ERR_FULL 4         /* (status word bit) some key did not fit */
#define FILTER_ERR_TIMEOUT 5      /* (status word bit) a bounded device wait gave up */
#define FILTER_ERR_CUDA 6         /* a CUDA runtime call failed */
#define FILTER_ERR_INTERNAL 7     /* (status word bit) a device consistency check failed */

/* ---- per-key status values written to d_status ---- */
#define FILTER_KEY_OK 0
#define FILTER_KEY_FULL 1      /* insert: no room (TCF blocks + backing full, GQF past the tail) */
#define FILTER_KEY_NOT_FOUND 2 /* remove: no stored copy left to remove */

/* ---- filter kinds and TCF modes ---- */
#define FILTER_TCF 1
#define FILTER_GQF 2
#define FILTER_MODE_BULK 0  /* TCF: sorted blocks, deterministic phased bulk insert */
#define FILTER_MODE_POINT 1 /* TCF: unsorted blocks, one atomic CAS per key (Alg. 1) */

typedef struct filter filter_t;

typedef struct filter_config {
    uint32_t kind;        /* FILTER_TCF or FILTER_GQF */
    uint32_t log2_slots;  /* TCF: log2 of total tag slots; GQF: q */
    uint32_t tag_bits;    /* TCF: slot bits f in {8, 12, 16} (tag + value; 12 only with
                             block_slots geometry, see below); GQF: r in {8, 16} */
    uint32_t mode;        /* TCF: FILTER_MODE_BULK or FILTER_MODE_POINT; GQF: 0 */
    uint64_t hash_seed;   /* xor-ed into keys before hashing */
    uint64_t max_batch;   /* largest n of one call; sizes the scratch memory (GQF: < 2^30) */
    uint32_t value_bits;  /* TCF: v bits of each slot hold a value below an (f - v)-bit tag,
                             0 <= v <= min(f / 2, 7); 0 = no values. GQF, groups: 0 */
    uint32_t block_slots; /* TCF: slots per block B; 0 = 256 / f (one 32-byte sector, 21 for
                             f = 12). Other block sizes (paper Sec. 4.1 blocks up to and past a
                             cache line, Sec. 4.2 128-slot bulk blocks): (f, B) in (16, 8),
                             (16, 32), (16, 64), (16, 128), (12, 21), (8, 64), bulk mode only,
                             no values, not in groups or the device view. The B slots of a
                             block are packed little-endian (slot s at bit f s) into the
                             smallest whole number of 32-byte sectors; the filter has nb
                             blocks, nb the largest power of two with nb B <= 2^log2_slots.
                             GQF: 0 */
} filter_config;

typedef struct filter_stats {
    uint64_t status_word;   /* sticky OR of (1 << FILTER_ERR_*) seen on the device */
    uint64_t failed_keys;   /* keys that got FILTER_KEY_FULL since creation */
    uint64_t backing_used;  /* TCF: entries in the backing table; GQF: 0 */
    uint64_t table_bytes;   /* bytes of the exported table image */
    uint64_t device_bytes;  /* table + scratch held on the device */
    uint64_t nslots;        /* TCF: tag slots; GQF: home + tail slots */
} filter_stats;

/*
 * filter_create: validate *cfg, allocate the table and the scratch for
 * batches of up to cfg->max_batch keys on the current device, and clear the
 * table on `stream`. The filter owns this memory until filter_destroy.
 * Returns FILTER_ERR_ARG for a bad geometry (TCF: f in {8,16}, or f = 12 and
 * the other (f, block_slots) pairs listed at filter_config in bulk mode
 * without values; 2^log2_slots >= 2 blocks, nb <= 2^32, value_bits <=
 * min(f / 2, 7); GQF: r in {8,16}, 6 <= q <= 36, q + r <= 64, value_bits and
 * block_slots 0),
 * FILTER_ERR_OOM if an allocation fails (nothing is leaked).
 */
int filter_create(const filter_config *cfg, void *stream, filter_t **out);

/* filter_destroy: synchronise the device and free everything. NULL is a no-op. */
int filter_destroy(filter_t *f);

/*
 * ---- tuning ----
 * Knobs of the bulk paths that change only the time taken: tables, answers
 * and statuses are the same under every setting (the GPU tests check both TCF
 * paths and the GQF in-place and merge paths against the same oracle).
 *   tcf_path: how a TCF bulk insert or remove groups its candidates by block.
 *     FILTER_TCF_PATH_BLOCK: a counting sort by block (a counter and an offset
 *     per block, an 8-byte record per key, scattered); fastest while that
 *     scratch stays in the L2. FILTER_TCF_PATH_TILED: a partition by tile of
 *     consecutive blocks in coalesced passes, then a shared-memory sort per
 *     tile; fastest for large tables and batches. FILTER_TCF_PATH_AUTO takes
 *     TILED when the table has at least tcf_tiled_min_blocks blocks and the
 *     batch at least as many keys (0: 2^23).
 *   tcf_tile_target: tiled path, the expected candidates per tile, 128 ..
 *     1024 (0: 1024).
 *   gqf_region_groups: GQF batches with at most this many distinct
 *     fingerprints per 256 quotients on average are inserted or removed in
 *     place (even-odd regions); denser ones take the merge (0: 8).
 * filter_set_tuning / filter_group_set_tuning: FILTER_ERR_ARG for values out
 * of range. filter_get_tuning: the current settings (0 fields = defaults).
 */
#define FILTER_TCF_PATH_AUTO 0
#define FILTER_TCF_PATH_BLOCK 1
#define FILTER_TCF_PATH_TILED 2

typedef struct filter_tuning {
    uint32_t tcf_path;
    uint32_t tcf_tile_target;
    uint32_t gqf_region_groups;
    uint32_t reserved;
    uint64_t tcf_tiled_min_blocks;
} filter_tuning;

/* filter_clear: empty the table (asynchronous) and reset the statistics. */
int filter_clear(filter_t *f, void *stream);

int filter_set_tuning(filter_t *f, const filter_tuning *t);
int filter_get_tuning(filter_t *f, filter_tuning *out);

/*
 * filter_insert: insert n keys (a multiset: duplicates are counted, Sec. 5 of
 * the paper, and stored as repeated tags by the TCF).
 *  TCF bulk mode: the phased deterministic batch insert (Sec. 4.1 shortcut,
 *  Sec. 4 two choices, Sec. 4.1 backing table, Sec. 4.2 sorted blocks).
 *  TCF point mode: each key independently, Alg. 1 (CAS into an empty slot).
 *  GQF: sort, reduce to <fingerprint, count> (Sec. 5.4), merge the groups
 *  into the runs (Sec. 5.3). If the table cannot hold every group, the
 *  longest prefix of the sorted groups that fits is kept.
 * d_keys: n uint64. d_status: NULL or n uint8 (FILTER_KEY_*). n <= max_batch.
 */
int filter_insert(filter_t *f, const uint64_t *d_keys, uint64_t n, uint8_t *d_status,
                  void *stream);

/*
 * filter_insert_values: as filter_insert, with a small value per key (the
 * paper's TCF associates small values with items, Sec. 1 and Sec. 4). TCF
 * with value_bits v > 0 only: a slot holds the key's (f - v)-bit tag and the
 * low v bits of d_values[i] below it. The value never changes where a key
 * goes: blocks, buckets and statuses are those filter_insert gives, and
 * copies of one tag are kept sorted by value. filter_insert on such a filter
 * stores value 0. d_values: n uint8. Returns FILTER_ERR_UNSUPPORTED for a
 * GQF or a TCF without values.
 */
int filter_insert_values(filter_t *f, const uint64_t *d_keys, const uint8_t *d_values, uint64_t n,
                         uint8_t *d_status, void *stream);

/*
 * filter_insert_counts: GQF only. Key i counts as d_counts[i] copies: its
 * fingerprint's count grows by that much, in the same single pass (sort,
 * reduce with the counts summed per fingerprint, merge). This is how the GQF
 * associates values with items: through its counters, as the counting
 * quotient filter it follows does (Sec. 2 of the paper); filter_count reads
 * them back. Statuses and the kept prefix on overflow are those of
 * filter_insert. Every count must be >= 1 and their sum below 2^32, else
 * FILTER_ERR_ARG and the table is unchanged (checked on the device; the call
 * synchronises `stream`). d_counts: n uint32. n <= max_batch. Returns
 * FILTER_ERR_UNSUPPORTED for a TCF.
 */
int filter_insert_counts(filter_t *f, const uint64_t *d_keys, const uint32_t *d_counts, uint64_t n,
                         uint8_t *d_status, void *stream);

/*
 * filter_query: d_found[i] = 1 if key i may be in the set (no false
 * negatives; false positives at the filter's rate), else 0.
 * TCF: tag in block b1 or b2 or the backing bucket. GQF: count > 0.
 * Any n (not limited by max_batch).
 */
int filter_query(filter_t *f, const uint64_t *d_keys, uint64_t n, uint8_t *d_found,
                 void *stream);

/*
 * filter_query_values: TCF with values only. d_values[i] = the smallest value
 * stored with key i's fingerprint (its tag in block b1 or b2, or its entry in
 * the backing bucket), or 0xFF when the fingerprint is absent; so
 * d_values[i] != 0xFF exactly when filter_query answers 1. Matching ignores
 * the value bits, and filter_remove deletes, per key, the copy with the
 * smallest value in the first of b1, b2 and the bucket that holds one.
 * Any n. Returns FILTER_ERR_UNSUPPORTED for a GQF or a TCF without values.
 */
int filter_query_values(filter_t *f, const uint64_t *d_keys, uint64_t n, uint8_t *d_values,
                        void *stream);

/*
 * filter_remove: delete one copy per key (Sec. 6.4 of the paper). Keys without a
 * stored copy get FILTER_KEY_NOT_FOUND (for the TCF, deleting a key that was
 * never inserted may remove another key's aliasing fingerprint, as in every
 * fingerprint filter). n <= max_batch.
 */
int filter_remove(filter_t *f, const uint64_t *d_keys, uint64_t n, uint8_t *d_status,
                  void *stream);

/*
 * filter_count: GQF only. d_counts[i] = stored count of key i's fingerprint
 * (never below the true count; exact when the fingerprint is injective on the
 * key universe). TCF returns FILTER_ERR_UNSUPPORTED. Any n.
 */
int filter_count(filter_t *f, const uint64_t *d_keys, uint64_t n, uint64_t *d_counts,
                 void *stream);

/* filter_get_stats: synchronise `stream`, then read the status word and counters. */
int filter_get_stats(filter_t *f, void *stream, filter_stats *out);

/*
 * filter_get_device_view: describe the filter's current table for the
 * device-side point queries of include/gpufilter_device.cuh (a caller's own
 * kernels call gf_device_tcf_contains / gf_device_gqf_count with the view
 * passed by value). The view holds device pointers owned by the filter and is
 * valid until the next insert, remove, clear or import on it; a GQF update
 * switches table buffers, so take the view again after one. Host only, does
 * not touch the device. Group members are not covered. A point-mode TCF can
 * also be updated from a caller's kernel (gf_device_tcf_insert / _remove),
 * and a GQF likewise (gf_device_gqf_insert / _remove, the locked point GQF
 * of Sec. 5.2: they update the current buffer in place, so the view stays
 * valid); those updates and the library's own calls on the filter must not
 * overlap, and GQF point updates must not overlap GQF counts of the filter.
 */
typedef struct filter_device_view {
    uint32_t kind;       /* FILTER_TCF or FILTER_GQF */
    uint32_t tag_bits;   /* TCF: slot bits f (tag + value); GQF: remainder bits r */
    uint32_t q;          /* GQF: quotient bits; TCF: 0 */
    uint32_t mode;       /* TCF: FILTER_MODE_BULK or FILTER_MODE_POINT; GQF: 0 */
    uint64_t seed;       /* the filter's hash seed (filter_config.hash_seed) */
    void *table;         /* TCF: nb blocks of 32 bytes; GQF: the 32-byte metadata records */
    void *aux;           /* TCF: the backing buckets (8 uint64 each); GQF: the remainders */
    uint64_t n_blocks;   /* TCF: nb (a power of two); GQF: metadata records */
    uint64_t n_aux;      /* TCF: backing buckets; GQF: slots */
    unsigned long long *counters;  /* the filter's device counters: [0] status word,
                                      [1] failed keys, [2] TCF backing entries */
    uint32_t value_bits; /* TCF: value bits below the tag in each slot; GQF: 0 */
    uint32_t reserved;
    uint32_t *locks;     /* GQF: the point-update locks, one 32-bit word per 8192 quotients,
                            32 words apart (gf_device_gqf_insert / _remove); TCF: NULL */
} filter_device_view;

int filter_get_device_view(filter_t *f, filter_device_view *out);

/*
 * filter_gqf_enumerate: the GQF's distinct fingerprints and their counts, in
 * ascending fingerprint order (the table is walked run by run, as counts read
 * it). *n_groups (host) receives the number of groups; the first min(cap,
 * *n_groups) are written to d_fingerprints / d_counts (device, cap entries
 * each). cap = 0 only counts. Synchronises `stream` once; takes (and returns)
 * (64-slot blocks + 1) x 4 bytes plus scan scratch of stream-ordered device
 * memory for the call. FILTER_ERR_ARG for a TCF.
 *
 * filter_gqf_keys_of: the keys whose fingerprints these are, by inverting the
 * fingerprint hash (Sec. 5.1: it is a bijection on p = q + r bits). Exact for
 * keys below 2^p; larger keys were folded to p bits first and come back as
 * that fold. With filter_gqf_enumerate this lists a GQF's contents, e.g. to
 * re-insert them into a larger filter (resize).
 */
int filter_gqf_enumerate(filter_t *f, uint64_t *d_fingerprints, uint64_t *d_counts, uint64_t cap,
                         uint64_t *n_groups, void *stream);
int filter_gqf_keys_of(filter_t *f, const uint64_t *d_fingerprints, uint64_t n, uint64_t *d_keys, void *stream);

/*
 * filter_gqf_point_update: GQF point inserts (remove = 0) or removes
 * (remove = 1) of n keys, one thread per key, in place on the current table
 * (paper Sec. 5.2, the point insertion API: locks on regions of 8192
 * quotients, the key's region and the next, taken in order with bounded
 * waits). The keys of one call are applied in no particular order; the table
 * is a function of the stored multiset, so it equals the table a bulk call
 * would leave. Asynchronous, no host synchronisation (graph-capturable), no
 * scratch. d_status (optional, n bytes): FILTER_KEY_OK, FILTER_KEY_FULL (the
 * shift would leave the two lock regions or the table; nothing changed;
 * counted), FILTER_KEY_NOT_FOUND (remove), or 3 (a lock wait gave up, or the
 * key's cluster is longer than the locked span; nothing changed; the status
 * word records FILTER_ERR_TIMEOUT). Meant for tables whose home slots are at
 * most about 95 % used, where clusters stay far shorter than a lock region.
 * FILTER_ERR_ARG for n > max_batch; FILTER_ERR_UNSUPPORTED for a TCF.
 */
int filter_gqf_point_update(filter_t *f, const uint64_t *d_keys, uint64_t n, int remove, uint8_t *d_status,
                            void *stream);

/* filter_export_size: bytes of the table image (see the layout above). */
int filter_export_size(filter_t *f, uint64_t *nbytes);

/*
 * filter_export: synchronise `stream` and copy the table image to host_buf
 * (nbytes must equal filter_export_size). TCF image: the blocks, then the
 * backing buckets. GQF image: all metadata records, then all remainders.
 * Used for parity checks and as a checkpoint.
 */
int filter_export(filter_t *f, void *host_buf, uint64_t nbytes, void *stream);

/* filter_import: load an image produced by filter_export of the same geometry. */
int filter_import(filter_t *f, const void *host_buf, uint64_t nbytes, void *stream);

/* filter_error_string: static text for a FILTER_* return code. */
const char *filter_error_string(int code);

/*
 * Kernel tracing (process-wide, off by default). While on, every kernel the
 * library launches is bracketed by two CUDA events on its stream and recorded
 * with its name and its work units (keys, slots or blocks, per kernel; the
 * sparse TCF phases count theirs on the device, in a 512 KB buffer that the
 * first filter_trace_enable(1) allocates).
 * filter_trace_summary synchronises the recorded events and returns, per
 * kernel name, the launch count, the summed units and the summed device time
 * in milliseconds. Enabling costs two event records per launch.
 * filter_trace_enable returns FILTER_ERR_OOM if that buffer cannot be allocated.
 */
typedef struct filter_trace_entry {
    char name[48];
    uint64_t launches;
    uint64_t units;
    double ms;
} filter_trace_entry;

int filter_trace_enable(int on);
int filter_trace_reset(void);
/* writes min(cap, number of kernels) entries to out; *n_kernels = number of kernels */
int filter_trace_summary(uint32_t cap, filter_trace_entry *out, uint32_t *n_kernels);

/*
 * filter_calibrate_gather: a measurement utility, not a filter operation.
 * For each of n keys, reads the key, `sectors_per_key` pseudo-random 32-byte
 * sectors of the table d_table (table_bytes bytes, 16-byte aligned, at most
 * 2^32 sectors; sector choice from mix64 of the key) and writes one byte to
 * d_out[i]: the memory pattern of a filter query without the filter
 * arithmetic. Timing it gives the random-access throughput the query kernels
 * are compared with at the same table footprint. Asynchronous on `stream`;
 * FILTER_ERR_ARG for null or misaligned pointers or an empty table.
 */
int filter_calibrate_gather(const void *d_table, uint64_t table_bytes, const uint64_t *d_keys, uint64_t n,
                            uint32_t sectors_per_key, uint8_t *d_out, void *stream);

/*
 * ---- failure-detection self-tests ----
 * These exist so that the failure paths can be exercised without a real
 * device fault (the paper has no counterpart).
 *
 * filter_debug_fail_alloc: make the nth device allocation the library
 *   attempts from now on (filter_create, filter_group_create,
 *   filter_server_create, filter_trace_enable, filter_gqf_enumerate) fail as
 *   if the device were full; nth = 0 cancels. The call then returns
 *   FILTER_ERR_OOM and frees what it had allocated. Process-wide.
 * filter_debug_live_allocations: *n = device allocations the library holds
 *   now (to check that a failed call leaked nothing).
 * filter_debug_wait_timeout: run, on `stream`, the library's bounded
 *   look-back wait (the one its scans and run-length encoding use) against a
 *   predecessor that never publishes, giving up after spin_limit loads. The
 *   wait records FILTER_ERR_TIMEOUT in f's sticky status word, which
 *   filter_get_stats then reports; the filter's table is not touched and the
 *   filter stays usable. FILTER_ERR_ARG for spin_limit 0.
 */
int filter_debug_fail_alloc(uint32_t nth);
int filter_debug_live_allocations(uint64_t *n);
int filter_debug_wait_timeout(filter_t *f, uint32_t spin_limit, void *stream);

/*
 * filter_gqf_insert_noalloc: a GQF bulk insert (the same work as
 * filter_insert on a GQF) that allocates no device memory at all. The paper
 * has no counterpart; this exists for callers that must not call cudaMalloc:
 * a process whose device memory is owned by its own allocator or by a fixed
 * arena reserved at start-up, where a cudaMalloc could fail on a full device
 * or fragment the arena, and latency-critical paths that cannot afford
 * cudaMalloc's implicit device synchronisation.
 *
 * d_table_in: the current table image of a GQF with this (q, r, hash_seed),
 *   in device memory, in the filter_export layout (all metadata records, then
 *   all remainders; filter_export_size bytes; an all-zero image is the empty
 *   table). d_table_out: receives the table after the insert, same size; it
 *   must not overlap d_table_in. d_keys: n uint64 keys. d_status: NULL or n
 *   uint8 per-key statuses, as for filter_insert. All device pointers are
 *   owned by the caller.
 * Limits: n <= FILTER_NOALLOC_MAX_KEYS, 6 <= q <= FILTER_NOALLOC_MAX_Q,
 *   r in {8, 16}; otherwise FILTER_ERR_ARG and nothing is enqueued.
 * Scratch: a static device array of 4 MiB inside the library, which every GPU
 *   that loads the library keeps until the process exits. All calls share it
 *   and it keeps the last call's contents (the call clears what it needs
 *   cleared), so calls whose GPU work overlaps - on different streams, or from
 *   several host threads - race on it and must be serialised by the caller.
 *   The first call on each device looks the array's device address up with
 *   cudaGetSymbolAddress, with that device current, and keeps it for the
 *   life of the process; a cudaDeviceReset invalidates it, so the call must
 *   not be used after one.
 * Synchronisation: like a GQF filter_insert, a call with n > 0 synchronises
 *   `stream` to read the number of distinct fingerprints in the batch and,
 *   after the merge, whether the table overflowed (an overflowing batch
 *   synchronises a few times more while it finds the prefix that fits). The
 *   GPU work is enqueued on `stream`; d_table_in is only read.
 */
#define FILTER_NOALLOC_MAX_KEYS 65536u
#define FILTER_NOALLOC_MAX_Q 20u
int filter_gqf_insert_noalloc(uint32_t q, uint32_t r, uint64_t hash_seed, const void *d_table_in,
                              void *d_table_out, const uint64_t *d_keys, uint64_t n,
                              uint8_t *d_status, void *stream);

/*
 * ---- filter groups ----
 * Many filters of one kind driven by one set of kernel launches per call: the
 * number of launches of a group call does not grow with the number of
 * members. The paper measures one filter per launch; groups serve workloads
 * with thousands of small filters (one per user, shard or sample), where
 * per-filter launches would be latency-bound. Each member's table is laid out
 * and behaves exactly as a standalone filter with the same configuration that
 * receives the same calls with its keys in the same order; its exported image
 * is byte-identical to that filter's.
 *
 * filter_group_create: cfgs[0 .. n_filters) configure the members. All share
 *   kind and tag_bits (TCF f / GQF r); TCF members use FILTER_MODE_BULK; each
 *   has its own log2_slots and hash_seed (cfgs[i].max_batch is ignored).
 *   max_total: the largest total key count of one insert or remove call (TCF
 *   < 2^32, GQF < 2^30). One device allocation holds every member's table and
 *   the shared scratch; the group owns it until filter_group_destroy.
 *   Returns FILTER_ERR_ARG for mixed kinds or tag widths, point mode, a bad
 *   member geometry (as filter_create), more than 2^32 TCF blocks in total, or
 *   GQF member index bits + the largest q + r above 64; FILTER_ERR_OOM if the
 *   allocation fails. Synchronises `stream`.
 */
typedef struct filter_group filter_group_t;

int filter_group_create(const filter_config *cfgs, uint32_t n_filters, uint64_t max_total, void *stream,
                        filter_group_t **out);

/* filter_group_destroy: synchronise the device and free everything. NULL is a no-op. */
int filter_group_destroy(filter_group_t *g);

/* filter_group_set_tuning: the tuning of every member's calls (see filter_set_tuning). */
int filter_group_set_tuning(filter_group_t *g, const filter_tuning *t);

/* filter_group_clear: empty every member (asynchronous) and reset the statistics. */
int filter_group_clear(filter_group_t *g, void *stream);

/*
 * Keys of a group call: member i's keys are d_keys[d_offsets[i] ..
 * d_offsets[i + 1]), in the order the member sees them. d_offsets: device
 * array of n_filters + 1 non-decreasing uint64 with d_offsets[0] = 0 and
 * d_offsets[n_filters] = n_total; n_total is passed by value so that launch
 * sizes are known without reading the device. Keys at or past n_total are
 * never read. Per-key outputs (d_status, d_found, d_counts) are indexed like
 * d_keys. Semantics per member are those of filter_insert, filter_remove,
 * filter_query and filter_count.
 *
 * filter_group_insert / filter_group_remove: n_total <= max_total, else
 *   FILTER_ERR_ARG. GQF inserts synchronise the stream once (overflow check);
 *   a member whose keys do not fit is redone alone from its previous table,
 *   keeping the longest prefix of its sorted groups that fits (as
 *   filter_insert), with extra synchronisations. GQF removes always take the
 *   merge path. All other group calls are asynchronous.
 * filter_group_query: any n_total.
 * filter_group_count: GQF groups only (TCF: FILTER_ERR_UNSUPPORTED); any n_total.
 */
int filter_group_insert(filter_group_t *g, const uint64_t *d_offsets, const uint64_t *d_keys, uint64_t n_total,
                        uint8_t *d_status, void *stream);
int filter_group_remove(filter_group_t *g, const uint64_t *d_offsets, const uint64_t *d_keys, uint64_t n_total,
                        uint8_t *d_status, void *stream);
int filter_group_query(filter_group_t *g, const uint64_t *d_offsets, const uint64_t *d_keys, uint64_t n_total,
                       uint8_t *d_found, void *stream);
int filter_group_count(filter_group_t *g, const uint64_t *d_offsets, const uint64_t *d_keys, uint64_t n_total,
                       uint64_t *d_counts, void *stream);

/*
 * filter_group_get_stats: synchronise `stream` and read member `member`'s
 * statistics. GQF members keep their own status word and failed-key count;
 * in a TCF group these counters, and backing_used, are shared by all members.
 * table_bytes and nslots are the member's; device_bytes is the whole group's.
 */
int filter_group_get_stats(filter_group_t *g, uint32_t member, void *stream, filter_stats *out);

/* filter_group_export_size / filter_group_export: member `member`'s table
 * image, in the filter_export layout of a standalone filter (synchronises). */
int filter_group_export_size(filter_group_t *g, uint32_t member, uint64_t *nbytes);
int filter_group_export(filter_group_t *g, uint32_t member, void *host_buf, uint64_t nbytes, void *stream);

/*
 * ---- batched work list ----
 * One call applies a list of work items to a TCF group and a GQF group (the
 * paper's batched bulk calls, Sec. 4.2 and Sec. 5.3, over thousands of
 * filters at once). Each item is (group, member, operation, device keys,
 * device results). The list itself is host memory, read during the call, so
 * that every launch is sized when it is enqueued; the call never
 * synchronises the host, so a sequence of calls on one stream can be captured
 * in one CUDA graph and replayed (the data in the items' buffers may change
 * between replays, the list may not).
 *
 * filter_batch_create: a batch context over `tcf` (a TCF group, or NULL) and
 *   `gqf` (a GQF group, or NULL), for calls of at most max_items items and at
 *   most max_keys keys per (group, operation) class. It allocates max_keys x
 *   16 bytes of device scratch and one device descriptor buffer (about
 *   40 bytes per item plus 8 per member and class). The groups stay owned by
 *   the caller and must outlive the batch.
 * filter_batch_run: per group, all inserts run first, then removes, then
 *   queries, then counts (GQF only); within one class, member m's items are
 *   concatenated in list order and applied as one batch (one group call for
 *   all members). d_out receives n uint8 statuses (insert, remove) or found
 *   flags (query), or n uint64 counts (count); NULL discards them. Inserts
 *   into a GQF member that do not fit leave that member's table unchanged and
 *   report FILTER_KEY_FULL for all of its keys in the call (unlike
 *   filter_group_insert, which keeps the longest prefix that fits and needs
 *   host round trips). A call's descriptors travel by value in the
 *   parameters of its own upload launches, so the list may be reused or
 *   freed as soon as the call returns, and direct calls and replays of
 *   captured graphs may be mixed freely; they share the batch's scratch, so
 *   they must run in order (one stream, or streams the caller orders).
 *   FILTER_ERR_ARG for a bad group, member or op, n_items >
 *   max_items, or a class above max_keys (inserts and removes also above the
 *   group's max_total); FILTER_ERR_UNSUPPORTED for a count on the TCF group.
 *   Nothing is enqueued when an item is rejected.
 */
typedef struct filter_batch filter_batch_t;

#define FILTER_BATCH_TCF 0
#define FILTER_BATCH_GQF 1

typedef struct filter_work {
    uint32_t group;         /* FILTER_BATCH_TCF or FILTER_BATCH_GQF */
    uint32_t member;        /* member index in that group */
    uint32_t op;            /* FILTER_OP_* */
    uint32_t reserved;      /* 0 */
    const uint64_t *d_keys; /* n keys, device */
    uint64_t n;
    void *d_out;            /* device results, or NULL */
} filter_work;

int filter_batch_create(filter_group_t *tcf, filter_group_t *gqf, uint64_t max_keys, uint32_t max_items,
                        filter_batch_t **out);
int filter_batch_run(filter_batch_t *b, const filter_work *items, uint32_t n_items, void *stream);
int filter_batch_destroy(filter_batch_t *b);

/*
 * ---- serving loop ----
 * Batches of host keys for many filters, run concurrently on several CUDA
 * streams with continuous batching. The paper measures isolated bulk calls;
 * this runtime serves a stream of requests (each a batch for one filter) as
 * they arrive.
 *
 * filter_server_create: serve the given filters (created by filter_create on
 *   the current device; the caller keeps ownership and must not use them
 *   while the server runs) with n_workers workers (1..64). Each worker is a
 *   host thread with its own CUDA stream and pinned bounce buffers of
 *   max_keys keys (16 bytes per key). All workers share one device staging
 *   pool sized for n_workers batches of max_keys keys (16 bytes per key),
 *   or, when the free device memory is smaller, for as many such batches as
 *   fit (FILTER_ERR_OOM when not even one fits; nothing is created).
 * Scheduling: each filter has a FIFO of requests and at most one batch in
 *   flight. Any idle worker takes the oldest waiting request among the
 *   filters with nothing in flight, together with the requests queued right
 *   behind it on the same filter that can run as one device batch without
 *   changing any result: queries, counts, and removes from a GQF (a GQF's
 *   table depends only on the stored multiset, and the earlier request's keys
 *   come first). TCF inserts and removes and GQF inserts run alone. A batch
 *   is admitted when its staging (8 bytes per key plus its results) fits in
 *   the free part of the pool; until then it waits while batches of other
 *   filters run and release theirs (a batch passed over 8 times blocks
 *   later ones until it fits). So every filter applies its requests in
 *   submission order, batches of different filters overlap on the device,
 *   and each request's results equal those of the same per-filter sequence
 *   run alone. Every filter's max_batch must be >= the requests submitted to
 *   it; merged batches stay within max_batch and max_keys.
 * filter_server_submit: enqueue one request and return at once with a
 *   ticket. The key buffer (host memory, pageable or pinned) and the output
 *   buffer must stay valid until the ticket is collected. Page-locked buffers
 *   (cudaHostAlloc / cudaHostRegister) are copied to and from the device
 *   directly; pageable ones go through the worker's pinned bounce buffers.
 *   host_out receives n bytes of statuses (insert, remove) or found flags
 *   (query), or n uint64 counts (count, GQF only); NULL discards the
 *   results. FILTER_ERR_ARG for a bad filter index or op, n > max_keys, or a
 *   server being destroyed.
 * filter_server_wait: block until the request is done, then return
 *   FILTER_OK with *op_rc = the operation's return code and *latency_s = the
 *   seconds from submit to results in host_out. Each ticket is collected
 *   once; an unknown or collected ticket gives FILTER_ERR_ARG.
 * filter_server_get_stats: counters since creation (see the struct).
 * filter_server_destroy: finish every submitted request, stop the workers
 *   and free the pool and the buffers. The filters are left to the caller.
 */
#define FILTER_OP_INSERT 0
#define FILTER_OP_QUERY 1
#define FILTER_OP_REMOVE 2
#define FILTER_OP_COUNT 3

typedef struct filter_request {
    uint32_t filter;            /* index into the server's filter list */
    uint32_t op;                /* FILTER_OP_* */
    const uint64_t *host_keys;  /* n keys, host memory */
    uint64_t n;
    void *host_out;             /* results, host memory, or NULL */
} filter_request;

typedef struct filter_server filter_server_t;

int filter_server_create(filter_t *const *filters, uint32_t n_filters, uint32_t n_workers, uint64_t max_keys,
                         filter_server_t **out);
int filter_server_submit(filter_server_t *s, const filter_request *req, uint64_t *ticket);
int filter_server_wait(filter_server_t *s, uint64_t ticket, int *op_rc, double *latency_s);

typedef struct filter_server_stats {
    uint64_t batches;          /* device batches run */
    uint64_t requests;         /* requests run */
    uint64_t merged_requests;  /* requests that ran in a batch with others */
    uint64_t max_concurrent;   /* most batches in flight at once */
    uint64_t pool_bytes;       /* size of the device staging pool */
    uint64_t pool_peak_bytes;  /* most of the pool reserved at once */
} filter_server_stats;

int filter_server_get_stats(filter_server_t *s, filter_server_stats *out);
int filter_server_destroy(filter_server_t *s);

#ifdef __cplusplus
}
#endif
#endif
