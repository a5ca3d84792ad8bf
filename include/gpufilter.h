/*
 * gpufilter: GPU two-choice filter (TCF) and counting quotient filter (GQF)
 * for NVIDIA GB300 (sm_103a), after "High-Performance Filters for GPUs"
 * (Pandey et al., arXiv 2212.09005).
 *
 * C ABI. Every pointer argument named d_* is a device pointer; host_* is host
 * memory. Streams are cudaStream_t values passed as void* (NULL = the legacy
 * default stream). All calls except filter_create, filter_destroy,
 * filter_get_stats, filter_export and filter_import are asynchronous: they
 * enqueue kernels on the stream and return; the caller's buffers must stay
 * valid until the stream reaches the call. Calls on one filter must be
 * ordered (same stream, or externally synchronised); different filters are
 * independent.
 *
 * Errors are returned synchronously for bad arguments, allocation failure
 * and unsupported operations. Conditions found on the device (a full table,
 * a bounded wait that gave up) are recorded in a sticky status word read by
 * filter_get_stats, and per key in the optional status arrays.
 *
 * Fingerprints and layouts
 *   TCF (paper Sec. 4): h = mix64(key ^ seed), block b1 = h mod nb, tag =
 *   bits 44.. of h (f bits, 0 and 1 moved to 2 and 3), b2 = b1 xor g(tag).
 *   nb = 2^log2_slots / B blocks of 32 bytes (B = 256 / f tags). Backing
 *   table: nbk buckets of 8 uint64 entries (min(b1,b2) << f | tag), nbk =
 *   max(8, ceil(ceil(N/100) / 8)) (Sec. 4.1, "backing table").
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
    uint32_t tag_bits;    /* TCF: f in {8, 16}; GQF: r in {8, 16} */
    uint32_t mode;        /* TCF: FILTER_MODE_BULK or FILTER_MODE_POINT; GQF: 0 */
    uint64_t hash_seed;   /* xor-ed into keys before hashing */
    uint64_t max_batch;   /* largest n of one call; sizes the scratch memory (GQF: < 2^30) */
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
 * Returns FILTER_ERR_ARG for a bad geometry (TCF: f in {8,16}, 2^log2_slots
 * >= 2 blocks, nb <= 2^32; GQF: r in {8,16}, 6 <= q <= 36, q + r <= 64),
 * FILTER_ERR_OOM if an allocation fails (nothing is leaked).
 */
int filter_create(const filter_config *cfg, void *stream, filter_t **out);

/* filter_destroy: synchronise the device and free everything. NULL is a no-op. */
int filter_destroy(filter_t *f);

/* filter_clear: empty the table (asynchronous) and reset the statistics. */
int filter_clear(filter_t *f, void *stream);

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
 * filter_query: d_found[i] = 1 if key i may be in the set (no false
 * negatives; false positives at the filter's rate), else 0.
 * TCF: tag in block b1 or b2 or the backing bucket. GQF: count > 0.
 * Any n (not limited by max_batch).
 */
int filter_query(filter_t *f, const uint64_t *d_keys, uint64_t n, uint8_t *d_found,
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
 * with its name and its work units (keys, slots or blocks, per kernel).
 * filter_trace_summary synchronises the recorded events and returns, per
 * kernel name, the launch count, the summed units and the summed device time
 * in milliseconds. Enabling costs two event records per launch.
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
 *   cudaGetSymbolAddress, with that device current; make that first call
 *   before any stream capture. The call is asynchronous on `stream` except
 *   when the table overflows, where it synchronises `stream`, as
 *   filter_insert does.
 */
#define FILTER_NOALLOC_MAX_KEYS 65536u
#define FILTER_NOALLOC_MAX_Q 20u
int filter_gqf_insert_noalloc(uint32_t q, uint32_t r, uint64_t hash_seed, const void *d_table_in,
                              void *d_table_out, const uint64_t *d_keys, uint64_t n,
                              uint8_t *d_status, void *stream);

#ifdef __cplusplus
}
#endif
#endif
