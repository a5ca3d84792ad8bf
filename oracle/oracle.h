/*
 * CPU oracle for the two GPU filters of "High-Performance Filters for GPUs"
 * (arXiv 2212.09005): the two-choice filter (TCF, Sec. 4) and the counting
 * quotient filter (GQF, Sec. 5).
 *
 * TEST INFRASTRUCTURE ONLY. This code is plain, single-threaded and slow on
 * purpose. It shares no code with the CUDA library. Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the
 * library path never calls it.
 *
 * Every function follows the filter specification written out in the
 * comments of hash.c, tcf.c and gqf.c, which state how each passage of the
 * paper is read where the paper is silent.
 */
#ifndef FILTER_ORACLE_H
#define FILTER_ORACLE_H
#include <stddef.h>
#include <stdint.h>

/* ---- hashing (hash.c) ---- */
uint64_t or_mix64(uint64_t x);
uint64_t or_unmix64(uint64_t x);
uint64_t or_mix_p(uint64_t x, unsigned p);
uint64_t or_unmix_p(uint64_t x, unsigned p);
uint64_t or_fold_p(uint64_t x, unsigned p);
void or_mix64_many(const uint64_t *in, uint64_t *out, uint64_t n);
void or_mix_p_many(const uint64_t *in, uint64_t *out, uint64_t n, unsigned p);

/* ---- TCF (tcf.c) ---- */
typedef struct or_tcf or_tcf;
or_tcf *or_tcf_new(unsigned log2_slots, unsigned tag_bits, uint64_t seed);
or_tcf *or_tcf_new_values(unsigned log2_slots, unsigned tag_bits, unsigned value_bits, uint64_t seed);
/* nb = 2^log2_blocks blocks of block_slots slots of tag_bits in {8, 12, 16} */
or_tcf *or_tcf_new_geom(unsigned log2_blocks, unsigned tag_bits, unsigned block_slots, unsigned value_bits,
                        uint64_t seed);
void or_tcf_free(or_tcf *T);
void or_tcf_keyinfo(const or_tcf *T, const uint64_t *keys, uint64_t n,
                    uint64_t *b1, uint64_t *b2, uint32_t *tag);
/* phase/where may be NULL; phase: 0 shortcut, 1 two-choice, 2 other block,
   3 backing, 4 rejected (full). where: block or backing bucket index. */
void or_tcf_insert(or_tcf *T, const uint64_t *keys, uint64_t n, uint8_t *status,
                   uint8_t *phase, uint64_t *where);
void or_tcf_insert_values(or_tcf *T, const uint64_t *keys, const uint8_t *values, uint64_t n,
                          uint8_t *status, uint8_t *phase, uint64_t *where);
void or_tcf_query(const or_tcf *T, const uint64_t *keys, uint64_t n, uint8_t *found);
void or_tcf_query_values(const or_tcf *T, const uint64_t *keys, uint64_t n, uint8_t *values);
void or_tcf_remove(or_tcf *T, const uint64_t *keys, uint64_t n, uint8_t *status);
uint64_t or_tcf_export_size(const or_tcf *T);
void or_tcf_export(const or_tcf *T, uint8_t *buf);
uint64_t or_tcf_backing_count(const or_tcf *T);
uint64_t or_tcf_stored_count(const or_tcf *T);
void or_tcf_geometry(const or_tcf *T, uint64_t *out8); /* nb, B, f, tsc, nbk, W, v, block bytes */

/* ---- GQF (gqf.c) ---- */
typedef struct or_gqf or_gqf;
or_gqf *or_gqf_new(unsigned q, unsigned r, uint64_t seed);
void or_gqf_free(or_gqf *G);
void or_gqf_fingerprints(const or_gqf *G, const uint64_t *keys, uint64_t n, uint64_t *fp);
void or_gqf_insert(or_gqf *G, const uint64_t *keys, uint64_t n, uint8_t *status);
void or_gqf_insert_counts(or_gqf *G, const uint64_t *keys, const uint32_t *counts, uint64_t n,
                          uint8_t *status);
void or_gqf_remove(or_gqf *G, const uint64_t *keys, uint64_t n, uint8_t *status);
void or_gqf_count(const or_gqf *G, const uint64_t *keys, uint64_t n, uint64_t *counts);
/* raw fingerprint groups (ascending, distinct); returns index of the first
   group that did not fit (m when all fit) */
uint64_t or_gqf_insert_groups(or_gqf *G, const uint64_t *fps, const uint64_t *cnts, uint64_t m);
uint64_t or_gqf_count_fp(const or_gqf *G, uint64_t fp);
uint64_t or_gqf_groups(const or_gqf *G, uint64_t *fps, uint64_t *cnts, uint64_t cap);
uint64_t or_gqf_export_size(const or_gqf *G);
void or_gqf_export(const or_gqf *G, uint8_t *buf);
uint64_t or_gqf_max_cluster(const or_gqf *G);
void or_gqf_geometry(const or_gqf *G, uint64_t *out5); /* N, S, nslots, nblk, p */
/* from-scratch canonical layout of a sorted distinct group list; returns 0 on
   success, 1 when the layout does not fit in the table */
int or_gqf_build(unsigned q, unsigned r, const uint64_t *fps, const uint64_t *cnts,
                 uint64_t m, uint8_t *buf);
uint64_t or_gqf_tail_slots(unsigned q);

#endif
