/*
 * famsa_gpu_debug.h -- test hooks of libfamsa_gpu.so (not needed by users).
 * The paper has no counterpart to these; they let the test suite reach
 * code paths that ordinary inputs rarely take.
 */
#ifndef FAMSA_GPU_DEBUG_H
#define FAMSA_GPU_DEBUG_H

#include "famsa_gpu.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Make the n-th next device allocation made while packing a family fail with
 * FAMSA_ENOMEM (n = 0: the next one); n < 0 disables.  Returns FAMSA_OK. */
int famsa_debug_fail_alloc_after(int n);

/* The family's packed match-bitmask (Peq) tables, copied to the host:
 * peq (n_words * 64 u32) in the family's (length, index) order -- per word
 * of a sequence, 32 u32 holding bits 0..31 of the mask of symbols 0..31,
 * then 32 u32 holding bits 32..63 --, word_off (k + 1 int64: the first word
 * of each sorted sequence, then the total) and perm (k int32: the caller's
 * label of each sorted sequence).  Any output may be NULL; n_words receives
 * the total.  EINVAL for a NULL handle. */
int famsa_debug_peq(const famsa_family *f, uint32_t *peq, int64_t *word_off, int32_t *perm, int64_t *n_words);

/* The number of device allocations the library has made in this process so
 * far (every one goes through one stream-ordered allocation routine).  Tests
 * use it to check that a call allocates nothing. */
int64_t famsa_debug_alloc_count(void);

/* The checked build (libfamsa_gpu_checked.so, compiled with -DFAMSA_CHECKED)
 * tests the invariants each kernel's indexing relies on (indices inside their
 * buffers, rows inside their kernel's width, ids inside their range) and
 * counts every failure, skipping the access it guards, instead of faulting.
 * Returns the failures counted so far on the current device, with the source
 * line of the first one in *first_line (may be NULL); -1 from the normal
 * build, which has no checks. */
int64_t famsa_debug_check_count(int64_t *first_line);

/* The checker's own test: in the checked build, launches one kernel whose one
 * check fails on purpose (it guards no access), so the count above grows by
 * one; returns FAMSA_OK (or ECUDA).  -1 from the normal build. */
int famsa_debug_check_selftest(void);

/* Rows wider than w 64-bit words do not use the thread-per-pair LCS kernel
 * (default 32, the thread-per-pair maximum): they take the sliced kernel
 * where famsa_debug_set_slices covers their width, else warp-per-pair (with
 * slices off, 0 sends every row to warp-per-pair).  Results are identical
 * either way.  Returns FAMSA_EINVAL for w outside 0..32. */
int famsa_debug_set_tpp_max_w(int w);

/* Rows of at least min_w words (64 residues each) run on the sliced kernel:
 * the row's bit vector split across up to 16 warps of at most `words` words
 * each (1..16; 0 = 16), the add's carries passed from warp to warp through
 * shared memory once per 16 column symbols.  min_w = 0 turns it off (rows
 * then take thread-per-pair up to famsa_debug_set_tpp_max_w, warp-per-pair
 * beyond); the default is 24.  Rows wider than 256 words always take
 * warp-per-pair.  Results are identical for every setting.  Returns
 * FAMSA_EINVAL for a negative min_w or words outside 0..16. */
int famsa_debug_set_slices(int min_w, int words);

/* Force the number of CTAs in the thread-block cluster that runs the SLINK
 * row update (1, 2, 4, 8 or 16; 0 = automatic, the largest that fits).
 * Results are identical for every size.  Returns FAMSA_EINVAL otherwise. */
int famsa_debug_set_cluster(int ctas);

/* Select the row update: 0 automatic (3 when every length is <= 32767,
 * else the insertion kernels: cluster shared memory when the family fits,
 * else global memory), 1 insertion in cluster shared memory (the tree call
 * returns FAMSA_EINVAL when the family does not fit), 2 insertion in global
 * memory, 3 minimum-spanning-tree rebuild per row block (FAMSA_EINVAL from
 * the tree call when a length is above 32767).  Results are identical.
 * Returns FAMSA_EINVAL outside 0..3. */
int famsa_debug_set_update_path(int path);

/* Rows per row block of famsa_slink_tree (0 = automatic; otherwise 1 to
 * 2048).  Small blocks make many blocks out of a small family.  Results are
 * identical.  Returns FAMSA_EINVAL outside 0..2048. */
int famsa_debug_set_row_block(int rows);

/* The pointer representation produced by the insertion row updates (paths
 * 1 and 2) of the last famsa_slink_tree call on f, in insertion labels: points are inserted in
 * the family's (length, index) order; perm[j] is the caller's label of the
 * j-th inserted point, pi[j] / (lam_num[j], lam_den[j]) its pointer and
 * height (reduced; +inf = (1, 0)).  Host arrays of k entries; any may be
 * NULL.  Returns FAMSA_EINVAL when no tree was built on f by an insertion
 * path. */
int famsa_debug_insertion_state(const famsa_family *f, int32_t *perm, int32_t *pi,
                                uint64_t *lam_num, uint32_t *lam_den);

/* Threads per CTA of the shared-memory row-update kernel (128, 256 or 512;
 * 0 = default 512).  Results are identical.  Returns FAMSA_EINVAL otherwise. */
int famsa_debug_set_update_threads(int threads);

/* 1: the LCS of a row block waits for the row update of the previous block
 * (no overlap of the two streams), for timing studies; 0: overlap (default). */
int famsa_debug_set_serial(int on);

/* Kilocycles spent by one thread of the row-update kernel in the sub-steps
 * of its last tree build on f (out16: 16 int64).  Shared-memory kernel: 0..7
 * the common path, 8..13 the run merge in shared memory.  Global-memory
 * kernel: 0 phase-A tiles, 1..3 warp totals and the cluster barrier, 4 CTA
 * prefixes, 5 forward scan, 6 backward scan and pointer update, 7..8 first
 * minimum and the barrier, 9 re-layout, 10 its barrier, 11 run merges. */
int famsa_debug_sub_kcycles(const famsa_family *f, int64_t *out16);

/* Rows per tile r (1, 2 or 4 with r * w <= 32; 0 = the default) of the
 * thread-per-pair LCS kernel for rows of w 64-bit words, as the batch
 * autotuner sets it.  Results are identical for every r.  EINVAL for other
 * values.  famsa_debug_tpp_rows returns the r in use for w (-1 for a bad w). */
int famsa_debug_set_tpp_rows(int w, int r);
int famsa_debug_tpp_rows(int w);

/* Batch autotuner on (1, default) or off (0; also forgets the widths tuned
 * so far, but keeps their choices until famsa_debug_set_tpp_rows resets them). */
int famsa_debug_set_autotune(int on);

/* Threads a CTA of the global-memory row-update kernel: -1 (default) by the
 * row block's size (512 below 100,000 points, else 1,024), 0 1,024, 1 512.
 * Results are identical.  EINVAL outside -1..1. */
int famsa_debug_set_global_variant(int v);

/* on != 0 (default): families of up to 4,096 points are finalised by one
 * CTA in one launch; 0: every family takes the multi-kernel finalisation.
 * Both give the same outputs.  Returns FAMSA_OK. */
int famsa_debug_set_fin_small(int on);

/* The row update's exact order code of the distance num / den (den in
 * 1..32767, num < 2^32): floor(num * 2^30 / den), and back from a code to the
 * distance as a reduced fraction.  Host-only arithmetic, no GPU needed;
 * FAMSA_EINVAL for a den out of range or a null pointer. */
int famsa_debug_order_code(uint32_t num, uint32_t den, uint64_t *code);
int famsa_debug_code_fraction(uint64_t code, uint64_t *num, uint32_t *den);

#ifdef __cplusplus
}
#endif

#endif /* FAMSA_GPU_DEBUG_H */
