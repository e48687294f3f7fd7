/*
 * famsa_gpu_debug.h -- test hooks of libfamsa_gpu.so (not needed by users).
 * The paper has no counterpart to these; they let the test suite reach
 * code paths that ordinary inputs rarely take.
 */
#ifndef FAMSA_GPU_DEBUG_H
#define FAMSA_GPU_DEBUG_H

#ifdef __cplusplus
extern "C" {
#endif

/* Make the n-th next device allocation made while packing a family fail with
 * FAMSA_ENOMEM (n = 0: the next one); n < 0 disables.  Returns FAMSA_OK. */
int famsa_debug_fail_alloc_after(int n);

/* Rows wider than w 64-bit words use the warp-per-pair LCS kernel instead of
 * thread-per-pair (default 32, the thread-per-pair maximum; 0 sends every
 * row to warp-per-pair).  Results are identical either way.  Returns
 * FAMSA_EINVAL for w outside 0..32. */
int famsa_debug_set_tpp_max_w(int w);

/* Force the number of CTAs in the thread-block cluster that runs the SLINK
 * row update (1, 2, 4, 8 or 16; 0 = automatic, the largest that fits).
 * Results are identical for every size.  Returns FAMSA_EINVAL otherwise. */
int famsa_debug_set_cluster(int ctas);

#ifdef __cplusplus
}
#endif

#endif /* FAMSA_GPU_DEBUG_H */
