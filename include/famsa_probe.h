/*
 * famsa_probe.h -- microbenchmarks behind the roofline figures, built into a
 * separate library (libfamsa_probe.so) that only the benchmark loads.  They
 * are not part of libfamsa_gpu.so and the paper has no counterpart.
 */
#ifndef FAMSA_PROBE_H
#define FAMSA_PROBE_H

#include "famsa_gpu.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Thread-instructions per second of one integer instruction kind run as
 * many independent chains over the whole device (kind 0 LOP3, 1 IADD3,
 * 2 IMAD, 3 LOP3 and IMAD alternating); it measures the width of the ALU
 * and FMA pipes for the LCS roofline.  Allocates a small output buffer. */
int famsa_probe_int_pipe_rate(int kind, double *inst_per_s);

/* SM clocks per repetition of one building block of the row update, on one
 * cluster of cluster_ctas (1, 2, 4, 8 or 16) CTAs of 512 threads, timed by
 * thread 0 of CTA 0 over 4,096 repetitions: kind 0 the block clamp scan with
 * order-code keys, 1 the same with cross-multiplied keys, 2 a cluster
 * barrier, 3 every CTA pushing one clamp into every CTA's shared memory and
 * a cluster barrier, 4 a dependent load from local shared memory, 5 a
 * dependent load from the next CTA's shared memory.  Allocates a few KB. */
int famsa_probe_cluster(int kind, int cluster_ctas, double *cycles);

#ifdef __cplusplus
}
#endif

#endif /* FAMSA_PROBE_H */
