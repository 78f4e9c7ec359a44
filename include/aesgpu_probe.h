/*
 * aesgpu_probe.h — micro-benchmarks behind the roofline denominators of the
 * bulk-AES kernels (libaesgpu_probe.so; used by bench.py, not by the
 * product path).  The paper has no counterpart: it measures CPU throughput
 * only (§V, Table I).  All calls are synchronous and allocate their own
 * scratch; they return 0 on success, non-zero on a bad argument (1) or a
 * CUDA failure (2-4).
 */
#ifndef AESGPU_PROBE_H
#define AESGPU_PROBE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Number of pipe-probe kinds: 0 LOP3, 1 PRMT, 2 32-bit add, 3 funnel shift,
 * 4 IMAD, 5 conflict-free 32-bit shared load, 6 LOP3+IMAD, 7 LOP3+LDS,
 * 8 PRMT+LDS, 9 LOP3+PRMT. */
int aesgpu_probe_num_kinds(void);

/* Thread-operations one probe unit counts (2 for the mixed kinds). */
int aesgpu_probe_ops_per_unit(int kind);

/* One CTA of `threads` threads per SM runs `iters` x 128 steps of 8
 * independent chains of the kind's instruction(s); writes the median over SMs
 * of thread-operations per SM clock, and the launch's wall time. */
int aesgpu_probe_pipe(int kind, int threads, int iters, double *ops_per_clk_per_sm,
                      double *seconds);

/* Streaming 128-bit device copy; best of `reps` read+write GB/s.
 * d_in, d_out: device, 16-byte aligned, nbytes a multiple of 16. */
int aesgpu_probe_copy(const void *d_in, void *d_out, size_t nbytes, int ctas_per_sm, int threads,
                      int reps, double *gbps);

#ifdef __cplusplus
}
#endif
#endif
