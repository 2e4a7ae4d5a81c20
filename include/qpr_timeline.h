/* Kernel timeline of the column-block RK4 stage: entry points of the
 * diagnostic build only (libqpr_timeline.so, compiled with -DQPR_TIMELINE by
 * paper_2003_04930_gb300.build.build_library(timeline=True)); the product
 * library libqpr.so does not export them. The timeline measures the RK4 step
 * of the method (Eq. 1 integrated by classical RK4, one SpMM grid and one
 * epilogue per stage) as it runs inside the library's captured CUDA graphs.
 *
 * Layout of the stamps (host buffer of 8 x 2048 x 8 unsigned 64-bit values,
 * row-major): [kind][launch][field], kind = (stage - 1) * 2 + {0: SpMM grid,
 * 1: epilogue}, launch = the kind's launch index modulo 2048 since the last
 * reset, field 2f = the first and 2f + 1 = the last CTA's global timer value
 * (ns) of event f: 0 entered, 1 left, 2 column block staged (whole-block
 * SpMM product CTAs), 3 rows done (same CTAs). Unset first fields hold
 * UINT64_MAX and unset last fields 0. counts (8 values) = CTAs that entered
 * each kind since the reset (launches = counts / grid size).
 *
 * Both calls act on the current CUDA device, synchronise it and return 0 on
 * success, 1 on a CUDA error. The caller owns both buffers. */
#ifndef QPR_TIMELINE_H
#define QPR_TIMELINE_H

#ifdef __cplusplus
extern "C" {
#endif

#define QPR_TIMELINE_KINDS 8
#define QPR_TIMELINE_LAUNCHES 2048
#define QPR_TIMELINE_FIELDS 8

/* Clears the stamps and counters. */
int qpr_timeline_reset(void);
/* Copies the stamps (QPR_TIMELINE_KINDS x QPR_TIMELINE_LAUNCHES x
 * QPR_TIMELINE_FIELDS values) and the counters (QPR_TIMELINE_KINDS values). */
int qpr_timeline_read(unsigned long long *stamps, unsigned long long *counts);

#ifdef __cplusplus
}
#endif

#endif
