/*
 * ia_measure.h — measurement aids of the sm_103a library (libia.so).
 *
 * Nothing here is part of the method (the paper has no counterpart): these
 * calls only measure the library's kernels and the hardware they run on, for
 * the benchmark's per-kernel timings and roofline denominators.  Conventions
 * as in ia.h (status codes, `stream` as a cudaStream_t passed as void*).
 */
#ifndef IA_MEASURE_H
#define IA_MEASURE_H

#include <stdint.h>

#include "ia.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Random-gather probe: every one of blocks x 256 threads reads `iters` records
 * of 48 bytes (three float4, the size of one vertex of the blended transform
 * grid) at xorshift-random indices of table [n_records][12] fp32 (device,
 * 16-byte aligned), and writes nothing that matters to sink (device, one
 * float).  Timing it on a table that fits L1 or L2 gives the random-gather
 * rate the correspondence search's gathers are measured against.
 * n_records 1..2^31, iters >= 1, blocks >= 1; IA_ERR_ARG otherwise. */
ia_status ia_gather_probe(const float *table, int64_t n_records, int iters, int blocks, float *sink, void *stream);

/* Per-kernel device times of the library's launches.  ia_profile_begin opens
 * a profile on the calling host thread; until ia_profile_end, every kernel the
 * library launches from this thread (any context, any stream) is bracketed by
 * two CUDA events recorded on its launch stream (a few microseconds of extra
 * host work per launch; results of the calls are unchanged).  ia_profile_end
 * waits for those events and returns one entry per kernel name, in order of
 * first launch: out [max_out] (host, may be NULL when max_out is 0), *n_out =
 * the number of distinct kernels (entries beyond max_out are dropped).
 * IA_ERR_STATE when no profile is open (end) or one is already open (begin);
 * IA_ERR_ARG for bad output arguments (the profile then stays open);
 * IA_ERR_CUDA when an event failed.  Messages: ia_profile_error(). */
typedef struct ia_kernel_time {
  char name[48];       /* kernel, with its precision / search variant */
  int64_t launches;
  double total_ms;     /* summed event-to-event device time */
  double max_ms;       /* longest single launch */
} ia_kernel_time;

ia_status ia_profile_begin(void);
ia_status ia_profile_end(ia_kernel_time *out, int max_out, int *n_out);
const char *ia_profile_error(void);

#ifdef __cplusplus
}
#endif
#endif /* IA_MEASURE_H */
