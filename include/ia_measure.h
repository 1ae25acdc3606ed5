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
 * of record_bytes bytes at xorshift-random indices of table (device,
 * n_records records, aligned to its records; 16-byte aligned for 48), and
 * writes nothing that matters to sink (device, one float).  record_bytes: 48
 * (three float4, one vertex of the blended transform grid: the correspondence
 * search's gathers), 16, 8 (an fp32 hash-table entry) or 4 (an fp16 entry).
 * Timing it on a table the size of a kernel's own gives the random-gather
 * rate that kernel's gathers are measured against.
 * n_records 1..2^31, iters >= 1, blocks >= 1; IA_ERR_ARG otherwise. */
ia_status ia_gather_probe(const float *table, int64_t n_records, int record_bytes, int iters, int blocks, float *sink,
                          void *stream);

/* Random-atomic probe: every one of blocks x 256 threads adds a small constant
 * to `iters` records of table (device, n_records records of record_bytes = 8
 * (float2, a hash-table gradient entry) or 16 (float4) bytes, aligned to its
 * records) at xorshift-random indices, with one vector atomicAdd each: the
 * rate of the training scatter's gradient atomics.  The table's values change.
 * n_records 1..2^31, iters >= 1, blocks >= 1; IA_ERR_ARG otherwise. */
ia_status ia_atomic_probe(float *table, int64_t n_records, int record_bytes, int iters, int blocks, void *stream);

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
