/*
 * ae_peak.h -- integer-ALU throughput of the current GPU, measured (libae.so).
 *
 * The search's row and sweep kernels are integer code: adds, maxima and the
 * DPX add-max of sm_90+ on int32 and packed int16x2 values.  Their roofline is
 * the rate at which the GPU retires those instructions, which no data sheet
 * states for this part.  This entry point measures it: every thread of a full
 * grid runs `chains` independent dependency chains of one operation kind, so
 * that the schedulers always have independent work, and the kernel is timed
 * with CUDA events on `stream`.  The paper has no counterpart (its method is
 * measured on a CPU).
 *
 * Kinds:
 *   AE_PEAK_IADD       int32 add                       (1 op per instruction)
 *   AE_PEAK_IMAX       int32 max                        (1 op)
 *   AE_PEAK_ADDMAX32   __viaddmax_s32: max(a + b, c)    (counted as 2 ops)
 *   AE_PEAK_ADDMAX16X2 __viaddmax_s16x2 on int16 pairs  (counted as 4 ops)
 * Every chain step depends on the previous step through values the compiler
 * cannot know (kernel arguments), so no step can be folded away.
 *
 * Outputs: *ops_per_s = operations retired per second over the whole GPU (as
 * counted above), *insts_per_s = the same for instructions, *ms = the kernel's
 * device time.  `blocks_per_sm` x the SM count blocks of 256 threads are
 * launched; each thread runs `iters` x 16 steps of each of `chains` (1..8)
 * chains.  The call allocates 4 bytes of device memory per thread for the
 * results (so the chains are live) and frees them before it returns; it
 * returns after the stream has finished.
 * Errors: AE_EINVAL (unknown kind, chains outside 1..8, iters < 1,
 * blocks_per_sm < 1), AE_ENOMEM, AE_ECUDA.
 */
#ifndef AE_PEAK_H
#define AE_PEAK_H

#include <stdint.h>

#include "ae.h"

#ifdef __cplusplus
extern "C" {
#endif

enum { AE_PEAK_IADD = 0, AE_PEAK_IMAX = 1, AE_PEAK_ADDMAX32 = 2, AE_PEAK_ADDMAX16X2 = 3 };

ae_status ae_int_peak(int32_t kind, int32_t chains, int32_t iters, int32_t blocks_per_sm, void *stream,
                      double *ops_per_s, double *insts_per_s, double *ms);

#ifdef __cplusplus
}
#endif

#endif /* AE_PEAK_H */
