/*
 * pthr_peaks.h -- on-device microbenchmarks of the rates that bound the PTHR
 * kernels (part of libpthr.so).
 *
 * The paper has no counterpart: it reports no throughput numbers and runs on
 * CPUs.  The local sweep of Sec. 3 item (i) is bound on GB300 by instruction
 * issue and shared-memory traffic, not by HBM, so its roofline fractions need
 * the shared-memory, L2 and per-pipe issue rates of the device it runs on.
 * These entry points measure them.
 */
#ifndef PTHR_PEAKS_H
#define PTHR_PEAKS_H

#include "pthr.h"

#ifdef __cplusplus
extern "C" {
#endif

enum {
    PTHR_PEAK_SMEM_READ = 0,  /* shared-memory load bandwidth, bytes/s (16-byte loads,
                                 conflict-free)                                        */
    PTHR_PEAK_L2_READ = 1,    /* L2 load bandwidth with L1 bypassed, bytes/s; reads up
                                 to 16 MB of the scratch buffer                        */
    PTHR_PEAK_ALU = 2,        /* integer-logic (lop3) instructions/s, thread level     */
    PTHR_PEAK_FMA = 3,        /* FP32 fma instructions/s, thread level                 */
    PTHR_PEAK_FMA2 = 4,       /* packed f32x2 fma instructions/s (two FMAs each)       */
    PTHR_PEAK_FP64 = 5,       /* FP64 fma instructions/s, thread level                 */
    PTHR_NPEAK = 6
};

/* Run microbenchmark `kind` (PTHR_PEAK_*) once to warm up and once timed with
 * CUDA events on `stream` (cudaStream_t; NULL = legacy default stream), over
 * every SM of the current device, and return its rate in *rate (bytes/s or
 * instructions/s) and the timed launch's duration in *seconds.
 * scratch_device: caller-owned device memory of scratch_bytes bytes (the
 * library allocates none); every kind stores a few words into its first
 * 4096 bytes, PTHR_PEAK_L2_READ also reads up to 16 MB after them (at least
 * 4096 + 16 MB recommended; less gives a smaller L2 working set).  Its
 * contents are not preserved.  Synchronises the stream.  Returns
 * PTHR_E_INVAL for a bad kind, NULL pointer or too little scratch and
 * PTHR_E_CUDA if a launch fails. */
PTHR_API pthr_status pthr_measure_peak(int kind, void *scratch_device, size_t scratch_bytes,
                                       void *stream, double *rate, double *seconds);

#ifdef __cplusplus
}
#endif
#endif /* PTHR_PEAKS_H */
