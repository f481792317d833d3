/*
 * ttcross_probe.h -- measurement helper of libttcross (not part of the method).
 *
 * The FP64 and FP32 pipes bound the residual screen of the TT cross (the
 * screen is a fused skinny contraction that never writes its result), so the
 * benchmark reports its arithmetic rate against a peak measured on the same
 * GPU with a dependent-FMA loop.
 */
#ifndef TTCROSS_PROBE_H
#define TTCROSS_PROBE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* Runs an FMA-throughput loop on the current device: `fp64` != 0 for binary64
   FMAs, else binary32.  Writes the sustained rate in FMA/s (one FMA = 2 flops)
   to *fma_per_s and the kernel time to *ms.  Launches blocks_per_sm CTAs of
   256 threads per SM, each thread running `iters` iterations of 8 independent
   FMA chains.  Returns 0 on success, else a ttc_status code (INVALID_ARG,
   CUDA).  Synchronizes the device. */
int ttcross_probe_fma_peak(int fp64, int blocks_per_sm, int64_t iters, double *fma_per_s,
                           double *ms);

#ifdef __cplusplus
}
#endif
#endif
