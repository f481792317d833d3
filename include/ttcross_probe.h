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

/* Latency of a dependent binary64 FMA chain on one SM of the current device,
   the quantity that bounds the serial parts of the cross (the pivot steps,
   Alg. 4 replays, the FP64 re-scores).  One CTA: warps 0..chain_warps-1 run
   `iters` dependent FMAs on their lanes 0..active_lanes-1 (the other lanes
   idle); warps chain_warps..chain_warps+busy_warps-1 run four independent
   chains each on all lanes, a throughput load on the same SM.  Writes the
   clock cycles per dependent FMA of warp 0 to *cycles.  Limits:
   1 <= chain_warps, 0 <= busy_warps, chain_warps + busy_warps <= 32,
   1 <= active_lanes <= 32, 1 <= iters <= 2^30; else TTC_ERR_INVALID_ARG (1).
   Returns 0 or a ttc_status code (6: CUDA).  Synchronizes the device. */
int ttcross_probe_fp64_chain(int chain_warps, int active_lanes, int busy_warps, int64_t iters,
                             double *cycles);

/* Issue rate of one warp's independent binary64 FMAs: one CTA of `warps`
   warps (1..32), each lane running `chains` (1, 2, 4 or 8) independent FMA
   chains for `iters` iterations; writes the clock cycles per FMA instruction
   of warp 0 to *cycles.  Returns 0, 1 (INVALID_ARG) or 6 (CUDA).
   Synchronizes the device. */
int ttcross_probe_fp64_ilp(int warps, int chains, int64_t iters, double *cycles);

#ifdef __cplusplus
}
#endif
#endif
