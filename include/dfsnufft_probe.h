/*
 * dfsnufft_probe -- arithmetic-rate probe used to state the ALU roofline of
 * the FP64 form (the paper has no counterpart: it is a measurement aid of
 * this library, exported by the same shared object as dfsnufft.h).
 */
#ifndef DFSNUFFT_PROBE_H
#define DFSNUFFT_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Measure the device's fused multiply-add rate in FLOP/s (2 per FMA) for
 * dtype DFSNUFFT_F64 (0) or DFSNUFFT_F32 (1): a kernel of independent FMA
 * chains, one CTA per SM slot, timed with CUDA events on the legacy default
 * stream for about target_ms milliseconds after a warm-up.  Synchronous.
 * Returns 0 and writes *flops_per_s, or a dfsnufft status code. */
int dfsnufft_probe_fma_rate(int dtype, double target_ms, double *flops_per_s);

#ifdef __cplusplus
}
#endif

#endif /* DFSNUFFT_PROBE_H */
