/*
 * dfsnufft_probe -- arithmetic-rate probe used to state the ALU roofline of
 * the FP64 form, and a self-test of the bounded waits (the paper has no
 * counterpart: measurement and test aids of this library, exported by the
 * same shared object as dfsnufft.h).
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

/* Self-test of the bounded waits: one CTA initialises an mbarrier that
 * nothing ever arrives on and waits on it with the same bounded wait the TMA
 * kernels use, giving up after `cycles` SM clock cycles (1 <= cycles <= 4e9,
 * about 2 s at 2 GHz).  The kernel then writes the timeout code to a device
 * status word and returns, as the TMA kernels do, so the context stays usable.
 * Synchronous.  *device_status receives the word (1 = timed out, the expected
 * outcome), *elapsed_ms the kernel's duration.  No paper counterpart: a check
 * of this library's failure detection that needs no GPU fault. */
int dfsnufft_selftest_wait_timeout(long long cycles, int *device_status, double *elapsed_ms);

/* Self-test of the persistent ensemble step's queue waits: the last step of an
 * ensemble in persistent mode is launched once more, uncaptured and
 * synchronously, with group 0's count of theta tasks one higher than it can
 * ever reach, so that its phi tasks wait for a completion that never comes.
 * Each wait gives up after `cycles` SM clock cycles (1 <= cycles <= 4e9); the
 * first that does raises the step's abort flag and timeout status, the other
 * CTAs skip their remaining tasks and the launch ends.  Returns
 * DFSNUFFT_ERR_TIMEOUT (the expected outcome) or DFSNUFFT_OK, without making
 * the failure sticky: the values of that launch are incomplete, and the next
 * dfsnufft_ensemble_run computes normally.  DFSNUFFT_ERR_NO_POINTS if the
 * ensemble is not in persistent mode or has not run a step yet. */
int dfsnufft_ensemble_selftest_queue_timeout(struct dfsnufft_ensemble_s *ens, long long cycles);

#ifdef __cplusplus
}
#endif

#endif /* DFSNUFFT_PROBE_H */
