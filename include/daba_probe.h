/*
 * daba_probe.h -- measurement helper of the DABA library (not part of the method): the
 * fused multiply-add rate of the current GPU, the denominator of the roofline of the
 * library's arithmetic-bound kernels (the FP64 path is bound by the FP64 pipe).
 */
#ifndef DABA_PROBE_H_
#define DABA_PROBE_H_

#ifdef __cplusplus
extern "C" {
#endif

/* Runs, over the whole current GPU (8 CTAs of 256 threads per SM), a kernel in which every
 * thread advances 8 independent fused multiply-add chains, and writes the best rate of three
 * timed launches (after one untimed) to *flops_per_s, counting 2 FLOP per multiply-add.
 * kind 0: FP32 fmaf; 1: packed FP32 (__ffma2_rn, two multiply-adds per instruction);
 * 2: FP64 fma. Allocates and frees a small device buffer. Returns 0 on success, 1 for an
 * invalid argument, 2 if a CUDA call failed, 3 if the allocation failed. */
int daba_probe_fma_rate(int kind, double* flops_per_s);

#ifdef __cplusplus
}
#endif

#endif /* DABA_PROBE_H_ */
