/*
 * me_probe.h -- measurement helper of libme_b300.so (not part of the method).
 *
 * The roofline of the amplitude kernels is the chip's non-tensor FP64 / FP32 rate,
 * which the device properties do not state.  me_probe_alu_peak measures it with a
 * dependent-chain-free FMA loop on every SM of the current device.
 */
#ifndef ME_B300_PROBE_H
#define ME_B300_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Sustained FMA throughput of the current device in flop/s (an FMA counts 2):
 * prec 0 = FP64, 1 = FP32, 2 = packed FP32 pairs (fma.rn.f32x2, two FMAs per
 * instruction).  Runs for roughly 'seconds' (0.05 .. 5).  Returns 0 and
 * writes *flops_per_s, or a negative status (-1 bad argument, -4 CUDA error). */
int me_probe_alu_peak(int prec, double seconds, double* flops_per_s);

#ifdef __cplusplus
}
#endif
#endif
