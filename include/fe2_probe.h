/*
 * fe2_probe.h - measurement helper shipped with the library (not part of the
 * method; the paper has no counterpart).
 *
 * fe2_probe_smem_bandwidth: aggregate shared-memory read bandwidth of the
 * current device, measured by every SM streaming 16-byte reads from its own
 * shared memory (best of 5 timed launches, CUDA events). The relaxation
 * kernels stage each RVE's positions in shared memory, so this is the
 * bandwidth ceiling their roofline is quoted against.
 *   gbs           out: GB/s (1e9 bytes per second), aggregate over all SMs
 *   sm_clock_mhz  out (may be NULL): the device's maximum SM clock
 * Returns 0, 1 for a NULL gbs, 2 if the scratch allocation fails, 3 on a CUDA
 * error. Allocates and frees its own scratch; synchronous.
 *
 * fe2_probe_fp64_rates: aggregate FP64 throughput of the current device for
 * the operations of the FP64 relaxation kernel, whose arithmetic is IEEE
 * double with explicit rounding: fused multiply-add (the rate of a plain add
 * or multiply), correctly rounded division and correctly rounded square root.
 * Each is timed on 8 independent dependency chains per thread, 8 CTAs of 256
 * threads per SM (best of 5 launches, CUDA events).
 *   fma_per_s, div_per_s, sqrt_per_s  out: operations per second, all SMs
 * Returns 0, 1 for a NULL pointer, 2 if the scratch allocation fails, 3 on a
 * CUDA error. Allocates and frees its own scratch; synchronous.
 */
#ifndef FE2_PROBE_H
#define FE2_PROBE_H
#ifdef __cplusplus
extern "C" {
#endif
int fe2_probe_smem_bandwidth(double *gbs, double *sm_clock_mhz);
int fe2_probe_fp64_rates(double *fma_per_s, double *div_per_s, double *sqrt_per_s);
#ifdef __cplusplus
}
#endif
#endif
