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
 */
#ifndef FE2_PROBE_H
#define FE2_PROBE_H
#ifdef __cplusplus
extern "C" {
#endif
int fe2_probe_smem_bandwidth(double *gbs, double *sm_clock_mhz);
#ifdef __cplusplus
}
#endif
#endif
