/*
 * rpim_probe.h -- measurement helpers of librpim: FP64 throughput probes used
 * to state the roofline of the assembly kernels (the paper gives no hardware
 * figures; the FP64 rate of the GPU is measured, not assumed), a count of
 * the library's kernel launches, and optional per-kernel device timing.
 *
 * Both run on the current CUDA device, synchronise it, and return the best
 * of `repeats` timed launches (CUDA events) in GFLOP/s through `gflops`
 * (host pointer).
 *   rpim_probe_dfma: independent fused multiply-add chains on the FP64 pipe
 *     (2 flops per DFMA).
 *   rpim_probe_dmma: mma.sync m8n8k4 FP64 tensor-core instructions
 *     (512 flops each).
 *   rpim_probe_fp64_mixed: half the warps on each of the two (equal flops
 *     per half): the combined rate tells whether the paths add up.
 * Errors: RPIM_E_ARG (null pointer), RPIM_E_CUDA.
 */
#ifndef RPIM_PROBE_H
#define RPIM_PROBE_H
#include "rpim.h"
#ifdef __cplusplus
extern "C" {
#endif
rpim_status rpim_probe_dfma(int32_t repeats, double *gflops);
rpim_status rpim_probe_dmma(int32_t repeats, double *gflops);
rpim_status rpim_probe_fp64_mixed(int32_t repeats, double *gflops);

/* Host-only (no GPU needed): the piecewise series that the shape-function
 * kernel uses for the multiquadric minus its chord, for the given
 * parameters: number of pieces, degree, number of FP64 (head) terms, and the
 * largest absolute error of the device evaluation order against the closed
 * form, measured on 129 points per piece of the range of s in long double.
 * Errors: RPIM_E_ARG (parameters out of range, or the check failed). */
rpim_status rpim_kernel_series_info(double alpha_c, double alpha_s, double q, int32_t *pieces,
                                    int32_t *degree, int32_t *fp64_terms, double *max_err);

/* The reciprocal the RPIM shape kernel takes of its pivots and of the
 * determinant of the pivot tetrahedron (Newton-Raphson from a
 * single-precision seed): r[i] = 1/d[i] for device arrays d, r of n doubles,
 * |d[i]| in [2^-126, 2^126] (d and 1/d single-precision normal). For
 * checking its accuracy against correctly rounded division. Synchronises
 * `stream`. Errors: RPIM_E_ARG, RPIM_E_CUDA. */
rpim_status rpim_probe_recip(int64_t n, const double *d, double *r, rpim_stream_t stream);

/* Number of kernels this library has launched since it was loaded. */
int64_t rpim_kernel_launches(void);

/* Number of device-memory allocations this library has requested since it
 * was loaded (every stream-ordered cudaMallocAsync of the stages and every
 * cudaMalloc of the probes above): the count does not change across a call
 * that allocates nothing. */
int64_t rpim_device_allocations(void);

/* Bytes currently in use from the current device's default stream-ordered
 * memory pool (cudaMemPoolAttrUsedMemCurrent), which serves every allocation
 * of the stages: the driver's own count, independent of the library's.
 * Errors: RPIM_E_ARG (null pointer), RPIM_E_CUDA. */
rpim_status rpim_pool_used_bytes(int64_t *bytes);

/* Turns per-kernel timing on or off (off at load). When on, every launch is
 * bracketed by two CUDA events recorded on the launch's own stream; this
 * adds two event records per launch and nothing else. */
rpim_status rpim_profile_enable(int32_t on);

/* Writes, as a JSON object into buf (host, cap bytes), the per-kernel totals
 * gathered while timing was on: {"name": [launches, total_ms], ...}.
 * Waits for the recorded events. reset != 0 clears the totals.
 * Errors: RPIM_E_ARG (null or too small buffer). */
rpim_status rpim_profile_read(char *buf, int64_t cap, int32_t reset);
#ifdef __cplusplus
}
#endif
#endif
