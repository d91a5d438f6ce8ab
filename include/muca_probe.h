/* muca_probe.h -- measurement probes of the device (not part of the method).
 *
 * The roofline of the sweep kernels needs two ceilings that a plain copy and
 * a bf16 GEMM do not give: the issue rate of 32-bit integer instructions and
 * the read bandwidth of the L2 cache.  These entry points measure them on the
 * current CUDA device with kernels of this library, timed with CUDA events on
 * the given stream (best of five launches after an untimed one).  They
 * allocate and free a few bytes (integer probe) or the probe buffer (L2 probe)
 * and synchronise the stream.
 *
 * Return codes: MUCA_PROBE_OK, MUCA_PROBE_ERR_INVALID_ARG (a bad argument, no
 * work done), MUCA_PROBE_ERR_CUDA (an allocation or launch failed).
 */
#ifndef MUCA_PROBE_H
#define MUCA_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MUCA_PROBE_OK 0
#define MUCA_PROBE_ERR_INVALID_ARG -1
#define MUCA_PROBE_ERR_CUDA -2

/* Integer instruction rate: eight 256-thread blocks per SM, each thread
 * running iters x 32 dependent-free 32-bit updates of one kind:
 *   0  multiply-add a = a * a + b  (one IMAD)
 *   1  three-input add a = a + b + c  (one IADD3)
 *   2  three-input logic a = (a & b) ^ c  (one LOP3)
 *   3  half multiply-adds, half three-input adds
 * ops_per_s: host FP64, updates (thread instructions) per second; ms: host
 * FP64, the best launch's duration, or NULL.  stream: a cudaStream_t (NULL =
 * the legacy default stream). */
int muca_probe_int(int32_t kind, int32_t iters, double *ops_per_s, double *ms, void *stream);

/* L2 read bandwidth: a device buffer of `bytes` (a multiple of 16, smaller
 * than the L2 for the result to mean L2), read whole reps times per launch by
 * four 512-thread blocks per SM with 16-byte loads that bypass L1.
 * bytes_per_s: host FP64; ms as above. */
int muca_probe_l2_read(int64_t bytes, int32_t reps, double *bytes_per_s, double *ms,
                       void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MUCA_PROBE_H */
