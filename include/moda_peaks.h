/* Measured on-chip peaks that bound the annealing kernel (integer work and
 * shared memory; it uses no tensor cores and little HBM bandwidth).  Used as
 * the denominators of its roofline fraction.
 *
 * Both probes run one launch of 4 x SM-count blocks of 512 threads on the
 * current device and time it with CUDA events on `cuda_stream` (NULL = the
 * legacy default stream); they block until it finished.
 */
#ifndef MODA_PEAKS_H_
#define MODA_PEAKS_H_

#include <stdint.h>

#include "moda.h"

#ifdef __cplusplus
extern "C" {
#endif

/* INT32 lane operations per second: every thread runs eight independent
 * dependency chains of single-instruction integer operations (multiply-add,
 * three-input xor, three-input add, min), `iters` rounds of 32 operations.
 * *ops_per_s receives lanes x operations / seconds, *ms the kernel time. */
moda_status moda_probe_int_peak(int32_t iters, void *cuda_stream, double *ops_per_s,
                                float *ms);

/* Shared-memory load bandwidth: every thread reads 16-byte vectors from a
 * 32 KiB shared buffer, conflict-free, `iters` rounds of 8 loads.
 * *bytes_per_s receives bytes loaded / seconds, *ms the kernel time. */
moda_status moda_probe_smem_peak(int32_t iters, void *cuda_stream, double *bytes_per_s,
                                 float *ms);

#ifdef __cplusplus
}
#endif

#endif /* MODA_PEAKS_H_ */
