/* A check of the annealing kernels' acceptance decision, exposed so that it
 * can be compared with the plain definition on any inputs.
 *
 * A bit whose acceptance penalty a (an integer >= 0: the strict sum or the
 * lenient minimum of max(0, Delta E_k), Eqs. pacceptms / pacceptml) lies
 * between the integer thresholds of R21 is accepted when
 *     a <= fl(delta * T[idx]),
 * T[idx] = -ln((idx + 0.5) / 65536) the quantised draw of Sec. 3.1 (R7) and
 * fl the IEEE double product.  The warp engine decides this in FP32 where
 * the FP32 result provably agrees and takes the double test otherwise;
 * moda_check_accept runs those same device functions.
 */
#ifndef MODA_CHECK_H_
#define MODA_CHECK_H_

#include <stdint.h>

#include "moda.h"

#ifdef __cplusplus
extern "C" {
#endif

/* For k < count: accept[k] = 1 if a[k] <= fl(delta[k] * T[idx[k]]), else 0,
 * as the device decides it; path[k] = 1 or 0 when the FP32 test decided,
 * -1 when the double test did.  a, delta, idx, accept and path are host
 * arrays of `count` entries owned by the caller (accept and path written).
 * Requires a[k] >= 0, delta[k] > 0 and finite, idx[k] < 65536
 * (MODA_EINVAL otherwise, before any device work).  Runs on the current
 * device on cuda_stream (NULL: the legacy default stream) and returns when
 * the results are on the host. */
moda_status moda_check_accept(const int64_t *a, const double *delta, const uint32_t *idx,
                              int32_t count, void *cuda_stream, uint8_t *accept, int8_t *path);

#ifdef __cplusplus
}
#endif

#endif /* MODA_CHECK_H_ */
