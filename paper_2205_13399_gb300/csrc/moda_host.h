// Host-side helpers shared by the C-ABI translation units (not part of the
// public ABI): the per-device cooling schedule and -ln(u) table cache.
#pragma once

#include <cstdint>

#include "moda.h"

namespace moda {

struct ScheduleView {
  const double *delta;      // [count] delta_t, t = 1..count
  const int64_t *lo, *hi;   // [count] floor(delta_t T_min), floor(delta_t T_max)
  int32_t count;            // later iterations reuse the last entry
  const double *table;      // [65536] -ln((idx + 0.5) / 65536)
  double tmin, tmax;
};

// The schedule of (delta0, deltaf, xi) covering I_max iterations and the
// table on `device`, built once and cached (Alg. 3's cooling rule).
moda_status schedule_view(int device, double delta0, double deltaf, double xi,
                          int64_t I_max, ScheduleView *out);

}  // namespace moda
