// Host check of moda::kernel_mode (the choice of annealing-kernel variant):
// the variants with the default algorithm compiled in (modes 3 to 5) are
// picked only for runs that use exactly that algorithm, and the variants
// with the placement compiled in (4, 5) only for runs with that placement.
// Exits nonzero on the first wrong choice.
#include <cstdio>

#include "moda_internal.h"

static int failures = 0;

static void expect(const moda::AnnealArgs &a, int rounds, int want, const char *what) {
  const int got = moda::kernel_mode(a, rounds);
  if (got != want) {
    std::printf("%s: rounds %d gave mode %d, want %d\n", what, rounds, got, want);
    ++failures;
  }
}

int main() {
  static unsigned char cache[16];
  moda::AnnealArgs base{};
  base.lookahead = 1;
  base.de_in_smem = 1;
  base.energies_in_smem = 1;
  base.bits_in_smem = 1;
  base.fcache = cache;

  expect(base, 1, 4, "default algorithm, on-chip placement");
  expect(base, 2, 3, "states on chip with two bits per thread");
  moda::AnnealArgs g = base;
  g.bits_in_smem = 0;
  for (int r : {2, 3, 4}) expect(g, r, 5, "states in global memory");
  for (int r : {1, 6, 8}) expect(g, r, 3, "states in global memory, other shapes");

  moda::AnnealArgs p = base;
  p.lookahead = 0;
  expect(p, 1, 3, "prefetch distance 0");
  p = base;
  p.lookahead = -1;
  expect(p, 1, 3, "cache read in place");
  p = base;
  p.fcache = nullptr;
  expect(p, 1, 3, "no field cache");
  p = base;
  p.de_in_smem = 0;
  expect(p, 1, 3, "Delta E not published");
  p = base;
  p.energies_in_smem = 0;
  expect(p, 1, 3, "energies in global memory");

  moda::AnnealArgs a = base;
  a.accept = 1;
  expect(a, 1, 0, "lenient acceptance");
  a = base;
  a.archive = 1;
  expect(a, 1, 0, "exploitative archive");
  a = base;
  a.escape = 1;
  expect(a, 1, 0, "offset escape");
  a = base;
  static int64_t trace[3];
  a.trace = trace;
  expect(a, 1, 0, "traced run");

  a = base;
  a.fast_forward = 1;
  expect(a, 1, 2, "fast-forward");
  a = base;
  a.normalize = 1;
  expect(a, 1, 1, "normalisation");
  a = base;
  a.snap_every = 10;
  expect(a, 1, 1, "snapshots");

  if (failures == 0) std::printf("kernel_mode: all choices as expected\n");
  return failures == 0 ? 0 : 1;
}
