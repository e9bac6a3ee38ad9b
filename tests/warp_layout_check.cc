// Host check of the warp engine's record and shared-memory layouts
// (moda::warp_rec, moda::warp_smem) for every n the library accepts and the
// buffer counts the launch planner can choose:
//  - every part a bulk copy (TMA) reads or writes starts on a 16-byte
//    boundary and has a multiple of 16 bytes: the jump record, its header
//    (candidate masks, state words, counts, energies), the header buffers
//    of the frozen-schedule layout;
//  - the frozen layout (one full record, a rebuild scratch of n^2 int32,
//    nbuf_f headers) stays inside the buffer region, and the region of the
//    normal layout holds nbuf full records;
//  - the parts of the team's and a warp's shared memory do not overlap,
//    and the per-target record ring holds the longest window plus prefetch.
// Exits nonzero on the first violation.
#include <cstdio>

#include "moda_internal.h"

static int failures = 0;

static void check(bool ok, const char *what, int n, int nbuf, int nbuf_f) {
  if (!ok) {
    std::printf("n %d nbuf %d nbuf_f %d: %s\n", n, nbuf, nbuf_f, what);
    ++failures;
  }
}

int main() {
  // (lookahead, window) pairs the planner tries
  static const int kOpts[][2] = {{14, 15}, {10, 11}, {8, 9}, {6, 7}, {5, 6}, {4, 5},
                                 {3, 4}, {2, 3}, {1, 2}, {2, 1}, {1, 1}, {0, 1}};
  for (int n = 2; n <= moda::kMaxN; ++n) {
    const int m = n * n;
    const moda::WarpRec r = moda::warp_rec(n, m);
    check(r.mp % 128 == 0 && r.mp >= m && r.mp - m < 128, "padded bits", n, 0, 0);
    check(r.off_cm == 4u * (uint32_t)r.mp, "masks follow the penalties", n, 0, 0);
    const uint32_t offs[] = {r.off_cm, r.off_xw, r.off_rc, r.off_E, r.jr, r.hb, r.lr};
    for (uint32_t o : offs) check(o % 16 == 0, "16-byte record part", n, 0, 0);
    check(r.off_xw - r.off_cm == (uint32_t)r.mp / 8, "one mask bit per bit", n, 0, 0);
    check(r.off_rc - r.off_xw == (uint32_t)r.mp / 8, "state words", n, 0, 0);
    check(r.off_E - r.off_rc >= (uint32_t)(2 * n), "counts fit", n, 0, 0);
    check(r.hb == r.jr - r.off_cm, "header bytes", n, 0, 0);
    for (const auto &o : kOpts) {
      const int nbuf = o[0] + o[1] + 1;
      for (const auto &f : kOpts) {
        const int nbuf_f = f[0] + f[1] + 1;
        for (int G = 1; G <= 8; ++G) {
          const moda::WarpSmem L =
              moda::warp_smem(n, m, m < 512 ? m : 512, nbuf, G, true, o[1], nbuf_f, f[1]);
          const size_t region = L.mbar - L.buf;
          check(L.buf % 16 == 0 && L.jr == r.jr, "buffer base and stride", n, nbuf, nbuf_f);
          check(region >= (size_t)nbuf * r.jr, "normal buffers fit", n, nbuf, nbuf_f);
          check(L.scr == r.jr && L.scr + 4 * (size_t)m <= L.hbuf, "scratch after the full record",
                n, nbuf, nbuf_f);
          check(L.hbuf % 16 == 0, "header buffers aligned", n, nbuf, nbuf_f);
          check(L.hbuf + (size_t)nbuf_f * r.hb <= region, "frozen layout fits", n, nbuf,
                nbuf_f);
          check(nbuf_f <= 30 && nbuf <= 30, "buffer indices below the sentinels", n, nbuf,
                nbuf_f);
          const int nb_max = nbuf > nbuf_f ? nbuf : nbuf_f;
          check(L.pfr >= nb_max && (L.pfr == 16 || L.pfr == 32), "record ring", n, nbuf,
                nbuf_f);
          const int w_max = o[1] > f[1] ? o[1] : f[1];
          check(L.cst == 8 * (w_max + 1), "count rows", n, nbuf, nbuf_f);
          check(L.mbar + 8 * (size_t)nb_max <= L.ring, "barriers fit", n, nbuf, nbuf_f);
          check(L.ring % 16 == 0 && L.aE % 16 == 0 && L.cnt % 16 == 0 && L.fld % 16 == 0 &&
                    L.team % 16 == 0,
                "team parts aligned", n, nbuf, nbuf_f);
          check(L.fld + 8 * (size_t)r.mp <= L.team, "fields fit", n, nbuf, nbuf_f);
          check(L.acc % 16 == 0 && L.rows % 16 == 0 && L.rc % 16 == 0 && L.pf % 16 == 0 &&
                    L.tbl % 16 == 0 && L.warp % 16 == 0,
                "warp parts aligned", n, nbuf, nbuf_f);
          check(L.total == L.team + (uint32_t)G * L.warp, "total", n, nbuf, nbuf_f);
          if (failures > 20) return 1;
        }
      }
    }
  }
  if (failures) return 1;
  std::printf("warp layouts ok\n");
  return 0;
}
