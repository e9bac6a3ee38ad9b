// The warp annealer: Alg. 3 of arXiv 2205.13399 (the multi-objective
// Digital Annealer, Sec. 3.3) for the bi-objective QAP with a team of G
// warps (G = 1 .. 8) per replica.  A persistent grid of teams pulls (run,
// replica) work items from a device list (largest runs first), so replicas
// of many instances of uneven n share the GPU in one launch; a team
// synchronises on a named barrier of its own, never on a block barrier.
// G = 1 suits launches with many more replicas than SMs (each warp a
// replica); larger G shortens one replica's iteration when replicas are
// few.
//
// State of a replica, the current point x of Alg. 3:
//   shared memory  its jump record: per bit the acceptance penalty
//                  a(p) = sum_k max(0, dE_k(p)) (strict, Eq. pacceptms) or
//                  min_k max(0, dE_k(p)) (lenient, Eq. pacceptml),
//                  saturated to uint32; the state words; the row and column
//                  counts R_i, C_u (each warp keeps its own copy of these);
//   global memory  its cost fields L_k(i,u) = sum_(j,v) Fs^k_ij d_uv x_jv
//                  (Fs^k = F^k + F^k^T), int32 pairs;
//   registers      E_1, E_2, |A| and the buffer bookkeeping, the same in
//                  every warp of the team.
// With h = R_i + C_u - 1 - 2 x_p and alpha_k = w_k / 2 (Eq. wqubom),
//   dE_k(p) = (1 - 2 x_p) (L_k(p) + w_k h)                         (Eq. cale),
// so a trial needs only a(p): bit p is accepted iff (double) a <=
// delta_t T[idx] (R7), decided by a <= lo_t or a > hi_t without a draw
// (R21).  Warp w of a team owns a contiguous range of 128-bit chunks; bit p
// of chunk c = p / 128 belongs to lane (p % 128) / 4, which owns bits
// 4g .. 4g + 3 of Philox group g = p / 4: one block per lane.
//
// A flip of bit (j, v) with s = +1 when it turns on adds s Fs^k_ij d_uv to
// every L_k(i, u) -- the outer product of flow row j and distance row v, so
// Q is never stored -- then recomputes every a(p) from L, the new counts
// and the new state.  Every archive slot keeps its jump and field records
// (the field cache); a jump to slot y takes y's jump record, prefetched by a
// bulk copy (TMA, mbarrier) `lookahead` iterations early when y is already
// known (the restart draw and |A| are), and y's field record in place.  A
// slot without records (beyond the cache) is rebuilt: M = X D, then
// L_k = Fs_k M.
#include <cstdint>
#include <type_traits>

#include "moda_device.cuh"
#include "moda_internal.h"

namespace moda {
namespace {

// Ring entry of one iteration: delta_t, its thresholds and the draws of the
// select, restart and exploit purposes.
struct WRing {
  double delta;
  int64_t lo, hi;
  uint32_t sel, rst, exp;
  float deltaf;  // fl32(delta), for the FP32 test of prefilter()
};
static_assert(sizeof(WRing) == 40, "ring entry layout");

// Named barrier `id` (1 .. 15) of `threads` threads; returns whether `v`
// held in any of them.
__device__ __forceinline__ bool team_sync_or(int id, int threads, bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(threads)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void team_sync(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

template <bool NARROW>
struct WarpAnnealer {
  using dE_t = typename std::conditional<NARROW, int32_t, int64_t>::type;

  // Penalty of a bit with Delta E (e1, e2), saturated to uint32.  In the
  // narrow variant each |dE_k| < 2^31, so the sum stays below 2^32 - 1.
  __device__ __forceinline__ static uint32_t penalty(dE_t e1, dE_t e2, bool lenient) {
    const dE_t u1 = e1 > 0 ? e1 : (dE_t)0, u2 = e2 > 0 ? e2 : (dE_t)0;
    if (NARROW) {
      return lenient ? (uint32_t)(u1 < u2 ? u1 : u2) : (uint32_t)u1 + (uint32_t)u2;
    } else {
      const int64_t a = lenient ? (int64_t)(u1 < u2 ? u1 : u2) : (int64_t)u1 + (int64_t)u2;
      return a >= 0xFFFFFFFFll ? 0xFFFFFFFFu : (uint32_t)a;
    }
  }
};

// The team's shape within its block.
struct Team {
  int G, wt, lane;     // warps per team, this warp's index in it, lane
  int bar;             // named barrier id (G > 1)
  unsigned char *ts;   // team shared memory
  unsigned char *ws0;  // warp 0's shared memory (warp w at ws0 + w * SL.warp)
};

// Runs replica `row` of run R on this team for all I_max iterations.
// `par` holds the phase parity of the team's mbarriers across items (the
// same in every warp).  Returns false when a bounded wait gave up (the
// error word is set).  FZ: the variant that carries the frozen layout
// (without it every test of `frozen` folds away).
template <bool NARROW, bool FZ>
__device__ bool team_run(const WarpRun &R, const int row, const Team &T, const WarpLaunch &Lc,
                         unsigned char *cache, uint32_t &par) {
  using WA = WarpAnnealer<NARROW>;
  using dE_t = typename WA::dE_t;
  const int lane = T.lane, G = T.G, wt = T.wt;
  const bool leader = wt == 0;
  // the warp that refills the ring and writes a flip's archive energies and
  // record header: the last, so that the leader (which starts the copies)
  // carries less of each iteration's serial work
  const bool scribe = wt == G - 1;
  const int n = R.n, m = R.m, W = R.W, s = R.s;
  const WarpRec rec = warp_rec(n, m);
  const int NC = rec.nc;
  // this warp's chunks [c0, c1): contiguous, so the team's accepted bits
  // in (warp, chunk, lane) order are in ascending bit order
  const int c0 = wt * NC / G, c1 = (wt + 1) * NC / G;
  const int cslots = R.cslots, se = R.se;
  const uint32_t rep = R.replica_base + (uint32_t)row;
  const uint32_t k0 = R.seed_lo, k1 = R.seed_hi;
  const uint32_t I_max = (uint32_t)R.I_max;
  const uint32_t nsched = (uint32_t)R.nsched;
  const int64_t w1l = R.w1, w2l = R.w2;
  const dE_t w1 = (dE_t)w1l, w2 = (dE_t)w2l;
  const bool lenient = R.accept != 0;
  const bool exploit = R.archive != 0;
  const uint32_t magic = R.magic;
  // prefetch distance and buffers of the current layout (the frozen layout
  // below has its own)
  int LA = Lc.lookahead, NB = Lc.nbuf;
  const WarpSmem &SL = Lc.sm;
  const double *const table = R.table;
  const float *const tablef = R.tablef;
  int64_t *const trace = R.trace;
  const int team_threads = 32 * G;
  auto sync = [&]() {
    if (G > 1) team_sync(T.bar, team_threads);
    else __syncwarp();
  };
  auto sync_or = [&](bool v) -> bool {
    if (G > 1) return team_sync_or(T.bar, team_threads, v);
    return __any_sync(kFull, v);
  };

  unsigned char *ts = T.ts;
  unsigned char *sbuf = ts + SL.buf;
  uint64_t *sbar = reinterpret_cast<uint64_t *>(ts + SL.mbar);
  WRing *ring = reinterpret_cast<WRing *>(ts + SL.ring);
  longlong2 *sAE = reinterpret_cast<longlong2 *>(ts + SL.aE);
  // accepted counts of the warps by round parity: [window position][warp],
  // then [warp] its first window position with an accepted bit (a warp may
  // write the next round's while another still reads this round's)
  int32_t *sCnt = reinterpret_cast<int32_t *>(ts + SL.cnt);
  // counts: [2 parities][window positions + 1][8 warps], SL.cst ints a parity
  const int cst = SL.cst;
  int64_t *sSum = reinterpret_cast<int64_t *>(ts + SL.cnt + 8 * cst + 16);  // [G][2] rebuild sums
  // explore: each warp's first dominated slot, [round parity][warp]
  int32_t *sScan = reinterpret_cast<int32_t *>(ts + SL.cnt + 8 * cst + 144);
  // the fields of the state the last flip reached, while Lc.sfields: flips
  // that follow flips read them here rather than from global memory
  int2 *const sF = reinterpret_cast<int2 *>(ts + SL.fld);
  const bool use_sf = Lc.sfields != 0;
  unsigned char *ws = T.ws0 + (size_t)wt * SL.warp;
  // this warp's prefetch bookkeeping (the same in every warp): sPf[tt & 15]
  // = {buffer or -1, slot, issuing iteration} of the copy for target
  // iteration tt; sWr[x & 15] = the slot iteration x wrote (-1: none)
  int4 *sPf = reinterpret_cast<int4 *>(ws + SL.pf);
  // per-target records and writes, a ring of SL.pfr iterations
  const uint32_t pfm = (uint32_t)SL.pfr - 1u;
  int32_t *sWr = reinterpret_cast<int32_t *>(ws + SL.pf + 16 * SL.pfr);
  uint4 *sAccW = reinterpret_cast<uint4 *>(ws + SL.acc);
  int32_t *sAccC = reinterpret_cast<int32_t *>(ws + SL.acc + 16 * (size_t)SL.nc_max);
  int32_t *sRow = reinterpret_cast<int32_t *>(ws + SL.rows);  // Fs1 row, Fs2 row, D row
  unsigned char *rcp = ws + SL.rc;  // this warp's row and column counts of the state
  // fl32(-ln u) of the acceptance draws of iteration `staged` for this
  // warp's (at most two) chunks, [chunk][lane][word], copied during the flip
  // before it: the draws do not depend on the state
  float *sTbl = reinterpret_cast<float *>(ws + SL.tbl);
  const bool can_stage = Lc.stage != 0 && c1 - c0 <= 2;
  uint32_t staged = 0;

  int64_t *gE = R.arch_E + (size_t)row * s * 2;
  uint32_t *gB = R.arch_bits + (size_t)row * s * W;
  unsigned char *gJR = cache;                                             // [cslots] jump records
  int2 *gLR = reinterpret_cast<int2 *>(cache + (size_t)cslots * rec.jr);  // [cslots][mp]
  int2 *gWork = gLR + (size_t)cslots * rec.mp;                            // [mp] working fields
  const int32_t *Fs1 = R.Fs1, *Fs2 = R.Fs2, *Dm = R.D;

  // Frozen layout (from iteration nsched on, when the launch has one): the
  // schedule no longer changes, so a jump record's candidate masks decide
  // which of its penalties can still be accepted and a copy brings only the
  // header.  The buffer region then holds one full record for the state a
  // flip or a rebuild reached (buffer kFull_b), a rebuild's scratch
  // (kScr_b) and Lc.nbuf_f header buffers.
  constexpr int kFull_b = 31, kScr_b = 30;
  const bool fz_on = FZ && Lc.nbuf_f > 0;
  bool frozen = false;
  auto base = [&](int b) -> unsigned char * {
    if (!frozen) return sbuf + (size_t)b * SL.jr;
    if (b == kFull_b) return sbuf;
    if (b == kScr_b) return sbuf + SL.scr;
    return sbuf + SL.hbuf + (size_t)b * rec.hb - rec.off_cm;  // header at base + off_cm
  };
  // penalties: only a full record (normal layout, or kFull_b / kScr_b)
  auto bA = [&](int b) { return reinterpret_cast<uint32_t *>(base(b)); };
  auto bCM = [&](int b) { return reinterpret_cast<const uint4 *>(base(b) + rec.off_cm); };
  auto bX = [&](int b) { return reinterpret_cast<uint32_t *>(base(b) + rec.off_xw); };
  auto bRC = [&](int b) { return base(b) + rec.off_rc; };
  auto bE = [&](int b) { return reinterpret_cast<int64_t *>(base(b) + rec.off_E); };
  // a buffer of header only (its penalties are read from the record)
  auto hdr_only = [&](int b) { return frozen && b != kFull_b; };
  // the frozen schedule's hi: masks mark a(p) <= it (saturated penalties
  // too when it reaches 2^32 - 1)
  const int64_t hiF = R.sch_hi[nsched - 1];
  const uint32_t hiF32 = hiF < 0xFFFFFFFFll ? (uint32_t)hiF : 0xFFFFFFFFu;
  auto divn = [&](int p) { return (int)__umulhi((uint32_t)p, magic); };

  // Iterations first .. first + 31 into the ring (one warp): schedule
  // entry (Alg. 3's cooling, the last entry held once delta reaches
  // delta_f) and the draws (0, q, replica, tag) of the select, restart and
  // exploit purposes.
  auto fill = [&](uint32_t first) {
    const uint32_t q = first + (uint32_t)lane;
    const uint32_t sn = (q <= nsched ? q : nsched) - 1u;
    WRing e;
    e.delta = R.sch_delta[sn];
    e.deltaf = __double2float_rn(e.delta);
    e.lo = R.sch_lo[sn];
    e.hi = R.sch_hi[sn];
    uint32_t c[4] = {0u, q, rep, kTagSelect};
    philox10(c, k0, k1);
    e.sel = c[0];
    uint32_t d[4] = {0u, q, rep, kTagRestart};
    philox10(d, k0, k1);
    e.rst = d[0];
    e.exp = 0u;
    if (exploit) {
      uint32_t x[4] = {0u, q, rep, kTagExploit};
      philox10(x, k0, k1);
      e.exp = x[0];
    }
    ring[q % kWarpRing] = e;
  };

  // Fields and penalties of the state in buffer b from scratch (Alg. 3's
  // initial state, or a jump to a slot without records), by the whole
  // team: the row and column counts into the buffer and every warp's copy,
  // M = X D in the a-array of buffer sc, then L_k(i,u) = sum_j Fs^k_ij M_ju
  // into gL and a(p) into buffer b.  Returns sum over set bits of L_1 and
  // of L_2 (2 c_k) and g (Eq. gqap), team totals.  Ends on a team barrier.
  auto rebuild = [&](int b, int sc, int2 *gL, int64_t &t1, int64_t &t2, int64_t &gp) {
    const uint32_t *xw = bX(b);
    unsigned char *rc = bRC(b);
    const int tid = wt * 32 + lane;
    for (int i = tid; i < n; i += team_threads) {
      int cr = 0, cc = 0;
      for (int u = 0; u < n; ++u) {
        const int p = i * n + u, q = u * n + i;
        cr += (int)((xw[p >> 5] >> (p & 31)) & 1u);
        cc += (int)((xw[q >> 5] >> (q & 31)) & 1u);
      }
      rc[i] = (unsigned char)cr;
      rc[n + i] = (unsigned char)cc;
    }
    int32_t *M = reinterpret_cast<int32_t *>(bA(sc));
    for (int e = tid; e < n * n; e += team_threads) {
      const int j = divn(e), u = e - j * n;
      int32_t acc = 0;
      for (int v = 0; v < n; ++v) {
        const int p = j * n + v;
        if ((xw[p >> 5] >> (p & 31)) & 1u) acc += __ldg(&Dm[v * n + u]);
      }
      M[e] = acc;
    }
    sync();
    for (int e = lane; e < 2 * n; e += 32) rcp[e] = rc[e];
    __syncwarp();
    uint32_t *ab = bA(b);
    t1 = 0;
    t2 = 0;
    for (int p = c0 * 128 + lane; p < c1 * 128; p += 32) {
      uint32_t a = 0xFFFFFFFFu;
      int2 L = make_int2(0, 0);
      if (p < m) {
        const int i = divn(p), u = p - i * n;
        int32_t a1 = 0, a2 = 0;
        for (int j = 0; j < n; ++j) {
          const int32_t mm = M[j * n + u];
          a1 += __ldg(&Fs1[i * n + j]) * mm;
          a2 += __ldg(&Fs2[i * n + j]) * mm;
        }
        L = make_int2(a1, a2);
        const int xv = (int)((xw[p >> 5] >> (p & 31)) & 1u);
        const dE_t g = (dE_t)(1 - 2 * xv);
        const dE_t h = (dE_t)rcp[i] + (dE_t)rcp[n + u] - 1 - 2 * xv;
        a = WA::penalty(g * ((dE_t)a1 + w1 * h), g * ((dE_t)a2 + w2 * h), lenient);
        if (xv) {
          t1 += a1;
          t2 += a2;
        }
      }
      gL[p] = L;
      ab[p] = a;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      t1 += __shfl_xor_sync(kFull, t1, o);
      t2 += __shfl_xor_sync(kFull, t2, o);
    }
    if (lane == 0) {
      sSum[2 * wt] = t1;
      sSum[2 * wt + 1] = t2;
    }
    sync();
    t1 = 0;
    t2 = 0;
    for (int w = 0; w < G; ++w) {
      t1 += sSum[2 * w];
      t2 += sSum[2 * w + 1];
    }
    gp = 0;
    for (int i = 0; i < n; ++i) {
      const int64_t dr = 1 - (int64_t)rcp[i], dc = 1 - (int64_t)rcp[n + i];
      gp += dr * dr + dc * dc;
    }
    sync();  // the scratch and the sums may be reused after this
  };

  // Exact penalty of bit p of the state in buffer b with fields gL (only
  // for a saturated a(p) in the int64 variant).
  auto exact_penalty = [&](int b, const int2 *gL, const unsigned char *rcq, int p) -> int64_t {
    const int2 L = gL[p];
    const int i = divn(p), u = p - i * n;
    const uint32_t *xw = bX(b);
    const int xv = (int)((xw[p >> 5] >> (p & 31)) & 1u);
    const int64_t g = 1 - 2 * xv, h = (int64_t)rcq[i] + rcq[n + u] - 1 - 2 * xv;
    const int64_t e1 = g * ((int64_t)L.x + w1l * h), e2 = g * ((int64_t)L.y + w2l * h);
    const int64_t u1 = e1 > 0 ? e1 : 0, u2 = e2 > 0 ? e2 : 0;
    return lenient ? (u1 < u2 ? u1 : u2) : u1 + u2;
  };

  bool fail = false;
  // Copies into buffer b complete phases of mbarrier b in turn; every warp
  // tracks the parity of the next phase.  A copy whose data the team uses
  // is waited for by every warp (take_buf).  One that is given up is
  // waited for by the thread that fills that buffer again, before it does
  // (the stale wait of the prefetch issue; retire_buf when the item ends),
  // and a barrier separates that wait from any take of the new copy; where
  // the new copy is taken at once (a jump to a member without a prefetched
  // record), every warp waits for the old copy and then for a barrier.  So
  // no warp polls a phase whose predecessor is still open, nor one that the
  // barrier may already have left twice: after a take the buffer is
  // refilled only one barrier later.
  auto take_buf = [&](int b) {
    const bool ok = mbar_wait(&sbar[b], (par >> b) & 1u);
    if (!__all_sync(kFull, ok)) fail = true;
    par ^= 1u << b;
  };
  auto retire_buf = [&](int b) {
    if (leader) {
      const bool ok = mbar_wait(&sbar[b], (par >> b) & 1u);
      if (!__all_sync(kFull, ok)) fail = true;
    }
    par ^= 1u << b;
  };
  // the leader's lane 0 starts the copy of slot y's jump record into b
  auto copy_record = [&](int b, int y) {
    if (leader && lane == 0) {
      fence_proxy_async_shared();
      if (frozen) {
        mbar_expect_tx(&sbar[b], rec.hb);
        bulk_g2s(base(b) + rec.off_cm, gJR + (size_t)y * rec.jr + rec.off_cm, rec.hb, &sbar[b]);
      } else {
        mbar_expect_tx(&sbar[b], rec.jr);
        bulk_g2s(base(b), gJR + (size_t)y * rec.jr, rec.jr, &sbar[b]);
      }
    }
  };

  // ---- initial state (Alg. 3: "a random binary solution", R10) ----------
  // Chunk c's 128 bits are the four words of Philox block (c, 0, replica,
  // init): state word 4c + w is word w.
  int cur = 0;
  // the archive slot whose record the state's buffer holds (-1: the buffer
  // holds a full record), for a header-only buffer's penalties
  int cur_slot = -1;
  {
    uint32_t *x0 = bX(0);
    for (int c = c0 + lane; c < c1; c += 32) {
      uint32_t b[4] = {(uint32_t)c, 0u, rep, kTagInit};
      philox10(b, k0, k1);
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int lo = 32 * (4 * c + w);
        uint32_t v = b[w];
        if (lo >= m) v = 0u;
        else if (lo + 32 > m) v &= (1u << (m - lo)) - 1u;
        x0[4 * c + w] = v;
      }
    }
    if (lane < SL.pfr) {
      sPf[lane] = make_int4(-1, 0, 0, 0);
      sWr[lane] = -1;
    }
    if (leader) {
      for (int q2 = lane; q2 < 2 * cst; q2 += 32)
        sCnt[q2] = 0;  // counts of warps beyond G stay 0
      fill(1);
      fill(33);
    }
    sync();
  }
  int64_t E1, E2;
  {
    int64_t t1, t2, gp;
    rebuild(0, 1, gWork, t1, t2, gp);
    E1 = t1 / 2 + w1l * (gp / 2);
    E2 = t2 / 2 + w2l * (gp / 2);
  }
  const int2 *curL = gWork;
  int acount = 0;
  // free buffers (bit b), copies in flight (bit b)
  uint32_t freeb = ((1u << NB) - 1u) & ~1u, pend = 0u;
  int flip_streak = 0;
  uint32_t nflip = 0, njump = 0, nempty = 0, npref = 0, ndirect = 0, nrebuild = 0;
  // the last iteration that wrote an archive slot; after a jump to a
  // cached slot this warp's counts are refreshed from the buffer only when
  // needed (rc_stale)
  uint32_t last_wr_t = 0;
  bool rc_stale = false;
  // this thread wrote records that later bulk copies (async proxy) read and
  // has not yet ordered them by fence.proxy.async: it does so at the start
  // of the next round, before any copy of the round is issued (a slot
  // written in the previous iteration is not copied until a barrier later)
  bool unfenced = false;

  // Rounds of up to KW iterations.  While the replica only jumps, the
  // states of the next iterations are known in advance -- iteration tau
  // jumps to the member its restart draw picks among |A| -- and their jump
  // records are prefetched, so the trials of a window of iterations t ..
  // t + K - 1 run together, iteration t + k on the member iteration
  // t + k - 1 would land on.  Every bit of every iteration is tested.  The
  // first iteration of the window that accepts a bit flips (the window's
  // earlier iterations were jumps, as assumed), and the trials after it
  // are discarded; a window without an accepted bit commits K jumps.
  int KW = Lc.window;
  uint32_t filled = 64;  // the ring holds the iterations up to `filled`
  // Every target iteration tau gets one record sPf[tau & 15], a copy or
  // none, written once, in the round that first reaches it; records up to
  // issued_to are written (none for 1 .. LA).
  uint32_t issued_to = (uint32_t)LA;
  uint32_t t = 1, rnd = 0;
  while (t <= I_max) {
    if (scribe)  // entries read before this round's barrier were written in earlier rounds
      while (filled < t + 48u) {
        fill(filled + 1u);
        filled += 32u;
      }
    if (fz_on && !frozen && t >= nsched) {
      // ---- the schedule is frozen from iteration t on: the copies in
      // flight land, the state's record moves to kFull_b, and jumps bring
      // headers into the frozen layout's buffers from now on
      bool ok = true;
      if ((pend >> lane) & 1u) ok = mbar_wait(&sbar[lane], (par >> lane) & 1u);
      if (!__all_sync(kFull, ok)) fail = true;
      par ^= pend;
      pend = 0u;
      sync();  // every warp is done with the old buffers
      if (cur != 0) {  // kFull_b is where buffer 0 was
        const int4 *src = reinterpret_cast<const int4 *>(sbuf + (size_t)cur * SL.jr);
        int4 *dst = reinterpret_cast<int4 *>(sbuf);
        for (int i = wt * 32 + lane; i < (int)(rec.jr / 16); i += team_threads) dst[i] = src[i];
      }
      frozen = true;
      cur = kFull_b;
      cur_slot = -1;
      LA = Lc.lookahead_f;
      KW = Lc.window_f;
      NB = Lc.nbuf_f;
      freeb = (1u << NB) - 1u;
      if (lane < SL.pfr) sPf[lane] = make_int4(-1, 0, 0, 0);
      __syncwarp();
      issued_to = t - 1u;
      sync();  // the record has moved before anyone reads it
    }
    if (unfenced) {
      fence_proxy_async_global();
      unfenced = false;
    }
    const int K = (KW > 1 && acount > 0 && flip_streak == 0)
                      ? (int)min((uint32_t)KW, I_max - t + 1u)
                      : 1;

    // ---- prefetch: the jump records of the members jumps up to t + K - 1
    // + LA would land on (their draws and |A| are known), unless the
    // replica is in a run of flips.  At most LA + K + 1 buffers are held:
    // the state's and those of targets t .. t + K - 1 + LA.  Lane k
    // handles target issued_to + 1 + k; every warp keeps the same books,
    // and warp k % G starts lane k's copy.
    if (LA > 0 && !(acount > 0 && flip_streak < 3)) {
      // no copies now: the targets get empty records
      const int nI = (int)(t + (uint32_t)(K - 1 + LA)) - (int)issued_to;
      if (lane < nI) sPf[(issued_to + 1u + (uint32_t)lane) & pfm] = make_int4(-1, 0, (int)t, 0);
      if (nI > 0) issued_to += (uint32_t)nI;
      __syncwarp();
    } else if (LA > 0) {
      // targets not yet given a record (none when an earlier, longer
      // window already reached t + K - 1 + LA)
      const int nI = (int)(t + (uint32_t)(K - 1 + LA)) - (int)issued_to;
      const uint32_t tt = issued_to + 1u + (uint32_t)lane;
      int sp = 0;
      bool want = false;
      if (lane < nI && acount > 0 && flip_streak < 3 && tt <= I_max) {
        sp = pick(ring[tt % kWarpRing].rst, acount);
        // a slot written in the previous iteration is left alone: warps
        // still writing it are ordered before the copy only by the next
        // barrier
        want = sp < cslots && sWr[(t - 1u) & pfm] != sp;
      }
      const uint32_t wm = __ballot_sync(kFull, want);
      // the r-th copy takes the r-th free buffer (there are enough: at
      // most NB - 1 - (issued_to - t + 1) >= nI are held)
      const int rank = __popc(wm & ((1u << lane) - 1u));
      int b = want ? nth_set_bit(freeb, rank) : -1;
      if (b >= NB || (b >= 0 && !((freeb >> b) & 1u))) {  // never: the books are kept so
        fail = true;
        b = -1;
      }
      const uint32_t bm = __reduce_or_sync(kFull, b >= 0 ? 1u << b : 0u);  // buffers taken now
      freeb &= ~bm;
      const uint32_t stale = pend & bm;  // unused earlier copies still land there
      // lane k's copy is started by warp k % G (the warps keep the same
      // books), which first waits for an unused earlier copy into its
      // buffer itself, so that the two cannot overlap
      const bool issuer = lane % G == wt;
      if (stale) {
        bool ok = true;
        if (issuer && b >= 0 && ((stale >> b) & 1u)) ok = mbar_wait(&sbar[b], (par >> b) & 1u);
        if (!__all_sync(kFull, ok)) fail = true;
        par ^= stale;
        pend &= ~stale;
      }
      if (issuer && b >= 0) {
        fence_proxy_async_shared();
        if (frozen) {  // the header: masks, state, counts, energies
          mbar_expect_tx(&sbar[b], rec.hb);
          bulk_g2s(base(b) + rec.off_cm, gJR + (size_t)sp * rec.jr + rec.off_cm, rec.hb,
                   &sbar[b]);
        } else {
          mbar_expect_tx(&sbar[b], rec.jr);
          bulk_g2s(base(b), gJR + (size_t)sp * rec.jr, rec.jr, &sbar[b]);
        }
      }
      pend |= bm;
      if (lane < nI) sPf[tt & pfm] = make_int4(b, b >= 0 ? sp : 0, (int)t, 0);
      if (nI > 0) issued_to += (uint32_t)nI;
      __syncwarp();
    }
    // The copy for target iteration tau is usable if it began for the slot
    // tau's draw picks now and no iteration before `lim` rewrote that slot
    // since (the iterations of this window write nothing before a flip).
    auto usable = [&](uint32_t tau, int slot, uint32_t lim) {
      const int4 pr = sPf[tau & pfm];
      bool ok = pr.x >= 0 && pr.y == slot;
      if (ok && last_wr_t >= (uint32_t)pr.z)
        for (uint32_t xi = (uint32_t)pr.z; xi < lim; ++xi)
          if (sWr[xi & pfm] == slot) ok = false;
      return ok;
    };
    // the window: iteration t + k (k >= 1) tries the member iteration
    // t + k - 1 would jump to, if its record is here (lane k - 1 checks)
    int Keff = 1;
    if (K > 1) {
      bool u = false;
      if (lane < K - 1) {
        const uint32_t tau = t + (uint32_t)lane;
        u = usable(tau, pick(ring[tau % kWarpRing].rst, acount), t);
      }
      const uint32_t um = __ballot_sync(kFull, u);
      Keff = 1 + __ffs(~um) - 1;  // leading usable targets
      if (Keff > K) Keff = K;
      // those records, for every warp: lane k waits for target t + k
      bool ok = true;
      int tb = -1;
      if (lane < Keff - 1) {
        tb = sPf[(t + (uint32_t)lane) & pfm].x;
        ok = mbar_wait(&sbar[tb], (par >> tb) & 1u);
      }
      if (!__all_sync(kFull, ok)) fail = true;
      const uint32_t tm = __reduce_or_sync(kFull, tb >= 0 ? 1u << tb : 0u);
      par ^= tm;
      pend &= ~tm;
    }

    // ---- the parallel trials (Eq. pacceptms / pacceptml) of the window,
    // this warp's chunks, up to its first accepted bit
    int32_t *cntr = sCnt + cst * (int)(rnd & 1u);  // [k][warp] counts, then [warp] first k
    int first_w = Keff, nl = 0;
    // A run of flips (one iteration, not staged): nearly every chunk
    // needs draws, so the draws and -ln(u) loads of two chunks are in
    // flight together, with no branch on the chunk's candidates.
    const bool hot = Keff == 1 && flip_streak > 0 && staged != t;
    // The iteration after a flip whose -ln(u) values were staged (it is
    // tried alone): the same, from the staged values.
    const bool hot_st = staged == t;
    // Otherwise first every bit of the window against its hi_t: usually
    // none can be accepted, and the window's trials end here.
    bool cand = hot || hot_st;
    if (!cand) {
      // lane k holds the buffer and threshold of window position k
      int sbl = cur;
      uint32_t hl = 0u;
      if (lane < Keff) {
        if (lane > 0) sbl = sPf[(t + (uint32_t)(lane - 1)) & pfm].x;
        const int64_t hk = ring[(t + (uint32_t)lane) % kWarpRing].hi;
        hl = hk < 0xFFFFFFFFll ? (uint32_t)hk : 0xFFFFFFFFu;
      }
      if (c1 - c0 <= 2) {
        // few chunks: every position's loads of a chunk issue together
        // (fully unrolled and predicated)
        for (int c = c0; c < c1; ++c) {
#pragma unroll
          for (int k = 0; k < kWarpMaxLA + 1; ++k) {
            const int sbk = __shfl_sync(kFull, sbl, k);
            const uint32_t h32 = __shfl_sync(kFull, hl, k);
            if (k < Keff) {
              if (hdr_only(sbk)) {  // the chunk's candidate masks
                const uint4 cm = bCM(sbk)[c];
                cand |= (cm.x | cm.y | cm.z | cm.w) != 0u;
              } else {
                const uint4 a4 = reinterpret_cast<const uint4 *>(bA(sbk))[c * 32 + lane];
                cand |= min(min(a4.x, a4.y), min(a4.z, a4.w)) <= h32;
              }
            }
          }
        }
      } else {
#pragma unroll
        for (int k = 0; k < kWarpMaxLA + 1; ++k) {
          if (k >= Keff) break;  // Keff is the same in every lane
          const int sbk = __shfl_sync(kFull, sbl, k);
          const uint32_t h32 = __shfl_sync(kFull, hl, k);
          if (hdr_only(sbk)) {  // the chunks' candidate masks
            const uint4 *cmp = bCM(sbk);
#pragma unroll 4
            for (int c = c0; c < c1; ++c) {
              const uint4 cm = cmp[c];
              cand |= (cm.x | cm.y | cm.z | cm.w) != 0u;
            }
          } else {
            const uint4 *ap = reinterpret_cast<const uint4 *>(bA(sbk));
#pragma unroll 4
            for (int c = c0; c < c1; ++c) {
              const uint4 a4 = ap[c * 32 + lane];
              cand |= min(min(a4.x, a4.y), min(a4.z, a4.w)) <= h32;
            }
          }
        }
      }
    }
    if (hot) {
      const WRing e = ring[t % kWarpRing];
      const double delta = e.delta;
      const float df = e.deltaf;
      const int64_t lo = e.lo, hi = e.hi;
      const uint32_t hi32 = hi < 0xFFFFFFFFll ? (uint32_t)hi : 0xFFFFFFFFu;
      const uint32_t lo32 = lo < 0xFFFFFFFFll ? (uint32_t)lo : 0xFFFFFFFFu;
      const unsigned char *rck = rc_stale ? bRC(cur) : rcp;
      const uint4 *a4p = reinterpret_cast<const uint4 *>(bA(cur));
      int cnt_w = 0;
#pragma unroll 2
      for (int c = c0; c < c1; ++c) {
        const uint4 a4 = a4p[c * 32 + lane];
        uint32_t d[4] = {(uint32_t)(c * 32 + lane), t, rep, kTagAccept};
        philox10(d, k0, k1);
        float tv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) tv[j] = __ldg(&tablef[d[j] >> 16]);
        const int p0 = c * 128 + lane * 4;
        const uint32_t av[4] = {a4.x, a4.y, a4.z, a4.w};
        bool acc[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[j] = false;
          if (p0 + j < m && av[j] <= hi32) {
            if (NARROW) {
              // a < 2^32 - 1: the clamped thresholds decide exactly
              const int r = av[j] <= lo32 ? 1 : prefilter(__uint2float_rn(av[j]), df, tv[j]);
              acc[j] = r > 0 ||
                       (r < 0 && (double)av[j] <= __dmul_rn(delta, __ldg(&table[d[j] >> 16])));
            } else {
              const int64_t ax =
                  av[j] == 0xFFFFFFFFu ? exact_penalty(cur, curL, rck, p0 + j) : (int64_t)av[j];
              const int r = ax <= lo ? 1 : ax > hi ? 0 : prefilter(penalty_f32(ax), df, tv[j]);
              acc[j] = r > 0 || (r < 0 && (double)ax <= __dmul_rn(delta, __ldg(&table[d[j] >> 16])));
            }
          }
        }
        const uint32_t b0 = __ballot_sync(kFull, acc[0]), b1 = __ballot_sync(kFull, acc[1]),
                       b2 = __ballot_sync(kFull, acc[2]), b3 = __ballot_sync(kFull, acc[3]);
        const int cnt = __popc(b0) + __popc(b1) + __popc(b2) + __popc(b3);
        if (cnt > 0) {
          if (lane == 0) {
            sAccW[nl] = make_uint4(b0, b1, b2, b3);
            sAccC[nl] = c;
          }
          ++nl;
          cnt_w += cnt;
        }
      }
      if (lane == 0) cntr[wt] = cnt_w;
      if (cnt_w > 0) first_w = 0;
    } else if (hot_st) {
      const WRing e = ring[t % kWarpRing];
      const double delta = e.delta;
      const float df = e.deltaf;
      const int64_t lo = e.lo, hi = e.hi;
      const uint32_t hi32 = hi < 0xFFFFFFFFll ? (uint32_t)hi : 0xFFFFFFFFu;
      const uint32_t lo32 = lo < 0xFFFFFFFFll ? (uint32_t)lo : 0xFFFFFFFFu;
      const unsigned char *rck = rc_stale ? bRC(cur) : rcp;
      const uint4 *a4p = reinterpret_cast<const uint4 *>(bA(cur));
      const float4 *t4p = reinterpret_cast<const float4 *>(sTbl);
      cp_async_wait_all();  // the staged values (copied during the flip)
      __syncwarp();
      int cnt_w = 0;
      for (int c = c0; c < c1; ++c) {
        const uint4 a4 = a4p[c * 32 + lane];
        const float4 t4 = t4p[(c - c0) * 32 + lane];
        const int p0 = c * 128 + lane * 4;
        const uint32_t av[4] = {a4.x, a4.y, a4.z, a4.w};
        const float tv[4] = {t4.x, t4.y, t4.z, t4.w};
        bool acc[4], amb[4];
        int64_t ai[4];
        bool anyamb = false;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[j] = false;
          amb[j] = false;
          ai[j] = (int64_t)av[j];
          if (p0 + j < m && av[j] <= hi32) {
            int r;
            if (NARROW) {
              // a < 2^32 - 1: the clamped thresholds decide exactly
              r = av[j] <= lo32 ? 1 : prefilter(__uint2float_rn(av[j]), df, tv[j]);
            } else {
              if (av[j] == 0xFFFFFFFFu) ai[j] = exact_penalty(cur, curL, rck, p0 + j);
              r = ai[j] <= lo ? 1 : ai[j] > hi ? 0 : prefilter(penalty_f32(ai[j]), df, tv[j]);
            }
            acc[j] = r > 0;
            amb[j] = r < 0;
            anyamb |= amb[j];
          }
        }
        if (__any_sync(kFull, anyamb)) {  // the double test near the boundary
          uint32_t d[4] = {(uint32_t)(c * 32 + lane), t, rep, kTagAccept};
          philox10(d, k0, k1);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (amb[j]) acc[j] = (double)ai[j] <= __dmul_rn(delta, __ldg(&table[d[j] >> 16]));
        }
        const uint32_t b0 = __ballot_sync(kFull, acc[0]), b1 = __ballot_sync(kFull, acc[1]),
                       b2 = __ballot_sync(kFull, acc[2]), b3 = __ballot_sync(kFull, acc[3]);
        const int cnt = __popc(b0) + __popc(b1) + __popc(b2) + __popc(b3);
        if (cnt > 0) {
          if (lane == 0) {
            sAccW[nl] = make_uint4(b0, b1, b2, b3);
            sAccC[nl] = c;
          }
          ++nl;
          cnt_w += cnt;
        }
      }
      if (lane == 0) cntr[wt] = cnt_w;
      if (cnt_w > 0) first_w = 0;
    } else if (!__any_sync(kFull, cand)) {
      if (lane < Keff) cntr[8 * lane + wt] = 0;
    } else
    for (int k = 0; k < Keff; ++k) {
      const uint32_t tk = t + (uint32_t)k;
      const WRing e = ring[tk % kWarpRing];
      const double delta = e.delta;
      const float df = e.deltaf;
      const int64_t lo = e.lo, hi = e.hi;
      const uint32_t hi32 = hi < 0xFFFFFFFFll ? (uint32_t)hi : 0xFFFFFFFFu;
      const uint32_t lo32 = lo < 0xFFFFFFFFll ? (uint32_t)lo : 0xFFFFFFFFu;
      int sb = cur, slot_k = cur_slot;
      const int2 *Lk = curL;
      const unsigned char *rck = rc_stale ? bRC(cur) : rcp;
      if (k > 0) {
        const int4 pr = sPf[(tk - 1u) & pfm];
        sb = pr.x;
        slot_k = pr.y;
        Lk = gLR + (size_t)pr.y * rec.mp;
        rck = bRC(sb);
      }
      // a header-only buffer: chunks with a candidate read their penalties
      // from the slot's record
      const bool ho = hdr_only(sb);
      const uint4 *a4p = ho ? reinterpret_cast<const uint4 *>(gJR + (size_t)slot_k * rec.jr)
                            : reinterpret_cast<const uint4 *>(bA(sb));
      int cnt_w = 0;
#pragma unroll 4
      for (int c = c0; c < c1; ++c) {
        if (ho) {
          const uint4 cm = bCM(sb)[c];
          if ((cm.x | cm.y | cm.z | cm.w) == 0u) continue;  // no bit of the chunk can be accepted
        }
        const uint4 a4 = a4p[c * 32 + lane];
        const uint32_t amin = min(min(a4.x, a4.y), min(a4.z, a4.w));
        if (__any_sync(kFull, amin <= hi32)) {
          // some bit of the chunk may be accepted: exact decisions
          const int p0 = c * 128 + lane * 4;
          const uint32_t av[4] = {a4.x, a4.y, a4.z, a4.w};
          bool acc[4], need[4];
          int64_t ai[4];
          bool anyneed = false;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[j] = false;
            need[j] = false;
            ai[j] = 0;
            if (p0 + j < m && av[j] <= hi32) {
              if (NARROW) {
                // a < 2^32 - 1: the clamped thresholds decide exactly
                if (av[j] <= lo32)
                  acc[j] = true;
                else
                  need[j] = true;
                ai[j] = (int64_t)av[j];
              } else {
                const int64_t ax =
                    av[j] == 0xFFFFFFFFu ? exact_penalty(sb, Lk, rck, p0 + j) : (int64_t)av[j];
                if (ax <= lo)
                  acc[j] = true;
                else if (ax <= hi)
                  need[j] = true;
                ai[j] = ax;
              }
            }
            anyneed |= need[j];
          }
          if (__any_sync(kFull, anyneed)) {
            // a in (lo, hi]: the draw decides (R7, R21); group 32c + lane
            bool amb[4];
            bool anyamb = false;
            uint32_t d[4] = {(uint32_t)(c * 32 + lane), tk, rep, kTagAccept};
            philox10(d, k0, k1);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              amb[j] = false;
              if (need[j]) {
                const float tf = __ldg(&tablef[d[j] >> 16]);
                const float af = NARROW ? __uint2float_rn((uint32_t)ai[j]) : penalty_f32(ai[j]);
                const int r = prefilter(af, df, tf);
                acc[j] = r > 0;
                amb[j] = r < 0;
                anyamb |= amb[j];
              }
            }
            if (__any_sync(kFull, anyamb)) {  // the double test near the boundary
#pragma unroll
              for (int j = 0; j < 4; ++j)
                if (amb[j]) acc[j] = (double)ai[j] <= __dmul_rn(delta, __ldg(&table[d[j] >> 16]));
            }
          }
          const uint32_t b0 = __ballot_sync(kFull, acc[0]), b1 = __ballot_sync(kFull, acc[1]),
                         b2 = __ballot_sync(kFull, acc[2]), b3 = __ballot_sync(kFull, acc[3]);
          const int cnt = __popc(b0) + __popc(b1) + __popc(b2) + __popc(b3);
          if (cnt > 0) {
            if (lane == 0) {
              sAccW[nl] = make_uint4(b0, b1, b2, b3);
              sAccC[nl] = c;
            }
            ++nl;
            cnt_w += cnt;
          }
        }
      }
      if (lane == 0) cntr[8 * k + wt] = cnt_w;
      if (cnt_w > 0) {
        first_w = k;
        break;
      }
    }
    if (lane == 0) cntr[cst - 8 + wt] = first_w;
    // every warp's counts, and whether any warp gave up a wait
    if (sync_or(fail)) {
      fail = true;
      break;
    }
    int kstar = Keff;  // the window's first iteration with an accepted bit
    for (int w = 0; w < G; ++w) kstar = min(kstar, (int)cntr[cst - 8 + w]);
    ++rnd;

    // ---- iterations t .. t + kstar - 1 jump (Alg. 3), or escape with an
    // empty archive (R12)
    if (kstar > 0) {
      if (lane < kstar) sWr[(t + (uint32_t)lane) & pfm] = -1;
      __syncwarp();
      if (acount == 0) {  // K = 1: one iteration
        const int4 pr = LA > 0 ? sPf[t & pfm] : make_int4(-1, 0, 0, 0);
        if (pr.x >= 0) freeb |= 1u << pr.x;
        ++nempty;
        if (trace != nullptr && leader && lane == 0) {
          int64_t *tr = trace + ((size_t)row * (size_t)I_max + (size_t)(t - 1)) * 3;
          tr[0] = E1;
          tr[1] = E2;
          tr[2] = INT64_MIN;
        }
      } else {
        // jumps to targets t .. t + ns - 1 land on records the window
        // took: the state passes through them and keeps the last
        const int ns = min(kstar, Keff - 1);
        if (trace != nullptr && leader && lane == 0)
          for (int k = 0; k < ns; ++k) {
            const int4 pr = sPf[(t + (uint32_t)k) & pfm];
            const int64_t *be = bE(pr.x);
            int64_t *tr = trace + ((size_t)row * (size_t)I_max + (size_t)(t + k - 1)) * 3;
            tr[0] = be[0];
            tr[1] = be[1];
            tr[2] = -1 - (int64_t)pr.y;
          }
        // (the records read for the trace are given up just below, and a
        // faster warp may refill them in its next round: the trace is
        // written first)
        if (trace != nullptr && ns > 0) sync();
        if (ns > 0) {
          const int pb = lane + 1 < ns ? sPf[(t + (uint32_t)lane) & pfm].x : -1;
          freeb |= __reduce_or_sync(kFull, pb >= 0 ? 1u << pb : 0u);  // passed through
          if (cur != kFull_b) freeb |= 1u << cur;
          const int4 pr = sPf[(t + (uint32_t)(ns - 1)) & pfm];
          cur = pr.x;
          cur_slot = pr.y;
          curL = gLR + (size_t)pr.y * rec.mp;
          const int64_t *be = bE(cur);
          E1 = be[0];
          E2 = be[1];
          rc_stale = true;
          npref += (uint32_t)ns;
          njump += (uint32_t)ns;
        }
        if (kstar > ns) {
          // the window's last iteration jumps to a member no trial holds
          const uint32_t tk = t + (uint32_t)(kstar - 1);
          const int slot = pick(ring[tk % kWarpRing].rst, acount);
          const int4 pr = LA > 0 ? sPf[tk & pfm] : make_int4(-1, 0, 0, 0);
          int nbuf;
          if (LA > 0 && usable(tk, slot, tk)) {
            nbuf = pr.x;
            take_buf(nbuf);
            pend &= ~(1u << nbuf);
            ++npref;
          } else {
            if (pr.x >= 0) freeb |= 1u << pr.x;
            if (frozen && slot >= cslots) {
              nbuf = kFull_b;  // a rebuild needs a full record
            } else {
              nbuf = __ffs(freeb) - 1;
              freeb &= ~(1u << nbuf);
              if ((pend >> nbuf) & 1u) {
                // an unused earlier copy still lands there: every warp
                // waits for it and the barrier orders that before the new
                // copy, which every warp then waits for in turn (a warp
                // must not poll the new copy's phase while the old one is
                // still open)
                take_buf(nbuf);
                pend &= ~(1u << nbuf);
                sync();
              }
            }
            if (slot < cslots) {
              copy_record(nbuf, slot);
              take_buf(nbuf);
            } else {
              // no records for this slot: rebuild from its state (the old
              // state's buffer is the scratch; kScr_b when frozen)
              uint32_t *xn = bX(nbuf);
              for (int q2 = 4 * c0 + lane; q2 < 4 * c1; q2 += 32)
                xn[q2] = q2 < W ? gB[(size_t)slot * W + q2] : 0u;
              sync();
              int64_t t1, t2, gp;
              rebuild(nbuf, frozen ? kScr_b : cur, gWork, t1, t2, gp);  // also this warp's counts
              ++nrebuild;
            }
            ++ndirect;
          }
          if (cur != kFull_b) freeb |= 1u << cur;
          cur = nbuf;
          cur_slot = slot < cslots ? slot : -1;
          if (slot < cslots) {
            curL = gLR + (size_t)slot * rec.mp;
            const int64_t *be = bE(cur);
            E1 = be[0];
            E2 = be[1];
            rc_stale = true;
          } else {
            curL = gWork;
            E1 = gE[2 * slot];
            E2 = gE[2 * slot + 1];
            rc_stale = false;
          }
          ++njump;
          if (trace != nullptr && leader && lane == 0) {
            int64_t *tr = trace + ((size_t)row * (size_t)I_max + (size_t)(tk - 1)) * 3;
            tr[0] = E1;
            tr[1] = E2;
            tr[2] = -1 - (int64_t)slot;
          }
        }
      }
    }
    if (kstar == Keff) {  // no bit accepted in the window
      t += (uint32_t)Keff;
      flip_streak = 0;
      __syncwarp();
      continue;
    }

    // ---- iteration tf = t + kstar flips.  Every record of targets tf
    // onwards is given up (the flip may change |A| or rewrite their slots):
    // a copy taken by the window has landed, one still in flight is waited
    // for before its buffer is filled again.  The next round copies again
    // from target tf + 1.
    const uint32_t tf = t + (uint32_t)kstar;
    // the next iteration, tried alone after a flip, will likely need
    // draws: their Philox blocks overlap the selection below, and their
    // -ln(u) values start coming now
    if (can_stage && tf < I_max) {
      cp_async_wait_all();  // no earlier copy may still be writing
      __syncwarp();
      for (int c = c0; c < c1; ++c) {
        uint32_t d[4] = {(uint32_t)(c * 32 + lane), tf + 1u, rep, kTagAccept};
        philox10(d, k0, k1);
        float *tv = sTbl + (size_t)(c - c0) * 128;
#pragma unroll
        for (int j = 0; j < 4; ++j) cp_async4(&tv[4 * lane + j], &tablef[d[j] >> 16]);
      }
      cp_async_commit();
      staged = tf + 1u;
    }
    if (LA > 0) {
      // lane k gives up target tf + k (at most K + LA < 32 of them)
      const int nd = (int)issued_to - (int)tf + 1;
      const uint32_t tau = tf + (uint32_t)lane;
      const int b = lane < nd ? sPf[tau & pfm].x : -1;
      freeb |= __reduce_or_sync(kFull, b >= 0 ? 1u << b : 0u);
      if (lane < nd) sPf[tau & pfm].x = -1;
      __syncwarp();
      issued_to = tf;
    }
    const WRing ef = ring[tf % kWarpRing];
    const int32_t *cntp = cntr + 8 * kstar;  // [warp] counts of iteration tf
    {
      const int4 ca = reinterpret_cast<const int4 *>(cntp)[0],
                 cb = reinterpret_cast<const int4 *>(cntp)[1];
      // prefix sums of the warps' counts, in registers
      const int s0 = ca.x, s1 = s0 + ca.y, s2 = s1 + ca.z, s3 = s2 + ca.w, s4 = s3 + cb.x,
                s5 = s4 + cb.y, s6 = s5 + cb.z, total = s6 + cb.w;
      // ---- one accepted flip at random (R11): rank r in ascending bit order
      int r = pick(ef.sel, total);
      // the warp holding rank r: the number of warps whose counts end at or
      // before it (warps past the team's G count 0 and end at `total`)
      const int ow = (r >= s0) + (r >= s1) + (r >= s2) + (r >= s3) + (r >= s4) + (r >= s5) +
                     (r >= s6);
      const int sw[8] = {0, s0, s1, s2, s3, s4, s5, s6};
      int before_w = 0;
#pragma unroll
      for (int w = 1; w < 8; ++w)
        if (ow == w) before_w = sw[w];
      r -= before_w;
      const unsigned char *ows = T.ws0 + (size_t)ow * SL.warp;
      const uint4 *oAccW = reinterpret_cast<const uint4 *>(ows + SL.acc);
      const int32_t *oAccC = reinterpret_cast<const int32_t *>(ows + SL.acc + 16 * (size_t)SL.nc_max);
      int q = 0, before = 0;
      uint4 bw = oAccW[0];
      for (;;) {
        const int k = __popc(bw.x) + __popc(bw.y) + __popc(bw.z) + __popc(bw.w);
        if (r < before + k) break;
        before += k;
        bw = oAccW[++q];
      }
      const int c = oAccC[q];
      // lane l's accepted bits (4l .. 4l + 3 of the chunk) as a nibble, and
      // the accepted bits of lanes 0 .. l (from the ballots, no shuffles)
      const uint32_t nib = ((bw.x >> lane) & 1u) | (((bw.y >> lane) & 1u) << 1) |
                           (((bw.z >> lane) & 1u) << 2) | (((bw.w >> lane) & 1u) << 3);
      const int cl = __popc(nib);
      const uint32_t upto = lane == 31 ? kFull : (2u << lane) - 1u;
      const int incl = __popc(bw.x & upto) + __popc(bw.y & upto) + __popc(bw.z & upto) +
                       __popc(bw.w & upto);
      const int rr = r - before;
      const bool mine = rr >= incl - cl && rr < incl;
      const unsigned who = __ballot_sync(kFull, mine);
      const int owner = __ffs(who) - 1;
      int jj = mine ? nth_set_bit(nib, rr - (incl - cl)) : 0;
      jj = __shfl_sync(kFull, jj, owner);
      const int ps = c * 128 + owner * 4 + jj;

      if (rc_stale) {  // this warp's counts of the state the jump reached
        const unsigned char *rc = bRC(cur);
        for (int q2 = lane; q2 < 2 * n; q2 += 32) rcp[q2] = rc[q2];
        __syncwarp();
        rc_stale = false;
      }
      const int j = divn(ps), v = ps - j * n;
      // the flip's global reads, issued together: L(ps), flow row j,
      // distance row v and this warp's first chunk of fields
      const int2 Lp = curL[ps];
      int32_t rf1[4], rf2[4], rdd[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = lane + 32 * k;
        rf1[k] = rf2[k] = rdd[k] = 0;
        if (i < n) {
          rf1[k] = __ldg(&Fs1[j * n + i]);  // Fs symmetric: row j = column j
          rf2[k] = __ldg(&Fs2[j * n + i]);
          rdd[k] = __ldg(&Dm[v * n + i]);
        }
      }
      int4 nx01 = make_int4(0, 0, 0, 0), nx23 = nx01;
      if (c0 < c1) {
        const int4 *src = reinterpret_cast<const int4 *>(curL + c0 * 128 + lane * 4);
        nx01 = src[0];
        nx23 = src[1];
      }
      // the rows into this warp's shared memory now: no registers held
      // across the archive scan
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = lane + 32 * k;
        if (i < n) {
          sRow[i] = rf1[k];
          sRow[kMaxN + i] = rf2[k];
          sRow[2 * kMaxN + i] = rdd[k];
        }
      }
      uint32_t *xw = bX(cur);
      const int xps = (int)((xw[ps >> 5] >> (ps & 31)) & 1u);
      const int sgn = 1 - 2 * xps;  // +1: the bit turns on
      const int64_t hps = (int64_t)rcp[j] + (int64_t)rcp[n + v] - 1 - 2 * xps;
      const int64_t nE1 = E1 + (int64_t)sgn * ((int64_t)Lp.x + w1l * hps);
      const int64_t nE2 = E2 + (int64_t)sgn * ((int64_t)Lp.y + w2l * hps);
      // frozen layout, state in a header buffer: the flip's state is built
      // in kFull_b, starting from this warp's state words (the header
      // buffer is read no more once every warp passes the next barrier)
      const int fdst = frozen && cur != kFull_b ? kFull_b : cur;
      if (fdst != cur) {
        uint32_t *xd = bX(fdst);
        for (int q2 = 4 * c0 + lane; q2 < 4 * c1; q2 += 32) xd[q2] = xw[q2];
        __syncwarp();
        xw = xd;
      }

      // ---- archive update: Alg. 4 (explore) or Alg. 5 (exploit), decided
      // the same way by every warp of the team
      int target = -1;
      int first_dom = -1;  // explore: this warp's first dominated slot of its stripes
      if (!exploit) {
        // the first member x dominates is replaced; else x is appended.
        // Warp w scans the stripes of 32 slots w, w + G, ...; the team's
        // first is the least of the warps' (after the barrier below).
        for (int base = 32 * wt; base < acount; base += 32 * G) {
          const int y = base + lane;
          bool dom = false;
          if (y < acount) {
            const longlong2 ye = y < se ? sAE[y] : make_longlong2(gE[2 * y], gE[2 * y + 1]);
            dom = dominates(nE1, nE2, ye.x, ye.y);
          }
          const unsigned bal = __ballot_sync(kFull, dom);
          if (bal) {
            first_dom = base + __ffs(bal) - 1;
            break;
          }
        }
        if (lane == 0) sScan[8 * (int)(rnd & 1u) + wt] = first_dom;
      } else {
        // no member may dominate x; then a random dominated member is
        // replaced (tag 3 draw, slot order), else x is appended
        int nb = 0;
        bool anyd = false;
        for (int base = 0; base < acount; base += 32) {
          const int y = base + lane;
          bool dom = false, domd = false;
          if (y < acount) {
            const longlong2 ye = y < se ? sAE[y] : make_longlong2(gE[2 * y], gE[2 * y + 1]);
            dom = dominates(nE1, nE2, ye.x, ye.y);
            domd = dominates(ye.x, ye.y, nE1, nE2);
          }
          nb += __popc(__ballot_sync(kFull, dom));
          anyd |= __any_sync(kFull, domd);
        }
        if (!anyd) {
          if (nb > 0) {
            int want = pick(ef.exp, nb);
            for (int base = 0; base < acount; base += 32) {
              const int y = base + lane;
              bool dom = false;
              if (y < acount) {
                const longlong2 ye = y < se ? sAE[y] : make_longlong2(gE[2 * y], gE[2 * y + 1]);
                dom = dominates(nE1, nE2, ye.x, ye.y);
              }
              const unsigned bal = __ballot_sync(kFull, dom);
              const int k = __popc(bal);
              if (want < k) {
                target = base + nth_set_bit(bal, want);
                break;
              }
              want -= k;
            }
          } else if (acount < s) {
            target = acount++;
          }
        }
      }

      // every warp has read the archive and the accepted lists: they may
      // change now
      sync();
      if (!exploit) {
        for (int w = 0; w < G; ++w) {
          const int f = sScan[8 * (int)(rnd & 1u) + w];
          if (f >= 0 && (target < 0 || f < target)) target = f;
        }
        if (target < 0 && acount < s) target = acount++;
      }
      sWr[tf & pfm] = target;
      if (target >= 0) last_wr_t = tf;
      if (target >= 0 && scribe && lane == 0) {
        gE[2 * target] = nE1;
        gE[2 * target + 1] = nE2;
        if (target < se) sAE[target] = make_longlong2(nE1, nE2);
      }

      // ---- apply the flip to this warp's chunks: outer product of flow
      // row j and distance row v; the counts read are the old ones, so
      // bits of row j or column v add the change
      __syncwarp();
      const bool cached = target >= 0 && target < cslots;
      int2 *const slotL = cached ? gLR + (size_t)target * rec.mp : nullptr;
      int2 *dstL = use_sf ? sF : cached ? slotL : gWork;
      unsigned char *jrec = cached ? gJR + (size_t)target * rec.jr : nullptr;
      uint4 *dA = reinterpret_cast<uint4 *>(jrec);
      uint4 *sa4 = reinterpret_cast<uint4 *>(bA(fdst));
      int c_next = c0;
      for (int cc = c0; cc < c1; ++cc) {
        const int p0 = cc * 128 + lane * 4;
        const int4 l01 = nx01, l23 = nx23;
        c_next = cc + 1;
        if (c_next < c1) {  // the next chunk's fields, loaded while this one computes
          const int4 *src = reinterpret_cast<const int4 *>(curL + c_next * 128 + lane * 4);
          nx01 = src[0];
          nx23 = src[1];
        }
        const uint32_t nibx = (xw[p0 >> 5] >> (p0 & 31)) & 15u;
        int Lx[4] = {l01.x, l01.z, l23.x, l23.z};
        int Ly[4] = {l01.y, l01.w, l23.y, l23.w};
        uint32_t an[4];
        // the four bits' (i, u), independent of one another, so that their
        // shared-memory reads issue together; a padding bit (p >= m) has
        // i <= 128, whose reads stay inside the rows and counts arrays
        int iq[4], uq[4];
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) {
          iq[q2] = divn(p0 + q2);
          uq[q2] = p0 + q2 - iq[q2] * n;
        }
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) {
          const int p = p0 + q2, i = iq[q2], u = uq[q2];
          const int32_t dd = sRow[2 * kMaxN + u];
          const int32_t f1 = sRow[i], f2 = sRow[kMaxN + i];
          const int hc = (int)rcp[i] + (int)rcp[n + u];
          if (p < m) {
            Lx[q2] += sgn * f1 * dd;
            Ly[q2] += sgn * f2 * dd;
            const int xq = (int)((nibx >> q2) & 1u) ^ (p == ps ? 1 : 0);
            const dE_t g = (dE_t)(1 - 2 * xq);
            const dE_t h = (dE_t)(hc + sgn * ((i == j ? 1 : 0) + (u == v ? 1 : 0)) - 1 - 2 * xq);
            an[q2] = WA::penalty(g * ((dE_t)Lx[q2] + w1 * h), g * ((dE_t)Ly[q2] + w2 * h), lenient);
          } else {
            an[q2] = 0xFFFFFFFFu;
          }
        }
        const int4 f01 = make_int4(Lx[0], Ly[0], Lx[1], Ly[1]);
        const int4 f23 = make_int4(Lx[2], Ly[2], Lx[3], Ly[3]);
        int4 *dst = reinterpret_cast<int4 *>(dstL + p0);
        dst[0] = f01;
        dst[1] = f23;
        if (use_sf && cached) {  // and the slot's field record
          int4 *dg = reinterpret_cast<int4 *>(slotL + p0);
          dg[0] = f01;
          dg[1] = f23;
        }
        const uint4 a4n = make_uint4(an[0], an[1], an[2], an[3]);
        sa4[cc * 32 + lane] = a4n;
        if (cached) dA[cc * 32 + lane] = a4n;
        if (FZ && cached) {
          // the record's candidate masks for the frozen schedule
          const uint32_t m0 = __ballot_sync(kFull, an[0] <= hiF32),
                         m1 = __ballot_sync(kFull, an[1] <= hiF32),
                         m2 = __ballot_sync(kFull, an[2] <= hiF32),
                         m3 = __ballot_sync(kFull, an[3] <= hiF32);
          if (lane == 0) reinterpret_cast<uint4 *>(jrec + rec.off_cm)[cc] = make_uint4(m0, m1, m2, m3);
        }
      }
      // this warp's state words of x' (bit ps toggled) into the archive
      const int qps = ps >> 5;
      const uint32_t bps = 1u << (ps & 31);
      if (target >= 0) {
        for (int q2 = 4 * c0 + lane; q2 < 4 * c1; q2 += 32) {
          const uint32_t wv = xw[q2] ^ (q2 == qps ? bps : 0u);
          if (q2 < W) gB[(size_t)target * W + q2] = wv;
          if (cached) reinterpret_cast<uint32_t *>(jrec + rec.off_xw)[q2] = wv;
        }
      }
      __syncwarp();
      // the warp owning bit ps toggles it (no other warp reads that word
      // before the next barrier); every warp updates its own counts
      if (lane == 0) {
        if (qps >= 4 * c0 && qps < 4 * c1) xw[qps] ^= bps;
        rcp[j] = (unsigned char)((int)rcp[j] + sgn);
        rcp[n + v] = (unsigned char)((int)rcp[n + v] + sgn);
      }
      __syncwarp();
      if (target >= 0 && scribe) {
        if (cached) {
          const uint32_t *rcw = reinterpret_cast<const uint32_t *>(rcp);
          uint32_t *jrc = reinterpret_cast<uint32_t *>(jrec + rec.off_rc);
          for (int q2 = lane; q2 < (int)(rec.off_E - rec.off_rc) / 4; q2 += 32) jrc[q2] = rcw[q2];
          if (lane == 0) {
            int64_t *je = reinterpret_cast<int64_t *>(jrec + rec.off_E);
            je[0] = nE1;
            je[1] = nE2;
          }
        }
      }
      if (cached) unfenced = true;  // fenced before the next bulk copy
      if (fdst != cur) {  // the header buffer is free again
        freeb |= 1u << cur;
        cur = fdst;
      }
      cur_slot = -1;
      curL = dstL;
      E1 = nE1;
      E2 = nE2;
      ++nflip;
      if (trace != nullptr && leader && lane == 0) {
        int64_t *tr = trace + ((size_t)row * (size_t)I_max + (size_t)(tf - 1)) * 3;
        tr[0] = E1;
        tr[1] = E2;
        tr[2] = (int64_t)ps;
      }
    }
    flip_streak = kstar == 0 ? flip_streak + 1 : 1;
    t = tf + 1u;
    __syncwarp();
  }
  // no copy may be in flight when the item ends
  cp_async_wait_all();
  for (int b = 0; b < 32; ++b)
    if ((pend >> b) & 1u) retire_buf(b);
  fail = sync_or(fail);
  if (fail) {
    if (leader && lane == 0) atomicExch(R.error, kErrCopyTimeout);
    return false;
  }
  const uint32_t *xw = bX(cur);
  for (int q2 = 4 * c0 + lane; q2 < 4 * c1 && q2 < W; q2 += 32)
    R.x_final[(size_t)row * W + q2] = xw[q2];
  if (leader && lane == 0) {
    R.E_final[2 * row] = E1;
    R.E_final[2 * row + 1] = E2;
    R.arch_count[row] = acount;
    int64_t *st = R.stats + (size_t)kStats * row;
    st[0] = nflip;
    st[1] = njump;
    st[2] = nempty;
    st[3] = 0;
    st[4] = npref;
    st[5] = ndirect;
    st[6] = 0;
    st[7] = nrebuild;
  }
  sync();  // the team's shared memory is reused by the next item
  return true;
}

// The register allocation is sized for one block per SM: no register
// spills (their local-memory reads missed L1 and sat on every iteration's
// chain), at the cost of resident warps.
template <bool NARROW, bool FZ>
__global__ void __launch_bounds__(256, 1) warp_anneal_kernel(const WarpLaunch L) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int G = L.team, nteams = (blockDim.x >> 5) / G;
  const int team = wid / G;
  Team T;
  T.G = G;
  T.wt = wid - team * G;
  T.lane = lane;
  T.bar = 1 + team;
  T.ts = smem + (size_t)team * L.sm.total;
  T.ws0 = T.ts + L.sm.team;
  uint64_t *bar = reinterpret_cast<uint64_t *>(T.ts + L.sm.mbar);
  int32_t *sItem = reinterpret_cast<int32_t *>(T.ts + L.sm.cnt + 8 * L.sm.cst);
  const bool leader = T.wt == 0;
  if (leader && lane == 0) {
    const int nbar = L.nbuf > L.nbuf_f ? L.nbuf : L.nbuf_f;
    for (int b = 0; b < nbar; ++b) mbar_init(&bar[b], 1);
    fence_mbar_init();
  }
  if (G > 1) team_sync(T.bar, 32 * G);
  else __syncwarp();
  unsigned char *cache =
      L.cache + (size_t)(blockIdx.x * nteams + team) * L.cache_stride;
  uint32_t par = 0;
  for (;;) {
    if (leader && lane == 0) *sItem = atomicAdd(L.counter, 1);
    if (G > 1) team_sync(T.bar, 32 * G);
    else __syncwarp();
    const int it = *sItem;
    if (G > 1) team_sync(T.bar, 32 * G);  // read before the next item is written
    if (it >= L.nitems) break;
    const int2 item = L.items[it];
    const WarpRun &R = L.runs[item.x];
    if ((R.narrow != 0) != NARROW) {  // the host launches matching variants only
      if (leader && lane == 0) atomicExch(R.error, kErrVariant);
      continue;
    }
    if (!team_run<NARROW, FZ>(R, item.y, T, L, cache, par)) break;
  }
}

}  // namespace

namespace {
// The warp engine's acceptance decision for given penalties, one per thread
// (the same device functions its trials run): accept[k] and the path taken
// (1 or 0 decided in FP32, -1 by the double test).
__global__ void check_accept_kernel(const int64_t *a, const double *delta, const uint32_t *idx,
                                    int count, const double *T, const float *Tf,
                                    uint8_t *accept, int8_t *path) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const int64_t ak = a[k];
  const double dk = delta[k];
  const uint32_t ik = idx[k];
  const int r = prefilter(penalty_f32(ak), __double2float_rn(dk), Tf[ik]);
  accept[k] = (uint8_t)(r > 0 || (r < 0 && (double)ak <= __dmul_rn(dk, T[ik])));
  path[k] = (int8_t)r;
}

// The kernel variant of a launch: narrow or not.
const void *warp_kernel(bool narrow, bool fz) {
  if (fz)
    return narrow ? reinterpret_cast<const void *>(warp_anneal_kernel<true, true>)
                  : reinterpret_cast<const void *>(warp_anneal_kernel<false, true>);
  return narrow ? reinterpret_cast<const void *>(warp_anneal_kernel<true, false>)
                : reinterpret_cast<const void *>(warp_anneal_kernel<false, false>);
}
}  // namespace

cudaError_t launch_warp(const WarpLaunch &L, bool narrow, int grid, int teams,
                        cudaStream_t stream) {
  const int warps = teams * L.team;
  if (L.team < 1 || L.team > 8 || teams < 1 || warps > 8 || teams > 15 || grid < 1)
    return cudaErrorInvalidValue;
  const size_t smem = (size_t)teams * L.sm.total;
  const void *f = warp_kernel(narrow, L.nbuf_f > 0);
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void *args[1] = {const_cast<WarpLaunch *>(&L)};
  e = cudaLaunchKernel(f, dim3((unsigned)grid), dim3((unsigned)(32 * warps)), args, smem, stream);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_check_accept(const int64_t *a, const double *delta, const uint32_t *idx,
                                int count, const double *T, const float *Tf, uint8_t *accept,
                                int8_t *path, cudaStream_t stream) {
  if (count < 1) return cudaSuccess;
  check_accept_kernel<<<(count + 255) / 256, 256, 0, stream>>>(a, delta, idx, count, T, Tf,
                                                               accept, path);
  return cudaGetLastError();
}

cudaError_t warp_function(bool narrow, bool fz, int team, size_t smem, const void **func) {
  (void)team;
  const void *f = warp_kernel(narrow, fz);
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) *func = f;
  return e;
}

cudaError_t warp_occupancy(bool narrow, bool fz, int team, size_t smem, int *blocks) {
  const void *f = warp_kernel(narrow, fz);
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, f, 32 * team, smem);
}

}  // namespace moda
