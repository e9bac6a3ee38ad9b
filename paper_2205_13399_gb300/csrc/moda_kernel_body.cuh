// Annealing kernel of the multi-objective Digital Annealer (MDA), Sec. 3.3,
// Alg. 3 of arXiv 2205.13399, for the bi-objective QAP: one thread block
// runs one replica for all I_max iterations, its state held on chip.
//
// A block is Tw worker threads plus two control warps.  Worker `tid` owns
// the bits p = k*Tw + tid, k < B ("rounds"), of the n*n-bit two-way
// one-hot state (bit p = i*n + u: facility i at location u, Sec. 2.2) and
// keeps in registers, per owned bit, x_p (a bit of `xmask`) and
//   Delta E_k(p) = (1 - 2 x_p)(L_k[p] + w_k (R_i + C_u - 1 - 2 x_p)),
// L_k[(i,u)] = sum_{(j,v)} Fs^k_ij d_uv x_jv the cost local field (Fs^k =
// F^k + F^k^T), R_i and C_u the row and column counts, alpha_k = w_k / 2
// (Eq. cale with the penalty of Eq. wqubom).  With zero-diagonal symmetric
// distances P^k_(i,u),(j,v) = Fs^k_ij d_uv, so Q is never stored: a flip of
// (j,v) with s = +1 when the bit turns on changes every other Delta E_k(q)
// by (1 - 2 x_q) s (Fs^k_ij d_uv + w_k [i == j or u == v]) -- the outer
// product of a flow column and a distance column -- and the flipped bit's
// Delta E changes sign.
//
// One iteration t (Alg. 3):
//   workers     the parallel trial of their bits; warp ballots give accept
//               masks in (round, warp, lane) order = ascending bit order;
//               accepted bits publish Delta E and their state bit.
//   warp A      meanwhile: every 8 iterations the draws and schedule
//               entries 8..15 iterations ahead; the jump record of t (the
//               member a jump would land on -- its draw and |A| are known
//               -- and whether its prefetched copy is usable).
//   warp B      meanwhile (field cache on, replica not in a run of flips):
//               a bulk copy (TMA, mbarrier) of the cached Delta E of the
//               member a jump at t + lookahead would land on; with the
//               cache read in place, an L2 prefetch of it instead.
//   -- barrier counting the threads that accepted a bit --
//   every warp  0: the jump (or escape) of warp A's record; otherwise the
//               rank selection of one accepted bit ("one flip at random").
//               Flip: workers apply it to their registers and ballot "x
//               dominates slot y" -- barrier -- every warp picks the target
//               slot (Alg. 4 / Alg. 5); workers store their part of x (and
//               of Delta E, into the cache).  Jump: workers take the
//               member's Delta E from the prefetch buffer, the cache, or
//               rebuild it as L_k = Fs_k (X D).  Otherwise: raise the
//               energy offset by beta.
#pragma once

#include <cstdint>
#include <type_traits>

#include "moda_device.cuh"
#include "moda_internal.h"

namespace moda {
namespace {

constexpr uint32_t kRing = 32;  // draw / schedule ring, iterations

// The two control warps alone (named barrier 1, 64 threads).
__device__ __forceinline__ void bar_sync_pair() {
  asm volatile("bar.sync 1, 64;" ::: "memory");
}

// ---- warp-level mask scans ----------------------------------------------

// Over `items` ballot masks in (round, warp) order: each lane sums a
// contiguous chunk; returns the total (all lanes) and the lane's inclusive
// prefix and own count.
__device__ __forceinline__ int warp_mask_total(const uint32_t *masks,
                                               int items, int lane, int &incl,
                                               int &cnt) {
  const int per = (items + 31) >> 5;
  cnt = 0;
  for (int q = 0; q < per; ++q) {
    const int it = lane * per + q;
    if (it < items) cnt += __popc(masks[it]);
  }
  incl = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += v;
  }
  return __shfl_sync(kFull, incl, 31);
}

// The same chunking as warp_mask_total without the scan: the lane's own
// count in `cnt`, the total in every lane.
__device__ __forceinline__ int warp_mask_count(const uint32_t *masks,
                                               int items, int lane, int &cnt) {
  const int per = (items + 31) >> 5;
  cnt = 0;
  for (int q = 0; q < per; ++q) {
    const int it = lane * per + q;
    if (it < items) cnt += __popc(masks[it]);
  }
  return (int)__reduce_add_sync(kFull, (unsigned)cnt);
}

// Flat index round*Tw + warp*32 + lane of the r-th set bit (r < total), in
// every lane.
__device__ __forceinline__ int warp_mask_select(const uint32_t *masks,
                                                int items, int nw, int Tw,
                                                int lane, int incl, int cnt,
                                                int r) {
  const int per = (items + 31) >> 5;
  const int excl = incl - cnt;
  int found = -1;
  if (r >= excl && r < incl) {
    int rr = r - excl;
    for (int q = 0; q < per; ++q) {
      const int it = lane * per + q;
      if (it >= items) break;
      const uint32_t mk = masks[it];
      const int pc = __popc(mk);
      if (rr < pc) {
        const int k = it / nw;
        const int w = it - k * nw;
        found = k * Tw + w * 32 + nth_set_bit(mk, rr);
        break;
      }
      rr -= pc;
    }
  }
  const unsigned who = __ballot_sync(kFull, found >= 0);
  return __shfl_sync(kFull, found, __ffs(who) - 1);
}

__device__ __forceinline__ int64_t block_sum(int64_t v, int64_t *red,
                                             int lane, int warp, int nw) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  int64_t t = 0;
  for (int w = 0; w < nw; ++w) t += red[w];
  __syncthreads();
  return t;
}

struct Bcast {
  int64_t dE1, dE2;  // Delta E of the flipped bit (owner-published path)
  int32_t sgn;       // +1: the bit turns on, -1: off
  int32_t pad;
};

// Kinds of iteration outcome (Alg. 3).  kFinish: this and every later
// iteration jump (fast-forward), the last one to the slot given.
enum : int32_t { kNone = 0, kFlip = 1, kJump = 2, kFinish = 3 };

// Prefetch bookkeeping entry for one target iteration.
struct PfRec {
  int32_t iter;    // iteration that issued the copy, 0 = none
  int32_t slot;    // archive slot copied
  int32_t parity;  // mbarrier phase parity that signals completion
  int32_t pad;
};

// Schedule entry of one iteration: delta_t and the thresholds, also
// clamped to int32 for the narrow variant.
struct SchEntry {
  double delta;
  int64_t lo, hi;
  uint32_t lo32, hi32;  // clamped to 2^32 - 1
  // normalised acceptance: fl(delta T_min) and fl(delta T_max); lo and hi
  // then bound the integer penalty (see fill_rings)
  double lod, hid;
  float deltaf;  // fl32(delta), for the FP32 test of prefilter()
  uint32_t pad;
};
static_assert(sizeof(SchEntry) == 56, "schedule entry layout (smem_layout reserves 56 bytes)");

// What iteration t does when no bit is accepted (Alg. 3), settled by
// control warp A before the iteration's barrier.
struct JumpRec {
  int32_t kind;     // kJump, kNone or kFinish
  int32_t slot;     // archive slot jumped to (kFinish: by iteration I_max)
  int32_t pbuf;     // prefetch buffer holding it, -1: read the cache record
  uint32_t parity;  // that buffer's mbarrier phase parity
  // pbuf >= 0: shared-memory byte offsets of the member's Delta E record,
  // its energies, its first state word and the buffer's mbarrier
  uint32_t rf, se, ws, bar;
};

// NARROW: Delta E in int32 and the acceptance penalty in uint32 (the host
// checked |Delta E_k| < 2^31 for every state and objective); otherwise
// int64.
// MODE 1 (EXT): the optional extensions -- QUBO normalisation (Sec. 4.2:
// objective k's Delta E scaled by s_k inside the acceptance test, in IEEE
// double) and archive snapshots -- compiled in; without them the loop
// carries neither.  MODE 2: the fast-forward bookkeeping compiled in.
// MODE 3: the default algorithm compiled in -- strict acceptance
// (Eq. pacceptms), the explorative archive (Alg. 4), the escape by a jump
// to the archive, no trace.  MODE 4 (B = 1): MODE 3 and the on-chip
// placement -- field cache on, prefetch distance 1, archive energies,
// archive states and published Delta E in shared memory.  MODE 5
// (2 <= B <= 4): the same with the archive states in global memory.  The
// host picks MODE 3 to 5 only for matching runs; a block given other
// arguments reports kErrVariant and does nothing.  MODE 0: none of these.
template <int B, bool NARROW, int MODE>
__global__ void __launch_bounds__(kMaxThreads, 1)
    anneal_kernel(const AnnealArgs A) {
  constexpr bool EXT = MODE == 1;
  constexpr bool DEF = MODE >= 3, DEFPL = MODE == 4 || MODE == 5;
  if (DEF) {
    bool match = A.accept == 0 && A.archive == 0 && A.escape == 0 && A.trace == nullptr &&
                 A.normalize == 0 && A.snap_every == 0 && A.fast_forward == 0;
    if (DEFPL)
      match = match && A.lookahead == 1 && A.de_in_smem != 0 && A.energies_in_smem != 0 &&
              (A.bits_in_smem != 0) == (MODE == 4) && A.fcache != nullptr;
    if (!match) {
      if (threadIdx.x == 0) atomicExch(A.error, kErrVariant);
      return;
    }
  }
  // Run settings, compile-time constants in the modes that fix them.
  const int cAccept = DEF ? 0 : A.accept;
  const int cArchive = DEF ? 0 : A.archive;
  const int cEscape = DEF ? 0 : A.escape;
  int64_t *const cTrace = DEF ? nullptr : A.trace;
  const int cLookahead = DEFPL ? 1 : A.lookahead;
  const bool cDeSmem = DEFPL || A.de_in_smem != 0;
  const bool cEnergiesSmem = DEFPL || A.energies_in_smem != 0;
  const bool cBitsSmem = MODE == 4 || (MODE != 5 && A.bits_in_smem != 0);
  using dE_t = typename std::conditional<NARROW, int32_t, int64_t>::type;
  using dE2_t = typename std::conditional<NARROW, int2, longlong2>::type;
  // acceptance penalty: a sum of two non-negative Delta E, so uint32 in
  // the narrow variant (each |Delta E_k| < 2^31)
  using pen_t = typename std::conditional<NARROW, uint32_t, int64_t>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = A.n, m = A.m, W = A.W, s = A.s;
  const int T = blockDim.x, tid = threadIdx.x;
  const int Tw = T - 64;                 // worker threads
  const int lane = tid & 31, warp = tid >> 5, NWB = Tw >> 5;
  const bool worker = tid < Tw;
  const bool control = !worker;          // the last two warps:
  const bool ctlA = warp == NWB;         // draws, schedule, jump records
  const bool ctlB = warp == NWB + 1;     // field-cache prefetch
  const int items = B * NWB;
  const int per = (items + 31) >> 5;     // ballot words per lane in scans
  const bool fc = DEFPL || A.fcache != nullptr;
  const bool de_smem = cDeSmem;
  const int LA = cLookahead;            // prefetch distance
  // Prefetch buffers: target iteration tt uses buffer tt % NB.  The copy
  // for t + LA starts before the barrier of iteration t, while a lagging
  // warp may still read the buffer of t - 1, so NB = LA + 2.
  // LA = -1: the cache is read in place, nothing is prefetched.
  const int NB = LA + 2;
  const bool pf = fc && LA >= 0;
  // Fast-forward (no extensions): stop once the rest of the run is settled.
  constexpr bool ff = MODE == 2;
  const Placement P{cEnergiesSmem, cBitsSmem, fc, LA,
                    de_smem, NARROW, ff};
  const SmemLayout lay = smem_layout(n, m, W, s, Tw, B, P);
  const bool NORM_ON = EXT && A.normalize != 0;
  const SlotLayout sl = slot_layout(m, NARROW);
  const dE_t w1 = (dE_t)A.w1, w2 = (dE_t)A.w2;
  int2 *sFs = reinterpret_cast<int2 *>(smem + lay.Fs);
  int32_t *sD = reinterpret_cast<int32_t *>(smem + lay.D);
  int32_t *sM = reinterpret_cast<int32_t *>(smem + lay.M);
  uint32_t *sMask = reinterpret_cast<uint32_t *>(smem + lay.mask);
  uint32_t *sAmask = reinterpret_cast<uint32_t *>(smem + lay.amask);
  // Rings of kRing iterations: sRnd[(t % kRing) * 4 + j] holds the draw of
  // tag kTagSelect + j of iteration t, sSch[t % kRing] its schedule entry.
  uint32_t *sRnd = reinterpret_cast<uint32_t *>(smem + lay.rnd);
  SchEntry *sSch = reinterpret_cast<SchEntry *>(smem + lay.sch);
  // Row and column counts of the last rebuilt state, two buffers used in
  // turn (rebuild q fills buffer q % 2 and clears the other one).
  int32_t *sRC = reinterpret_cast<int32_t *>(smem + lay.RC);
  int64_t *sRed = reinterpret_cast<int64_t *>(smem + lay.red);
  Bcast *bc = reinterpret_cast<Bcast *>(smem + lay.bc);
  uint32_t *sInit = reinterpret_cast<uint32_t *>(smem + lay.init);
  uint64_t *sBar = reinterpret_cast<uint64_t *>(smem + lay.mbar);
  dE2_t *sDE = reinterpret_cast<dE2_t *>(smem + lay.dE);  // [bits]
  // state bit of each accepted bit, published beside its Delta E
  uint8_t *sXb = reinterpret_cast<uint8_t *>(smem + lay.dE) + sizeof(dE2_t) * (size_t)B * Tw;
  // Prefetch bookkeeping (after initialisation; shares the reduction
  // space): sPf[target iteration % 8], the copies warp B started, and
  // sWr[iteration % 8] = the archive slot that iteration wrote (-1 = none),
  // kept by warp A.
  PfRec *sPf = reinterpret_cast<PfRec *>(smem + lay.red);
  int32_t *sWr = reinterpret_cast<int32_t *>(smem + lay.red + 8 * sizeof(PfRec));
  JumpRec *sJr = reinterpret_cast<JumpRec *>(smem + lay.jr);  // [t % 8]
  // Fast-forward: sLive[t % 4] == t when some bit of iteration t's trial
  // had its acceptance penalty in (lo_t, hi_t].  Kept by control warp A's
  // lane 0 alone: sFF[0] the archive slot whose state the current
  // iteration tries (-1: the state is no member), sFF[1] the number of
  // slots marked in sDead, and sDead bit y when slot y's state was tried
  // and no bit had a penalty <= hi.  hi_t never rises, so no later trial
  // of that state accepts a bit either, until the slot is rewritten.
  uint32_t *sLive = reinterpret_cast<uint32_t *>(smem + lay.ff);
  int32_t *sFF = reinterpret_cast<int32_t *>(sLive + 4);
  uint32_t *sDead = sLive + 8;
  // One bit per thread: bits 4g .. 4g + 3 take the four words of one
  // acceptance Philox block (group g = p / 4), so a warp's 32 bits need 8
  // blocks per iteration.  A warp that must draw computes the blocks of
  // iterations t .. t + 3 at once (lane l: group 8 warp + l % 8, iteration
  // t + l / 8) into sDraw[32 warp + l] and reuses them while they cover
  // the iteration; sDrawT[warp] is t (0: none yet).
  uint4 *sDraw = reinterpret_cast<uint4 *>(smem + lay.draw);
  uint32_t *sDrawT = reinterpret_cast<uint32_t *>(smem + lay.draw + 16 * (size_t)Tw);

  const int rb = blockIdx.x;
  const uint32_t rep = A.replica_base + (uint32_t)rb;
  const uint32_t k0 = A.seed_lo, k1 = A.seed_hi;
  int64_t *gE = A.arch_E + (size_t)rb * s * 2;
  uint32_t *gBits = A.arch_bits + (size_t)rb * s * W;
  unsigned char *gF = fc ? A.fcache + (size_t)rb * s * sl.bytes : nullptr;
  longlong2 *aE = cEnergiesSmem
                      ? reinterpret_cast<longlong2 *>(smem + lay.archE)
                      : reinterpret_cast<longlong2 *>(gE);
  uint32_t *aBits = cBitsSmem
                        ? reinterpret_cast<uint32_t *>(smem + lay.archB)
                        : gBits;
  int rc_buf = 0;
  const uint32_t I_max = (uint32_t)A.I_max;
  const uint32_t nsched = (uint32_t)A.nsched;

  for (int e = tid; e < n * n; e += T) {
    sFs[e] = make_int2(A.Fs1[e], A.Fs2[e]);
    sD[e] = A.D[e];
  }
  for (int e = tid; e < 4 * n; e += T) sRC[e] = 0;
  // Control warp: draws (select, restart, exploit) and schedule entries of
  // iterations first .. first + 7 into the rings, all lanes on one path:
  // lane l < 24 draws tag kTagSelect + l % 3 of iteration first + l / 3,
  // lane l < 8 copies the schedule entry of iteration first + l.
  // Normalised: the exact thresholds are fl(delta T_min) and fl(delta
  // T_max) on the scaled penalty a'; lo and hi become integer bounds on the
  // unscaled penalty A (a1 + a2, or their minimum), with s_min A <= a' <=
  // s_max A up to a few roundings: A <= lo implies a' <= fl(delta T_min)
  // and A > hi implies a' > fl(delta T_max), by margins of 1e-12.
  const double s_min = A.s1 < A.s2 ? A.s1 : A.s2, s_max = A.s1 < A.s2 ? A.s2 : A.s1;
  auto fill_rings = [&](uint32_t first) {
    const uint32_t it = first + (uint32_t)(lane & 7);
    const uint32_t sn = (it <= nsched ? it : nsched) - 1;
    const double sd = A.sch_delta[sn];
    int64_t slo = A.sch_lo[sn], shi = A.sch_hi[sn];
    double lod = 0, hid = 0;
    if (NORM_ON) {
      lod = __dmul_rn(sd, A.tmin);
      hid = __dmul_rn(sd, A.tmax);
      const double ql = floor(lod / (s_max * (1.0 + 1e-12)));
      const double qh = floor(hid / (s_min * (1.0 - 1e-12)));
      slo = ql < 4.0e18 ? (int64_t)ql : (int64_t)4000000000000000000ll;
      shi = qh < 4.0e18 ? (int64_t)qh : (int64_t)4000000000000000000ll;
    }
    const uint32_t q = first + (uint32_t)(lane < 24 ? lane / 3 : 7);
    const uint32_t tag = (uint32_t)(lane % 3);
    uint32_t c[4] = {0u, q, rep, kTagSelect + tag};
    philox10(c, k0, k1);
    if (lane < 24) sRnd[(q % kRing) * 4 + tag] = c[0];
    if (lane < 8)
      sSch[it % kRing] = SchEntry{sd, slo, shi,
                                  (uint32_t)(slo < 4294967295ll ? slo : 4294967295ll),
                                  (uint32_t)(shi < 4294967295ll ? shi : 4294967295ll), lod, hid,
                                  __double2float_rn(sd), 0u};
  };
  if (ctlB && lane == 0 && pf) {
    for (int b = 0; b < NB; ++b) mbar_init(&sBar[b], 1);
    fence_mbar_init();
  }
  if (ctlA) fill_rings(1);  // iterations 1..8; iteration t = 8i + 1 fills t+8..t+15

  // Own bit k is valid when worker && k*Tw + tid < m: own[k] packs its
  // facility i (bits 8..15) and location u (bits 0..7); D1[k], D2[k] hold
  // Delta E_1, Delta E_2 of flipping it (Eq. cale), kept up to date.
  int own[B];
  dE_t D1[B], D2[B];
  uint32_t xmask = 0;
  auto valid = [&](int k) { return worker && k * Tw + tid < m; };
#pragma unroll
  for (int k = 0; k < B; ++k) {
    const int p = k * Tw + tid;
    own[k] = valid(k) ? (((p / n) << 8) | (p % n)) : 0;
    D1[k] = 0;
    D2[k] = 0;
  }
  // Initial state (Alg. 3: "a random binary solution"): bit p is bit p % 32
  // of word (p / 32) % 4 of the draw (p / 128, 0, replica, init).
#pragma unroll
  for (int k = 0; k < B; ++k) {
    if (!valid(k)) continue;
    const int p = k * Tw + tid;
    uint32_t c[4] = {(uint32_t)p >> 7, 0u, rep, kTagInit};
    philox10(c, k0, k1);
    xmask |= ((word_of(c, (p >> 5) & 3) >> (p & 31)) & 1u) << k;
  }
  if (worker) {
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const uint32_t wv = __ballot_sync(kFull, (xmask >> k) & 1u);
      if (lane == 0 && k * NWB + warp < W) sInit[k * NWB + warp] = wv;
    }
  }
  __syncthreads();

  // Delta E of every owned bit of the state held in `words`, from scratch,
  // in two passes around one barrier: (1) M = X * D (M_ju = sum_v x_jv d_vu)
  // and the row / column counts R, C into shared memory; (2) every worker
  // forms the cost fields L_k[(i,u)] = sum_j Fs^k_ij M_ju and
  //   Delta E_k = (1 - 2x)(L_k + w_k (R_i + C_u - 1 - 2x)).
  // Fields are exact int32 (the instance check bounds them).  Returns the
  // sum over set bits of L_1 and of L_2 (2 c_k) in s1, s2.
  auto rebuild = [&](const uint32_t *words, int64_t &s1, int64_t &s2) {
    for (int e = tid; e < n * n; e += T) {
      const int j = (int)__umulhi((uint32_t)e, A.magic);
      const int u = e - j * n;
      const int lo_bit = j * n, hi_bit = j * n + n;  // row j: [lo_bit, hi_bit)
      int32_t acc = 0;
      for (int w = lo_bit >> 5; w <= (hi_bit - 1) >> 5; ++w) {
        uint32_t word = words[w];
        const int base = w * 32;
        if (base < lo_bit) word &= ~0u << (lo_bit - base);
        if (base + 32 > hi_bit) word &= ~0u >> (base + 32 - hi_bit);
        while (word) {
          const int v = base + __ffs(word) - 1 - lo_bit;
          word &= word - 1;
          acc += sD[v * n + u];
        }
      }
      sM[e] = acc;
      if ((words[e >> 5] >> (e & 31)) & 1u) {  // bit e = (j, u) is set
        atomicAdd(&sRC[rc_buf * 2 * n + j], 1);
        atomicAdd(&sRC[rc_buf * 2 * n + n + u], 1);
      }
    }
    xmask = 0;
#pragma unroll
    for (int k = 0; k < B; ++k) {
      if (!valid(k)) continue;
      const int q = k * Tw + tid;
      xmask |= ((words[q >> 5] >> (q & 31)) & 1u) << k;
    }
    __syncthreads();
    const int32_t *cR = sRC + rc_buf * 2 * n, *cC = cR + n;
    for (int e = tid; e < 2 * n; e += T) sRC[(1 - rc_buf) * 2 * n + e] = 0;
    s1 = 0;
    s2 = 0;
#pragma unroll
    for (int k = 0; k < B; ++k) {
      if (!valid(k)) continue;
      const int i = own[k] >> 8, u = own[k] & 255;
      int32_t a1 = 0, a2 = 0;
      const int2 *frow = sFs + i * n;  // Fs symmetric: row i = column i
#pragma unroll 5
      for (int j = 0; j < n; ++j) {
        const int2 f = frow[j];
        const int32_t mm = sM[j * n + u];
        a1 += f.x * mm;
        a2 += f.y * mm;
      }
      const int xv = (int)((xmask >> k) & 1u);
      const dE_t g = (dE_t)(1 - 2 * xv);
      const dE_t h = (dE_t)(cR[i] + cC[u] - 1 - 2 * xv);
      D1[k] = g * ((dE_t)a1 + w1 * h);
      D2[k] = g * ((dE_t)a2 + w2 * h);
      if (xv) {
        s1 += a1;
        s2 += a2;
      }
    }
    rc_buf ^= 1;
  };
  int64_t E1, E2;
  {
    // E_k = c_k + w_k g / 2 with c_k = (sum_p x_p L_k[p]) / 2 and g from
    // the row and column counts.
    int64_t s1, s2, gp = 0;
    rebuild(sInit, s1, s2);
    for (int e = tid; e < n; e += T) {
      const int64_t dr = 1 - sRC[e], dc = 1 - sRC[n + e];
      gp += dr * dr + dc * dc;
    }
    s1 = block_sum(s1, sRed, lane, warp, T >> 5);
    s2 = block_sum(s2, sRed, lane, warp, T >> 5);
    gp = block_sum(gp, sRed, lane, warp, T >> 5);
    E1 = s1 / 2 + A.w1 * (gp / 2);
    E2 = s2 / 2 + A.w2 * (gp / 2);
  }
  if (tid < 8) {
    sPf[tid] = PfRec{0, 0, 0, 0};
    sWr[tid] = -1;
  }
  if (ff)
    for (int e = tid; e < 8 + ((s + 31) >> 5); e += T) sLive[e] = e == 4 ? 0xFFFFFFFFu : 0u;
  if (B == 1 && tid < NWB) sDrawT[tid] = 0;
  __syncthreads();

  int64_t Eoff = 0;
  int acount = 0;
  // Outcome counters, kept by control warp A's lane 0 in shared memory:
  // flips, jumps, empty escapes, offset raises, prefetched jumps, direct
  // reads, iterations fast-forwarded.
  uint32_t *sStat = reinterpret_cast<uint32_t *>(smem + lay.stat);
  if (tid < 8) sStat[tid] = 0;
  // A bounded wait gave up: the thread sets `fail` and the shared flag
  // sStat[7]; the iteration barrier counts it like an accepted bit, and a
  // nonzero count with the flag set ends the loop in every thread.
  int fail = 0;
  auto set_fail = [&]() {
    fail = 1;
    sStat[7] = 1;
  };
  int flip_streak = 0;  // consecutive flip iterations: no prefetch while hot
  // Control lane 0's copy bookkeeping: buffer b has a copy in flight when
  // pend >> b & 1; its mbarrier's next phase parity is ph >> b & 1.
  uint32_t pend = 0, ph = 0;
  // buffer of iteration t (warp A) and of t + LA (warp B): t % NB kept
  // by counting; the slot the previous flip wrote (warp B)
  int jb = NB > 1 ? 1 : 0;
  int pb_next = (int)((1u + (uint32_t)(LA > 0 ? LA : 0)) % (uint32_t)NB);
  uint32_t last_t = 0;
  int last_target = -1;
  // Fast-forward: sets or clears slot y's mark (control warp A, lane 0).
  auto mark_dead = [&](int y, bool on) {
    const uint32_t w = sDead[y >> 5], b = 1u << (y & 31);
    sDead[y >> 5] = on ? (w | b) : (w & ~b);
    sFF[1] += (int)on - (int)((w & b) != 0);
  };
  const uint32_t bits_lo = (uint32_t)(uintptr_t)gBits;  // low bits of the state array
  // Archive snapshots (Fig. mdasl), taken by control warp A alone: the
  // archive as it stood after iteration t is copied right after the
  // barrier of iteration t + 1 (or after the loop), in that iteration's
  // decision; it cannot change before then, and the next change (a flip's
  // writes) comes after a barrier this warp reaches only when the copy is
  // done.
  const bool snap = EXT && A.snap_every > 0;
  int32_t snap_left = A.snap_every;
  int32_t snap_j = 0;
  bool snap_mark = false;  // this iteration is followed by a snapshot
  bool snap_due = false;   // the previous one was
  auto take_snapshot = [&]() {
    const size_t row = (size_t)rb * (size_t)A.nsnap + (size_t)snap_j;
    int64_t *dE = A.snap_E + row * (size_t)s * 2;
    uint32_t *dB = A.snap_bits + row * (size_t)s * W;
    for (int e = lane; e < acount; e += 32) {
      const longlong2 v = aE[e];
      dE[2 * e] = v.x;
      dE[2 * e + 1] = v.y;
    }
    for (int e = lane; e < acount * W; e += 32) dB[e] = aBits[e];
    if (lane == 0) A.snap_count[row] = acount;
    ++snap_j;
    snap_due = false;
  };
  // schedule entry of the current iteration, in registers
  double cur_delta, cur_lod = 0, cur_hid = 0;
  float cur_deltaf;
  pen_t cur_lo, cur_hi;
  {
    const SchEntry e = sSch[1];
    cur_delta = e.delta;
    cur_deltaf = e.deltaf;
    cur_lo = NARROW ? (pen_t)e.lo32 : (pen_t)e.lo;
    cur_hi = NARROW ? (pen_t)e.hi32 : (pen_t)e.hi;
    if (NORM_ON) {
      cur_lod = e.lod;
      cur_hid = e.hid;
    }
  }

  for (uint32_t t = 1; t <= I_max; ++t) {
    const int buf = (int)(t & 1u);
    // this iteration's jump record: settled by warp A before the barrier,
    // read by the other warps after it
    JumpRec jr{kNone, 0, -1, 0, 0, 0, 0, 0};
    uint32_t *mask = sMask + buf * items;        // accept ballots

    bool acc_any = false;  // this thread accepted a bit
    if (worker) {
      // ---- workers: the parallel trial of their bits --------------------
      const double delta = cur_delta;
      const pen_t lo = cur_lo, hi = cur_hi;
      // 2 <= B <= 4: this lane's acceptance Philox block of the iteration
      bool drawn = false;
      uint32_t dc[4];
#pragma unroll
      for (int k = 0; k < B; ++k) {
        const dE_t e1 = D1[k], e2 = D2[k];
        if (NORM_ON) {
          const bool in = k * Tw + tid < m;
          const dE_t u1 = e1 > 0 ? e1 : 0, u2 = e2 > 0 ? e2 : 0;
          const pen_t ai = cAccept == 0 ? (pen_t)u1 + (pen_t)u2 : (pen_t)(u1 < u2 ? u1 : u2);
          bool acc = false, need = in;  // offset escape: every bit exactly
          if (cEscape == 0) {
            acc = in && ai <= lo;
            need = in && ai > lo && ai <= hi;
          }
          if (__any_sync(kFull, need)) {
            // a' = s_1 Delta E_1 (- E_off), ... in IEEE double, as written
            double x1 = __dmul_rn(A.s1, (double)e1), x2 = __dmul_rn(A.s2, (double)e2);
            if (cEscape == 1) {
              x1 = __dsub_rn(x1, (double)Eoff);
              x2 = __dsub_rn(x2, (double)Eoff);
            }
            const double b1 = x1 > 0 ? x1 : 0.0, b2 = x2 > 0 ? x2 : 0.0;
            const double ad = cAccept == 0 ? __dadd_rn(b1, b2) : (b1 < b2 ? b1 : b2);
            if (need && ad <= cur_lod) acc = true;
            const bool draw = need && ad > cur_lod && ad <= cur_hid;
            if (__any_sync(kFull, draw)) {
              const int p = k * Tw + tid;
              uint32_t c[4] = {(uint32_t)p >> 2, t, rep, kTagAccept};
              philox10(c, k0, k1);
              const uint32_t w = word_of(c, p & 3);
              if (draw) acc = ad <= __dmul_rn(delta, A.table[w >> 16]);
            }
          }
          if (acc && de_smem) {
            dE2_t v;
            v.x = e1;
            v.y = e2;
            sDE[k * Tw + tid] = v;
            sXb[k * Tw + tid] = (uint8_t)((xmask >> k) & 1u);
          }
          const uint32_t bal = __ballot_sync(kFull, acc);
          if (lane == 0) mask[k * NWB + warp] = bal;
          acc_any |= acc;
          continue;
        }
        dE_t a1, a2;
        if (cEscape == 1) {  // the offset lowers Delta E (Alg. 1)
          const dE_t off = NARROW ? (dE_t)(Eoff < 2147483647ll ? Eoff : 2147483647ll) : (dE_t)Eoff;
          a1 = e1 > off ? e1 - off : 0;
          a2 = e2 > off ? e2 - off : 0;
        } else {
          a1 = e1 > 0 ? e1 : 0;
          a2 = e2 > 0 ? e2 : 0;
        }
        const pen_t a = cAccept == 0 ? (pen_t)a1 + (pen_t)a2 : (pen_t)(a1 < a2 ? a1 : a2);
        const bool in = k * Tw + tid < m;
        bool acc = in && a <= lo;
        // a in (lo, hi]: the draw decides (warp-uniform branch; cold
        // iterations rarely take it)
        const bool need = in && a > lo && a <= hi;
        if (__any_sync(kFull, need)) {
          if (ff && lane == 0) sLive[t & 3u] = t;
          const int p = k * Tw + tid;
          uint32_t w;
          if (B == 1) {
            const uint32_t t0 = sDrawT[warp];
            if (t0 == 0u || t - t0 >= 4u) {
              uint32_t c[4] = {(uint32_t)(warp * 8 + (lane & 7)), t + (uint32_t)(lane >> 3), rep,
                               kTagAccept};
              philox10(c, k0, k1);
              sDraw[warp * 32 + lane] = make_uint4(c[0], c[1], c[2], c[3]);
              __syncwarp();
              if (lane == 0) sDrawT[warp] = t;
              w = reinterpret_cast<const uint32_t *>(sDraw)[(warp * 32 + (lane >> 2)) * 4 + (lane & 3)];
            } else {
              w = reinterpret_cast<const uint32_t *>(
                  sDraw)[(warp * 32 + (int)(t - t0) * 8 + (lane >> 2)) * 4 + (lane & 3)];
            }
            __syncwarp();
          } else if (B <= 4) {
            // The warp's bits of round k form 8 groups, so one block per
            // lane covers every round: lane l computes group l % 8 of round
            // l / 8 (once per iteration), and bit lane l of round k takes
            // word l % 4 from lane 8k + l / 4.
            if (!drawn) {
              const uint32_t kk = (uint32_t)(lane >> 3);
              dc[0] = (kk * (uint32_t)Tw + (uint32_t)warp * 32u) / 4u + (uint32_t)(lane & 7);
              dc[1] = t;
              dc[2] = rep;
              dc[3] = kTagAccept;
              philox10(dc, k0, k1);
              drawn = true;
            }
            const int src = k * 8 + (lane >> 2);
            const uint32_t v0 = __shfl_sync(kFull, dc[0], src), v1 = __shfl_sync(kFull, dc[1], src),
                           v2 = __shfl_sync(kFull, dc[2], src), v3 = __shfl_sync(kFull, dc[3], src);
            const int wi = lane & 3;
            w = wi == 0 ? v0 : wi == 1 ? v1 : wi == 2 ? v2 : v3;
          } else {
            uint32_t c[4] = {(uint32_t)p >> 2, t, rep, kTagAccept};
            philox10(c, k0, k1);
            w = word_of(c, p & 3);
          }
          if (need) {  // FP32 where exact, else the double test (prefilter)
            const uint32_t ix = w >> 16;
            const int r = prefilter(penalty_f32((int64_t)a), cur_deltaf, A.tablef[ix]);
            acc = r > 0 || (r < 0 && (double)a <= __dmul_rn(delta, A.table[ix]));
          }
        }
        if (acc && de_smem) {
          dE2_t v;
          v.x = e1;
          v.y = e2;
          sDE[k * Tw + tid] = v;
          sXb[k * Tw + tid] = (uint8_t)((xmask >> k) & 1u);
        }
        const uint32_t bal = __ballot_sync(kFull, acc);
        if (lane == 0) mask[k * NWB + warp] = bal;
        acc_any |= acc;
      }
    } else if (ctlA) {
      // ---- control warp A: draws, schedule, the jump record -------------
      if (t % 8u == 1u) fill_rings(t + 8);
      if (snap && --snap_left == 0) {  // iteration t ends with a snapshot
        snap_left = A.snap_every;
        snap_mark = true;
      }
      if (lane == 0) sWr[t & 7] = -1;  // set to the written slot by a flip below
      if (pf && LA == 0) bar_sync_pair();  // warp B recorded its copy for t
      // The jump iteration t makes if it accepts no bit (its draw and |A|
      // are known now).  Its copy is usable if it was started LA iterations
      // ago for this slot and no iteration since rewrote that slot.
      jr = JumpRec{kNone, 0, -1, 0, 0, 0, 0, 0};
      if (cEscape == 0 && acount > 0) {
        jr.kind = kJump;
        jr.slot = pick(sRnd[(t % kRing) * 4 + 1], acount);
        if (pf) {
          const PfRec rec = sPf[t & 7];
          bool ok = rec.iter != 0 && rec.slot == jr.slot && (uint32_t)rec.iter + LA == t;
          for (uint32_t x = (uint32_t)rec.iter; ok && x < t; ++x)
            if (sWr[x & 7] == jr.slot) ok = false;
          if (ok) {
            const uint32_t pb = (uint32_t)lay.pf + (uint32_t)jb * (uint32_t)lay.pf_slot;
            jr.pbuf = jb;
            jr.parity = (uint32_t)rec.parity;
            jr.rf = pb;
            jr.se = cEnergiesSmem ? (uint32_t)lay.archE + 16u * (uint32_t)jr.slot
                                       : pb + (uint32_t)lay.pfE;
            jr.ws = cBitsSmem
                        ? (uint32_t)lay.archB + 4u * (uint32_t)(jr.slot * W)
                        : pb + (uint32_t)lay.pfW + ((bits_lo + 4u * (uint32_t)(jr.slot * W)) & 15u);
            jr.bar = (uint32_t)lay.mbar + 8u * (uint32_t)jb;
          }
        }
      }
      if (ff) {
        // Every member is marked and iteration t tries one of them: no
        // bit is accepted in t or later, so t .. I_max all jump and the
        // run ends on the member iteration I_max draws.
        int fin = -1;
        if (lane == 0 && acount > 0 && sFF[1] == acount && sFF[0] >= 0) {
          uint32_t c[4] = {0u, I_max, rep, kTagRestart};
          philox10(c, k0, k1);
          fin = pick(c[0], acount);
        }
        fin = __shfl_sync(kFull, fin, 0);
        if (fin >= 0) jr = JumpRec{kFinish, fin, -1, 0, 0, 0, 0, 0};
      }
      if (lane == 0) sJr[t & 7] = jr;
      if (++jb == NB) jb = 0;
    } else {
      // ---- control warp B: the field-cache prefetch ---------------------
      if (pf && lane == 0) {
        // Copy for the jump iteration t + LA would make.  A slot written in
        // the previous iteration is left alone: its writes are ordered for
        // the copy engine only by a later barrier.
        const uint32_t tt = t + (uint32_t)LA;
        const int b = pb_next;
        bool issue = cEscape == 0 && acount > 0 && flip_streak < 3 && tt <= I_max;
        int slot_p = 0;
        if (issue) {
          slot_p = pick(sRnd[(tt % kRing) * 4 + 1], acount);
          if (last_t + 1 == t && last_target == slot_p) issue = false;
        }
        uint32_t par = 0;
        if (issue) {
          if ((pend >> b) & 1u) {  // retire the unused copy in this buffer
            if (!mbar_wait(&sBar[b], (ph >> b) & 1u)) set_fail();
            ph ^= 1u << b;
            pend &= ~(1u << b);
          }
          unsigned char *pb = smem + lay.pf + (size_t)b * lay.pf_slot;
          uint32_t eb = 0, bb = 0, boff = 0;
          if (!cEnergiesSmem) eb = 16;
          if (!cBitsSmem) {
            boff = (bits_lo + 4u * (uint32_t)(slot_p * W)) & 15u;
            bb = (boff + 4u * (uint32_t)W + 15u) & ~15u;
          }
          fence_proxy_async_shared();
          mbar_expect_tx(&sBar[b], (uint32_t)sl.bytes + eb + bb);
          bulk_g2s(pb, gF + (size_t)slot_p * sl.bytes, (uint32_t)sl.bytes, &sBar[b]);
          if (eb) bulk_g2s(pb + lay.pfE, gE + 2 * (size_t)slot_p, 16, &sBar[b]);
          if (bb)
            bulk_g2s(pb + lay.pfW,
                     reinterpret_cast<const unsigned char *>(gBits + (size_t)slot_p * W) - boff,
                     bb, &sBar[b]);
          par = (ph >> b) & 1u;
          pend |= 1u << b;
        }
        sPf[tt & 7] = PfRec{issue ? (int)t : 0, slot_p, (int)par, 0};
      } else if (!NARROW && fc && lane == 0 && cEscape == 0 && acount > 0 &&
                 t + 2 <= I_max) {
        // Records read in place (no prefetch buffers; the large 16-byte
        // records of the int64 variant): bring the record and state of the
        // member a jump two iterations ahead would land on into L2.  Only a
        // hint -- the jump reads the current data anyway.
        const uint32_t tt = t + 2;
        const int slot_p = pick(sRnd[(tt % kRing) * 4 + 1], acount);
        bulk_prefetch_l2(gF + (size_t)slot_p * sl.bytes, (uint32_t)sl.bytes);
        if (!cBitsSmem) {
          const uint32_t boff = (bits_lo + 4u * (uint32_t)(slot_p * W)) & 15u;
          bulk_prefetch_l2(reinterpret_cast<const unsigned char *>(gBits + (size_t)slot_p * W) - boff,
                           (boff + 4u * (uint32_t)W + 15u) & ~15u);
        }
      }
      if (++pb_next == NB) pb_next = 0;
      if (pf && LA == 0) {
        __syncwarp();
        bar_sync_pair();  // the copy for t is recorded for warp A
      }
    }
    // The barrier counts the threads that accepted a bit (or gave up a
    // wait): 0 means no bit was accepted, the common case once the
    // schedule has cooled, settled without reading the ballots.
    const int nacc = __syncthreads_count(acc_any || fail);
    if (nacc > 0 && sStat[7]) break;  // a bounded wait gave up (uniform)
    // schedule entry of the next iteration, loaded early
    const SchEntry nse = sSch[(t + 1) % kRing];

    // ---- every warp: the decision (the same in all of them) -------------
    const uint32_t *rnd = sRnd + (t % kRing) * 4;
    int kind, ps = 0;
    {
      if (worker) {
        if (nacc > 0) {
          kind = kFlip;
          int cnt = 0;
#pragma unroll
          for (int q = 0; q < B; ++q) {  // items <= B * 31, so per <= B
            const int it = lane * per + q;
            if (q < per && it < items) cnt += __popc(mask[it]);
          }
          // one bit per thread: the count is the number of accepted bits
          const int total = B == 1 ? nacc : (int)__reduce_add_sync(kFull, (unsigned)cnt);
          const int incl = warp_incl_scan(cnt, lane);
          ps = warp_mask_select(mask, items, NWB, Tw, lane, incl, cnt, pick(rnd[0], total));
        } else {
          jr = sJr[t & 7];
          kind = jr.kind;
        }
      } else if (ctlA) {
        kind = nacc > 0 ? kFlip : jr.kind;
        // the state tried in t is member sFF[0] and no penalty was <= hi
        if (ff && nacc == 0 && lane == 0 && sFF[0] >= 0 && sLive[t & 3u] != t)
          mark_dead(sFF[0], true);
        // the archive as it stood after the previous iteration
        if (snap_due) take_snapshot();
        snap_due = snap_mark;
        snap_mark = false;
      } else {
        if (nacc == 0) jr = sJr[t & 7];  // settled by warp A
        kind = nacc > 0 ? kFlip : jr.kind;
        if (nacc == 0 && lane == 0 && jr.pbuf >= 0) {  // the copy is consumed
          ph ^= 1u << jr.pbuf;
          pend &= ~(1u << jr.pbuf);
        }
      }
    }

    // ---- all: carry out the decision ------------------------------------
    if (kind == kFlip) {
      int64_t dE1, dE2;
      int sg;
      if (de_smem) {
        const dE2_t v = sDE[ps];
        dE1 = (int64_t)v.x;
        dE2 = (int64_t)v.y;
        // ballot word of bit ps: (round, warp) = ps / 32 because Tw % 32 == 0
        sg = 1 - 2 * (int)sXb[ps];
      } else {
        const int kk = ps / Tw;
        if (ps - kk * Tw == tid) {  // the owner publishes Delta E and its sign
#pragma unroll
          for (int k = 0; k < B; ++k) {
            if (k != kk) continue;
            bc->dE1 = (int64_t)D1[k];
            bc->dE2 = (int64_t)D2[k];
            bc->sgn = 1 - 2 * (int)((xmask >> k) & 1u);
          }
        }
        __syncthreads();
        dE1 = bc->dE1;
        dE2 = bc->dE2;
        sg = bc->sgn;
      }
      const int64_t nE1 = E1 + dE1, nE2 = E2 + dE2;
      const int j = (int)__umulhi((uint32_t)ps, A.magic);
      const int v = ps - j * n;
      int anyd = 0;
      if (worker) {
        // Delta E after flipping (j, v): the flipped bit's changes sign;
        // every other bit q = (i, u) gains (1 - 2 x_q) s P_qp with
        // P_qp = Fs^k_ij d_uv + w_k [i == j or u == v] (Eq. cale, Y / Z).
#pragma unroll
        for (int k = 0; k < B; ++k) {
          if (k * Tw + tid >= m) continue;
          if (k * Tw + tid == ps) {
            D1[k] = -D1[k];
            D2[k] = -D2[k];
            xmask ^= 1u << k;
            continue;
          }
          const int i = own[k] >> 8, u = own[k] & 255;
          const int2 f = sFs[j * n + i];
          const int32_t dd = sD[v * n + u];
          const bool coupled = (i == j) | (u == v);
          const int gs = sg * (1 - 2 * (int)((xmask >> k) & 1u));
          D1[k] += (dE_t)gs * ((dE_t)(f.x * dd) + (coupled ? w1 : (dE_t)0));
          D2[k] += (dE_t)gs * ((dE_t)(f.y * dd) + (coupled ? w2 : (dE_t)0));
        }
        // Archive: ballots of "x dominates slot y" in slot order, and (for
        // the exploitative update) whether some member dominates x.
#pragma unroll
        for (int k = 0; k < B; ++k) {
          const int y = k * Tw + tid;
          bool dom = false;
          if (y < acount) {
            const longlong2 ye = aE[y];
            dom = dominates(nE1, nE2, ye.x, ye.y);
            if (dominates(ye.x, ye.y, nE1, nE2)) anyd = 1;
          }
          const uint32_t bal = __ballot_sync(kFull, dom);
          if (lane == 0) sAmask[k * NWB + warp] = bal;
        }
      }
      anyd = __syncthreads_or(anyd);
      int target = -1;
      if (cArchive == 0) {
        // Alg. 4: replace the first dominated member, else append.
        target = warp_mask_first(sAmask, items, NWB, Tw, lane);
        if (target < 0 && acount < s) target = acount++;
      } else if (!anyd) {
        // Alg. 5: replace a random dominated member, else append.
        int aincl, acnt;
        const int nb = warp_mask_total(sAmask, items, lane, aincl, acnt);
        if (nb > 0)
          target = warp_mask_select(sAmask, items, NWB, Tw, lane, aincl, acnt,
                                    pick(rnd[2], nb));
        else if (acount < s)
          target = acount++;
      }
      if (target >= 0) {
        if (worker) {
#pragma unroll
          for (int k = 0; k < B; ++k) {
            const uint32_t wv = __ballot_sync(kFull, (xmask >> k) & 1u);
            const int wi = k * NWB + warp;
            if (lane == 0 && wi < W) aBits[(size_t)target * W + wi] = wv;
          }
          if (tid == 0) aE[target] = make_longlong2(nE1, nE2);
          if (fc) {
            dE2_t *rf = reinterpret_cast<dE2_t *>(gF + (size_t)target * sl.bytes);
#pragma unroll
            for (int k = 0; k < B; ++k) {
              const int q = k * Tw + tid;
              if (q >= m) continue;
              dE2_t v2;
              v2.x = D1[k];
              v2.y = D2[k];
              rf[q] = v2;
            }
            fence_proxy_async_global();  // later bulk copies read these
          }
        } else {
          if (ctlA && pf && lane == 0) sWr[t & 7] = target;
          last_target = target;
          last_t = t;
        }
      }
      if (ff && ctlA && lane == 0) {  // the new state is member `target` (if stored)
        if (target >= 0) mark_dead(target, false);
        sFF[0] = target;
      }
      E1 = nE1;
      E2 = nE2;
      Eoff = 0;
      if (ctlA && lane == 0) ++sStat[0];
    } else if (kind == kJump) {
      // Alg. 3: jump to a random archive member.
      const int slot = jr.slot, pbuf = jr.pbuf;
      if (fc) {
        if (worker) {
          if (pbuf >= 0) {  // from the prefetch buffer (shared memory)
            if (!mbar_wait(reinterpret_cast<uint64_t *>(smem + jr.bar), jr.parity)) set_fail();
            const dE2_t *rf = reinterpret_cast<const dE2_t *>(smem + jr.rf);
            const uint32_t *ws = reinterpret_cast<const uint32_t *>(smem + jr.ws);
            const longlong2 se = *reinterpret_cast<const longlong2 *>(smem + jr.se);
            E1 = se.x;
            E2 = se.y;
            xmask = 0;
#pragma unroll
            for (int k = 0; k < B; ++k) {
              if (!valid(k)) continue;
              const dE2_t v2 = rf[k * Tw + tid];
              D1[k] = v2.x;
              D2[k] = v2.y;
              xmask |= ((ws[k * NWB + warp] >> lane) & 1u) << k;
            }
          } else {  // read the record where it is
            const dE2_t *rf = reinterpret_cast<const dE2_t *>(gF + (size_t)slot * sl.bytes);
            const uint32_t *wsrc = aBits + (size_t)slot * W;
            const longlong2 se = aE[slot];
            E1 = se.x;
            E2 = se.y;
            xmask = 0;
#pragma unroll
            for (int k = 0; k < B; ++k) {
              if (!valid(k)) continue;
              const dE2_t v2 = rf[k * Tw + tid];
              D1[k] = v2.x;
              D2[k] = v2.y;
              xmask |= ((wsrc[k * NWB + warp] >> lane) & 1u) << k;
            }
          }
        } else if (pbuf >= 0) {
          if (ctlA && lane == 0) ++sStat[4];
        } else {
          if (ctlA && lane == 0) ++sStat[5];
        }
      } else {
        const longlong2 se = aE[slot];
        E1 = se.x;
        E2 = se.y;
        int64_t s1, s2;
        rebuild(aBits + (size_t)slot * W, s1, s2);
      }
      if (ctlA && lane == 0) ++sStat[1];
      if (ff && ctlA && lane == 0) sFF[0] = slot;
    } else if (ff && kind == kFinish) {
      // Iterations t .. I_max each jump to the member their draw picks
      // (the archive no longer changes); the state ends as member
      // jr.slot.  Delta E is not needed any more.
      const int slot = jr.slot;
      const longlong2 se = aE[slot];
      E1 = se.x;
      E2 = se.y;
      if (worker) {
        const uint32_t *wsrc = aBits + (size_t)slot * W;
        xmask = 0;
#pragma unroll
        for (int k = 0; k < B; ++k)
          if (valid(k)) xmask |= ((wsrc[k * NWB + warp] >> lane) & 1u) << k;
      }
      if (cTrace != nullptr) {
        for (uint64_t q = (uint64_t)t + (uint64_t)tid; q <= (uint64_t)I_max; q += (uint64_t)T) {
          uint32_t c[4] = {0u, (uint32_t)q, rep, kTagRestart};
          philox10(c, k0, k1);
          const int y = pick(c[0], acount);
          const longlong2 v = aE[y];
          int64_t *tr = cTrace + ((size_t)rb * (size_t)I_max + (size_t)(q - 1)) * 3;
          tr[0] = v.x;
          tr[1] = v.y;
          tr[2] = -1 - (int64_t)y;
        }
      }
      if (ctlA && lane == 0) {
        sStat[1] += I_max - t + 1;
        sStat[6] = I_max - t;
      }
      break;
    } else if (cEscape == 0) {
      if (ctlA && lane == 0) ++sStat[2];
    } else {
      Eoff += A.beta;
      if (ctlA && lane == 0) ++sStat[3];
    }
    if (ctlB) flip_streak = kind == kFlip ? flip_streak + 1 : 0;
    cur_delta = nse.delta;
    cur_deltaf = nse.deltaf;
    cur_lo = NARROW ? (pen_t)nse.lo32 : (pen_t)nse.lo;
    cur_hi = NARROW ? (pen_t)nse.hi32 : (pen_t)nse.hi;
    if (NORM_ON) {
      cur_lod = nse.lod;
      cur_hid = nse.hid;
    }
    if (cTrace != nullptr && tid == 0) {
      int64_t *tr = cTrace + ((size_t)rb * (size_t)I_max + (size_t)(t - 1)) * 3;
      tr[0] = E1;
      tr[1] = E2;
      tr[2] = kind == kFlip ? (int64_t)ps : kind == kJump ? -1 - (int64_t)jr.slot : INT64_MIN;
    }
  }
  __syncthreads();  // the last iteration's archive writes
  if (ctlA && (snap_due || snap_mark)) take_snapshot();
  // No bulk copy may be in flight when the block exits.
  if (pf && ctlB && lane == 0) {
    for (int b = 0; b < NB; ++b)
      if ((pend >> b) & 1u)
        if (!mbar_wait(&sBar[b], (ph >> b) & 1u)) fail = 1;
  }
  if (__syncthreads_or(fail) && tid == 0) atomicExch(A.error, kErrCopyTimeout);
  if (worker) {
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const uint32_t wv = __ballot_sync(kFull, (xmask >> k) & 1u);
      const int wi = k * NWB + warp;
      if (lane == 0 && wi < W) A.x_final[(size_t)rb * W + wi] = wv;
    }
  }
  if (cEnergiesSmem) {
    for (int e = tid; e < acount; e += T) {
      const longlong2 v = aE[e];
      gE[2 * e] = v.x;
      gE[2 * e + 1] = v.y;
    }
  }
  if (cBitsSmem) {
    for (int e = tid; e < acount * W; e += T) gBits[e] = aBits[e];
  }
  if (tid == Tw) {  // control warp A counted the outcomes
    int64_t *st = A.stats + (size_t)kStats * rb;
    for (int q = 0; q < 7; ++q) st[q] = sStat[q];
    st[7] = 0;
    A.arch_count[rb] = acount;
  }
  if (tid == 0) {  // workers track the energies
    A.E_final[2 * rb] = E1;
    A.E_final[2 * rb + 1] = E2;
  }
}

template <int B, bool NARROW, int MODE>
cudaError_t launch_bn(const AnnealArgs &args, int replicas, int workers,
                      size_t smem, cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(
      anneal_kernel<B, NARROW, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  anneal_kernel<B, NARROW, MODE><<<replicas, workers + 64, smem, stream>>>(args);
  return cudaGetLastError();
}

template <int B, bool NARROW, int MODE>
const void *kernel_ptr() {
  return reinterpret_cast<const void *>(anneal_kernel<B, NARROW, MODE>);
}

}  // namespace
}  // namespace moda
