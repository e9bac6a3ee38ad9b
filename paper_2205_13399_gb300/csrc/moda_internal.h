// Internal declarations shared by the host library (moda_api.cu,
// moda_noalloc.cu) and the annealing kernel (moda_kernel.cu).  Not part of
// the public C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

namespace moda {

constexpr int kMaxN = 128;          // n <= 128: a bit index fits (i << 8) | u
constexpr int kMaxThreads = 1024;   // threads of a block, control warps included
constexpr int kMaxWorkers = kMaxThreads - 64;
constexpr int kTableSize = 65536;   // -ln(u) table, u quantised to 2^-16
constexpr int kMaxLookahead = 3;    // field-cache prefetch distance
constexpr int kStats = 8;           // counters per replica (see moda.h)

// Purposes of a Philox draw (fourth counter word).
enum : uint32_t { kTagAccept = 0, kTagSelect = 1, kTagRestart = 2,
                  kTagExploit = 3, kTagInit = 4 };

// Device status codes written to AnnealArgs::error.
// kErrVariant: a kernel variant was launched for a run it does not fit.
enum : int32_t { kErrNone = 0, kErrCopyTimeout = 1, kErrVariant = 2 };

__host__ __device__ inline size_t align_up(size_t v, size_t a) {
  return (v + a - 1) / a * a;
}

// Per-slot record of the field cache: (Delta E_1, Delta E_2) of every bit
// of the member's state, as int32 pairs (narrow variant) or int64 pairs.
struct SlotLayout {
  size_t bytes;
};
__host__ __device__ inline SlotLayout slot_layout(int m, bool narrow) {
  SlotLayout S;
  S.bytes = (narrow ? 8 : 16) * align_up((size_t)m, 8);
  return S;
}

// Everything one launch of the annealing kernel needs.  All pointers are
// device pointers.
struct AnnealArgs {
  int32_t n, m, W;          // W = ceil(m / 32) words per bit vector
  int32_t s;                // archive capacity
  int64_t I_max;
  uint32_t replica_base;
  uint32_t seed_lo, seed_hi;
  uint32_t magic;           // ceil(2^32 / n): q / n = umulhi(q, magic), q < 2^14
  int64_t w1, w2;           // penalty weights, alpha_k = w_k / 2
  int64_t beta;
  int32_t accept, archive, escape;
  int32_t nsched;           // entries of the schedule; later iterations
                            // reuse the last one
  int32_t energies_in_smem; // archive energies kept in shared memory
  int32_t bits_in_smem;     // archive states kept in shared memory
  int32_t lookahead;        // field-cache prefetch distance (iterations)
  int32_t de_in_smem;       // accepted bits publish Delta E in shared memory
  int32_t normalize;        // Sec. 4.2 normalisation in the acceptance test
  double s1, s2;            // its per-objective scales (1 when off)
  double tmin, tmax;        // -ln(u) at the largest and smallest u
  int32_t snap_every;       // > 0: archive snapshot after every such iteration
  int32_t nsnap;            // I_max / snap_every
  int32_t *snap_count;      // [R][nsnap]
  int64_t *snap_E;          // [R][nsnap][s][2]
  uint32_t *snap_bits;      // [R][nsnap][s][W]
  const double *sch_delta;  // [nsched] delta_t, t = 1..nsched
  const int64_t *sch_lo;    // [nsched] floor(delta_t * T_min): a <= lo accepts
  const int64_t *sch_hi;    // [nsched] floor(delta_t * T_max): a > hi rejects
  const double *table;      // [65536] -ln((idx + 0.5) / 65536)
  const float *tablef;      // [65536] the same rounded to float (FP32 test)
  const int32_t *Fs1, *Fs2; // [n][n] F_k + F_k^T (symmetric)
  const int32_t *D;         // [n][n] symmetric distances, zero diagonal
  // Field cache, [R][s] records of slot_layout(m, narrow).bytes, or
  // nullptr: Delta E of every bit of every archive member, written when
  // the member is stored and brought back by a bulk copy (TMA), started up
  // to `lookahead` iterations early, when the replica jumps to it.
  unsigned char *fcache;
  // outputs, one block per replica of this launch
  int64_t *arch_E;          // [R][s][2]
  uint32_t *arch_bits;      // [R][s][W] (+ 32 spare bytes)
  int32_t *arch_count;      // [R]
  uint32_t *x_final;        // [R][W]
  int64_t *E_final;         // [R][2]
  int64_t *stats;           // [R][kStats]
  int64_t *trace;           // [R][I_max][3] or nullptr
  int32_t *error;           // device status word, kErrNone = fine
  // 1: stop once every archive member is known unable to accept and the
  // state about to be tried is a member (moda_params.fast_forward)
  int32_t fast_forward;
};

// Placement choices of one launch (decided on the host).
struct Placement {
  bool energies_in_smem;  // archive energies on chip
  bool bits_in_smem;      // archive states on chip
  bool field_cache;       // jumps reload cached fields
  int lookahead;          // prefetch distance, iterations
  bool de_in_smem;        // accepted bits publish Delta E in shared memory
  bool narrow;            // Delta E fits int32 (kernel variant)
  bool ff;                // fast-forward bookkeeping (moda_params.fast_forward)
};

// Byte offsets of the shared-memory carve-up of one annealing block with
// `workers` bit-owning threads (plus one control warp).
struct SmemLayout {
  size_t Fs, D, M, mask, amask, rnd, sch, RC, red, bc, jr, stat, ff, draw, init, mbar, dE,
      pf, pf_slot, pfE, pfW, archE, archB, total;
};

__host__ __device__ inline SmemLayout smem_layout(int n, int m, int W, int s,
                                                  int workers, int rounds,
                                                  const Placement &P) {
  SmemLayout L;
  size_t o = 0;
  const size_t nn = (size_t)n * n;
  const size_t items = (size_t)rounds * (workers / 32);
  const size_t bits = (size_t)rounds * workers;
  L.Fs = o;    o = align_up(o + 8 * nn, 16);                 // int2 pairs
  L.D = o;     o = align_up(o + 4 * nn, 16);
  L.mask = o;  o = align_up(o + 4 * 2 * items, 16);  // accept ballots x 2
  L.amask = o; o = align_up(o + 4 * items, 16);
  L.rnd = o;   o = align_up(o + 32 * 4 * 4, 16);             // 32 iterations
  L.sch = o;   o = align_up(o + 32 * 56, 16);                // 32 entries
  L.RC = o;    o = align_up(o + 4 * 4 * (size_t)n, 16);      // 2 x (R, C)
  L.red = o;   o = align_up(o + 8 * 32, 16);
  L.bc = o;    o = align_up(o + 32, 16);
  L.jr = o;    o = align_up(o + 8 * 32, 16);                 // 8 entries
  L.stat = o;  o = align_up(o + 8 * 4, 16);                  // counters
  // fast-forward: 4 iteration stamps, 4 words of bookkeeping, then one
  // bit per archive slot
  L.ff = o;    if (P.ff) o = align_up(o + 4 * (8 + ((size_t)s + 31) / 32), 16);
  // one bit per thread: each warp's acceptance draws of 4 iterations (one
  // Philox block per lane), then the first iteration they cover
  L.draw = o;  if (rounds == 1) o = align_up(o + 16 * (size_t)workers + 4 * (workers / 32), 16);
  L.init = o;  o = align_up(o + 4 * (size_t)W, 16);
  L.mbar = o;  o = align_up(o + 8 * (kMaxLookahead + 2), 16);
  L.dE = o;    if (P.de_in_smem) o = align_up(o + (P.narrow ? 8 : 16) * bits + bits, 16);  // + state bytes
  // Prefetch buffers (lookahead + 2: the one being filled, the one of the
  // current iteration and the one a lagging warp may still read): one
  // field-cache record, then the member's energies and the 16-byte-aligned
  // span of its state words when those live in HBM.  M = X * D (only used
  // by rebuilds, which never overlap a prefetch) shares this space.
  L.pfE = slot_layout(m, P.narrow).bytes;
  L.pfW = L.pfE + (P.energies_in_smem ? 0 : 16);
  L.pf_slot = align_up(L.pfW + (P.bits_in_smem ? 0 : align_up(4 * (size_t)W, 16) + 16), 16);
  L.pf = o;
  size_t pf_bytes = P.field_cache && P.lookahead >= 0
                        ? L.pf_slot * (size_t)(P.lookahead + 2) : 0;
  if (pf_bytes < 4 * nn) pf_bytes = 4 * nn;
  L.M = o;
  o = align_up(o + pf_bytes, 16);
  L.archE = o; if (P.energies_in_smem) o = align_up(o + 16 * (size_t)s, 16);
  L.archB = o; if (P.bits_in_smem) o = align_up(o + 4 * (size_t)s * W, 16);
  L.total = o;
  return L;
}

// True when every |Delta E_k| stays below 2^31 for every state:
// |Delta E_k| <= B_k + w_k (2n + 1), B_k the bound of the fields.  The
// kernel then keeps Delta E in int32 and the acceptance penalty (a sum of
// two values in [0, 2^31)) in uint32.
inline bool narrow_ok(int n, int64_t b1, int64_t b2, int64_t w1, int64_t w2) {
  const long double e1 = (long double)b1 + (long double)w1 * (2 * n + 1);
  const long double e2 = (long double)b2 + (long double)w2 * (2 * n + 1);
  return e1 < 2147483647.0L && e2 < 2147483647.0L;
}

// Sec. 4.2 normalisation: objective k's scale 2^23 / (largest coefficient
// of its cost QUBO), that coefficient being max Fs^k_ij * max d_uv for
// non-negative flows and distances; 1 for an objective without cost.
inline double norm_scale(int64_t max_coef) {
  return max_coef > 0 ? 8388608.0 / (double)max_coef : 1.0;
}

// Normalisation or snapshots: the kernel variant that carries them.
inline bool uses_extensions(const AnnealArgs &a) {
  return a.normalize != 0 || a.snap_every > 0;
}

// Kernel variant of a launch with `rounds` bits per thread: 1 with the
// extensions, 2 with the fast-forward bookkeeping (never together with an
// extension), 3 the default algorithm (strict acceptance, Alg. 4 archive,
// archive escape, no trace) compiled in, 4 that and the on-chip placement
// (one bit per thread, field cache with prefetch distance 1, archive and
// published Delta E in shared memory), 5 the same placement with the
// archive states in global memory (2 to 4 bits per thread), else 0.
inline int kernel_mode(const AnnealArgs &a, int rounds) {
  if (uses_extensions(a)) return 1;
  if (a.fast_forward) return 2;
  if (a.accept == 0 && a.archive == 0 && a.escape == 0 && a.trace == nullptr) {
    if (a.lookahead == 1 && a.de_in_smem && a.energies_in_smem && a.fcache != nullptr) {
      if (rounds == 1 && a.bits_in_smem) return 4;
      if (rounds >= 2 && rounds <= 4 && !a.bits_in_smem) return 5;
    }
    return 3;
  }
  return 0;
}

// Bits per thread the kernel is instantiated for.
bool supported_rounds(int b);

// Launch one block of `workers` + 64 threads per replica on `stream`.
cudaError_t launch_anneal(const AnnealArgs &args, int replicas, int workers,
                          int rounds, bool narrow, size_t smem_bytes,
                          cudaStream_t stream);

// The kernel for `rounds` bits per thread (one block of workers + 64
// threads, two control warps, per replica, `smem` bytes of dynamic shared memory, which this
// call allows), for launching from a CUDA graph node with one AnnealArgs
// argument.
cudaError_t anneal_function(int rounds, bool narrow, int mode, size_t smem,
                            const void **func);

// Modes 2 to 4 of launch_anneal and anneal_function (a second translation
// unit, moda_kernel_special.cu).
cudaError_t launch_anneal_special(const AnnealArgs &args, int replicas, int workers, int rounds,
                                  bool narrow, int mode, size_t smem, cudaStream_t stream);
cudaError_t anneal_function_special(int rounds, bool narrow, int mode, size_t smem,
                                    const void **func);

// ---- the warp annealer: a team of G warps per replica ----------------------
//
// A throughput form of the same loop: each team of G warps (G = 1 .. 8)
// runs one replica, synchronised by a named barrier of its own (no block
// barriers), pulling (run, replica) work items from a device list.  Warp w
// of a team owns a contiguous range of 128-bit chunks; bit p of a chunk
// belongs to lane (p % 128) / 4, so a lane holds 4 consecutive bits of
// each chunk (one acceptance Philox block: bits 4g .. 4g + 3 take the words
// of block g).  The state a trial
// reads is, per bit, its acceptance penalty a (strict: sum_k max(0, dE_k);
// lenient: min_k max(0, dE_k)) saturated to uint32; the integer cost fields
// L_k (int32 pairs) live in global memory and are read only by flips.

constexpr int kWarpRing = 128;  // draw / schedule ring entries (iterations)
constexpr int kWarpMaxLA = 14;  // prefetch distance (iterations ahead)

// Records of one archive slot for a run of n, m (the field cache of the
// warp annealer):
//   jump record  a[mp] uint32 penalties, the candidate masks [mp / 32],
//                the state words [mp / 32], the row and column counts [2n]
//                uint8 (16-byte padded), (E1, E2) int64 -- brought into
//                shared memory by one bulk copy when the replica jumps to
//                the slot (once the schedule is frozen, the header alone:
//                the masks say which penalties can still be accepted);
//   field record (L1, L2) int32 pairs [mp].
// mp = 128 ceil(m / 128): bits past m carry a = 0xFFFFFFFF and no state.
struct WarpRec {
  int32_t nc, mp;                        // chunks of 128 bits, padded bits
  uint32_t off_cm;                       // candidate masks (the header starts here)
  uint32_t off_xw, off_rc, off_E, jr;    // jump-record offsets and bytes
  uint32_t hb;                           // header bytes: jr - off_cm
  uint32_t lr;                           // field-record bytes
};
// Jump record: the penalties a(p) (uint32 each), then the header: per chunk
// four 32-bit candidate masks (word j, bit l: bit 128 c + 4 l + j has
// a <= hi of the frozen schedule), the state words, the row and column
// counts and the energies.  Every part starts on a 16-byte boundary.
__host__ __device__ inline WarpRec warp_rec(int n, int m) {
  WarpRec r;
  r.nc = (m + 127) / 128;
  r.mp = 128 * r.nc;
  r.off_cm = 4u * (uint32_t)r.mp;
  r.off_xw = r.off_cm + (uint32_t)(r.mp / 8);
  r.off_rc = r.off_xw + 4u * (uint32_t)(r.mp / 32);
  r.off_E = r.off_rc + (uint32_t)align_up((size_t)(2 * n), 16);
  r.jr = r.off_E + 16u;
  r.hb = r.jr - r.off_cm;
  r.lr = 8u * (uint32_t)r.mp;
  return r;
}

// Shared-memory carve-up of one team (the G warps that run one replica),
// sized for the largest run of a launch: nbuf jump-record buffers, their
// mbarriers, the ring of draws and schedule entries, the archive energies
// of slots < se, the prefetch bookkeeping and the warps' accepted counts;
// then per warp its accepted-chunk list, the flow and distance rows of a
// flip and its copy of the row and column counts.
struct WarpSmem {
  uint32_t jr;     // buffer stride
  uint32_t scr, hbuf;  // frozen layout, from buf: rebuild scratch, header buffers
  uint32_t buf, mbar, ring, aE, cnt, fld, team;   // team part (bytes: team)
  uint32_t acc, rows, rc, pf, tbl, warp;          // warp part (bytes: warp)
  int32_t nc_max;
  int32_t pfr;     // per-target record ring entries: 16, or 32 past 16 buffers
  int32_t cst;     // ints per round parity of the counts: 8 (window + 1)
  uint32_t total;  // team + G warps
};
// stage: each warp owns at most two chunks of the largest run (then the
// -ln(u) values of the draws after a flip are staged on chip).
__host__ __device__ inline bool warp_stage(int m_max, int G) {
  return (m_max + 127) / 128 <= 2 * G;
}
// sfields: the team part also holds the fields of the state a flip
// reached (8 bytes per bit), so that flips following flips read them on chip.
// nbuf_f > 0: the frozen layout's header buffers (window_f iterations), in
// the same region: one full record, a rebuild scratch, nbuf_f headers.
__host__ __device__ inline WarpSmem warp_smem(int n_max, int m_max, int se_max, int nbuf, int G,
                                              bool sfields, int window, int nbuf_f = 0,
                                              int window_f = 1) {
  const WarpRec r = warp_rec(n_max, m_max);
  WarpSmem L;
  size_t o = 0;
  L.jr = r.jr;
  L.nc_max = r.nc;
  const int nb_max = nbuf > nbuf_f ? nbuf : nbuf_f;
  const int w_max = window > window_f ? window : window_f;
  L.pfr = nb_max <= 16 ? 16 : 32;  // holds targets t .. t + window - 1 + lookahead
  L.cst = 8 * (w_max + 1);
  L.scr = r.jr;
  L.hbuf = r.jr + (uint32_t)align_up(4 * (size_t)m_max, 16);
  size_t region = (size_t)nbuf * r.jr;
  if (nbuf_f > 0 && L.hbuf + (size_t)nbuf_f * r.hb > region) region = L.hbuf + (size_t)nbuf_f * r.hb;
  L.buf = 0;                 o = align_up(o + region, 16);
  L.mbar = (uint32_t)o;      o = align_up(o + 8 * (size_t)nb_max, 16);
  L.ring = (uint32_t)o;      o = align_up(o + 40 * (size_t)kWarpRing, 16);
  L.aE = (uint32_t)o;        o = align_up(o + 16 * (size_t)se_max, 16);
  // accepted counts of the warps by round parity [2][window positions +
  // 1][8], the work item, the warps' partial sums of a rebuild [8][2], the
  // warps' first dominated archive slots by round parity [2][8]
  L.cnt = (uint32_t)o;       o = align_up(o + 8 * (size_t)L.cst + 16 + 128 + 64, 16);
  L.fld = (uint32_t)o;       if (sfields) o = align_up(o + 8 * (size_t)r.mp, 16);
  L.team = (uint32_t)o;
  o = 0;
  L.acc = 0;                 o = align_up(o + 20 * (size_t)r.nc, 16);
  L.rows = (uint32_t)o;      o = align_up(o + 3 * 4 * (size_t)kMaxN, 16);
  L.rc = (uint32_t)o;        o = align_up(o + 2 * (size_t)kMaxN, 16);
  L.pf = (uint32_t)o;        o = align_up(o + 20 * (size_t)L.pfr, 16);
  L.tbl = (uint32_t)o;       // staged -ln(u), 2 chunks
  if (warp_stage(m_max, G)) o = align_up(o + 8 * 4 * 32 * 2, 16);
  L.warp = (uint32_t)o;
  L.total = L.team + (uint32_t)G * L.warp;
  return L;
}

// One run of a warp-annealer launch (device memory; every pointer a
// device pointer).
struct WarpRun {
  int32_t n, m, W, s;
  int32_t cslots;            // slots < cslots have field-cache records; a
                             // jump to a later slot rebuilds the fields
  int32_t se;                // archive energies of slots < se on chip
  int32_t narrow;            // |Delta E_k| < 2^31 for every state
  int32_t accept, archive;   // moda_accept, moda_archive (escape: archive)
  int32_t nsched, replicas;
  uint32_t replica_base, seed_lo, seed_hi, magic;
  int32_t pad;
  int64_t I_max;
  int64_t w1, w2;
  const double *sch_delta;
  const int64_t *sch_lo, *sch_hi;
  const double *table;
  const float *tablef;       // table rounded to float: the FP32 prefilter
  const int32_t *Fs1, *Fs2, *D;
  int64_t *arch_E;
  uint32_t *arch_bits;
  int32_t *arch_count;
  uint32_t *x_final;
  int64_t *E_final;
  int64_t *stats;
  int64_t *trace;            // [R][I_max][3] or nullptr
  int32_t *error;
};

// Kernel argument of a warp-annealer launch.
struct WarpLaunch {
  const WarpRun *runs;
  const int2 *items;         // (run, replica row), largest runs first
  int32_t nitems;
  int32_t nbuf;              // jump-record buffers per team: lookahead + window + 1
  // the frozen layout (nbuf_f > 0): header buffers, prefetch distance and
  // window once the schedule no longer changes
  int32_t nbuf_f, lookahead_f, window_f;
  int32_t lookahead;         // prefetch distance, 0 .. kWarpMaxLA
  int32_t team;              // G: warps per replica (1 .. 8)
  int32_t window;            // iterations tried together, 1 .. lookahead + 1
  int32_t stage;             // warp_stage() of the launch's largest run
  int32_t sfields;           // fields of a flip's state in shared memory (sm.fld)
  int32_t *counter;          // next item; zero before the launch
  unsigned char *cache;      // field-cache region of each resident team
  size_t cache_stride;       // bytes per team
  WarpSmem sm;               // shared memory of one team
};

// Field-cache bytes of one team for a run: cslots jump and field records
// plus a working field record.
inline size_t warp_cache_bytes(int n, int m, int cslots) {
  const WarpRec r = warp_rec(n, m);
  return (size_t)cslots * ((size_t)r.jr + r.lr) + r.lr;
}

// Launches the warp annealer: `grid` blocks of `teams` teams of L.team warps.
cudaError_t launch_warp(const WarpLaunch &L, bool narrow, int grid, int teams,
                        cudaStream_t stream);
// The warp annealer's kernel (one WarpLaunch argument; fz: the variant with
// the frozen layout, for launches with nbuf_f > 0) for teams of `team`
// warps, for a CUDA graph node, with `smem` bytes of dynamic shared memory
// allowed.
cudaError_t warp_function(bool narrow, bool fz, int team, size_t smem, const void **func);
// The warp engine's acceptance decisions for `count` (penalty, delta, table
// index) triples in device memory (moda_check_accept).
cudaError_t launch_check_accept(const int64_t *a, const double *delta, const uint32_t *idx,
                                int count, const double *T, const float *Tf, uint8_t *accept,
                                int8_t *path, cudaStream_t stream);
// Resident blocks (one team of `team` warps each) per SM of that variant.
cudaError_t warp_occupancy(bool narrow, bool fz, int team, size_t smem, int *blocks);

// Sets the thread-local message that moda_last_error() returns.
void set_last_error(const char *msg);
inline void set_last_error(const std::string &msg) { set_last_error(msg.c_str()); }

}  // namespace moda
