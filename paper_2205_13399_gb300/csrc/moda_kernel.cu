// Annealing kernel of the multi-objective Digital Annealer (MDA), Sec. 3.3,
// Alg. 3 of arXiv 2205.13399, for the bi-objective QAP: one thread block
// runs one replica for all I_max iterations, its state held on chip.
//
// State of a replica.  Thread `tid` of a T-thread block owns the bits
// p = k*T + tid, k < B ("rounds"), of the n*n-bit two-way one-hot state
// (bit p = i*n + u: facility i at location u, Sec. 2.2) and keeps in
// registers, per owned bit:
//   x_p                 (a bit of `xmask`),
//   rc_p = R_i + C_u    (row count of facility i plus column count of u),
//   L1_p, L2_p          cost-only local fields
//                       L_k[(i,u)] = sum_{(j,v)} Fs^k_ij d_uv x_jv,
//                       Fs^k = F^k + F^k^T.
// With zero-diagonal symmetric distances, P^k_(i,u),(j,v) = Fs^k_ij d_uv is
// the off-diagonal of Eq. cale's P for the cost QUBO and its diagonal is 0,
// so the cost part of Delta E_k at bit p is (1 - 2 x_p) L_k[p].  Flipping
// bit (i,u) changes g (Eq. gqap) by 2 (1 - 2x)(rc - 1 - 2x), hence
//   Delta E_k = (1 - 2x) L_k + w_k (1 - 2x)(rc - 1 - 2x),  alpha_k = w_k/2
// (Eq. wqubom).  Q is never stored: a flip of (j,v) changes every field by
// s * Fs^k_ij * d_uv -- the outer product of a flow column and a distance
// column, s = +1 when the bit turns on.
//
// One iteration t (Alg. 3):
//   0  if the replica could jump to the archive this iteration, the slot it
//      would jump to is already known (the draw and |A| are), so one thread
//      starts a bulk copy (TMA) of that member's cached fields into shared
//      memory, completion tracked by an mbarrier.
//   A  every thread: Delta E and the parallel trial of its bits; warp
//      ballots give accept masks in (round, warp, lane) order = ascending
//      bit order.  One warp draws the next iteration's select / restart /
//      exploit words meanwhile.
//   -- barrier --
//   B  every warp, redundantly: count the accepted bits and rank-select one.
//      Flip:    its owner publishes Delta E -- barrier -- every thread
//               applies the flip to its registers and ballots "x dominates
//               slot y" -- barrier -- every warp picks the target slot
//               (Alg. 4 / Alg. 5) and stores its part of x (and of the
//               fields, into the cache).
//      No flip: jump to a random archive member: wait for the prefetched
//               fields (or rebuild them as L_k = Fs_k (X D)), or raise the
//               energy offset by beta.
#include <cstdint>

#include "moda_internal.h"

namespace moda {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWaitLimit = 1 << 22;  // bounded mbarrier polls

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64
// multiplies with a Weyl-sequence key schedule.
__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0,
                                         uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c[0];
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0;
    const uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

__device__ __forceinline__ uint32_t word_of(const uint32_t c[4], int w) {
  return w == 0 ? c[0] : w == 1 ? c[1] : w == 2 ? c[2] : c[3];
}

// floor(u * count / 2^32): uniform index in [0, count).
__device__ __forceinline__ int pick(uint32_t u, int count) {
  return (int)(((uint64_t)u * (uint32_t)count) >> 32);
}

__device__ __forceinline__ int nth_set_bit(uint32_t mask, int r) {
  for (int q = 0; q < r; ++q) mask &= mask - 1;
  return __ffs(mask) - 1;
}

__device__ __forceinline__ bool dominates(int64_t a1, int64_t a2, int64_t b1,
                                          int64_t b2) {
  return a1 <= b1 && a2 <= b2 && !(a1 == b1 && a2 == b2);
}

// ---- mbarrier and bulk-copy (TMA) helpers --------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
          smem_addr(bar)),
      "r"(bytes)
      : "memory");
}
// Bulk copy global -> shared; both addresses 16-byte aligned, bytes a
// multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src,
                                         uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], "
      "%2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for phase `parity` of `bar` to complete, at most kWaitLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (int i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
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

// Flat index round*T + warp*32 + lane of the r-th set bit (r < total), in
// every lane.
__device__ __forceinline__ int warp_mask_select(const uint32_t *masks,
                                                int items, int nw, int T,
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
        found = k * T + w * 32 + nth_set_bit(mk, rr);
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
  int64_t dE1, dE2;  // Delta E of the flipped bit
  int32_t sgn;       // +1: the bit turns on, -1: off
  int32_t pad;
};

template <int B>
__global__ void __launch_bounds__(kMaxThreads, 1)
    anneal_kernel(const AnnealArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = A.n, m = A.m, W = A.W, s = A.s;
  const int T = blockDim.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, NW = T >> 5;
  const int items = B * NW;
  const bool fc = A.fcache != nullptr;
  const SmemLayout lay =
      smem_layout(n, m, W, s, T, B, A.energies_in_smem != 0,
                  A.bits_in_smem != 0, fc);
  const SlotLayout sl = slot_layout(m);
  int2 *sFs = reinterpret_cast<int2 *>(smem + lay.Fs);
  int32_t *sD = reinterpret_cast<int32_t *>(smem + lay.D);
  int32_t *sM = reinterpret_cast<int32_t *>(smem + lay.M);
  uint32_t *sMask = reinterpret_cast<uint32_t *>(smem + lay.mask);
  uint32_t *sAmask = reinterpret_cast<uint32_t *>(smem + lay.amask);
  uint32_t *sRnd = reinterpret_cast<uint32_t *>(smem + lay.rnd);
  // Row and column counts of the last rebuilt state, two buffers used in
  // turn (rebuild q fills buffer q % 2 and clears the other one).
  int32_t *sRC = reinterpret_cast<int32_t *>(smem + lay.RC);
  int64_t *sRed = reinterpret_cast<int64_t *>(smem + lay.red);
  Bcast *bc = reinterpret_cast<Bcast *>(smem + lay.bc);
  uint32_t *sInit = reinterpret_cast<uint32_t *>(smem + lay.init);
  uint64_t *sBar = reinterpret_cast<uint64_t *>(smem + lay.mbar);

  const int rb = blockIdx.x;
  const uint32_t rep = A.replica_base + (uint32_t)rb;
  const uint32_t k0 = A.seed_lo, k1 = A.seed_hi;
  int64_t *gE = A.arch_E + (size_t)rb * s * 2;
  uint32_t *gBits = A.arch_bits + (size_t)rb * s * W;
  unsigned char *gF = fc ? A.fcache + (size_t)rb * s * sl.bytes : nullptr;
  longlong2 *aE = A.energies_in_smem
                      ? reinterpret_cast<longlong2 *>(smem + lay.archE)
                      : reinterpret_cast<longlong2 *>(gE);
  uint32_t *aBits = A.bits_in_smem
                        ? reinterpret_cast<uint32_t *>(smem + lay.archB)
                        : gBits;
  int rc_buf = 0;

  for (int e = tid; e < n * n; e += T) {
    sFs[e] = make_int2(A.Fs1[e], A.Fs2[e]);
    sD[e] = A.D[e];
  }
  for (int e = tid; e < 4 * n; e += T) sRC[e] = 0;
  if (tid == 0 && fc) {
    mbar_init(&sBar[0], 1);
    mbar_init(&sBar[1], 1);
    fence_mbar_init();
  }
  // Draws (select, restart, exploit) of iteration t live in sRnd[t % 3]:
  // they are drawn one iteration ahead, while a slow warp may still read
  // those of the previous iteration.
  if (warp == NW - 1 && lane < 3) {
    uint32_t c[4] = {0u, 1u, rep, kTagSelect + (uint32_t)lane};
    philox10(c, k0, k1);
    sRnd[4 + lane] = c[0];
  }
  int *sFail = reinterpret_cast<int *>(&bc->pad);
  if (tid == 0) *sFail = 0;

  // Own bit k (valid when k*T + tid < m): own[k] packs facility i (bits
  // 8..15), location u (bits 0..7) and rc = R_i + C_u (bits 16..31).
  int own[B];
  int32_t L1[B], L2[B];
  uint32_t xmask = 0;
#pragma unroll
  for (int k = 0; k < B; ++k) {
    const int p = k * T + tid;
    own[k] = p < m ? (((p / n) << 8) | (p % n)) : 0;
    L1[k] = 0;
    L2[k] = 0;
  }
  // Initial state (Alg. 3: "a random binary solution"): bit p is bit p % 32
  // of word (p / 32) % 4 of the draw (p / 128, 0, replica, init).
#pragma unroll
  for (int k = 0; k < B; ++k) {
    if (k * T + tid >= m) continue;
    const int p = k * T + tid;
    uint32_t c[4] = {(uint32_t)p >> 7, 0u, rep, kTagInit};
    philox10(c, k0, k1);
    xmask |= ((word_of(c, (p >> 5) & 3) >> (p & 31)) & 1u) << k;
  }
#pragma unroll
  for (int k = 0; k < B; ++k) {
    const uint32_t wv = __ballot_sync(kFull, (xmask >> k) & 1u);
    if (lane == 0 && k * NW + warp < W) sInit[k * NW + warp] = wv;
  }
  __syncthreads();

  // Fields, counts and owned bits of the state held in `words`, in two
  // passes around one barrier: (1) M = X * D (M_ju = sum_v x_jv d_vu) and
  // the row / column counts into shared memory; (2) every thread forms
  // L_k[(i,u)] = sum_j Fs^k_ij M_ju for its own bits.  Both passes are
  // exact int32 arithmetic (the instance check bounds every field).
  auto rebuild = [&](const uint32_t *words) {
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
      if (k * T + tid >= m) continue;
      const int q = k * T + tid;
      xmask |= ((words[q >> 5] >> (q & 31)) & 1u) << k;
    }
    __syncthreads();
    const int32_t *cR = sRC + rc_buf * 2 * n, *cC = cR + n;
    for (int e = tid; e < 2 * n; e += T) sRC[(1 - rc_buf) * 2 * n + e] = 0;
#pragma unroll
    for (int k = 0; k < B; ++k) {
      if (k * T + tid >= m) continue;
      const int i = (own[k] >> 8) & 255, u = own[k] & 255;
      int32_t a1 = 0, a2 = 0;
      const int2 *frow = sFs + i * n;  // Fs symmetric: row i = column i
#pragma unroll 5
      for (int j = 0; j < n; ++j) {
        const int2 f = frow[j];
        const int32_t mm = sM[j * n + u];
        a1 += f.x * mm;
        a2 += f.y * mm;
      }
      L1[k] = a1;
      L2[k] = a2;
      own[k] = ((cR[i] + cC[u]) << 16) | (i << 8) | u;
    }
    rc_buf ^= 1;
  };
  rebuild(sInit);

  // E_k = c_k + w_k g / 2 with c_k = (sum_p x_p L_k[p]) / 2 and g from the
  // row and column counts.
  int64_t E1, E2;
  {
    int64_t s1 = 0, s2 = 0, gp = 0;
#pragma unroll
    for (int k = 0; k < B; ++k) {
      if (k * T + tid >= m || !((xmask >> k) & 1u)) continue;
      s1 += L1[k];
      s2 += L2[k];
    }
    for (int e = tid; e < n; e += T) {
      const int64_t dr = 1 - sRC[e], dc = 1 - sRC[n + e];
      gp += dr * dr + dc * dc;
    }
    s1 = block_sum(s1, sRed, lane, warp, NW);
    s2 = block_sum(s2, sRed, lane, warp, NW);
    gp = block_sum(gp, sRed, lane, warp, NW);
    E1 = s1 / 2 + A.w1 * (gp / 2);
    E2 = s2 / 2 + A.w2 * (gp / 2);
  }

  int64_t Eoff = 0;
  int acount = 0;
  int64_t st_flip = 0, st_jump = 0, st_empty = 0, st_off = 0;
  // Prefetch state (uniform across the block): buffer b has a copy in
  // flight when pend & (1 << b); its mbarrier's next phase is ph >> b & 1.
  uint32_t pend = 0, ph = 0;
  bool failed = false;

  for (int64_t it = 1; it <= A.I_max; ++it) {
    const uint32_t t = (uint32_t)it;
    const int buf = (int)(t & 1u);
    uint32_t *mask = sMask + buf * items;
    const uint32_t *rnd = sRnd + (t % 3u) * 4;
    const int si = (int)((it <= A.nsched ? it : (int64_t)A.nsched) - 1);
    const double delta = A.sch_delta[si];
    const int64_t lo = A.sch_lo[si], hi = A.sch_hi[si];

    // Step 0: prefetch the member a jump in this iteration would land on.
    unsigned char *pb = smem + lay.pbuf + (size_t)buf * lay.pbuf_bytes;
    const bool jump_possible = fc && A.escape == 0 && acount > 0;
    if (jump_possible) {
      if (pend & (1u << buf)) {  // retire the unused copy of iteration t-2
        if (!mbar_wait(&sBar[buf], (ph >> buf) & 1u)) {
          failed = true;
          *sFail = 1;
        }
        ph ^= 1u << buf;
        pend &= ~(1u << buf);
      }
      if (tid == 0) {
        const int slot = pick(rnd[1], acount);
        const uint32_t bytes = (uint32_t)sl.bytes;
        uint32_t eb = 0, bb = 0, boff = 0;
        if (!A.energies_in_smem) eb = 16;
        if (!A.bits_in_smem) {
          const uintptr_t b0 = (uintptr_t)(gBits + (size_t)slot * W);
          boff = (uint32_t)(b0 & 15);
          bb = (uint32_t)align_up(boff + 4 * (size_t)W, 16);
        }
        fence_proxy_async_shared();
        mbar_expect_tx(&sBar[buf], bytes + eb + bb);
        bulk_g2s(pb, gF + (size_t)slot * sl.bytes, bytes, &sBar[buf]);
        if (eb)
          bulk_g2s(pb + sl.bytes, gE + (size_t)slot * 2, 16, &sBar[buf]);
        if (bb)
          bulk_g2s(pb + sl.bytes + eb,
                   reinterpret_cast<const unsigned char *>(gBits + (size_t)slot * W) - boff,
                   bb, &sBar[buf]);
      }
      pend |= 1u << buf;
    }

    // Phase A: Delta E (Eq. cale) and the parallel trial of every bit.
#pragma unroll
    for (int k = 0; k < B; ++k) {
      bool acc = false;
      const uint32_t xv = (xmask >> k) & 1u;
      if (k * T + tid < m) {
        const int p = k * T + tid;
        const int sg = 1 - 2 * (int)xv;
        const int h = sg * ((own[k] >> 16) - 1 - 2 * (int)xv);
        int64_t f1 = (int64_t)(sg * L1[k]) + A.w1 * h;
        int64_t f2 = (int64_t)(sg * L2[k]) + A.w2 * h;
        if (A.escape == 1) {
          f1 -= Eoff;
          f2 -= Eoff;
        }
        const int64_t a1 = f1 > 0 ? f1 : 0, a2 = f2 > 0 ? f2 : 0;
        const int64_t a = A.accept == 0 ? a1 + a2 : (a1 < a2 ? a1 : a2);
        if (a <= lo) {
          acc = true;
        } else if (a <= hi) {
          uint32_t c[4] = {(uint32_t)p >> 2, t, rep, kTagAccept};
          philox10(c, k0, k1);
          const uint32_t w = word_of(c, p & 3);
          acc = (double)a <= __dmul_rn(delta, A.table[w >> 16]);
        }
      }
      const uint32_t bal = __ballot_sync(kFull, acc);
      if (lane == 0) mask[k * NW + warp] = bal;
    }
    if (warp == NW - 1 && lane < 3) {  // draws of iteration t + 1
      uint32_t c[4] = {0u, t + 1u, rep, kTagSelect + (uint32_t)lane};
      philox10(c, k0, k1);
      sRnd[((t + 1u) % 3u) * 4 + lane] = c[0];
    }
    __syncthreads();
    if (fc && *sFail) break;  // a bulk copy did not complete (uniform exit)

    // Phase B: every warp reaches the same decision from shared memory.
    int incl, cnt;
    const int total = warp_mask_total(mask, items, lane, incl, cnt);
    int64_t event = INT64_MIN;
    if (total > 0) {
      const int ps = warp_mask_select(mask, items, NW, T, lane, incl, cnt,
                                      pick(rnd[0], total));
      const int kk = ps / T;
      if (ps - kk * T == tid) {  // the owner publishes Delta E of the flip
#pragma unroll
        for (int k = 0; k < B; ++k) {
          if (k != kk) continue;
          const int xv = (int)((xmask >> k) & 1u);
          const int sg = 1 - 2 * xv;
          const int h = sg * ((own[k] >> 16) - 1 - 2 * xv);
          bc->dE1 = (int64_t)(sg * L1[k]) + A.w1 * h;
          bc->dE2 = (int64_t)(sg * L2[k]) + A.w2 * h;
          bc->sgn = sg;
        }
      }
      __syncthreads();
      const int64_t nE1 = E1 + bc->dE1, nE2 = E2 + bc->dE2;
      const int sg = bc->sgn;
      const int j = (int)__umulhi((uint32_t)ps, A.magic);
      const int v = ps - j * n;
      // Apply the flip of (j, v) to the owned registers.
#pragma unroll
      for (int k = 0; k < B; ++k) {
        if (k * T + tid >= m) continue;
        const int i = (own[k] >> 8) & 255, u = own[k] & 255;
        const int2 f = sFs[j * n + i];
        const int32_t d = sg * sD[v * n + u];
        L1[k] += f.x * d;
        L2[k] += f.y * d;
        own[k] += (sg * ((i == j) + (u == v))) * 65536;
        if (k * T + tid == ps) xmask ^= 1u << k;
      }
      // Archive: ballots of "x dominates slot y" in slot order, and (for
      // the exploitative update) whether some member dominates x.
      int anyd = 0;
#pragma unroll
      for (int k = 0; k < B; ++k) {
        const int y = k * T + tid;
        bool dom = false;
        if (y < acount) {
          const longlong2 ye = aE[y];
          dom = dominates(nE1, nE2, ye.x, ye.y);
          if (dominates(ye.x, ye.y, nE1, nE2)) anyd = 1;
        }
        const uint32_t bal = __ballot_sync(kFull, dom);
        if (lane == 0) sAmask[k * NW + warp] = bal;
      }
      anyd = __syncthreads_or(anyd);
      int aincl, acnt;
      const int nb = warp_mask_total(sAmask, items, lane, aincl, acnt);
      int target = -1;
      if (A.archive == 0) {
        // Alg. 4: replace the first dominated member, else append.
        if (nb > 0)
          target = warp_mask_select(sAmask, items, NW, T, lane, aincl, acnt, 0);
        else if (acount < s)
          target = acount++;
      } else if (!anyd) {
        // Alg. 5: replace a random dominated member, else append.
        if (nb > 0)
          target = warp_mask_select(sAmask, items, NW, T, lane, aincl, acnt,
                                    pick(rnd[2], nb));
        else if (acount < s)
          target = acount++;
      }
      if (target >= 0) {
#pragma unroll
        for (int k = 0; k < B; ++k) {
          const uint32_t wv = __ballot_sync(kFull, (xmask >> k) & 1u);
          const int wi = k * NW + warp;
          if (lane == 0 && wi < W) aBits[(size_t)target * W + wi] = wv;
        }
        if (tid == 0) aE[target] = make_longlong2(nE1, nE2);
        if (fc) {
          unsigned char *rec = gF + (size_t)target * sl.bytes;
          int2 *rf = reinterpret_cast<int2 *>(rec + sl.fields);
          uint16_t *rr = reinterpret_cast<uint16_t *>(rec + sl.rc);
#pragma unroll
          for (int k = 0; k < B; ++k) {
            const int q = k * T + tid;
            if (q >= m) continue;
            rf[q] = make_int2(L1[k], L2[k]);
            rr[q] = (uint16_t)(own[k] >> 16);
          }
          fence_proxy_async_global();  // later bulk copies read these
        }
        // The next iteration's bulk copy may read this slot.
        if (fc) __syncthreads();
      }
      E1 = nE1;
      E2 = nE2;
      Eoff = 0;
      ++st_flip;
      event = ps;
    } else if (A.escape == 0) {
      if (acount > 0) {
        // Alg. 3: jump to a random archive member.
        const int slot = pick(rnd[1], acount);
        if (fc) {
          if (!mbar_wait(&sBar[buf], (ph >> buf) & 1u)) {
            failed = true;
            *sFail = 1;
          }
          ph ^= 1u << buf;
          pend &= ~(1u << buf);
          const int2 *rf = reinterpret_cast<const int2 *>(pb + sl.fields);
          const uint16_t *rr = reinterpret_cast<const uint16_t *>(pb + sl.rc);
          longlong2 se;
          if (A.energies_in_smem)
            se = aE[slot];
          else
            se = *reinterpret_cast<const longlong2 *>(pb + sl.bytes);
          const uint32_t *words;
          if (A.bits_in_smem) {
            words = aBits + (size_t)slot * W;
          } else {
            const uintptr_t b0 = (uintptr_t)(gBits + (size_t)slot * W);
            words = reinterpret_cast<const uint32_t *>(
                pb + sl.bytes + (A.energies_in_smem ? 0 : 16) + (b0 & 15));
          }
          E1 = se.x;
          E2 = se.y;
          xmask = 0;
#pragma unroll
          for (int k = 0; k < B; ++k) {
            const int q = k * T + tid;
            if (q >= m) continue;
            const int2 f = rf[q];
            L1[k] = f.x;
            L2[k] = f.y;
            own[k] = ((int)rr[q] << 16) | (own[k] & 0xFFFF);
            xmask |= ((words[q >> 5] >> (q & 31)) & 1u) << k;
          }
        } else {
          const longlong2 se = aE[slot];
          E1 = se.x;
          E2 = se.y;
          rebuild(aBits + (size_t)slot * W);
        }
        ++st_jump;
        event = -1 - (int64_t)slot;
      } else {
        ++st_empty;
      }
    } else {
      Eoff += A.beta;
      ++st_off;
    }
    if (A.trace != nullptr && tid == 0) {
      int64_t *tr = A.trace + ((size_t)rb * (size_t)A.I_max + (size_t)(it - 1)) * 3;
      tr[0] = E1;
      tr[1] = E2;
      tr[2] = event;
    }
  }

  // No bulk copy may be in flight when the block exits.
  for (int b = 0; b < 2; ++b)
    if (pend & (1u << b)) {
      if (!mbar_wait(&sBar[b], (ph >> b) & 1u)) failed = true;
    }
  if (failed && tid == 0) atomicExch(A.error, kErrCopyTimeout);

  __syncthreads();
#pragma unroll
  for (int k = 0; k < B; ++k) {
    const uint32_t wv = __ballot_sync(kFull, (xmask >> k) & 1u);
    const int wi = k * NW + warp;
    if (lane == 0 && wi < W) A.x_final[(size_t)rb * W + wi] = wv;
  }
  if (A.energies_in_smem) {
    for (int e = tid; e < acount; e += T) {
      const longlong2 v = aE[e];
      gE[2 * e] = v.x;
      gE[2 * e + 1] = v.y;
    }
  }
  if (A.bits_in_smem) {
    for (int e = tid; e < acount * W; e += T) gBits[e] = aBits[e];
  }
  if (tid == 0) {
    A.arch_count[rb] = acount;
    A.E_final[2 * rb] = E1;
    A.E_final[2 * rb + 1] = E2;
    A.stats[4 * rb + 0] = st_flip;
    A.stats[4 * rb + 1] = st_jump;
    A.stats[4 * rb + 2] = st_empty;
    A.stats[4 * rb + 3] = st_off;
  }
}

template <int B>
cudaError_t launch_b(const AnnealArgs &args, int replicas, int threads,
                     size_t smem, cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(
      anneal_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  anneal_kernel<B><<<replicas, threads, smem, stream>>>(args);
  return cudaGetLastError();
}

}  // namespace

bool supported_rounds(int b) {
  return b == 1 || b == 2 || b == 3 || b == 4 || b == 6 || b == 8;
}

cudaError_t launch_anneal(const AnnealArgs &args, int replicas, int threads,
                          int rounds, size_t smem, cudaStream_t stream) {
  switch (rounds) {
    case 1: return launch_b<1>(args, replicas, threads, smem, stream);
    case 2: return launch_b<2>(args, replicas, threads, smem, stream);
    case 3: return launch_b<3>(args, replicas, threads, smem, stream);
    case 4: return launch_b<4>(args, replicas, threads, smem, stream);
    case 6: return launch_b<6>(args, replicas, threads, smem, stream);
    case 8: return launch_b<8>(args, replicas, threads, smem, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace moda
