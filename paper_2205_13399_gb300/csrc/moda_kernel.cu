// Annealing kernel of the multi-objective Digital Annealer (MDA), Sec. 3.3,
// Alg. 3 of arXiv 2205.13399, for the bi-objective QAP: one thread block
// runs one replica for all I_max iterations, its state held on chip.
//
// State of a replica (shared memory):
//   X[p]        the n*n-bit two-way one-hot state, bit p = i*n + u
//               (facility i at location u, Sec. 2.2);
//   R[i], C[u]  row and column counts of X;
//   L1[p], L2[p] cost-only local fields
//               L_k[(i,u)] = sum_{(j,v)} Fs^k_ij d_uv x_jv,  Fs^k = F^k + F^k^T.
// With zero-diagonal symmetric distances, P^k_(i,u),(j,v) = Fs^k_ij d_uv is
// the off-diagonal of Eq. cale's P for the cost QUBO and its diagonal is 0,
// so the cost part of Delta E_k at bit p is (1 - 2 x_p) L_k[p].  The
// penalty part follows from the counts: flipping (i,u) changes g by
//   2 (1 - 2 x)(R_i + C_u - 1 - 2 x)          (Eq. gqap),
// so Delta E_k = (1 - 2x) L_k + w_k (1 - 2x)(R_i + C_u - 1 - 2x) with
// alpha_k = w_k / 2 (Eq. wqubom).  Q is never stored: a flip of (j,v)
// updates every field by s * Fs^k_ij * d_uv (the outer product of a flow
// column and a distance column), s = +1 when the bit turns on.
//
// Bit ownership is round-robin: thread `tid` owns bits p = k*T + tid,
// k < B, so a warp ballot per k yields accept masks whose (k, warp, lane)
// order is ascending bit order -- the order in which "one flip at random"
// (Alg. 3) is ranked.
#include <cstdint>

#include "moda_internal.h"

namespace moda {
namespace {

constexpr unsigned kFull = 0xffffffffu;

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

struct Bcast {
  int32_t count;   // accepted bits this iteration
  int32_t p;       // the flipped bit
  int32_t sgn;     // +1: the bit turned on, -1: off
  int32_t slot;    // restart slot, or archive target (-1: none)
  int32_t acount;  // archive size after the update
  int32_t nones;   // set bits collected by a rebuild
  int32_t pad0, pad1;
  int64_t E1, E2;  // energies after the flip
};

__device__ __forceinline__ bool dominates(int64_t a1, int64_t a2, int64_t b1,
                                          int64_t b2) {
  return a1 <= b1 && a2 <= b2 && !(a1 == b1 && a2 == b2);
}

// Warp-0 helper: over `items` ballot masks in (k, warp) order, the total
// number of set bits and, for rank r (r < total, uniform), the flat index
// k*T + warp*32 + lane of the r-th set bit (valid in every lane).
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

template <int B>
__global__ void __launch_bounds__(kMaxThreads, 1)
    anneal_kernel(const AnnealArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = A.n, m = A.m, W = A.W;
  const int T = blockDim.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, NW = T >> 5;
  const SmemLayout lay = smem_layout(n, m, T, B);
  int32_t *sFs1 = reinterpret_cast<int32_t *>(smem + lay.Fs1);
  int32_t *sFs2 = reinterpret_cast<int32_t *>(smem + lay.Fs2);
  int32_t *sD = reinterpret_cast<int32_t *>(smem + lay.D);
  int32_t *sL1 = reinterpret_cast<int32_t *>(smem + lay.L1);
  int32_t *sL2 = reinterpret_cast<int32_t *>(smem + lay.L2);
  int32_t *sR = reinterpret_cast<int32_t *>(smem + lay.R);
  int32_t *sC = reinterpret_cast<int32_t *>(smem + lay.C);
  uint32_t *sMask = reinterpret_cast<uint32_t *>(smem + lay.mask);
  uint32_t *sAmask = reinterpret_cast<uint32_t *>(smem + lay.amask);
  uint16_t *sOnes = reinterpret_cast<uint16_t *>(smem + lay.ones);
  uint8_t *sX = reinterpret_cast<uint8_t *>(smem + lay.X);
  int64_t *sRed = reinterpret_cast<int64_t *>(smem + lay.red);
  Bcast *bc = reinterpret_cast<Bcast *>(smem + lay.bcast);

  const int rb = blockIdx.x;
  const uint32_t rep = A.replica_base + (uint32_t)rb;
  const uint32_t k0 = A.seed_lo, k1 = A.seed_hi;
  const int s = A.s;
  int64_t *aE = A.arch_E + (size_t)rb * s * 2;
  uint32_t *aBits = A.arch_bits + (size_t)rb * s * W;
  const int items = B * NW;

  for (int e = tid; e < n * n; e += T) {
    sFs1[e] = A.Fs1[e];
    sFs2[e] = A.Fs2[e];
    sD[e] = A.D[e];
  }
  // Own bits: facility i and location u packed as (i << 8) | u, -1 if p >= m.
  int own[B];
#pragma unroll
  for (int k = 0; k < B; ++k) {
    const int p = k * T + tid;
    own[k] = p < m ? (((p / n) << 8) | (p % n)) : -1;
  }
  // Initial state (Alg. 3: "a random binary solution"): bit p is bit p % 32
  // of word (p / 32) % 4 of the draw (p / 128, 0, replica, init).
#pragma unroll
  for (int k = 0; k < B; ++k) {
    if (own[k] < 0) continue;
    const int p = k * T + tid;
    uint32_t c[4] = {(uint32_t)p >> 7, 0u, rep, kTagInit};
    philox10(c, k0, k1);
    sX[p] = (uint8_t)((word_of(c, (p >> 5) & 3) >> (p & 31)) & 1u);
  }
  for (int e = tid; e < n; e += T) {
    sR[e] = 0;
    sC[e] = 0;
  }
  if (tid == 0) bc->nones = 0;
  __syncthreads();

  // Counts, the list of set bits and the fields from scratch.
  auto collect = [&]() {
#pragma unroll
    for (int k = 0; k < B; ++k) {
      if (own[k] < 0) continue;
      const int p = k * T + tid;
      if (sX[p]) {
        atomicAdd(&sR[own[k] >> 8], 1);
        atomicAdd(&sC[own[k] & 255], 1);
        const int pos = atomicAdd(&bc->nones, 1);
        sOnes[pos] = (uint16_t)own[k];
      }
    }
  };
  auto rebuild_fields = [&]() {
    const int no = bc->nones;
#pragma unroll
    for (int k = 0; k < B; ++k) {
      if (own[k] < 0) continue;
      const int p = k * T + tid;
      const int i = own[k] >> 8, u = own[k] & 255;
      int32_t acc1 = 0, acc2 = 0;
      for (int q = 0; q < no; ++q) {
        const int jv = sOnes[q];
        const int j = jv >> 8, v = jv & 255;
        const int32_t d = sD[v * n + u];
        acc1 += sFs1[j * n + i] * d;
        acc2 += sFs2[j * n + i] * d;
      }
      sL1[p] = acc1;
      sL2[p] = acc2;
    }
  };
  collect();
  __syncthreads();
  rebuild_fields();
  __syncthreads();

  // E_k = c_k + w_k g / 2 with c_k = (sum_p x_p L_k[p]) / 2.
  int64_t E1, E2;
  {
    int64_t s1 = 0, s2 = 0, gp = 0;
#pragma unroll
    for (int k = 0; k < B; ++k) {
      if (own[k] < 0) continue;
      const int p = k * T + tid;
      if (sX[p]) {
        s1 += sL1[p];
        s2 += sL2[p];
      }
    }
    for (int e = tid; e < n; e += T) {
      const int64_t dr = 1 - sR[e], dc = 1 - sC[e];
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

  for (int64_t it = 1; it <= A.I_max; ++it) {
    const uint32_t t = (uint32_t)it;
    const int si = (int)((it <= A.nsched ? it : (int64_t)A.nsched) - 1);
    const double delta = A.sch_delta[si];
    const int64_t lo = A.sch_lo[si], hi = A.sch_hi[si];

    // Phase A: Delta E (Eq. cale) and the parallel trial of every bit.
#pragma unroll
    for (int k = 0; k < B; ++k) {
      bool acc = false;
      if (own[k] >= 0) {
        const int p = k * T + tid;
        const int xv = sX[p];
        const int sg = 1 - 2 * xv;
        const int h = sg * (sR[own[k] >> 8] + sC[own[k] & 255] - 1 - 2 * xv);
        int64_t e1 = (int64_t)(sg * sL1[p]) + A.w1 * h;
        int64_t e2 = (int64_t)(sg * sL2[p]) + A.w2 * h;
        if (A.escape == 1) {
          e1 -= Eoff;
          e2 -= Eoff;
        }
        const int64_t a1 = e1 > 0 ? e1 : 0, a2 = e2 > 0 ? e2 : 0;
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
      if (lane == 0) sMask[k * NW + warp] = bal;
    }
    __syncthreads();

    // Phase B (warp 0): count, pick one accepted bit, apply it to X, R, C.
    if (warp == 0) {
      int incl, cnt;
      const int total = warp_mask_total(sMask, items, lane, incl, cnt);
      if (lane == 0) bc->count = total;
      if (total > 0) {
        uint32_t c[4] = {0u, t, rep, kTagSelect};
        philox10(c, k0, k1);
        const int r = pick(c[0], total);
        const int p = warp_mask_select(sMask, items, NW, T, lane, incl, cnt, r);
        if (lane == 0) {
          const int i = p / n, u = p - (p / n) * n;
          const int xv = sX[p];
          const int sg = 1 - 2 * xv;
          const int h = sg * (sR[i] + sC[u] - 1 - 2 * xv);
          bc->p = p;
          bc->sgn = sg;
          bc->E1 = E1 + (int64_t)(sg * sL1[p]) + A.w1 * h;
          bc->E2 = E2 + (int64_t)(sg * sL2[p]) + A.w2 * h;
          sX[p] = (uint8_t)(1 - xv);
          sR[i] += sg;
          sC[u] += sg;
        }
      } else if (A.escape == 0 && acount > 0) {
        uint32_t c[4] = {0u, t, rep, kTagRestart};
        philox10(c, k0, k1);
        if (lane == 0) {
          bc->slot = pick(c[0], acount);
          bc->nones = 0;
        }
        for (int e = lane; e < n; e += 32) {
          sR[e] = 0;
          sC[e] = 0;
        }
      }
    }
    __syncthreads();

    int64_t event = INT64_MIN;
    const int count = bc->count;
    if (count > 0) {
      const int p = bc->p, sg = bc->sgn;
      const int64_t nE1 = bc->E1, nE2 = bc->E2;
      const int j = p / n, v = p - (p / n) * n;
      // Outer-product field update for the flip of (j, v).
#pragma unroll
      for (int k = 0; k < B; ++k) {
        if (own[k] < 0) continue;
        const int q = k * T + tid;
        const int32_t d = sg * sD[v * n + (own[k] & 255)];
        sL1[q] += sFs1[j * n + (own[k] >> 8)] * d;
        sL2[q] += sFs2[j * n + (own[k] >> 8)] * d;
      }
      // Archive: ballots of "x dominates slot y" in slot order; for the
      // exploitative update also whether some member dominates x.
      int anyd = 0;
#pragma unroll
      for (int k = 0; k < B; ++k) {
        const int y = k * T + tid;
        bool dom = false;
        if (y < acount) {
          const int64_t y1 = aE[2 * y], y2 = aE[2 * y + 1];
          dom = dominates(nE1, nE2, y1, y2);
          if (dominates(y1, y2, nE1, nE2)) anyd = 1;
        }
        const uint32_t bal = __ballot_sync(kFull, dom);
        if (lane == 0) sAmask[k * NW + warp] = bal;
      }
      anyd = __syncthreads_or(anyd);
      if (warp == 0) {
        int incl, cnt;
        const int nb = warp_mask_total(sAmask, items, lane, incl, cnt);
        int target = -1, newcount = acount;
        if (A.archive == 0) {
          // Alg. 4: replace the first dominated member, else append.
          if (nb > 0)
            target = warp_mask_select(sAmask, items, NW, T, lane, incl, cnt, 0);
          else if (acount < s)
            target = newcount++;
        } else if (!anyd) {
          // Alg. 5: replace a random dominated member, else append.
          if (nb > 0) {
            uint32_t c[4] = {0u, t, rep, kTagExploit};
            philox10(c, k0, k1);
            target = warp_mask_select(sAmask, items, NW, T, lane, incl, cnt,
                                      pick(c[0], nb));
          } else if (acount < s) {
            target = newcount++;
          }
        }
        if (lane == 0) {
          bc->slot = target;
          bc->acount = newcount;
        }
      }
      __syncthreads();
      const int target = bc->slot;
      acount = bc->acount;
      if (target >= 0) {
        for (int w = warp; w < W; w += NW) {
          const int q = w * 32 + lane;
          const uint32_t word = __ballot_sync(kFull, q < m && sX[q] != 0);
          if (lane == 0) aBits[(size_t)target * W + w] = word;
        }
        if (tid == 0) {
          aE[2 * target] = nE1;
          aE[2 * target + 1] = nE2;
        }
      }
      E1 = nE1;
      E2 = nE2;
      Eoff = 0;
      ++st_flip;
      event = p;
    } else if (A.escape == 0) {
      if (acount > 0) {
        // Alg. 3: jump to a random archive member; rebuild its fields.
        const int slot = bc->slot;
        E1 = aE[2 * slot];
        E2 = aE[2 * slot + 1];
        const uint32_t *src = aBits + (size_t)slot * W;
#pragma unroll
        for (int k = 0; k < B; ++k) {
          if (own[k] < 0) continue;
          const int q = k * T + tid;
          sX[q] = (uint8_t)((src[q >> 5] >> (q & 31)) & 1u);
        }
        collect();
        __syncthreads();
        rebuild_fields();
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

  __syncthreads();
  for (int w = warp; w < W; w += NW) {
    const int q = w * 32 + lane;
    const uint32_t word = __ballot_sync(kFull, q < m && sX[q] != 0);
    if (lane == 0) A.x_final[(size_t)rb * W + w] = word;
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
                     cudaStream_t stream) {
  const SmemLayout lay = smem_layout(args.n, args.m, threads, B);
  cudaError_t e = cudaFuncSetAttribute(anneal_kernel<B>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)lay.total);
  if (e != cudaSuccess) return e;
  anneal_kernel<B><<<replicas, threads, lay.total, stream>>>(args);
  return cudaGetLastError();
}

}  // namespace

bool supported_bits_per_thread(int b) {
  return b == 1 || b == 2 || b == 4 || b == 8;
}

cudaError_t launch_anneal(const AnnealArgs &args, int replicas, int threads,
                          int bits_per_thread, cudaStream_t stream) {
  switch (bits_per_thread) {
    case 1: return launch_b<1>(args, replicas, threads, stream);
    case 2: return launch_b<2>(args, replicas, threads, stream);
    case 4: return launch_b<4>(args, replicas, threads, stream);
    case 8: return launch_b<8>(args, replicas, threads, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace moda
