// Multi-objective Digital Annealer (Alg. 3 of arXiv 2205.13399) on K
// objectives given as explicit QUBO matrices: the generalisation of the
// bi-objective QAP path from outer-product fields to a stored P (Eq. cale),
// for QUBOs without QAP structure and for more than two objectives.
//
// One thread block per replica; thread tid owns bits q = k*T + tid, k < B,
// and keeps Delta E_j(q) of every objective j in registers.  A flip of bit
// p changes every other Delta E_j(q) by (1 - 2 x_q) s P_j[p][q] (s = +1
// when p turns on): one coalesced read of row p of each P_j.  Draws, the
// acceptance rule, the selection and the archive updates are those of the
// bQAP kernel, with K-dimensional dominance; a jump to an archive member
// reloads its Delta E from a per-slot record in global memory (or rebuilds
// it from the member's state when the records do not fit).
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "moda_host.h"
#include "moda_internal.h"

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxK = 3;
constexpr int kMaxQThreads = 1024;

enum : uint32_t { kTagAccept = 0, kTagSelect = 1, kTagRestart = 2, kTagExploit = 3,
                  kTagInit = 4 };

// Philox4x32-10 (Salmon et al., SC'11).
__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

__device__ __forceinline__ int pick(uint32_t u, int count) {
  return (int)(((uint64_t)u * (uint32_t)count) >> 32);
}

__device__ __forceinline__ int nth_bit(uint32_t mask, int r) {
  for (int q = 0; q < r; ++q) mask &= mask - 1;
  return __ffs(mask) - 1;
}

// Ballot words in (round, warp) order, one word per lane per pass: the
// r-th set bit (r < total) as a flat index round*T + warp*32 + lane.
__device__ int select_bit(const uint32_t *masks, int items, int nw, int T, int lane, int r) {
  int base = 0;
  for (int it0 = 0; it0 < items; it0 += 32) {
    const int it = it0 + lane;
    const uint32_t mk = it < items ? masks[it] : 0u;
    const int c = __popc(mk);
    int incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += v;
    }
    const int tot = __shfl_sync(kFull, incl, 31);
    if (r < base + tot) {
      const int excl = base + incl - c;
      int found = -1;
      if (r >= excl && r < base + incl) {
        const int kk = it / nw, w = it - kk * nw;
        found = kk * T + w * 32 + nth_bit(mk, r - excl);
      }
      const unsigned who = __ballot_sync(kFull, found >= 0);
      return __shfl_sync(kFull, found, __ffs(who) - 1);
    }
    base += tot;
  }
  return -1;
}

__device__ int count_bits(const uint32_t *masks, int items, int lane) {
  int c = 0;
  for (int it = lane; it < items; it += 32) c += __popc(masks[it]);
  return (int)__reduce_add_sync(kFull, (unsigned)c);
}

template <int K>
__device__ __forceinline__ bool dominates(const int64_t *a, const int64_t *b) {
  bool strict = false;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    if (a[j] > b[j]) return false;
    if (a[j] < b[j]) strict = true;
  }
  return strict;
}

// Shared-memory carve-up (byte offsets, 16-byte aligned regions).
struct QLayout {
  size_t mask, amask, rnd, bc, red, init, total;
};
__host__ __device__ inline size_t qalign(size_t v) { return (v + 15) / 16 * 16; }
__host__ __device__ inline QLayout qubo_layout(int T, int B, int W) {
  const size_t items = (size_t)B * (T / 32);
  QLayout L;
  size_t o = 0;
  L.mask = o;  o = qalign(o + 4 * 2 * items);          // accept ballots x 2
  L.amask = o; o = qalign(o + 4 * items);              // archive ballots
  L.rnd = o;   o = qalign(o + 4 * 8);                  // draws x 2 iterations
  L.bc = o;    o = qalign(o + 8 * (kMaxK + 2));        // flipped bit's Delta E, x
  L.red = o;   o = qalign(o + 8 * 32 * (kMaxK + 1));   // block sums
  L.init = o;  o = qalign(o + 4 * (size_t)W);          // initial state
  L.total = o;
  return L;
}

struct QArgs {
  int32_t m, W, s, nsched;
  int64_t I_max, beta;
  uint32_t replica_base, seed_lo, seed_hi;
  int32_t accept, archive, escape;
  const int32_t *P;          // [K][m][m]: P_j = Q_j + Q_j^T, diagonal Q_pp
  const double *sch_delta;
  const int64_t *sch_lo, *sch_hi;
  const double *table;
  int64_t *fcache;           // [R][s][K][m] Delta E records, or nullptr
  int64_t *arch_E;           // [R][s][K]
  uint32_t *arch_bits;       // [R][s][W]
  int32_t *arch_count;       // [R]
  uint32_t *x_final;         // [R][W]
  int64_t *E_final;          // [R][K]
  int64_t *stats;            // [R][4]
  int64_t *trace;            // [R][I_max][K + 1] or nullptr
};

template <int K, int B>
__global__ void __launch_bounds__(kMaxQThreads, 1) qubo_kernel(const QArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int NW = T >> 5, items = B * NW;
  const int m = A.m, W = A.W, s = A.s;
  const size_t mm = (size_t)m * m;
  const int rb = blockIdx.x;
  const uint32_t rep = A.replica_base + (uint32_t)rb;
  const uint32_t k0 = A.seed_lo, k1 = A.seed_hi;
  const uint32_t I_max = (uint32_t)A.I_max;
  const QLayout L = qubo_layout(T, B, W);
  uint32_t *sMask = reinterpret_cast<uint32_t *>(smem + L.mask);   // [2][items]
  uint32_t *sAmask = reinterpret_cast<uint32_t *>(smem + L.amask); // [items]
  uint32_t *sRnd = reinterpret_cast<uint32_t *>(smem + L.rnd);     // [2][4]
  int64_t *sBc = reinterpret_cast<int64_t *>(smem + L.bc);         // [K + 1]
  int64_t *sRed = reinterpret_cast<int64_t *>(smem + L.red);       // [32][K + 1]
  int64_t *gE = A.arch_E + (size_t)rb * s * K;
  uint32_t *gBits = A.arch_bits + (size_t)rb * s * W;
  int64_t *gF = A.fcache ? A.fcache + (size_t)rb * s * K * m : nullptr;

  int64_t dE[K][B];
  uint32_t xm = 0;  // bit k: x of own bit k * T + tid
  auto valid = [&](int k) { return k * T + tid < m; };

  // Delta E of every own bit of the state `x_of(q)`, from scratch, and the
  // block's energies: Delta E_j(q) = (1 - 2 x_q)(P_j[q][q] + sum_{r in x,
  // r != q} P_j[r][q]); E_j = sum_{q in x} (P_j[q][q] + phi_j(q) / 2).
  auto rebuild = [&](const uint32_t *words, int64_t *E) {
    int64_t part[K];
#pragma unroll
    for (int j = 0; j < K; ++j) part[j] = 0;
    xm = 0;
#pragma unroll
    for (int k = 0; k < B; ++k) {
      if (!valid(k)) continue;
      const int q = k * T + tid;
      const int xq = (int)((words[q >> 5] >> (q & 31)) & 1u);
      xm |= (uint32_t)xq << k;
      int64_t phi[K];
#pragma unroll
      for (int j = 0; j < K; ++j) phi[j] = 0;
      for (int w = 0; w < W; ++w) {
        uint32_t word = words[w];
        while (word) {
          const int r = w * 32 + __ffs(word) - 1;
          word &= word - 1;
          if (r == q) continue;
#pragma unroll
          for (int j = 0; j < K; ++j) phi[j] += A.P[j * mm + (size_t)r * m + q];
        }
      }
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const int64_t d = A.P[j * mm + (size_t)q * m + q];
        dE[j][k] = (1 - 2 * xq) * (d + phi[j]);
        if (xq) part[j] += 2 * d + phi[j];
      }
    }
    // block sums of 2 E_j (phi counts every pair twice)
#pragma unroll
    for (int j = 0; j < K; ++j) {
      int64_t v = part[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
      if (lane == 0) sRed[warp * (K + 1) + j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < K; ++j) {
      int64_t t2 = 0;
      for (int w = 0; w < NW; ++w) t2 += sRed[w * (K + 1) + j];
      E[j] = t2 / 2;
    }
    __syncthreads();
  };

  // initial state: bit p is bit p % 32 of word (p / 32) % 4 of the draw
  // (p / 128, 0, replica, init) -- Alg. 3 "a random binary solution"
  uint32_t *sInit = reinterpret_cast<uint32_t *>(smem + L.init);  // [W]
  for (int w = tid; w < W; w += T) {
    uint32_t c[4] = {(uint32_t)w >> 2, 0u, rep, kTagInit};
    philox(c, k0, k1);
    const uint32_t v = (w & 3) == 0 ? c[0] : (w & 3) == 1 ? c[1] : (w & 3) == 2 ? c[2] : c[3];
    const int lo_bit = w * 32;
    sInit[w] = lo_bit + 32 <= m ? v : (v & ((1u << (m - lo_bit)) - 1u));
  }
  __syncthreads();
  int64_t E[K];
  rebuild(sInit, E);

  int acount = 0;
  int64_t Eoff = 0;
  uint32_t st[4] = {0, 0, 0, 0};
  for (uint32_t t = 1; t <= I_max; ++t) {
    const int buf = (int)(t & 1u);
    uint32_t *mask = sMask + buf * items;
    const uint32_t sn = (t <= (uint32_t)A.nsched ? t : (uint32_t)A.nsched) - 1;
    const double delta = A.sch_delta[sn];
    const int64_t lo = A.sch_lo[sn], hi = A.sch_hi[sn];
    bool acc_any = false;
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const bool in = valid(k);
      int64_t a = 0;
#pragma unroll
      for (int j = 0; j < K; ++j) {
        int64_t e = dE[j][k];
        if (A.escape == 1) e -= Eoff;
        const int64_t aj = e > 0 ? e : 0;
        if (A.accept == 0) a += aj;
        else a = (j == 0 || aj < a) ? aj : a;
      }
      bool acc = in && a <= lo;
      const bool need = in && a > lo && a <= hi;
      if (__any_sync(kFull, need)) {
        const int p = k * T + tid;
        uint32_t c[4] = {(uint32_t)p >> 2, t, rep, kTagAccept};
        philox(c, k0, k1);
        const uint32_t w = (p & 3) == 0 ? c[0] : (p & 3) == 1 ? c[1] : (p & 3) == 2 ? c[2] : c[3];
        if (need) acc = (double)a <= __dmul_rn(delta, A.table[w >> 16]);
      }
      const uint32_t bal = __ballot_sync(kFull, acc);
      if (lane == 0) mask[k * NW + warp] = bal;
      acc_any |= acc;
    }
    if (tid < 3) {  // select, restart, exploit draws of iteration t
      uint32_t c[4] = {0u, t, rep, kTagSelect + (uint32_t)tid};
      philox(c, k0, k1);
      sRnd[buf * 4 + tid] = c[0];
    }
    const int nacc = __syncthreads_count(acc_any);
    const uint32_t *rnd = sRnd + buf * 4;
    int64_t event = INT64_MIN;
    if (nacc > 0) {
      // Alg. 3: one flip at random among the accepted bits (ascending)
      const int total = count_bits(mask, items, lane);
      const int ps = select_bit(mask, items, NW, T, lane, pick(rnd[0], total));
      const int kk = ps / T;
      if (ps - kk * T == tid) {
#pragma unroll
        for (int k = 0; k < B; ++k) {
          if (k != kk) continue;
#pragma unroll
          for (int j = 0; j < K; ++j) sBc[j] = dE[j][k];
          sBc[K] = (xm >> k) & 1u;
        }
      }
      __syncthreads();
      const int sg = 1 - 2 * (int)sBc[K];  // +1: bit ps turns on
#pragma unroll
      for (int j = 0; j < K; ++j) E[j] += sBc[j];
#pragma unroll
      for (int k = 0; k < B; ++k) {
        if (!valid(k)) continue;
        const int q = k * T + tid;
        if (q == ps) {
#pragma unroll
          for (int j = 0; j < K; ++j) dE[j][k] = -dE[j][k];
          xm ^= 1u << k;
          continue;
        }
        const int g = sg * (1 - 2 * (int)((xm >> k) & 1u));
#pragma unroll
        for (int j = 0; j < K; ++j) dE[j][k] += (int64_t)g * A.P[j * mm + (size_t)ps * m + q];
      }
      Eoff = 0;
      // archive (Alg. 4 / Alg. 5): ballots of "x dominates slot y"
      int anyd = 0;
#pragma unroll
      for (int k = 0; k < B; ++k) {
        const int y = k * T + tid;
        bool dom = false;
        if (y < acount) {
          int64_t ye[K];
#pragma unroll
          for (int j = 0; j < K; ++j) ye[j] = gE[(size_t)y * K + j];
          dom = dominates<K>(E, ye);
          if (dominates<K>(ye, E)) anyd = 1;
        }
        const uint32_t bal = __ballot_sync(kFull, dom);
        if (lane == 0) sAmask[k * NW + warp] = bal;
      }
      anyd = __syncthreads_or(anyd);
      const int nb = count_bits(sAmask, items, lane);
      int target = -1;
      if (A.archive == 0) {
        if (nb > 0) target = select_bit(sAmask, items, NW, T, lane, 0);
        else if (acount < s) target = acount++;
      } else if (!anyd) {
        if (nb > 0) target = select_bit(sAmask, items, NW, T, lane, pick(rnd[2], nb));
        else if (acount < s) target = acount++;
      }
      if (target >= 0) {
#pragma unroll
        for (int k = 0; k < B; ++k) {
          const uint32_t wv = __ballot_sync(kFull, (xm >> k) & 1u);
          const int wi = k * NW + warp;
          if (lane == 0 && wi < W) gBits[(size_t)target * W + wi] = wv;
        }
        if (tid == 0)
          for (int j = 0; j < K; ++j) gE[(size_t)target * K + j] = E[j];
        if (gF) {
#pragma unroll
          for (int k = 0; k < B; ++k) {
            if (!valid(k)) continue;
#pragma unroll
            for (int j = 0; j < K; ++j)
              gF[((size_t)target * K + j) * m + k * T + tid] = dE[j][k];
          }
        }
      }
      ++st[0];
      event = ps;
    } else if (A.escape == 0 && acount > 0) {
      // Alg. 3: jump to a random archive member
      const int slot = pick(rnd[1], acount);
#pragma unroll
      for (int j = 0; j < K; ++j) E[j] = gE[(size_t)slot * K + j];
      const uint32_t *words = gBits + (size_t)slot * W;
      if (gF) {
        xm = 0;
#pragma unroll
        for (int k = 0; k < B; ++k) {
          if (!valid(k)) continue;
          const int q = k * T + tid;
          xm |= ((words[q >> 5] >> (q & 31)) & 1u) << k;
#pragma unroll
          for (int j = 0; j < K; ++j) dE[j][k] = gF[((size_t)slot * K + j) * m + q];
        }
      } else {
        int64_t Er[K];
        rebuild(words, Er);
      }
      ++st[1];
      event = -1 - (int64_t)slot;
    } else if (A.escape == 0) {
      ++st[2];
    } else {
      Eoff += A.beta;
      ++st[3];
    }
    if (A.trace && tid == 0) {
      int64_t *tr = A.trace + ((size_t)rb * I_max + (t - 1)) * (K + 1);
      for (int j = 0; j < K; ++j) tr[j] = E[j];
      tr[K] = event;
    }
  }
#pragma unroll
  for (int k = 0; k < B; ++k) {
    const uint32_t wv = __ballot_sync(kFull, (xm >> k) & 1u);
    const int wi = k * NW + warp;
    if (lane == 0 && wi < W) A.x_final[(size_t)rb * W + wi] = wv;
  }
  if (tid == 0) {
    A.arch_count[rb] = acount;
    for (int j = 0; j < K; ++j) A.E_final[(size_t)rb * K + j] = E[j];
    for (int q = 0; q < 4; ++q) A.stats[(size_t)rb * 4 + q] = st[q];
  }
}


template <int K, int B>
cudaError_t launch_qb(const QArgs &a, int R, int T, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(qubo_kernel<K, B>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  qubo_kernel<K, B><<<R, T, smem, st>>>(a);
  return cudaGetLastError();
}

template <int K>
cudaError_t launch_qk(const QArgs &a, int R, int T, int B, size_t smem, cudaStream_t st) {
  switch (B) {
    case 1: return launch_qb<K, 1>(a, R, T, smem, st);
    case 2: return launch_qb<K, 2>(a, R, T, smem, st);
    case 4: return launch_qb<K, 4>(a, R, T, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

moda_status qfail(moda_status st, const std::string &msg) {
  moda::set_last_error(msg);
  return st;
}

}  // namespace

struct moda_qubo_s {
  int32_t K = 0, m = 0, W = 0;
  int device = 0;
  int32_t *dP = nullptr;
};

struct moda_qrun_s {
  moda_qubo q = nullptr;
  int32_t R = 0, s = 0;
  int64_t I_max = 0;
  bool traced = false;
  cudaStream_t stream = nullptr;
  cudaEvent_t start = nullptr, stop = nullptr;
  int64_t *fcache = nullptr, *arch_E = nullptr, *E_final = nullptr, *stats = nullptr,
          *trace = nullptr;
  uint32_t *arch_bits = nullptr, *x_final = nullptr;
  int32_t *arch_count = nullptr;
};

namespace {
void free_qrun(moda_qrun r) {
  void *ptrs[] = {r->fcache, r->arch_E, r->E_final, r->stats, r->trace, r->arch_bits,
                  r->x_final, r->arch_count};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (r->start) cudaEventDestroy(r->start);
  if (r->stop) cudaEventDestroy(r->stop);
}
}  // namespace

extern "C" {

moda_status moda_qubo_create(int32_t K, int32_t m, const int32_t *Q, moda_qubo *out) {
  if (!out) return qfail(MODA_EINVAL, "out is NULL");
  *out = nullptr;
  if (!Q) return qfail(MODA_EINVAL, "NULL matrix");
  if (K < 1 || K > kMaxK) return qfail(MODA_EINVAL, "K must be in [1, 3]");
  if (m < 1 || m > 4 * kMaxQThreads) return qfail(MODA_EINVAL, "m must be in [1, 4096]");
  const size_t mm = (size_t)m * m;
  std::vector<int32_t> P((size_t)K * mm);
  for (int j = 0; j < K; ++j) {
    const int32_t *Qj = Q + (size_t)j * mm;
    for (int p = 0; p < m; ++p)
      for (int r = 0; r < m; ++r) {
        const int lo = p < r ? p : r, hi = p < r ? r : p;
        const int64_t v = p == r ? (int64_t)Qj[(size_t)p * m + p]
                                 : (int64_t)Qj[(size_t)lo * m + hi];  // upper triangle
        if (v > 2147483647ll || v < -2147483647ll)
          return qfail(MODA_EOVERFLOW, "an entry of Q + Q^T exceeds int32");
        P[(size_t)j * mm + (size_t)p * m + r] = (int32_t)v;
      }
  }
  moda_qubo q = new (std::nothrow) moda_qubo_s;
  if (!q) return qfail(MODA_ENOMEM, "host allocation");
  q->K = K;
  q->m = m;
  q->W = (m + 31) / 32;
  cudaGetDevice(&q->device);
  cudaError_t e = cudaMalloc(&q->dP, sizeof(int32_t) * P.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(q->dP, P.data(), sizeof(int32_t) * P.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (q->dP) cudaFree(q->dP);
    delete q;
    return qfail(MODA_ECUDA, std::string("upload: ") + cudaGetErrorString(e));
  }
  *out = q;
  return MODA_OK;
}

void moda_qubo_destroy(moda_qubo q) {
  if (!q) return;
  cudaFree(q->dP);
  delete q;
}

moda_status moda_qubo_anneal(moda_qubo q, const moda_params *p, void *cuda_stream,
                             moda_qrun *out) {
  if (!out) return qfail(MODA_EINVAL, "out is NULL");
  *out = nullptr;
  if (!q || !p) return qfail(MODA_EINVAL, "NULL argument");
  const int m = q->m, K = q->K;
  if (p->replicas < 1) return qfail(MODA_EINVAL, "replicas must be >= 1");
  if (p->I_max < 0 || p->I_max > 0xFFFFFFFFll)
    return qfail(MODA_EINVAL, "I_max must be in [0, 2^32)");
  if (!(p->delta0 > 0) || !(p->deltaf > 0) || !(p->xi > 0) || !(p->xi < 1))
    return qfail(MODA_EINVAL, "need delta0 > 0, deltaf > 0, 0 < xi < 1");
  if (p->beta < 0) return qfail(MODA_EINVAL, "beta must be >= 0");
  if (p->archive_size < 0 || p->archive_size > m)
    return qfail(MODA_EINVAL, "archive_size must be in [0, m]");
  if ((p->accept != MODA_STRICT && p->accept != MODA_LENIENT) ||
      (p->archive != MODA_EXPLORE && p->archive != MODA_EXPLOIT) ||
      (p->escape != MODA_ESC_ARCHIVE && p->escape != MODA_ESC_OFFSET))
    return qfail(MODA_EINVAL, "bad accept, archive or escape mode");
  if (p->normalize || p->snapshot_every || p->fast_forward)
    return qfail(MODA_EUNSUPPORTED,
                 "normalisation, snapshots and fast-forward are bQAP-path options");
  int B = 0;
  for (int b : {1, 2, 4})
    if ((int64_t)b * kMaxQThreads >= m) {
      B = b;
      break;
    }
  const int T = ((m + B - 1) / B + 31) / 32 * 32;
  const int s = p->archive_size > 0 ? p->archive_size : m;
  moda::ScheduleView sv{};
  cudaSetDevice(q->device);
  moda_status st = moda::schedule_view(q->device, p->delta0, p->deltaf, p->xi, p->I_max, &sv);
  if (st != MODA_OK) return st;
  moda_qrun r = new (std::nothrow) moda_qrun_s;
  if (!r) return qfail(MODA_ENOMEM, "host allocation");
  r->q = q;
  r->R = p->replicas;
  r->s = s;
  r->I_max = p->I_max;
  r->traced = p->trace != 0 && p->I_max > 0;
  r->stream = static_cast<cudaStream_t>(cuda_stream);
  const size_t R = (size_t)r->R, W = (size_t)q->W;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void **ptr, size_t nb) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, nb);
  };
  alloc((void **)&r->arch_E, R * s * K * sizeof(int64_t));
  alloc((void **)&r->arch_bits, R * s * W * sizeof(uint32_t));
  alloc((void **)&r->arch_count, R * sizeof(int32_t));
  alloc((void **)&r->x_final, R * W * sizeof(uint32_t));
  alloc((void **)&r->E_final, R * K * sizeof(int64_t));
  alloc((void **)&r->stats, R * 4 * sizeof(int64_t));
  if (r->traced) alloc((void **)&r->trace, R * (size_t)p->I_max * (K + 1) * sizeof(int64_t));
  // Delta E records of the archive members, when the escape jumps and they
  // fit in 60 % of the free memory (else jumps rebuild Delta E)
  const size_t cache_bytes = R * s * (size_t)K * m * sizeof(int64_t);
  if (e == cudaSuccess && p->escape == MODA_ESC_ARCHIVE && p->field_cache != 2) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && cache_bytes <= free_b / 10 * 6)
      alloc((void **)&r->fcache, cache_bytes);
  }
  if (e == cudaSuccess) e = cudaEventCreate(&r->start);
  if (e == cudaSuccess) e = cudaEventCreate(&r->stop);
  if (e != cudaSuccess) {
    free_qrun(r);
    delete r;
    return qfail(MODA_ENOMEM, std::string("device allocation: ") + cudaGetErrorString(e));
  }
  QArgs a{};
  a.m = m;
  a.W = q->W;
  a.s = s;
  a.nsched = sv.count;
  a.I_max = p->I_max;
  a.beta = p->beta;
  a.replica_base = (uint32_t)p->replica_base;
  a.seed_lo = (uint32_t)(p->seed & 0xFFFFFFFFull);
  a.seed_hi = (uint32_t)(p->seed >> 32);
  a.accept = p->accept;
  a.archive = p->archive;
  a.escape = p->escape;
  a.P = q->dP;
  a.sch_delta = sv.delta;
  a.sch_lo = sv.lo;
  a.sch_hi = sv.hi;
  a.table = sv.table;
  a.fcache = r->fcache;
  a.arch_E = r->arch_E;
  a.arch_bits = r->arch_bits;
  a.arch_count = r->arch_count;
  a.x_final = r->x_final;
  a.E_final = r->E_final;
  a.stats = r->stats;
  a.trace = r->trace;
  const size_t smem = qubo_layout(T, B, q->W).total;
  e = cudaEventRecord(r->start, r->stream);
  if (e == cudaSuccess) {
    switch (K) {
      case 1: e = launch_qk<1>(a, r->R, T, B, smem, r->stream); break;
      case 2: e = launch_qk<2>(a, r->R, T, B, smem, r->stream); break;
      default: e = launch_qk<3>(a, r->R, T, B, smem, r->stream); break;
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(r->stop, r->stream);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(r->stream);
    free_qrun(r);
    delete r;
    return qfail(MODA_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  }
  *out = r;
  return MODA_OK;
}

moda_status moda_qrun_wait(moda_qrun r) {
  if (!r) return qfail(MODA_EINVAL, "NULL run");
  cudaSetDevice(r->q->device);
  const cudaError_t e = cudaEventSynchronize(r->stop);
  if (e != cudaSuccess) return qfail(MODA_ECUDA, std::string("run: ") + cudaGetErrorString(e));
  return MODA_OK;
}

moda_status moda_qrun_read(moda_qrun r, int32_t *count, int64_t *E, uint32_t *bits,
                           uint32_t *x, int64_t *E_final, int64_t *stats, int64_t *trace) {
  if (!r) return qfail(MODA_EINVAL, "NULL run");
  cudaSetDevice(r->q->device);
  if (cudaEventQuery(r->stop) != cudaSuccess) return qfail(MODA_EBUSY, "run still executing");
  const size_t R = (size_t)r->R, s = (size_t)r->s, K = (size_t)r->q->K, W = (size_t)r->q->W;
  struct Item {
    void *dst;
    const void *src;
    size_t bytes;
  } items[] = {
      {count, r->arch_count, R * sizeof(int32_t)},
      {E, r->arch_E, R * s * K * sizeof(int64_t)},
      {bits, r->arch_bits, R * s * W * sizeof(uint32_t)},
      {x, r->x_final, R * W * sizeof(uint32_t)},
      {E_final, r->E_final, R * K * sizeof(int64_t)},
      {stats, r->stats, R * 4 * sizeof(int64_t)},
      {trace, r->trace, r->traced ? R * (size_t)r->I_max * (K + 1) * sizeof(int64_t) : 0},
  };
  for (const Item &it : items) {
    if (!it.dst || !it.bytes) continue;
    const cudaError_t e = cudaMemcpy(it.dst, it.src, it.bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return qfail(MODA_ECUDA, std::string("read: ") + cudaGetErrorString(e));
  }
  if (trace && !r->traced) return qfail(MODA_EINVAL, "the run kept no trace");
  return MODA_OK;
}

moda_status moda_qrun_elapsed_ms(moda_qrun r, float *ms) {
  if (!r || !ms) return qfail(MODA_EINVAL, "NULL argument");
  const cudaError_t e = cudaEventElapsedTime(ms, r->start, r->stop);
  if (e != cudaSuccess) return qfail(MODA_ECUDA, cudaGetErrorString(e));
  return MODA_OK;
}

void moda_qrun_destroy(moda_qrun r) {
  if (!r) return;
  cudaSetDevice(r->q->device);
  if (r->stop) cudaEventSynchronize(r->stop);
  free_qrun(r);
  delete r;
}

}  // extern "C"
