// Device helpers shared by the annealing kernels (moda_kernel_body.cuh,
// moda_warp.cuh): the Philox4x32-10 counter generator, index picks, bit
// selection, dominance, and the mbarrier / bulk-copy (TMA) wrappers.
#pragma once

#include <cstdint>

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

// Position of the r-th (0-based) set bit of `mask`, r < popc(mask): a
// binary search on the set-bit counts of halves, quarters, ...
__device__ __forceinline__ int nth_set_bit(uint32_t mask, int r) {
  int pos = 0;
  int c = __popc(mask & 0xFFFFu);
  if (r >= c) {
    r -= c;
    pos = 16;
  }
  uint32_t m = mask >> pos;
  c = __popc(m & 0xFFu);
  if (r >= c) {
    r -= c;
    pos += 8;
    m >>= 8;
  }
  c = __popc(m & 0xFu);
  if (r >= c) {
    r -= c;
    pos += 4;
    m >>= 4;
  }
  c = __popc(m & 0x3u);
  if (r >= c) {
    r -= c;
    pos += 2;
    m >>= 2;
  }
  if (r >= (int)(m & 1u)) pos += 1;
  return pos;
}

// Flat index round*Tw + warp*32 + lane of the lowest set bit over `items`
// ballot masks in (round, warp) order, or -1 if none, in every lane.
__device__ __forceinline__ int warp_mask_first(const uint32_t *masks, int items, int nw,
                                               int Tw, int lane) {
  for (int q0 = 0; q0 < items; q0 += 32) {
    const int it = q0 + lane;
    const uint32_t mk = it < items ? masks[it] : 0u;
    const unsigned nz = __ballot_sync(kFull, mk != 0u);
    if (nz) {
      const int L = __ffs(nz) - 1;
      const uint32_t w = __shfl_sync(kFull, mk, L);
      const int k = (q0 + L) / nw;
      const int wi = q0 + L - k * nw;
      return k * Tw + wi * 32 + __ffs(w) - 1;
    }
  }
  return -1;
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
// Bulk prefetch of global memory into L2 (no destination, no completion
// signal); address 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// Asynchronous 8-byte copy global -> shared (both 8-byte aligned); a
// thread's copies complete at cp_async_wait_all.
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}
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
// Waits for the phase of parity `parity` of `bar` to complete, at most
// kWaitLimit polls; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (int i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// The acceptance test of a bit whose penalty a (an integer >= 0) lies in
// (lo_t, hi_t] is a <= fl(delta T) (R7).  This part's FP64 rate is low, so
// it is first decided in FP32 where that is exact: with df = fl32(delta),
// Tf = fl32(T) and pf = fl32(df Tf), pf lies within (1 +- 2^-24)^3 of
// delta T, fl(delta T) within 2^-53 of it, and af = fl32(a) within 2^-24 of
// a.  Hence af <= fl32(pf (1 - 2^-20)) implies a <= (1 - 11 2^-24)
// fl(delta T) (accept, 1), and af >= fl32(pf (1 + 2^-20)) implies
// a >= (1 + 11 2^-24) fl(delta T) (reject, 0).  Otherwise (-1, a within
// about 2^-20 of the product, rare) the caller takes the double test.
// fl32(a) of a penalty a >= 0: the 32-bit conversion whenever a fits it
// (the 64-bit one is slow here), both rounding to nearest.
__device__ __forceinline__ float penalty_f32(int64_t a) {
  return a < 0x100000000ll ? __uint2float_rn((uint32_t)a) : __ll2float_rn(a);
}

__device__ __forceinline__ int prefilter(float af, float df, float Tf) {
  const float pf = __fmul_rn(df, Tf);
  if (af <= __fmul_rn(pf, 1.0f - 0x1p-20f)) return 1;
  if (af >= __fmul_rn(pf, 1.0f + 0x1p-20f)) return 0;
  return -1;
}

// Inclusive prefix sum of `v` over the lanes.
__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int u = __shfl_up_sync(kFull, v, d);
    if (lane >= d) v += u;
  }
  return v;
}

}  // namespace
}  // namespace moda
