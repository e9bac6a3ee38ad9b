// On-chip peak probes declared in include/moda_peaks.h: integer lane
// operations per second and shared-memory load bandwidth, the two limits of
// the annealing kernel's roofline.
#include <cstdint>
#include <string>

#include "moda_internal.h"
#include "moda_peaks.h"

namespace {

constexpr int kThreads = 512;
constexpr int kChains = 8;

// Eight independent chains; each round applies 4 single-instruction
// operations to each chain (32 per thread per round).  The result feeds a
// conditional store so that nothing is dead.
__global__ void __launch_bounds__(kThreads) int_probe(int32_t iters, uint32_t seed,
                                                      uint32_t *sink) {
  uint32_t a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed ^ (threadIdx.x * 0x9E3779B9u + c);
  const uint32_t k1 = seed | 1u, k2 = seed * 3u + 7u, k3 = seed ^ 0x85EBCA6Bu;
  for (int32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      a[c] = a[c] * k1 + k2;               // multiply-add
      a[c] = a[c] ^ k3 ^ (uint32_t)i;      // three-input xor
      a[c] = a[c] + k2 + (uint32_t)c;      // three-input add
      a[c] = a[c] < k1 ? a[c] : a[c] - k1; // min-like select
    }
  }
  uint32_t r = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) r ^= a[c];
  if (r == seed) sink[blockIdx.x] = r;  // practically never taken
}

__global__ void __launch_bounds__(kThreads) smem_probe(int32_t iters, uint32_t seed,
                                                       uint32_t *sink) {
  __shared__ uint4 buf[2048];  // 32 KiB
  for (int e = threadIdx.x; e < 2048; e += kThreads)
    buf[e] = make_uint4(seed + e, seed ^ e, seed * e, e);
  __syncthreads();
  uint4 acc = make_uint4(0, 0, 0, 0);
  // lane l reads vector (base + l) % 2048: a warp covers 512 consecutive
  // bytes, four conflict-free wavefronts of 128 bytes
  uint32_t base = (threadIdx.x >> 5) * 64u;
  for (int32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint4 v = buf[(base + q * 256u + (threadIdx.x & 31)) & 2047u];
      acc.x ^= v.x;
      acc.y += v.y;
      acc.z ^= v.z;
      acc.w += v.w;
    }
    base += 32u;
  }
  if ((acc.x ^ acc.y ^ acc.z ^ acc.w) == seed) sink[blockIdx.x] = acc.x;
}

template <typename K>
moda_status run_probe(K kernel, int32_t iters, void *cuda_stream, float *ms, int *blocks) {
  if (iters < 1) {
    moda::set_last_error("iters must be >= 1");
    return MODA_EINVAL;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  uint32_t *sink = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(uint32_t) * 4 * (size_t)sms);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  *blocks = 4 * sms;
  if (e == cudaSuccess) {
    kernel<<<*blocks, kThreads, 0, st>>>(1, 12345u, sink);  // warm-up
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  if (e == cudaSuccess) {
    kernel<<<*blocks, kThreads, 0, st>>>(iters, 12345u, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) {
    moda::set_last_error(std::string("probe: ") + cudaGetErrorString(e));
    return MODA_ECUDA;
  }
  return MODA_OK;
}

}  // namespace

extern "C" {

moda_status moda_probe_int_peak(int32_t iters, void *cuda_stream, double *ops_per_s,
                                float *ms) {
  if (!ops_per_s || !ms) {
    moda::set_last_error("NULL output");
    return MODA_EINVAL;
  }
  int blocks = 0;
  moda_status st = run_probe(int_probe, iters, cuda_stream, ms, &blocks);
  if (st != MODA_OK) return st;
  const double ops = (double)blocks * kThreads * (double)iters * kChains * 4.0;
  *ops_per_s = ops / (*ms * 1e-3);
  return MODA_OK;
}

moda_status moda_probe_smem_peak(int32_t iters, void *cuda_stream, double *bytes_per_s,
                                 float *ms) {
  if (!bytes_per_s || !ms) {
    moda::set_last_error("NULL output");
    return MODA_EINVAL;
  }
  int blocks = 0;
  moda_status st = run_probe(smem_probe, iters, cuda_stream, ms, &blocks);
  if (st != MODA_OK) return st;
  const double bytes = (double)blocks * kThreads * (double)iters * 8.0 * 16.0;
  *bytes_per_s = bytes / (*ms * 1e-3);
  return MODA_OK;
}

}  // extern "C"
