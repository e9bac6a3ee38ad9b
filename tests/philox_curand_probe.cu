// Test helper: raw Philox4x32-10 words from NVIDIA's cuRAND device API, used
// to pin the oracle's own Philox (and, through parity, the kernel's) to an
// independent implementation.  curand_init(seed, subsequence, offset) with
// offset = 4 * (c0 + 2^32 c1) and subsequence = c2 + 2^32 c3 leaves the
// generator at counter (c0, c1, c2, c3) under key (seed lo, seed hi); the
// first curand4() returns the Philox output of that counter.
#include <cstdint>

#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void probe(const uint32_t *ctr, const uint64_t *seed, uint32_t *out, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  curandStatePhilox4_32_10_t st;
  const uint64_t off = 4ull * ((uint64_t)ctr[4 * i] | ((uint64_t)ctr[4 * i + 1] << 32));
  const uint64_t sub = (uint64_t)ctr[4 * i + 2] | ((uint64_t)ctr[4 * i + 3] << 32);
  curand_init(seed[i], sub, off, &st);
  const uint4 v = curand4(&st);
  out[4 * i + 0] = v.x;
  out[4 * i + 1] = v.y;
  out[4 * i + 2] = v.z;
  out[4 * i + 3] = v.w;
}

extern "C" int philox_curand(const uint32_t *ctr, const uint64_t *seed, uint32_t *out,
                             int count) {
  uint32_t *dc = nullptr, *dout = nullptr;
  uint64_t *ds = nullptr;
  if (cudaMalloc(&dc, 16ull * count) != cudaSuccess) return 1;
  if (cudaMalloc(&ds, 8ull * count) != cudaSuccess) return 1;
  if (cudaMalloc(&dout, 16ull * count) != cudaSuccess) return 1;
  cudaMemcpy(dc, ctr, 16ull * count, cudaMemcpyHostToDevice);
  cudaMemcpy(ds, seed, 8ull * count, cudaMemcpyHostToDevice);
  probe<<<(count + 127) / 128, 128>>>(dc, ds, dout, count);
  cudaError_t e = cudaMemcpy(out, dout, 16ull * count, cudaMemcpyDeviceToHost);
  cudaFree(dc);
  cudaFree(ds);
  cudaFree(dout);
  return e == cudaSuccess ? 0 : 2;
}
