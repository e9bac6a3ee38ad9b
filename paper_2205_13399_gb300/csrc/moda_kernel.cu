// Launches of the annealing kernel (moda_kernel_body.cuh): the plain and
// the extensions variants (modes 0 and 1) and the default algorithm with
// archive states in global memory (mode 5, 2 to 4 bits per thread) are
// instantiated here, modes 2 to 4 in moda_kernel_special.cu, so the two
// compile side by side.  This file also holds the dispatch on (rounds,
// narrow, mode) used by the host library.
#include "moda_kernel_body.cuh"

namespace moda {
namespace {

template <int B, bool NARROW>
cudaError_t launch_bm(const AnnealArgs &args, int replicas, int workers, int mode,
                      size_t smem, cudaStream_t stream) {
  if constexpr (B >= 2 && B <= 4)
    if (mode == 5) return launch_bn<B, NARROW, 5>(args, replicas, workers, smem, stream);
  return mode == 1 ? launch_bn<B, NARROW, 1>(args, replicas, workers, smem, stream)
                   : launch_bn<B, NARROW, 0>(args, replicas, workers, smem, stream);
}

template <int B>
cudaError_t launch_b(const AnnealArgs &args, int replicas, int workers, bool narrow, int mode,
                     size_t smem, cudaStream_t stream) {
  return narrow ? launch_bm<B, true>(args, replicas, workers, mode, smem, stream)
                : launch_bm<B, false>(args, replicas, workers, mode, smem, stream);
}

template <int B, bool NARROW>
const void *kernel_of(int mode) {
  if constexpr (B >= 2 && B <= 4)
    if (mode == 5) return kernel_ptr<B, NARROW, 5>();
  return mode == 1 ? kernel_ptr<B, NARROW, 1>() : kernel_ptr<B, NARROW, 0>();
}

template <int B>
cudaError_t function_b(bool narrow, int mode, size_t smem, const void **func) {
  const void *f = narrow ? kernel_of<B, true>(mode) : kernel_of<B, false>(mode);
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) *func = f;
  return e;
}

}  // namespace

bool supported_rounds(int b) {
  return b == 1 || b == 2 || b == 3 || b == 4 || b == 6 || b == 8;
}

cudaError_t anneal_function(int rounds, bool narrow, int mode, size_t smem,
                            const void **func) {
  if (mode >= 2 && mode <= 4) return anneal_function_special(rounds, narrow, mode, smem, func);
  switch (rounds) {
    case 1: return function_b<1>(narrow, mode, smem, func);
    case 2: return function_b<2>(narrow, mode, smem, func);
    case 3: return function_b<3>(narrow, mode, smem, func);
    case 4: return function_b<4>(narrow, mode, smem, func);
    case 6: return function_b<6>(narrow, mode, smem, func);
    case 8: return function_b<8>(narrow, mode, smem, func);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_anneal(const AnnealArgs &args, int replicas, int workers,
                          int rounds, bool narrow, size_t smem, cudaStream_t stream) {
  if (workers % 32 || workers < 32 || workers > kMaxWorkers) return cudaErrorInvalidValue;
  const int mode = kernel_mode(args, rounds);
  if (mode >= 2 && mode <= 4)
    return launch_anneal_special(args, replicas, workers, rounds, narrow, mode, smem, stream);
  switch (rounds) {
    case 1: return launch_b<1>(args, replicas, workers, narrow, mode, smem, stream);
    case 2: return launch_b<2>(args, replicas, workers, narrow, mode, smem, stream);
    case 3: return launch_b<3>(args, replicas, workers, narrow, mode, smem, stream);
    case 4: return launch_b<4>(args, replicas, workers, narrow, mode, smem, stream);
    case 6: return launch_b<6>(args, replicas, workers, narrow, mode, smem, stream);
    case 8: return launch_b<8>(args, replicas, workers, narrow, mode, smem, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace moda
