// Launches of the annealing kernel (moda_kernel_body.cuh) in modes 2 to 4:
// the fast-forward bookkeeping (2), the default algorithm compiled in (3),
// and the default algorithm with the on-chip placement, one bit per thread
// (4).  Instantiated apart from modes 0 and 1 (moda_kernel.cu) so that the
// two translation units compile side by side.
#include "moda_kernel_body.cuh"

namespace moda {
namespace {

template <int B, bool NARROW>
cudaError_t launch_bm(const AnnealArgs &args, int replicas, int workers, int mode,
                      size_t smem, cudaStream_t stream) {
  if constexpr (B == 1)
    if (mode == 4) return launch_bn<B, NARROW, 4>(args, replicas, workers, smem, stream);
  return mode == 3 ? launch_bn<B, NARROW, 3>(args, replicas, workers, smem, stream)
                   : launch_bn<B, NARROW, 2>(args, replicas, workers, smem, stream);
}

template <int B>
cudaError_t launch_b(const AnnealArgs &args, int replicas, int workers, bool narrow, int mode,
                     size_t smem, cudaStream_t stream) {
  return narrow ? launch_bm<B, true>(args, replicas, workers, mode, smem, stream)
                : launch_bm<B, false>(args, replicas, workers, mode, smem, stream);
}

template <int B, bool NARROW>
const void *kernel_of(int mode) {
  if constexpr (B == 1)
    if (mode == 4) return kernel_ptr<B, NARROW, 4>();
  return mode == 3 ? kernel_ptr<B, NARROW, 3>() : kernel_ptr<B, NARROW, 2>();
}

template <int B>
cudaError_t function_b(bool narrow, int mode, size_t smem, const void **func) {
  const void *f = narrow ? kernel_of<B, true>(mode) : kernel_of<B, false>(mode);
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) *func = f;
  return e;
}

}  // namespace

cudaError_t anneal_function_special(int rounds, bool narrow, int mode, size_t smem,
                                    const void **func) {
  if (mode < 2 || mode > 4) return cudaErrorInvalidValue;
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

cudaError_t launch_anneal_special(const AnnealArgs &args, int replicas, int workers, int rounds,
                                  bool narrow, int mode, size_t smem, cudaStream_t stream) {
  if (mode < 2 || mode > 4) return cudaErrorInvalidValue;
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
