// Batch kernels (one persistent launch over many (text, DFA) items).
#define PAREM_BATCH_KERNELS
#include "parem_launch.h"
#include "parem_scan.cuh"

namespace parem {

cudaError_t launch_batch_scan(const BatchParams& bp, int grid, int block, size_t smem, cudaStream_t s) {
  // two block shapes: 24 warps at 80 registers, or 16 warps at 128
  if (block == 768) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_batch_scan<768>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_batch_scan<768><<<grid, block, smem, s>>>(bp);
  } else if (block == 512) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_batch_scan<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_batch_scan<512><<<grid, block, smem, s>>>(bp);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_emit(const BatchParams& bp, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_batch_emit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_batch_emit<<<grid, 256, smem, s>>>(bp);
  return cudaGetLastError();
}

cudaError_t launch_batch_tiny(const BatchParams& bp, const uint32_t* tiny_items, uint32_t n_tiny, cudaStream_t s) {
  k_batch_tiny<<<(n_tiny + 127) / 128, 128, 0, s>>>(bp, tiny_items, n_tiny);
  return cudaGetLastError();
}

}  // namespace parem
