// Kernels for the class-indexed table in shared memory.
#include "parem_launch.h"
#include "parem_scan.cuh"

namespace parem {

cudaError_t scan_class(uint32_t esize, uint32_t P, const CUtensorMap& tm, const ScanParams& p, int grid,
                       int block, size_t smem, cudaStream_t s) {
  if (esize == 1)
    return P == 1 ? launch_spec_scan<kClassSmem, 1, 1>(tm, p, grid, block, smem, s)
                  : launch_spec_scan<kClassSmem, 1, 8>(tm, p, grid, block, smem, s);
  return P == 1 ? launch_spec_scan<kClassSmem, 2, 1>(tm, p, grid, block, smem, s)
                : launch_spec_scan<kClassSmem, 2, 8>(tm, p, grid, block, smem, s);
}

cudaError_t emit_class(uint32_t esize, const ScanParams& p, int grid, int block, size_t smem, cudaStream_t s) {
  return esize == 1 ? launch_emit<kClassSmem, 1>(p, grid, block, smem, s)
                    : launch_emit<kClassSmem, 2>(p, grid, block, smem, s);
}

cudaError_t tiny_class(uint32_t esize, const ScanParams& p, size_t smem, cudaStream_t s) {
  return esize == 1 ? launch_tiny<kClassSmem, 1>(p, smem, s) : launch_tiny<kClassSmem, 2>(p, smem, s);
}

}  // namespace parem
