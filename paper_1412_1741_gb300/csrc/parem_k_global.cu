// Kernels for tables too large for shared memory: class-indexed, read from global memory
// through the read-only path (the table stays resident in the 126 MB L2).
#include "parem_launch.h"
#include "parem_scan.cuh"

namespace parem {

cudaError_t scan_global(uint32_t esize, uint32_t P, const CUtensorMap& tm, const ScanParams& p, int grid,
                        int block, size_t smem, cudaStream_t s) {
  (void)esize;
  return P == 1 ? launch_spec_scan<kClassGlobal, 2, 1>(tm, p, grid, block, smem, s)
                : launch_spec_scan<kClassGlobal, 2, 8>(tm, p, grid, block, smem, s);
}

cudaError_t emit_global(uint32_t esize, const ScanParams& p, int grid, int block, size_t smem, cudaStream_t s) {
  (void)esize;
  return launch_emit<kClassGlobal, 2>(p, grid, block, smem, s);
}

cudaError_t tiny_global(uint32_t esize, const ScanParams& p, size_t smem, cudaStream_t s) {
  (void)esize;
  return launch_tiny<kClassGlobal, 2>(p, smem, s);
}

cudaError_t launch_scan_dispatch(uint32_t layout, uint32_t esize, uint32_t P, const CUtensorMap& tm,
                                 const ScanParams& p, int grid, int block, size_t smem, cudaStream_t s) {
  switch (layout) {
    case kByteSmem: return scan_byte(esize, P, tm, p, grid, block, smem, s);
    case kClassSmem: return scan_class(esize, P, tm, p, grid, block, smem, s);
    default: return scan_global(esize, P, tm, p, grid, block, smem, s);
  }
}

cudaError_t launch_emit_dispatch(uint32_t layout, uint32_t esize, const ScanParams& p, int grid, int block,
                                 size_t smem, cudaStream_t s) {
  switch (layout) {
    case kByteSmem: return emit_byte(esize, p, grid, block, smem, s);
    case kClassSmem: return emit_class(esize, p, grid, block, smem, s);
    default: return emit_global(esize, p, grid, block, smem, s);
  }
}

cudaError_t launch_tiny_dispatch(uint32_t layout, uint32_t esize, const ScanParams& p, size_t smem,
                                 cudaStream_t s) {
  switch (layout) {
    case kByteSmem: return tiny_byte(esize, p, smem, s);
    case kClassSmem: return tiny_class(esize, p, smem, s);
    default: return tiny_global(esize, p, smem, s);
  }
}

}  // namespace parem
