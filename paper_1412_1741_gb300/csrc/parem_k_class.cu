// Kernels for the class-indexed table in shared memory.
#include "parem_launch.h"
#include "parem_scan.cuh"

namespace parem {

cudaError_t scan_class(uint32_t esize, uint32_t P, const CUtensorMap& tm, const ScanParams& p, int grid,
                       int block, size_t smem, cudaStream_t s) {
  switch (esize * 16 + P) {
    case 16 + 1: return launch_spec_scan<kClassSmem, 1, 1>(tm, p, grid, block, smem, s);
    case 16 + 2: return launch_spec_scan<kClassSmem, 1, 2>(tm, p, grid, block, smem, s);
    case 16 + 4: return launch_spec_scan<kClassSmem, 1, 4>(tm, p, grid, block, smem, s);
    case 16 + 8: return launch_spec_scan<kClassSmem, 1, 8>(tm, p, grid, block, smem, s);
    case 32 + 1: return launch_spec_scan<kClassSmem, 2, 1>(tm, p, grid, block, smem, s);
    case 32 + 2: return launch_spec_scan<kClassSmem, 2, 2>(tm, p, grid, block, smem, s);
    case 32 + 4: return launch_spec_scan<kClassSmem, 2, 4>(tm, p, grid, block, smem, s);
    default: return launch_spec_scan<kClassSmem, 2, 8>(tm, p, grid, block, smem, s);
  }
}

// wide column map (column offsets above 255): class counts above 127 with 2-byte entries
cudaError_t scan_class_wide(uint32_t P, const CUtensorMap& tm, const ScanParams& p, int grid, int block,
                            size_t smem, cudaStream_t s) {
  switch (P) {
    case 1: return launch_spec_scan<kClassSmemW, 2, 1>(tm, p, grid, block, smem, s);
    case 2: return launch_spec_scan<kClassSmemW, 2, 2>(tm, p, grid, block, smem, s);
    case 4: return launch_spec_scan<kClassSmemW, 2, 4>(tm, p, grid, block, smem, s);
    default: return launch_spec_scan<kClassSmemW, 2, 8>(tm, p, grid, block, smem, s);
  }
}

cudaError_t emit_class(uint32_t esize, const ScanParams& p, const CUtensorMap* tm,
                       int grid, int block, size_t smem, cudaStream_t s) {
  return esize == 1 ? launch_emit<kClassSmem, 1>(p, tm, grid, block, smem, s)
                    : launch_emit<kClassSmem, 2>(p, tm, grid, block, smem, s);
}

cudaError_t emit_class_wide(const ScanParams& p, const CUtensorMap* tm,
                            int grid, int block, size_t smem, cudaStream_t s) {
  return launch_emit<kClassSmemW, 2>(p, tm, grid, block, smem, s);
}

cudaError_t tiny_class(uint32_t esize, const ScanParams& p, size_t smem, cudaStream_t s) {
  return esize == 1 ? launch_tiny<kClassSmem, 1>(p, smem, s) : launch_tiny<kClassSmem, 2>(p, smem, s);
}

cudaError_t tiny_class_wide(const ScanParams& p, size_t smem, cudaStream_t s) {
  return launch_tiny<kClassSmemW, 2>(p, smem, s);
}

}  // namespace parem
