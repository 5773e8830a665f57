// Kernels for the class table in shared memory with computed columns (kClassWin): bytes of
// one ASCII window and one extra byte have their own columns, every other byte shares one.
#include "parem_launch.h"
#include "parem_scan.cuh"

namespace parem {

cudaError_t scan_win(uint32_t esize, uint32_t P, const CUtensorMap& tm, const ScanParams& p, int grid, int block,
                     size_t smem, cudaStream_t s) {
  switch (esize * 16 + P) {
    case 16 + 1: return launch_spec_scan<kClassWin, 1, 1>(tm, p, grid, block, smem, s);
    case 16 + 2: return launch_spec_scan<kClassWin, 1, 2>(tm, p, grid, block, smem, s);
    case 16 + 4: return launch_spec_scan<kClassWin, 1, 4>(tm, p, grid, block, smem, s);
    case 16 + 8: return launch_spec_scan<kClassWin, 1, 8>(tm, p, grid, block, smem, s);
    case 32 + 1: return launch_spec_scan<kClassWin, 2, 1>(tm, p, grid, block, smem, s);
    case 32 + 2: return launch_spec_scan<kClassWin, 2, 2>(tm, p, grid, block, smem, s);
    case 32 + 4: return launch_spec_scan<kClassWin, 2, 4>(tm, p, grid, block, smem, s);
    default: return launch_spec_scan<kClassWin, 2, 8>(tm, p, grid, block, smem, s);
  }
}

cudaError_t emit_win(uint32_t esize, const ScanParams& p, const CUtensorMap* tm,
                     int grid, int block, size_t smem, cudaStream_t s) {
  return esize == 1 ? launch_emit<kClassWin, 1>(p, tm, grid, block, smem, s)
                    : launch_emit<kClassWin, 2>(p, tm, grid, block, smem, s);
}

cudaError_t tiny_win(uint32_t esize, const ScanParams& p, size_t smem, cudaStream_t s) {
  return esize == 1 ? launch_tiny<kClassWin, 1>(p, smem, s) : launch_tiny<kClassWin, 2>(p, smem, s);
}

}  // namespace parem
