// Pass-1 kernels for the class table with computed columns plus the two-byte stride table
// over the hot states (kClassPair).  Its emit and tiny kernels are those of kClassWin: the
// class table sits at the same place and the pair table is used by the main run only.
#include "parem_launch.h"
#include "parem_scan.cuh"

namespace parem {

cudaError_t scan_pair(uint32_t esize, uint32_t P, const CUtensorMap& tm, const ScanParams& p, int grid, int block,
                      size_t smem, cudaStream_t s) {
  switch (esize * 16 + P) {
    case 16 + 1: return launch_spec_scan<kClassPair, 1, 1>(tm, p, grid, block, smem, s);
    case 16 + 2: return launch_spec_scan<kClassPair, 1, 2>(tm, p, grid, block, smem, s);
    case 16 + 4: return launch_spec_scan<kClassPair, 1, 4>(tm, p, grid, block, smem, s);
    case 16 + 8: return launch_spec_scan<kClassPair, 1, 8>(tm, p, grid, block, smem, s);
    case 32 + 1: return launch_spec_scan<kClassPair, 2, 1>(tm, p, grid, block, smem, s);
    case 32 + 2: return launch_spec_scan<kClassPair, 2, 2>(tm, p, grid, block, smem, s);
    case 32 + 4: return launch_spec_scan<kClassPair, 2, 4>(tm, p, grid, block, smem, s);
    default: return launch_spec_scan<kClassPair, 2, 8>(tm, p, grid, block, smem, s);
  }
}

}  // namespace parem
