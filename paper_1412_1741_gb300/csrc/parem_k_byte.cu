// Kernels for the byte-indexed table in shared memory (up to ~96 KiB of table).
#include "parem_launch.h"
#include "parem_scan.cuh"

namespace parem {

cudaError_t scan_byte(uint32_t esize, uint32_t P, const CUtensorMap& tm, const ScanParams& p, int grid,
                      int block, size_t smem, cudaStream_t s) {
  switch (esize * 16 + P) {
    case 16 + 1: return launch_spec_scan<kByteSmem, 1, 1>(tm, p, grid, block, smem, s);
    case 16 + 2: return launch_spec_scan<kByteSmem, 1, 2>(tm, p, grid, block, smem, s);
    case 16 + 4: return launch_spec_scan<kByteSmem, 1, 4>(tm, p, grid, block, smem, s);
    case 16 + 8: return launch_spec_scan<kByteSmem, 1, 8>(tm, p, grid, block, smem, s);
    case 32 + 1: return launch_spec_scan<kByteSmem, 2, 1>(tm, p, grid, block, smem, s);
    case 32 + 2: return launch_spec_scan<kByteSmem, 2, 2>(tm, p, grid, block, smem, s);
    case 32 + 4: return launch_spec_scan<kByteSmem, 2, 4>(tm, p, grid, block, smem, s);
    default: return launch_spec_scan<kByteSmem, 2, 8>(tm, p, grid, block, smem, s);
  }
}

cudaError_t emit_byte(uint32_t esize, const ScanParams& p, const CUtensorMap* tm,
                      int grid, int block, size_t smem, cudaStream_t s) {
  return esize == 1 ? launch_emit<kByteSmem, 1>(p, tm, grid, block, smem, s)
                    : launch_emit<kByteSmem, 2>(p, tm, grid, block, smem, s);
}

cudaError_t tiny_byte(uint32_t esize, const ScanParams& p, size_t smem, cudaStream_t s) {
  return esize == 1 ? launch_tiny<kByteSmem, 1>(p, smem, s) : launch_tiny<kByteSmem, 2>(p, smem, s);
}

}  // namespace parem

namespace parem {

// Small DFAs with the 4-byte stride table (candidate sets of at most 32 states: P = 1).
cudaError_t scan_byte_stride(const CUtensorMap& tm, const ScanParams& p, int grid, int block, size_t smem,
                             cudaStream_t s) {
  return launch_spec_scan<kByteStride, 1, 1>(tm, p, grid, block, smem, s);
}

cudaError_t emit_byte_stride(const ScanParams& p, const CUtensorMap* tm,
                             int grid, int block, size_t smem, cudaStream_t s) {
  return launch_emit<kByteStride, 1>(p, tm, grid, block, smem, s);
}

cudaError_t tiny_byte_stride(const ScanParams& p, size_t smem, cudaStream_t s) {
  return launch_tiny<kByteStride, 1>(p, smem, s);
}

}  // namespace parem
