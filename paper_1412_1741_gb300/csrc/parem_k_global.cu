// Kernels for tables too large for shared memory: class-indexed, read from global memory
// through the read-only path (the table stays resident in the 126 MB L2).
#include "parem_launch.h"
#include "parem_scan.cuh"

namespace parem {

cudaError_t scan_global(uint32_t wide, uint32_t P, const CUtensorMap& tm, const ScanParams& p, int grid,
                        int block, size_t smem, cudaStream_t s) {
  if (wide) {
    switch (P) {
      case 1: return launch_spec_scan<kClassGlobalW, 2, 1>(tm, p, grid, block, smem, s);
      case 2: return launch_spec_scan<kClassGlobalW, 2, 2>(tm, p, grid, block, smem, s);
      case 4: return launch_spec_scan<kClassGlobalW, 2, 4>(tm, p, grid, block, smem, s);
      default: return launch_spec_scan<kClassGlobalW, 2, 8>(tm, p, grid, block, smem, s);
    }
  }
  switch (P) {
    case 1: return launch_spec_scan<kClassGlobal, 2, 1>(tm, p, grid, block, smem, s);
    case 2: return launch_spec_scan<kClassGlobal, 2, 2>(tm, p, grid, block, smem, s);
    case 4: return launch_spec_scan<kClassGlobal, 2, 4>(tm, p, grid, block, smem, s);
    default: return launch_spec_scan<kClassGlobal, 2, 8>(tm, p, grid, block, smem, s);
  }
}

cudaError_t emit_global(uint32_t wide, const ScanParams& p, const CUtensorMap* tm,
                        int grid, int block, size_t smem, cudaStream_t s) {
  return wide ? launch_emit<kClassGlobalW, 2>(p, tm, grid, block, smem, s)
              : launch_emit<kClassGlobal, 2>(p, tm, grid, block, smem, s);
}

cudaError_t tiny_global(uint32_t wide, const ScanParams& p, size_t smem, cudaStream_t s) {
  return wide ? launch_tiny<kClassGlobalW, 2>(p, smem, s) : launch_tiny<kClassGlobal, 2>(p, smem, s);
}

cudaError_t launch_scan_dispatch(uint32_t layout, uint32_t esize, uint32_t P, const CUtensorMap& tm,
                                 const ScanParams& p, int grid, int block, size_t smem, cudaStream_t s) {
  switch (layout) {
    case kByteSmem: return scan_byte(esize, P, tm, p, grid, block, smem, s);
    case kClassWin: return scan_win(esize, P, tm, p, grid, block, smem, s);
    case kClassPair: return scan_pair(esize, P, tm, p, grid, block, smem, s);
    case kByteStride:
      // at most 32 compact states, so at most 32 candidates (P == 1); anything else would be
      // a planning error
      return P == 1 ? scan_byte_stride(tm, p, grid, block, smem, s) : cudaErrorInvalidValue;
    case kClassSmem: return scan_class(esize, P, tm, p, grid, block, smem, s);
    case kClassSmemW: return scan_class_wide(P, tm, p, grid, block, smem, s);
    case kClassGlobal: return scan_global(0, P, tm, p, grid, block, smem, s);
    default: return scan_global(1, P, tm, p, grid, block, smem, s);
  }
}

cudaError_t launch_emit_dispatch(uint32_t layout, uint32_t esize, const ScanParams& p, const CUtensorMap* tm,
                                 int grid, int block, size_t smem, cudaStream_t s) {
  switch (layout) {
    case kByteSmem: return emit_byte(esize, p, tm, grid, block, smem, s);
    case kByteStride: return emit_byte_stride(p, tm, grid, block, smem, s);
    case kClassWin:
    case kClassPair: return emit_win(esize, p, tm, grid, block, smem, s);
    case kClassSmem: return emit_class(esize, p, tm, grid, block, smem, s);
    case kClassSmemW: return emit_class_wide(p, tm, grid, block, smem, s);
    case kClassGlobal: return emit_global(0, p, tm, grid, block, smem, s);
    default: return emit_global(1, p, tm, grid, block, smem, s);
  }
}

cudaError_t launch_tiny_dispatch(uint32_t layout, uint32_t esize, const ScanParams& p, size_t smem,
                                 cudaStream_t s) {
  switch (layout) {
    case kByteSmem: return tiny_byte(esize, p, smem, s);
    case kByteStride: return tiny_byte_stride(p, smem, s);
    case kClassWin:
    case kClassPair: return tiny_win(esize, p, smem, s);
    case kClassSmem: return tiny_class(esize, p, smem, s);
    case kClassSmemW: return tiny_class_wide(p, smem, s);
    case kClassGlobal: return tiny_global(0, p, smem, s);
    default: return tiny_global(1, p, smem, s);
  }
}

}  // namespace parem
