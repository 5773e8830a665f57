// parem_launch.h -- launch plan and the kernel dispatch entry points (one translation unit
// per table layout instantiates the kernels).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>

#include "parem_internal.h"

#include "../../include/parem.h"

// A loaded DFA: the host preparation and its device copy (opaque in the C ABI).
struct parem_dfa {
  int device = 0;
  parem::Prepared host;
  parem::DeviceDfa dev{};
  void* dmem = nullptr;
  parem_dfa_info info{};
  // the batch kernels' copy (u16 class table, u16 column map), built on first batch use
  parem::DeviceDfa batch{};
  void* batch_mem = nullptr;
  // longest speculative prefix (bytes) the candidates of this DFA needed so far, learned from
  // earlier scans; plans make rows several times longer than this
  std::atomic<uint32_t> conv_hint{0};
  // matches per MiB of text in the last scan of at least 1 MiB (kEmpty: none yet); scans
  // of DFAs that matched rarely count matches only in the 16-byte vectors that have one
  std::atomic<uint32_t> density_hint{0xFFFFFFFFu};
  // The two-byte stride variant (kClassPair) of a kClassWin DFA, learned once from a sample
  // of a large text: a copy of the prepared DFA renumbered with the most visited states
  // first, its pair table appended, and its device copy.  pair_state: kPairNone (not tried),
  // kPairBusy (being built by one call), kPairReady (pair_host / pair_dev usable, never
  // changed again), kPairOff (not worth it for the texts seen).
  std::atomic<uint32_t> pair_state{0};
  parem::Prepared pair_host;
  parem::DeviceDfa pair_dev{};
  void* pair_mem = nullptr;
};

namespace parem {

// A named range on the host timeline of profilers that read NVTX (one per API call); without
// a profiler attached the calls do nothing.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
// Shortest row length worth speculating for this DFA: a multiple of its learned convergence
// length, or for DFAs whose candidate sets are large relative to their states (random-like
// automata, which need about twice their state count to synchronise) a multiple of n.
uint64_t min_row_bytes(const parem_dfa* dfa, uint32_t P);
// Longest row worth planning for m candidates: bounds the slot-map cost of a row whose
// candidates never merge.
uint64_t max_row_bytes(const parem_dfa* dfa, uint32_t m);
// Rows whose candidates have not merged are run from their resolved start instead of through
// slot maps: for more candidates than one pass of the lanes, when the DFA synchronises.
bool serial_rows(const parem_dfa* dfa, uint32_t m);
// Record what a scan with the given speculation cap observed about convergence.
void learn_convergence(const parem_dfa* dfa, uint32_t spec_cap, uint32_t nonconv_rows, uint32_t conv_max);

constexpr uint32_t kPairNone = 0, kPairBusy = 1, kPairReady = 2, kPairOff = 3;
// Texts at least this long teach a kClassWin DFA its hot states (parem_pair.cpp).
constexpr uint64_t kPairLearnBytes = 64ull << 20;
// The kClassPair variant of a kClassWin DFA planned from a host text sample (nwin windows of
// wlen bytes): hot states, the renumbered copy with its pair table, and the estimated share
// of 32-lane vector steps that would need the byte loop (parem_pair.cpp).
struct PairPlan {
  bool ok = false;               // worth using (the share is small enough)
  uint32_t hot = 0;              // hot states H (0: no variant)
  double warp_slow = 1.0;
  std::vector<uint32_t> hot_orig;  // original id of hot state e
  Prepared Q;
};
int plan_pairs(const Prepared& P, const uint8_t* sample, uint64_t nwin, uint64_t wlen, PairPlan* out);
// Sample the device text, plan the variant and upload it when it pays; sets pair_state to
// kPairReady or kPairOff.  Host call, blocking.
int learn_pairs(parem_dfa* dfa, const uint8_t* text, uint64_t len, cudaStream_t stream);
// The device copy of a prepared DFA: one allocation (table, column map, byte classes,
// candidate lists, ranks) and the DeviceDfa that points into it (parem_api.cu).
int upload_prepared(const Prepared& P, DeviceDfa* D, void** dmem);
}  // namespace parem

namespace parem {

struct Plan {
  const Prepared* prep;  // the prepared DFA the scan runs (the pair variant when it is used)
  const DeviceDfa* ddfa; // and its device copy
  uint32_t layout;       // its table layout
  uint32_t P;            // candidate registers per lane in the warp-wide phase (1, 2, 4, 8)
  uint32_t enum_all;
  uint32_t cand_stride;
  uint32_t group;        // lanes per row in the grouped speculation (P == 1)
  uint32_t bitmap_words; // per-warp candidate bitmap words (P > 1 and candidate sets > 32 * P)
  uint32_t spec_bytes;   // per-warp speculation scratch
  int warps, grid;
  uint32_t table_smem;   // table bytes staged in shared memory (0 for the global layouts)
  size_t smem;
  uint64_t h, S, R, tail, n_chunks;
  uint32_t spec_cap;
  uint32_t serial;       // unmerged rows run from their resolved start (no slot maps)
  uint32_t sparse;       // count matches per 16-byte vector only where one occurs
  uint32_t dense;        // matches were dense in the DFA's last large scan: the emit pass
                         // streams the rows through shared memory (k_emit_stream)
};

// The launch plan of one scan (parem_api.cu).
int plan_scan(const parem_dfa* dfa, const uint8_t* text, uint64_t len, const parem_match_opts* o, Plan* pl);

cudaError_t launch_scan_dispatch(uint32_t layout, uint32_t esize, uint32_t P, const CUtensorMap& tm,
                                 const ScanParams& p, int grid, int block, size_t smem, cudaStream_t s);
cudaError_t launch_emit_dispatch(uint32_t layout, uint32_t esize, const ScanParams& p, const CUtensorMap* tm,
                                 int grid, int block, size_t smem, cudaStream_t s);
cudaError_t launch_tiny_dispatch(uint32_t layout, uint32_t esize, const ScanParams& p, size_t smem,
                                 cudaStream_t s);

// per-layout entry points (parem_k_byte.cu, parem_k_class.cu, parem_k_global.cu)
cudaError_t scan_byte(uint32_t esize, uint32_t P, const CUtensorMap& tm, const ScanParams& p, int grid,
                      int block, size_t smem, cudaStream_t s);
cudaError_t scan_class(uint32_t esize, uint32_t P, const CUtensorMap& tm, const ScanParams& p, int grid,
                       int block, size_t smem, cudaStream_t s);
cudaError_t scan_class_wide(uint32_t P, const CUtensorMap& tm, const ScanParams& p, int grid, int block,
                            size_t smem, cudaStream_t s);
cudaError_t scan_global(uint32_t wide, uint32_t P, const CUtensorMap& tm, const ScanParams& p, int grid,
                        int block, size_t smem, cudaStream_t s);
cudaError_t emit_byte(uint32_t esize, const ScanParams& p, const CUtensorMap* tm,
                      int grid, int block, size_t smem, cudaStream_t s);
cudaError_t emit_class(uint32_t esize, const ScanParams& p, const CUtensorMap* tm,
                       int grid, int block, size_t smem, cudaStream_t s);
cudaError_t emit_class_wide(const ScanParams& p, const CUtensorMap* tm,
                            int grid, int block, size_t smem, cudaStream_t s);
cudaError_t emit_global(uint32_t wide, const ScanParams& p, const CUtensorMap* tm,
                        int grid, int block, size_t smem, cudaStream_t s);
cudaError_t tiny_byte(uint32_t esize, const ScanParams& p, size_t smem, cudaStream_t s);
cudaError_t scan_byte_stride(const CUtensorMap& tm, const ScanParams& p, int grid, int block, size_t smem,
                             cudaStream_t s);
cudaError_t emit_byte_stride(const ScanParams& p, const CUtensorMap* tm,
                             int grid, int block, size_t smem, cudaStream_t s);
cudaError_t tiny_byte_stride(const ScanParams& p, size_t smem, cudaStream_t s);
cudaError_t scan_win(uint32_t esize, uint32_t P, const CUtensorMap& tm, const ScanParams& p, int grid, int block,
                     size_t smem, cudaStream_t s);
cudaError_t emit_win(uint32_t esize, const ScanParams& p, const CUtensorMap* tm,
                     int grid, int block, size_t smem, cudaStream_t s);
cudaError_t tiny_win(uint32_t esize, const ScanParams& p, size_t smem, cudaStream_t s);
cudaError_t scan_pair(uint32_t esize, uint32_t P, const CUtensorMap& tm, const ScanParams& p, int grid, int block,
                      size_t smem, cudaStream_t s);
cudaError_t tiny_class(uint32_t esize, const ScanParams& p, size_t smem, cudaStream_t s);
cudaError_t tiny_class_wide(const ScanParams& p, size_t smem, cudaStream_t s);
cudaError_t tiny_global(uint32_t wide, const ScanParams& p, size_t smem, cudaStream_t s);

cudaError_t launch_batch_scan(const BatchParams& bp, int grid, int block, size_t smem, cudaStream_t s);
cudaError_t launch_batch_emit(const BatchParams& bp, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_batch_tiny(const BatchParams& bp, const uint32_t* tiny_items, uint32_t n_tiny, cudaStream_t s);

}  // namespace parem
