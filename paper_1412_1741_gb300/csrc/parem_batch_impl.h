// parem_batch_impl.h -- the batch builder as used by the request server: batches planned
// into caller-owned buffers (no allocation per batch) and read back item by item.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/parem.h"
#include "parem_internal.h"

namespace parem {

// Buffers lent to one batch at a time.  The host descriptor image is pinned so that its copy
// to `desc` can be asynchronous on `stream`; the caller must not reuse the arena before the
// batch's work on that stream has completed.
struct BatchArena {
  uint8_t* scratch = nullptr;  // device
  uint64_t scratch_cap = 0;
  uint8_t* desc = nullptr;  // device
  uint8_t* host_desc = nullptr;  // pinned host, desc_cap bytes
  uint64_t desc_cap = 0;
  DevResult* host_res = nullptr;  // pinned host, res_cap entries
  uint32_t res_cap = 0;
  EarlyResult* host_early = nullptr;  // pinned, mapped: res_cap early results (optional)
  EarlyResult* dev_early = nullptr;   // its device address
  cudaStream_t stream = nullptr;
};

// Plan items (positions kept, no graph, the whole GPU) into the arena; seg_for[i] != 0 fixes
// item i's row length.  PAREM_ERR_TOO_LARGE when the batch does not fit the arena.
int batch_create_in(const parem_batch_item* items, uint32_t n, const std::vector<uint64_t>& seg_for,
                    const BatchArena* arena, parem_batch** out);
// Clear the scratch, launch the kernels and copy the results to the arena's host results.
int batch_enqueue(parem_batch* b, cudaStream_t st);
void batch_release(parem_batch* b);
// After the batch's stream has completed: the result of the item at sorted position k, its
// status (OK, CAPACITY, TIMEOUT or INTERNAL), and what it taught about the DFA's convergence.
int batch_sorted_result(const parem_batch* b, uint32_t k, parem_result* res);
int batch_item_result(const parem_batch* b, uint32_t i, parem_result* res);
// While the batch runs: the result of the item at sorted position k if its kernel has
// published it early (items without positions, arenas with early results); false otherwise.
bool batch_early_result(const parem_batch* b, uint32_t k, parem_result* res);
uint32_t batch_size(const parem_batch* b);
uint32_t batch_kernels(const parem_batch* b);  // kernel launches of one batch_enqueue
uint32_t batch_order(const parem_batch* b, uint32_t k);  // sorted position -> given index
// The batch kernels' copy of a DFA (built once).
int batch_prepare_dfa(parem_dfa* d);
// Row length the batch planner uses for this DFA when nothing else is known.
uint64_t batch_default_segment(const parem_dfa* d);

}  // namespace parem
