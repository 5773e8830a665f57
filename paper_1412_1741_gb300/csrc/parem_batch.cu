// parem_batch.cu -- batched matching: many (text, DFA) items in one persistent launch, the
// whole run captured in a CUDA graph; an autotuner for each DFA's segment size and
// speculation form and for the batch's block shape.
//
// Planning (parem_batch_create):
//   * every DFA of the batch gets its batch-kernel copy (u16 class table, u16 column map);
//   * items are grouped by DFA ("slots"); each item gets rows of S bytes (per-DFA S from the
//     autotuner, or the planner's default: about two rows per lane of the whole GPU); each
//     slot gets a speculation form (grouped, warp-wide in registers, warp-wide through a
//     state bitmap);
//   * texts shorter than one 64-byte row go to a one-thread-per-item kernel;
//   * one scratch allocation holds every item's status words, row records, recorded positions,
//     slot maps and result word; one descriptor allocation holds the per-item scan parameters
//     and TMA tensor maps, the slots, and the initial CTA -> slot assignment (first enough CTAs
//     for the slots of long serial chunks to start all of them at once, then the rest in
//     proportion to each slot's bytes, weighted up when its table is read from L2);
//   * clearing the scratch, the kernels and the copy of the results to pinned host memory are
//     captured in one CUDA graph, which parem_batch_run replays.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/parem.h"
#include "parem_batch_impl.h"
#include "parem_internal.h"
#include "parem_launch.h"

using namespace parem;

struct parem_batch {
  int device = 0;
  std::vector<parem_batch_item> items;  // as given
  std::vector<uint32_t> order;          // sorted position -> given index
  std::vector<uint64_t> seg;            // per given item: S (0 for texts shorter than a row)
  std::vector<uint32_t> cap;            // per given item: speculation cap (bytes)
  std::vector<uint32_t> spec;           // per given item: speculation form (PAREM_BATCH_SPEC_*)
  std::vector<uint8_t> smem_table;      // per given item: its DFA's table is in shared memory
  void* desc = nullptr;
  void* scratch = nullptr;
  DevResult* host_res = nullptr;        // pinned, per sorted item
  DevResult* dev_res = nullptr;
  EarlyResult* host_early = nullptr;    // arena's early results, per sorted item (or nullptr)
  EarlyResult* dev_early = nullptr;
  BatchParams bp{};
  uint64_t zero_bytes = 0;
  int grid = 0, block = 0;
  size_t smem = 0;
  int emit_grid = 0;
  size_t emit_smem = 0;
  uint32_t n_scan_items = 0;
  uint32_t n_tiny = 0;
  const uint32_t* tiny_dev = nullptr;
  bool any_positions = false;
  bool use_graph = true;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint32_t n_items = 0;
  bool borrowed = false;  // scratch, descriptors and results live in a caller's BatchArena
};

namespace {

uint64_t up(uint64_t x, uint64_t m) { return (x + m - 1) / m * m; }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn_batch() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

int encode_item_rows(CUtensorMap* tm, const uint8_t* base, uint64_t S, uint64_t R) {
  auto fn = encode_fn_batch();
  if (!fn) return PAREM_ERR_CUDA;
  cuuint64_t dims[2] = {(cuuint64_t)S, (cuuint64_t)R};
  cuuint64_t strides[1] = {(cuuint64_t)S};
  cuuint32_t box[2] = {kBox, kLanes};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(base), dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? PAREM_OK : PAREM_ERR_CUDA;
}

// The batch kernels' copy of a DFA: class-indexed rows of u16 entries and a u16 column map
// (byte -> class * 2).  The candidate lists, ranks and byte classes are shared with the
// plain copy.
int ensure_batch_dfa(parem_dfa* d) {
  if (d->batch_mem) return PAREM_OK;
  const Prepared& P = d->host;
  const uint32_t n = P.n, nc = P.n_classes;
  uint32_t rb = nc * 2;
  if (rb % 4 == 0 && (rb / 4) % 2 == 0) rb += 4;
  const uint64_t tbytes = up((uint64_t)n * rb, 16);
  if (tbytes > 0xFFFFFFFFull) return PAREM_ERR_UNSUPPORTED;
  std::vector<uint8_t> tab(tbytes, 0);
  std::vector<int> rep(nc, -1);
  for (int b = 0; b < 256; ++b)
    if (rep[P.byte_class[b]] < 0) rep[P.byte_class[b]] = b;
  for (uint32_t s = 0; s < n; ++s)
    for (uint32_t c = 0; c < nc; ++c) {
      const uint8_t* src = &P.table[(uint64_t)s * P.rowbytes + P.colmap[rep[c]]];
      uint16_t v = P.esize == 1 ? (uint16_t)src[0] : (uint16_t)(src[0] | (src[1] << 8));
      std::memcpy(&tab[(uint64_t)s * rb + 2 * c], &v, 2);
    }
  std::vector<uint16_t> cm(256);
  for (int b = 0; b < 256; ++b) cm[b] = (uint16_t)(P.byte_class[b] * 2);
  void* mem = nullptr;
  if (cudaMalloc(&mem, tbytes + 512) != cudaSuccess) return PAREM_ERR_OOM;
  uint8_t* base = static_cast<uint8_t*>(mem);
  if (cudaMemcpy(base, tab.data(), tbytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(base + tbytes, cm.data(), 512, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(mem);
    return PAREM_ERR_CUDA;
  }
  d->batch = d->dev;
  d->batch.table = base;
  d->batch.colmap = base + tbytes;
  d->batch.layout = kBatchDyn;
  d->batch.esize = 2;
  d->batch.rowbytes = rb;
  d->batch.table_bytes = (uint32_t)tbytes;
  d->batch_mem = mem;
  return PAREM_OK;
}

void release(parem_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (!b->borrowed) {
    if (b->desc) cudaFree(b->desc);
    if (b->scratch) cudaFree(b->scratch);
    if (b->host_res) cudaFreeHost(b->host_res);
  }
  delete b;
}

// Launch the batch's kernels on a stream (also used while capturing the graph).
int enqueue(parem_batch* b, cudaStream_t st) {
  if (cudaMemsetAsync(b->scratch, 0, b->zero_bytes, st) != cudaSuccess) return PAREM_ERR_CUDA;
  if (b->n_tiny && launch_batch_tiny(b->bp, b->tiny_dev, b->n_tiny, st) != cudaSuccess) return PAREM_ERR_CUDA;
  if (b->n_scan_items) {
    if (launch_batch_scan(b->bp, b->grid, b->block, b->smem, st) != cudaSuccess) return PAREM_ERR_CUDA;
    if (b->any_positions && b->emit_grid > 0 &&
        launch_batch_emit(b->bp, b->emit_grid, b->emit_smem, st) != cudaSuccess)
      return PAREM_ERR_CUDA;
  }
  if (cudaMemcpyAsync(b->host_res, b->dev_res, sizeof(DevResult) * b->n_items, cudaMemcpyDeviceToHost, st) !=
      cudaSuccess)
    return PAREM_ERR_CUDA;
  return PAREM_OK;
}

// The speculation form a DFA gets in a batch: `want` where it applies, else the default
// (grouped for candidate sets of one warp or less; the state bitmap for sets beyond the
// registers, or for DFAs of many states that synchronise slowly; else registers).
uint32_t resolve_spec(const parem_dfa* d, uint32_t want) {
  const Prepared& P = d->host;
  const bool bitmap_ok = P.n <= 16384;
  if (want == PAREM_BATCH_SPEC_GROUPED && P.max_cand <= kLanes) return want;
  if (want == PAREM_BATCH_SPEC_WARP && P.max_cand <= 8 * kLanes) return want;
  if (want == PAREM_BATCH_SPEC_WARP_BITMAP && bitmap_ok) return want;
  if (P.max_cand <= kLanes) return PAREM_BATCH_SPEC_GROUPED;
  if (bitmap_ok && (P.max_cand > 8 * kLanes || (P.sync_len > 16 && P.n >= 256))) return PAREM_BATCH_SPEC_WARP_BITMAP;
  return PAREM_BATCH_SPEC_WARP;
}

struct Slot {
  parem_dfa* dfa;
  std::vector<uint32_t> items;  // given indices
  uint32_t spec = PAREM_BATCH_SPEC_AUTO;
  uint32_t bitmap_words = 0;
  uint32_t spec_bytes = kSpecBytes;
  bool smem_tier = false;
  double weight = 0;
};

// Plan a batch.  seg_for: per given item, the segment size to use (0 = default); spec_for
// (optional): per given item, the speculation form of its DFA (AUTO = o->spec, else the
// default; an item's DFA takes the form of its first item).  With an arena, nothing is
// allocated: the batch lives in the arena's buffers (PAREM_ERR_TOO_LARGE when it does not
// fit) and its descriptors are copied on the arena's stream.
int create_internal(const parem_batch_item* items, uint32_t n, const parem_batch_opts* o, int grid_limit,
                    const std::vector<uint64_t>& seg_for, bool use_graph, bool keep_positions,
                    parem_batch** out, const BatchArena* arena = nullptr,
                    const std::vector<uint32_t>* spec_for = nullptr) {
  *out = nullptr;
  if (!items || n == 0) return PAREM_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return PAREM_ERR_CUDA;
  for (uint32_t i = 0; i < n; ++i) {
    const parem_batch_item& it = items[i];
    if (!it.dfa || it.dfa->device != dev || (it.len > 0 && !it.text) || it.len > kMaxText) return PAREM_ERR_INVALID_ARG;
  }
  int sms = 0, smem_optin = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  parem_batch* b = new (std::nothrow) parem_batch();
  if (!b) return PAREM_ERR_OOM;
  b->device = dev;
  b->items.assign(items, items + n);
  b->n_items = n;
  b->use_graph = use_graph;

  // slots: distinct DFAs in order of first appearance
  std::map<const parem_dfa*, uint32_t> slot_of;
  std::vector<Slot> slots;
  for (uint32_t i = 0; i < n; ++i) {
    auto it = slot_of.find(items[i].dfa);
    if (it == slot_of.end()) {
      it = slot_of.emplace(items[i].dfa, (uint32_t)slots.size()).first;
      Slot s;
      s.dfa = const_cast<parem_dfa*>(items[i].dfa);
      uint32_t want = o ? o->spec : PAREM_BATCH_SPEC_AUTO;
      if (spec_for && i < spec_for->size() && (*spec_for)[i]) want = (*spec_for)[i];
      s.spec = resolve_spec(s.dfa, want);
      slots.push_back(s);
    }
  }
  for (Slot& s : slots) {
    int rc = ensure_batch_dfa(s.dfa);
    if (rc != PAREM_OK) {
      release(b);
      return rc;
    }
    const Prepared& P = s.dfa->host;
    if (s.spec == PAREM_BATCH_SPEC_WARP_BITMAP) {
      s.bitmap_words = (P.n + 31) / 32;
      s.spec_bytes = kSpecBytes + (uint32_t)up(8ull * s.bitmap_words, 16) + 512u;
    }
  }
  // launch shape and shared-memory carve-up
  // the two block shapes of k_batch_scan
  const int warps = (o && o->warps_per_block && o->warps_per_block <= 16) ? 16 : 24;
  uint32_t spec_bytes = kSpecBytes;
  for (const Slot& s : slots) spec_bytes = std::max(spec_bytes, s.spec_bytes);
  const uint32_t per_warp = kStages * kStageBytes + kStages * 8 + spec_bytes;
  const int64_t budget = (int64_t)smem_optin - kTableOff - 1024 - (int64_t)warps * per_warp;
  uint32_t max_table = 0;
  for (Slot& s : slots) {
    s.smem_tier = (int64_t)s.dfa->batch.table_bytes <= budget;
    if (s.smem_tier) max_table = std::max(max_table, s.dfa->batch.table_bytes);
  }
  b->grid = grid_limit > 0 ? std::min(grid_limit, sms) : sms;
  b->block = warps * 32;
  b->smem = kTableOff + max_table + 1024 + (size_t)warps * per_warp;
  b->emit_smem = kTableOff + max_table;

  // per-item plans
  uint64_t total = 0;
  for (uint32_t i = 0; i < n; ++i) total += items[i].len;
  const uint64_t lanes = (uint64_t)sms * warps * kLanes;
  uint64_t s_default = up(std::max<uint64_t>(total / (2 * lanes + 1), 1), kBox);
  s_default = std::min<uint64_t>(std::max<uint64_t>(s_default, 4096), 1u << 20);
  struct Plan1 {
    uint64_t h, S, R, tail, chunks;
    uint32_t cap;
  };
  std::vector<Plan1> plan(n);
  b->seg.assign(n, 0);
  b->cap.assign(n, 0);
  b->spec.assign(n, 0);
  b->smem_table.assign(n, 0);
  for (uint32_t i = 0; i < n; ++i) {
    const parem_batch_item& it = items[i];
    Plan1& pl = plan[i];
    const uint64_t addr = reinterpret_cast<uint64_t>(it.text);
    pl.h = std::min<uint64_t>(it.len, (16 - (addr & 15)) & 15);
    const uint64_t body = it.len - pl.h;
    uint64_t S = (i < seg_for.size() && seg_for[i]) ? seg_for[i]
                 : (o && o->segment_bytes) ? o->segment_bytes
                                           : std::min(std::max<uint64_t>(s_default, min_row_bytes(it.dfa, 8)),
                                                      max_row_bytes(it.dfa, it.dfa->host.max_cand));
    S = up(S, kBox);
    while (body / S >= (1ull << 31)) S *= 2;
    if (body < S) S = body / kBox * kBox;
    pl.S = S;
    pl.R = S ? body / S : 0;
    pl.tail = S ? body - pl.R * S : body;
    pl.chunks = (pl.R + kLanes - 1) / kLanes;
    const Prepared& P = it.dfa->host;
    uint64_t cap = std::min<uint64_t>(
        std::max<uint64_t>(std::max<uint64_t>(2048, 16ull * P.n), 4ull * it.dfa->conv_hint.load()), S);
    pl.cap = (uint32_t)(cap / 16 * 16);
    if (pl.cap == 0) pl.cap = 16;
    b->seg[i] = pl.R ? S : 0;
    b->cap[i] = pl.cap;
    b->spec[i] = slots[slot_of[it.dfa]].spec;
    b->smem_table[i] = slots[slot_of[it.dfa]].smem_tier ? 1 : 0;
    if (pl.R) slots[slot_of[it.dfa]].items.push_back(i);
  }
  // sorted order: scanned items by slot, then the short ones
  std::vector<uint32_t> tiny;
  for (uint32_t i = 0; i < n; ++i)
    if (!plan[i].R) tiny.push_back(i);
  for (const Slot& s : slots) b->order.insert(b->order.end(), s.items.begin(), s.items.end());
  b->n_scan_items = (uint32_t)b->order.size();
  b->order.insert(b->order.end(), tiny.begin(), tiny.end());
  b->n_tiny = (uint32_t)tiny.size();

  // scratch: [tickets][results][status words] (cleared each run), then per item the row
  // records, recorded positions and slot maps
  const uint64_t o_res = up(4ull * slots.size(), 256);
  const uint64_t o_status = up(o_res + sizeof(DevResult) * (uint64_t)n, 256);
  uint64_t off = o_status;
  std::vector<uint64_t> st_off(n);
  for (uint32_t k = 0; k < n; ++k) {
    const uint32_t i = b->order[k];
    st_off[i] = off;
    off += plan[i].chunks * 8;
  }
  b->zero_bytes = up(off, 16);
  off = up(off, 256);
  std::vector<uint64_t> rec_off(n), pos_off(n), map_off(n);
  for (uint32_t k = 0; k < n; ++k) {
    const uint32_t i = b->order[k];
    const bool emit = keep_positions && items[i].positions && items[i].capacity > 0;
    b->any_positions = b->any_positions || (emit && plan[i].R);
    rec_off[i] = off;
    if (emit && plan[i].R) off = up(off + plan[i].R * sizeof(SegRec), 256);
    pos_off[i] = off;
    if (emit && plan[i].R) off = up(off + plan[i].R * kRowSlotBytes, 256);
    map_off[i] = off;
    const uint32_t stride = std::max<uint32_t>(1, items[i].dfa->host.max_cand);
    if (!serial_rows(items[i].dfa, items[i].dfa->host.max_cand)) off = up(off + 2 * plan[i].R * stride * 4, 256);
  }
  if (arena) {
    b->borrowed = true;
    if (off > arena->scratch_cap || n > arena->res_cap) {
      release(b);
      return PAREM_ERR_TOO_LARGE;
    }
    b->scratch = arena->scratch;
    b->host_res = arena->host_res;
    if (arena->host_early && arena->dev_early) {
      // the arena is idle: no kernel writes these slots while they are cleared
      b->host_early = arena->host_early;
      b->dev_early = arena->dev_early;
      for (uint32_t k = 0; k < n; ++k) reinterpret_cast<volatile uint32_t*>(&b->host_early[k].ready)[0] = 0u;
    }
  } else {
    if (cudaMalloc(&b->scratch, std::max<uint64_t>(off, 256)) != cudaSuccess) {
      release(b);
      return PAREM_ERR_OOM;
    }
    if (cudaMallocHost(&b->host_res, sizeof(DevResult) * n) != cudaSuccess) {
      release(b);
      return PAREM_ERR_OOM;
    }
  }
  uint8_t* sb = static_cast<uint8_t*>(b->scratch);
  b->dev_res = reinterpret_cast<DevResult*>(sb + o_res);

  // descriptors
  const uint32_t ns = (uint32_t)slots.size();
  std::vector<uint32_t> cta_slot(b->grid, 0);
  std::vector<uint32_t> emit_slot;
  std::vector<uint64_t> emit_row0;
  const uint64_t d_items = 0;
  const uint64_t d_slots = up(d_items + sizeof(BatchItem) * (uint64_t)n, 256);
  const uint64_t d_cta = up(d_slots + sizeof(BatchSlot) * (uint64_t)ns, 256);
  const uint64_t d_tiny = up(d_cta + 4ull * b->grid, 256);
  // emit blocks: 256 rows of one slot per block
  std::vector<uint64_t> slot_rows(ns, 0), slot_chunks(ns, 0);
  for (uint32_t si = 0; si < ns; ++si)
    for (uint32_t i : slots[si].items) {
      slot_rows[si] += plan[i].R;
      slot_chunks[si] += plan[i].chunks;
    }
  if (b->any_positions)
    for (uint32_t si = 0; si < ns; ++si)
      for (uint64_t r0 = 0; r0 < slot_rows[si]; r0 += 256) {
        emit_slot.push_back(si);
        emit_row0.push_back(r0);
      }
  b->emit_grid = (int)emit_slot.size();
  const uint64_t d_eslot = up(d_tiny + 4ull * std::max<size_t>(tiny.size(), 1), 256);
  const uint64_t d_erow = up(d_eslot + 4ull * std::max<size_t>(emit_slot.size(), 1), 256);
  const uint64_t d_total = up(d_erow + 8ull * std::max<size_t>(emit_row0.size(), 1), 256);
  std::vector<uint8_t> host_vec;
  uint8_t* host = nullptr;  // descriptor image (pinned in an arena)
  if (arena) {
    if (d_total > arena->desc_cap) {
      release(b);
      return PAREM_ERR_TOO_LARGE;
    }
    b->desc = arena->desc;
    host = arena->host_desc;
    std::memset(host, 0, d_total);
  } else {
    if (cudaMalloc(&b->desc, d_total) != cudaSuccess) {
      release(b);
      return PAREM_ERR_OOM;
    }
    host_vec.assign(d_total, 0);
    host = host_vec.data();
  }
  uint8_t* db = static_cast<uint8_t*>(b->desc);
  std::vector<BatchItem> hitems(n);  // typed (aligned) staging, copied into `host` below
  std::vector<BatchSlot> hslots(ns);
  std::memset(static_cast<void*>(hitems.data()), 0, sizeof(BatchItem) * n);
  std::memset(static_cast<void*>(hslots.data()), 0, sizeof(BatchSlot) * ns);
  // slot item ranges in the sorted order
  uint32_t pos_k = 0;
  for (uint32_t si = 0; si < ns; ++si) {
    BatchSlot& bs = hslots[si];
    bs.dfa = slots[si].dfa->batch;
    bs.smem_tier = slots[si].smem_tier ? 1u : 0u;
    bs.grouped = slots[si].spec == PAREM_BATCH_SPEC_GROUPED ? 1u : 0u;
    bs.item_begin = pos_k;
    bs.item_end = pos_k + (uint32_t)slots[si].items.size();
    bs.n_chunks = slot_chunks[si];
    bs.n_rows = slot_rows[si];
    bs.ticket = reinterpret_cast<uint32_t*>(sb + 4ull * si);
    uint64_t cb = 0, rb = 0;
    for (uint32_t i : slots[si].items) {
      BatchItem& bi = hitems[pos_k++];
      bi.chunk_base = cb;
      bi.row_base = rb;
      cb += plan[i].chunks;
      rb += plan[i].R;
    }
  }
  for (uint32_t k = 0; k < n; ++k) {
    const uint32_t i = b->order[k];
    const parem_batch_item& it = items[i];
    const Plan1& pl = plan[i];
    const Prepared& P = it.dfa->host;
    BatchItem& bi = hitems[k];
    ScanParams& p = bi.p;
    std::memset(&p, 0, sizeof(p));
    p.dfa = it.dfa->batch;
    p.text = it.text;
    p.n = it.len;
    p.h = pl.h;
    p.S = pl.S;
    p.R = pl.R;
    p.tail = pl.tail;
    p.n_chunks = pl.chunks;
    p.init_state = P.start;
    // lanes per row of the grouped speculation: the smallest power of two holding the
    // largest candidate set (used when the slot is grouped)
    p.group = 1;
    while (p.group < P.max_cand && p.group < kLanes) p.group *= 2;
    p.bitmap_words = slots[slot_of[it.dfa]].bitmap_words;
    p.spec_bytes = spec_bytes;
    p.smem_table_bytes = 0;
    p.enum_all = 0;
    p.spec_cap = pl.cap;
    p.cand_stride = std::max<uint32_t>(1, P.max_cand);
    p.serial_fallback = serial_rows(it.dfa, P.max_cand) ? 1u : 0u;
    p.wait_budget = 4000000000ull;
    p.skip_publish = -1;
    p.status = reinterpret_cast<unsigned long long*>(sb + st_off[i]);
    const bool emit = keep_positions && it.positions && it.capacity > 0;
    p.segrec = (emit && pl.R) ? reinterpret_cast<SegRec*>(sb + rec_off[i]) : nullptr;
    p.slots = (emit && pl.R) ? reinterpret_cast<uint32_t*>(sb + pos_off[i]) : nullptr;
    p.slot_end = reinterpret_cast<uint32_t*>(sb + map_off[i]);
    p.slot_cnt = reinterpret_cast<uint32_t*>(sb + map_off[i] + pl.R * (uint64_t)p.cand_stride * 4);
    p.result = b->dev_res + k;
    p.early = (!emit && b->dev_early) ? b->dev_early + k : nullptr;
    p.positions = emit ? it.positions : nullptr;
    p.capacity = emit ? it.capacity : 0;
    if (pl.R) {
      int rc = encode_item_rows(&bi.tmap, it.text + pl.h, pl.S, pl.R);
      if (rc != PAREM_OK) {
        release(b);
        return rc;
      }
    }
  }
  // initial CTA -> slot assignment in proportion to the slots' work (largest remainders)
  double wsum = 0;
  for (uint32_t si = 0; si < ns; ++si) {
    uint64_t bytes = 0;
    for (uint32_t i : slots[si].items) bytes += items[i].len;
    slots[si].weight = (double)bytes * (slots[si].smem_tier ? 1.0 : 4.0);
    wsum += slots[si].weight;
  }
  {
    // Slots whose chunks are long serial chains (candidate sets beyond the registers, merged
    // through the state bitmap) first get enough blocks to start all their chunks at once:
    // otherwise their last chunks start when the first ones end, and the batch waits on two
    // chunk lengths.  The rest of the grid goes by weight.
    std::vector<int> quota(ns, 0);
    int floor_sum = 0;
    for (uint32_t si = 0; si < ns; ++si) {
      if (slots[si].spec == PAREM_BATCH_SPEC_WARP_BITMAP && slots[si].dfa->host.max_cand > 8 * kLanes) {
        quota[si] = (int)((slot_chunks[si] + warps - 1) / warps);
        floor_sum += quota[si];
      }
    }
    if (floor_sum > b->grid) {
      const int want = floor_sum;
      floor_sum = 0;
      for (uint32_t si = 0; si < ns; ++si) {
        quota[si] = (int)((int64_t)quota[si] * b->grid / want);
        floor_sum += quota[si];
      }
    }
    const int rest = b->grid - floor_sum;
    std::vector<std::pair<double, uint32_t>> rem;
    int given = floor_sum;
    for (uint32_t si = 0; si < ns; ++si) {
      if (slots[si].weight <= 0) continue;
      const double q = wsum > 0 ? slots[si].weight / wsum * rest : 0;
      quota[si] += (int)std::floor(q);
      given += (int)std::floor(q);
      rem.push_back({q - std::floor(q), si});
    }
    std::sort(rem.begin(), rem.end(), [](auto& a, auto& c) { return a.first > c.first; });
    for (size_t r = 0; given < b->grid && r < rem.size(); ++r, ++given) quota[rem[r].second]++;
    int c = 0;
    for (uint32_t si = 0; si < ns && c < b->grid; ++si)
      for (int q = 0; q < quota[si] && c < b->grid; ++q) cta_slot[c++] = si;
    for (; c < b->grid; ++c) cta_slot[c] = rem.empty() ? 0 : rem[0].second;
  }
  std::memcpy(host + d_items, hitems.data(), sizeof(BatchItem) * n);
  std::memcpy(host + d_slots, hslots.data(), sizeof(BatchSlot) * ns);
  std::memcpy(host + d_cta, cta_slot.data(), 4ull * b->grid);
  for (size_t t = 0; t < tiny.size(); ++t) {
    const uint32_t k = b->n_scan_items + (uint32_t)t;
    std::memcpy(host + d_tiny + 4 * t, &k, 4);
  }
  if (!emit_slot.empty()) {
    std::memcpy(host + d_eslot, emit_slot.data(), 4 * emit_slot.size());
    std::memcpy(host + d_erow, emit_row0.data(), 8 * emit_row0.size());
  }
  const cudaError_t ce = arena ? cudaMemcpyAsync(db, host, d_total, cudaMemcpyHostToDevice, arena->stream)
                               : cudaMemcpy(db, host, d_total, cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) {
    release(b);
    return PAREM_ERR_CUDA;
  }
  BatchParams& bp = b->bp;
  bp.items = reinterpret_cast<const BatchItem*>(db + d_items);
  bp.slots = reinterpret_cast<const BatchSlot*>(db + d_slots);
  bp.cta_slot = reinterpret_cast<const uint32_t*>(db + d_cta);
  bp.emit_slot = reinterpret_cast<const uint32_t*>(db + d_eslot);
  bp.emit_row0 = reinterpret_cast<const uint64_t*>(db + d_erow);
  bp.n_slots = ns;
  bp.max_table_smem = max_table;
  bp.spec_bytes = spec_bytes;
  bp.wait_budget = 4000000000ull;
  b->tiny_dev = reinterpret_cast<const uint32_t*>(db + d_tiny);

  if (use_graph) {
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
      release(b);
      return PAREM_ERR_CUDA;
    }
    int rc = PAREM_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) rc = PAREM_ERR_CUDA;
    if (rc == PAREM_OK) rc = enqueue(b, cs);
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(cs, &g) != cudaSuccess && rc == PAREM_OK) rc = PAREM_ERR_CUDA;
    b->graph = g;
    if (rc == PAREM_OK && cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) rc = PAREM_ERR_CUDA;
    cudaStreamDestroy(cs);
    if (rc != PAREM_OK) {
      release(b);
      return rc;
    }
  }
  *out = b;
  return PAREM_OK;
}

int run_internal(parem_batch* b, cudaStream_t st) {
  int rc = PAREM_OK;
  if (b->use_graph) {
    if (cudaGraphLaunch(b->exec, st) != cudaSuccess) return PAREM_ERR_CUDA;
  } else {
    rc = enqueue(b, st);
    if (rc != PAREM_OK) return rc;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return PAREM_ERR_CUDA;
  bool capacity = false;
  for (uint32_t k = 0; k < b->n_items; ++k) {
    const DevResult& r = b->host_res[k];
    if (r.error == kErrTimeout) return PAREM_ERR_TIMEOUT;
    if (r.error) return PAREM_ERR_INTERNAL;
    const uint32_t i = b->order[k];
    const parem_batch_item& it = b->items[i];
    if (it.positions && it.capacity > 0 && r.count > it.capacity) capacity = true;
    if (k < b->n_scan_items) learn_convergence(it.dfa, b->cap[i], r.nonconv_rows, r.conv_max);
  }
  return capacity ? PAREM_ERR_CAPACITY : PAREM_OK;
}

// Time a trial batch without positions (the best of `reps` runs after one warm-up run):
// items with segment size S and speculation form `spec`, or (S == 0) with seg_for and
// spec_for per item, as planned for the whole GPU.
float time_trial(const std::vector<parem_batch_item>& its, uint64_t S, int warps, int grid, uint32_t spec,
                 const std::vector<uint64_t>& seg_for = {}, const std::vector<uint32_t>* spec_for = nullptr,
                 int reps = 2) {
  parem_batch_opts o{};
  o.warps_per_block = (uint32_t)warps;
  o.segment_bytes = S;
  o.spec = spec;
  parem_batch* t = nullptr;
  if (create_internal(its.data(), (uint32_t)its.size(), &o, grid, seg_for, false, false, &t, nullptr, spec_for) !=
      PAREM_OK)
    return 1e30f;
  cudaStream_t st;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  run_internal(t, st);  // warm-up
  for (int rep = 0; rep < reps; ++rep) {
    cudaEventRecord(e0, st);
    if (run_internal(t, st) != PAREM_OK) {
      best = 1e30f;
      break;
    }
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  release(t);
  return best;
}

}  // namespace

extern "C" int parem_batch_create(const parem_batch_item* items, uint32_t n_items, const parem_batch_opts* opts,
                                  parem_batch** out) {
  if (!out) return PAREM_ERR_INVALID_ARG;
  *out = nullptr;
  const bool graph = opts ? opts->use_graph != 0 : true;
  std::vector<uint64_t> seg_for;
  std::vector<uint32_t> spec_for;
  parem_batch_opts o = opts ? *opts : parem_batch_opts{};
  if (!opts) o.use_graph = 1;
  if (o.autotune && !o.segment_bytes && items && n_items) {
    // Per DFA: time candidate segment sizes and speculation forms on all of that DFA's items
    // alone on the whole GPU (no positions).  That time is the larger of the DFA's work over
    // the GPU and its critical path (the longest chain of dependent lookups of one chunk:
    // speculation of its 32 rows, then the longest row), and in a batch that mixes DFAs the
    // slowest DFA's critical path is what the others cannot hide.  A change must gain 3 %.
    // Then the whole batch: the tuned and the default plans, with 24 and with 16 warps.
    parem_batch* probe = nullptr;
    int rc = create_internal(items, n_items, &o, 0, seg_for, false, false, &probe);
    if (rc != PAREM_OK) return rc;
    const int warps = probe->block / 32;
    std::map<const parem_dfa*, std::vector<parem_batch_item>> by_dfa;
    std::map<const parem_dfa*, uint64_t> base_s;
    std::map<const parem_dfa*, uint32_t> base_spec;
    std::vector<uint64_t> seg_default(n_items, 0);
    std::vector<uint32_t> spec_default(n_items, 0);
    for (uint32_t i = 0; i < n_items; ++i) {
      seg_default[i] = probe->seg[i];
      spec_default[i] = probe->spec[i];
      if (probe->seg[i] == 0) continue;
      parem_batch_item it = items[i];
      it.positions = nullptr;
      it.capacity = 0;
      by_dfa[items[i].dfa].push_back(it);
      base_s[items[i].dfa] = std::max(base_s[items[i].dfa], probe->seg[i]);
      base_spec[items[i].dfa] = probe->spec[i];
    }
    release(probe);
    constexpr float kGain = 0.97f;
    std::map<const parem_dfa*, std::pair<uint64_t, uint32_t>> best_of;
    for (auto& kv : by_dfa) {
      const parem_dfa* d = kv.first;
      uint64_t bytes = 0;
      for (auto& it : kv.second) bytes += it.len;
      const uint64_t s0 = base_s[d];
      const uint32_t f0 = base_spec[d];
      if (bytes < (4u << 20)) {
        best_of[d] = {s0, f0};
        continue;
      }
      // a first trial at the default size and form teaches the DFA's convergence length
      float best = time_trial(kv.second, s0, warps, 0, f0);
      uint64_t pick_s = s0;
      uint32_t pick_f = f0;
      // sizes from a quarter to four times the default, no shorter than the longest merge
      // seen so far (plus a quarter) nor than 1 KiB: shorter rows than the planner's default
      // (several merge lengths) cost more speculation per byte but shorten each chunk
      const uint64_t conv = d->conv_hint.load();
      const uint64_t smin = std::max<uint64_t>(1024, up(conv + conv / 4, kBox));
      const uint64_t smax = std::max(smin, std::min<uint64_t>(max_row_bytes(d, d->host.max_cand), 4u << 20));
      auto clamp_s = [&](double v) {
        return std::min<uint64_t>(std::max<uint64_t>(up((uint64_t)std::llround(v), kBox), smin), smax);
      };
      std::vector<std::pair<uint64_t, uint32_t>> tried{{s0, f0}};
      auto trial = [&](uint64_t S, uint32_t f) {
        if (std::find(tried.begin(), tried.end(), std::make_pair(S, f)) != tried.end()) return;
        tried.push_back({S, f});
        const float ms = time_trial(kv.second, S, warps, 0, f);
        if (ms < best * kGain) {
          best = ms;
          pick_s = S;
          pick_f = f;
        }
      };
      for (double g : {0.25, 0.5, 2.0, 4.0}) trial(clamp_s((double)s0 * g), f0);
      // the other forms that apply to this DFA, around the best size so far (unless the caller
      // fixed the form)
      const uint64_t s1 = pick_s;
      for (uint32_t f : {PAREM_BATCH_SPEC_GROUPED, PAREM_BATCH_SPEC_WARP, PAREM_BATCH_SPEC_WARP_BITMAP}) {
        if (o.spec != PAREM_BATCH_SPEC_AUTO || f == f0 || resolve_spec(d, f) != f) continue;
        for (double g : {1.0, 0.5, 2.0}) trial(clamp_s((double)s1 * g), f);
      }
      best_of[d] = {pick_s, pick_f};
    }
    std::vector<uint64_t> seg_tuned(n_items, 0);
    std::vector<uint32_t> spec_tuned(n_items, 0);
    for (uint32_t i = 0; i < n_items; ++i) {
      auto it = best_of.find(items[i].dfa);
      if (it != best_of.end()) {
        seg_tuned[i] = it->second.first;
        spec_tuned[i] = it->second.second;
      }
    }
    // the whole batch: tuned against default plans, and the block shape (unless given)
    std::vector<parem_batch_item> all(items, items + n_items);
    for (auto& it : all) {
      it.positions = nullptr;
      it.capacity = 0;
    }
    float best = 1e30f;
    bool tuned = true;
    int pick_w = warps;
    for (int w : {24, 16}) {
      if (o.warps_per_block && w != warps) continue;
      const float tt = time_trial(all, 0, w, 0, PAREM_BATCH_SPEC_AUTO, seg_tuned, &spec_tuned, 3);
      const float td = time_trial(all, 0, w, 0, PAREM_BATCH_SPEC_AUTO, seg_default, &spec_default, 3);
      // the first shape tried is the default; another must gain 3 %
      const float scale = best < 1e29f ? kGain : 1.0f;
      if (std::min(tt, td) < best * scale) {
        best = std::min(tt, td);
        tuned = tt <= td;
        pick_w = w;
      }
    }
    seg_for = tuned ? seg_tuned : seg_default;
    spec_for = tuned ? spec_tuned : spec_default;
    o.warps_per_block = (uint32_t)pick_w;
  }
  return create_internal(items, n_items, &o, 0, seg_for, graph, true, out, nullptr, &spec_for);
}

extern "C" int parem_batch_run(parem_batch* batch, void* stream) {
  if (!batch) return PAREM_ERR_INVALID_ARG;
  NvtxRange range("parem_batch_run");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return PAREM_ERR_CUDA;
  if (dev != batch->device) return PAREM_ERR_INVALID_ARG;
  return run_internal(batch, static_cast<cudaStream_t>(stream));
}

extern "C" int parem_batch_results(const parem_batch* batch, parem_result* out) {
  if (!batch || !out) return PAREM_ERR_INVALID_ARG;
  for (uint32_t k = 0; k < batch->n_items; ++k) {
    const uint32_t i = batch->order[k];
    const parem_batch_item& it = batch->items[i];
    const Prepared& P = it.dfa->host;
    const DevResult& r = batch->host_res[k];
    parem_result& res = out[i];
    std::memset(&res, 0, sizeof(res));
    if (it.len == 0) {
      res.final_state = P.orig_of[P.start];
      res.accepted = P.start >= P.first_accept;
      continue;
    }
    res.final_state = r.final_state < P.n ? P.orig_of[r.final_state] : PAREM_NONE;
    res.accepted = (r.final_state < P.n && r.final_state >= P.first_accept) ? 1 : 0;
    res.match_count = r.count;
    res.n_written = (it.positions && it.capacity) ? std::min<uint64_t>(r.count, it.capacity) : 0;
  }
  return PAREM_OK;
}

extern "C" int parem_batch_stats(const parem_batch* batch, parem_stats* out) {
  if (!batch || !out) return PAREM_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  for (uint32_t k = 0; k < batch->n_items; ++k) {
    const DevResult& r = batch->host_res[k];
    out->nonconv_rows += r.nonconv_rows;
    out->conv_max = std::max(out->conv_max, r.conv_max);
    out->cycles_spec += r.cyc_spec;
    out->cycles_main += r.cyc_main;
    out->cycles_resolve += r.cyc_resolve;
    out->cycles_bitmap += r.cyc_bitmap;
    out->cycles_lane += r.cyc_lane;
    out->spec_lookups += r.spec_lookups;
  }
  out->kernels = batch_kernels(batch);
  return PAREM_OK;
}

extern "C" int parem_batch_item_segment(const parem_batch* batch, uint32_t i, uint64_t* segment_bytes) {
  if (!batch || !segment_bytes || i >= batch->n_items) return PAREM_ERR_INVALID_ARG;
  *segment_bytes = batch->seg[i];
  return PAREM_OK;
}

extern "C" int parem_batch_item_config(const parem_batch* batch, uint32_t i, parem_batch_config* out) {
  if (!batch || !out || i >= batch->n_items) return PAREM_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->segment_bytes = batch->seg[i];
  out->spec = batch->spec[i];
  out->warps_per_block = (uint32_t)(batch->block / 32);
  out->smem_table = batch->smem_table[i];
  return PAREM_OK;
}

extern "C" void parem_batch_free(parem_batch* batch) {
  if (!batch) return;
  cudaDeviceSynchronize();
  release(batch);
}

namespace parem {

int batch_create_in(const parem_batch_item* items, uint32_t n, const std::vector<uint64_t>& seg_for,
                    const BatchArena* arena, parem_batch** out) {
  return create_internal(items, n, nullptr, 0, seg_for, false, true, out, arena);
}

int batch_enqueue(parem_batch* b, cudaStream_t st) { return enqueue(b, st); }

void batch_release(parem_batch* b) { release(b); }

int batch_item_result(const parem_batch* b, uint32_t i, parem_result* res) {
  uint32_t k = 0;
  while (k < b->n_items && b->order[k] != i) ++k;
  if (k == b->n_items) return PAREM_ERR_INVALID_ARG;
  return batch_sorted_result(b, k, res);
}

int batch_sorted_result(const parem_batch* b, uint32_t k, parem_result* res) {
  const uint32_t i = b->order[k];
  const parem_batch_item& it = b->items[i];
  const Prepared& P = it.dfa->host;
  const DevResult& r = b->host_res[k];
  std::memset(res, 0, sizeof(*res));
  if (it.len == 0) {
    res->final_state = P.orig_of[P.start];
    res->accepted = P.start >= P.first_accept;
    return PAREM_OK;
  }
  if (r.error == kErrTimeout) return PAREM_ERR_TIMEOUT;
  if (r.error) return PAREM_ERR_INTERNAL;
  if (k < b->n_scan_items) learn_convergence(it.dfa, b->cap[i], r.nonconv_rows, r.conv_max);
  res->final_state = r.final_state < P.n ? P.orig_of[r.final_state] : PAREM_NONE;
  res->accepted = (r.final_state < P.n && r.final_state >= P.first_accept) ? 1 : 0;
  res->match_count = r.count;
  res->n_written = (it.positions && it.capacity) ? std::min<uint64_t>(r.count, it.capacity) : 0;
  return (it.positions && it.capacity > 0 && r.count > it.capacity) ? PAREM_ERR_CAPACITY : PAREM_OK;
}

bool batch_early_result(const parem_batch* b, uint32_t k, parem_result* res) {
  if (!b->host_early || k >= b->n_items) return false;
  const volatile EarlyResult& e = b->host_early[k];
  if (e.ready == 0) return false;
  std::atomic_thread_fence(std::memory_order_acquire);
  const uint32_t i = b->order[k];
  const parem_batch_item& it = b->items[i];
  if (it.len == 0 || e.error != 0 || (it.positions && it.capacity > 0)) return false;
  const Prepared& P = it.dfa->host;
  const uint32_t fs = e.final_state;
  std::memset(res, 0, sizeof(*res));
  res->final_state = fs < P.n ? P.orig_of[fs] : PAREM_NONE;
  res->accepted = (fs < P.n && fs >= P.first_accept) ? 1 : 0;
  res->match_count = e.count;
  return true;
}

uint32_t batch_size(const parem_batch* b) { return b->n_items; }

uint32_t batch_kernels(const parem_batch* b) {
  return (b->n_tiny ? 1u : 0u) + (b->n_scan_items ? 1u : 0u) +
         ((b->n_scan_items && b->any_positions && b->emit_grid > 0) ? 1u : 0u);
}

uint32_t batch_order(const parem_batch* b, uint32_t k) { return b->order[k]; }

int batch_prepare_dfa(parem_dfa* d) { return ensure_batch_dfa(d); }

uint64_t batch_default_segment(const parem_dfa* d) {
  // latency first: a request is answered when its slowest chunk is, and a chunk's main run is
  // one dependent lookup per byte of its rows, so rows are a few synchronisation lengths long
  // (4 x the estimate, 1.25 x the longest merge seen) rather than the planner's 16 x, which
  // pays for throughput with rows of up to several hundred KiB on many-state DFAs
  const Prepared& H = d->host;
  const uint64_t est = H.sync_len == kNoSync ? 0 : H.sync_len;
  const uint64_t conv = d->conv_hint.load();
  uint64_t S = std::max<uint64_t>(4096, std::max<uint64_t>(4 * est, conv + conv / 4));
  S = (S + kBox - 1) / kBox * kBox;
  return std::min(std::min(S, std::max<uint64_t>(4096, min_row_bytes(d, 8))), max_row_bytes(d, H.max_cand));
}

}  // namespace parem
