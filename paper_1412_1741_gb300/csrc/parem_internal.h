// parem_internal.h -- structures shared by the host planner (parem_api.cu, parem_prep.cpp)
// and the kernels (parem_scan.cuh).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda.h>

namespace parem {

constexpr uint32_t kLanes = 32;          // segments per chunk: one per lane of the owning warp
constexpr uint32_t kBox = 64;            // bytes of one TMA column block per row (64B swizzle)
constexpr uint32_t kStages = 2;          // TMA stages per warp
constexpr uint32_t kStageBytes = kLanes * kBox;  // 2 KiB: 32 rows x 64 B
constexpr uint32_t kEmpty = 0xFFFFFFFFu; // an empty candidate register / "no state"
constexpr uint32_t kNoSlot = 0xFFFFu;    // rank(c, q) when q is not a candidate of class c
constexpr uint32_t kLaneCand = 8;        // survivors a lane takes over from the warp-wide phase
// per-warp speculation scratch in shared memory: hand-over lists (32 rows x 8 states, u16),
// a 32-word compaction buffer and five 64-bit phase cycle counters (48 bytes with padding)
constexpr uint32_t kSpecBytes = kLanes * kLaneCand * 2 + kLanes * 4 + 48;
constexpr uint32_t kHeadFlag = 1u;       // SegRec.flags: row 0 re-runs the unaligned head
constexpr uint32_t kSlotsFlag = 2u;      // SegRec.flags: every main-run match of the row is in its slots
constexpr uint32_t kPreFlag = 4u;        // SegRec.flags: replay the merged prefix [0, t) from x
constexpr uint32_t kBitsFlag = 8u;       // SegRec.flags: the main-run matches of [t, row end) are in
                                         // the match bitmap
constexpr uint32_t kRowSlots = 16;       // match positions pass 1 records per row
constexpr uint64_t kMaxText = 1ull << 45;

// Table layouts (parem_dfa_info.layout).  The class layouts read a 256-entry byte -> column
// map; its entries are u8 when every column offset fits a byte, else u16 (the *W layouts).
enum Layout : uint32_t { kByteSmem = 0, kClassSmem = 1, kClassGlobal = 2, kClassSmemW = 3, kClassGlobalW = 4,
                         // batch kernels: class-indexed u16 table with a u16 column map, staged in
                         // shared memory
                         kBatchDyn = 5,
                         // byte-indexed table plus a 4-symbol-stride table for the main run (small
                         // DFAs whose bytes 0..K-2 are distinct classes and all others one class)
                         kByteStride = 6,
                         // class table in shared memory whose columns are computed from the byte:
                         // bytes [lo, lo + w) -> columns 2.., byte xb -> column 1, others column 0
                         kClassWin = 7,
                         // kClassWin plus a two-byte stride table over the hot states for the main
                         // run (texts of lowercase letters and spaces; see the pair table below)
                         kClassPair = 8,
                         // batch kernels: the kBatchDyn copy read from global memory (L2), for
                         // DFAs whose table does not fit the shared memory the stages leave
                         kBatchGlobal = 9 };
// Two-byte stride ("pair") table of kClassPair.  A byte b of {0x20, 0x61..0x7A} has the code
// f = b & 0x1F (0 for the space, 1..26 for a..z); two bytes form the pair index 27 f0 + f1.
// The hot states are the compact states 0 .. H-1 (non-accepting, the most visited ones); row
// e < H holds, for every pair, the hot state reached after both bytes, or the escape value H
// when an intermediate or final state is accepting or not hot.  Row H is all H, so an escaped
// run stays escaped.  Entries are bytes; H <= 254 (in practice shared memory bounds H).
constexpr uint32_t kPairCodes = 27;
constexpr uint32_t kPairRow = kPairCodes * kPairCodes;  // 729 entries per row
constexpr uint32_t kPairMaxHot = 254;
constexpr uint32_t kPairMaxWarps = 24;  // warps per block of its pass 1 (registers and shared memory)
// Text box of pass 1's TMA stages per row: 32 bytes (32-byte swizzle) for kClassPair, whose
// tables leave less shared memory for stages, 64 bytes (64-byte swizzle) otherwise.
constexpr uint32_t box_bytes(uint32_t layout) { return layout == kClassPair ? 32u : kBox; }
constexpr uint32_t kNoSync = 0xFFFFFFFFu;  // Prepared::sync_len: the candidate sets did not synchronise
// Shared memory of every kernel starts with the column map (512 B reserved), then the
// synchronising-byte table (256 u16 at kSyncOff), then the table at this fixed offset, so
// table reads use an immediate offset.
constexpr uint32_t kSyncOff = 512;
constexpr uint32_t kTableOff = 1024;
constexpr uint32_t kNoSync16 = 0xFFFFu;  // sync_state entry of a byte that does not synchronise

// Chunk status word (64 bit), published with release semantics:
//   [63:62] flag  0 none, 1 MAPPED (end state E known), 2 AGGREGATE (E, dead, count),
//                 3 INCLUSIVE (E, prefix dead, prefix count)
//   [61]    dead flag
//   [60:45] E, the compact end state of the chunk assuming a live start
//   [44:0]  count
constexpr uint32_t kFlagMapped = 1, kFlagAggregate = 2, kFlagInclusive = 3;
constexpr uint64_t kCountMask = (1ull << 45) - 1;

// Device error codes (written to the error word; the first one wins).
constexpr uint32_t kErrTimeout = 1, kErrInternal = 2;

// A prepared DFA on the host, in the layout the kernels read.
struct Prepared {
  uint32_t n_in = 0, n_sym = 0;     // as given
  uint32_t n = 0;                   // compact states (incl. dead)
  uint32_t has_dead = 0;
  uint32_t dead = kEmpty;           // compact id of the dead state
  uint32_t first_accept = 0;        // compact ids >= first_accept are in F
  uint32_t start = 0;               // compact q0
  uint32_t n_classes = 0;           // classes of the bytes (the "all states" list is extra)
  uint32_t layout = 0, esize = 1, rowbytes = 0, table_bytes = 0;
  uint32_t max_cand = 0;            // over byte classes
  double mean_cand = 0;
  uint32_t sync_len = 0;            // estimated synchronisation length (symbols), or kNoSync
  uint32_t stride_k = 0;            // kByteStride: symbols K of the stride table (byte b -> min(b, K-1))
  uint32_t stride_off = 0;          // kByteStride: offset of the stride table inside `table`
  uint32_t win = 0;                 // kClassWin, kClassPair: lo | w << 8 | xb << 16
  uint32_t pair_hot = 0;            // kClassPair: hot states H (escape value)
  uint32_t pair_off = 0;            // kClassPair: offset of the pair table inside `table`
  uint32_t main_bytes = 0;          // kClassPair: bytes of the class table before the pair table
  std::vector<uint32_t> orig_of;    // compact -> original (dead -> 0xFFFFFFFF)
  std::vector<uint32_t> compact_of; // original -> compact
  std::vector<uint16_t> byte_class; // 256
  std::vector<uint16_t> colmap;     // 256: column byte offset of each byte in a table row
  std::vector<uint8_t> table;       // n * rowbytes (padded to 16)
  std::vector<uint32_t> img_off;    // n_classes + 2 offsets; list n_classes = all live states
  std::vector<uint16_t> img;        // candidate lists, sorted, dead excluded
  std::vector<uint16_t> rank;       // (n_classes + 1) * n
};

// Host preparation (parem_prep.cpp).  Returns 0 or a PAREM_ERR_* code.
int prepare_dfa(const uint32_t* table, uint32_t n_states, uint32_t n_symbols,
                const uint16_t* byte_to_symbol, uint32_t start, const uint8_t* accept,
                uint32_t smem_table_budget, Prepared* out);

// Device-resident DFA, passed by value to kernels.
struct DeviceDfa {
  const uint8_t* table;
  const uint8_t* colmap;          // 256 entries of 1 or 2 bytes (layout)
  const uint16_t* byte_class;
  const uint32_t* img_off;
  const uint16_t* img;
  const uint16_t* rank;
  uint32_t n, n_classes, first_accept, dead, start;
  uint32_t layout, esize, rowbytes, table_bytes, max_cand;
  uint32_t stride_k, stride_off;  // kByteStride (see Prepared)
  // kByteStride constants of the main run, computed on the host so that the loop reads them
  // as kernel-parameter operands: K^4, the byte dot-product weights (K^3, K^2, K, 1) for
  // K <= 6, and K and K - 1 in every byte
  uint32_t stride_k4, stride_wts, stride_krep, stride_kmrep;
  uint32_t win;                   // kClassWin (see Prepared)
  uint32_t pair_hot, pair_off;    // kClassPair (see Prepared)
  // 256 entries: for a byte whose class leads every live state to one state (its candidate
  // list img(c) has one state), that state; the dead state when the list is empty; kNoSync16
  // otherwise (or for every byte when a state id could be 0xFFFF)
  const uint16_t* sync_state;
};

// Per-segment record for the emit pass: the matches of the row lie in the row-relative
// window [fv, lv), which the emit pass re-runs from state fs.
struct SegRec {
  uint32_t fs;      // state at row offset fv, where the main-run window starts
  uint32_t count;   // matches inside the segment
  uint64_t offset;  // index of the segment's first match in the global position order
  uint32_t fv, lv;  // main-run window (row-relative bytes; the last row extends into the tail)
  uint32_t lvv, ls; // last matching vector [lvv, lv) and the state at lvv (fast replay)
  uint32_t x;       // true start state of the row (before the head bytes for row 0)
  uint32_t flags;   // kHeadFlag | kPreFlag | kSlotsFlag
  uint32_t t;       // length of the merged prefix replayed from x (kPreFlag)
  uint32_t pre;     // matches in the head and the merged prefix
};

// Scratch bytes per row for recorded match positions (row-relative u32).
constexpr uint32_t kRowSlotBytes = kRowSlots * 4;
// Streaming emit pass: positions a lane collects in shared memory before the warp writes them.
constexpr uint32_t kEmitBuf = 32;

// Words of the ticket area (256 B at the start of a scan's header): the chunk ticket, the
// counters of blocks that finished pass 1 and the emit pass, the streaming emit's ticket.
constexpr uint32_t kDoneScanWord = 16, kDoneEmitWord = 32, kEmitTicketWord = 48;

// Result word filled on the device.
struct DevResult {
  uint32_t final_state;  // compact
  uint32_t error;        // kErr* or 0
  uint64_t count;
  uint32_t emit_replays;     // rows whose positions the emit pass had to replay
  uint32_t emit_max_window;  // longest replayed window (bytes)
  uint32_t nonconv_rows;     // rows whose candidates did not merge within the speculation cap
  uint32_t conv_max;         // longest merged prefix t over the rows (bytes)
  uint32_t progress;         // bumped by long serial steps; device waits time out only
                             // when it has not moved for their whole budget
  uint32_t pad;
  // SM cycles spent by the chunk-owning warps, summed over chunks: speculation (with slot
  // maps), main run, resolution (waits, look-back, row records)
  unsigned long long cyc_spec, cyc_main, cyc_resolve;
  unsigned long long cyc_bitmap, cyc_lane;  // parts of cyc_spec: bitmap phase, lane phase
  unsigned long long spec_lookups;          // lookups of candidate runs (see parem_stats)
};
static_assert(sizeof(DevResult) % 8 == 0, "the result word is copied in 8-byte words");

// A batch item's result in host-mapped memory, written by the kernel that finishes the item
// (its last chunk, or the tiny kernel) as soon as it is known, so that a server can answer
// the request before the rest of its batch is done.  `ready` is written last, after a
// system-scope fence.
struct EarlyResult {
  uint32_t final_state;  // compact
  uint32_t error;
  uint64_t count;
  uint32_t ready;
  uint32_t pad;
};

// Parameters of one plain scan (one text).
struct ScanParams {
  DeviceDfa dfa;
  const uint8_t* text;     // text base (any alignment)
  uint64_t n;              // text bytes
  uint64_t h;              // head bytes before the first 16-byte aligned address (< 16)
  uint64_t S;              // bytes per full row (segment), multiple of kBox
  uint64_t R;              // full rows; row r covers [h + r*S, h + (r+1)*S)
  uint64_t tail;           // bytes after the last full row, appended to row R-1
  uint64_t n_chunks;       // ceil(R / 32)
  uint32_t init_state;     // compact start state (q0 or carried in)
  uint32_t group;          // lanes per row in the speculation when P == 1 (power of two <= 32)
  uint32_t bitmap_words;   // words of the per-warp candidate bitmap (0: no bitmap phase)
  uint32_t spec_bytes;     // per-warp speculation scratch in shared memory
  uint32_t enum_all;       // candidates = all live states
  uint32_t spec_cap;       // bytes of speculation before a segment counts as non-converged
  uint32_t cand_stride;    // slots per segment in the slot map
  uint32_t serial_fallback;  // rows that did not merge are run from their resolved start
                             // (no slot maps); else every candidate gets a slot-map entry
  uint64_t pos_base;       // added to every position written (text offset of a piece)
  uint32_t sparse_count;   // main run: track the largest state of each 16-byte vector and
                           // count (by a replay of the vector) only where it is accepting
  uint32_t stream_emit;    // dense matches: the emit pass streams the rows through shared
                           // memory by TMA as pass 1 does (k_emit_stream)
  uint32_t* match_bits;    // dense matches: one bit per body byte (bit i: body byte i ends a
                           // match), written by pass 1's main run and read by k_emit_bits;
                           // nullptr = off
  uint64_t wait_budget;    // clock64 cycles
  int64_t skip_publish;    // test hook (-1 off)
  // scratch
  uint32_t* ticket;
  unsigned long long* status;
  SegRec* segrec;          // nullptr when positions are not requested
  uint32_t* slots;         // R * kRowSlots row-relative match positions (with segrec)
  uint32_t* slot_end;      // R * cand_stride
  uint32_t* slot_cnt;      // R * cand_stride
  DevResult* result;
  DevResult* host_result;  // host-mapped copy of *result, written by the last block of the
                           // scan's last kernel (nullptr: the host copies the result itself)
  EarlyResult* early;      // batch items without positions: early copy of the result (or nullptr)
  uint4* clear;            // zeroed by the kernel (clear_n16 16-byte words): the header
  uint64_t clear_n16;      // region of the previous scan, which the next scan reuses
  // outputs
  uint64_t* positions;
  uint64_t capacity;
  // shared memory: [colmap | table at kTableOff] then, from the first 1024-aligned address
  // at or after kTableOff + smem_table_bytes: per-warp stages, barriers and speculation scratch
  uint32_t smem_table_bytes;
};

// ---------------------------------------------------------------------------------------
// Batch: many (text, DFA) items in one persistent launch.
// ---------------------------------------------------------------------------------------
// One DFA of a batch ("slot"): its items are contiguous in the item array.
struct BatchSlot {
  DeviceDfa dfa;           // kBatchDyn copy: u16 class table, u16 column map
  uint32_t smem_tier;      // 1: the table is staged in shared memory
  uint32_t item_begin, item_end;
  uint32_t grouped;        // 1: candidate sets of at most 32 states, grouped speculation
  uint64_t n_chunks;       // chunks of all its items
  uint64_t n_rows;         // rows of all its items
  uint32_t* ticket;        // chunk ticket counter of the slot
};

// One (text, DFA) item: its scan parameters (scratch pointers inside the batch scratch) and
// the tensor map of its rows.  64-byte aligned for the tensor map.
struct alignas(64) BatchItem {
  CUtensorMap tmap;
  ScanParams p;
  uint64_t chunk_base;     // first chunk ticket of the item within its slot
  uint64_t row_base;       // first row of the item within its slot
};

struct BatchParams {
  const BatchItem* items;
  const BatchSlot* slots;
  const uint32_t* cta_slot;     // first slot of each persistent CTA of the scan kernel
  const uint32_t* emit_slot;    // slot of each CTA of the emit kernel
  const uint64_t* emit_row0;    // first row (within the slot) of each CTA of the emit kernel
  uint32_t n_slots;
  uint32_t max_table_smem;      // largest table staged in shared memory (carve-up)
  uint32_t spec_bytes;          // per-warp speculation scratch (largest over the slots)
  uint32_t pad;
  uint64_t wait_budget;
};

}  // namespace parem
