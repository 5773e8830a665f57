// parem_scan.cuh -- sm_103a kernels of the chunked speculative DFA scan.
//
// Mapping of Algorithm 1 onto the GPU
//   * Domain decomposition: the text is cut into rows ("segments") of S bytes; 32
//     consecutive rows form a chunk, owned by one warp, one row per lane.  Chunks are
//     taken in order from an atomic ticket counter by persistent warps.
//   * Candidate speculation (R = S n L): for row r > 0 the candidates are img(c), the
//     distinct states reachable on the class c of the byte that ends row r-1, minus the
//     dead state (a dead run needs no simulation).  Row 0 starts from q0 exactly.
//   * Candidate runs: lanes hold candidates and advance in lockstep over the row's bytes;
//     lanes whose states meet are merged with __match_any_sync.  Small candidate sets use
//     G lanes per row, so 32/G rows are speculated per pass; large ones use all 32 lanes
//     and P registers per lane for one row, compact the survivors into one register once
//     they fit, and hand the last few (<= 8) to the lane that owns the row, all lanes then
//     finishing their own rows in parallel.  Once one live state is left the row's map is
//     constant from that offset t on; the lane runs that single state over the rest of its
//     row out of shared memory, where a TMA pipeline stages 32 rows x 64 bytes per step
//     (64-byte swizzle, conflict-free 16-byte reads).
//   * Reduction / join: each chunk publishes its end state (MAPPED), then its match count
//     and dead flag given the end state of the previous chunk (AGGREGATE), then the prefix
//     (INCLUSIVE), found by a decoupled look-back over 32 predecessors at a time.  A row
//     whose candidates never merge keeps a full slot map (end, count per candidate).
//   * The matches inside [0, t) of each row are counted by re-running that prefix from the
//     resolved start; the same re-run checks that the start reaches the merged state.
//   * Emit pass: pass 1 records, per row, the first and last 16-byte vectors that hold
//     matches and the states at their starts; rows with matches replay those vectors (the
//     whole window only when matches lie between them) and write the positions at the
//     row's offset in the global order.
#pragma once

// Per-chunk counters in the result word: SM cycles per phase (PAREM_PHASE_STATS) and the
// convergence statistics the planner learns from (PAREM_CONV_STATS).
#ifndef PAREM_PHASE_STATS
#define PAREM_PHASE_STATS 1
#endif
#ifndef PAREM_CONV_STATS
#define PAREM_CONV_STATS 1
#endif

#include <atomic>
#include <cstdint>

#include "parem_internal.h"

namespace parem {

constexpr unsigned kFull = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int32_t x, int32_t y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint4 ldg16(const uint8_t* p) {
  uint4 v;
  asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

__device__ __forceinline__ uint32_t ldg8(const uint8_t* p) {
  uint16_t v;
  asm volatile("ld.global.nc.u8 %0, [%1];" : "=h"(v) : "l"(p));
  return v;
}

// byte i (0..15) of a 16-byte vector, zero-extended (one PRMT)
__device__ __forceinline__ uint32_t byte_of(const uint4& v, int i) {
  const uint32_t w = (i < 4) ? v.x : (i < 8) ? v.y : (i < 12) ? v.z : v.w;
  return __byte_perm(w, 0u, 0x4440u + (uint32_t)(i & 3));
}

__device__ __forceinline__ void set_error(DevResult* r, uint32_t code) {
  atomicCAS(&r->error, 0u, code);
}

__device__ __forceinline__ uint32_t read_error(const DevResult* r) {
  return *reinterpret_cast<const volatile uint32_t*>(&r->error);
}

__device__ __forceinline__ uint32_t read_progress(const DevResult* r) {
  return *reinterpret_cast<const volatile uint32_t*>(&r->progress);
}

// A device wait gives up when its budget has passed with no serial progress anywhere in the
// scan: *t0 and *seen restart while the progress word moves.  *seen starts as kEmpty ("not
// read yet"), so a wait that ends within its budget never reads the progress word; the first
// expiry reads it and grants one more budget.
__device__ __forceinline__ bool wait_expired(const DevResult* r, uint64_t budget, long long* t0, uint32_t* seen) {
  if ((uint64_t)(clock64() - *t0) <= budget) return false;
  const uint32_t pr = read_progress(r);
  if (pr != *seen) {
    *seen = pr;
    *t0 = clock64();
    return false;
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// Transition table access.  The column map sits at shared offset 0 and the table (shared
// layouts) at kTableOff, both addressed from the dynamic shared base, so a lookup is one
// IMAD and one LDS with an immediate offset.
// ---------------------------------------------------------------------------------------
template <int LAYOUT, int ESIZE>
struct Tab {
  static constexpr bool kByte = LAYOUT == kByteSmem || LAYOUT == kByteStride;
  static constexpr bool kGlobal = LAYOUT == kClassGlobal || LAYOUT == kClassGlobalW || LAYOUT == kBatchGlobal;
  static constexpr bool kWide =
      LAYOUT == kClassSmemW || LAYOUT == kClassGlobalW || LAYOUT == kBatchDyn || LAYOUT == kBatchGlobal;
  static constexpr bool kWin = LAYOUT == kClassWin || LAYOUT == kClassPair;
  const uint8_t* sm;       // dynamic shared memory base
  const uint8_t* gtable;   // global table (global layouts)
  uint32_t rowbytes;
  // kClassWin, from the window [lo, lo + w) and the extra byte xb: 2 * (2 - lo) (mod 2^32),
  // 2 * (w + 2) and 2 * (w + 3) (column byte offsets for 2-byte entries), and xb
  uint32_t win_k, win_cap, win_xcol, win_xb;

  __device__ __forceinline__ void set_win(uint32_t win) {
    const uint32_t lo = win & 0xFFu, w = (win >> 8) & 0xFFu;
    win_k = 4u - 2u * lo;
    win_cap = 2u * (w + 2u);
    win_xcol = 2u * (w + 3u);
    win_xb = win >> 16;
  }
  __device__ __forceinline__ uint32_t col(uint32_t b) const {
    if (kByte) return b * ESIZE;
    if (kWin) {
      // a shift-add, a minimum and a select instead of a column-map read from shared memory:
      // column min(b - lo + 2, w + 2) (unsigned), or w + 3 for the extra byte
      uint32_t c2 = min(2u * b + win_k, win_cap);
      c2 = b == win_xb ? win_xcol : c2;
      return ESIZE == 2 ? c2 : c2 >> 1;
    }
    if (kWide) return *reinterpret_cast<const uint16_t*>(sm + 2 * b);
    return sm[b];
  }
  __device__ __forceinline__ uint32_t next(uint32_t s, uint32_t c) const {
    const uint32_t o = s * rowbytes + c;
    if (kGlobal) {
      return ESIZE == 1 ? (uint32_t)__ldg(gtable + o)
                        : (uint32_t)__ldg(reinterpret_cast<const uint16_t*>(gtable + o));
    }
    return ESIZE == 1 ? (uint32_t)sm[kTableOff + o]
                      : (uint32_t)*reinterpret_cast<const uint16_t*>(sm + kTableOff + o);
  }
};

// The synchronising-byte table into shared memory at kSyncOff (all kNoSync16 when the DFA
// has none).
__device__ __forceinline__ void load_sync(uint8_t* sm, const DeviceDfa& D) {
  uint4* dst = reinterpret_cast<uint4*>(sm + kSyncOff);
  const uint4* src = reinterpret_cast<const uint4*>(D.sync_state);
  for (uint32_t i = threadIdx.x; i < 512 / 16; i += blockDim.x)
    dst[i] = src != nullptr ? src[i] : make_uint4(kFull, kFull, kFull, kFull);
}

// Stage the column map, the synchronising-byte table and (shared layouts) the table into
// shared memory.
template <int LAYOUT, int ESIZE>
__device__ __forceinline__ void load_tables(uint8_t* sm, const DeviceDfa& D) {
  const uint32_t cm_bytes = Tab<LAYOUT, ESIZE>::kWide ? 512u : 256u;
  const uint4* src = reinterpret_cast<const uint4*>(D.colmap);
  uint4* dst = reinterpret_cast<uint4*>(sm);
  for (uint32_t i = threadIdx.x; i < cm_bytes / 16; i += blockDim.x) dst[i] = src[i];
  load_sync(sm, D);
  if (!Tab<LAYOUT, ESIZE>::kGlobal) {
    const uint4* ts = reinterpret_cast<const uint4*>(D.table);
    uint4* td = reinterpret_cast<uint4*>(sm + kTableOff);
    for (uint32_t i = threadIdx.x; i < D.table_bytes / 16; i += blockDim.x) td[i] = ts[i];
  }
}

// Batch kernels: the column map, and the table when it is staged, of one slot's DFA.
__device__ __forceinline__ void load_tables_dyn(uint8_t* sm, const DeviceDfa& D, uint32_t smem_tier) {
  const uint4* src = reinterpret_cast<const uint4*>(D.colmap);
  uint4* dst = reinterpret_cast<uint4*>(sm);
  for (uint32_t i = threadIdx.x; i < 512 / 16; i += blockDim.x) dst[i] = src[i];
  load_sync(sm, D);
  if (smem_tier) {
    const uint4* ts = reinterpret_cast<const uint4*>(D.table);
    uint4* td = reinterpret_cast<uint4*>(sm + kTableOff);
    for (uint32_t i = threadIdx.x; i < D.table_bytes / 16; i += blockDim.x) td[i] = ts[i];
  }
}

// Run [0, len) of a 16-byte aligned global range from state x.  Adds the matches to *cnt
// and returns the end state; stops early (returning dead) once the run is dead.  With bits,
// also writes each vector's 16 match bits (bits[o / 16] for the vector at o) to the match
// bitmap of the range.
template <int LAYOUT, int ESIZE>
__device__ uint32_t run_range16(const Tab<LAYOUT, ESIZE>& tab, const uint8_t* p, uint64_t len,
                                uint32_t x, uint32_t dead, uint32_t first_accept, uint32_t* cnt,
                                uint16_t* bits = nullptr) {
  uint32_t c = 0;
  const uint4 zero = make_uint4(0, 0, 0, 0);
  // two vectors in flight ahead of the one being consumed
  uint4 a = len >= 16 ? ldg16(p) : zero, b = len >= 32 ? ldg16(p + 16) : zero;
  for (uint64_t o = 0; o < len; o += 16) {
    const uint4 v = a;
    a = b;
    b = o + 48 <= len ? ldg16(p + o + 32) : zero;
    if (bits != nullptr) {
      uint32_t m = 0;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        x = tab.next(x, tab.col(byte_of(v, i)));
        m |= (x >= first_accept ? 1u : 0u) << i;
      }
      c += __popc(m);
      bits[o / 16] = (uint16_t)m;
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        x = tab.next(x, tab.col(byte_of(v, i)));
        c += (x >= first_accept);
      }
    }
    if (x == dead) break;
  }
  // a dead run cannot have counted matches after dying (dead < first_accept)
  *cnt += c;
  return x;
}

// The whole warp runs one state chain x (warp-uniform) over a 16-byte aligned global range
// [0, len): the lanes load the next 512 bytes while the current 512 are consumed from
// registers by shuffles.  Returns the (uniform) end state; adds the matches to *cnt.
template <int LAYOUT, int ESIZE>
__device__ uint32_t warp_run_range16(const Tab<LAYOUT, ESIZE>& tab, const uint8_t* p, uint64_t len,
                                     uint32_t x, uint32_t dead, uint32_t first_accept, uint32_t* cnt,
                                     uint32_t lane) {
  uint32_t c = 0;
  const uint4 zero = make_uint4(0, 0, 0, 0);
  uint4 cur = (uint64_t)lane * 16 < len ? ldg16(p + lane * 16) : zero;
  for (uint64_t base = 0; base < len && x != dead; base += 512) {
    const uint64_t nb = base + 512 + (uint64_t)lane * 16;
    const uint4 nxt = nb < len ? ldg16(p + nb) : zero;
    const uint64_t left16 = (len - base) / 16;
    const uint32_t nv = left16 < 32 ? (uint32_t)left16 : 32u;
    for (uint32_t k = 0; k < nv; ++k) {
      uint4 v;
      v.x = __shfl_sync(kFull, cur.x, k);
      v.y = __shfl_sync(kFull, cur.y, k);
      v.z = __shfl_sync(kFull, cur.z, k);
      v.w = __shfl_sync(kFull, cur.w, k);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        x = tab.next(x, tab.col(byte_of(v, i)));
        c += (x >= first_accept);
      }
    }
    cur = nxt;
  }
  *cnt += c;
  return x;
}

// Run an arbitrary (unaligned) global byte range [0, len) from x, byte by byte.
template <int LAYOUT, int ESIZE>
__device__ uint32_t run_bytes(const Tab<LAYOUT, ESIZE>& tab, const uint8_t* p, uint64_t len,
                              uint32_t x, uint32_t dead, uint32_t first_accept, uint32_t* cnt) {
  uint32_t c = 0;
  for (uint64_t o = 0; o < len; ++o) {
    x = tab.next(x, tab.col(ldg8(p + o)));
    c += (x >= first_accept);
    if (x == dead) break;
  }
  *cnt += c;
  return x;
}

// Early copy of a finished item's result for the host (see EarlyResult).
__device__ __forceinline__ void write_early(EarlyResult* e, uint32_t final_state, uint64_t count, uint32_t error) {
  e->final_state = final_state;
  e->count = count;
  e->error = error;
  __threadfence_system();
  *reinterpret_cast<volatile uint32_t*>(&e->ready) = 1u;
}

// Associative join of (dead, count) pairs in text order: everything after a death counts 0.
struct Pfx {
  uint32_t dead;
  uint64_t count;
};
__device__ __forceinline__ Pfx pfx_op(Pfx a, Pfx b) {  // a before b
  Pfx r;
  r.dead = a.dead | b.dead;
  r.count = a.dead ? a.count : a.count + b.count;
  return r;
}

__device__ __forceinline__ unsigned long long pack_status(uint32_t flag, uint32_t dead, uint32_t E,
                                                          uint64_t cnt) {
  return ((unsigned long long)flag << 62) | ((unsigned long long)(dead & 1u) << 61) |
         ((unsigned long long)(E & 0xFFFFu) << 45) | (cnt & kCountMask);
}

// Bounded wait on a stage barrier.  Returns false on timeout or when another warp failed.
__device__ __forceinline__ bool stage_wait(uint32_t bar, uint32_t parity, uint64_t budget,
                                           const DevResult* res) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if ((uint64_t)(clock64() - t0) > budget || read_error(res)) return false;
  }
  return true;
}

// Offset of pass 1's per-warp region: the first 1024-aligned shared address after the
// tables (the host reserves 1024 bytes of slack for this alignment).
__device__ __forceinline__ uint32_t stage_region_off(const uint8_t* smem_raw, uint32_t table_bytes) {
  const uint32_t base = smem_u32(smem_raw);
  const uint32_t a = base + kTableOff + table_bytes;
  return ((a + 1023u) & ~1023u) - base;
}

// Per-warp state of pass 1 that persists from chunk to chunk.
struct WarpCtx {
  uint8_t* sm;          // dynamic shared memory base
  uint32_t lane;
  uint32_t stage0;      // offset of this warp's TMA stages
  uint32_t bar0;        // offset of this warp's stage barriers
  uint16_t* hand;       // hand-over lists (32 rows x 8 states)
  uint32_t* cbuf;       // compaction buffer (32 words)
  uint32_t* bitmaps;    // candidate bitmaps and state list (bitmap phase)
  uint32_t phase_bits;  // expected parity of each stage barrier
  uint32_t pending;     // stages issued and not yet waited
  // SM cycles per phase, kept by lane 0 in the warp's shared scratch: speculation, main run,
  // resolution, bitmap, lane phase; summed over chunks, added to the result word by flush_cycles
  unsigned long long* cyc;
};

__device__ __forceinline__ void flush_cycles(WarpCtx& wc, DevResult* r) {
#if PAREM_PHASE_STATS
  if (wc.lane == 0) {
    if (wc.cyc[0] | wc.cyc[1] | wc.cyc[2]) {
      atomicAdd(&r->cyc_spec, wc.cyc[0]);
      atomicAdd(&r->cyc_main, wc.cyc[1]);
      atomicAdd(&r->cyc_resolve, wc.cyc[2]);
      if (wc.cyc[3]) atomicAdd(&r->cyc_bitmap, wc.cyc[3]);
      if (wc.cyc[4]) atomicAdd(&r->cyc_lane, wc.cyc[4]);
    }
    for (int i = 0; i < 5; ++i) wc.cyc[i] = 0;
  }
#endif
}

// One chunk (32 rows) of one text: speculation, main run, look-back, row records.
__device__ __forceinline__ uint4 row_load16(const uint8_t* row, uint32_t pos, uint32_t lim) {
  return pos + 16 <= lim ? ldg16(row + pos) : make_uint4(0, 0, 0, 0);
}

// Sequential 16-byte reads of one row of text [0, lim).  With PF, the vector at the reader's
// position is loaded one step ahead of its use (the kernels for large candidate sets, whose
// speculation runs long past the staged bytes); without, it is loaded when used (fewer live
// registers).
template <bool PF>
struct RowAhead;
template <>
struct RowAhead<true> {
  uint4 v0;
  __device__ __forceinline__ void init(const uint8_t* row, uint32_t pos, uint32_t lim) { v0 = row_load16(row, pos, lim); }
  __device__ __forceinline__ uint4 get(const uint8_t*, uint32_t, uint32_t) const { return v0; }
  // advance from pos to pos + 16
  __device__ __forceinline__ void shift(const uint8_t* row, uint32_t pos, uint32_t lim) {
    v0 = row_load16(row, pos + 16, lim);
  }
};
template <>
struct RowAhead<false> {
  __device__ __forceinline__ void init(const uint8_t*, uint32_t, uint32_t) {}
  __device__ __forceinline__ uint4 get(const uint8_t* row, uint32_t pos, uint32_t lim) const {
    return row_load16(row, pos, lim);
  }
  __device__ __forceinline__ void shift(const uint8_t*, uint32_t, uint32_t) {}
};

// The steps of one chunk (scan_chunk below), each a function of the chunk context and
// the lane's row state; every step is inlined, so the state stays in registers.

// What a warp knows about its chunk j: the rows it covers, the staged bytes and the
// table; constant for the chunk once its first stages have landed.
template <int LAYOUT, int ESIZE>
struct ChunkCtx {
  // the row's bytes arrive in boxes of BOX bytes (32 rows x BOX per stage), swizzled in
  // 16-byte chunks by the TMA unit: chunk c of row k sits at c ^ ((k / SWZ_DIV) & SWZ_MASK)
  static constexpr uint32_t BOX = box_bytes(LAYOUT), SB = kLanes * BOX;
  static constexpr uint32_t SWZ_DIV = 128u / BOX, SWZ_MASK = BOX / 16u - 1u;
  WarpCtx& wc;
  const Tab<LAYOUT, ESIZE>& tab;
  const ScanParams& p;
  const CUtensorMap* tmap;
  uint64_t j;
  uint32_t lane;
  uint32_t dead;         // kEmpty when the DFA has no dead state
  uint32_t A;            // first accepting state
  uint32_t nblk;         // boxes per row
  uint32_t issue_first;  // stages issued at the start of the chunk
  uint32_t cap;          // speculation cap (bytes)
  unsigned lt_mask;
  uint64_t row0, myrow;  // first row of the chunk, the lane's row
  bool active, last_row; // the lane has a row; it is the text's last full row
  uint32_t nrows;        // rows of the chunk
  const uint8_t* body;   // the text after the head (16-byte aligned)
  uint64_t rowlen;       // the lane's row length (the last row takes the tail)
  uint32_t staged = 0;   // bytes of every row in the first stages (set by chunk_begin)

  __device__ __forceinline__ ChunkCtx(WarpCtx& w, const Tab<LAYOUT, ESIZE>& t, const ScanParams& pp,
                                      const CUtensorMap* tm, uint64_t jj)
      : wc(w), tab(t), p(pp), tmap(tm), j(jj) {
    lane = wc.lane;
    dead = p.dfa.dead;
    A = p.dfa.first_accept;
    nblk = (uint32_t)(p.S / BOX);
    issue_first = nblk < kStages ? nblk : kStages;
    cap = p.spec_cap;
    lt_mask = (1u << lane) - 1u;
    row0 = j * kLanes;
    myrow = row0 + lane;
    active = myrow < p.R;
    nrows = (uint32_t)((p.R - row0) < kLanes ? (p.R - row0) : kLanes);
    body = p.text + p.h;
    last_row = active && myrow == p.R - 1;
    rowlen = p.S + (last_row ? p.tail : 0);
  }
  // 16 staged bytes of row k at offset pos (pos < staged)
  __device__ __forceinline__ uint4 staged16(uint32_t k, uint32_t pos) const {
    const uint32_t b = pos / BOX;
    const uint32_t ch = ((pos % BOX) / 16u) ^ ((k / SWZ_DIV) & SWZ_MASK);
    return *reinterpret_cast<const uint4*>(wc.sm + wc.stage0 + b * SB + k * BOX + ch * 16u);
  }
  // the class whose candidate list speculates row r: that of the byte ending row r - 1
  __device__ __forceinline__ uint32_t cand_class(uint64_t r) const {
    return p.enum_all ? p.dfa.n_classes : (uint32_t)p.dfa.byte_class[ldg8(body + r * p.S - 1)];
  }
};

// The lane's row through the speculation steps.
struct RowSpec {
  uint32_t my_off = 0, my_m = 0;  // the row's candidate list (offset, size)
  bool failed = false;            // a stage wait ran out (the error word is set)
  uint32_t my_t = 0;              // offset where the candidates merged (S: never)
  uint32_t my_sigma = kEmpty;     // the merged state at my_t
  uint32_t my_conv = 1;           // the candidates merged
  uint32_t head_cnt = 0;          // row 0: matches in the head bytes
  uint32_t my_hand = 0;           // survivors handed to the lane-parallel phase
  uint32_t my_sync = 0;           // merged at a synchronising byte
  unsigned long long spec_lk = 0; // speculation lookups of the chunk (warp-uniform)
};

// The lane's main run: its end state, match count and the vectors holding matches.
struct RowMain {
  uint32_t s = 0, mu = 0, fv = kEmpty, fs = 0, lvv = 0, ls = 0, lv = 0, nrec = 0, E = 0;
};

// 1. Start the chunk's TMA pipeline, look up every row's candidate list while the first
// stages are in flight, and wait for those stages.
template <int LAYOUT, int ESIZE>
__device__ __forceinline__ void chunk_begin(ChunkCtx<LAYOUT, ESIZE>& C, RowSpec& R) {
  uint8_t* const sm = C.wc.sm;
  const uint32_t lane = C.lane;
  const uint32_t stage0 = C.wc.stage0;
  const uint32_t bar0 = C.wc.bar0;
  uint32_t& phase_bits = C.wc.phase_bits;
  uint32_t& pending = C.wc.pending;
  const DeviceDfa& D = C.p.dfa;
  const uint32_t issue_first = C.issue_first;
  const uint64_t row0 = C.row0;
  const uint64_t myrow = C.myrow;
  const bool active = C.active;
  const ScanParams& p = C.p;
  const CUtensorMap* const tmap = C.tmap;
  constexpr uint32_t BOX = ChunkCtx<LAYOUT, ESIZE>::BOX;
  constexpr uint32_t SB = ChunkCtx<LAYOUT, ESIZE>::SB;
  auto cand_class = [&](uint64_t r) -> uint32_t { return C.cand_class(r); };
  auto& my_off = R.my_off;
  auto& my_m = R.my_m;
  auto& failed = R.failed;
  // 1. start the TMA pipeline for this chunk
  if (lane == 0) {
    for (uint32_t b = 0; b < issue_first; ++b) {
      const uint32_t bar = smem_u32(sm + bar0 + 8 * b);
      mbar_arrive_expect_tx(bar, SB);
      tma_load_2d(smem_u32(sm + stage0 + b * SB), tmap, bar, (int32_t)(b * BOX), (int32_t)row0);
    }
  }
  pending |= (1u << issue_first) - 1u;
  // the candidate list of every row of the chunk (row k: lane k), looked up by the lanes at
  // once while the first stages are in flight: the class of the byte that ends the previous
  // row and the bounds of its list (a chain of dependent global loads, paid once per chunk)
  if (active && myrow > 0) {
    const uint32_t cls = cand_class(myrow);
    my_off = D.img_off[cls];
    my_m = D.img_off[cls + 1] - my_off;
  }
  for (uint32_t b = 0; b < issue_first && !failed; ++b) {
    if (!stage_wait(smem_u32(sm + bar0 + 8 * b), (phase_bits >> b) & 1u, p.wait_budget, p.result)) {
      set_error(p.result, kErrTimeout);
      failed = true;
    }
  }
  C.staged = issue_first * BOX;
}

// Rows merged at a synchronising byte in their staged bytes.
template <int LAYOUT, int ESIZE>
__device__ __forceinline__ void find_sync_byte(const ChunkCtx<LAYOUT, ESIZE>& C, RowSpec& R) {
  uint8_t* const sm = C.wc.sm;
  const uint32_t lane = C.lane;
  const uint64_t myrow = C.myrow;
  const bool active = C.active;
  const uint32_t staged = C.staged;
  const Tab<LAYOUT, ESIZE>& tab = C.tab;
  const ScanParams& p = C.p;
  auto staged16 = [&](uint32_t k, uint32_t pos) -> uint4 { return C.staged16(k, pos); };
  auto& failed = R.failed;
  auto& my_t = R.my_t;
  auto& my_sigma = R.my_sigma;
  auto& my_sync = R.my_sync;
  // Rows that reach a synchronising byte early need no speculation: a byte whose class has
  // a one-state candidate list (Algorithm 1's R = S n L of the position after it is that
  // state for every live start) fixes the run.  Each lane looks for one in the staged bytes of
  // its row and runs that state to the next 16-byte boundary; the row is then merged at that
  // offset (the resolved start replays the bytes before it, as for any merged prefix).
  if (active && myrow > 0 && !p.enum_all && !failed && staged >= 32) {
    const uint16_t* sync = reinterpret_cast<const uint16_t*>(sm + kSyncOff);
    uint32_t t0 = kEmpty, x = 0;
    for (uint32_t pos = 0; pos + 16 < staged && t0 == kEmpty; pos += 16) {
      const uint4 v = staged16(lane, pos);
#pragma unroll
      for (uint32_t q = 0; q < 16; ++q) {
        if (t0 == kEmpty) {
          const uint32_t z = sync[byte_of(v, (int)q)];
          if (z != kNoSync16) {
            t0 = pos + q;
            x = z;
          }
        }
      }
    }
    if (t0 != kEmpty) {
      const uint32_t t1 = (t0 + 16u) & ~15u;
      const uint4 v = staged16(lane, t0 & ~15u);
#pragma unroll
      for (uint32_t q = 0; q < 16; ++q)
        if (q > (t0 & 15u)) x = tab.next(x, tab.col(byte_of(v, (int)q)));
      my_t = t1;
      my_sigma = x;
      my_sync = 1;
    }
  }
}

// 2. Grouped speculation (candidate sets of at most 32 states).
template <int LAYOUT, int ESIZE>
__device__ __forceinline__ void speculate_grouped(const ChunkCtx<LAYOUT, ESIZE>& C, RowSpec& R) {
  const uint32_t lane = C.lane;
  const DeviceDfa& D = C.p.dfa;
  const uint32_t dead = C.dead;
  const uint32_t A = C.A;
  const uint32_t cap = C.cap;
  const uint64_t row0 = C.row0;
  const uint32_t nrows = C.nrows;
  const uint8_t* const body = C.body;
  const uint32_t staged = C.staged;
  const Tab<LAYOUT, ESIZE>& tab = C.tab;
  const ScanParams& p = C.p;
  auto staged16 = [&](uint32_t k, uint32_t pos) -> uint4 { return C.staged16(k, pos); };
  auto& my_off = R.my_off;
  auto& my_m = R.my_m;
  auto& failed = R.failed;
  auto& my_t = R.my_t;
  auto& my_sigma = R.my_sigma;
  auto& my_conv = R.my_conv;
  auto& head_cnt = R.head_cnt;
  auto& my_sync = R.my_sync;
  auto& spec_lk = R.spec_lk;
  // 2. grouped speculation: G lanes per row, 32/G rows per pass
  const uint32_t G = p.group;
  const uint32_t rpp = kLanes / G;
  const uint32_t gi = lane / G, gl = lane % G;
  const unsigned gmask = (G == 32u) ? kFull : (((1u << G) - 1u) << (gi * G));
  for (uint32_t k0 = 0; k0 < nrows && !failed; k0 += rpp) {
    const uint32_t k = k0 + gi;
    const bool valid = k < nrows;
    const uint64_t r = row0 + k;
    const uint32_t off = __shfl_sync(kFull, my_off, k & 31u), m = __shfl_sync(kFull, my_m, k & 31u);
    const bool synced = __shfl_sync(kFull, my_sync, k & 31u) != 0;
    uint32_t st = kEmpty, hc = 0;
    bool exact = false;
    if (valid) {
      if (r == 0) {
        // row 0 starts from the exact state: the initial state run over the head bytes
        if (gl == 0) {
          st = run_bytes(tab, p.text, p.h, p.init_state, dead, A, &hc);
          if (st == dead) st = kEmpty;
        }
        exact = true;
      } else if (!synced) {
        if (gl < m && m <= G) st = (uint32_t)D.img[off + gl];
      }
    }
    // a row whose group has at most one live lane is already merged at t = 0
    unsigned live = __ballot_sync(kFull, st != kEmpty);
    bool done = exact || !valid || synced || __popc(live & gmask) <= 1;
    uint32_t pos = 0, outcome = 1;
    const uint8_t* grow = body + (row0 + (valid ? k : 0u)) * p.S;
    const uint32_t kk = valid ? k : 0u;
    RowAhead<false> ra;
    ra.init(grow, staged, (uint32_t)p.S);
    while (!__all_sync(kFull, done)) {
      if (!done && pos >= cap) {
        done = true;
        outcome = 3;
      }
#if PAREM_CONV_STATS
      spec_lk += 16u * (uint32_t)__popc(__ballot_sync(kFull, !done && st != kEmpty));
#endif
      const uint4 v = pos < staged ? staged16(kk, pos) : ra.get(grow, pos, (uint32_t)p.S);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int i2 = 0; i2 < 4; ++i2) {
          if (!done && st != kEmpty) {
            const uint32_t s2 = tab.next(st, tab.col(byte_of(v, q * 4 + i2)));
            st = (s2 == dead) ? kEmpty : s2;
          }
        }
        const uint32_t key = st == kEmpty ? kEmpty : ((gi << 16) | st);
        const unsigned grp = __match_any_sync(kFull, key);
        if (st != kEmpty && (uint32_t)(__ffs(grp) - 1) != lane) st = kEmpty;
      }
      if (!done) {
        if (pos >= staged) ra.shift(grow, pos, (uint32_t)p.S);
        pos += 16;
      }
      live = __ballot_sync(kFull, st != kEmpty);
      if (!done && __popc(live & gmask) <= 1) done = true;
    }
    // the surviving state of each row (or dead) and the outcome go to the row's lane
    live = __ballot_sync(kFull, st != kEmpty);
    const unsigned mine = live & gmask;
    const uint32_t sig = __shfl_sync(kFull, st, mine ? (uint32_t)(__ffs(mine) - 1) : gi * G);
    const uint32_t sigma_row = mine ? sig : dead;
    const uint32_t hcg = __shfl_sync(kFull, hc, gi * G);
    // lane k (k in [k0, k0 + rpp)) collects from group k - k0
    const uint32_t from = ((lane - k0) % rpp) * G;
    const uint32_t o_sig = __shfl_sync(kFull, sigma_row, from);
    const uint32_t o_out = __shfl_sync(kFull, outcome, from);
    const uint32_t o_pos = __shfl_sync(kFull, pos, from);
    const uint32_t o_hc = __shfl_sync(kFull, hcg, from);
    if (lane >= k0 && lane < k0 + rpp && lane < nrows && !my_sync) {
      my_conv = o_out == 1;
      my_t = o_out == 3 ? (uint32_t)p.S : o_pos;
      my_sigma = o_out == 1 ? o_sig : kEmpty;
      head_cnt = o_hc;
    }
  }
  if (row0 != 0 || lane != 0) head_cnt = 0;
}

// 2a. Warp-wide speculation over P registers per lane.
template <int LAYOUT, int ESIZE, int P>
__device__ __forceinline__ void speculate_warp(const ChunkCtx<LAYOUT, ESIZE>& C, RowSpec& R) {
  const uint32_t lane = C.lane;
  uint16_t* const hand = C.wc.hand;
  uint32_t* const cbuf = C.wc.cbuf;
  uint32_t* const bitmaps = C.wc.bitmaps;
  const DeviceDfa& D = C.p.dfa;
  const uint32_t dead = C.dead;
  const uint32_t A = C.A;
  const uint32_t cap = C.cap;
  const unsigned lt_mask = C.lt_mask;
  const uint64_t row0 = C.row0;
  const uint32_t nrows = C.nrows;
  const uint8_t* const body = C.body;
  const uint32_t staged = C.staged;
  const Tab<LAYOUT, ESIZE>& tab = C.tab;
  const ScanParams& p = C.p;
  WarpCtx& wc = C.wc;
  auto staged16 = [&](uint32_t k, uint32_t pos) -> uint4 { return C.staged16(k, pos); };
  auto& my_off = R.my_off;
  auto& my_m = R.my_m;
  auto& failed = R.failed;
  auto& my_t = R.my_t;
  auto& my_sigma = R.my_sigma;
  auto& my_conv = R.my_conv;
  auto& head_cnt = R.head_cnt;
  auto& my_hand = R.my_hand;
  auto& my_sync = R.my_sync;
  auto& spec_lk = R.spec_lk;
  // 2a. warp-wide speculation, one row at a time, candidates across lanes and registers
  for (uint32_t k = 0; k < nrows && !failed; ++k) {
    const uint64_t r = row0 + k;
    if (r == 0) {
      uint32_t c0 = 0;
      const uint32_t sh = run_bytes(tab, p.text, p.h, p.init_state, dead, A, &c0);
      if (lane == 0) {
        my_t = 0;
        my_sigma = sh;
        head_cnt = c0;
      }
      continue;
    }
    if (__shfl_sync(kFull, my_sync, k)) continue;  // merged at a synchronising byte
    const uint32_t off = __shfl_sync(kFull, my_off, k), m = __shfl_sync(kFull, my_m, k);
    const bool big = m > 32u * P;
    if (m <= 1 || (big && p.bitmap_words == 0)) {
      if (lane == k) {
        my_t = big ? (uint32_t)p.S : 0u;
        my_conv = m <= 1;
        my_sigma = m == 1 ? (uint32_t)D.img[off] : dead;
      }
      continue;
    }
    uint32_t st[P];
    uint32_t lr = 0;  // registers that may hold live candidates (warp-uniform)
    uint32_t live_n = m;  // live candidates after the last merge check (warp-uniform)
    uint32_t pos = 0, sigma = kEmpty, outcome = 0;  // 1 merged, 2 handed to the lane, 3 not merging
#if PAREM_PHASE_STATS
    const uint32_t cb0 = (uint32_t)clock64();
#endif
    if (big) {
      // More candidates than registers: the warp keeps the candidate set as a bitmap over
      // the states (duplicates merge by construction) until it fits 32 * P registers.
      const uint32_t W = p.bitmap_words;
      uint32_t* bm0 = bitmaps;
      uint32_t* bm1 = bitmaps + W;
      for (uint32_t w = lane; w < W; w += 32) bm0[w] = 0;
      __syncwarp();
      for (uint32_t slot = lane; slot < m; slot += 32) {
        const uint32_t q = D.img[off + slot];
        atomicOr(&bm0[q >> 5], 1u << (q & 31u));
      }
      __syncwarp();
      uint32_t cnt = m;
      const uint8_t* brow = body + r * p.S;
      RowAhead<(P >= 4)> ra;
      ra.init(brow, pos > staged ? pos : staged, (uint32_t)p.S);
      for (;;) {
        if (pos >= cap) {
          outcome = 3;
          break;
        }
        const uint4 v = pos < staged ? staged16(k, pos) : ra.get(brow, pos, (uint32_t)p.S);
        if (pos >= staged) ra.shift(brow, pos, (uint32_t)p.S);
#if PAREM_CONV_STATS
        spec_lk += 16u * live_n;
#endif
#pragma unroll 1
        for (int q = 0; q < 16; ++q) {
          const uint32_t c = tab.col(byte_of(v, q));
          for (uint32_t w = lane; w < W; w += 32) bm1[w] = 0;
          __syncwarp();
          for (uint32_t w = lane; w < W; w += 32) {
            uint32_t bits = bm0[w];
            while (bits) {
              // up to four independent lookups in flight
              uint32_t qs[4], nq[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                qs[u] = kEmpty;
                if (bits) {
                  qs[u] = w * 32u + (uint32_t)(__ffs(bits) - 1);
                  bits &= bits - 1;
                }
              }
#pragma unroll
              for (int u = 0; u < 4; ++u) nq[u] = qs[u] != kEmpty ? tab.next(qs[u], c) : dead;
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (qs[u] != kEmpty && nq[u] != dead) atomicOr(&bm1[nq[u] >> 5], 1u << (nq[u] & 31u));
            }
          }
          __syncwarp();
          uint32_t* tmp = bm0;
          bm0 = bm1;
          bm1 = tmp;
        }
        pos += 16;
        uint32_t local = 0;
        for (uint32_t w = lane; w < W; w += 32) local += __popc(bm0[w]);
        cnt = __reduce_add_sync(kFull, local);
        live_n = cnt;
        if (cnt <= 32u * P) break;
      }
#if PAREM_PHASE_STATS
      if (lane == 0) wc.cyc[3] += (uint32_t)clock64() - cb0;
#endif
      if (outcome == 0) {
        // list the surviving states in the hand-over buffer, then load the registers
        uint32_t local = 0;
        for (uint32_t w = lane; w < W; w += 32) local += __popc(bm0[w]);
        uint32_t incl = local;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t o = __shfl_up_sync(kFull, incl, d);
          if (lane >= (uint32_t)d) incl += o;
        }
        uint32_t idx = incl - local;
        // the list has its own buffer after the two bitmaps: the hand-over lists of
        // earlier rows of this chunk must survive until phase 2b
        uint16_t* list = reinterpret_cast<uint16_t*>(bitmaps + 2 * W);
        for (uint32_t w = lane; w < W; w += 32) {
          uint32_t bits = bm0[w];
          while (bits) {
            list[idx++] = (uint16_t)(w * 32u + (uint32_t)(__ffs(bits) - 1));
            bits &= bits - 1;
          }
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < P; ++i) {
          const uint32_t slot = (uint32_t)i * 32u + lane;
          st[i] = slot < cnt ? (uint32_t)list[slot] : kEmpty;
          if ((uint32_t)i * 32u < cnt) lr |= 1u << i;
        }
        __syncwarp();
      }
    } else {
#pragma unroll
      for (int i = 0; i < P; ++i) {
        const uint32_t slot = (uint32_t)i * 32u + lane;
        st[i] = slot < m ? (uint32_t)D.img[off + slot] : kEmpty;
        if ((uint32_t)i * 32u < m) lr |= 1u << i;
      }
    }
    const uint8_t* wrow = body + r * p.S;
    RowAhead<(P >= 4)> wa;
    wa.init(wrow, pos > staged ? pos : staged, (uint32_t)p.S);
    for (; outcome == 0;) {
      if (pos >= cap) {
        outcome = 3;
        break;
      }
      const uint4 v = pos < staged ? staged16(k, pos) : wa.get(wrow, pos, (uint32_t)p.S);
      if (pos >= staged) wa.shift(wrow, pos, (uint32_t)p.S);
#if PAREM_CONV_STATS
      spec_lk += 16u * live_n;
#endif
      if (p.bitmap_words) {
        // 16 steps with no merging inside them, then one merge of equal states across all
        // lanes and registers through the state bitmap, which also packs the survivors
        // densely into the first registers
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const uint32_t c = tab.col(byte_of(v, q));
#pragma unroll
          for (int i = 0; i < P; ++i) {
            if ((lr >> i) & 1u) {
              if (st[i] != kEmpty) {
                const uint32_t s2 = tab.next(st[i], c);
                st[i] = (s2 == dead) ? kEmpty : s2;
              }
            }
          }
        }
        pos += 16;
        const uint32_t W = p.bitmap_words;
        uint32_t* bm = bitmaps;
        for (uint32_t w = lane; w < W; w += 32) bm[w] = 0;
        __syncwarp();
#pragma unroll
        for (int i = 0; i < P; ++i)
          if (((lr >> i) & 1u) && st[i] != kEmpty) atomicOr(&bm[st[i] >> 5], 1u << (st[i] & 31u));
        __syncwarp();
        uint32_t local = 0;
        for (uint32_t w = lane; w < W; w += 32) local += __popc(bm[w]);
        uint32_t incl = local;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t o = __shfl_up_sync(kFull, incl, d);
          if (lane >= (uint32_t)d) incl += o;
        }
        const uint32_t cnt = __shfl_sync(kFull, incl, 31);
        live_n = cnt;
        uint32_t idx = incl - local;
        uint16_t* list = reinterpret_cast<uint16_t*>(bitmaps + 2 * W);
        for (uint32_t w = lane; w < W; w += 32) {
          uint32_t bits = bm[w];
          while (bits) {
            list[idx++] = (uint16_t)(w * 32u + (uint32_t)(__ffs(bits) - 1));
            bits &= bits - 1;
          }
        }
        __syncwarp();
        lr = 0;
#pragma unroll
        for (int i = 0; i < P; ++i) {
          const uint32_t slot = (uint32_t)i * 32u + lane;
          st[i] = slot < cnt ? (uint32_t)list[slot] : kEmpty;
          if ((uint32_t)i * 32u < cnt) lr |= 1u << i;
        }
        __syncwarp();
        if (cnt <= 1) {
          outcome = 1;
          sigma = cnt ? __shfl_sync(kFull, st[0], 0) : dead;
          break;
        }
        if (cnt <= kLaneCand) {
          // few survivors left: the lane that owns the row finishes them (phase 2b)
          if (lane < cnt) hand[k * kLaneCand + lane] = (uint16_t)st[0];
          sigma = cnt;
          outcome = 2;
          break;
        }
        continue;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int i2 = 0; i2 < 4; ++i2) {
          const uint32_t c = tab.col(byte_of(v, q * 4 + i2));
#pragma unroll
          for (int i = 0; i < P; ++i) {
            if ((lr >> i) & 1u) {
              if (st[i] != kEmpty) {
                const uint32_t s2 = tab.next(st[i], c);
                st[i] = (s2 == dead) ? kEmpty : s2;
              }
            }
          }
        }
        // merge lanes whose candidates met (within each register)
#pragma unroll
        for (int i = 0; i < P; ++i) {
          if ((lr >> i) & 1u) {
            const unsigned grp = __match_any_sync(kFull, st[i]);
            if (st[i] != kEmpty && (uint32_t)(__ffs(grp) - 1) != lane) st[i] = kEmpty;
          }
        }
      }
      pos += 16;
      uint32_t total = 0, nlr = 0;
      unsigned bl[P];
#pragma unroll
      for (int i = 0; i < P; ++i) {
        bl[i] = ((lr >> i) & 1u) ? __ballot_sync(kFull, st[i] != kEmpty) : 0u;
        total += __popc(bl[i]);
        if (bl[i]) nlr |= 1u << i;
      }
      lr = nlr;
      if (total <= 32 && (lr & ~1u)) {
        // all survivors fit one register: compact them into register 0, then merge
        uint32_t base = 0;
#pragma unroll
        for (int i = 0; i < P; ++i) {
          if (st[i] != kEmpty) cbuf[base + __popc(bl[i] & lt_mask)] = st[i];
          base += __popc(bl[i]);
        }
        __syncwarp();
        st[0] = lane < total ? cbuf[lane] : kEmpty;
#pragma unroll
        for (int i = 1; i < P; ++i) st[i] = kEmpty;
        __syncwarp();
        const unsigned grp = __match_any_sync(kFull, st[0]);
        if (st[0] != kEmpty && (uint32_t)(__ffs(grp) - 1) != lane) st[0] = kEmpty;
        bl[0] = __ballot_sync(kFull, st[0] != kEmpty);
#pragma unroll
        for (int i = 1; i < P; ++i) bl[i] = 0;
        total = __popc(bl[0]);
        lr = 1;
      }
      live_n = total;
      if (total <= 1) {
        outcome = 1;
        if (total == 0) {
          sigma = dead;
        } else {
          uint32_t reg = 0, holder = 0;
#pragma unroll
          for (int i = P - 1; i >= 0; --i)
            if (bl[i]) {
              reg = (uint32_t)i;
              holder = __ffs(bl[i]) - 1;
            }
          uint32_t val = kEmpty;
#pragma unroll
          for (int i = 0; i < P; ++i)
            if ((uint32_t)i == reg) val = st[i];
          sigma = __shfl_sync(kFull, val, holder);
        }
        break;
      }
      if (total <= kLaneCand && lr == 1u) {
        // few survivors left: the lane that owns the row finishes them (phase 2b)
        if (st[0] != kEmpty) hand[k * kLaneCand + __popc(bl[0] & lt_mask)] = (uint16_t)st[0];
        sigma = total;
        outcome = 2;
        break;
      }
    }
    if (lane == k) {
      my_conv = outcome == 1;
      my_t = outcome == 3 ? (uint32_t)p.S : pos;
      my_sigma = outcome == 1 ? sigma : kEmpty;
      my_hand = outcome == 2 ? sigma : 0u;
    }
  }

}

// 2b. Lane-parallel speculation of the survivors the warp-wide phase handed over.
template <int LAYOUT, int ESIZE, int P>
__device__ __forceinline__ void speculate_lanes(const ChunkCtx<LAYOUT, ESIZE>& C, RowSpec& R) {
  const uint32_t lane = C.lane;
  uint16_t* const hand = C.wc.hand;
  const uint32_t dead = C.dead;
  const uint32_t cap = C.cap;
  const uint64_t row0 = C.row0;
  const uint64_t myrow = C.myrow;
  const bool active = C.active;
  const uint8_t* const body = C.body;
  const uint32_t staged = C.staged;
  const Tab<LAYOUT, ESIZE>& tab = C.tab;
  const ScanParams& p = C.p;
  WarpCtx& wc = C.wc;
  auto staged16 = [&](uint32_t k, uint32_t pos) -> uint4 { return C.staged16(k, pos); };
  auto& failed = R.failed;
  auto& my_t = R.my_t;
  auto& my_sigma = R.my_sigma;
  auto& my_conv = R.my_conv;
  auto& my_hand = R.my_hand;
  auto& spec_lk = R.spec_lk;
#if PAREM_PHASE_STATS
  const uint32_t cl0 = (uint32_t)clock64();
#endif
  // 2b. lane-parallel speculation: each lane runs the few survivors of its own row
  if (__ballot_sync(kFull, my_hand != 0) && !failed) {
    __syncwarp();
    // every lane runs the loop (lanes without survivors idle through it); the survivor
    // slots it touches are bounded by the warp's largest survivor count, which is uniform,
    // so slots nobody uses cost nothing
    {
      uint32_t ls[kLaneCand];
#pragma unroll
      for (uint32_t i = 0; i < kLaneCand; ++i)
        ls[i] = i < my_hand ? (uint32_t)hand[lane * kLaneCand + i] : kEmpty;
      uint32_t L = my_hand, pos = my_t, lk2 = 0;
      bool busy = my_hand != 0;
      const uint8_t* lrow = body + (active ? myrow : row0) * p.S;
      RowAhead<(P >= 4)> la;
      if (busy) la.init(lrow, pos > staged ? pos : staged, (uint32_t)p.S);
      for (;;) {
        if (busy && pos >= cap) {
          my_conv = 0;
          my_t = (uint32_t)p.S;
          busy = false;
        }
        const uint32_t lmax = __reduce_max_sync(kFull, busy ? L : 0u);
        if (lmax == 0) break;
        lk2 += busy ? 16u * L : 0u;
        const uint4 v = !busy ? make_uint4(0, 0, 0, 0) : pos < staged ? staged16(lane, pos) : la.get(lrow, pos, (uint32_t)p.S);
        if (busy && pos >= staged) la.shift(lrow, pos, (uint32_t)p.S);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const uint32_t c = tab.col(byte_of(v, q));
#pragma unroll
          for (uint32_t i = 0; i < kLaneCand; ++i) {
            if (i < lmax) {  // warp-uniform
              if (ls[i] != kEmpty) {
                const uint32_t s2 = tab.next(ls[i], c);
                ls[i] = (s2 == dead) ? kEmpty : s2;
              }
            }
          }
        }
        pos += 16;
        // merge equal survivors and compact them to the front
        uint32_t out[kLaneCand];
#pragma unroll
        for (uint32_t i = 0; i < kLaneCand; ++i) out[i] = kEmpty;
        uint32_t np = 0;
#pragma unroll
        for (uint32_t i = 0; i < kLaneCand; ++i) {
          if (i < lmax) {
            bool keep = ls[i] != kEmpty;
#pragma unroll
            for (uint32_t jj = 0; jj < i; ++jj)
              if (ls[jj] == ls[i]) keep = false;
#pragma unroll
            for (uint32_t qq = 0; qq < kLaneCand; ++qq)
              if (qq <= i && keep && qq == np) out[qq] = ls[i];
            np += keep ? 1u : 0u;
          }
        }
#pragma unroll
        for (uint32_t i = 0; i < kLaneCand; ++i) ls[i] = out[i];
        if (busy) {
          L = np;
          if (L <= 1) {
            my_conv = 1;
            my_t = pos;
            my_sigma = L ? ls[0] : dead;
            busy = false;
          }
        }
      }
      my_hand = 0;
#if PAREM_CONV_STATS
      spec_lk += __reduce_add_sync(kFull, lk2);
#endif
    }
    __syncwarp();
  }
#if PAREM_PHASE_STATS
  if (lane == 0) wc.cyc[4] += (uint32_t)clock64() - cl0;
#endif
}

// Convergence counters of the chunk for the planner.
template <int LAYOUT, int ESIZE>
__device__ __forceinline__ void record_convergence(const ChunkCtx<LAYOUT, ESIZE>& C, const RowSpec& R) {
  const uint32_t lane = C.lane;
  const bool active = C.active;
  const ScanParams& p = C.p;
  auto& my_t = R.my_t;
  auto& my_conv = R.my_conv;
  auto& spec_lk = R.spec_lk;
#if PAREM_CONV_STATS
  // convergence statistics for the planner (one update per chunk)
  {
    const unsigned nc = __ballot_sync(kFull, active && !my_conv);
    uint32_t tmax = (active && my_conv) ? my_t : 0u;
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) tmax = max(tmax, __shfl_xor_sync(kFull, tmax, d));
    if (lane == 0) {
      if (nc) atomicAdd(&p.result->nonconv_rows, (uint32_t)__popc(nc));
      if (tmax) atomicMax(&p.result->conv_max, tmax);
      if (spec_lk) atomicAdd(&p.result->spec_lookups, spec_lk);
    }
  }
#endif
}

// 3. Slot maps of the rows that did not merge.
template <int LAYOUT, int ESIZE>
__device__ __forceinline__ void run_slot_maps(const ChunkCtx<LAYOUT, ESIZE>& C, RowSpec& R) {
  const uint32_t lane = C.lane;
  const DeviceDfa& D = C.p.dfa;
  const uint32_t dead = C.dead;
  const uint32_t A = C.A;
  const uint64_t row0 = C.row0;
  const bool active = C.active;
  const uint8_t* const body = C.body;
  const Tab<LAYOUT, ESIZE>& tab = C.tab;
  const ScanParams& p = C.p;
  auto cand_class = [&](uint64_t r) -> uint32_t { return C.cand_class(r); };
  auto& failed = R.failed;
  auto& my_conv = R.my_conv;
  // 3. slot maps of rows whose candidates did not merge (rare): every candidate runs
  //    the whole row (and the tail on the last row), lanes over candidates
  unsigned nonconv = p.serial_fallback ? 0u : __ballot_sync(kFull, active && !my_conv);
  while (nonconv && !failed) {
    const uint32_t k = __ffs(nonconv) - 1;
    nonconv &= nonconv - 1;
    const uint64_t r = row0 + k;
    const uint32_t cls = cand_class(r);
    const uint32_t off = D.img_off[cls];
    const uint32_t m = D.img_off[cls + 1] - off;
    for (uint32_t base = 0; base < m; base += 32) {
      const uint32_t slot = base + lane;
      uint32_t x = slot < m ? (uint32_t)D.img[off + slot] : 0u;
      uint32_t c = 0;
      x = run_range16(tab, body + r * p.S, p.S, x, dead, A, &c);
      if (r == p.R - 1 && p.tail) x = run_bytes(tab, body + p.R * p.S, p.tail, x, dead, A, &c);
      if (slot < m) {
        p.slot_end[r * p.cand_stride + slot] = x;
        p.slot_cnt[r * p.cand_stride + slot] = c;
      }
    }
    if (lane == 0) atomicAdd(&p.result->progress, 1u);
#if PAREM_CONV_STATS
    if (lane == 0)
      atomicAdd(&p.result->spec_lookups, (unsigned long long)m * (p.S + (r == p.R - 1 ? p.tail : 0)));
#endif
  }
}

// 4. The main run of every merged row (and the tail on the last row); false when a stage
// wait ran out.
template <int LAYOUT, int ESIZE>
__device__ __forceinline__ bool main_run(ChunkCtx<LAYOUT, ESIZE>& C, RowSpec& R, RowMain& M) {
  // the match bitmap (dense emission) is never planned for the stride layouts: no code for it
  constexpr bool kBits = LAYOUT != kByteStride && LAYOUT != kClassPair;
  uint8_t* const sm = C.wc.sm;
  const uint32_t lane = C.lane;
  const uint32_t stage0 = C.wc.stage0;
  const uint32_t bar0 = C.wc.bar0;
  uint32_t& phase_bits = C.wc.phase_bits;
  uint32_t& pending = C.wc.pending;
  const DeviceDfa& D = C.p.dfa;
  const uint32_t A = C.A;
  const uint32_t nblk = C.nblk;
  const uint64_t row0 = C.row0;
  const uint64_t myrow = C.myrow;
  const bool active = C.active;
  const uint8_t* const body = C.body;
  const bool last_row = C.last_row;
  const Tab<LAYOUT, ESIZE>& tab = C.tab;
  const ScanParams& p = C.p;
  const CUtensorMap* const tmap = C.tmap;
  constexpr uint32_t BOX = ChunkCtx<LAYOUT, ESIZE>::BOX;
  constexpr uint32_t SB = ChunkCtx<LAYOUT, ESIZE>::SB;
  constexpr uint32_t SWZ_DIV = ChunkCtx<LAYOUT, ESIZE>::SWZ_DIV;
  constexpr uint32_t SWZ_MASK = ChunkCtx<LAYOUT, ESIZE>::SWZ_MASK;
  auto& failed = R.failed;
  auto& my_t = R.my_t;
  auto& my_sigma = R.my_sigma;
  auto& my_conv = R.my_conv;
  auto& s = M.s;
  auto& mu = M.mu;
  auto& fv = M.fv;
  auto& fs = M.fs;
  auto& lvv = M.lvv;
  auto& ls = M.ls;
  auto& lv = M.lv;
  auto& nrec = M.nrec;
  auto& E = M.E;
  // 4. main run: each lane runs its merged state over the rest of its row from smem,
  //    remembering the first and last 16-byte vectors that contain matches
  s = my_sigma;
  const bool run = active && my_conv;
  uint32_t* myslots = p.slots ? p.slots + myrow * kRowSlots : nullptr;
  for (uint32_t blk = 0; blk < nblk && !failed; ++blk) {
    const uint32_t b = blk % kStages;
    const uint32_t bar = smem_u32(sm + bar0 + 8 * b);
    if (!stage_wait(bar, (phase_bits >> b) & 1u, p.wait_budget, p.result)) {
      set_error(p.result, kErrTimeout);
      failed = true;
      break;
    }
    phase_bits ^= 1u << b;
    pending &= ~(1u << b);
    uint4 v[BOX / 16];
    const uint8_t* stg = sm + stage0 + b * SB + lane * BOX;
#pragma unroll
    for (uint32_t i = 0; i < BOX / 16; ++i)
      v[i] = *reinterpret_cast<const uint4*>(stg + ((i ^ ((lane / SWZ_DIV) & SWZ_MASK)) * 16u));
    __syncwarp();
    if (blk + kStages < nblk) {
      if (lane == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(bar, SB);
        tma_load_2d(smem_u32(sm + stage0 + b * SB), tmap, bar, (int32_t)((blk + kStages) * BOX), (int32_t)row0);
      }
      pending |= 1u << b;
    }
    if (run) {
      const uint32_t col0 = blk * BOX;
      unsigned long long bmask = 0;  // match bits of this block (match bitmap only)
#pragma unroll
      for (uint32_t i = 0; i < BOX / 16; ++i) {
        const uint32_t col = col0 + i * 16u;
        if (col >= my_t) {
          bool exact = true;  // the vector is run byte by byte below
          if constexpr (LAYOUT == kClassPair) {
            // Two bytes per lookup while the run stays in the hot states and every byte is a
            // space or a lowercase letter.  Each word's codes f = b & 0x1F index the pair table
            // by one byte dot product (27 f0 + f1, 27 f2 + f3) on top of the row base.  The
            // fold is exact only for {0x20, 0x61..0x7A}: per byte, bit 7 must be clear, bit 5
            // set, bit 6 equal to (f != 0) and f < 27; any other byte, and any escape (a
            // cold or accepting state within the vector), sends the vector to the byte loop
            // from its start state.  A vector taken here has no match (hot states are not
            // accepting and the table escapes on an accepting step).
            const uint32_t H = D.pair_hot, t2 = D.pair_off;
            const uint32_t ws[4] = {v[i].x, v[i].y, v[i].z, v[i].w};
            uint32_t e = min(s, H);
            uint32_t acc_a = 0, acc_b = 0, acc_c = 0xFFFFFFFFu;
#pragma unroll
            for (int g = 0; g < 4; g += 2) {
              const uint32_t w0 = ws[g], w1 = ws[g + 1];
              const uint32_t f0 = w0 & 0x1F1F1F1Fu, f1 = w1 & 0x1F1F1F1Fu;
              // bit 7: b >= 0x80; bit 6: bit 6 of b != (f != 0)
              acc_a |= (f0 + 0x3F3F3F3Fu) ^ w0;
              acc_a |= (f1 + 0x3F3F3F3Fu) ^ w1;
              acc_b |= (f0 + 0x65656565u) | (f1 + 0x65656565u);  // bit 7: f >= 27
              acc_c &= w0 & w1;                                  // bit 5 must stay set
              // the pair offsets do not depend on the state: only one multiply-add and the
              // lookup are on the dependent chain
              const uint32_t q0 = __dp4a(f0, 0x0000011Bu, t2), q1 = __dp4a(f0, 0x011B0000u, t2);
              const uint32_t q2 = __dp4a(f1, 0x0000011Bu, t2), q3 = __dp4a(f1, 0x011B0000u, t2);
              e = sm[kTableOff + e * kPairRow + q0];
              e = sm[kTableOff + e * kPairRow + q1];
              e = sm[kTableOff + e * kPairRow + q2];
              e = sm[kTableOff + e * kPairRow + q3];
            }
            const uint32_t bad = (acc_a & 0xC0C0C0C0u) | (acc_b & 0x80808080u) | (~acc_c & 0x20202020u);
            exact = (bad != 0u) | (e >= H);
            if (!exact) s = e;
          }
          if (exact) {
          const uint32_t mu0 = mu, s0 = s;
          if constexpr (LAYOUT == kByteStride) {
            // four bytes per lookup: the stride table holds the state after them and how
            // many of the four steps end in an accepting state
            const uint32_t K = D.stride_k, km = K - 1, k4 = D.stride_k4;
            const uint8_t* stab = sm + kTableOff + D.stride_off;
            const uint32_t ws[4] = {v[i].x, v[i].y, v[i].z, v[i].w};
            if (D.stride_wts != 0) {
              // the four symbols of a word at once (K <= 6): clamp every byte to K - 1 (bit 7
              // of (b | 0x80) - K is set when b & 0x7F >= K; bytes >= 128 clamp too), then
              // the mixed-radix index m0 K^3 + m1 K^2 + m2 K + m3 as one byte dot product
#pragma unroll
              for (int g = 0; g < 4; ++g) {
                const uint32_t w = ws[g];
                const uint32_t over = (((w | 0x80808080u) - D.stride_krep) | w) & 0x80808080u;
                const uint32_t mask = (over >> 7) * 0xFFu;
                const uint32_t m = (w & ~mask) | (D.stride_kmrep & mask);
                const uint32_t e = stab[__dp4a(m, D.stride_wts, s * k4)];
                s = e & 31u;
                mu += e >> 5;
              }
            } else {
#pragma unroll
              for (int g = 0; g < 4; ++g) {
                const uint32_t w = ws[g];
                const uint32_t m0 = min(w & 0xFFu, km), m1 = min((w >> 8) & 0xFFu, km);
                const uint32_t m2 = min((w >> 16) & 0xFFu, km), m3 = min(w >> 24, km);
                const uint32_t e = stab[s * k4 + ((m0 * K + m1) * K + m2) * K + m3];
                s = e & 31u;
                mu += e >> 5;
              }
            }
          } else if (p.sparse_count) {
            // the largest state of the 16 steps says whether any was accepting (accepting
            // states are numbered last); only then is the vector replayed to count
            uint32_t mx = 0;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              s = tab.next(s, tab.col(byte_of(v[i], q)));
              mx = max(mx, s);
            }
            if (mx >= A) {
              uint32_t x = s0;
#pragma unroll
              for (int q = 0; q < 16; ++q) {
                x = tab.next(x, tab.col(byte_of(v[i], q)));
                mu += (x >= A);
              }
            }
          } else if (kBits && p.match_bits != nullptr) {
            // dense matches: the accepting steps of the vector as a 16-bit mask for the match
            // bitmap (stored once per block below)
            uint32_t mb = 0;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              s = tab.next(s, tab.col(byte_of(v[i], q)));
              mb |= (s >= A ? 1u : 0u) << q;
            }
            mu += __popc(mb);
            bmask |= (unsigned long long)mb << (16u * i);
          } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              s = tab.next(s, tab.col(byte_of(v[i], q)));
              mu += (s >= A);
            }
          }
          if (mu != mu0) {
            if (fv == kEmpty) {
              fv = col;
              fs = s0;
            }
            lvv = col;
            ls = s0;
            if (myslots != nullptr && nrec < kRowSlots) {
              // replay this vector to record its match positions (rare for sparse matches)
              uint32_t x = s0;
#pragma unroll
              for (int q = 0; q < 16; ++q) {
                x = tab.next(x, tab.col(byte_of(v[i], q)));
                if (x >= A) {
                  if (nrec < kRowSlots) myslots[nrec] = col + (uint32_t)q;
                  ++nrec;
                }
              }
            }
          }
          }
        }
      }
      if (kBits && p.match_bits != nullptr) {
        // bits [myrow * S + col0, + BOX) of the body: BOX-bit aligned (S and col0 are)
        const uint64_t bit0 = myrow * p.S + col0;
        if constexpr (BOX == 64) {
          reinterpret_cast<unsigned long long*>(p.match_bits)[bit0 / 64] = bmask;
        } else {
          p.match_bits[bit0 / 32] = (uint32_t)bmask;
        }
      }
    }
  }
  if (failed) return false;
  lv = (fv == kEmpty) ? 0u : lvv + 16u;
  if (run && last_row && p.tail) {
    // the tail after the last full row (16-byte aligned, shorter than a row) is on the critical
    // path of the scan: it is read 16 bytes at a time with the next vector's load in flight,
    // and its last partial vector by independent byte loads
    const uint8_t* tp = body + p.R * p.S;
    const uint32_t tl = (uint32_t)p.tail;
    const uint32_t full = tl & ~15u;
    uint4 nx = full ? ldg16(tp) : make_uint4(0, 0, 0, 0);
    for (uint32_t o = 0; o < tl; o += 16) {
      uint4 cur = nx;
      if (o + 16 < full) nx = ldg16(tp + o + 16);
      if (o >= full) {  // the last partial vector
        uint32_t wv[4] = {0, 0, 0, 0};
#pragma unroll
        for (uint32_t q = 0; q < 16; ++q)
          if (o + q < tl) wv[q >> 2] |= ldg8(tp + o + q) << (8 * (q & 3));
        cur = make_uint4(wv[0], wv[1], wv[2], wv[3]);
      }
      const uint32_t n_here = min(16u, tl - o);
      uint32_t tbits = 0;
#pragma unroll
      for (uint32_t q = 0; q < 16; ++q) {
        if (q < n_here) {
          const uint32_t s0 = s;
          s = tab.next(s, tab.col(byte_of(cur, (int)q)));
          if (s >= A) {
            ++mu;
            tbits |= 1u << q;
            const uint32_t at = (uint32_t)p.S + o + q;
            if (fv == kEmpty) {
              fv = at;
              fs = s0;
            }
            lvv = at;
            ls = s0;
            lv = lvv + 1;
            if (myslots != nullptr && nrec < kRowSlots) myslots[nrec] = lvv;
            ++nrec;
          }
        }
      }
      // bits [R * S + o, + 16) of the body (16-bit aligned)
      if (kBits && p.match_bits != nullptr)
        reinterpret_cast<uint16_t*>(p.match_bits)[(p.R * p.S + o) / 16] = (uint16_t)tbits;
    }
  }
  E = s;  // main end (assumes the row's start reaches my_sigma at my_t)
  return true;
}

// 5.-9. Resolve the chunk: row starts from the chunk's start state, the aggregate, the
// look-back for the exclusive prefix, the row records; false when a wait ran out.
template <int LAYOUT, int ESIZE>
__device__ __forceinline__ bool resolve_chunk(const ChunkCtx<LAYOUT, ESIZE>& C, const RowSpec& R,
                                              const RowMain& M) {
  // the match bitmap (dense emission) is never planned for the stride layouts: no code for it
  constexpr bool kBits = LAYOUT != kByteStride && LAYOUT != kClassPair;
  const uint32_t lane = C.lane;
  const DeviceDfa& D = C.p.dfa;
  const uint32_t dead = C.dead;
  const uint32_t A = C.A;
  const uint64_t row0 = C.row0;
  const uint64_t myrow = C.myrow;
  const bool active = C.active;
  const uint32_t nrows = C.nrows;
  const uint8_t* const body = C.body;
  const uint64_t rowlen = C.rowlen;
  const Tab<LAYOUT, ESIZE>& tab = C.tab;
  const ScanParams& p = C.p;
  const uint64_t j = C.j;
  auto cand_class = [&](uint64_t r) -> uint32_t { return C.cand_class(r); };
  auto& my_t = R.my_t;
  auto& my_sigma = R.my_sigma;
  auto& my_conv = R.my_conv;
  auto& head_cnt = R.head_cnt;
  auto& mu = M.mu;
  auto& fv = M.fv;
  auto& fs = M.fs;
  auto& lvv = M.lvv;
  auto& ls = M.ls;
  auto& lv = M.lv;
  auto& nrec = M.nrec;
  auto& E = M.E;
  // the match bitmap of row r (the merged prefix replays below write its bits [0, t))
  auto row_bits = [&](uint64_t r) -> uint16_t* {
    return kBits && p.match_bits != nullptr ? reinterpret_cast<uint16_t*>(p.match_bits) + (r * p.S) / 16 : nullptr;
  };
  // 5. the chunk's end state is known now if every row merged
  //    (or if at least its last row did: E_last does not depend on the chunk's start, and
  //    publishing it now keeps chunks with unmerged rows from forming a chain)
  const bool fast = __ballot_sync(kFull, active && !my_conv) == 0;
  const bool skip = (int64_t)j == p.skip_publish;
  const uint32_t E_last = __shfl_sync(kFull, E, nrows - 1);
  const bool last_merged = __shfl_sync(kFull, my_conv, nrows - 1) != 0;
  if (last_merged && lane == 0 && !skip) st_release(&p.status[j], pack_status(kFlagMapped, 0, E_last, 0));

  // rows k >= 1: start = end of row k-1 (fast path), count the merged prefix [0, t)
  uint32_t x_k = __shfl_up_sync(kFull, E, 1);
  uint32_t cnt_k = 0, dies_k = 0, pre_k = 0, died_pre = 0;
  if (fast && active && lane >= 1) {
    if (x_k == dead) {
      dies_k = 1;
      died_pre = 1;
    } else {
      const uint32_t y = run_range16(tab, body + myrow * p.S, my_t, x_k, dead, A, &pre_k, row_bits(myrow));
      if (y == dead) {
        dies_k = 1;
        died_pre = 1;
        cnt_k = pre_k;
      } else {
        if (y != my_sigma) set_error(p.result, kErrInternal);
        cnt_k = pre_k + mu;
        dies_k = (E == dead);
      }
    }
  }

  // 6. start state of the chunk: the end state published by chunk j-1
  uint32_t s_j = p.init_state;
  if (j > 0) {
    unsigned long long w = 0;
    if (lane == 0) {
      long long t0 = clock64();
      uint32_t seen = kEmpty;
      for (;;) {
        w = ld_acquire(&p.status[j - 1]);
        if ((w >> 62) != 0) break;
        if (read_error(p.result) || wait_expired(p.result, p.wait_budget, &t0, &seen)) {
          set_error(p.result, kErrTimeout);
          w = 0;
          break;
        }
      }
    }
    w = __shfl_sync(kFull, w, 0);
    if ((w >> 62) == 0) return false;  // failed: the error word is set
    s_j = (uint32_t)((w >> 45) & 0xFFFFu);
    if (s_j >= D.n) {  // never happens for a consistent status word; keep indices valid
      set_error(p.result, kErrInternal);
      s_j = 0;
    }
  }

  uint32_t E_chunk = E_last;
  if (fast) {
    if (lane == 0) {
      x_k = s_j;
      if (j == 0) {
        pre_k = 0;
        cnt_k = head_cnt + mu;
        dies_k = (E == dead);
      } else if (s_j == dead) {
        dies_k = 1;
        died_pre = 1;
        cnt_k = 0;
      } else {
        const uint32_t y = run_range16(tab, body + myrow * p.S, my_t, s_j, dead, A, &pre_k, row_bits(myrow));
        if (y == dead) {
          dies_k = 1;
          died_pre = 1;
          cnt_k = pre_k;
        } else {
          if (y != my_sigma) set_error(p.result, kErrInternal);
          cnt_k = pre_k + mu;
          dies_k = (E == dead);
        }
      }
    }
  } else {
    // slow path: walk the rows in order from s_j (lane 0 works, the lanes keep results); the
    // match bitmap words the lanes' main runs wrote are ordered before lane 0's prefix bits
    __syncwarp();
    uint32_t x = s_j;
    for (uint32_t k = 0; k < nrows; ++k) {
      const uint32_t tk = __shfl_sync(kFull, my_t, k);
      const uint32_t sk = __shfl_sync(kFull, my_sigma, k);
      const uint32_t Ek = __shfl_sync(kFull, E, k);
      const uint32_t muk = __shfl_sync(kFull, mu, k);
      const uint32_t ck = __shfl_sync(kFull, my_conv, k);
      const uint32_t hk = __shfl_sync(kFull, head_cnt, k);
      uint32_t cnt = 0, xin = x, pre = 0, dpre = 0;
      const uint64_t rr = row0 + k;
      if (p.serial_fallback && !ck && rr != 0 && x != dead) {
        // unmerged row: the warp runs the resolved start over the whole row
        x = warp_run_range16(tab, body + rr * p.S, p.S, x, dead, A, &cnt, lane);
        if (rr == p.R - 1 && p.tail && x != dead) x = run_bytes(tab, body + p.R * p.S, p.tail, x, dead, A, &cnt);
        if (lane == 0) atomicAdd(&p.result->progress, 1u);
      } else if (lane == 0) {
        const uint64_t r = rr;
        if (x == dead) {
          dpre = 1;
        } else if (r == 0) {
          cnt = hk + muk;
          x = Ek;
        } else if (ck) {
          const uint32_t y = run_range16(tab, body + r * p.S, tk, x, dead, A, &pre, row_bits(r));
          if (y == dead) {
            cnt = pre;
            dpre = 1;
            x = dead;
          } else {
            if (y != sk) set_error(p.result, kErrInternal);
            cnt = pre + muk;
            x = Ek;
          }
        } else {
          const uint32_t cls = cand_class(r);
          const uint32_t slot = D.rank[(uint64_t)cls * D.n + x];
          if (slot == kNoSlot) {
            set_error(p.result, kErrInternal);
            x = 0;  // any valid state: the call reports an error
          } else {
            cnt = p.slot_cnt[r * p.cand_stride + slot];
            x = p.slot_end[r * p.cand_stride + slot];
          }
        }
      }
      xin = __shfl_sync(kFull, xin, 0);
      cnt = __shfl_sync(kFull, cnt, 0);
      pre = __shfl_sync(kFull, pre, 0);
      dpre = __shfl_sync(kFull, dpre, 0);
      x = __shfl_sync(kFull, x, 0);
      if (lane == k) {
        x_k = xin;
        cnt_k = cnt;
        pre_k = pre;
        died_pre = dpre;
        dies_k = (x == dead);
      }
    }
    E_chunk = last_merged ? E_last : x;
    if (!last_merged && lane == 0 && !skip) st_release(&p.status[j], pack_status(kFlagMapped, 0, E_chunk, 0));
  }

  // 7. aggregate: counts up to and including the first row whose run dies
  const unsigned dmask = __ballot_sync(kFull, active && dies_k);
  const uint32_t first_dead = dmask ? (uint32_t)(__ffs(dmask) - 1) : 32u;
  uint64_t c = (active && lane <= first_dead) ? cnt_k : 0;
  uint64_t csum = c;
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) csum += __shfl_xor_sync(kFull, csum, d);
  const Pfx agg = {dmask ? 1u : 0u, csum};
  if (lane == 0 && !skip)
    st_release(&p.status[j], pack_status(kFlagAggregate, agg.dead, E_chunk, agg.count));


  // 8. decoupled look-back for the exclusive prefix
  Pfx ex = {0, 0};
  if (j > 0) {
    int64_t base = (int64_t)j - 1;
    bool ok = true;
    for (;;) {
      const int64_t idx = base - (int64_t)lane;
      unsigned long long w = 0;
      unsigned inc = 0;
      uint32_t limit = 31;
      long long t0 = clock64();
      uint32_t seen = kEmpty;
      for (;;) {
        w = idx >= 0 ? ld_acquire(&p.status[idx]) : ((unsigned long long)kFlagInclusive << 62);
        const uint32_t flag = (uint32_t)(w >> 62);
        inc = __ballot_sync(kFull, flag == kFlagInclusive);
        const unsigned notready = __ballot_sync(kFull, flag < kFlagAggregate);
        limit = inc ? (uint32_t)(__ffs(inc) - 1) : 31u;
        const unsigned need = limit == 31 ? kFull : ((1u << (limit + 1)) - 1u);
        if (!(notready & need)) break;
        bool stop = false;
        if (lane == 0) stop = read_error(p.result) || wait_expired(p.result, p.wait_budget, &t0, &seen);
        if (__shfl_sync(kFull, stop, 0)) {
          ok = false;
          break;
        }
      }
      if (!ok) break;
      Pfx v = {0, 0};
      if (lane <= limit) {
        v.dead = (uint32_t)((w >> 61) & 1u);
        v.count = w & kCountMask;
      }
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        Pfx o;
        o.dead = __shfl_down_sync(kFull, v.dead, d);
        o.count = __shfl_down_sync(kFull, v.count, d);
        if (lane + d < 32) v = pfx_op(o, v);
      }
      Pfx win;
      win.dead = __shfl_sync(kFull, v.dead, 0);
      win.count = __shfl_sync(kFull, v.count, 0);
      ex = pfx_op(win, ex);
      if (inc) break;
      base -= 32;
    }
    if (!ok) {
      set_error(p.result, kErrTimeout);
      return false;
    }
  }
  const Pfx inc = pfx_op(ex, agg);
  if (lane == 0 && !skip)
    st_release(&p.status[j], pack_status(kFlagInclusive, inc.dead, E_chunk, inc.count));

  // 9. per-row records for the emit pass: offset and the windows holding the matches
  if (p.segrec != nullptr) {
    const bool live_row = active && !ex.dead && lane <= first_dead;
    const uint64_t rc = live_row ? cnt_k : 0;
    uint64_t incl = rc;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t o = __shfl_up_sync(kFull, incl, d);
      if (lane >= (uint32_t)d) incl += o;
    }
    if (active) {
      SegRec sr;
      sr.x = live_row ? x_k : dead;
      sr.count = (uint32_t)rc;
      sr.offset = ex.count + incl - rc;
      sr.flags = 0;
      sr.t = 0;
      sr.pre = 0;
      sr.lvv = kEmpty;
      sr.ls = 0;
      if (!my_conv) {
        // slot-map row: no merged run, replay the whole row from its start
        sr.fv = 0;
        sr.fs = x_k;
        sr.lv = (uint32_t)rowlen;
      } else {
        if (myrow == 0 && head_cnt > 0) {
          sr.flags |= kHeadFlag;
          sr.pre = head_cnt;
        } else if (pre_k > 0) {
          sr.flags |= kPreFlag;
          sr.t = my_t;
          sr.pre = pre_k;
        }
        // main-run window (empty when the run died inside the prefix)
        const bool main_live = !died_pre && mu > 0;
        sr.fv = (main_live && fv != kEmpty) ? fv : 0u;
        sr.fs = fs;
        sr.lv = main_live ? lv : 0u;
        sr.lvv = main_live ? lvv : kEmpty;
        sr.ls = ls;
        // every main-run match was recorded by pass 1: the emit pass only copies them
        if (main_live && p.slots != nullptr && nrec == mu && mu <= kRowSlots) sr.flags |= kSlotsFlag;
        // or every match of the row is in the match bitmap: the prefix [0, t) replayed from the
        // row's true start wrote its bits, the main run the rest (a run that died inside the
        // prefix is replayed by the emit pass instead)
        if (!died_pre && kBits && p.match_bits != nullptr) sr.flags |= kBitsFlag;
      }
      p.segrec[myrow] = sr;
    }
  }
  if (j == p.n_chunks - 1 && lane == 0) {
    p.result->final_state = inc.dead ? dead : E_chunk;
    p.result->count = inc.count;
    if (p.early != nullptr) write_early(p.early, inc.dead ? dead : E_chunk, inc.count, read_error(p.result));
  }
  return true;
}

// One chunk of 32 rows (row k on lane k) by one warp: Algorithm 1 per row.  The rows'
// candidate sets (the states entered on the byte that ends the previous row) are run until
// they merge (steps 1-3); each lane then runs its merged state over the rest of its row
// (step 4); the chunk's start state from chunk j - 1 fixes every row's true start, the merged
// prefixes are counted, and the chunk publishes its aggregate and inclusive prefix for the
// look-back of later chunks (steps 5-9).
template <int LAYOUT, int ESIZE, int P>
__device__ __forceinline__ void scan_chunk(WarpCtx& wc, const Tab<LAYOUT, ESIZE>& tab, const ScanParams& p,
                                           const CUtensorMap* tmap, const uint64_t j) {
#if PAREM_PHASE_STATS
  const uint32_t clk0 = (uint32_t)clock64();
#endif
  ChunkCtx<LAYOUT, ESIZE> C(wc, tab, p, tmap, j);
  RowSpec R;
  chunk_begin(C, R);
  find_sync_byte(C, R);
  if constexpr (P == 1) {
    speculate_grouped(C, R);
  } else {
    speculate_warp<LAYOUT, ESIZE, P>(C, R);
    speculate_lanes<LAYOUT, ESIZE, P>(C, R);
  }
  record_convergence(C, R);
  run_slot_maps(C, R);
#if PAREM_PHASE_STATS
  const uint32_t clk1 = (uint32_t)clock64();
#endif
  RowMain M;
  if (!main_run(C, R, M)) return;
#if PAREM_PHASE_STATS
  const uint32_t clk2 = (uint32_t)clock64();
#endif
  if (!resolve_chunk(C, R, M)) return;
#if PAREM_PHASE_STATS
  if (C.lane == 0) {
    // 32-bit cycle differences (a chunk takes far less than 2^32 cycles)
    wc.cyc[0] += clk1 - clk0;
    wc.cyc[1] += clk2 - clk1;
    wc.cyc[2] += (uint32_t)clock64() - clk2;
  }
#endif
}

// Wait (bounded) for stages still in flight before the CTA may release its shared memory.
__device__ __forceinline__ void drain_stages(const WarpCtx& wc, uint64_t budget) {
  for (uint32_t b = 0; b < kStages; ++b) {
    if (wc.pending & (1u << b)) {
      const uint32_t bar = smem_u32(wc.sm + wc.bar0 + 8 * b);
      const long long t0 = clock64();
      while (!mbar_try_wait(bar, (wc.phase_bits >> b) & 1u)) {
        if ((uint64_t)(clock64() - t0) > budget) break;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Pass 1: speculation, main run, look-back.  P = candidate registers per lane when one row
// is speculated by the whole warp (32 * P candidates); with P == 1, p.group lanes per row.
// ---------------------------------------------------------------------------------------
// The last block of a kernel to finish copies the result word to the host-mapped copy the
// host reads after the stream synchronises (no separate device-to-host copy).  Every block
// counts itself done after a fence, so the last one sees every block's result updates.
__device__ __forceinline__ void publish_result(const ScanParams& p, uint32_t* done) {
  if (p.host_result == nullptr) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(done, 1u) == gridDim.x - 1) {
      __threadfence();
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(p.result);
      volatile unsigned long long* dst = reinterpret_cast<volatile unsigned long long*>(p.host_result);
      for (uint32_t i = 0; i < sizeof(DevResult) / 8; ++i) dst[i] = __ldcg(src + i);
    }
  }
}

// Zero the previous scan's header region (its ticket, result and status words), which the
// next scan on the stream reuses; every thread of the grid takes a strided share.
__device__ __forceinline__ void clear_prev_header(const ScanParams& p) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.clear_n16; i += stride)
    p.clear[i] = make_uint4(0, 0, 0, 0);
}

// Threads per block the pass-1 kernel is compiled for: the pair variant's tables leave room
// for at most kPairMaxWarps warps, so it gets the registers of 512 threads.
template <int LAYOUT, int P>
constexpr int spec_scan_threads() {
  return LAYOUT == kClassPair ? (int)(kPairMaxWarps * 32) : (P >= 4 ? 768 : 1024);
}

template <int LAYOUT, int ESIZE, int P>
__global__ void __launch_bounds__(spec_scan_threads<LAYOUT, P>(), 1)
    k_spec_scan(const __grid_constant__ CUtensorMap tmap, const ScanParams p) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  uint8_t* const sm = smem_raw;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  clear_prev_header(p);
  load_tables<LAYOUT, ESIZE>(sm, p.dfa);
  const uint32_t region = stage_region_off(smem_raw, Tab<LAYOUT, ESIZE>::kGlobal ? 0u : p.smem_table_bytes);
  constexpr uint32_t SB = kLanes * box_bytes(LAYOUT);  // bytes of one stage
  WarpCtx wc;
  wc.sm = sm;
  wc.lane = lane;
  wc.stage0 = region + warp * (kStages * SB);
  wc.bar0 = region + nwarps * (kStages * SB) + warp * (kStages * 8);
  const uint32_t spec0 = region + nwarps * (kStages * SB + kStages * 8) + warp * p.spec_bytes;
  wc.hand = reinterpret_cast<uint16_t*>(sm + spec0);
  wc.cbuf = reinterpret_cast<uint32_t*>(sm + spec0 + kLanes * kLaneCand * 2);
  // 2 x bitmap_words words of candidate bitmaps, then a list of up to 256 states
  wc.bitmaps = reinterpret_cast<uint32_t*>(sm + spec0 + kSpecBytes);
  wc.phase_bits = 0;
  wc.pending = 0;
  wc.cyc = reinterpret_cast<unsigned long long*>(sm + spec0 + kLanes * kLaneCand * 2 + kLanes * 4);
  if (lane == 0)
    for (int i = 0; i < 5; ++i) wc.cyc[i] = 0;
  if (lane == 0) {
    for (uint32_t s = 0; s < kStages; ++s) mbar_init(smem_u32(sm + wc.bar0 + 8 * s), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  Tab<LAYOUT, ESIZE> tab;
  tab.sm = sm;
  tab.gtable = p.dfa.table;
  tab.rowbytes = p.dfa.rowbytes;
  tab.set_win(p.dfa.win);
  for (;;) {
    uint32_t ticket = 0;
    if (lane == 0) ticket = read_error(p.result) ? 0xFFFFFFFFu : atomicAdd(p.ticket, 1u);
    ticket = __shfl_sync(kFull, ticket, 0);
    if ((uint64_t)ticket >= p.n_chunks) break;
    scan_chunk<LAYOUT, ESIZE, P>(wc, tab, p, &tmap, ticket);
  }
  flush_cycles(wc, p.result);
  drain_stages(wc, p.wait_budget);
  publish_result(p, p.ticket + kDoneScanWord);
}


// ---------------------------------------------------------------------------------------
// Emit pass: one thread per row with matches.  It first replays the first and the last
// matching vectors; when that does not account for every match of the row, it replays the
// whole window [fv, lv) instead.  Positions are written at the row's offset.
// ---------------------------------------------------------------------------------------
template <int LAYOUT, int ESIZE>
__device__ __forceinline__ void emit_range(const Tab<LAYOUT, ESIZE>& tab, const ScanParams& p, uint64_t r,
                                           uint32_t from, uint32_t to, uint32_t& x, uint64_t& o,
                                           uint64_t end) {
  const uint8_t* rowp = p.text + p.h + r * p.S;
  const uint64_t gbase = p.h + r * p.S;
  const uint32_t A = p.dfa.first_accept;
  uint64_t off = from;
  // aligned whole vectors inside the row, with the next vector's load in flight: the steps
  // of a vector collect a 16-bit mask of accepting positions, written after the vector
  // (one store per match instead of a predicated store at every byte)
  if ((off & 15u) == 0 && off + 16 <= p.S && off + 16 <= to) {
    // two vectors in flight ahead of the one consumed (a replay is a single dependent chain
    // per thread: the loads must cover the memory latency on their own)
    const uint4 zero = make_uint4(0, 0, 0, 0);
    uint4 nxt = ldg16(rowp + off);
    uint4 nxt2 = (off + 32 <= p.S && off + 32 <= to) ? ldg16(rowp + off + 16) : zero;
    while (off + 16 <= p.S && off + 16 <= to && o < end) {
      const uint4 v = nxt;
      nxt = nxt2;
      if (off + 48 <= p.S && off + 48 <= to) nxt2 = ldg16(rowp + off + 32);
      uint32_t m = 0;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        x = tab.next(x, tab.col(byte_of(v, i)));
        m |= (x >= A ? 1u : 0u) << i;
      }
      const uint64_t pb = p.pos_base + gbase + off;
      while (m != 0 && o < end) {
        p.positions[o++] = pb + (uint64_t)(__ffs(m) - 1);
        m &= m - 1u;
      }
      off += 16;
    }
  }
  while (off < to && o < end) {
    if ((off & 15u) == 0 && off + 16 <= p.S && off + 16 <= to) {
      const uint4 v = ldg16(rowp + off);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        x = tab.next(x, tab.col(byte_of(v, i)));
        if (x >= A && o < end) p.positions[o++] = p.pos_base + gbase + off + (uint64_t)i;
      }
      off += 16;
    } else {
      x = tab.next(x, tab.col(ldg8(rowp + off)));
      if (x >= A) p.positions[o++] = p.pos_base + gbase + off;
      off += 1;
    }
  }
}

// The positions of row r of one text (see k_emit).
template <int LAYOUT, int ESIZE>
__device__ __forceinline__ void emit_row(const Tab<LAYOUT, ESIZE>& tab, const ScanParams& p, uint64_t r) {
  const uint32_t A = p.dfa.first_accept;
  const SegRec sr = p.segrec[r];
  if (sr.count == 0 || sr.offset >= p.capacity) return;
  const uint64_t end = (sr.offset + sr.count < p.capacity) ? sr.offset + sr.count : p.capacity;
  uint64_t o = sr.offset;
  if (sr.flags & kHeadFlag) {
    // row 0: the unaligned head bytes before the first full row
    uint32_t x = sr.x;
    for (uint64_t i = 0; i < p.h && o < end; ++i) {
      x = tab.next(x, tab.col(ldg8(p.text + i)));
      if (x >= A) p.positions[o++] = p.pos_base + i;
    }
  }
  if (sr.flags & kBitsFlag) return;  // the rest of the row comes from the match bitmap (k_emit_bits)
  if (!(sr.flags & kHeadFlag) && (sr.flags & kPreFlag)) {
    // matches inside the merged prefix [0, t), replayed from the row's true start
    uint32_t x = sr.x;
    emit_range(tab, p, r, 0u, sr.t, x, o, end);
  }
  if (o >= end || sr.lv == 0) return;
  if (sr.flags & kSlotsFlag) {
    // pass 1 recorded every main-run match of this row
    const uint64_t gbase = p.h + r * p.S;
    const uint32_t* sl = p.slots + r * kRowSlots;
    for (uint32_t i = 0; o < end; ++i) p.positions[o++] = p.pos_base + gbase + sl[i];
    return;
  }
  atomicAdd(&p.result->emit_replays, 1u);
  atomicMax(&p.result->emit_max_window, sr.lv - sr.fv);
  const uint64_t o_main = o;
  uint32_t x = sr.fs;
  if (sr.lvv != kEmpty && sr.lvv > sr.fv) {
    // fast replay: the first matching vector, then the last one
    const uint32_t first_end = sr.fv + 16 <= sr.lvv ? sr.fv + 16 : sr.lvv;
    emit_range(tab, p, r, sr.fv, first_end, x, o, end);
    uint32_t y = sr.ls;
    emit_range(tab, p, r, sr.lvv, sr.lv, y, o, end);
    if (o == end) return;
    // matches lie between the two vectors: replay the whole window
    o = o_main;
    x = sr.fs;
  }
  emit_range(tab, p, r, sr.fv, sr.lv, x, o, end);
}

template <int LAYOUT, int ESIZE>
__global__ void __launch_bounds__(1024) k_emit(const ScanParams p) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  uint8_t* const sm = smem_raw;
  const DeviceDfa& D = p.dfa;
  // The table is staged only by blocks with a row to replay: rows whose matches pass 1
  // recorded are copied (sparse texts: nearly all of them), so most blocks never read it.
  bool replay = false;
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < p.R;
       r += (uint64_t)gridDim.x * blockDim.x) {
    const SegRec& sr = p.segrec[r];
    replay = replay || (sr.count > 0 && sr.offset < p.capacity &&
                        ((sr.flags & kHeadFlag) ||
                         (!(sr.flags & kBitsFlag) && ((sr.flags & kPreFlag) || (!(sr.flags & kSlotsFlag) && sr.lv > 0)))));
  }
  if (__syncthreads_or(replay)) {
    load_tables<LAYOUT, ESIZE>(sm, D);
    __syncthreads();
  }
  Tab<LAYOUT, ESIZE> tab;
  tab.sm = sm;
  tab.gtable = D.table;
  tab.rowbytes = D.rowbytes;
  tab.set_win(p.dfa.win);
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < p.R;
       r += (uint64_t)gridDim.x * blockDim.x)
    emit_row<LAYOUT, ESIZE>(tab, p, r);
  publish_result(p, p.ticket + kDoneEmitWord);
}

// Dense emission, streamed: warps take chunk tickets as in pass 1 and the chunk's rows arrive
// through the same TMA stages; each lane replays its row's match window [fv, lv) from the
// state pass 1 recorded at fv, collecting per 16-byte vector a mask of accepting steps from
// which it writes positions at the row's offset.  The head or merged-prefix matches (before
// the window) and the last row's tail (after the last full row) are replayed from global
// memory by the lane; rows whose matches pass 1 recorded are copied.
template <int LAYOUT, int ESIZE>
__global__ void __launch_bounds__(1024, 1)
    k_emit_stream(const __grid_constant__ CUtensorMap tmap, const ScanParams p) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  uint8_t* const sm = smem_raw;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  load_tables<LAYOUT, ESIZE>(sm, p.dfa);
  const uint32_t region = stage_region_off(smem_raw, Tab<LAYOUT, ESIZE>::kGlobal ? 0u : p.smem_table_bytes);
  WarpCtx wc;
  wc.sm = sm;
  wc.lane = lane;
  wc.stage0 = region + warp * (kStages * kStageBytes);
  wc.bar0 = region + nwarps * (kStages * kStageBytes) + warp * (kStages * 8);
  wc.phase_bits = 0;
  wc.pending = 0;
  // per lane kEmitBuf u16 positions (relative to the warp's base column), lane-major
  uint16_t* const buf = reinterpret_cast<uint16_t*>(
      sm + region + nwarps * (kStages * kStageBytes + kStages * 8) + warp * (kLanes * kEmitBuf * 2)) + lane * kEmitBuf;
  if (lane == 0) {
    for (uint32_t b = 0; b < kStages; ++b) mbar_init(smem_u32(sm + wc.bar0 + 8 * b), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  Tab<LAYOUT, ESIZE> tab;
  tab.sm = sm;
  tab.gtable = p.dfa.table;
  tab.rowbytes = p.dfa.rowbytes;
  tab.set_win(p.dfa.win);
  const uint32_t A = p.dfa.first_accept;
  const uint32_t nblk = (uint32_t)(p.S / kBox);
  uint32_t* const tickets = p.ticket + kEmitTicketWord;
  uint16_t* const wbuf = buf - lane * kEmitBuf;  // the warp's buffers
  bool failed = false;
  for (;;) {
    uint32_t ticket = 0;
    if (lane == 0) ticket = read_error(p.result) ? 0xFFFFFFFFu : atomicAdd(tickets, 1u);
    ticket = __shfl_sync(kFull, ticket, 0);
    if ((uint64_t)ticket >= p.n_chunks) break;
    const uint64_t row0 = (uint64_t)ticket * kLanes;
    const uint64_t r = row0 + lane;
    // this lane's window [fv, lv) with its state x and output range [o, end)
    uint32_t fv = kEmpty, lv = 0, x = 0;
    uint64_t o = 0, end = 0;
    if (r < p.R) {
      const SegRec sr = p.segrec[r];
      if (sr.count > 0 && sr.offset < p.capacity) {
        end = (sr.offset + sr.count < p.capacity) ? sr.offset + sr.count : p.capacity;
        o = sr.offset;
        if (sr.flags & kHeadFlag) {
          uint32_t y = sr.x;
          for (uint64_t i = 0; i < p.h && o < end; ++i) {
            y = tab.next(y, tab.col(ldg8(p.text + i)));
            if (y >= A) p.positions[o++] = p.pos_base + i;
          }
        } else if (sr.flags & kPreFlag) {
          uint32_t y = sr.x;
          emit_range(tab, p, r, 0u, sr.t, y, o, end);
        }
        if (o < end && sr.lv > 0) {
          if (sr.flags & kSlotsFlag) {
            const uint64_t gbase = p.pos_base + p.h + r * p.S;
            const uint32_t* sl = p.slots + r * kRowSlots;
            for (uint32_t i = 0; o < end; ++i) p.positions[o++] = gbase + sl[i];
          } else {
            fv = sr.fv;
            lv = sr.lv;
            x = sr.fs;
          }
        }
      }
    }
    // the blocks that hold some lane's window inside the full rows
    uint32_t fmin = fv, lmax = (fv == kEmpty) ? 0u : lv;
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
      fmin = min(fmin, __shfl_xor_sync(kFull, fmin, d));
      lmax = max(lmax, __shfl_xor_sync(kFull, lmax, d));
    }
    if (fmin == kEmpty) continue;
    const uint32_t b0 = fmin / kBox;
    const uint32_t b1 = min((lmax + kBox - 1) / kBox, nblk);
    const uint32_t in_row_end = min(lv, (uint32_t)p.S);
    // Positions are collected per lane in shared memory and written by the whole warp one
    // lane's run at a time (consecutive addresses, full sectors) instead of one scattered
    // 8-byte store per position: flushed when a lane has no room for another vector's, or
    // when the columns would no longer fit 16 bits above the warp's base column.
    const uint64_t rowbase = p.pos_base + p.h + r * p.S;
    uint32_t cnt = 0, base = b0 * kBox;
    auto flush = [&]() {
      __syncwarp();  // every lane's buffer writes are visible to the warp
      for (uint32_t src = 0; src < kLanes; ++src) {
        const uint32_t n = __shfl_sync(kFull, cnt, src);
        if (n == 0) continue;
        const uint64_t os = __shfl_sync(kFull, o, src);
        const uint64_t vb = __shfl_sync(kFull, rowbase, src) + base;
        if (lane < n) p.positions[os + lane] = vb + wbuf[src * kEmitBuf + lane];
      }
      __syncwarp();
      o += cnt;
      cnt = 0;
    };
    if (b0 < b1) {
      const uint32_t nb = b1 - b0;
      const uint32_t first = nb < kStages ? nb : kStages;
      if (lane == 0) {
        for (uint32_t k = 0; k < first; ++k) {
          const uint32_t bar = smem_u32(sm + wc.bar0 + 8 * k);
          mbar_arrive_expect_tx(bar, kStageBytes);
          tma_load_2d(smem_u32(sm + wc.stage0 + k * kStageBytes), &tmap, bar, (int32_t)((b0 + k) * kBox),
                      (int32_t)row0);
        }
      }
      wc.pending |= (1u << first) - 1u;
      for (uint32_t k = 0; k < nb; ++k) {
        const uint32_t b = k % kStages;
        const uint32_t bar = smem_u32(sm + wc.bar0 + 8 * b);
        if (!stage_wait(bar, (wc.phase_bits >> b) & 1u, p.wait_budget, p.result)) {
          set_error(p.result, kErrTimeout);
          failed = true;
          break;
        }
        wc.phase_bits ^= 1u << b;
        wc.pending &= ~(1u << b);
        uint4 v[kBox / 16];
        const uint8_t* stg = sm + wc.stage0 + b * kStageBytes + lane * kBox;
#pragma unroll
        for (uint32_t i = 0; i < kBox / 16; ++i)
          v[i] = *reinterpret_cast<const uint4*>(stg + ((i ^ ((lane >> 1) & 3u)) * 16u));
        __syncwarp();
        if (k + kStages < nb) {
          if (lane == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive_expect_tx(bar, kStageBytes);
            tma_load_2d(smem_u32(sm + wc.stage0 + b * kStageBytes), &tmap, bar, (int32_t)((b0 + k + kStages) * kBox),
                        (int32_t)row0);
          }
          wc.pending |= 1u << b;
        }
        const uint32_t col0 = (b0 + k) * kBox;
        if (col0 + kBox - base > 0xFFFFu) {  // warp-uniform
          flush();
          base = col0;
        }
#pragma unroll
        for (uint32_t i = 0; i < kBox / 16; ++i) {
          const uint32_t col = col0 + i * 16u;
          if (col >= fv && col + 16u <= in_row_end && o + cnt < end) {
            uint32_t m = 0;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              x = tab.next(x, tab.col(byte_of(v[i], q)));
              m |= (x >= A ? 1u : 0u) << q;
            }
            const uint32_t rel = col - base;
            while (m != 0 && o + cnt < end) {
              buf[cnt++] = (uint16_t)(rel + (uint32_t)(__ffs(m) - 1));
              m &= m - 1u;
            }
          }
          if (__any_sync(kFull, cnt > kEmitBuf - 16)) flush();
        }
      }
      flush();
      if (failed) break;
    }
    // the last row's window past the last full row (its tail)
    if (fv != kEmpty && lv > p.S && o < end) {
      const uint32_t from = fv > (uint32_t)p.S ? fv : (uint32_t)p.S;
      emit_range(tab, p, r, from, lv, x, o, end);
    }
  }
  drain_stages(wc, p.wait_budget);
  publish_result(p, p.ticket + kDoneEmitWord);
}

// Dense emission from the match bitmap of pass 1: one warp per row whose matches are all in
// the bitmap, without the transition table (so more warps fit an SM).  1,024 bytes of the row
// at a time, every lane takes 32 bits of the bitmap and writes its positions (relative to
// the round, 16 bits each) into a per-warp buffer in shared memory at its scan offset -- two
// bits per step, the lowest from the front and the highest from the back -- and the warp
// writes the buffer in order with consecutive addresses.  k_emit runs after it for what
// needs the table: row 0's head bytes (before the aligned body, outside the bitmap; their
// positions come first, so this kernel starts row 0 after them) and the rows without bits
// (a run that died inside its merged prefix, or speculation that never merged).
constexpr uint32_t kEmitBitsWarps = 16;    // warps per block of k_emit_bits
constexpr uint32_t kEmitBitsRound = 1024;  // row bytes per round (32 lanes x 32 bits)

static __global__ void __launch_bounds__(kEmitBitsWarps * 32, 4) k_emit_bits(const ScanParams p) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint16_t* const buf = reinterpret_cast<uint16_t*>(smem_raw) + warp * kEmitBitsRound;
  const uint32_t* bits32 = p.match_bits;
  const uint64_t step = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t r = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp; r < p.R; r += step) {
    const SegRec sr = p.segrec[r];
    if (sr.count == 0 || sr.offset >= p.capacity || !(sr.flags & kBitsFlag)) continue;
    const uint64_t end = (sr.offset + sr.count < p.capacity) ? sr.offset + sr.count : p.capacity;
    uint64_t o = sr.offset + ((sr.flags & kHeadFlag) ? sr.pre : 0u);
    const uint32_t rowlen = (uint32_t)(p.S + (r == p.R - 1 ? p.tail : 0));
    const uint64_t rword = (r * p.S) / 32;              // bitmap word of the row's first byte
    const uint64_t gpos = p.pos_base + p.h + r * p.S;   // text position of the row's first byte
    // the next round's bits are loaded while this round's positions are written
    auto load_bits = [&](uint32_t at) -> uint32_t {
      if (at >= rowlen) return 0u;
      uint32_t m = bits32[rword + at / 32];
      if (rowlen - at < 32u) m &= (1u << (rowlen - at)) - 1u;
      return m;
    };
    uint32_t m_next = load_bits(32u * lane);
    for (uint32_t base = 0; base < rowlen && o < end; base += kEmitBitsRound) {
      uint32_t m = m_next;
      m_next = load_bits(base + kEmitBitsRound + 32u * lane);
      const uint32_t c = __popc(m);
      uint32_t incl = c;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, d);
        if (lane >= (uint32_t)d) incl += y;
      }
      const uint32_t total = __shfl_sync(kFull, incl, 31);
      uint32_t lo = incl - c, hi = incl;
      const uint32_t rel = 32u * lane;
      while (m != 0u) {
        buf[lo++] = (uint16_t)(rel + (uint32_t)(__ffs(m) - 1));
        m &= m - 1u;
        if (m != 0u) {
          const uint32_t qh = 31u - (uint32_t)__clz(m);
          buf[--hi] = (uint16_t)(rel + qh);
          m ^= 1u << qh;
        }
      }
      __syncwarp();
      const uint64_t rb = gpos + base;
      const uint32_t lim = (uint32_t)(end - o < total ? end - o : total);
      for (uint32_t i = lane; i < lim; i += 32) p.positions[o + i] = rb + buf[i];
      __syncwarp();
      o += total;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Texts too short for one row: a single thread runs the plain loop on the device.
// ---------------------------------------------------------------------------------------
template <int LAYOUT, int ESIZE>
__global__ void k_tiny(const ScanParams p) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  uint8_t* const sm = smem_raw;
  const DeviceDfa& D = p.dfa;
  clear_prev_header(p);
  load_tables<LAYOUT, ESIZE>(sm, D);
  __syncthreads();
  if (threadIdx.x != 0) return;
  Tab<LAYOUT, ESIZE> tab;
  tab.sm = sm;
  tab.gtable = D.table;
  tab.rowbytes = D.rowbytes;
  tab.set_win(p.dfa.win);
  uint32_t x = p.init_state;
  uint64_t cnt = 0;
  for (uint64_t i = 0; i < p.n; ++i) {
    if (x == D.dead) break;
    x = tab.next(x, tab.col(ldg8(p.text + i)));
    if (x >= D.first_accept) {
      if (p.positions && cnt < p.capacity) p.positions[cnt] = p.pos_base + i;
      ++cnt;
    }
  }
  p.result->final_state = x;
  p.result->count = cnt;
  if (p.host_result != nullptr) {  // one block, one thread: it wrote the word itself
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(p.result);
    volatile unsigned long long* dst = reinterpret_cast<volatile unsigned long long*>(p.host_result);
    for (uint32_t i = 0; i < sizeof(DevResult) / 8; ++i) dst[i] = src[i];
  }
}

#ifdef PAREM_BATCH_KERNELS  // compiled in parem_k_batch.cu only
// ---------------------------------------------------------------------------------------
// Batch: many (text, DFA) items in one persistent launch.  Each CTA serves one slot (DFA) at
// a time: it stages that DFA's tables once, its warps take the slot's chunk tickets (the
// chunks of all the slot's items in order), and when the slot runs dry the CTA moves to
// another slot that still has chunks.  Within a slot the chunk protocol is the one of
// k_spec_scan, per item.
// ---------------------------------------------------------------------------------------
// One chunk of a batch item, with the slot's table tier (shared memory or global) and
// speculation form (grouped, or warp-wide over P registers) fixed at compile time.  Not
// inlined: each form gets its own register allocation under the kernel's launch bound.
template <int LAYOUT, int P>
__device__ __noinline__ void batch_chunk(WarpCtx& wc, uint8_t* sm, const BatchSlot& S, const BatchItem& it,
                                         uint64_t j) {
  Tab<LAYOUT, 2> tab;
  tab.sm = sm;
  tab.gtable = S.dfa.table;
  tab.rowbytes = S.dfa.rowbytes;
  tab.set_win(0);
  scan_chunk<LAYOUT, 2, P>(wc, tab, it.p, &it.tmap, j);
}

// THREADS: 768 (24 warps at 80 registers) or 512 (16 warps at 128 registers).
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1) k_batch_scan(const __grid_constant__ BatchParams bp) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  __shared__ uint32_t s_next;
  uint8_t* const sm = smem_raw;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const uint32_t region = stage_region_off(smem_raw, bp.max_table_smem);
  WarpCtx wc;
  wc.sm = sm;
  wc.lane = lane;
  wc.stage0 = region + warp * (kStages * kStageBytes);
  wc.bar0 = region + nwarps * (kStages * kStageBytes) + warp * (kStages * 8);
  const uint32_t spec0 = region + nwarps * (kStages * kStageBytes + kStages * 8) + warp * bp.spec_bytes;
  wc.hand = reinterpret_cast<uint16_t*>(sm + spec0);
  wc.cbuf = reinterpret_cast<uint32_t*>(sm + spec0 + kLanes * kLaneCand * 2);
  wc.bitmaps = reinterpret_cast<uint32_t*>(sm + spec0 + kSpecBytes);
  wc.phase_bits = 0;
  wc.pending = 0;
  wc.cyc = reinterpret_cast<unsigned long long*>(sm + spec0 + kLanes * kLaneCand * 2 + kLanes * 4);
  if (lane == 0)
    for (int i = 0; i < 5; ++i) wc.cyc[i] = 0;
  if (lane == 0) {
    for (uint32_t s = 0; s < kStages; ++s) mbar_init(smem_u32(sm + wc.bar0 + 8 * s), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  uint32_t slot = bp.cta_slot[blockIdx.x];
  while (slot < bp.n_slots) {
    const BatchSlot& S = bp.slots[slot];
    load_tables_dyn(sm, S.dfa, S.smem_tier);
    __syncthreads();
    for (;;) {
      uint32_t ticket = 0;
      if (lane == 0) ticket = atomicAdd(S.ticket, 1u);
      ticket = __shfl_sync(kFull, ticket, 0);
      if ((uint64_t)ticket >= S.n_chunks) break;
      // the item that owns this chunk: the last one whose first ticket is <= ticket
      uint32_t lo = S.item_begin, hi = S.item_end - 1;
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) / 2;
        if (bp.items[mid].chunk_base <= ticket) lo = mid; else hi = mid - 1;
      }
      const BatchItem& it = bp.items[lo];
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&it.tmap) : "memory");
      const uint64_t j = ticket - it.chunk_base;
      if (S.smem_tier) {
        if (S.grouped)
          batch_chunk<kBatchDyn, 1>(wc, sm, S, it, j);
        else
          batch_chunk<kBatchDyn, 8>(wc, sm, S, it, j);
      } else {
        if (S.grouped)
          batch_chunk<kBatchGlobal, 1>(wc, sm, S, it, j);
        else
          batch_chunk<kBatchGlobal, 8>(wc, sm, S, it, j);
      }
      flush_cycles(wc, it.p.result);  // items differ from chunk to chunk
    }
    __syncthreads();  // every warp is done with this slot's tables
    if (threadIdx.x == 0) {
      uint32_t nx = 0xFFFFFFFFu;
      for (uint32_t k = 1; k <= bp.n_slots; ++k) {
        const uint32_t c = (slot + k) % bp.n_slots;
        if ((uint64_t)*reinterpret_cast<volatile uint32_t*>(bp.slots[c].ticket) < bp.slots[c].n_chunks) {
          nx = c;
          break;
        }
      }
      s_next = nx;
    }
    __syncthreads();
    slot = s_next;
  }
  drain_stages(wc, bp.wait_budget);
}

// Batch emit: each CTA handles 256 rows of one slot's items.
__global__ void __launch_bounds__(256) k_batch_emit(const __grid_constant__ BatchParams bp) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  uint8_t* const sm = smem_raw;
  const uint32_t slot = bp.emit_slot[blockIdx.x];
  const BatchSlot& S = bp.slots[slot];
  load_tables_dyn(sm, S.dfa, S.smem_tier);
  __syncthreads();
  const uint64_t rr = bp.emit_row0[blockIdx.x] + threadIdx.x;
  if (rr >= S.n_rows) return;
  uint32_t lo = S.item_begin, hi = S.item_end - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) / 2;
    if (bp.items[mid].row_base <= rr) lo = mid; else hi = mid - 1;
  }
  const BatchItem& it = bp.items[lo];
  if (it.p.segrec == nullptr || it.p.R == 0) return;
  if (S.smem_tier) {
    Tab<kBatchDyn, 2> tab;
    tab.sm = sm;
    tab.gtable = S.dfa.table;
    tab.rowbytes = S.dfa.rowbytes;
    emit_row<kBatchDyn, 2>(tab, it.p, rr - it.row_base);
  } else {
    Tab<kBatchGlobal, 2> tab;
    tab.sm = sm;
    tab.gtable = S.dfa.table;
    tab.rowbytes = S.dfa.rowbytes;
    emit_row<kBatchGlobal, 2>(tab, it.p, rr - it.row_base);
  }
}

// Batch items too short for one row: one thread per item.
__global__ void k_batch_tiny(const __grid_constant__ BatchParams bp, const uint32_t* tiny_items, uint32_t n_tiny) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tiny) return;
  const BatchItem& it = bp.items[tiny_items[t]];
  const ScanParams& p = it.p;
  const DeviceDfa& D = p.dfa;
  uint32_t x = p.init_state;
  uint64_t cnt = 0;
  for (uint64_t i = 0; i < p.n; ++i) {
    if (x == D.dead) break;
    const uint32_t c = *reinterpret_cast<const uint16_t*>(D.colmap + 2 * ldg8(p.text + i));
    x = __ldg(reinterpret_cast<const uint16_t*>(D.table + x * D.rowbytes + c));
    if (x >= D.first_accept) {
      if (p.positions && cnt < p.capacity) p.positions[cnt] = p.pos_base + i;
      ++cnt;
    }
  }
  p.result->final_state = x;
  p.result->count = cnt;
  if (p.early != nullptr) write_early(p.early, x, cnt, 0u);
}

#endif  // PAREM_BATCH_KERNELS

// Launch wrappers, instantiated in the per-layout translation units.
//
// The dynamic shared memory limit of a kernel is raised once per device to the largest size
// launched so far (one slot per device ordinal below 64; others set it at every launch).
template <typename K>
cudaError_t raise_smem_limit(K kern, size_t smem, std::atomic<size_t>* limits) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorInvalidDevice;
  if (dev >= 0 && dev < 64 && limits[dev].load(std::memory_order_relaxed) >= smem) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && dev >= 0 && dev < 64) {
    size_t cur = limits[dev].load(std::memory_order_relaxed);
    while (cur < smem && !limits[dev].compare_exchange_weak(cur, smem)) {
    }
  }
  return e;
}

template <int LAYOUT, int ESIZE, int P>
cudaError_t launch_spec_scan(const CUtensorMap& tmap, const ScanParams& p, int grid, int block,
                             size_t smem, cudaStream_t stream) {
  static std::atomic<size_t> limits[64];
  auto kern = k_spec_scan<LAYOUT, ESIZE, P>;
  cudaError_t e = raise_smem_limit(kern, smem, limits);
  if (e != cudaSuccess) return e;
  kern<<<grid, block, smem, stream>>>(tmap, p);
  return cudaGetLastError();
}

template <int LAYOUT, int ESIZE>
cudaError_t launch_emit(const ScanParams& p, const CUtensorMap* tm, int grid, int block, size_t smem,
                        cudaStream_t stream) {
  static std::atomic<size_t> limits[64], limits_stream[64];
  // the chosen block size per (device, shared memory size), packed as smem << 24 | blocks << 12 | block
  static std::atomic<uint64_t> choice[64];
  if (p.match_bits != nullptr) {
    // dense matches recorded as bits by pass 1: four blocks of 16 warps per SM expand them;
    // k_emit below then writes what needs the table (row 0's head, rows without bits)
    const size_t sm_bytes = (size_t)kEmitBitsWarps * kEmitBitsRound * 2;
    const uint64_t want = (p.R + kEmitBitsWarps - 1) / kEmitBitsWarps;
    const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)grid * 4, want));
    k_emit_bits<<<blocks, kEmitBitsWarps * 32, sm_bytes, stream>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (p.stream_emit && tm != nullptr) {
    // dense matches: pass 1's launch shape (one block per SM, warps as shared memory allows)
    auto kern = k_emit_stream<LAYOUT, ESIZE>;
    const size_t per_warp = kStages * kStageBytes + kStages * 8 + kLanes * kEmitBuf * 2;
    const size_t fixed = smem + 1024;  // column map and table, then alignment of the stages
    int optin = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int warps = (int)std::min<size_t>(32, ((size_t)optin - fixed) / per_warp);
    if (warps < 1) return cudaErrorInvalidValue;
    const size_t sm_bytes = fixed + (size_t)warps * per_warp;
    cudaError_t e = raise_smem_limit(kern, sm_bytes, limits_stream);
    if (e != cudaSuccess) return e;
    const uint64_t chunk_blocks = (p.n_chunks + warps - 1) / warps;
    const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sms, chunk_blocks));
    kern<<<blocks, warps * 32, sm_bytes, stream>>>(*tm, p);
    return cudaGetLastError();
  }
  auto kern = k_emit<LAYOUT, ESIZE>;
  cudaError_t e = raise_smem_limit(kern, smem, limits);
  if (e != cudaSuccess) return e;
  // One thread per row: the block size that keeps the most threads resident (the table in
  // shared memory is per block, so larger blocks share it among more rows), one wave of
  // resident blocks.  `grid` carries the SM count and `block` the smallest block size.
  int dev = 0;
  cudaGetDevice(&dev);
  int best_threads = 0, best_block = block, best_blocks = 1;
  const uint64_t c = (dev >= 0 && dev < 64) ? choice[dev].load(std::memory_order_relaxed) : 0;
  if (c && (c >> 24) == smem) {
    best_blocks = (int)((c >> 12) & 0xFFF);
    best_block = (int)(c & 0xFFF);
  } else {
    for (int b = block; b <= 1024; b *= 2) {
      int nb = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, b, smem) != cudaSuccess) continue;
      if (nb * b > best_threads) {
        best_threads = nb * b;
        best_block = b;
        best_blocks = nb;
      }
    }
    if (dev >= 0 && dev < 64 && best_blocks < 4096)
      choice[dev].store((uint64_t)smem << 24 | (uint64_t)best_blocks << 12 | (uint64_t)best_block,
                        std::memory_order_relaxed);
  }
  // no more blocks than there are rows to cover: every block stages the table
  const uint64_t need = (p.R + best_block - 1) / best_block;
  const int blocks = (int)std::min<uint64_t>((uint64_t)grid * best_blocks, std::max<uint64_t>(need, 1));
  kern<<<blocks, best_block, smem, stream>>>(p);
  return cudaGetLastError();
}

template <int LAYOUT, int ESIZE>
cudaError_t launch_tiny(const ScanParams& p, size_t smem, cudaStream_t stream) {
  static std::atomic<size_t> limits[64];
  auto kern = k_tiny<LAYOUT, ESIZE>;
  cudaError_t e = raise_smem_limit(kern, smem, limits);
  if (e != cudaSuccess) return e;
  kern<<<1, 128, smem, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace parem
