// parem_noalloc.cu -- parem_match_noalloc: the scan of parem_match with its scratch in a
// fixed, statically defined device array instead of memory allocated by the library.
//
// For callers that cannot allocate device memory (their memory belongs to their own pool
// allocator, or allocation and its implicit synchronisation are not acceptable on their
// path).  The kernels are the ones parem_match launches; only where their scratch lives
// differs.  Calls share the array: overlapping calls race, so callers serialise them.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/parem.h"
#include "parem_internal.h"
#include "parem_launch.h"

using namespace parem;

namespace {

// The fixed scratch area: ticket counter, result word, chunk status words, per-row records
// and slot maps of one scan.  Host code must not take this name as a device address; it
// asks the runtime for the address once per device (scratch_address below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[PAREM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on device `dev` (which must be current); looked up on
// the first call for that device and kept.
int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return PAREM_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return PAREM_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return PAREM_OK;
}

int encode_rows_noalloc(CUtensorMap* tm, const uint8_t* base, uint64_t S, uint64_t R, uint32_t box_w) {
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
  if (!fn) return PAREM_ERR_CUDA;
  cuuint64_t dims[2] = {(cuuint64_t)S, (cuuint64_t)R};
  cuuint64_t strides[1] = {(cuuint64_t)S};
  cuuint32_t box[2] = {box_w, kLanes};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(base), dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        box_w == 32 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? PAREM_OK : PAREM_ERR_CUDA;
}

uint64_t up256(uint64_t x) { return (x + 255) & ~255ull; }

}  // namespace

extern "C" int parem_match_noalloc(const parem_dfa* dfa, const uint8_t* text, uint64_t len, uint64_t* positions,
                                   uint64_t capacity, void* stream, parem_result* out) {
  if (!dfa || !out || (len > 0 && !text) || len > kMaxText) return PAREM_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return PAREM_ERR_CUDA;
  if (dev != dfa->device) return PAREM_ERR_INVALID_ARG;
  void* area = nullptr;
  int rc = scratch_address(dev, &area);
  if (rc != PAREM_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (len == 0) {
    const Prepared& P0 = dfa->host;
    std::memset(out, 0, sizeof(*out));
    out->final_state = P0.orig_of[P0.start];
    out->accepted = P0.start >= P0.first_accept;
    return PAREM_OK;
  }
  Plan pl;
  rc = plan_scan(dfa, text, len, nullptr, &pl);
  if (rc != PAREM_OK) return rc;
  // the prepared DFA of this scan (its two-byte stride variant once parem_match has learned it)
  const Prepared& P = *pl.prep;
  // the layout of parem_match's scratch, inside the fixed area
  const bool emit = positions != nullptr && capacity > 0;
  const uint64_t o_status = 512;
  const uint64_t o_segrec = up256(o_status + pl.n_chunks * 8);
  const uint64_t o_rows = up256(o_segrec + (emit ? pl.R * sizeof(SegRec) : 0));
  const uint64_t o_slot = up256(o_rows + (emit ? pl.R * kRowSlotBytes : 0));
  const uint64_t slot_bytes = pl.serial ? 0 : pl.R * (uint64_t)pl.cand_stride * 4;
  const uint64_t total = up256(o_slot + 2 * slot_bytes);
  if (total > PAREM_NOALLOC_SCRATCH_BYTES) return PAREM_ERR_TOO_LARGE;
  uint8_t* sb = static_cast<uint8_t*>(area);
  // the ticket counter, the result word and the status words must start at zero
  if (cudaMemsetAsync(sb, 0, o_status + pl.n_chunks * 8, st) != cudaSuccess) return PAREM_ERR_CUDA;

  ScanParams p;
  std::memset(&p, 0, sizeof(p));
  p.dfa = *pl.ddfa;
  p.text = text;
  p.n = len;
  p.h = pl.h;
  p.S = pl.S;
  p.R = pl.R;
  p.tail = pl.tail;
  p.n_chunks = pl.n_chunks;
  p.init_state = P.start;
  p.group = pl.group;
  p.bitmap_words = pl.bitmap_words;
  p.spec_bytes = pl.spec_bytes;
  p.smem_table_bytes = pl.table_smem;
  p.enum_all = 0;
  p.spec_cap = pl.spec_cap;
  p.cand_stride = pl.cand_stride;
  p.serial_fallback = pl.serial;
  p.sparse_count = pl.sparse;
  p.wait_budget = 4000000000ull;
  p.skip_publish = -1;
  p.ticket = reinterpret_cast<uint32_t*>(sb);
  p.result = reinterpret_cast<DevResult*>(sb + 256);
  p.status = reinterpret_cast<unsigned long long*>(sb + o_status);
  p.segrec = emit ? reinterpret_cast<SegRec*>(sb + o_segrec) : nullptr;
  p.slots = emit ? reinterpret_cast<uint32_t*>(sb + o_rows) : nullptr;
  p.slot_end = reinterpret_cast<uint32_t*>(sb + o_slot);
  p.slot_cnt = reinterpret_cast<uint32_t*>(sb + o_slot + slot_bytes);
  p.positions = emit ? positions : nullptr;
  p.capacity = emit ? capacity : 0;
  // dense matches (learned from the DFA's earlier scans): the streaming emit pass, as in
  // parem_match; it reads the same row records and needs no other scratch
  p.stream_emit = (emit && pl.dense && pl.R) ? 1u : 0u;

  const bool global_table = P.layout == kClassGlobal || P.layout == kClassGlobalW;
  const size_t small_smem = kTableOff + (global_table ? 0 : P.table_bytes);
  cudaError_t e;
  if (pl.R == 0) {
    e = launch_tiny_dispatch(P.layout, P.esize, p, small_smem, st);
  } else {
    // pass 1 reads boxes of box_bytes(layout); the streaming emit pass always 64-byte boxes
    CUtensorMap tm, tm_emit;
    rc = encode_rows_noalloc(&tm, text + pl.h, pl.S, pl.R, box_bytes(P.layout));
    if (rc == PAREM_OK) rc = encode_rows_noalloc(&tm_emit, text + pl.h, pl.S, pl.R, kBox);
    if (rc != PAREM_OK) return rc;
    e = launch_scan_dispatch(P.layout, P.esize, pl.P, tm, p, pl.grid, pl.warps * 32, pl.smem, st);
    if (e == cudaSuccess && emit) {
      int sms = 0;
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PAREM_ERR_CUDA;
      e = launch_emit_dispatch(P.layout, P.esize, p, &tm_emit, sms, 256, small_smem, st);
    }
  }
  if (e != cudaSuccess) return PAREM_ERR_CUDA;
  DevResult r;
  if (cudaMemcpyAsync(&r, p.result, sizeof(DevResult), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return PAREM_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PAREM_ERR_CUDA;
  // what this scan taught about the DFA (how long its candidates took to merge, how dense its
  // matches are) feeds the plans of later scans, whichever entry point makes them
  if (pl.R) learn_convergence(dfa, pl.spec_cap, r.nonconv_rows, r.conv_max);
  if (len >= (1u << 20) && !r.error)
    const_cast<parem_dfa*>(dfa)->density_hint.store(
        (uint32_t)std::min<uint64_t>(r.count / std::max<uint64_t>(1, len >> 20), 0xFFFFFFFEull));
  if (r.error == kErrTimeout) return PAREM_ERR_TIMEOUT;
  if (r.error) return PAREM_ERR_INTERNAL;
  std::memset(out, 0, sizeof(*out));
  const uint32_t fs = r.final_state;
  out->final_state = (fs < P.n) ? P.orig_of[fs] : PAREM_NONE;
  out->accepted = (fs < P.n && fs >= P.first_accept) ? 1 : 0;
  out->match_count = r.count;
  out->n_written = emit ? (r.count < capacity ? r.count : capacity) : 0;
  if (emit && r.count > capacity) return PAREM_ERR_CAPACITY;
  return PAREM_OK;
}
