// parem_api.cu -- the C ABI of libparem (include/parem.h): DFA loading, scratch memory,
// the launch planner and the scan entry points.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "../../include/parem.h"
#include "parem_internal.h"
#include "parem_launch.h"

using namespace parem;

namespace {

constexpr uint32_t kSmemTableBudget = 160 * 1024;

#define PAREM_CUDA_TRY(expr)                              \
  do {                                                    \
    cudaError_t _e = (expr);                              \
    if (_e != cudaSuccess) {                              \
      return _e == cudaErrorMemoryAllocation ? PAREM_ERR_OOM : PAREM_ERR_CUDA; \
    }                                                     \
  } while (0)

// ---------------------------------------------------------------------------------------
// scratch memory, cached per (device, stream)
// ---------------------------------------------------------------------------------------
struct Scratch {
  void* dev = nullptr;
  size_t bytes = 0;
  // Two header regions [ticket 256 B][result 256 B][status words], hdr_bytes each.  A scan
  // uses region cur, which is all zero, and its first kernel zeroes the other region (the
  // previous scan's), so no memset precedes the launches.  used[i]: bytes of region i that
  // its last scan may have written (0: clean).
  void* hdr = nullptr;
  size_t hdr_bytes = 0;
  uint32_t cur = 0;
  size_t used[2] = {0, 0};
  DevResult* host_res = nullptr;  // pinned, mapped: the kernels write the result word here
  DevResult* host_res_dev = nullptr;  // its device address
  void* dev_text = nullptr;       // staging for parem_match_host
  size_t text_bytes = 0;
  void* dev_pos = nullptr;
  size_t pos_bytes = 0;
  cudaStream_t copy_st[2] = {nullptr, nullptr};  // host-text pieces are copied on these
  std::vector<cudaEvent_t> piece_ev;              // one per piece: its copy has landed
  cudaEvent_t host_ev = nullptr;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};  // before pass 1, after pass 1, after emit
  bool timed = false, emitted = false, have_stats = false;
  parem_stats stats{};
};

std::mutex g_mu;
std::map<std::pair<int, void*>, Scratch*> g_scratch;

Scratch* get_scratch(int dev, void* stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto& s = g_scratch[{dev, stream}];
  if (!s) s = new (std::nothrow) Scratch();
  return s;
}

int ensure(void** p, size_t* have, size_t need) {
  if (*have >= need && *p) return PAREM_OK;
  size_t sz = std::max(need, (size_t)(*have * 3 / 2));
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  sz = (sz + 4095) & ~(size_t)4095;
  cudaError_t e = cudaMalloc(p, sz);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? PAREM_ERR_OOM : PAREM_ERR_CUDA;
  }
  *have = sz;
  return PAREM_OK;
}

// ---------------------------------------------------------------------------------------
// tensor map encoding through the driver entry point
// ---------------------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// Tensor map of R rows of S bytes: boxes of `box` bytes (32 or 64) x 32 rows, swizzled by the
// box width so that the 32 lanes' 16-byte reads of one chunk fall in distinct banks.
int encode_rows(CUtensorMap* tm, const uint8_t* base, uint64_t S, uint64_t R, uint32_t box_w = kBox) {
  auto fn = encode_fn();
  if (!fn) return PAREM_ERR_CUDA;
  cuuint64_t dims[2] = {(cuuint64_t)S, (cuuint64_t)R};
  cuuint64_t strides[1] = {(cuuint64_t)S};
  cuuint32_t box[2] = {box_w, kLanes};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(base), dims, strides, box,
                  estr, CU_TENSOR_MAP_INTERLEAVE_NONE, box_w == 32 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? PAREM_OK : PAREM_ERR_CUDA;
}

struct DevProps {
  int sms = 0;
  int smem_optin = 0;
};

DevProps dev_props(int dev) {
  static std::mutex mu;
  static std::map<int, DevProps> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  DevProps p;
  cudaDeviceGetAttribute(&p.sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&p.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cache[dev] = p;
  return p;
}

uint64_t round_up(uint64_t x, uint64_t m) { return (x + m - 1) / m * m; }

void fill_info(const Prepared& P, parem_dfa_info* info) {
  std::memset(info, 0, sizeof(*info));
  info->n_states = P.n_in;
  info->n_symbols = P.n_sym;
  info->compact_states = P.n;
  info->n_classes = P.n_classes;
  info->has_dead = P.has_dead;
  info->entry_bytes = P.esize;
  info->layout = P.layout;
  info->table_bytes = P.table_bytes;
  info->max_candidates = P.max_cand;
  info->mean_candidates = P.mean_cand;
  info->sync_estimate = P.sync_len;
}

}  // namespace

namespace parem {

int upload_prepared(const Prepared& P, DeviceDfa* out, void** dmem) {
  // one allocation: table | colmap | byte_class | img_off | img | rank
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = round_up(off + bytes, 256);
    return o;
  };
  const size_t o_table = take(P.table.size());
  const bool wide = P.layout == kClassSmemW || P.layout == kClassGlobalW;
  std::vector<uint8_t> cm(512, 0);
  for (int b = 0; b < 256; ++b) {
    if (wide) {
      std::memcpy(&cm[2 * b], &P.colmap[b], 2);
    } else {
      cm[b] = (uint8_t)P.colmap[b];
    }
  }
  const size_t o_colmap = take(512);
  const size_t o_cls = take(256 * 2);
  const size_t o_imgoff = take(P.img_off.size() * 4);
  const size_t o_img = take(P.img.size() * 2);
  const size_t o_rank = take(P.rank.size() * 2);
  const size_t o_sync = take(256 * 2);
  // the synchronising bytes: classes whose candidate list has at most one state
  std::vector<uint16_t> sync(256, (uint16_t)kNoSync16);
  if (P.n < 0xFFFFu) {
    for (int b = 0; b < 256; ++b) {
      const uint32_t c = P.byte_class[b];
      const uint32_t m = P.img_off[c + 1] - P.img_off[c];
      if (m == 1) sync[b] = P.img[P.img_off[c]];
      else if (m == 0 && P.has_dead) sync[b] = (uint16_t)P.dead;
    }
  }
  void* mem = nullptr;
  if (cudaMalloc(&mem, off) != cudaSuccess) return PAREM_ERR_OOM;
  uint8_t* base = static_cast<uint8_t*>(mem);
  cudaError_t e = cudaSuccess;
  e = e == cudaSuccess ? cudaMemcpy(base + o_table, P.table.data(), P.table.size(), cudaMemcpyHostToDevice) : e;
  e = e == cudaSuccess ? cudaMemcpy(base + o_colmap, cm.data(), 512, cudaMemcpyHostToDevice) : e;
  e = e == cudaSuccess ? cudaMemcpy(base + o_cls, P.byte_class.data(), 256 * 2, cudaMemcpyHostToDevice) : e;
  e = e == cudaSuccess ? cudaMemcpy(base + o_imgoff, P.img_off.data(), P.img_off.size() * 4, cudaMemcpyHostToDevice) : e;
  e = e == cudaSuccess ? cudaMemcpy(base + o_img, P.img.data(), P.img.size() * 2, cudaMemcpyHostToDevice) : e;
  e = e == cudaSuccess ? cudaMemcpy(base + o_rank, P.rank.data(), P.rank.size() * 2, cudaMemcpyHostToDevice) : e;
  e = e == cudaSuccess ? cudaMemcpy(base + o_sync, sync.data(), 256 * 2, cudaMemcpyHostToDevice) : e;
  if (e != cudaSuccess) {
    cudaFree(mem);
    return PAREM_ERR_CUDA;
  }
  DeviceDfa D{};
  D.table = base + o_table;
  D.colmap = base + o_colmap;
  D.byte_class = reinterpret_cast<const uint16_t*>(base + o_cls);
  D.img_off = reinterpret_cast<const uint32_t*>(base + o_imgoff);
  D.img = reinterpret_cast<const uint16_t*>(base + o_img);
  D.rank = reinterpret_cast<const uint16_t*>(base + o_rank);
  D.n = P.n;
  D.n_classes = P.n_classes;
  D.first_accept = P.first_accept;
  D.dead = P.dead;
  D.start = P.start;
  D.layout = P.layout;
  D.esize = P.esize;
  D.rowbytes = P.rowbytes;
  D.table_bytes = P.table_bytes;
  D.max_cand = P.max_cand;
  D.stride_k = P.stride_k;
  D.stride_off = P.stride_off;
  {
    const uint32_t K = P.stride_k;
    D.stride_k4 = K * K * K * K;
    D.stride_wts = K <= 6 ? (K * K * K | (K * K) << 8 | K << 16 | 1u << 24) : 0u;
    D.stride_krep = K * 0x01010101u;
    D.stride_kmrep = K ? (K - 1) * 0x01010101u : 0u;
  }
  D.win = P.win;
  D.pair_hot = P.pair_hot;
  D.pair_off = P.pair_off;
  D.sync_state = reinterpret_cast<const uint16_t*>(base + o_sync);
  *out = D;
  *dmem = mem;
  return PAREM_OK;
}

}  // namespace parem

// =======================================================================================
// ABI
// =======================================================================================
extern "C" const char* parem_strerror(int status) {
  switch (status) {
    case PAREM_OK: return "ok";
    case PAREM_ERR_INVALID_ARG: return "invalid argument";
    case PAREM_ERR_OOM: return "out of memory";
    case PAREM_ERR_CAPACITY: return "more matches than the position buffer holds";
    case PAREM_ERR_TIMEOUT: return "a bounded device-side wait ran out";
    case PAREM_ERR_CUDA: return "CUDA runtime error";
    case PAREM_ERR_INTERNAL: return "device-side self-check failed";
    case PAREM_ERR_UNSUPPORTED: return "unsupported request";
    case PAREM_ERR_TOO_LARGE: return "the request needs more scratch than the fixed area of parem_match_noalloc";
    default: return "unknown status";
  }
}

extern "C" const char* parem_version(void) { return "0.1.0"; }

extern "C" int parem_prepare_info(const uint32_t* table, uint32_t n_states, uint32_t n_symbols,
                                  const uint16_t* byte_to_symbol, uint32_t start, const uint8_t* accept,
                                  parem_dfa_info* info) {
  if (!info) return PAREM_ERR_INVALID_ARG;
  Prepared P;
  int rc = prepare_dfa(table, n_states, n_symbols, byte_to_symbol, start, accept, kSmemTableBudget, &P);
  if (rc != PAREM_OK) return rc;
  fill_info(P, info);
  return PAREM_OK;
}

extern "C" int parem_load_dfa(const uint32_t* table, uint32_t n_states, uint32_t n_symbols,
                              const uint16_t* byte_to_symbol, uint32_t start, const uint8_t* accept,
                              parem_dfa** out) {
  if (!out) return PAREM_ERR_INVALID_ARG;
  *out = nullptr;
  parem_dfa* d = new (std::nothrow) parem_dfa();
  if (!d) return PAREM_ERR_OOM;
  int rc = prepare_dfa(table, n_states, n_symbols, byte_to_symbol, start, accept, kSmemTableBudget, &d->host);
  if (rc != PAREM_OK) {
    delete d;
    return rc;
  }
  const Prepared& P = d->host;
  if (cudaGetDevice(&d->device) != cudaSuccess) {
    delete d;
    return PAREM_ERR_CUDA;
  }
  rc = upload_prepared(P, &d->dev, &d->dmem);
  if (rc != PAREM_OK) {
    delete d;
    return rc;
  }
  fill_info(P, &d->info);
  *out = d;
  return PAREM_OK;
}

extern "C" int parem_dfa_get_info(const parem_dfa* dfa, parem_dfa_info* info) {
  if (!dfa || !info) return PAREM_ERR_INVALID_ARG;
  *info = dfa->info;
  info->pair_hot_states =
      dfa->pair_state.load(std::memory_order_acquire) == kPairReady ? dfa->pair_host.pair_hot : 0u;
  return PAREM_OK;
}

extern "C" void parem_free_dfa(parem_dfa* dfa) {
  if (!dfa) return;
  cudaDeviceSynchronize();
  if (dfa->dmem) cudaFree(dfa->dmem);
  if (dfa->batch_mem) cudaFree(dfa->batch_mem);
  if (dfa->pair_mem) cudaFree(dfa->pair_mem);
  delete dfa;
}

extern "C" int parem_last_stats(void* stream, parem_stats* out) {
  if (!out) return PAREM_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PAREM_ERR_CUDA;
  Scratch* s = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_scratch.find({dev, stream});
    if (it == g_scratch.end()) return PAREM_ERR_INVALID_ARG;
    s = it->second;
  }
  if (!s->have_stats) return PAREM_ERR_INVALID_ARG;
  *out = s->stats;
  out->scan_ms = -1.f;
  out->emit_ms = -1.f;
  if (s->timed) {
    PAREM_CUDA_TRY(cudaEventSynchronize(s->ev[2]));
    PAREM_CUDA_TRY(cudaEventElapsedTime(&out->scan_ms, s->ev[0], s->ev[1]));
    if (s->emitted) {
      PAREM_CUDA_TRY(cudaEventElapsedTime(&out->emit_ms, s->ev[1], s->ev[2]));
    } else {
      out->emit_ms = 0.f;
    }
  }
  return PAREM_OK;
}

extern "C" int parem_release_scratch(void* stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PAREM_ERR_CUDA;
  Scratch* s = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_scratch.find({dev, stream});
    if (it == g_scratch.end()) return PAREM_OK;
    s = it->second;
    g_scratch.erase(it);
  }
  cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (s->dev) cudaFree(s->dev);
  if (s->hdr) cudaFree(s->hdr);
  if (s->dev_text) cudaFree(s->dev_text);
  if (s->dev_pos) cudaFree(s->dev_pos);
  if (s->host_res) cudaFreeHost(s->host_res);
  for (auto& ev : s->ev)
    if (ev) cudaEventDestroy(ev);
  delete s;
  return PAREM_OK;
}

// ---------------------------------------------------------------------------------------
// planning and launching one scan
// ---------------------------------------------------------------------------------------
namespace parem {

// Candidate sets of DFAs with at least 256 states that take longer than this to shrink to
// one state (estimated, symbols) merge through the state bitmap every 16 steps: merging
// with match_any only finds equal states within one register, so a long shrinking phase
// would keep every register live.
constexpr uint32_t kBitmapSync = 16;

// Row length in units of the estimated synchronisation length, and in units of the longest
// merge seen so far (measured on random DFAs with 126 to 2,000 states and 1 GiB of text:
// throughput rises up to 16-32 x the estimate, where the speculation is a small part of a row).
constexpr uint64_t kRowsPerSync = 16;
constexpr uint64_t kRowsPerMerge = 2;

bool serial_rows(const parem_dfa* dfa, uint32_t m) { return m > kLanes && dfa->host.sync_len != kNoSync; }

uint64_t max_row_bytes(const parem_dfa* dfa, uint32_t m) {
  // An unmerged row run from its resolved start costs S lookups on the chunk's warp.
  if (serial_rows(dfa, m)) return 16u << 20;
  // Through slot maps it costs m * S lookups; bound that to 2^27 lookups so that even a text
  // that never synchronises the automaton keeps every chunk well inside the device wait limit.
  return std::max<uint64_t>(4096, ((1ull << 27) / std::max<uint32_t>(m, 1)) / kBox * kBox);
}

uint64_t min_row_bytes(const parem_dfa* dfa, uint32_t P) {
  const Prepared& H = dfa->host;
  // grouped speculation of small candidate sets costs little per row: short rows keep small
  // texts spread over many warps
  uint64_t smin = P == 1 ? 128 : 4096;
  // rows several times longer than the candidates need to merge: the estimate from random
  // input (prepare time) or the longest merge seen on real input, whichever is larger
  const uint64_t est = H.sync_len == kNoSync ? 0 : H.sync_len;
  smin = std::max<uint64_t>(smin, std::max<uint64_t>(kRowsPerSync * est, kRowsPerMerge * dfa->conv_hint.load()));
  smin = std::min<uint64_t>(round_up(smin, kBox), 64u << 20);
  return std::min(smin, max_row_bytes(dfa, H.max_cand));
}

void learn_convergence(const parem_dfa* dfa, uint32_t spec_cap, uint32_t nonconv_rows, uint32_t conv_max) {
  // Only DFAs whose candidates do merge teach anything: when some rows merged and others ran
  // out of the speculation cap, the next plans get a larger cap (4x) and longer rows (8x). A
  // DFA whose rows never merge (a permutation automaton) keeps its plan: longer rows would
  // not make its slot maps cheaper.
  if (conv_max == 0) return;
  uint32_t want = nonconv_rows ? std::max(conv_max, spec_cap) : conv_max;
  want = std::min<uint32_t>(want, 1u << 24);
  auto& h = const_cast<parem_dfa*>(dfa)->conv_hint;
  uint32_t cur = h.load();
  while (want > cur && !h.compare_exchange_weak(cur, want)) {
  }
}

int plan_scan(const parem_dfa* dfa, const uint8_t* text, uint64_t len, const parem_match_opts* o,
              Plan* pl) {
  const DevProps props = dev_props(dfa->device);
  std::memset(pl, 0, sizeof(*pl));
  // the two-byte stride variant once it has been learned (and unless the call declines it)
  const bool pair = !(o && o->pair_mode == PAREM_PAIR_OFF) &&
                    dfa->pair_state.load(std::memory_order_acquire) == kPairReady;
  pl->prep = pair ? &dfa->pair_host : &dfa->host;
  pl->ddfa = pair ? &dfa->pair_dev : &dfa->dev;
  const Prepared& P = *pl->prep;
  pl->layout = P.layout;
  pl->enum_all = o && o->enumerate_all ? 1u : 0u;
  const uint32_t m_need = pl->enum_all ? (P.n - P.has_dead) : P.max_cand;
  pl->P = m_need <= 32 ? 1 : m_need <= 64 ? 2 : m_need <= 128 ? 4 : 8;
  pl->cand_stride = std::max<uint32_t>(1, std::max(P.max_cand, pl->enum_all ? P.n : 0u));
  pl->serial = serial_rows(dfa, m_need) ? 1u : 0u;
  // fewer than one match per KiB in the last large scan: matches are rare enough that
  // replaying the few vectors that hold one is cheaper than counting at every byte
  const uint32_t density = dfa->density_hint.load();
  pl->sparse = density < 1024u ? 1u : 0u;
  // at least one match per 64 bytes: a row's replay in the emit pass is long serial work,
  // so it is split into pieces that run in parallel
  pl->dense = (density != 0xFFFFFFFFu && density >= 16384u) ? 1u : 0u;
  // lanes per row in the grouped speculation (P == 1): the smallest power of two that holds
  // the largest candidate set
  pl->group = 1;
  while (pl->group < m_need && pl->group < 32) pl->group *= 2;
  // shared memory of pass 1: [colmap | table at kTableOff][slack to 1024][per-warp region]
  const uint32_t table_smem = (P.layout == kClassGlobal || P.layout == kClassGlobalW) ? 0 : P.table_bytes;
  pl->table_smem = table_smem;
  const uint32_t fixed = kTableOff + table_smem + 1024;
  // candidate sets larger than the registers run through a per-warp bitmap of the states
  pl->bitmap_words = 0;
  if (pl->P > 1 && P.n <= 16384 && (m_need > 32u * pl->P || (P.sync_len > kBitmapSync && P.n >= 256)))
    pl->bitmap_words = (P.n + 31) / 32;
  pl->spec_bytes = kSpecBytes + (pl->bitmap_words ? (uint32_t)round_up(8ull * pl->bitmap_words, 16) + 512u : 0u);
  const uint32_t per_warp = kStages * kLanes * box_bytes(P.layout) + kStages * 8 + pl->spec_bytes;
  int warps = (int)((props.smem_optin - (int)fixed) / (int)per_warp);
  // the launch bounds of the kernel variants
  warps = std::min(warps, P.layout == kClassPair ? (int)kPairMaxWarps : pl->P >= 4 ? 24 : 32);
  if (o && o->warps_per_block) warps = std::min<int>(warps, (int)o->warps_per_block);
  if (warps < 1) return PAREM_ERR_UNSUPPORTED;
  pl->warps = warps;
  pl->grid = props.sms;
  pl->smem = fixed + (size_t)warps * per_warp;
  // rows
  const uint64_t addr = reinterpret_cast<uint64_t>(text);
  pl->h = std::min<uint64_t>(len, (16 - (addr & 15)) & 15);
  const uint64_t body = len - pl->h;
  const uint64_t lanes_total = (uint64_t)pl->grid * warps * kLanes;
  uint64_t S;
  if (o && o->segment_bytes) {
    S = round_up(o->segment_bytes, kBox);
  } else {
    const uint64_t smax = max_row_bytes(dfa, m_need);
    const uint64_t smin = std::min(min_row_bytes(dfa, pl->P), smax);
    const uint64_t shi = std::max<uint64_t>(smin, std::min<uint64_t>(smax, 1u << 20));
    // One wave: rows long enough that every warp owns at most one chunk.  All chunks then
    // run at once and finish together, so no look-back waits on a predecessor that started
    // later, and the per-chunk work (speculation, pipeline fill) is paid once per warp.
    S = round_up(std::max<uint64_t>((body + lanes_total - 1) / lanes_total, 1), kBox);
    S = std::min<uint64_t>(std::max(S, smin), shi);
    // The tail (body mod S) is run by the last row's lane after its row, which puts it on
    // the critical path: among the next 64 row lengths (still one wave) take the one with
    // the least S + tail.
    if (body >= S) {
      uint64_t best = S, best_cost = S + body % S;
      for (uint64_t c = S + kBox; c <= std::min<uint64_t>(S + 64 * kBox, shi); c += kBox) {
        const uint64_t cost = c + body % c;
        if (cost < best_cost) {
          best = c;
          best_cost = cost;
        }
      }
      S = best;
    }
  }
  // keep the row index inside the TMA coordinate range
  while (body / S >= (1ull << 31)) S *= 2;
  if (body < S) S = body / kBox * kBox;
  pl->S = S;
  pl->R = S ? body / S : 0;
  pl->tail = S ? body - pl->R * S : body;
  pl->n_chunks = (pl->R + kLanes - 1) / kLanes;
  // Fewer chunks than warps: warps take chunks in ticket order, and the warps of the first
  // blocks would take them all, crowding a few SMs.  Spread them: one block per chunk up to
  // the SM count, then as many warps per block as the chunks need.
  if (!(o && o->warps_per_block) && pl->n_chunks < (uint64_t)pl->grid * pl->warps) {
    if (pl->n_chunks <= (uint64_t)pl->grid) {
      pl->grid = (int)std::max<uint64_t>(1, pl->n_chunks);
      pl->warps = 1;
    } else {
      pl->warps = (int)((pl->n_chunks + pl->grid - 1) / pl->grid);
    }
    pl->smem = fixed + (size_t)pl->warps * per_warp;
  }
  uint64_t cap = o && o->spec_cap_bytes ? o->spec_cap_bytes
                                        : std::max<uint64_t>(std::max<uint64_t>(2048, 16ull * P.n),
                                                             4ull * dfa->conv_hint.load());
  cap = std::min<uint64_t>(cap, S);
  pl->spec_cap = (uint32_t)(cap / 16 * 16);
  if (pl->spec_cap == 0) pl->spec_cap = 16;
  return PAREM_OK;
}

}  // namespace parem

static int run_scan(const parem_dfa* dfa, const uint8_t* text, uint64_t len, uint64_t* positions,
                    uint64_t capacity, const parem_match_opts* o, cudaStream_t stream, parem_result* out,
                    uint64_t pos_base = 0) {
  if (o && o->use_start_state && o->start_state >= dfa->host.n_in) return PAREM_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  if (len == 0) {
    const Prepared& P0 = dfa->host;
    const uint32_t init0 = (o && o->use_start_state) ? P0.compact_of[o->start_state] : P0.start;
    out->final_state = P0.orig_of[init0];
    out->accepted = init0 >= P0.first_accept;
    return PAREM_OK;
  }
  Plan pl;
  int rc = plan_scan(dfa, text, len, o, &pl);
  if (rc != PAREM_OK) return rc;
  // the prepared DFA of this scan (the two-byte stride variant when it is used): its state
  // numbering applies to the start state and the result
  const Prepared& P = *pl.prep;
  const uint32_t init = (o && o->use_start_state) ? P.compact_of[o->start_state] : P.start;
  Scratch* sc = get_scratch(dfa->device, stream);
  if (!sc) return PAREM_ERR_OOM;
  if (!sc->host_res) {
    if (cudaHostAlloc(&sc->host_res, sizeof(DevResult), cudaHostAllocMapped) != cudaSuccess) {
      sc->host_res = nullptr;
      return PAREM_ERR_OOM;
    }
    if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&sc->host_res_dev), sc->host_res, 0) != cudaSuccess) {
      cudaFreeHost(sc->host_res);
      sc->host_res = nullptr;
      return PAREM_ERR_CUDA;
    }
  }
  // header (double-buffered, see Scratch): [ticket 256][result 256][status K*8]
  const uint64_t o_status = 512;
  const uint64_t hdr_need = round_up(o_status + pl.n_chunks * 8, 256);
  if (!sc->hdr || sc->hdr_bytes < hdr_need) {
    if (sc->hdr) cudaFree(sc->hdr);
    sc->hdr = nullptr;
    sc->hdr_bytes = 0;
    const size_t sz = round_up(std::max<uint64_t>(hdr_need, sc->hdr_bytes * 3 / 2), 4096);
    cudaError_t ae = cudaMalloc(&sc->hdr, 2 * sz);
    if (ae != cudaSuccess) {
      sc->hdr = nullptr;
      return ae == cudaErrorMemoryAllocation ? PAREM_ERR_OOM : PAREM_ERR_CUDA;
    }
    sc->hdr_bytes = sz;
    sc->cur = 0;
    sc->used[0] = sc->used[1] = 0;
    PAREM_CUDA_TRY(cudaMemsetAsync(sc->hdr, 0, 2 * sz, stream));
  }
  if (sc->used[sc->cur]) {  // an earlier scan stopped before its kernel cleared this region
    PAREM_CUDA_TRY(cudaMemsetAsync(static_cast<uint8_t*>(sc->hdr) + sc->cur * sc->hdr_bytes, 0,
                                   sc->used[sc->cur], stream));
    sc->used[sc->cur] = 0;
  }
  uint8_t* hb = static_cast<uint8_t*>(sc->hdr) + sc->cur * sc->hdr_bytes;
  uint8_t* hb_other = static_cast<uint8_t*>(sc->hdr) + (sc->cur ^ 1u) * sc->hdr_bytes;
  // scratch: [segrec R*16][row slots][slot_end][slot_cnt]
  const bool emit = positions != nullptr && capacity > 0;
  const uint64_t o_segrec = 0;
  const uint64_t o_rows = round_up(o_segrec + (emit ? pl.R * sizeof(SegRec) : 0), 256);
  const uint64_t o_slot = round_up(o_rows + (emit ? pl.R * kRowSlotBytes : 0), 256);
  const uint64_t slot_bytes = pl.serial ? 0 : pl.R * (uint64_t)pl.cand_stride * 4;
  // dense matches: pass 1 records them as one bit per body byte and the emit pass expands
  // the bits (the pair and stride layouts count in their own ways and keep the replay)
  const bool bits = emit && pl.dense && pl.R && P.layout != kByteStride && P.layout != kClassPair;
  const uint64_t o_bits = round_up(o_slot + 2 * slot_bytes, 256);
  const uint64_t bits_bytes = bits ? round_up((pl.R * pl.S + pl.tail + 7) / 8 + 16, 256) : 0;
  const uint64_t total = round_up(std::max<uint64_t>(o_bits + bits_bytes, 256), 256);
  rc = ensure(&sc->dev, &sc->bytes, total);
  if (rc != PAREM_OK) return rc;
  uint8_t* sb = static_cast<uint8_t*>(sc->dev);

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
  p.init_state = init;
  p.group = pl.group;
  p.bitmap_words = pl.bitmap_words;
  p.spec_bytes = pl.spec_bytes;
  p.smem_table_bytes = pl.table_smem;
  p.enum_all = pl.enum_all;
  p.spec_cap = pl.spec_cap;
  p.cand_stride = pl.cand_stride;
  p.serial_fallback = pl.serial;
  p.pos_base = pos_base;
  p.sparse_count = pl.sparse;
  p.wait_budget = o && o->wait_budget_cycles ? o->wait_budget_cycles : 4000000000ull;
  p.skip_publish = (o && o->debug_skip_publish_chunk > 0) ? o->debug_skip_publish_chunk : -1;
  if (!o) p.skip_publish = -1;
  p.ticket = reinterpret_cast<uint32_t*>(hb);
  p.result = reinterpret_cast<DevResult*>(hb + 256);
  p.status = reinterpret_cast<unsigned long long*>(hb + o_status);
  p.host_result = sc->host_res_dev;
  p.clear = reinterpret_cast<uint4*>(hb_other);
  p.clear_n16 = round_up(sc->used[sc->cur ^ 1u], 16) / 16;
  p.segrec = emit ? reinterpret_cast<SegRec*>(sb + o_segrec) : nullptr;
  p.slots = emit ? reinterpret_cast<uint32_t*>(sb + o_rows) : nullptr;
  p.slot_end = reinterpret_cast<uint32_t*>(sb + o_slot);
  p.slot_cnt = reinterpret_cast<uint32_t*>(sb + o_slot + slot_bytes);
  p.stream_emit = (emit && pl.dense && pl.R && !bits) ? 1u : 0u;
  p.match_bits = bits ? reinterpret_cast<uint32_t*>(sb + o_bits) : nullptr;
  if (bits) p.sparse_count = 0;
  p.positions = emit ? positions : nullptr;
  p.capacity = emit ? capacity : 0;

  const bool global_table = P.layout == kClassGlobal || P.layout == kClassGlobalW;
  const size_t small_smem = kTableOff + (global_table ? 0 : P.table_bytes);
  const bool timed = o && o->record_kernel_times;
  if (timed && !sc->ev[0]) {
    for (auto& ev : sc->ev) PAREM_CUDA_TRY(cudaEventCreate(&ev));
  }
  sc->timed = timed;
  sc->emitted = false;
  sc->have_stats = true;
  sc->stats = parem_stats{};
  sc->stats.segment_bytes = pl.S;
  sc->stats.rows = pl.R;
  sc->stats.chunks = pl.n_chunks;
  sc->stats.blocks = pl.R ? (uint32_t)pl.grid : 1;
  sc->stats.warps_per_block = pl.R ? (uint32_t)pl.warps : 1;
  sc->stats.candidate_regs = pl.P;
  sc->stats.spec_cap_bytes = pl.spec_cap;
  sc->stats.kernels = 1 + ((pl.R && emit) ? 1 : 0) + (bits ? 1 : 0);
  sc->stats.layout = P.layout;
  sc->stats.pair_hot_states = P.layout == kClassPair ? P.pair_hot : 0u;
  if (timed) PAREM_CUDA_TRY(cudaEventRecord(sc->ev[0], stream));
  cudaError_t e;
  if (pl.R == 0) {
    e = launch_tiny_dispatch(P.layout, P.esize, p, small_smem, stream);
  } else {
    // pass 1 reads boxes of box_bytes(layout); the streaming emit pass always 64-byte boxes
    CUtensorMap tm, tm_emit;
    rc = encode_rows(&tm, text + pl.h, pl.S, pl.R, box_bytes(P.layout));
    if (rc == PAREM_OK && box_bytes(P.layout) != kBox) rc = encode_rows(&tm_emit, text + pl.h, pl.S, pl.R);
    if (rc != PAREM_OK) return rc;
    if (box_bytes(P.layout) == kBox) tm_emit = tm;
    e = launch_scan_dispatch(P.layout, P.esize, pl.P, tm, p, pl.grid, pl.warps * 32, pl.smem, stream);
    if (e == cudaSuccess && timed) e = cudaEventRecord(sc->ev[1], stream);
    if (e == cudaSuccess && emit) {
      sc->emitted = true;
      const DevProps props = dev_props(dfa->device);
      e = launch_emit_dispatch(P.layout, P.esize, p, &tm_emit, props.sms, 256, small_smem, stream);
    }
  }
  if (e == cudaSuccess && timed && pl.R == 0) e = cudaEventRecord(sc->ev[1], stream);
  if (e == cudaSuccess && timed) e = cudaEventRecord(sc->ev[2], stream);
  // region cur is written from here on; the kernel (if it launched) cleared the other one
  sc->used[sc->cur] = hdr_need;
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? PAREM_ERR_OOM : PAREM_ERR_CUDA;
  sc->used[sc->cur ^ 1u] = 0;
  sc->cur ^= 1u;
  // the last kernel's last block wrote the result word to host_res (publish_result)
  PAREM_CUDA_TRY(cudaStreamSynchronize(stream));
  const DevResult r = *sc->host_res;
  sc->stats.emit_replays = r.emit_replays;
  sc->stats.emit_max_window = r.emit_max_window;
  sc->stats.nonconv_rows = r.nonconv_rows;
  sc->stats.conv_max = r.conv_max;
  sc->stats.cycles_spec = r.cyc_spec;
  sc->stats.cycles_main = r.cyc_main;
  sc->stats.cycles_resolve = r.cyc_resolve;
  sc->stats.cycles_bitmap = r.cyc_bitmap;
  sc->stats.cycles_lane = r.cyc_lane;
  sc->stats.spec_lookups = r.spec_lookups;
  if (pl.R) learn_convergence(dfa, pl.spec_cap, r.nonconv_rows, r.conv_max);
  if (len >= (1u << 20) && !r.error)
    const_cast<parem_dfa*>(dfa)->density_hint.store(
        (uint32_t)std::min<uint64_t>(r.count / std::max<uint64_t>(1, len >> 20), 0xFFFFFFFEull));
  // a large text (or a call that asks) teaches a computed-column DFA its hot states once; the
  // two-byte stride variant is used from the next scan on
  if (!r.error && dfa->host.layout == kClassWin && !(o && o->pair_mode == PAREM_PAIR_OFF) &&
      (len >= kPairLearnBytes || (o && o->pair_mode == PAREM_PAIR_LEARN && len >= 4096))) {
    uint32_t expect = kPairNone;
    parem_dfa* md = const_cast<parem_dfa*>(dfa);
    if (md->pair_state.compare_exchange_strong(expect, kPairBusy)) learn_pairs(md, text, len, stream);
  }
  if (r.error == kErrTimeout) return PAREM_ERR_TIMEOUT;
  if (r.error) return PAREM_ERR_INTERNAL;
  const uint32_t fs = r.final_state;
  out->final_state = (fs < P.n) ? P.orig_of[fs] : PAREM_NONE;
  out->accepted = (fs < P.n && fs >= P.first_accept) ? 1 : 0;
  out->match_count = r.count;
  out->n_written = emit ? std::min<uint64_t>(r.count, capacity) : 0;
  if (emit && r.count > capacity) return PAREM_ERR_CAPACITY;
  return PAREM_OK;
}

extern "C" int parem_match_ex(const parem_dfa* dfa, const uint8_t* text, uint64_t len, uint64_t* positions,
                              uint64_t capacity, const parem_match_opts* opts, void* stream, parem_result* out) {
  if (!dfa || !out || (len > 0 && !text) || len > kMaxText) return PAREM_ERR_INVALID_ARG;
  NvtxRange range("parem_match");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return PAREM_ERR_CUDA;
  if (dev != dfa->device) return PAREM_ERR_INVALID_ARG;
  return run_scan(dfa, text, len, positions, capacity, opts, static_cast<cudaStream_t>(stream), out);
}

extern "C" int parem_match(const parem_dfa* dfa, const uint8_t* text, uint64_t len, uint64_t* positions,
                           uint64_t capacity, void* stream, parem_result* out) {
  return parem_match_ex(dfa, text, len, positions, capacity, nullptr, stream, out);
}

extern "C" int parem_match_host(const parem_dfa* dfa, const uint8_t* text, uint64_t len, uint64_t* positions,
                                uint64_t capacity, void* stream, parem_result* out) {
  if (!dfa || !out || (len > 0 && !text) || len > kMaxText) return PAREM_ERR_INVALID_ARG;
  NvtxRange range("parem_match_host");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return PAREM_ERR_CUDA;
  if (dev != dfa->device) return PAREM_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch* sc = get_scratch(dev, stream);
  if (!sc) return PAREM_ERR_OOM;
  int rc = ensure(&sc->dev_text, &sc->text_bytes, std::max<uint64_t>(len, 16));
  if (rc != PAREM_OK) return rc;
  const bool want = positions != nullptr && capacity > 0;
  if (want) {
    rc = ensure(&sc->dev_pos, &sc->pos_bytes, capacity * 8);
    if (rc != PAREM_OK) return rc;
  }
  std::memset(out, 0, sizeof(*out));
  // Pieces of the text are copied on two copy streams, all enqueued at once; each piece is
  // scanned as soon as it has landed, from the state the previous piece ended in (the
  // carry-in start of the scan), while the later pieces are still being copied.
  const uint64_t piece = len <= (64ull << 20) ? std::max<uint64_t>(len, 16)
                                              : std::min<uint64_t>(512ull << 20,
                                                                   std::max<uint64_t>(64ull << 20, (len / 8 + 15) & ~15ull));
  const uint64_t n_pieces = len ? (len + piece - 1) / piece : 0;
  if (!sc->host_ev && cudaEventCreateWithFlags(&sc->host_ev, cudaEventDisableTiming) != cudaSuccess) return PAREM_ERR_CUDA;
  for (int k = 0; k < 2; ++k)
    if (!sc->copy_st[k] && cudaStreamCreateWithFlags(&sc->copy_st[k], cudaStreamNonBlocking) != cudaSuccess)
      return PAREM_ERR_CUDA;
  while (sc->piece_ev.size() < n_pieces) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return PAREM_ERR_CUDA;
    sc->piece_ev.push_back(e);
  }
  // the staging buffer is free once the work already queued on the stream is done
  PAREM_CUDA_TRY(cudaEventRecord(sc->host_ev, st));
  uint8_t* dtext = static_cast<uint8_t*>(sc->dev_text);
  for (uint64_t k = 0; k < n_pieces; ++k) {
    cudaStream_t cs = sc->copy_st[k & 1];
    if (k < 2) PAREM_CUDA_TRY(cudaStreamWaitEvent(cs, sc->host_ev, 0));
    const uint64_t off = k * piece, n = std::min(piece, len - off);
    PAREM_CUDA_TRY(cudaMemcpyAsync(dtext + off, text + off, n, cudaMemcpyHostToDevice, cs));
    PAREM_CUDA_TRY(cudaEventRecord(sc->piece_ev[k], cs));
  }
  const Prepared& P = dfa->host;
  uint32_t state = P.orig_of[P.start];
  bool dead = false;
  uint64_t total = 0, written = 0;
  uint8_t accepted = P.start >= P.first_accept ? 1 : 0;
  rc = PAREM_OK;
  for (uint64_t k = 0; k < n_pieces && !dead; ++k) {
    const uint64_t off = k * piece, n = std::min(piece, len - off);
    PAREM_CUDA_TRY(cudaStreamWaitEvent(st, sc->piece_ev[k], 0));
    parem_match_opts o{};
    o.start_state = state;
    o.use_start_state = 1;
    parem_result r;
    const bool room = want && written < capacity;
    const int rk = run_scan(dfa, dtext + off, n, room ? static_cast<uint64_t*>(sc->dev_pos) + written : nullptr,
                            room ? capacity - written : 0, &o, st, &r, off);
    if (rk != PAREM_OK && rk != PAREM_ERR_CAPACITY) {
      rc = rk;
      break;
    }
    total += r.match_count;
    written += r.n_written;
    accepted = r.accepted;
    if (r.final_state == PAREM_NONE) dead = true;
    else state = r.final_state;
  }
  // copies of pieces after a dead end (or an error) may still be in flight
  for (int k = 0; k < 2; ++k) cudaStreamSynchronize(sc->copy_st[k]);
  if (rc != PAREM_OK) return rc;
  out->final_state = dead ? PAREM_NONE : state;
  out->accepted = dead ? 0 : accepted;
  out->match_count = total;
  out->n_written = want ? std::min<uint64_t>(total, capacity) : 0;
  if (want && out->n_written) {
    PAREM_CUDA_TRY(cudaMemcpyAsync(positions, sc->dev_pos, out->n_written * 8, cudaMemcpyDeviceToHost, st));
  }
  PAREM_CUDA_TRY(cudaStreamSynchronize(st));
  return (want && total > capacity) ? PAREM_ERR_CAPACITY : PAREM_OK;
}
