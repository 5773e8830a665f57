// parem_pair.cpp -- the two-byte stride variant (kClassPair) of a DFA whose class table has
// computed columns (kClassWin).
//
// The main run of Algorithm 1's candidate runs costs one dependent table lookup per byte.
// For texts of lowercase letters and spaces (the byte codes f = b & 0x1F of {0x20, 0x61..0x7A}
// are 0..26), one lookup in a table indexed by (state, f0, f1) advances two bytes.  Such a
// table over every state would be |Q| * 729 bytes; it is built for the H hot states only,
// the ones a run visits most, and a run that leaves them (or meets an accepting state, or a
// byte outside the set) takes the byte loop for that 16-byte vector.  Which states are hot
// depends on the text, so it is learned once: the first scan of at least kPairLearnBytes
// (or one that asks for it) copies a sample of its text to the host, runs the DFA over it,
// and keeps the variant when its estimated share of vectors needing the byte loop is small.
// The variant is a copy of the prepared DFA with the hot states renumbered 0 .. H-1 (so the
// hot index of a state is its compact id) and the pair table appended to its table; the
// original stays in use for everything else (batches, servers).  Results do not change: the
// pair table holds exactly the composed transitions, and the byte loop handles the rest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "../../include/parem.h"
#include "parem_internal.h"
#include "parem_launch.h"

namespace parem {

namespace {

// Byte of pair code f (0 space, 1..26 a..z) and the code of a byte (-1: outside the set).
inline uint8_t code_byte(uint32_t f) { return f == 0 ? 0x20 : (uint8_t)(0x60 + f); }
inline int pair_code(uint8_t b) { return b == 0x20 ? 0 : (b >= 0x61 && b <= 0x7A) ? b - 0x60 : -1; }

// One step of the prepared class table (compact states, computed-column layout).
inline uint32_t step(const Prepared& P, uint32_t s, uint8_t b) {
  const uint8_t* e = &P.table[(uint64_t)s * P.rowbytes + P.colmap[b]];
  if (P.esize == 1) return *e;
  uint16_t v;
  std::memcpy(&v, e, 2);
  return v;
}

// P with its states renumbered by pi (new id of old state s; a permutation of the non-accepting
// live states, the identity on the dead and accepting states): same DFA, same classes.
Prepared permute(const Prepared& P, const std::vector<uint32_t>& pi) {
  Prepared Q = P;
  const uint32_t n = P.n;
  const uint32_t ncols = ((P.win >> 8) & 0xFFu) + 4u;  // computed-column layout: w + 4 columns
  for (uint32_t s = 0; s < n; ++s)
    for (uint32_t c = 0; c < ncols; ++c) {
      const uint64_t from = (uint64_t)s * P.rowbytes + c * P.esize;
      const uint64_t to = (uint64_t)pi[s] * P.rowbytes + c * P.esize;
      uint32_t v = 0;
      std::memcpy(&v, &P.table[from], P.esize);
      v = pi[v];
      std::memcpy(&Q.table[to], &v, P.esize);
    }
  for (uint32_t s = 0; s < n; ++s) Q.orig_of[pi[s]] = P.orig_of[s];
  for (uint32_t q = 0; q < P.n_in; ++q) Q.compact_of[q] = pi[P.compact_of[q]];
  Q.start = pi[P.start];
  const uint32_t nl = (uint32_t)P.img_off.size() - 1;
  Q.rank.assign((uint64_t)nl * n, (uint16_t)kNoSlot);
  for (uint32_t c = 0; c < nl; ++c) {
    const uint32_t a = P.img_off[c], b = P.img_off[c + 1];
    std::vector<uint16_t> list;
    for (uint32_t k = a; k < b; ++k) list.push_back((uint16_t)pi[P.img[k]]);
    std::sort(list.begin(), list.end());
    for (uint32_t k = 0; k < list.size(); ++k) {
      Q.img[a + k] = list[k];
      Q.rank[(uint64_t)c * n + list[k]] = (uint16_t)k;
    }
  }
  return Q;
}

// Largest prepared table (class table and pair table): pass 1 then still runs kPairMaxWarps
// warps per block (2,752 bytes of stages, barriers and speculation scratch each) in the
// 227 KiB of shared memory a block may have, to cover the latency of the dependent lookups.
constexpr uint64_t kPairSmemCap = 160u << 10;
// Escape bytes after the last row of the pair table (see its construction).
constexpr uint64_t kPairPad = 144;
static_assert(27 * 31 + 31 - kPairRow < kPairPad, "pair table padding");
// Share of 32-lane vector steps allowed to need the byte loop (estimated on the sample).
constexpr double kPairMaxWarpSlow = 0.4;

}  // namespace

int plan_pairs(const Prepared& P, const uint8_t* sample, uint64_t nwin, uint64_t wlen, PairPlan* out) {
  out->ok = false;
  out->hot = 0;
  out->warp_slow = 1.0;
  const uint32_t k_live = P.first_accept - P.has_dead;  // non-accepting live states: 0 .. k-1
  if (P.layout != kClassWin || k_live < 2 || nwin == 0 || wlen < 16) return PAREM_OK;
  // visits per state, from the start state in every window (the first 64 bytes only settle
  // the run onto the text's states and are not counted)
  const uint64_t settle = std::min<uint64_t>(64, wlen / 4);
  std::vector<uint64_t> visits(P.n, 0);
  for (uint64_t k = 0; k < nwin; ++k) {
    uint32_t s = P.start;
    const uint8_t* w = sample + k * wlen;
    for (uint64_t j = 0; j < wlen; ++j) {
      s = step(P, s, w[j]);
      if (j >= settle) ++visits[s];
    }
  }
  // hot states: the most visited non-accepting live states (ties by id), at most 254 and as
  // many as fit the shared-memory cap next to the class table
  std::vector<uint32_t> order(k_live);
  std::iota(order.begin(), order.end(), 0u);
  std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return visits[a] > visits[b]; });
  const uint64_t main_bytes = (P.table_bytes + 15) & ~15ull;
  const uint64_t room = kPairSmemCap - std::min<uint64_t>(kPairSmemCap, main_bytes + kPairPad);
  const uint64_t fit = room >= 2 * kPairRow ? room / kPairRow - 1 : 0;
  uint32_t H = (uint32_t)std::min<uint64_t>({kPairMaxHot, (uint64_t)k_live, fit});
  while (H > 0 && visits[order[H - 1]] == 0) --H;
  if (H < 2) return PAREM_OK;
  std::vector<uint32_t> pi(P.n);
  std::iota(pi.begin(), pi.end(), 0u);
  for (uint32_t i = 0; i < k_live; ++i) pi[order[i]] = i;
  Prepared Q = permute(P, pi);
  // the pair table: rows 0 .. H-1 for the hot states, row H all escape, then kPairPad escape
  // bytes: a vector with a byte outside the set has codes up to 31 (index up to 27*31 + 31 =
  // 868 inside a row), and its lookups must still read entries <= H, inside the table
  std::vector<uint8_t> t2((uint64_t)(H + 1) * kPairRow + kPairPad, (uint8_t)H);
  for (uint32_t e = 0; e < H; ++e)
    for (uint32_t f0 = 0; f0 < kPairCodes; ++f0) {
      const uint32_t y = step(Q, e, code_byte(f0));
      for (uint32_t f1 = 0; f1 < kPairCodes; ++f1) {
        const uint32_t z = step(Q, y, code_byte(f1));
        const bool esc = y >= Q.first_accept || z >= Q.first_accept || z >= H;
        t2[(uint64_t)e * kPairRow + f0 * kPairCodes + f1] = (uint8_t)(esc ? H : z);
      }
    }
  // estimated share of 16-byte vectors (16-byte steps of a lane) that need the byte loop
  uint64_t vec = 0, slow = 0;
  for (uint64_t k = 0; k < nwin; ++k) {
    uint32_t s = Q.start;
    const uint8_t* w = sample + k * wlen;
    for (uint64_t j = 0; j + 16 <= wlen; j += 16) {
      bool fast = s < H;
      uint32_t e = std::min(s, H);
      for (int i = 0; i < 16 && fast; i += 2) {
        const int a = pair_code(w[j + i]), b = pair_code(w[j + i + 1]);
        if (a < 0 || b < 0) fast = false;
        else e = t2[(uint64_t)e * kPairRow + a * kPairCodes + b];
      }
      fast = fast && e < H;
      for (int i = 0; i < 16; ++i) s = step(Q, s, w[j + i]);
      if (j >= settle) {
        ++vec;
        slow += fast ? 0 : 1;
      }
    }
  }
  const double p_slow = vec ? (double)slow / (double)vec : 1.0;
  out->warp_slow = 1.0 - std::pow(1.0 - p_slow, 32.0);
  out->hot = H;
  out->hot_orig.resize(H);
  for (uint32_t e = 0; e < H; ++e) out->hot_orig[e] = Q.orig_of[e];
  Q.layout = kClassPair;
  Q.pair_hot = H;
  Q.main_bytes = (uint32_t)main_bytes;
  Q.pair_off = (uint32_t)main_bytes;
  Q.table.resize(main_bytes + ((t2.size() + 15) & ~(size_t)15), 0);
  std::memcpy(Q.table.data() + main_bytes, t2.data(), t2.size());
  Q.table_bytes = (uint32_t)Q.table.size();
  out->Q = std::move(Q);
  out->ok = out->warp_slow <= kPairMaxWarpSlow;
  return PAREM_OK;
}

int learn_pairs(parem_dfa* dfa, const uint8_t* text, uint64_t len, cudaStream_t stream) {
  auto give_up = [&](int rc) {
    dfa->pair_state.store(kPairOff, std::memory_order_release);
    return rc;
  };
  if (dfa->host.layout != kClassWin) return give_up(PAREM_OK);
  // sample: up to 64 windows of 64 KiB spread over the text (the whole text when short)
  uint64_t nwin = 64, wlen = std::min<uint64_t>(64u << 10, len / 64) & ~15ull;
  if (wlen < 4096) {
    nwin = 1;
    wlen = std::min<uint64_t>(len, 4u << 20);
  }
  std::vector<uint8_t> buf(nwin * wlen);
  for (uint64_t k = 0; k < nwin; ++k) {
    const uint64_t off = nwin == 1 ? 0 : (len - wlen) / (nwin - 1) * k;
    if (cudaMemcpyAsync(buf.data() + k * wlen, text + off, wlen, cudaMemcpyDeviceToHost, stream) != cudaSuccess)
      return give_up(PAREM_ERR_CUDA);
  }
  if (cudaStreamSynchronize(stream) != cudaSuccess) return give_up(PAREM_ERR_CUDA);
  PairPlan pp;
  plan_pairs(dfa->host, buf.data(), nwin, wlen, &pp);
  if (!pp.ok) return give_up(PAREM_OK);
  DeviceDfa D{};
  void* mem = nullptr;
  const int rc = upload_prepared(pp.Q, &D, &mem);
  if (rc != PAREM_OK) return give_up(rc);
  dfa->pair_host = std::move(pp.Q);
  dfa->pair_dev = D;
  dfa->pair_mem = mem;
  dfa->pair_state.store(kPairReady, std::memory_order_release);
  return PAREM_OK;
}

}  // namespace parem

// Host-only preview of the pair variant (no GPU): see include/parem.h.
extern "C" int parem_pair_preview(const uint32_t* table, uint32_t n_states, uint32_t n_symbols,
                                  const uint16_t* byte_to_symbol, uint32_t start, const uint8_t* accept,
                                  const uint8_t* sample, uint64_t sample_len, parem_pair_info* info,
                                  uint32_t* hot_states, uint8_t* pair_table, uint64_t pair_table_cap) {
  if (!info || (sample_len > 0 && !sample)) return PAREM_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  parem::Prepared P;
  int rc = parem::prepare_dfa(table, n_states, n_symbols, byte_to_symbol, start, accept, 160u << 10, &P);
  if (rc != PAREM_OK) return rc;
  info->layout = P.layout;
  parem::PairPlan pp;
  parem::plan_pairs(P, sample, 1, sample_len, &pp);
  info->hot_states = pp.hot;
  info->accepted = pp.ok ? 1u : 0u;
  info->warp_slow_share = pp.warp_slow;
  if (pp.hot == 0) return PAREM_OK;
  info->pair_table_bytes = (uint64_t)(pp.hot + 1) * parem::kPairRow;
  if (hot_states)
    for (uint32_t e = 0; e < pp.hot; ++e) hot_states[e] = pp.hot_orig[e];
  if (pair_table) {
    if (pair_table_cap < info->pair_table_bytes) return PAREM_ERR_CAPACITY;
    std::memcpy(pair_table, pp.Q.table.data() + pp.Q.pair_off, info->pair_table_bytes);
  }
  return PAREM_OK;
}
