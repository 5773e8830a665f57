// parem_prep.cpp -- host-side preparation of a DFA for the GPU scan (no CUDA calls).
//
// Input is the DFA (Q, Sigma, delta, q0, F) of Section II-A with the byte -> symbol map.
// Output (parem::Prepared) is what the kernels read:
//   * completion with an explicit dead state when some transition is undefined or some
//     byte lies outside the alphabet (the "not in Q" case of Algorithm 1's tests);
//   * renumbering: non-accepting states first, then the dead state, then the accepting
//     states, so "state in F" is one comparison with first_accept;
//   * byte classes: bytes whose symbols have identical transition columns share a class;
//   * the transition table, either byte-indexed (256 columns: no class lookup in the hot
//     loop) or class-indexed, with a row pitch chosen to spread rows over the 32 banks;
//   * for every class c the candidate list img(c): the distinct states reached on c from
//     any state, without the dead state (the set L of Algorithm 1; S n L for a complete
//     DFA, and the dead state needs no simulation), plus one extra list with every live
//     state for the enumeration mode;
//   * rank(c, q): slot of state q in img(c), used to read a chunk map at its true start.
#include <algorithm>
#include <cstring>
#include <map>
#include <unordered_map>

#include "../../include/parem.h"
#include "parem_internal.h"

namespace parem {

namespace {

struct VecHash {
  size_t operator()(const std::vector<uint32_t>& v) const {
    uint64_t h = 1469598103934665603ull;
    for (uint32_t x : v) {
      h ^= x;
      h *= 1099511628211ull;
    }
    return (size_t)h;
  }
};

// Row pitch in bytes: a multiple of the entry size whose word stride is odd when it is a
// whole number of words, so consecutive rows start in different banks.
uint32_t row_pitch(uint32_t cols, uint32_t esize) {
  uint32_t rb = cols * esize;
  if (rb % 4 == 0 && (rb / 4) % 2 == 0) rb += 4;
  return rb;
}

}  // namespace

// How many symbols a speculative candidate set needs before it shrinks to one state, for the
// planner's row length: median over 5 seeded trials, each starting from the candidate set of
// a random live class and driven by live classes drawn uniformly (splitmix64).  A trial that
// has not synchronised when its work (the sum of the set sizes) reaches 2^24 gives kNoSync.
uint32_t estimate_sync(const std::vector<std::vector<uint32_t>>& cols, const Prepared& P) {
  std::vector<uint32_t> live;
  for (uint32_t c = 0; c < P.n_classes; ++c)
    if (P.img_off[c + 1] - P.img_off[c] > 0) live.push_back(c);
  if (live.empty() || P.max_cand <= 1) return 0;
  uint64_t x = 0x9E3779B97F4A7C15ull ^ P.n;
  auto next_rand = [&x]() {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  std::vector<uint32_t> res;
  std::vector<uint32_t> cur, nxt;
  std::vector<uint32_t> mark(P.n, 0);
  uint32_t stamp = 0;
  for (int trial = 0; trial < 5; ++trial) {
    const uint32_t c0 = live[next_rand() % live.size()];
    cur.assign(P.img.begin() + P.img_off[c0], P.img.begin() + P.img_off[c0 + 1]);
    uint64_t work = 0;
    uint32_t t = 0;
    bool sync = true;
    while (cur.size() > 1) {
      if (work > (1ull << 24)) {
        sync = false;
        break;
      }
      const uint32_t c = live[next_rand() % live.size()];
      ++stamp;
      nxt.clear();
      for (uint32_t q : cur) {
        const uint32_t r = cols[c][q];
        if (r == P.dead || mark[r] == stamp) continue;
        mark[r] = stamp;
        nxt.push_back(r);
      }
      work += cur.size();
      cur.swap(nxt);
      ++t;
    }
    res.push_back(sync ? t : kNoSync);
  }
  std::sort(res.begin(), res.end());
  return res[res.size() / 2];
}

int prepare_dfa(const uint32_t* table, uint32_t n_states, uint32_t n_symbols,
                const uint16_t* byte_to_symbol, uint32_t start, const uint8_t* accept,
                uint32_t smem_table_budget, Prepared* out) {
  if (!table || !accept || !out) return PAREM_ERR_INVALID_ARG;
  if (n_states < 1 || n_states > 65535 || n_symbols < 1 || n_symbols > 256 || start >= n_states)
    return PAREM_ERR_INVALID_ARG;
  const uint64_t cells = (uint64_t)n_states * n_symbols;
  bool any_none = false;
  for (uint64_t i = 0; i < cells; ++i) {
    if (table[i] == PAREM_NONE) {
      any_none = true;
    } else if (table[i] >= n_states) {
      return PAREM_ERR_INVALID_ARG;
    }
  }
  // symbol of each byte
  uint32_t sym[256];
  bool byte_outside = false;
  for (int b = 0; b < 256; ++b) {
    uint32_t a;
    if (byte_to_symbol) {
      a = byte_to_symbol[b];
      if (a == PAREM_NONE16) {
        a = PAREM_NONE;
      } else if (a >= n_symbols) {
        return PAREM_ERR_INVALID_ARG;
      }
    } else {
      a = (uint32_t)b < n_symbols ? (uint32_t)b : PAREM_NONE;
    }
    sym[b] = a;
    if (a == PAREM_NONE) byte_outside = true;
  }
  // A dead state is needed when an undefined entry can be used by some byte, or a byte is
  // outside the alphabet.
  bool used_sym[256] = {false};
  for (int b = 0; b < 256; ++b)
    if (sym[b] != PAREM_NONE) used_sym[sym[b]] = true;
  bool none_used = false;
  if (any_none) {
    for (uint32_t q = 0; q < n_states && !none_used; ++q)
      for (uint32_t a = 0; a < n_symbols; ++a)
        if (used_sym[a] && table[(uint64_t)q * n_symbols + a] == PAREM_NONE) {
          none_used = true;
          break;
        }
  }
  Prepared P;
  P.n_in = n_states;
  P.n_sym = n_symbols;
  P.has_dead = (none_used || byte_outside) ? 1 : 0;
  P.n = n_states + P.has_dead;
  // renumber: non-accepting, dead, accepting
  P.compact_of.assign(n_states, 0);
  P.orig_of.assign(P.n, 0);
  uint32_t next = 0;
  for (uint32_t q = 0; q < n_states; ++q)
    if (!accept[q]) {
      P.compact_of[q] = next;
      P.orig_of[next++] = q;
    }
  if (P.has_dead) {
    P.dead = next;
    P.orig_of[next++] = PAREM_NONE;
  }
  P.first_accept = next;
  for (uint32_t q = 0; q < n_states; ++q)
    if (accept[q]) {
      P.compact_of[q] = next;
      P.orig_of[next++] = q;
    }
  P.start = P.compact_of[start];
  const uint32_t n = P.n;

  // transition column of a symbol over compact states (dead row -> dead)
  auto column = [&](uint32_t a) {
    std::vector<uint32_t> col(n);
    for (uint32_t c = 0; c < n; ++c) {
      uint32_t q = P.orig_of[c];
      if (q == PAREM_NONE || a == PAREM_NONE) {
        col[c] = P.dead;
      } else {
        uint32_t e = table[(uint64_t)q * n_symbols + a];
        col[c] = e == PAREM_NONE ? P.dead : P.compact_of[e];
      }
    }
    return col;
  };
  // classes over the symbols the bytes use (NONE is its own column)
  std::unordered_map<std::vector<uint32_t>, uint32_t, VecHash> cls_of_col;
  std::vector<std::vector<uint32_t>> cols;
  std::map<uint32_t, uint32_t> cls_of_sym;
  P.byte_class.assign(256, 0);
  for (int b = 0; b < 256; ++b) {
    uint32_t a = sym[b];
    auto it = cls_of_sym.find(a);
    if (it == cls_of_sym.end()) {
      std::vector<uint32_t> col = column(a);
      auto jt = cls_of_col.find(col);
      uint32_t c;
      if (jt == cls_of_col.end()) {
        c = (uint32_t)cols.size();
        cls_of_col.emplace(col, c);
        cols.push_back(std::move(col));
      } else {
        c = jt->second;
      }
      it = cls_of_sym.emplace(a, c).first;
    }
    P.byte_class[b] = (uint16_t)it->second;
  }
  P.n_classes = (uint32_t)cols.size();

  // layout
  P.esize = n <= 256 ? 1 : 2;
  const uint32_t rb_byte = row_pitch(256, P.esize);
  const uint32_t rb_cls = row_pitch(P.n_classes, P.esize);
  if ((uint64_t)n * rb_byte <= smem_table_budget) {
    P.layout = kByteSmem;
    P.rowbytes = rb_byte;
  } else if ((uint64_t)n * rb_cls <= smem_table_budget) {
    P.layout = kClassSmem;
    P.rowbytes = rb_cls;
  } else {
    P.layout = kClassGlobal;
    P.rowbytes = rb_cls;
  }
  // column offsets that do not fit a byte need the wide column map
  if (P.layout != kByteSmem && (P.n_classes - 1) * P.esize > 255)
    P.layout = P.layout == kClassSmem ? kClassSmemW : kClassGlobalW;
  uint64_t tbytes = (uint64_t)n * P.rowbytes;
  tbytes = (tbytes + 15) & ~15ull;
  if (tbytes > 0xFFFFFFFFull) return PAREM_ERR_UNSUPPORTED;
  P.table_bytes = (uint32_t)tbytes;
  P.table.assign(P.table_bytes, 0);
  auto put = [&](uint32_t s, uint32_t colbyte, uint32_t v) {
    uint8_t* p = &P.table[(uint64_t)s * P.rowbytes + colbyte];
    if (P.esize == 1) {
      *p = (uint8_t)v;
    } else {
      uint16_t w = (uint16_t)v;
      std::memcpy(p, &w, 2);
    }
  };
  P.colmap.assign(256, 0);
  if (P.layout == kByteSmem) {
    for (int b = 0; b < 256; ++b) {
      const auto& col = cols[P.byte_class[b]];
      for (uint32_t s = 0; s < n; ++s) put(s, (uint32_t)b * P.esize, col[s]);
      P.colmap[b] = (uint16_t)(b * P.esize);
    }
  } else {
    for (uint32_t c = 0; c < P.n_classes; ++c)
      for (uint32_t s = 0; s < n; ++s) put(s, c * P.esize, cols[c][s]);
    for (int b = 0; b < 256; ++b) P.colmap[b] = (uint16_t)(P.byte_class[b] * P.esize);
  }

  // Computed columns: when every byte outside one window [lo, lo + w) of ASCII (w <= 64) and
  // one extra byte xb shares a single class, the column of a byte is arithmetic, so the scan
  // needs no column-map lookup per byte: column min(b - lo + 2, w + 2) (unsigned; window
  // bytes 2.., every byte below or above the window w + 2, and the bytes lo - 2, lo - 1 land
  // on columns 0, 1), except xb -> w + 3.  Columns 0, 1 and w + 2 hold the shared class.
  // The table then has w + 4 columns (each window byte its own, even where classes repeat);
  // it must fit shared memory.
  if (P.layout != kByteSmem && P.n_classes >= 2) {
    std::vector<uint32_t> freq(P.n_classes, 0);
    for (int b = 0; b < 256; ++b) freq[P.byte_class[b]]++;
    uint32_t other = 0;
    for (uint32_t c = 1; c < P.n_classes; ++c)
      if (freq[c] > freq[other]) other = c;
    std::vector<int> B;
    int other_byte = -1;
    for (int b = 0; b < 256; ++b) {
      if (P.byte_class[b] != other) B.push_back(b);
      else if (other_byte < 0) other_byte = b;
    }
    int lo = -1, w = 0, xb = other_byte;
    auto fits = [](int l, int h) { return l >= 0 && h < 128 && h - l + 1 <= 64; };
    if (!B.empty() && fits(B.front(), B.back())) {
      lo = B.front();
      w = B.back() - lo + 1;
    } else if (B.size() >= 2 && fits(B[1], B.back())) {
      lo = B[1];
      w = B.back() - lo + 1;
      xb = B.front();
    } else if (B.size() >= 2 && fits(B.front(), B[B.size() - 2])) {
      lo = B.front();
      w = B[B.size() - 2] - lo + 1;
      xb = B.back();
    }
    const uint32_t rb_win = row_pitch((uint32_t)w + 4, P.esize);
    if (lo >= 0 && xb >= 0 && (uint64_t)n * rb_win <= smem_table_budget) {
      P.layout = kClassWin;
      P.rowbytes = rb_win;
      P.table_bytes = (uint32_t)(((uint64_t)n * rb_win + 15) & ~15ull);
      P.table.assign(P.table_bytes, 0);
      auto column_of = [&](int b) -> uint32_t {
        if (b == xb) return (uint32_t)w + 3u;
        if (b >= lo && b < lo + w) return 2u + (uint32_t)(b - lo);
        if (b == lo - 2 || b == lo - 1) return (uint32_t)(b - lo + 2);
        return (uint32_t)w + 2u;
      };
      std::vector<int> rep(w + 4, other_byte);
      rep[w + 3] = xb;
      for (int i = 0; i < w; ++i) rep[2 + i] = lo + i;
      for (uint32_t c = 0; c < (uint32_t)w + 4; ++c)
        for (uint32_t s = 0; s < n; ++s) put(s, c * P.esize, cols[P.byte_class[rep[c]]][s]);
      for (int b = 0; b < 256; ++b) P.colmap[b] = (uint16_t)(column_of(b) * P.esize);
      P.win = (uint32_t)lo | ((uint32_t)w << 8) | ((uint32_t)xb << 16);
    }
  }

  // Multi-stride table: for a small DFA (<= 32 compact states) whose bytes 0..K-2 are classes
  // 0..K-2 and whose other bytes all share class K-1, one lookup advances 4 bytes.  Entry for
  // (state s, bytes b1..b4) at s * K^4 + ((m1 * K + m2) * K + m3) * K + m4, m = min(b, K - 1):
  // the state after the 4 bytes (5 bits) and how many of the 4 states after each byte are
  // accepting (3 bits).  The main run of the scan uses it; every other step stays byte-wise.
  if (P.layout == kByteSmem && n <= 32 && P.n_classes >= 2) {
    const uint32_t K = P.n_classes;
    bool ok = K <= 16;
    for (int b = 0; b < 256 && ok; ++b) ok = P.byte_class[b] == std::min<uint32_t>((uint32_t)b, K - 1);
    const uint64_t k4 = (uint64_t)K * K * K * K;
    if (ok && (uint64_t)n * k4 <= (48u << 10)) {
      const uint32_t off = P.table_bytes;
      P.table.resize(off + (((uint64_t)n * k4 + 15) & ~15ull), 0);
      for (uint32_t s = 0; s < n; ++s)
        for (uint64_t idx = 0; idx < k4; ++idx) {
          const uint32_t d[4] = {(uint32_t)(idx / (K * K * K)), (uint32_t)(idx / (K * K) % K),
                                 (uint32_t)(idx / K % K), (uint32_t)(idx % K)};
          uint32_t x = s, cnt = 0;
          for (int i = 0; i < 4; ++i) {
            x = cols[d[i]][x];
            cnt += x >= P.first_accept ? 1u : 0u;
          }
          P.table[off + (uint64_t)s * k4 + idx] = (uint8_t)(x | (cnt << 5));
        }
      P.table_bytes = (uint32_t)P.table.size();
      P.layout = kByteStride;
      P.stride_k = K;
      P.stride_off = off;
    }
  }

  // candidate lists and ranks; list n_classes holds every live state (enumeration mode)
  const uint32_t nl = P.n_classes + 1;
  P.img_off.assign(nl + 1, 0);
  P.rank.assign((uint64_t)nl * n, (uint16_t)kNoSlot);
  std::vector<uint8_t> seen(n);
  P.max_cand = 0;
  for (uint32_t c = 0; c < nl; ++c) {
    std::fill(seen.begin(), seen.end(), 0);
    if (c < P.n_classes) {
      for (uint32_t s = 0; s < n; ++s) seen[cols[c][s]] = 1;
    } else {
      std::fill(seen.begin(), seen.end(), 1);
    }
    P.img_off[c] = (uint32_t)P.img.size();
    for (uint32_t s = 0; s < n; ++s) {
      if (!seen[s] || s == P.dead) continue;
      P.rank[(uint64_t)c * n + s] = (uint16_t)(P.img.size() - P.img_off[c]);
      P.img.push_back((uint16_t)s);
    }
    uint32_t m = (uint32_t)P.img.size() - P.img_off[c];
    if (c < P.n_classes) P.max_cand = std::max(P.max_cand, m);
  }
  P.img_off[nl] = (uint32_t)P.img.size();
  double tot = 0;
  for (int b = 0; b < 256; ++b) {
    uint32_t c = P.byte_class[b];
    tot += P.img_off[c + 1] - P.img_off[c];
  }
  P.mean_cand = tot / 256.0;
  P.sync_len = estimate_sync(cols, P);
  if (P.img.empty()) P.img.push_back(0);
  *out = std::move(P);
  return PAREM_OK;
}

}  // namespace parem
