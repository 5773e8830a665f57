// parem_regex.cpp -- host front-end: a regular expression (the operators of Table III:
// concatenation, Kleene star, union, positive closure, range, optionality, group) compiled
// to a DFA table for parem_load_dfa.
//
// The pipeline follows the paper's Section III (Implementation): the expression is parsed into a syntax tree
// by a recursive-descent parser of the operator grammar (precedence, lowest first: union,
// concatenation, the postfix quantifiers * + ?); the tree becomes an NFA by the
// McNaughton-Yamada-Thompson construction (one fragment per node, joined by empty
// transitions); the subset construction turns the NFA into a DFA.  Bytes that every NFA
// edge treats alike share one DFA symbol (byte classes), so the table has one column per
// class; the DFA is then minimized (Moore's partition refinement).  For a search (the
// default) the NFA's start state also loops on every byte, so the DFA accepts after
// position j exactly when some suffix of text[0..j], possibly empty, matches (Sigma* R);
// anchored compilation accepts when text[0..j] matches.
//
// Syntax: a byte stands for itself; '\' escapes the next byte (\n \t \r \0 \xHH as usual);
// '.' is any byte; [..] is a set of bytes and ranges, written a-z or (as in the paper)
// a..z, negated by a leading '^'; ( ) groups; | * + ? as in Table III.  An empty
// alternative matches the empty string.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/parem.h"

namespace {

using ByteSet = std::vector<bool>;  // 256 flags
constexpr uint64_t kMaxPattern = 16384;  // pattern bytes

struct Node {
  enum Kind { kBytes, kEmpty, kConcat, kUnion, kStar, kPlus, kOpt } kind;
  ByteSet bytes;          // kBytes
  std::vector<int> kids;  // kConcat, kUnion: two; quantifiers: one
};

struct Parser {
  const uint8_t* s;
  size_t n, i = 0;
  std::vector<Node> nodes;
  bool ok = true;

  int add(Node nd) {
    nodes.push_back(std::move(nd));
    return (int)nodes.size() - 1;
  }
  bool more() const { return i < n; }
  uint8_t peek() const { return s[i]; }

  static int hexval(uint8_t c) {
    if (c >= '0' && c <= '9') return c - '0';
    if (c >= 'a' && c <= 'f') return c - 'a' + 10;
    if (c >= 'A' && c <= 'F') return c - 'A' + 10;
    return -1;
  }
  // one byte after a backslash
  int escaped() {
    if (!more()) {
      ok = false;
      return 0;
    }
    const uint8_t c = s[i++];
    switch (c) {
      case 'n': return '\n';
      case 't': return '\t';
      case 'r': return '\r';
      case '0': return 0;
      case 'x': {
        if (i + 2 > n || hexval(s[i]) < 0 || hexval(s[i + 1]) < 0) {
          ok = false;
          return 0;
        }
        const int v = hexval(s[i]) * 16 + hexval(s[i + 1]);
        i += 2;
        return v;
      }
      default: return c;
    }
  }
  // a byte inside a set: escaped or literal
  int set_byte() {
    if (!more()) {
      ok = false;
      return 0;
    }
    const uint8_t c = s[i++];
    return c == '\\' ? escaped() : c;
  }
  int parse_set() {  // after '['
    ByteSet b(256, false);
    bool neg = false;
    if (more() && peek() == '^') {
      neg = true;
      ++i;
    }
    bool first = true;
    while (more() && (peek() != ']' || first)) {
      first = false;
      const int lo = set_byte();
      int hi = lo;
      if (i + 1 < n && s[i] == '.' && s[i + 1] == '.') {  // the paper's a..z
        i += 2;
        hi = set_byte();
      } else if (i + 1 < n && s[i] == '-' && s[i + 1] != ']') {
        i += 1;
        hi = set_byte();
      }
      if (!ok || hi < lo) {
        ok = false;
        return -1;
      }
      for (int c = lo; c <= hi; ++c) b[c] = true;
    }
    if (!more()) {
      ok = false;
      return -1;
    }
    ++i;  // ']'
    if (neg)
      for (int c = 0; c < 256; ++c) b[c] = !b[c];
    return add(Node{Node::kBytes, b, {}});
  }
  int atom() {
    const uint8_t c = s[i];
    if (c == '(') {
      ++i;
      const int e = alt();
      if (!ok || !more() || peek() != ')') {
        ok = false;
        return -1;
      }
      ++i;
      return e;
    }
    if (c == '[') {
      ++i;
      return parse_set();
    }
    ++i;
    ByteSet b(256, false);
    if (c == '.') {
      b.assign(256, true);
    } else if (c == '\\') {
      b[escaped()] = true;
    } else if (c == '*' || c == '+' || c == '?' || c == ')') {
      ok = false;  // a quantifier with nothing to repeat, or an unopened group
      return -1;
    } else {
      b[c] = true;
    }
    return add(Node{Node::kBytes, b, {}});
  }
  int repeat() {
    int e = atom();
    while (ok && more() && (peek() == '*' || peek() == '+' || peek() == '?')) {
      const uint8_t q = s[i++];
      e = add(Node{q == '*' ? Node::kStar : q == '+' ? Node::kPlus : Node::kOpt, {}, {e}});
    }
    return e;
  }
  int concat() {
    int e = -1;
    while (ok && more() && peek() != '|' && peek() != ')') {
      const int r = repeat();
      e = e < 0 ? r : add(Node{Node::kConcat, {}, {e, r}});
    }
    return e < 0 ? add(Node{Node::kEmpty, {}, {}}) : e;
  }
  int alt() {
    int e = concat();
    while (ok && more() && peek() == '|') {
      ++i;
      const int r = concat();
      e = add(Node{Node::kUnion, {}, {e, r}});
    }
    return e;
  }
};

// Thompson NFA: every state has at most one byte-set edge and any number of empty edges.
struct Nfa {
  std::vector<int> set_of;                // per state: index into sets (-1: none)
  std::vector<int> next;                  // per state: target of the byte-set edge
  std::vector<std::vector<int>> eps;      // per state: empty-edge targets
  std::vector<ByteSet> sets;

  int state() {
    set_of.push_back(-1);
    next.push_back(-1);
    eps.emplace_back();
    return (int)set_of.size() - 1;
  }
  // fragment of node k: (entry, exit)
  std::pair<int, int> build(const std::vector<Node>& t, int k) {
    const Node& nd = t[k];
    switch (nd.kind) {
      case Node::kBytes: {
        const int a = state(), b = state();
        sets.push_back(nd.bytes);
        set_of[a] = (int)sets.size() - 1;
        next[a] = b;
        return {a, b};
      }
      case Node::kEmpty: {
        const int a = state(), b = state();
        eps[a].push_back(b);
        return {a, b};
      }
      case Node::kConcat: {
        const auto x = build(t, nd.kids[0]);
        const auto y = build(t, nd.kids[1]);
        eps[x.second].push_back(y.first);
        return {x.first, y.second};
      }
      case Node::kUnion: {
        const auto x = build(t, nd.kids[0]);
        const auto y = build(t, nd.kids[1]);
        const int a = state(), b = state();
        eps[a].push_back(x.first);
        eps[a].push_back(y.first);
        eps[x.second].push_back(b);
        eps[y.second].push_back(b);
        return {a, b};
      }
      default: {  // quantifiers around fragment x
        const auto x = build(t, nd.kids[0]);
        const int a = state(), b = state();
        eps[a].push_back(x.first);
        if (nd.kind != Node::kPlus) eps[a].push_back(b);   // zero occurrences (* and ?)
        eps[x.second].push_back(b);
        if (nd.kind != Node::kOpt) eps[x.second].push_back(x.first);  // repeat (* and +)
        return {a, b};
      }
    }
  }
};

// Moore's partition refinement: the minimal DFA of the same language.  The empty subset
// (no match can continue: table entry PAREM_NONE) is an explicit dead state during the
// refinement and PAREM_NONE again afterwards; the start state keeps number 0.
void minimize(uint32_t& n, uint32_t k, std::vector<uint32_t>& table, std::vector<uint8_t>& accept) {
  const uint32_t dead = n;  // extra state: every transition to itself, not accepting
  auto next = [&](uint32_t q, uint32_t c) -> uint32_t {
    if (q == dead) return dead;
    const uint32_t t = table[(uint64_t)q * k + c];
    return t == PAREM_NONE ? dead : t;
  };
  std::vector<uint32_t> cls(n + 1);
  for (uint32_t q = 0; q < n; ++q) cls[q] = accept[q] ? 1u : 0u;
  cls[dead] = 0;
  uint32_t n_cls = 0;
  for (;;) {
    std::map<std::vector<uint32_t>, uint32_t> id;
    std::vector<uint32_t> nc(n + 1);
    std::vector<uint32_t> sig(k + 1);
    for (uint32_t q = 0; q <= n; ++q) {
      sig[0] = cls[q];
      for (uint32_t c = 0; c < k; ++c) sig[c + 1] = cls[next(q, c)];
      nc[q] = id.emplace(sig, (uint32_t)id.size()).first->second;
    }
    const uint32_t m = (uint32_t)id.size();
    cls.swap(nc);
    if (m == n_cls) break;
    n_cls = m;
  }
  // new numbering: the start's class first, the dead class dropped
  const uint32_t dead_cls = cls[dead];
  std::vector<uint32_t> renum(n_cls, PAREM_NONE);
  uint32_t m = 0;
  renum[cls[0]] = m++;
  for (uint32_t q = 0; q < n; ++q)
    if (cls[q] != dead_cls && renum[cls[q]] == PAREM_NONE) renum[cls[q]] = m++;
  std::vector<uint32_t> t2((uint64_t)m * k, PAREM_NONE);
  std::vector<uint8_t> a2(m, 0);
  std::vector<char> done(m, 0);
  for (uint32_t q = 0; q < n; ++q) {
    const uint32_t r = renum[cls[q]];
    if (r == PAREM_NONE || done[r]) continue;
    done[r] = 1;
    a2[r] = accept[q];
    for (uint32_t c = 0; c < k; ++c) {
      const uint32_t t = next(q, c);
      t2[(uint64_t)r * k + c] = (t == dead || cls[t] == dead_cls) ? PAREM_NONE : renum[cls[t]];
    }
  }
  n = m;
  table.swap(t2);
  accept.swap(a2);
}

}  // namespace

struct parem_regex {
  uint32_t n_states = 0, n_symbols = 0, start = 0;
  std::vector<uint32_t> table;   // n_states * n_symbols, PAREM_NONE for the empty subset
  std::vector<uint16_t> byte_to_symbol;
  std::vector<uint8_t> accept;
};

extern "C" int parem_regex_compile(const char* pattern, uint64_t len, uint32_t flags, uint32_t max_states,
                                   parem_regex** out) {
  if (!out || (len > 0 && !pattern) || (flags & ~PAREM_REGEX_ANCHORED)) return PAREM_ERR_INVALID_ARG;
  *out = nullptr;
  if (len > kMaxPattern) return PAREM_ERR_TOO_LARGE;  // the tree is built and walked recursively
  const uint32_t limit = max_states ? std::min<uint32_t>(max_states, 65535u) : 65535u;
  Parser ps{reinterpret_cast<const uint8_t*>(pattern), (size_t)len};
  const int root = ps.alt();
  if (!ps.ok || ps.more() || root < 0) return PAREM_ERR_INVALID_ARG;  // syntax error

  Nfa nfa;
  const auto frag = nfa.build(ps.nodes, root);
  const int accept_state = frag.second;
  const bool search = !(flags & PAREM_REGEX_ANCHORED);
  // Sigma* R: a start state that loops on every byte and enters R
  int nfa_start = frag.first;
  if (search) {
    const int loop = nfa.state();
    nfa.sets.push_back(ByteSet(256, true));
    nfa.set_of[loop] = (int)nfa.sets.size() - 1;
    nfa.next[loop] = loop;
    nfa.eps[loop].push_back(frag.first);
    nfa_start = loop;
  }

  // byte classes: bytes with the same membership in every edge set
  std::map<std::vector<bool>, uint16_t> cls_of_sig;
  std::vector<uint16_t> cls(256);
  std::vector<int> rep;  // a byte of each class
  for (int b = 0; b < 256; ++b) {
    std::vector<bool> sig(nfa.sets.size());
    for (size_t k = 0; k < nfa.sets.size(); ++k) sig[k] = nfa.sets[k][b];
    auto it = cls_of_sig.find(sig);
    if (it == cls_of_sig.end()) {
      it = cls_of_sig.emplace(sig, (uint16_t)rep.size()).first;
      rep.push_back(b);
    }
    cls[b] = it->second;
  }
  const uint32_t n_sym = (uint32_t)rep.size();

  // subset construction
  const size_t ns = nfa.set_of.size();
  auto closure = [&](std::vector<int> seed) {
    std::vector<char> in(ns, 0);
    std::vector<int> stack;
    for (int q : seed)
      if (!in[q]) {
        in[q] = 1;
        stack.push_back(q);
      }
    while (!stack.empty()) {
      const int q = stack.back();
      stack.pop_back();
      for (int r : nfa.eps[q])
        if (!in[r]) {
          in[r] = 1;
          stack.push_back(r);
        }
    }
    std::vector<int> sorted;
    for (size_t q = 0; q < ns; ++q)
      if (in[q]) sorted.push_back((int)q);
    return sorted;
  };
  auto* re = new (std::nothrow) parem_regex();
  if (!re) return PAREM_ERR_OOM;
  std::map<std::vector<int>, uint32_t> id_of;
  std::vector<std::vector<int>> subsets;
  const auto s0 = closure({nfa_start});
  id_of.emplace(s0, 0u);
  subsets.push_back(s0);
  for (size_t d = 0; d < subsets.size(); ++d) {
    const std::vector<int> cur = subsets[d];
    for (uint32_t c = 0; c < n_sym; ++c) {
      std::vector<int> moved;
      for (int q : cur)
        if (nfa.set_of[q] >= 0 && nfa.sets[nfa.set_of[q]][rep[c]]) moved.push_back(nfa.next[q]);
      if (moved.empty()) {
        re->table.push_back(PAREM_NONE);
        continue;
      }
      const auto nxt = closure(moved);
      auto it = id_of.find(nxt);
      if (it == id_of.end()) {
        if (subsets.size() >= limit) {
          delete re;
          return PAREM_ERR_TOO_LARGE;
        }
        it = id_of.emplace(nxt, (uint32_t)subsets.size()).first;
        subsets.push_back(nxt);
      }
      re->table.push_back(it->second);
    }
  }
  re->n_states = (uint32_t)subsets.size();
  re->n_symbols = n_sym;
  re->start = 0;
  re->byte_to_symbol = cls;
  re->accept.resize(re->n_states);
  for (uint32_t q = 0; q < re->n_states; ++q) {
    re->accept[q] = 0;
    for (int x : subsets[q])
      if (x == accept_state) re->accept[q] = 1;
  }
  // the subset construction can leave equivalent states (e.g. the start subset of a search);
  // the scan prefers the minimal DFA: fewer states, fewer speculation candidates
  minimize(re->n_states, re->n_symbols, re->table, re->accept);
  *out = re;
  return PAREM_OK;
}

extern "C" int parem_regex_info(const parem_regex* re, uint32_t* n_states, uint32_t* n_symbols) {
  if (!re || !n_states || !n_symbols) return PAREM_ERR_INVALID_ARG;
  *n_states = re->n_states;
  *n_symbols = re->n_symbols;
  return PAREM_OK;
}

extern "C" int parem_regex_export(const parem_regex* re, uint32_t* table, uint16_t* byte_to_symbol,
                                  uint8_t* accept, uint32_t* start) {
  if (!re || !table || !byte_to_symbol || !accept || !start) return PAREM_ERR_INVALID_ARG;
  std::memcpy(table, re->table.data(), re->table.size() * sizeof(uint32_t));
  std::memcpy(byte_to_symbol, re->byte_to_symbol.data(), 256 * sizeof(uint16_t));
  std::memcpy(accept, re->accept.data(), re->accept.size());
  *start = re->start;
  return PAREM_OK;
}

extern "C" int parem_regex_load(const parem_regex* re, parem_dfa** out) {
  if (!re || !out) return PAREM_ERR_INVALID_ARG;
  return parem_load_dfa(re->table.data(), re->n_states, re->n_symbols, re->byte_to_symbol.data(), re->start,
                        re->accept.data(), out);
}

extern "C" void parem_regex_free(parem_regex* re) { delete re; }
