"""Seeded synthetic inputs: DFAs and texts shaped like the workloads of the paper.

This module only BUILDS inputs (transition tables, accept sets, byte maps and texts).  It
never runs a DFA over a text, so it holds none of the matching arithmetic; both the CUDA
path and the CPU oracle consume what it produces.

DFA builders
  kmp_dfa             -- the string-matching automaton of one literal (the automaton of
                         Fig. 1 / Table I is kmp_dfa("parallel") over {p,a,r,e,l}).
  aho_corasick_dfa    -- the complete DFA of a keyword union (trie + failure links).
  random_dfa          -- a random complete DFA (every transition uniform).
Texts
  uniform_text        -- i.i.d. uniform symbols.
  zipf_words_text     -- space-separated Zipf-distributed words with planted keywords.
Workload recipes (the configurations that the tests and the benchmark use) are the
``*_workload`` functions at the end, with their sizes and seeds.
"""
from __future__ import annotations

from collections import deque
from dataclasses import dataclass, field

import numpy as np

NONE = 0xFFFFFFFF
NONE16 = 0xFFFF


@dataclass
class DfaSpec:
    """A DFA in the library's input format (see include/parem.h, parem_load_dfa)."""
    table: np.ndarray                     # uint32 [n_states, n_symbols], entry < n_states or NONE
    start: int
    accept: np.ndarray                    # uint8 [n_states]
    byte_to_symbol: np.ndarray | None     # uint16 [256] or None (identity)
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_states(self) -> int:
        return int(self.table.shape[0])

    @property
    def n_symbols(self) -> int:
        return int(self.table.shape[1])


# ----------------------------------------------------------------------------------------
# DFA builders
# ----------------------------------------------------------------------------------------
def kmp_dfa(pattern, n_symbols: int) -> tuple[np.ndarray, np.ndarray]:
    """String-matching automaton of ``pattern`` (a sequence of symbols < n_symbols).

    State q = length of the longest prefix of the pattern that is a suffix of the text read
    so far; state m = len(pattern) is the only accepting state, and on the next symbol it
    continues through the pattern's longest proper border, so overlapping matches are found.
    """
    pat = [int(c) for c in pattern]
    m = len(pat)
    assert m >= 1 and all(0 <= c < n_symbols for c in pat)
    table = np.zeros((m + 1, n_symbols), dtype=np.uint32)
    border = 0  # state reached by the pattern minus its first symbol (KMP restart state)
    table[0, pat[0]] = 1
    for q in range(1, m + 1):
        table[q, :] = table[border, :]
        if q < m:
            table[q, pat[q]] = q + 1
            border = int(table[border, pat[q]])
    accept = np.zeros(m + 1, dtype=np.uint8)
    accept[m] = 1
    return table, accept


def aho_corasick_dfa(keywords, n_symbols: int) -> tuple[np.ndarray, np.ndarray]:
    """Complete DFA for "some keyword ends here": trie nodes, goto + failure transitions.

    State = trie node of the longest suffix of the text read so far that is a prefix of some
    keyword.  A state accepts iff some keyword is a suffix of its string.
    """
    goto = [dict()]
    out = [False]
    for kw in keywords:
        node = 0
        for c in kw:
            c = int(c)
            assert 0 <= c < n_symbols
            if c not in goto[node]:
                goto.append(dict())
                out.append(False)
                goto[node][c] = len(goto) - 1
            node = goto[node][c]
        out[node] = True
    n = len(goto)
    table = np.zeros((n, n_symbols), dtype=np.uint32)
    fail = [0] * n
    queue = deque()
    for c in range(n_symbols):
        child = goto[0].get(c)
        if child is None:
            table[0, c] = 0
        else:
            table[0, c] = child
            fail[child] = 0
            queue.append(child)
    while queue:
        node = queue.popleft()
        out[node] = out[node] or out[fail[node]]
        for c in range(n_symbols):
            child = goto[node].get(c)
            if child is None:
                table[node, c] = table[fail[node], c]
            else:
                table[node, c] = child
                fail[child] = int(table[fail[node], c])
                queue.append(child)
    accept = np.array(out, dtype=np.uint8)
    return table, accept


def random_dfa(n_states: int, n_symbols: int, n_accept: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Random complete DFA: every transition uniform in [0, n_states); ``n_accept`` accepting
    states drawn without replacement; start state 0."""
    rng = np.random.default_rng(seed)
    table = rng.integers(0, n_states, size=(n_states, n_symbols), dtype=np.uint32)
    accept = np.zeros(n_states, dtype=np.uint8)
    if n_accept > 0:
        accept[rng.choice(n_states, size=n_accept, replace=False)] = 1
    return table, accept


def letters_byte_map() -> np.ndarray:
    """a-z (ASCII 97..122) -> symbols 0..25, space (32) -> 26, every other byte outside Sigma."""
    m = np.full(256, NONE16, dtype=np.uint16)
    m[97:123] = np.arange(26, dtype=np.uint16)
    m[32] = 26
    return m


# ----------------------------------------------------------------------------------------
# Texts
# ----------------------------------------------------------------------------------------
def uniform_text(n: int, n_symbols: int, seed: int) -> np.ndarray:
    """n i.i.d. uniform symbols in [0, n_symbols) as uint8 (numpy default_rng(seed))."""
    return np.random.default_rng(seed).integers(0, n_symbols, size=n, dtype=np.uint8)


def zipf_vocabulary(n_words: int = 65536, min_len: int = 2, max_len: int = 12, seed: int = 2):
    """Random lowercase words with lengths uniform in [min_len, max_len]."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(min_len, max_len + 1, size=n_words)
    letters = rng.integers(97, 123, size=int(lens.sum()), dtype=np.uint8)
    padded = np.full((n_words, max_len + 1), 32, dtype=np.uint8)
    o = 0
    for i, L in enumerate(lens):
        padded[i, :L] = letters[o:o + L]
        o += L
    return padded, lens.astype(np.int64)


def zipf_probabilities(n_words: int, s: float = 1.1) -> np.ndarray:
    r = np.arange(1, n_words + 1, dtype=np.float64)
    p = r ** (-s)
    return p / p.sum()


def random_keywords(n_keywords: int = 64, min_len: int = 8, max_len: int = 24, seed: int = 1):
    """Random lowercase keywords (bytes) with lengths uniform in [min_len, max_len]."""
    rng = np.random.default_rng(seed)
    kws = []
    for _ in range(n_keywords):
        L = int(rng.integers(min_len, max_len + 1))
        kws.append(bytes(rng.integers(97, 123, size=L, dtype=np.uint8)))
    return kws


def plant_plan(n: int, keywords, rate: float, seed: int):
    """Byte indices and values that plant keywords at positions chosen i.i.d. with
    probability ``rate`` per byte.  Later plants overwrite earlier ones; the returned
    indices are unique, so applying them in any order gives the same text."""
    rng = np.random.default_rng(seed)
    if n == 0 or rate <= 0:
        return np.zeros(0, np.int64), np.zeros(0, np.uint8)
    expect = int(n * rate * 1.2) + 64
    pos = []
    cur = -1
    while True:
        gaps = rng.geometric(rate, size=expect)
        starts = cur + np.cumsum(gaps)
        keep = starts[starts < n]
        pos.append(keep)
        if keep.size < starts.size:
            break
        cur = int(starts[-1])
    pos = np.concatenate(pos).astype(np.int64)
    which = rng.integers(0, len(keywords), size=pos.size)
    idx_parts, val_parts = [], []
    for p, w in zip(pos, which):
        kw = np.frombuffer(keywords[w], dtype=np.uint8)
        L = min(kw.size, n - int(p))
        idx_parts.append(np.arange(p, p + L, dtype=np.int64))
        val_parts.append(kw[:L])
    if not idx_parts:
        return np.zeros(0, np.int64), np.zeros(0, np.uint8)
    idx = np.concatenate(idx_parts)
    val = np.concatenate(val_parts)
    # last writer wins: unique over the reversed sequence keeps the last occurrence
    ridx = idx[::-1]
    rval = val[::-1]
    u, first = np.unique(ridx, return_index=True)
    return u, rval[first]


def zipf_words_text(n: int, seed_words: int = 2, seed_plants: int = 3, plant_rate: float = 1e-5,
                    keywords=None, zipf_s: float = 1.1) -> np.ndarray:
    """Host (numpy) version: words drawn by Zipf rank, separated by single spaces, truncated
    to n bytes, then keywords planted by overwriting."""
    padded, lens = zipf_vocabulary(seed=seed_words)
    p = zipf_probabilities(padded.shape[0], zipf_s)
    rng = np.random.default_rng(seed_words + 1000)
    mean = float((p * (lens + 1)).sum())
    out = np.empty(n, dtype=np.uint8)
    filled = 0
    while filled < n:
        k = int((n - filled) / mean * 1.05) + 16
        idx = rng.choice(padded.shape[0], size=k, p=p)
        L = lens[idx] + 1
        rows = padded[idx]
        mask = np.arange(padded.shape[1])[None, :] < L[:, None]
        chunk = rows[mask]
        take = min(chunk.size, n - filled)
        out[filled:filled + take] = chunk[:take]
        filled += take
    if keywords is None:
        keywords = random_keywords()
    pi, pv = plant_plan(n, keywords, plant_rate, seed_plants)
    out[pi] = pv
    return out


def zipf_words_text_device(n: int, device, seed: int = 2, seed_plants: int = 3, plant_rate: float = 1e-5,
                           keywords=None, zipf_s: float = 1.1):
    """Device (torch) version for multi-GiB texts: same distribution as zipf_words_text, word
    draws from torch's seeded generator on ``device`` (inverse-CDF sampling), plants from
    numpy default_rng(seed_plants).  Returns a uint8 CUDA tensor."""
    import torch

    padded, lens = zipf_vocabulary(seed=seed)
    V, W = padded.shape
    p = zipf_probabilities(V, zipf_s)
    cdf = torch.tensor(np.cumsum(p), dtype=torch.float64, device=device)
    padded_t = torch.tensor(padded, dtype=torch.uint8, device=device)
    lens_t = torch.tensor(lens, dtype=torch.int64, device=device)
    mean = float((p * (lens + 1)).sum())
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    out = torch.empty(n, dtype=torch.uint8, device=device)
    filled = 0
    while filled < n:
        k = min(48 << 20, int((n - filled) / mean * 1.02) + 1024)
        u = torch.rand(k, generator=g, device=device, dtype=torch.float64)
        idx = torch.searchsorted(cdf, u).clamp_(max=V - 1)
        L = lens_t[idx] + 1
        offs = torch.cumsum(L, 0) - L
        total = int(offs[-1].item() + L[-1].item())
        take = min(total, n - filled)
        word_of_byte = torch.repeat_interleave(torch.arange(k, device=device), L)[:take]
        char = torch.arange(take, device=device, dtype=torch.int64) - offs[word_of_byte]
        out[filled:filled + take] = padded_t[idx[word_of_byte], char]
        del word_of_byte, char, idx, L, offs, u
        filled += take
    if keywords is None:
        keywords = random_keywords()
    pi, pv = plant_plan(n, keywords, plant_rate, seed_plants)
    if pi.size:
        out[torch.from_numpy(pi).to(device)] = torch.from_numpy(pv).to(device)
    return out


def uniform_text_device(n: int, n_symbols: int, device, seed: int):
    """Device (torch) uniform symbols in [0, n_symbols), seeded torch generator."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    out = torch.empty(n, dtype=torch.uint8, device=device)
    step = 1 << 30
    for o in range(0, n, step):
        m = min(step, n - o)
        out[o:o + m] = torch.randint(0, n_symbols, (m,), generator=g, device=device, dtype=torch.int16).to(torch.uint8)
    return out


# ----------------------------------------------------------------------------------------
# Workload recipes
# ----------------------------------------------------------------------------------------
PARALLEL_ALPHABET = b"parel"      # column order of Table I
ACGT = {"A": 0, "C": 1, "G": 2, "T": 3}


def parallel_dfa() -> DfaSpec:
    """The automaton of Fig. 1 / Table I: all occurrences of "parallel" over {p,a,r,e,l}.
    Text bytes are the symbol indices 0..4 (identity byte map)."""
    pat = [PARALLEL_ALPHABET.index(c) for c in b"parallel"]
    table, accept = kmp_dfa(pat, 5)
    return DfaSpec(table, 0, accept, None, "parallel")


def gattaca_dfa() -> DfaSpec:
    """KMP automaton of Sigma*.GATTACA over A=0,C=1,G=2,T=3 (8 states, accept = 7)."""
    table, accept = kmp_dfa([ACGT[c] for c in "GATTACA"], 4)
    return DfaSpec(table, 0, accept, None, "gattaca")


def keywords_ac_dfa(n_keywords: int = 64, seed: int = 1) -> DfaSpec:
    """Aho-Corasick DFA of 64 random lowercase keywords (lengths 8-24) over a-z + space."""
    kws = random_keywords(n_keywords, seed=seed)
    sym = letters_byte_map()
    table, accept = aho_corasick_dfa([[int(sym[b]) for b in kw] for kw in kws], 27)
    return DfaSpec(table, 0, accept, sym, "ac64", {"keywords": kws})


def dense_dfa(n_states: int = 256, seed: int = 4, accept_frac: float = 0.10) -> DfaSpec:
    """Random complete DFA over all 256 byte values, ~10% accepting, start 0."""
    table, accept = random_dfa(n_states, 256, int(round(accept_frac * n_states)), seed)
    return DfaSpec(table, 0, accept, None, f"dense{n_states}")


def gattaca_workload(n: int = 1 << 20):
    return gattaca_dfa(), uniform_text(n, 4, 0)


def parallel_workload(n: int, seed: int = 11):
    return parallel_dfa(), uniform_text(n, 5, seed)


# ----------------------------------------------------------------------------------------
# Batched workload: many texts of uneven length, each paired with one of several DFAs
# ----------------------------------------------------------------------------------------
def keyword_union_dfa(target_states: int, alphabet: int, seed: int):
    """Aho-Corasick DFA of random keywords over `alphabet` symbols, adding keywords (lengths
    4-16) until the trie has at least `target_states` states.  For the 27-symbol alphabet the
    keywords use the letters only (symbol 26 is the space)."""
    rng = np.random.default_rng(seed)
    letters = 26 if alphabet == 27 else alphabet
    kws, nodes = [], {()}
    while len(nodes) < target_states:
        kw = tuple(int(x) for x in rng.integers(0, letters, size=int(rng.integers(4, 17))))
        kws.append(kw)
        for i in range(1, len(kw) + 1):
            nodes.add(kw[:i])
    table, accept = aho_corasick_dfa(kws, alphabet)
    return table, accept, kws


def batch_dfas(n_dfas: int = 32, seed: int = 6, max_states: int = 4096):
    """DFAs of the batched workload: states log-uniform in [4, max_states], alphabet uniform
    over {4, 27, 256}; even ids are keyword unions, odd ids random complete DFAs (10%
    accepting).  Byte maps: 27 symbols use letters_byte_map, 4 and 256 the identity."""
    rng = np.random.default_rng(seed)
    out = []
    for d in range(n_dfas):
        states = int(round(np.exp(rng.uniform(np.log(4), np.log(max_states)))))
        alphabet = int(rng.choice([4, 27, 256]))
        if d % 2 == 0:
            table, accept, kws = keyword_union_dfa(states, alphabet, seed * 1000 + d)
            meta = {"family": "keywords", "alphabet": alphabet, "keywords": len(kws)}
        else:
            table, accept = random_dfa(states, alphabet, max(1, int(round(0.1 * states))), seed * 1000 + d)
            meta = {"family": "random", "alphabet": alphabet}
        b2s = letters_byte_map() if alphabet == 27 else None
        out.append(DfaSpec(table, 0, accept, b2s, f"batch{d}", meta))
    return out


def batch_lengths(n_texts: int = 4096, lo: int = 1 << 10, hi: int = 16 << 20, seed: int = 6):
    """Text lengths log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed + 100)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_texts)).astype(np.int64)


def batch_texts_device(dfas, lengths, device, seed: int = 6, pool_bytes: int = 64 << 20):
    """Texts of the batched workload in one device arena (each text its own bytes): text i
    goes with DFA i mod len(dfas).  Keyword DFAs read Zipf words mapped into their alphabet
    (letters and space as is for 27 and 256 symbols; (letter - 'a') mod 4 and space -> 0 for
    4 symbols); random DFAs read uniform symbols.  Texts are copied from seeded pools at
    seeded offsets.  Returns (arena, offsets)."""
    import torch

    pool_bytes = max(pool_bytes, int(lengths.max()) + 1)
    zipf = zipf_words_text_device(pool_bytes, device, seed=seed)
    z4 = torch.where(zipf == 32, torch.zeros_like(zipf), (zipf - 97) % 4)
    pools = {("keywords", 27): zipf, ("keywords", 256): zipf, ("keywords", 4): z4,
             ("random", 4): uniform_text_device(pool_bytes, 4, device, seed + 1),
             ("random", 27): uniform_text_device(pool_bytes, 27, device, seed + 2),
             ("random", 256): uniform_text_device(pool_bytes, 256, device, seed + 3)}
    offsets = np.zeros(len(lengths) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)
    arena = torch.empty(int(offsets[-1]), dtype=torch.uint8, device=device)
    rng = np.random.default_rng(seed + 200)
    for i, L in enumerate(lengths):
        spec = dfas[i % len(dfas)]
        pool = pools[(spec.meta["family"], spec.meta["alphabet"])]
        start = int(rng.integers(0, pool_bytes - int(L)))
        arena[int(offsets[i]):int(offsets[i + 1])] = pool[start:start + int(L)]
    return arena, offsets


# ---------------------------------------------------------------------------------------
# serving workload: 128 DFAs, Poisson arrivals of requests that are slices of device pools
# ---------------------------------------------------------------------------------------
def serve_dfas(n_dfas: int = 128, seed: int = 7, max_states: int = 8192):
    """DFAs of the serving workload: the batch families with states log-uniform in
    [4, max_states]."""
    return batch_dfas(n_dfas, seed=seed, max_states=max_states)


def serve_trace(n_dfas: int, rate_per_s: float, duration_s: float, lo: int = 256, hi: int = 64 << 20,
                seed: int = 7):
    """Open-loop request trace: exponential inter-arrival gaps at rate_per_s for duration_s,
    DFA uniform over n_dfas, lengths log-uniform in [lo, hi].  Returns (arrival_ns, dfa, length)."""
    rng = np.random.default_rng(seed)
    n = int(rate_per_s * duration_s * 1.2) + 16
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
    n = int(np.searchsorted(t, duration_s))
    arrival = (t[:n] * 1e9).astype(np.int64)
    dfa = rng.integers(0, n_dfas, size=n).astype(np.uint32)
    length = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n)).astype(np.int64)
    return arrival, dfa, length


def serve_pools_device(device, pool_bytes: int = 1536 << 20, seed: int = 7):
    """Device text pools of the serving workload, one per (family, alphabet), filled as the
    batched workload's texts: 6 x pool_bytes (9 GiB at the default)."""
    import torch

    zipf = zipf_words_text_device(pool_bytes, device, seed=seed)
    z4 = torch.where(zipf == 32, torch.zeros_like(zipf), (zipf - 97) % 4)
    return {("keywords", 27): zipf, ("keywords", 256): zipf.clone(), ("keywords", 4): z4,
            ("random", 4): uniform_text_device(pool_bytes, 4, device, seed + 1),
            ("random", 27): uniform_text_device(pool_bytes, 27, device, seed + 2),
            ("random", 256): uniform_text_device(pool_bytes, 256, device, seed + 3)}


def serve_slices(specs, pools, dfa, length, seed: int = 7):
    """Device address of each request's text: a seeded slice of its DFA's pool."""
    rng = np.random.default_rng(seed + 300)
    addr = np.zeros(len(dfa), dtype=np.uint64)
    keys = [(s.meta["family"], s.meta["alphabet"]) for s in specs]
    for i, (d, L) in enumerate(zip(dfa, length)):
        pool = pools[keys[int(d)]]
        start = int(rng.integers(0, pool.numel() - int(L)))
        addr[i] = pool.data_ptr() + start
    return addr
