"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each pin is written as a function of a scan implementation, so the same pin checks the C
oracle, its pure-Python mirror and (in test_pins_catch_planted_mistakes) deliberately
broken copies of the mirror, which shows that a plausible mistake fails at least one pin.

Pins:
  * Table I (Section II-C): the printed transition table equals the KMP automaton of
    "parallel" -- this pins the input builder that every test relies on.
  * Table II (Section II-C): the candidate sets and visited-state rows of the worked
    example, and the result of the whole scan.
  * The image of "l" is {0,5,6,8}; 28 runs for enumeration vs 13 worst case (Section II-C).
  * KMP automata vs brute-force substring search (textbook special case).
  * Aho-Corasick automata vs Python's ``re`` (library routine) and brute force.
  * The matrix-product formulation of a DFA run (numpy matmul, the formulation of Maine
    cited in Section I) on random partial DFAs with bytes outside the alphabet.
  * Closed forms: parity of a symbol count; a binary number modulo 3.
  * Algorithm 1 restated on the CPU: every split into p slices joins to the sequential result.
  * Exhaustive enumeration of all short texts over a small partial DFA.
"""
import itertools
import os
import re

import numpy as np
import pytest

from oracle import oracle
from paper_1412_1741_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NONE = oracle.NONE
NONE16 = oracle.NONE16


def load_table1():
    rows = []
    with open(os.path.join(GOLDEN, "paper_table1_parallel.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                v = [int(x) for x in line.split()]
                rows.append(v)
    rows.sort()
    assert [r[0] for r in rows] == list(range(9))
    return np.array([r[1:] for r in rows], dtype=np.uint32)


def load_table2():
    d = {"rows": []}
    with open(os.path.join(GOLDEN, "paper_table2_chunks.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *rest = line.split()
            if k == "TEXT":
                d["text"] = rest[0]
            elif k == "UNITS":
                d["units"] = int(rest[0])
            elif k.startswith("P"):
                d["rows"].append((int(k[1:]), int(rest[0]), [int(x) for x in rest[1:]]))
            elif k == "IMAGE":
                d["image"] = (rest[0], [int(x) for x in rest[1:]])
            else:
                d[k] = int(rest[0])
    return d


def parallel_spec():
    table = load_table1()
    accept = np.zeros(9, np.uint8)
    accept[8] = 1
    return table, accept


def encode_parel(s):
    return np.frombuffer(bytes(wl.PARALLEL_ALPHABET.index(c) for c in s.encode()), dtype=np.uint8)


# ----------------------------------------------------------------------------------------
# pins as functions of a scan implementation
# ----------------------------------------------------------------------------------------
def c_scan(table, b2s, start, accept, text):
    return oracle.scan(table, b2s, start, accept, np.asarray(text, dtype=np.uint8))


def py_scan(table, b2s, start, accept, text):
    return oracle.scan_py(table, b2s, start, accept, bytes(np.asarray(text, dtype=np.uint8)))


def pin_worked_example(scan_fn):
    table, accept = parallel_spec()
    d = load_table2()
    text = encode_parel(d["text"])
    r = scan_fn(table, None, 0, accept, text)
    # The only occurrence of "parallel" ends at index 12 (0-based); the text ends in state 0.
    assert r.match_count == 1
    assert list(map(int, r.positions)) == [12]
    assert r.final_state == 0 and not r.accepted


def pin_kmp_bruteforce(scan_fn, trials=60, seed=123):
    rng = np.random.default_rng(seed)
    for t in range(trials):
        k = int(rng.integers(2, 5))
        m = int(rng.integers(1, 7))
        pat = rng.integers(0, k, size=m)
        if t % 3 == 0:  # periodic patterns exercise overlapping matches
            pat = np.resize(pat[: max(1, m // 2)], m)
        table, accept = wl.kmp_dfa(pat, k)
        text = rng.integers(0, k, size=int(rng.integers(0, 200)), dtype=np.uint8)
        r = scan_fn(table, None, 0, accept, text)
        want = [j for j in range(m - 1, text.size) if np.array_equal(text[j - m + 1:j + 1], pat)]
        assert list(map(int, r.positions)) == want
        assert r.match_count == len(want)
        # the final state is the longest suffix of the text that is a prefix of the pattern
        best = 0
        for L in range(min(m, text.size), -1, -1):
            if L == 0 or np.array_equal(text[text.size - L:], pat[:L]):
                best = L
                break
        assert r.final_state == best


def matrix_scan(table, b2s, start, accept, text):
    """The run as products of 0/1 transition matrices (one per symbol) with a one-hot state
    row vector; index n (one past the states) is the dead state."""
    table = np.asarray(table, dtype=np.int64)
    n, k = table.shape
    M = np.zeros((k + 1, n + 1, n + 1), dtype=np.int64)  # symbol k = outside the alphabet
    for a in range(k):
        for q in range(n):
            e = table[q, a]
            M[a, q, n if e == NONE else e] = 1
        M[a, n, n] = 1
    M[k, :, n] = 1
    f = np.zeros(n + 1, dtype=np.int64)
    f[:n] = np.asarray(accept, dtype=np.int64)
    v = np.zeros(n + 1, dtype=np.int64)
    v[start] = 1
    pos = []
    for j, b in enumerate(np.asarray(text, dtype=np.uint8)):
        if b2s is None:
            a = int(b) if int(b) < k else k
        else:
            a = int(b2s[b])
            a = k if a == NONE16 else a
        v = v @ M[a]
        if int(v @ f) == 1:
            pos.append(j)
    final = int(np.argmax(v))
    assert v.sum() == 1
    return oracle.ScanResult(NONE if final == n else final, final != n and bool(accept[final]), len(pos),
                             np.array(pos, dtype=np.uint64))


def random_partial_dfa(rng, n, k, p_none=0.15):
    table = rng.integers(0, n, size=(n, k)).astype(np.uint32)
    table[rng.random((n, k)) < p_none] = NONE
    accept = (rng.random(n) < 0.3).astype(np.uint8)
    b2s = np.full(256, NONE16, dtype=np.uint16)
    for b in range(256):
        if rng.random() < 0.8:
            b2s[b] = rng.integers(0, k)
    return table, accept, b2s


def pin_matrix(scan_fn, trials=40, seed=7):
    rng = np.random.default_rng(seed)
    for t in range(trials):
        n = int(rng.integers(1, 9))
        k = int(rng.integers(1, 6))
        table, accept, b2s = random_partial_dfa(rng, n, k)
        if t % 2:
            b2s = None
        text = rng.integers(0, 8 if b2s is None else 256, size=int(rng.integers(0, 120)), dtype=np.uint8)
        start = int(rng.integers(0, n))
        a = scan_fn(table, b2s, start, accept, text)
        b = matrix_scan(table, b2s, start, accept, text)
        assert (a.final_state, a.accepted, a.match_count) == (b.final_state, b.accepted, b.match_count)
        assert np.array_equal(a.positions, b.positions)


def pin_closed_forms(scan_fn, seed=5):
    rng = np.random.default_rng(seed)
    # parity of the number of a's (symbol 0) over {a,b}: state = count mod 2, F = {even}
    table = np.array([[1, 0], [0, 1]], dtype=np.uint32)
    accept = np.array([1, 0], np.uint8)
    text = rng.integers(0, 2, size=300, dtype=np.uint8)
    r = scan_fn(table, None, 0, accept, text)
    want = [j for j in range(text.size) if int((text[: j + 1] == 0).sum()) % 2 == 0]
    assert list(map(int, r.positions)) == want
    assert r.final_state == int((text == 0).sum()) % 2
    # value of a binary number read MSB first, modulo 3; F = {0}
    table = np.array([[(2 * q + a) % 3 for a in range(2)] for q in range(3)], dtype=np.uint32)
    accept = np.array([1, 0, 0], np.uint8)
    bits = rng.integers(0, 2, size=200, dtype=np.uint8)
    r = scan_fn(table, None, 0, accept, bits)
    want = [j for j in range(bits.size) if int("".join(map(str, bits[: j + 1])), 2) % 3 == 0]
    assert list(map(int, r.positions)) == want
    assert r.final_state == int("".join(map(str, bits)), 2) % 3


def pin_ac_re(scan_fn, seed=9):
    rng = np.random.default_rng(seed)
    for t in range(12):
        alpha = b"abcd"
        kws = sorted({rng.choice(list(alpha), size=int(rng.integers(1, 6))).astype(np.uint8).tobytes()
                      for _ in range(int(rng.integers(1, 7)))})
        sym = np.full(256, NONE16, np.uint16)
        for i, c in enumerate(alpha):
            sym[c] = i
        table, accept = wl.aho_corasick_dfa([[int(sym[c]) for c in kw] for kw in kws], len(alpha))
        text = rng.choice(list(alpha + b"x"), size=int(rng.integers(0, 300))).astype(np.uint8).tobytes()
        r = scan_fn(table, sym, 0, accept, np.frombuffer(text, np.uint8))
        ends = set()
        for kw in kws:  # library routine: overlapping matches of each keyword via lookahead
            for m in re.finditer(b"(?=" + re.escape(kw) + b")", text):
                ends.add(m.start() + len(kw) - 1)
        brute = {j for j in range(len(text)) for kw in kws if text[: j + 1].endswith(kw)}
        assert ends == brute
        # A byte outside the alphabet ('x') kills the run (dead state, reading c4/c10), so the
        # DFA can only report the matches that end before the first 'x'.
        cut = text.find(b"x")
        cut = len(text) if cut < 0 else cut
        want = sorted(e for e in ends if e < cut)
        assert list(map(int, r.positions)) == want
        if cut < len(text):
            assert r.final_state == NONE


ALL_PINS = [pin_worked_example, pin_kmp_bruteforce, pin_matrix, pin_closed_forms, pin_ac_re]


@pytest.mark.parametrize("impl", [c_scan, py_scan], ids=["C", "python"])
@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda f: f.__name__)
def test_pin(impl, pin):
    pin(impl)


# ----------------------------------------------------------------------------------------
# paper fixtures
# ----------------------------------------------------------------------------------------
def test_table1_is_kmp_automaton_of_parallel():
    spec = wl.parallel_dfa()
    assert np.array_equal(spec.table, load_table1())
    assert list(np.nonzero(spec.accept)[0]) == [8]


def test_table2_candidates_and_visited_rows():
    table, accept = parallel_spec()
    d = load_table2()
    text = encode_parel(d["text"])
    slices = oracle.alg1_parallel(table, None, 0, accept, text, d["units"])
    assert [(lo, hi) for lo, hi, _ in slices] == [(0, 6), (6, 12), (12, 18), (18, 24)]
    for unit, cand, visited in d["rows"]:
        lo, hi, runs = slices[unit]
        assert cand in runs, (unit, cand)
        assert runs[cand][0] == visited
        # the C trace gives the same visited vector
        assert list(map(int, oracle.trace(table, None, cand, text[lo:hi]))) == visited
    # candidate sets by the rule of Algorithm 1 (R3 = {0, 7}: reading of the printed row)
    assert [sorted(runs) for _, _, runs in slices] == [[0], [1], [0, 7], [0, 7]]
    res = oracle.alg1_join(slices, 0, accept, text.size)
    seq = oracle.scan(table, None, 0, accept, text)
    assert (res.final_state, res.match_count, list(res.positions)) == (seq.final_state, 1, [12])


def test_image_of_l_and_run_counts():
    table, _ = parallel_spec()
    d = load_table2()
    sym, img = d["image"]
    tl = [list(map(int, r)) for r in table]
    assert sorted(oracle.alg1_L(tl, wl.PARALLEL_ALPHABET.index(sym.encode()))) == img
    n_states = table.shape[0]
    units = d["units"]
    assert (units - 1) * n_states + 1 == d["ENUM_RUNS"]
    assert (units - 1) * len(img) + 1 == d["WORST_RUNS"]
    assert round(d["ENUM_RUNS"] / d["WORST_RUNS"], 2) == 2.15


def test_kmp_builder_matches_its_definition():
    rng = np.random.default_rng(1)
    for _ in range(40):
        k = int(rng.integers(1, 5))
        pat = list(rng.integers(0, k, size=int(rng.integers(1, 8))))
        table, accept = wl.kmp_dfa(pat, k)
        m = len(pat)
        for q in range(m + 1):
            for a in range(k):
                w = pat[:q] + [a]
                best = 0
                for L in range(min(m, len(w)), 0, -1):
                    if w[len(w) - L:] == pat[:L]:
                        best = L
                        break
                assert table[q, a] == best


def test_ac_builder_matches_its_definition():
    rng = np.random.default_rng(2)
    for _ in range(10):
        k = 3
        kws = [list(rng.integers(0, k, size=int(rng.integers(1, 5)))) for _ in range(int(rng.integers(1, 5)))]
        table, accept = wl.aho_corasick_dfa(kws, k)
        # rebuild node strings by BFS over the trie edges
        prefixes = sorted({tuple(kw[:i]) for kw in kws for i in range(len(kw) + 1)}, key=lambda t: (len(t), t))
        # map each node to its string by walking the table from the root
        node_of = {}
        for p in prefixes:
            s = 0
            for c in p:
                s = int(table[s, c])
            node_of[p] = s
        assert len(set(node_of.values())) == table.shape[0] == len(prefixes)
        for p, s in node_of.items():
            for a in range(k):
                w = list(p) + [a]
                best = ()
                for L in range(len(w), -1, -1):
                    if tuple(w[len(w) - L:]) in node_of:
                        best = tuple(w[len(w) - L:])
                        break
                assert int(table[s, a]) == node_of[best]
            assert bool(accept[s]) == any(list(p[len(p) - len(kw):]) == kw for kw in kws if len(kw) <= len(p))


# ----------------------------------------------------------------------------------------
# Algorithm 1 and exhaustive checks
# ----------------------------------------------------------------------------------------
def test_every_split_joins_to_the_sequential_result():
    rng = np.random.default_rng(3)
    for t in range(25):
        n_states = int(rng.integers(1, 7))
        k = int(rng.integers(1, 4))
        table, accept, b2s = random_partial_dfa(rng, n_states, k, p_none=0.1 if t % 2 else 0.0)
        b2s = None
        text = rng.integers(0, k + (1 if t % 3 == 0 else 0), size=int(rng.integers(0, 40)), dtype=np.uint8)
        seq = oracle.scan(table, None, 0, accept, text)
        for p in range(1, max(2, text.size + 2)):
            res = oracle.alg1_join(oracle.alg1_parallel(table, None, 0, accept, text, p), 0, accept, text.size)
            assert (res.final_state, res.match_count) == (seq.final_state, seq.match_count), (t, p)
            assert np.array_equal(res.positions, seq.positions)


def test_exhaustive_short_texts():
    rng = np.random.default_rng(4)
    table, accept, _ = random_partial_dfa(rng, 4, 3, p_none=0.2)
    for L in range(0, 7):
        for text in itertools.product(range(4), repeat=L):  # byte 3 lies outside the alphabet
            t = np.array(text, dtype=np.uint8)
            a = oracle.scan(table, None, 1, accept, t)
            b = oracle.scan_py(table, None, 1, accept, bytes(t))
            assert (a.final_state, a.match_count, list(a.positions)) == (b.final_state, b.match_count, list(b.positions))
    # and the matrix formulation on a sample of the longest texts
    for text in list(itertools.product(range(4), repeat=7))[::97]:
        t = np.array(text, dtype=np.uint8)
        a = oracle.scan(table, None, 1, accept, t)
        m = matrix_scan(table, None, 1, accept, t)
        assert (a.final_state, a.match_count, list(a.positions)) == (m.final_state, m.match_count, list(m.positions))


def test_empty_text_and_capacity():
    table, accept = parallel_spec()
    r = oracle.scan(table, None, 8, accept, np.zeros(0, np.uint8))
    assert (r.final_state, r.accepted, r.match_count) == (8, True, 0)
    text = encode_parel("parallel" * 5)
    r = oracle.scan(table, None, 0, accept, text, capacity=3)
    assert r.match_count == 5 and list(map(int, r.positions)) == [7, 15, 23]


def test_invalid_arguments_are_rejected():
    table = np.array([[0, 5]], dtype=np.uint32)  # entry 5 >= n_states
    with pytest.raises(ValueError):
        oracle.scan(table, None, 0, np.zeros(1, np.uint8), np.array([1], np.uint8))
    with pytest.raises(ValueError):
        oracle.scan(np.zeros((1, 2), np.uint32), None, 3, np.zeros(1, np.uint8), np.zeros(1, np.uint8))


# ----------------------------------------------------------------------------------------
# the pins have teeth: plausible mistakes planted in copies of the mirror fail a pin
# ----------------------------------------------------------------------------------------
def _mutant(kind):
    def scan_fn(table, b2s, start, accept, text):
        table = np.asarray(table)
        n, k = table.shape
        s = int(start)
        pos = []
        for j, b in enumerate(np.asarray(text, dtype=np.uint8)):
            a = oracle.symbol_of(b2s, k, int(b))
            if kind == "count_before_step" and s != NONE and accept[s]:
                pos.append(j)
            if kind == "transposed" and s != NONE and a != NONE:
                s = int(table.T.reshape(-1)[(a * n + s) % (n * k)]) if n == k else int(table[a % n][s % k])
            elif kind == "dead_not_absorbing" and s == NONE:
                s = int(table[start][a]) if a != NONE else NONE
            elif kind == "off_by_one_position":
                s = oracle.step(table, s, a)
                if s != NONE and accept[s]:
                    pos.append(j + 1)
                continue
            else:
                s = oracle.step(table, s, a)
            if kind != "count_before_step" and s != NONE and accept[s]:
                pos.append(j)
        acc = s != NONE and bool(accept[s])
        return oracle.ScanResult(s, acc, len(pos), np.array(pos, dtype=np.uint64))
    return scan_fn


@pytest.mark.parametrize("kind", ["count_before_step", "transposed", "dead_not_absorbing", "off_by_one_position"])
def test_pins_catch_planted_mistakes(kind):
    bad = _mutant(kind)
    failed = []
    for pin in ALL_PINS:
        try:
            pin(bad)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"no pin caught the planted mistake {kind}"
