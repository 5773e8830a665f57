"""Regular-expression front-end (host only, no GPU): the operators of Table III compiled by the
Thompson and subset constructions (Section III) into a DFA, checked by running that DFA with
the oracle against a brute force with Python's `re` module (every position j such that some suffix of
the text up to j, possibly empty, matches, or for anchored compilation the prefix up to j), and
against the paper's own automaton of Table I for the literal "parallel"."""
import os
import re

import numpy as np
import pytest

import paper_1412_1741_gb300 as pm
from oracle import oracle
from paper_1412_1741_gb300 import build as pbuild

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def lib():
    pbuild.build()
    return pm.load_library()


def to_python(pattern: str) -> str:
    """The same expression in Python's syntax: inside [...] sets the paper's ranges a..z
    become a-z (outside a set, '..' is two any-byte atoms and stays)."""
    return re.sub(r"\[[^\]]*\]", lambda m: re.sub(r"(\\?.)\.\.(\\?.)", r"\1-\2", m.group(0)), pattern)


def brute_force(pattern: str, text: bytes, anchored: bool) -> np.ndarray:
    rx = re.compile(to_python(pattern).encode(), re.S)
    ends = []
    for j in range(len(text)):
        # a suffix of text[0..j], possibly empty (a pattern that matches the empty string
        # matches after every symbol), or the whole prefix when anchored
        starts = [0] if anchored else range(j + 2)
        if any(rx.fullmatch(text, i, j + 1) for i in starts):
            ends.append(j)
    return np.array(ends, np.uint64)


def dfa_positions(r: pm.RegexDfa, text: bytes) -> np.ndarray:
    return oracle.scan(r.table, r.byte_to_symbol, r.start, r.accept, np.frombuffer(text, np.uint8)).positions


PATTERNS = [
    "ab", "a*", "a|b", "a+", "[0..9]", "a?", "(ab|c)*",          # one per row of Table III
    "(a|b)?c*[0..3]b+",                                          # the expression of Fig. 2
    "ab*c", "(a|bc)+d?", "a(b|)c", "[a-c]+b", "x[^ab]y", "a.c", "(aa|a)*b", "((a|b)(c|d))+",
    "c(a|b)*c", "\\x61\\.b", "[0..2][1..3]?", "(ab)?(ab)?a",
]


@pytest.mark.parametrize("pattern", PATTERNS)
@pytest.mark.parametrize("anchored", [False, True])
def test_compiled_dfa_matches_re_brute_force(pattern, anchored):
    r = pm.parem_regex_compile(pattern, pm.PAREM_REGEX_ANCHORED if anchored else 0)
    assert r.table.shape[0] == r.accept.size and r.table.shape[1] == int(r.byte_to_symbol.max()) + 1
    rng = np.random.default_rng(len(pattern) * 7 + anchored)
    alphabet = np.frombuffer(b"abcdxy0123.", np.uint8)
    for n in (0, 1, 5, 40, 160):
        text = bytes(rng.choice(alphabet, size=n))
        assert np.array_equal(dfa_positions(r, text), brute_force(pattern, text, anchored)), (pattern, text)


def test_literal_search_dfa_is_the_automaton_of_table1():
    # the search DFA of "parallel" needs exactly the paper's 9 states, and on the paper's
    # example input it reports the one match the example finds (ending at index 12)
    r = pm.parem_regex_compile("parallel")
    assert r.table.shape[0] == 9
    text = b"plarap" + b"aralle" + b"lapare" + b"parapl"
    assert dfa_positions(r, text).tolist() == [12]
    # same language as Table I's automaton on every text over {p,a,r,e,l}
    t1 = np.loadtxt(os.path.join(GOLDEN, "paper_table1_parallel.txt"), dtype=np.uint32)[:, 1:]
    acc = np.zeros(9, np.uint8)
    acc[8] = 1
    b2s = np.full(256, pm.PAREM_NONE16, np.uint16)
    for k, c in enumerate(b"parel"):
        b2s[c] = k
    rng = np.random.default_rng(12)
    for _ in range(50):
        text = bytes(rng.choice(np.frombuffer(b"parel", np.uint8), size=200))
        want = oracle.scan(t1, b2s, 0, acc, np.frombuffer(text, np.uint8)).positions
        assert np.array_equal(dfa_positions(r, text), want)


def test_byte_classes_and_dead_transitions():
    r = pm.parem_regex_compile("[a..z]+q", pm.PAREM_REGEX_ANCHORED)
    b2s = r.byte_to_symbol
    assert len(set(b2s[[ord(c) for c in "abcp"]])) == 1          # letters other than q: one class
    assert b2s[ord("q")] != b2s[ord("a")] and b2s[ord("0")] != b2s[ord("a")]
    # anchored: a byte outside [a..z] at the start leaves no way to match
    assert r.table[r.start, b2s[ord("0")]] == pm.PAREM_NONE


@pytest.mark.parametrize("bad", ["(", "a)", "*a", "a|*", "[ab", "[z..a]", "\\x4", "a(b"])
def test_syntax_errors_are_rejected(bad):
    with pytest.raises(pm.ParemError) as e:
        pm.parem_regex_compile(bad)
    assert e.value.status == -1


def test_state_limit():
    # the 10th symbol from the end is 'a': any DFA for it has at least 2^10 states
    pattern = "(a|b)*a" + "(a|b)" * 9
    with pytest.raises(pm.ParemError) as e:
        pm.parem_regex_compile(pattern, max_states=256)
    assert e.value.status == pm.PAREM_ERR_TOO_LARGE
    r = pm.parem_regex_compile(pattern, max_states=4096)
    assert r.table.shape[0] == 1024  # minimal
    rng = np.random.default_rng(3)
    text = bytes(rng.choice(np.frombuffer(b"ab", np.uint8), size=60))
    assert np.array_equal(dfa_positions(r, text), brute_force(pattern, text, False))


@pytest.mark.parametrize("pattern,anchored,states", [
    ("a*", False, 1),            # every suffix matches (the empty one): one accepting state
    ("(a|b)*", True, 1),         # the empty prefix matches too: one accepting state (others: dead)
    ("a|aa|aaa", True, 4),       # a, aa, aaa: the start and three accepting states
    ("(ab|ab)c", True, 4),       # the duplicate alternative collapses
    ("x*y", False, 2),
])
def test_minimal_dfa_sizes(pattern, anchored, states):
    # the compiled DFA is minimal: its state count is the Myhill-Nerode index of the language
    # (the dead state is implicit, as PAREM_NONE entries)
    r = pm.parem_regex_compile(pattern, pm.PAREM_REGEX_ANCHORED if anchored else 0)
    assert r.table.shape[0] == states, r.table


def random_pattern(rng, depth=0):
    """A random expression over a small alphabet from Table III's operators."""
    r = rng.random()
    if depth >= 3 or r < 0.3:
        kind = rng.integers(4)
        if kind == 0:
            return str(rng.choice(list("abc")))
        if kind == 1:
            lo, hi = sorted(rng.choice(list("abcd"), size=2))
            return f"[{lo}..{hi}]"
        if kind == 2:
            return "[^" + str(rng.choice(list("abc"))) + "]"
        return "."
    if r < 0.55:
        return random_pattern(rng, depth + 1) + random_pattern(rng, depth + 1)
    if r < 0.7:
        return "(" + random_pattern(rng, depth + 1) + "|" + random_pattern(rng, depth + 1) + ")"
    return "(" + random_pattern(rng, depth + 1) + ")" + str(rng.choice(list("*+?")))


def test_random_expressions_match_re_brute_force():
    # 200 random expressions of nested operators, each on random texts, search and anchored
    rng = np.random.default_rng(2024)
    alphabet = np.frombuffer(b"abcdx", np.uint8)
    for _ in range(200):
        pattern = random_pattern(rng)
        for anchored in (False, True):
            r = pm.parem_regex_compile(pattern, pm.PAREM_REGEX_ANCHORED if anchored else 0)
            text = bytes(rng.choice(alphabet, size=int(rng.integers(0, 30))))
            assert np.array_equal(dfa_positions(r, text), brute_force(pattern, text, anchored)), (pattern, text)
