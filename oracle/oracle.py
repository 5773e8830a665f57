"""Reference oracle for PaREM DFA matching.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` (the
``cpu_baseline`` of a bench line and the ``--impl reference`` arm) may import this module.  The product package never imports it, and it imports nothing from the
product package: the two share no code, tables or helpers.

Contents
--------
* ``scan``            -- the plain sequential DFA run (Section II-A; Section II-B: start in
                         q0, one step per symbol), in C (``parem_oracle.c``) via ctypes.
* ``scan_py``         -- the same definition as a pure-Python loop, for tiny cases.
* ``trace``           -- the visited-state vector of one run (the vector Rr of Algorithm 1).
* ``alg1_*``          -- Algorithm 1 restated step by step on the CPU for small inputs: the
                         domain decomposition, the sets S, L and R = S n L, one run per
                         candidate, and the join of the per-chunk results (Section II-B,
                         Section II-C).  It is used to pin the oracle against Table II and
                         to check that every chunking composes to the sequential result.

All arithmetic is on integers and exact; there is no tolerance anywhere.
Conventions (readings of the paper):
  NONE (0xFFFFFFFF) in a table entry = undefined transition; a byte that maps to NONE16
  (0xFFFF) is outside the alphabet.  Both lead to the absorbing, non-accepting dead state,
  reported as NONE.  A match is counted after each symbol whose transition lands in F, at
  the 0-based index of that symbol; q0 itself is never counted.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

NONE = 0xFFFFFFFF
NONE16 = 0xFFFF

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "parem_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libparem_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile parem_oracle.c into a shared library with gcc (portable flags only)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.oracle_dfa_scan.argtypes = [
            ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint32,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64,
            u32p, ctypes.POINTER(ctypes.c_uint64)]
        lib.oracle_dfa_scan.restype = ctypes.c_int
        lib.oracle_dfa_trace.argtypes = [
            ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint32,
            ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
        lib.oracle_dfa_trace.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass
class ScanResult:
    final_state: int          # NONE when the run died
    accepted: bool            # final_state in F (Section II-A)
    match_count: int
    positions: np.ndarray     # uint64, ascending 0-based indices of match-ending symbols


def _prep(table, byte_to_symbol, accept):
    table = np.ascontiguousarray(table, dtype=np.uint32)
    assert table.ndim == 2
    accept = np.ascontiguousarray(accept, dtype=np.uint8)
    assert accept.shape == (table.shape[0],)
    b2s = None
    if byte_to_symbol is not None:
        b2s = np.ascontiguousarray(byte_to_symbol, dtype=np.uint16)
        assert b2s.shape == (256,)
    return table, b2s, accept


def _ptr(a):
    return None if a is None else a.ctypes.data


def scan(table, byte_to_symbol, start, accept, text, want_positions=True, capacity=None, times=None) -> ScanResult:
    """Plain sequential DFA run over ``text`` (C implementation).

    ``times``: optional list; the wall time (s) of each pass over the text is appended to it
    (one pass without positions; with positions a counting pass, then the pass that writes
    them), so that a caller can time one pass of the definition on its own."""
    import time

    lib = _load()
    table, b2s, accept = _prep(table, byte_to_symbol, accept)
    text = np.ascontiguousarray(np.frombuffer(text, dtype=np.uint8) if isinstance(text, (bytes, bytearray)) else text,
                                dtype=np.uint8)
    n = int(text.size)
    fs = ctypes.c_uint32()
    cnt = ctypes.c_uint64()
    if want_positions:
        # First pass counts, second pass fills exactly; keeps memory bounded by the count.
        t0 = time.perf_counter()
        rc = lib.oracle_dfa_scan(_ptr(table), table.shape[0], table.shape[1], _ptr(b2s), int(start),
                                 _ptr(accept), _ptr(text), n, None, 0, ctypes.byref(fs), ctypes.byref(cnt))
        if times is not None:
            times.append(time.perf_counter() - t0)
        if rc != 0:
            raise ValueError(f"oracle_dfa_scan: invalid argument ({rc})")
        cap = cnt.value if capacity is None else min(int(capacity), cnt.value)
        pos = np.zeros(max(cap, 1), dtype=np.uint64)
        t0 = time.perf_counter()
        rc = lib.oracle_dfa_scan(_ptr(table), table.shape[0], table.shape[1], _ptr(b2s), int(start),
                                 _ptr(accept), _ptr(text), n, _ptr(pos), cap, ctypes.byref(fs), ctypes.byref(cnt))
        if times is not None:
            times.append(time.perf_counter() - t0)
        pos = pos[:cap]
    else:
        t0 = time.perf_counter()
        rc = lib.oracle_dfa_scan(_ptr(table), table.shape[0], table.shape[1], _ptr(b2s), int(start),
                                 _ptr(accept), _ptr(text), n, None, 0, ctypes.byref(fs), ctypes.byref(cnt))
        if times is not None:
            times.append(time.perf_counter() - t0)
        pos = np.zeros(0, dtype=np.uint64)
    if rc != 0:
        raise ValueError(f"oracle_dfa_scan: invalid argument ({rc})")
    final = int(fs.value)
    accepted = final != NONE and bool(accept[final])
    return ScanResult(final, accepted, int(cnt.value), pos)


def trace(table, byte_to_symbol, start, text) -> np.ndarray:
    """Visited-state vector of one run from ``start`` (NONE once dead): Rr of Algorithm 1."""
    lib = _load()
    table = np.ascontiguousarray(table, dtype=np.uint32)
    b2s = None if byte_to_symbol is None else np.ascontiguousarray(byte_to_symbol, dtype=np.uint16)
    text = np.ascontiguousarray(np.frombuffer(text, dtype=np.uint8) if isinstance(text, (bytes, bytearray)) else text,
                                dtype=np.uint8)
    out = np.zeros(max(text.size, 1), dtype=np.uint32)
    rc = lib.oracle_dfa_trace(_ptr(table), table.shape[0], table.shape[1], _ptr(b2s), int(start),
                              _ptr(text), int(text.size), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_dfa_trace: invalid argument")
    return out[: text.size]


# ----------------------------------------------------------------------------------------
# Pure-Python mirror of the definition (tiny inputs only).
# ----------------------------------------------------------------------------------------
def symbol_of(byte_to_symbol, n_symbols, b):
    """Symbol of text byte b, or NONE when b lies outside the alphabet."""
    if byte_to_symbol is None:
        return b if b < n_symbols else NONE
    a = int(byte_to_symbol[b])
    return NONE if a == NONE16 else a


def step(table, s, a):
    """One application of delta; NONE (dead) absorbs, an undefined entry leads to NONE."""
    if s == NONE or a == NONE:
        return NONE
    return int(table[s][a])


def scan_py(table, byte_to_symbol, start, accept, text) -> ScanResult:
    table = [list(map(int, row)) for row in np.asarray(table)]
    n_symbols = len(table[0])
    s = int(start)
    pos = []
    for j, b in enumerate(bytes(text)):
        s = step(table, s, symbol_of(byte_to_symbol, n_symbols, b))
        if s != NONE and accept[s]:
            pos.append(j)
    accepted = s != NONE and bool(accept[s])
    return ScanResult(s, accepted, len(pos), np.array(pos, dtype=np.uint64))


# ----------------------------------------------------------------------------------------
# Algorithm 1, restated step by step (small inputs).
# ----------------------------------------------------------------------------------------
def alg1_slices(n, p):
    """Domain decomposition: processing unit i takes [i*(n//p), (i+1)*(n//p)); the last unit
    also takes the remainder that n//p leaves over (reading of the slice length n/p)."""
    size = n // p
    out = []
    for i in range(p):
        lo = i * size
        hi = (i + 1) * size if i < p - 1 else n
        out.append((lo, hi))
    return out


def alg1_S(table, first_symbol):
    """S: states with a transition defined on the first symbol of this slice."""
    return {q for q in range(len(table)) if step(table, q, first_symbol) != NONE}


def alg1_L(table, prev_last_symbol):
    """L: the distinct states reached from any state on the last symbol of the previous slice."""
    return {step(table, q, prev_last_symbol) for q in range(len(table))} - {NONE}


def alg1_candidates(table, byte_to_symbol, start, text, lo, hi, first_slice):
    """R = S n L for a slice (the first slice starts from q0 alone)."""
    if first_slice or lo == 0:
        # The first slice, or a slice preceded only by empty slices, starts from q0 exactly.
        return [int(start)]
    n_symbols = len(table[0])
    if hi <= lo:
        return sorted(alg1_L(table, symbol_of(byte_to_symbol, n_symbols, text[lo - 1])))
    S = alg1_S(table, symbol_of(byte_to_symbol, n_symbols, text[lo]))
    L = alg1_L(table, symbol_of(byte_to_symbol, n_symbols, text[lo - 1]))
    return sorted(S & L)


def alg1_run(table, byte_to_symbol, accept, r, text, lo, hi):
    """One candidate run over a slice: the visited vector Rr, the found counter and the match
    positions, counted per (slice, candidate) (reading of found++)."""
    n_symbols = len(table[0])
    s = r
    visited, pos = [], []
    for j in range(lo, hi):
        s = step(table, s, symbol_of(byte_to_symbol, n_symbols, text[j]))
        visited.append(s)
        if s != NONE and accept[s]:
            pos.append(j)
    return visited, pos


def alg1_parallel(table, byte_to_symbol, start, accept, text, p):
    """All slices of Algorithm 1: for every slice its candidate set R and one run per candidate.
    Returns a list of (lo, hi, {r: (visited, positions)})."""
    table = [list(map(int, row)) for row in np.asarray(table)]
    text = bytes(text)
    out = []
    for i, (lo, hi) in enumerate(alg1_slices(len(text), p)):
        R = alg1_candidates(table, byte_to_symbol, start, text, lo, hi, i == 0)
        runs = {r: alg1_run(table, byte_to_symbol, accept, r, text, lo, hi) for r in R}
        out.append((lo, hi, runs))
    return out


def alg1_join(slices, start, accept, n):
    """The reduction: connect the last state of slice i's chosen run to the candidate of slice
    i+1 that equals it, in text order.  A start state that is not among the candidates of a
    slice means the true run dies on that slice's first symbol (it is not in S), or was dead
    already; the rest of the text is then dead."""
    s = int(start)
    pos = []
    first = True
    for lo, hi, runs in slices:
        if first:
            visited, p = runs[s]
            first = False
        elif s in runs:
            visited, p = runs[s]
        else:
            s = NONE
            break
        pos.extend(p)
        if visited:
            s = visited[-1]
    accepted = s != NONE and bool(accept[s])
    return ScanResult(s, accepted, len(pos), np.array(pos, dtype=np.uint64))
