/*
 * parem_oracle.c -- the reference oracle for DFA matching.  TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU legs (the cpu_baseline of a bench
 * line and the --impl reference arm) may load this library.  The product path (libparem) never links, loads or calls it, and it shares no
 * header, table or helper with the CUDA path.
 *
 * What it computes is the plain definition of running a DFA (Q, Sigma, delta, q0, F) over a
 * text, one symbol at a time (Section II-A, the DFA quintuple; Section II-B, where the
 * sequential run starts in q0 and takes one step per symbol).  There is no chunking and no
 * speculation here; the parallel method of Algorithm 1 must reproduce exactly this result.
 *
 * Readings of the paper that this file fixes:
 *   - Undefined transitions (Algorithm 1 tests "Tt[q][c] in Q", i.e. an entry may be
 *     missing) and bytes outside the alphabet lead to an implicit absorbing, non-accepting
 *     dead state.  The dead state is reported as ORACLE_NONE.
 *   - A match is counted after each symbol whose transition lands in F (Algorithm 1 counts
 *     found++ when Tt[r][char] is in F).  The position reported is the 0-based index of
 *     that symbol, so positions are ascending and there is at most one per index.  The
 *     start state itself is never counted, even when q0 is in F.
 *   - "accepted" (Section II-A) is final_state in F; for an empty text it is q0 in F.
 *
 * Written in plain C99 so that it builds with gcc on both x86-64 and aarch64.
 */
#include <stddef.h>
#include <stdint.h>

#define ORACLE_NONE 0xFFFFFFFFu
#define ORACLE_NONE16 0xFFFFu

#define ORACLE_OK 0
#define ORACLE_EINVAL -1

/*
 * oracle_dfa_scan
 *   table          n_states * n_symbols entries, row-major table[q * n_symbols + a]; each
 *                  entry is a state index < n_states or ORACLE_NONE (undefined).
 *   byte_to_symbol 256 entries mapping a text byte to a symbol < n_symbols or ORACLE_NONE16;
 *                  NULL means byte b is symbol b when b < n_symbols, else outside Sigma.
 *   start          q0.
 *   accept         n_states flags, nonzero = state in F.
 *   text, n        the input T.
 *   positions      optional (may be NULL): receives the first `capacity` match positions.
 *   final_state    receives the state after the last symbol (ORACLE_NONE when dead).
 *   match_count    receives the number of matches (all of them, even beyond capacity).
 * Returns ORACLE_OK, or ORACLE_EINVAL when an argument is out of range.
 */
int oracle_dfa_scan(const uint32_t* table, uint32_t n_states, uint32_t n_symbols,
                    const uint16_t* byte_to_symbol, uint32_t start, const uint8_t* accept,
                    const uint8_t* text, uint64_t n, uint64_t* positions, uint64_t capacity,
                    uint32_t* final_state, uint64_t* match_count) {
  if (!table || !accept || !final_state || !match_count) return ORACLE_EINVAL;
  if (n_states == 0 || n_symbols == 0 || n_symbols > 256 || start >= n_states) return ORACLE_EINVAL;
  if (n > 0 && !text) return ORACLE_EINVAL;

  uint32_t s = start; /* ORACLE_NONE once the run has died */
  uint64_t count = 0;
  for (uint64_t j = 0; j < n; ++j) {
    if (s == ORACLE_NONE) break; /* the dead state absorbs the rest of the text */
    uint32_t b = text[j];
    uint32_t a;
    if (byte_to_symbol) {
      a = byte_to_symbol[b];
      if (a == ORACLE_NONE16) a = ORACLE_NONE;
    } else {
      a = (b < n_symbols) ? b : ORACLE_NONE;
    }
    if (a != ORACLE_NONE && a >= n_symbols) return ORACLE_EINVAL;
    uint32_t next = (a == ORACLE_NONE) ? ORACLE_NONE : table[(uint64_t)s * n_symbols + a];
    if (next != ORACLE_NONE && next >= n_states) return ORACLE_EINVAL;
    s = next;
    if (s != ORACLE_NONE && accept[s]) {
      if (positions && count < capacity) positions[count] = j;
      ++count;
    }
  }
  *final_state = s;
  *match_count = count;
  return ORACLE_OK;
}

/*
 * oracle_dfa_trace: the visited-state vector of one run (the vector Rr of Algorithm 1),
 * i.e. the state after each of the n symbols, ORACLE_NONE once dead.  Used by the tests
 * that pin the oracle against the worked example (Table II).
 */
int oracle_dfa_trace(const uint32_t* table, uint32_t n_states, uint32_t n_symbols,
                     const uint16_t* byte_to_symbol, uint32_t start, const uint8_t* text,
                     uint64_t n, uint32_t* visited) {
  if (!table || !visited || n_states == 0 || n_symbols == 0 || n_symbols > 256) return ORACLE_EINVAL;
  if (start != ORACLE_NONE && start >= n_states) return ORACLE_EINVAL;
  uint32_t s = start;
  for (uint64_t j = 0; j < n; ++j) {
    if (s != ORACLE_NONE) {
      uint32_t b = text[j];
      uint32_t a;
      if (byte_to_symbol) {
        a = byte_to_symbol[b];
        if (a == ORACLE_NONE16) a = ORACLE_NONE;
      } else {
        a = (b < n_symbols) ? b : ORACLE_NONE;
      }
      s = (a == ORACLE_NONE) ? ORACLE_NONE : table[(uint64_t)s * n_symbols + a];
      if (s != ORACLE_NONE && s >= n_states) return ORACLE_EINVAL;
    }
    visited[j] = s;
  }
  return ORACLE_OK;
}
