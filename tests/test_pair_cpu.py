"""The two-byte stride variant's plan on the host (no GPU), through parem_pair_preview: every
entry of its pair table against two steps of the oracle's transition function, the choice of
hot states against the state visits of the oracle's run over the sample, and the estimated
share of 16-byte vector steps that need the byte loop against a direct count."""
import numpy as np
import pytest

import paper_1412_1741_gb300 as pm
from oracle import oracle
from paper_1412_1741_gb300 import workloads as wl

NONE = oracle.NONE


def _ac(n_keywords, lo, hi, seed):
    kws = wl.random_keywords(n_keywords, lo, hi, seed=seed)
    sym = wl.letters_byte_map()
    t, acc = wl.aho_corasick_dfa([[int(sym[b]) for b in kw] for kw in kws], 27)
    return wl.DfaSpec(t, 0, acc, sym, f"ac{n_keywords}", {"keywords": kws})


def _code_byte(f):
    return 0x20 if f == 0 else 0x60 + f


@pytest.fixture(scope="module")
def lib():
    from paper_1412_1741_gb300 import build

    build.build()
    return pm.load_library()


@pytest.mark.parametrize("n_keywords,lo,hi,seed", [(64, 8, 24, 1), (48, 6, 16, 7)])
def test_pair_table_entries_are_two_oracle_steps(lib, n_keywords, lo, hi, seed):
    spec = wl.keywords_ac_dfa() if seed == 1 else _ac(n_keywords, lo, hi, seed)
    sample = wl.zipf_words_text(1 << 20, seed_words=3, seed_plants=4, plant_rate=1e-4, keywords=spec.meta["keywords"])
    pv = pm.parem_pair_preview(spec.table, spec.byte_to_symbol, spec.start, spec.accept, sample)
    assert pv.layout == 7 and 2 <= pv.hot_states <= 254
    H = pv.hot_states
    table = [list(map(int, r)) for r in np.asarray(spec.table)]
    acc = np.asarray(spec.accept).astype(bool)
    n_sym = len(table[0])
    hot = [int(q) for q in pv.hot_orig]
    assert len(set(hot)) == H and not any(acc[q] for q in hot)
    index = {q: e for e, q in enumerate(hot)}

    def step(q, b):
        return oracle.step(table, q, oracle.symbol_of(spec.byte_to_symbol, n_sym, b))

    for e, q in enumerate(hot):
        for f0 in range(27):
            y = step(q, _code_byte(f0))
            for f1 in range(27):
                z = step(y, _code_byte(f1))
                esc = (y == NONE or acc[y] or z == NONE or acc[z] or z not in index)
                assert int(pv.pair_table[e, f0 * 27 + f1]) == (H if esc else index[z]), (e, f0, f1)
    assert (pv.pair_table[H] == H).all()
    # the hot states are the most visited non-accepting states of the run over the sample
    # (after its first 64 bytes)
    vis = oracle.trace(spec.table, spec.byte_to_symbol, spec.start, sample).astype(np.int64)[64:]
    counts = np.bincount(vis[vis >= 0], minlength=len(table))
    cold_live = [q for q in range(len(table)) if not acc[q] and q not in index]
    assert min(counts[q] for q in hot) >= max([counts[q] for q in cold_live] or [0])
    # the estimate: a 16-byte vector (aligned to the sample) is fast when it starts in a hot
    # state, holds only spaces and lowercase letters, and every pair stays hot and non-accepting
    states = oracle.trace(spec.table, spec.byte_to_symbol, spec.start, sample).astype(np.int64)
    before = np.concatenate([[spec.start], states[:-1]])
    ok_byte = (sample == 0x20) | ((sample >= 0x61) & (sample <= 0x7A))
    hot_mask = np.zeros(len(table) + 1, bool)
    hot_mask[hot] = True
    acc_mask = np.zeros(len(table) + 1, bool)
    acc_mask[:len(table)] = acc
    m = sample.size // 16 * 16
    s_all = np.where(states[:m] < 0, len(table), states[:m])
    fast = (hot_mask[np.where(before[:m] < 0, len(table), before[:m])].reshape(-1, 16)[:, 0] &
            ok_byte[:m].reshape(-1, 16).all(axis=1) &
            (~acc_mask[s_all]).reshape(-1, 16).all(axis=1) &
            hot_mask[s_all].reshape(-1, 2)[:, 1].reshape(-1, 8).all(axis=1))
    p_slow = 1.0 - fast[4:].mean()  # the first 64 bytes are not counted
    assert pv.warp_slow_share == pytest.approx(1.0 - (1.0 - p_slow) ** 32, rel=1e-9)


def test_pair_preview_declines_where_hot_states_do_not_cover(lib):
    spec = _ac(200, 3, 10, 9)
    sample = wl.zipf_words_text(1 << 20, seed_words=3, seed_plants=4, plant_rate=1e-4, keywords=spec.meta["keywords"])
    pv = pm.parem_pair_preview(spec.table, spec.byte_to_symbol, spec.start, spec.accept, sample)
    assert pv.layout == 7 and pv.hot_states >= 100 and not pv.accepted and pv.warp_slow_share > 0.4


def test_pair_preview_needs_computed_columns(lib):
    # a DFA whose table is byte-indexed (layout 0) has no pair variant
    spec = wl.gattaca_dfa()
    pv = pm.parem_pair_preview(spec.table, spec.byte_to_symbol, spec.start, spec.accept, wl.uniform_text(4096, 4, 0))
    assert pv.layout != 7 and pv.hot_states == 0 and not pv.accepted
