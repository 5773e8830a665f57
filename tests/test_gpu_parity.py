"""Parity of the CUDA path (through the C ABI) with the CPU oracle: bit-exact final state,
acceptance, match count and match positions.  All inputs are seeded and synthetic."""
import numpy as np
import pytest

import paper_1412_1741_gb300 as pm
from oracle import oracle
from paper_1412_1741_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
NONE = pm.PAREM_NONE


@pytest.fixture(scope="module")
def torch():
    import torch as _t

    from paper_1412_1741_gb300 import build

    build.build()
    pm.load_library()
    assert _t.cuda.is_available()
    return _t


_DFA_CACHE = {}


def load(spec):
    key = id(spec)
    if key not in _DFA_CACHE:
        _DFA_CACHE[key] = (spec, pm.parem_load_dfa(spec.table, spec.byte_to_symbol, spec.start, spec.accept))
    return _DFA_CACHE[key][1]


def device_text(torch, text, offset=0):
    n = int(text.size)
    buf = torch.zeros(n + offset + 64, dtype=torch.uint8, device="cuda")
    view = buf[offset:offset + n]
    if n:
        view.copy_(torch.from_numpy(np.ascontiguousarray(text)))
    return buf, view


def check(torch, spec, text, offset=0, opts=None, positions=True, capacity=None, start=None):
    dfa = load(spec)
    _, view = device_text(torch, text, offset)
    st = spec.start if start is None else start
    want = oracle.scan(spec.table, spec.byte_to_symbol, st, spec.accept, text, want_positions=positions)
    cap = capacity if capacity is not None else max(want.match_count, 1)
    pos = torch.full((cap,), -1, dtype=torch.int64, device="cuda") if positions else None
    if opts is None and start is None:
        got = pm.parem_match(dfa, view, pos, length=text.size)
    else:
        o = opts or pm.MatchOpts()
        if start is not None:
            o.start_state = start
            o.use_start_state = 1
        got = pm.parem_match_ex(dfa, view, pos, o, length=text.size)
    assert got.final_state == want.final_state
    assert got.accepted == want.accepted
    assert got.match_count == want.match_count
    if positions:
        k = min(cap, want.match_count)
        assert got.n_written == k
        g = pos[:k].cpu().numpy().astype(np.uint64)
        assert np.array_equal(g, want.positions[:k])
        if want.match_count > cap:
            assert got.status == -3
    return got, want


def random_partial(seed, n, k, p_none=0.1, b2s_frac=0.9):
    rng = np.random.default_rng(seed)
    t = rng.integers(0, n, size=(n, k)).astype(np.uint32)
    t[rng.random((n, k)) < p_none] = NONE
    acc = (rng.random(n) < 0.2).astype(np.uint8)
    b2s = np.full(256, pm.PAREM_NONE16, np.uint16)
    keep = rng.random(256) < b2s_frac
    b2s[keep] = rng.integers(0, k, size=int(keep.sum()))
    return wl.DfaSpec(t, int(rng.integers(0, n)), acc, b2s, f"partial{seed}")


# ---------------------------------------------------------------------------------------
GATTACA = wl.gattaca_dfa()
PARALLEL = wl.parallel_dfa()
AC = wl.keywords_ac_dfa()
DENSE = wl.dense_dfa()
PARITY = wl.DfaSpec(np.array([[1, 0], [0, 1]], np.uint32), 0, np.array([1, 0], np.uint8), None, "parity")
MOD3 = wl.DfaSpec(np.array([[(2 * q + a) % 3 for a in range(2)] for q in range(3)], np.uint32), 0,
                  np.array([1, 0, 0], np.uint8), None, "mod3")


def test_paper_worked_example(torch):
    text = np.frombuffer(bytes(wl.PARALLEL_ALPHABET.index(c) for c in b"plaraparallelapareparapl"), np.uint8)
    got, want = check(torch, PARALLEL, text)
    assert (got.match_count, want.positions.tolist()) == (1, [12])


@pytest.mark.parametrize("n", [0, 1, 15, 16, 17, 100, 143, 144, 145, 1000, 4095, 4096, 4097, 65549, 300001])
@pytest.mark.parametrize("offset", [0, 1, 7, 15])
def test_lengths_and_alignments_gattaca(torch, n, offset):
    check(torch, GATTACA, wl.uniform_text(n, 4, seed=n + offset), offset=offset)


@pytest.mark.parametrize("seg", [128, 256, 384, 2048])
@pytest.mark.parametrize("spec", [GATTACA, PARALLEL, AC, DENSE], ids=lambda s: s.name)
def test_many_chunks_forced_segments(torch, spec, seg):
    n = 200_000 + 37
    if spec is AC:
        text = wl.zipf_words_text(n, plant_rate=3e-4)
    elif spec is DENSE:
        text = wl.uniform_text(n, 256, seed=5)
    else:
        text = wl.uniform_text(n, spec.n_symbols, seed=seg)
    check(torch, spec, text, offset=3, opts=pm.MatchOpts(segment_bytes=seg))


@pytest.mark.parametrize("seed", range(6))
def test_partial_dfas_with_dead_states(torch, seed):
    spec = random_partial(seed, n=int(np.random.default_rng(seed).integers(2, 40)), k=3, p_none=0.02 * seed)
    rng = np.random.default_rng(100 + seed)
    text = rng.integers(0, 256, size=150_000, dtype=np.uint8)
    check(torch, spec, text, opts=pm.MatchOpts(segment_bytes=256))
    check(torch, spec, text[:5000], offset=5)


@pytest.mark.parametrize("spec", [PARITY, MOD3], ids=lambda s: s.name)
def test_non_converging_dfas_use_slot_maps(torch, spec):
    text = wl.uniform_text(120_000 + 5, 2, seed=1)
    check(torch, spec, text, opts=pm.MatchOpts(segment_bytes=128))
    check(torch, spec, text, opts=pm.MatchOpts(segment_bytes=1024), offset=9)


def test_more_candidates_than_registers(torch):
    # 1200 states over 4 symbols: |img(c)| ~ 760 > 256 candidates held in registers
    t, acc = wl.random_dfa(1200, 4, 100, seed=21)
    spec = wl.DfaSpec(t, 0, acc, None, "rand1200")
    text = wl.uniform_text(40_000, 4, seed=2)
    check(torch, spec, text, opts=pm.MatchOpts(segment_bytes=256))


def test_large_table_in_global_memory(torch):
    t, acc = wl.random_dfa(3000, 40, 300, seed=22)  # 3000 x 40 x 2 B > shared-memory budget
    spec = wl.DfaSpec(t, 0, acc, None, "rand3000")
    assert pm.parem_prepare_info(t, None, 0, acc).layout == 2
    check(torch, spec, wl.uniform_text(300_000, 40, seed=3), opts=pm.MatchOpts(segment_bytes=4096))


@pytest.mark.parametrize("spec", [GATTACA, PARALLEL], ids=lambda s: s.name)
def test_enumeration_mode(torch, spec):
    text = wl.uniform_text(100_000, spec.n_symbols, seed=4)
    check(torch, spec, text, opts=pm.MatchOpts(enumerate_all=1, segment_bytes=256))


def test_carry_in_start_state(torch):
    text = wl.uniform_text(250_000, 4, seed=6)
    whole = oracle.scan(GATTACA.table, None, 0, GATTACA.accept, text)
    cut = 123_457
    a, _ = check(torch, GATTACA, text[:cut])
    b, _ = check(torch, GATTACA, text[cut:], start=a.final_state, opts=pm.MatchOpts(segment_bytes=512))
    assert a.match_count + b.match_count == whole.match_count
    assert b.final_state == whole.final_state


def test_capacity_and_count_only(torch):
    text = wl.uniform_text(500_000, 4, seed=7)
    got, want = check(torch, GATTACA, text, capacity=5)
    assert got.status == -3 and got.n_written == 5
    got, _ = check(torch, GATTACA, text, positions=False)
    assert got.n_written == 0


def test_zipf_words_ac_64mb(torch):
    text = wl.zipf_words_text(64 << 20)
    check(torch, AC, text, offset=1)


def test_dense_64mb(torch):
    text = wl.uniform_text(64 << 20, 256, seed=5)
    check(torch, DENSE, text, offset=2)


def test_timeout_hook_reports_error_and_context_survives(torch):
    text = wl.uniform_text(300_000, 4, seed=8)
    dfa = load(GATTACA)
    _, view = device_text(torch, text)
    o = pm.MatchOpts(segment_bytes=128, debug_skip_publish_chunk=3, wait_budget_cycles=200_000_000)
    with pytest.raises(pm.ParemError) as e:
        pm.parem_match_ex(dfa, view, None, o, length=text.size)
    assert e.value.status == -4
    check(torch, GATTACA, text)  # the context is still usable


def test_host_buffers(torch):
    text = wl.uniform_text(1 << 20, 4, seed=0)
    want = oracle.scan(GATTACA.table, None, 0, GATTACA.accept, text)
    pos = np.zeros(max(1, want.match_count), np.uint64)
    got = pm.parem_match_host(load(GATTACA), text, pos)
    assert (got.final_state, got.match_count) == (want.final_state, want.match_count)
    assert np.array_equal(pos[:got.n_written], want.positions)


@pytest.mark.parametrize("n_sym,n_states", [(1, 3), (2, 5), (3, 17), (4, 31), (5, 12)])
def test_four_byte_stride_table(torch, n_sym, n_states):
    # small DFAs over bytes 0..n_sym-1 (every other byte is outside the alphabet): the main
    # run advances 4 bytes per lookup (layout 6); texts include outside bytes and lengths
    # that are not multiples of 4 or 16
    t, acc = wl.random_dfa(n_states, n_sym, max(1, n_states // 4), seed=100 + n_states)
    spec = wl.DfaSpec(t, 0, acc, None, f"stride{n_sym}x{n_states}")
    assert pm.parem_prepare_info(t, None, 0, acc).layout == 6
    rng = np.random.default_rng(n_states)
    text = rng.integers(0, n_sym, size=300_003).astype(np.uint8)
    text[rng.random(text.size) < 0.001] = 200  # outside bytes kill the run
    check(torch, spec, text, offset=3, opts=pm.MatchOpts(segment_bytes=1024))
    check(torch, spec, text[:77_777], opts=pm.MatchOpts(segment_bytes=128))
    clean = rng.integers(0, n_sym, size=250_001).astype(np.uint8)
    check(torch, spec, clean, offset=5)
    # outside bytes next to the clamp boundaries of the four-at-once symbol clamp (K - 1,
    # K, 127, 128, 128 + K - 1, 255 for K = n_sym + 1 classes) must all take the outside class
    edge = np.array([n_sym, n_sym + 1, 6, 7, 127, 128, 128 + n_sym - 1, 128 + n_sym, 133, 255], np.uint8)
    sprinkled = rng.integers(0, n_sym, size=200_001).astype(np.uint8)
    where = rng.random(sprinkled.size) < 3e-4
    sprinkled[where] = rng.choice(edge, size=int(where.sum()))
    check(torch, spec, sprinkled, offset=1, opts=pm.MatchOpts(segment_bytes=512))


@pytest.mark.parametrize("extra", [32, 200, None])
def test_computed_columns(torch, extra):
    # bytes 97..122 are symbols 0..25 and one extra byte (below or above 128) symbol 26; all
    # other bytes are outside the alphabet: layout 7 computes the column from the byte.
    # Texts draw every byte value so the in-register column arithmetic sees them all.
    n_sym = 27 if extra is not None else 26
    t, acc = wl.random_dfa(600, n_sym, 60, seed=31 + (extra or 0))
    b2s = np.full(256, pm.PAREM_NONE16, np.uint16)
    b2s[97:123] = np.arange(26)
    if extra is not None:
        b2s[extra] = 26
    spec = wl.DfaSpec(t, 0, acc, b2s, f"win{extra}")
    assert pm.parem_prepare_info(t, b2s, 0, acc).layout == 7
    rng = np.random.default_rng(7)
    letters = rng.integers(97, 123, size=400_000).astype(np.uint8)
    noise = rng.random(letters.size)
    letters[noise < 0.02] = extra if extra is not None else 97
    letters[noise > 0.99995] = rng.integers(0, 256, size=int((noise > 0.99995).sum())).astype(np.uint8)
    check(torch, spec, letters, offset=9, opts=pm.MatchOpts(segment_bytes=4096))
    check(torch, spec, rng.integers(0, 256, size=50_001).astype(np.uint8), opts=pm.MatchOpts(segment_bytes=256))


def test_sparse_counting_after_a_sparse_scan(torch):
    # the first scan of a DFA learns its match density; once it is below one match per KiB,
    # scans count matches only in the 16-byte vectors whose largest state is accepting
    # (with a replay of that vector).  Both modes must give the oracle's result.
    kws = wl.random_keywords(24, 6, 12, seed=8)
    sym = wl.letters_byte_map()
    t, acc = wl.aho_corasick_dfa([[int(sym[b]) for b in kw] for kw in kws], 27)
    spec = wl.DfaSpec(t, 0, acc, sym, "ac24-sparse", {"keywords": kws})
    text = wl.zipf_words_text(6 << 20, seed_words=4, seed_plants=5, plant_rate=2e-4, keywords=kws)
    want = oracle.scan(spec.table, spec.byte_to_symbol, spec.start, spec.accept, text)
    assert 0 < want.match_count < 1024 * 6
    dfa = pm.parem_load_dfa(spec.table, spec.byte_to_symbol, spec.start, spec.accept)
    _, view = device_text(torch, text, 3)
    for _ in range(3):  # dense first, then sparse
        pos = torch.full((want.match_count,), -1, dtype=torch.int64, device="cuda")
        got = pm.parem_match(dfa, view, pos, length=text.size)
        assert (got.final_state, got.match_count) == (want.final_state, want.match_count)
        assert np.array_equal(pos.cpu().numpy().astype(np.uint64), want.positions)
        cnt = pm.parem_match(dfa, view, length=text.size)  # count only
        assert cnt.match_count == want.match_count
    dfa.free()


@pytest.mark.parametrize("offset,cap_div", [(0, 1), (7, 1), (3, 3)])
def test_clustered_matches_after_a_sparse_scan(torch, offset, cap_div):
    # a DFA whose last scan was sparse counts per vector (sparse counting); a text with a
    # dense cluster of keywords (rows with more matches than pass 1 records), keywords at
    # row starts (matches inside merged prefixes) and in the unaligned head must still give
    # every position in order, with and without capacity truncation
    kws = wl.random_keywords(24, 6, 12, seed=8)
    sym = wl.letters_byte_map()
    t, acc = wl.aho_corasick_dfa([[int(sym[b]) for b in kw] for kw in kws], 27)
    spec = wl.DfaSpec(t, 0, acc, sym, "ac24-cluster", {"keywords": kws})
    sparse = wl.zipf_words_text(4 << 20, seed_words=4, seed_plants=5, plant_rate=1e-5, keywords=kws)
    text = wl.zipf_words_text(5 << 20, seed_words=6, seed_plants=7, plant_rate=2e-5, keywords=kws)
    rng = np.random.default_rng(offset)
    pos = 1000
    while pos < 300_000:  # cluster: a keyword every ~20 bytes
        kw = kws[int(rng.integers(len(kws)))]
        text[pos:pos + len(kw)] = np.frombuffer(kw, np.uint8)
        pos += len(kw) + int(rng.integers(1, 12))
    for start in range(0, text.size - 64, 4096 * 7 + 64):  # keywords at scattered 64-aligned offsets
        kw = kws[start % len(kws)]
        text[start:start + len(kw)] = np.frombuffer(kw, np.uint8)
    text[:len(kws[0])] = np.frombuffer(kws[0], np.uint8)  # a match inside the head bytes
    dfa = pm.parem_load_dfa(spec.table, spec.byte_to_symbol, spec.start, spec.accept)
    _, sview = device_text(torch, sparse, 0)
    want = oracle.scan(spec.table, spec.byte_to_symbol, spec.start, spec.accept, text)
    assert want.match_count > 10_000
    _, view = device_text(torch, text, offset)
    for opts in (None, pm.MatchOpts(segment_bytes=1024), pm.MatchOpts(segment_bytes=128)):
        # a sparse scan first, so that this scan of the clustered text counts sparsely
        assert pm.parem_match(dfa, sview, length=sparse.size).match_count < 1024 * 4
        cap = want.match_count // cap_div
        pos_t = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
        got = pm.parem_match_ex(dfa, view, pos_t, opts, length=text.size)
        assert (got.final_state, got.match_count, got.n_written) == (want.final_state, want.match_count, cap)
        assert np.array_equal(pos_t.cpu().numpy().astype(np.uint64), want.positions[:cap])
    dfa.free()


@pytest.mark.parametrize("seg", [0, 4160, 8192, 196608])
def test_dense_emission(torch, seg):
    # dense matches (10 %, then a stretch where every byte matches): positions in order,
    # with and without capacity truncation
    spec = wl.dense_dfa()
    rng = np.random.default_rng(seg)
    text = rng.integers(0, 256, size=(6 << 20) + 4099).astype(np.uint8)
    # in the last 1 MiB the automaton accepts after every byte (ten times the density)
    t = np.asarray(spec.table)
    acc = np.asarray(spec.accept).astype(bool)
    q = int(oracle.scan(spec.table, None, spec.start, spec.accept, text[: -(1 << 20)]).final_state)
    first_acc = np.argmax(acc[t], axis=1)  # per state, the first byte that leads to F
    tail = np.empty(1 << 20, np.uint8)
    for j in range(tail.size):
        tail[j] = first_acc[q]
        q = int(t[q, tail[j]])
    text[-(1 << 20):] = tail
    _, view = device_text(torch, text, 5)
    o = pm.MatchOpts(segment_bytes=seg)
    want = oracle.scan(spec.table, spec.byte_to_symbol, spec.start, spec.accept, text)
    assert want.match_count > (text.size >> 6) + (1 << 20)
    # a fresh DFA emits row by row; once a scan of it has seen the density, the emit pass
    # streams the rows through shared memory and writes each lane's positions warp-wide
    # (rows of 192 KiB take the buffers' base column past 64 KiB; the last row's tail is
    # replayed from global memory)
    for learn in (False, True):
        dfa = pm.parem_load_dfa(spec.table, spec.byte_to_symbol, spec.start, spec.accept)
        if learn:
            assert pm.parem_match_ex(dfa, view, None, o, length=text.size).match_count == want.match_count
        for cap in (want.match_count, want.match_count // 3):
            pos = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
            got = pm.parem_match_ex(dfa, view, pos, o, length=text.size)
            assert (got.final_state, got.match_count, got.n_written) == (want.final_state, want.match_count, cap)
            assert np.array_equal(pos.cpu().numpy().astype(np.uint64), want.positions[:cap])
        dfa.free()


def test_host_buffers_in_pieces(torch):
    # 200 MiB: the host path copies and scans 64 MiB pieces, each from the state the previous
    # one ended in; positions of all pieces land in one buffer, in order, with a capacity
    # that runs out inside a later piece
    n = 200 << 20
    text_dev = wl.uniform_text_device(n, 4, torch.device("cuda"), seed=12)
    host = text_dev.cpu().numpy()
    dfa = load(GATTACA)
    ref_pos = torch.full((4096,), -1, dtype=torch.int64, device="cuda")
    ref = pm.parem_match(dfa, text_dev, ref_pos)
    assert ref.match_count > 2000
    for cap in (4096, 1500):
        pos = np.zeros(cap, np.uint64)
        got = pm.parem_match_host(dfa, host, pos)
        assert (got.final_state, got.accepted, got.match_count) == (ref.final_state, ref.accepted, ref.match_count)
        assert got.n_written == min(cap, ref.match_count)
        assert np.array_equal(pos[:got.n_written], ref_pos[:got.n_written].cpu().numpy().astype(np.uint64))
    # a partial DFA (KMP of "GAT" with C undefined) whose run dies in the second piece: the
    # matches before the death count, nothing after it does
    t, acc = wl.kmp_dfa([2, 0, 3], 4)
    t = np.array(t, dtype=np.uint32)
    t[:, 1] = NONE
    spec = wl.DfaSpec(t, 0, acc, None, "gat-no-C")
    host2 = host.copy()
    head = host2[: 100 << 20]
    head[head == 1] = 0  # no C before 100 MiB
    host2[(100 << 20) + 5] = 1
    want = oracle.scan(spec.table, None, 0, spec.accept, host2[: (100 << 20) + 64])
    assert want.match_count > 1000 and want.final_state == NONE
    got = pm.parem_match_host(load(spec), host2, None)
    assert got.final_state == pm.PAREM_NONE and not got.accepted
    assert got.match_count == want.match_count


@pytest.mark.parametrize("n_states,n_sym,layout", [(400, 140, 3), (450, 200, 4), (150, 4, 0), (700, 100, 1),
                                                   (700, 30, 7), (500, 60, 7)])
def test_table_layouts_and_register_counts(torch, n_states, n_sym, layout):
    t, acc = wl.random_dfa(n_states, n_sym, max(1, n_states // 10), seed=n_states + n_sym)
    spec = wl.DfaSpec(t, 0, acc, None, f"rand{n_states}x{n_sym}")
    assert pm.parem_prepare_info(t, None, 0, acc).layout == layout
    text = wl.uniform_text(150_000, n_sym, seed=n_sym)
    check(torch, spec, text, offset=6, opts=pm.MatchOpts(segment_bytes=2048))
    check(torch, spec, text[:40_000], opts=pm.MatchOpts(segment_bytes=128))


@pytest.mark.parametrize("seg", [128, 640, 4096])
def test_grouped_speculation_row_packing(torch, seg):
    # candidate sets of 1..4 states (G = 4): eight rows speculated per warp pass
    for spec in (GATTACA, PARALLEL):
        text = wl.uniform_text(300_000 + 11, spec.n_symbols + 1, seed=seg)  # includes bytes outside Sigma
        check(torch, spec, text, offset=seg % 16, opts=pm.MatchOpts(segment_bytes=seg))


def test_emit_windows_with_sparse_and_clustered_matches(torch):
    # rows with one match, two distant matches and many matches in between
    kws = wl.random_keywords(8, 3, 6, seed=3)
    sym = wl.letters_byte_map()
    t, acc = wl.aho_corasick_dfa([[int(sym[b]) for b in kw] for kw in kws], 27)
    spec = wl.DfaSpec(t, 0, acc, sym, "ac8")
    text = wl.zipf_words_text(1 << 20, plant_rate=2e-3, keywords=kws)
    text[300_000:300_400] = np.frombuffer((kws[0] + b" ") * 100, np.uint8)[:400]
    check(torch, spec, text, offset=4, opts=pm.MatchOpts(segment_bytes=1024))
    check(torch, spec, text, offset=0)


@pytest.mark.parametrize("n_states,n_sym,seg", [(4096, 256, 8192), (2000, 27, 2048), (600, 4, 1024)])
def test_bitmap_phase_for_large_candidate_sets(torch, n_states, n_sym, seg):
    # |img(c)| ~ 0.63 n > 256: candidates start as a per-warp bitmap, then move to registers
    t, acc = wl.random_dfa(n_states, n_sym, n_states // 10, seed=n_states)
    spec = wl.DfaSpec(t, 0, acc, None, f"rand{n_states}x{n_sym}")
    assert pm.parem_prepare_info(t, None, 0, acc).max_candidates > 256
    text = wl.uniform_text(400_000 + 3, n_sym, seed=9)
    check(torch, spec, text, offset=5, opts=pm.MatchOpts(segment_bytes=seg))


def test_enumeration_mode_with_bitmap(torch):
    t, acc = wl.random_dfa(600, 8, 60, seed=33)
    spec = wl.DfaSpec(t, 0, acc, None, "rand600x8")
    text = wl.uniform_text(200_000, 8, seed=10)
    check(torch, spec, text, opts=pm.MatchOpts(enumerate_all=1, segment_bytes=2048))


@pytest.mark.parametrize("pattern,anchored", [("(a|b)?c*[0..3]b+", False), ("(ab|c)*d", True),
                                               ("x[^ab]y|[0..9]+\\.[0..9]", False),
                                               ("(a|b)*a(a|b)(a|b)(a|b)(a|b)", False)])
def test_regex_dfa_scan(torch, pattern, anchored):
    # a DFA compiled from a regular expression (Table III operators) scanned on the GPU
    # equals the oracle's run of the same DFA (layouts and speculation as for any DFA)
    r = pm.parem_regex_compile(pattern, pm.PAREM_REGEX_ANCHORED if anchored else 0)
    spec = wl.DfaSpec(r.table, r.start, r.accept, r.byte_to_symbol, f"re:{pattern}")
    rng = np.random.default_rng(len(pattern))
    text = rng.choice(np.frombuffer(b"abcdxy0123.", np.uint8), size=(3 << 20) + 77)
    check(torch, spec, text, offset=3)
    check(torch, spec, text[:50_001], opts=pm.MatchOpts(segment_bytes=256))


def test_text_longer_than_4gib_against_the_oracle(torch):
    # The sparse-DFA workload at 4 GiB + 4,097 bytes viewed at an odd offset: row index x row
    # length, the position bases and the chunk count pass 2^32 here.  Final state, count and
    # every position are compared with the oracle's run over the same bytes, through the
    # device entry point and through the host-buffer entry point (pieces, carry-in starts).
    n = (4 << 30) + 4097
    dev = torch.device("cuda")
    src = wl.zipf_words_text_device(n, dev, seed=2, keywords=AC.meta["keywords"])
    # keywords planted past 2^32 (the last 4,097 bytes hold none at the generator's rate)
    for k, at in enumerate((100, 1500, 3900)):
        kw = AC.meta["keywords"][k]
        src[(1 << 32) + at:(1 << 32) + at + len(kw)] = torch.frombuffer(bytearray(kw), dtype=torch.uint8).to(dev)
    buf = torch.empty(n + 64, dtype=torch.uint8, device=dev)
    view = buf[3:3 + n]
    view.copy_(src)
    del src
    host = view.cpu().numpy()
    want = oracle.scan(AC.table, AC.byte_to_symbol, AC.start, AC.accept, host)
    assert want.match_count > 40_000 and int(want.positions[-1]) > (1 << 32)
    dfa = load(AC)
    pos = torch.full((want.match_count,), -1, dtype=torch.int64, device=dev)
    got = pm.parem_match(dfa, view, pos)
    assert (got.final_state, got.accepted, got.match_count, got.n_written) == \
        (want.final_state, want.accepted, want.match_count, want.match_count)
    assert np.array_equal(pos.cpu().numpy().view(np.uint64), want.positions)
    st = pm.parem_last_stats()
    assert st["rows"] * st["segment_bytes"] > (1 << 32)
    del pos, buf, view
    torch.cuda.empty_cache()
    hpos = np.zeros(want.match_count, np.uint64)
    got = pm.parem_match_host(dfa, host, hpos)
    assert (got.final_state, got.match_count, got.n_written) == (want.final_state, want.match_count, want.match_count)
    assert np.array_equal(hpos, want.positions)


def _pair_spec(n_keywords=64, seed=1, lo=8, hi=24):
    if (n_keywords, seed, lo, hi) == (64, 1, 8, 24):
        return AC
    kws = wl.random_keywords(n_keywords, lo, hi, seed=seed)
    sym = wl.letters_byte_map()
    t, acc = wl.aho_corasick_dfa([[int(sym[b]) for b in kw] for kw in kws], 27)
    return wl.DfaSpec(t, 0, acc, sym, f"ac{n_keywords}-{seed}", {"keywords": kws})


@pytest.mark.parametrize("n_keywords,seed,lo,hi", [(64, 1, 8, 24), (48, 7, 6, 16), (64, 5, 8, 24)])
def test_two_byte_stride_variant(torch, n_keywords, seed, lo, hi):
    # The two-byte stride variant (layout 8) of a computed-column keyword DFA, learned from the
    # first text: scans that use it give the oracle's result on texts of letters and spaces,
    # texts with every other kind of byte sprinkled in (each sends its vector to the byte loop),
    # texts dense with keywords (escapes through accepting states), carry-in starts, capacity
    # limits, count-only calls and forced row lengths.
    spec = _pair_spec(n_keywords, seed, lo, hi)
    kws = spec.meta["keywords"]
    dfa = pm.parem_load_dfa(spec.table, spec.byte_to_symbol, spec.start, spec.accept)
    assert pm.parem_dfa_get_info(dfa).layout == 7
    learn_text = wl.zipf_words_text(6 << 20, seed_words=3, seed_plants=4, plant_rate=1e-4, keywords=kws)
    _, lview = device_text(torch, learn_text, 0)
    first = pm.parem_match_ex(dfa, lview, None, pm.MatchOpts(pair_mode=pm.PAREM_PAIR_LEARN), length=learn_text.size)
    assert pm.parem_last_stats()["layout"] == 7  # the scan that learns still runs layout 7
    want0 = oracle.scan(spec.table, spec.byte_to_symbol, spec.start, spec.accept, learn_text, want_positions=False)
    assert (first.final_state, first.match_count) == (want0.final_state, want0.match_count)
    hot = pm.parem_dfa_get_info(dfa).pair_hot_states
    assert 2 <= hot <= 254
    rng = np.random.default_rng(seed)
    plain = wl.zipf_words_text((3 << 20) + 11, seed_words=7, seed_plants=8, plant_rate=3e-4, keywords=kws)
    noisy = plain.copy()
    odd = np.array([0x00, 0x1F, 0x21, 0x3A, 0x3F, 0x40, 0x41, 0x5A, 0x5F, 0x60, 0x7B, 0x7E, 0x7F, 0x80, 0xC1, 0xE0,
                    0xFA, 0xFF], np.uint8)
    where = rng.random(noisy.size) < 2e-4
    noisy[where] = rng.choice(odd, size=int(where.sum()))
    dense = plain.copy()
    p = 5000
    while p < 400_000:  # a keyword every few bytes
        kw = kws[int(rng.integers(len(kws)))]
        dense[p:p + len(kw)] = np.frombuffer(kw, np.uint8)
        p += len(kw) + int(rng.integers(0, 4))
    for text, offset, opts in ((plain, 3, None), (noisy, 0, None), (dense, 5, None),
                               (plain, 7, pm.MatchOpts(segment_bytes=1024)), (noisy, 1, pm.MatchOpts(segment_bytes=128))):
        want = oracle.scan(spec.table, spec.byte_to_symbol, spec.start, spec.accept, text)
        _, view = device_text(torch, text, offset)
        for cap in (max(1, want.match_count), max(1, want.match_count // 3)):
            pos = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
            got = pm.parem_match_ex(dfa, view, pos, opts, length=text.size)
            assert pm.parem_last_stats()["layout"] == 8
            assert (got.final_state, got.accepted, got.match_count) == (want.final_state, want.accepted, want.match_count)
            k = min(cap, want.match_count)
            assert got.n_written == k
            assert np.array_equal(pos[:k].cpu().numpy().view(np.uint64), want.positions[:k])
        cnt = pm.parem_match_ex(dfa, view, None, opts, length=text.size)
        assert (cnt.final_state, cnt.match_count) == (want.final_state, want.match_count)
        # the plain variant, declined for one call, agrees
        off = pm.parem_match_ex(dfa, view, None, pm.MatchOpts(pair_mode=pm.PAREM_PAIR_OFF), length=text.size)
        assert pm.parem_last_stats()["layout"] == 7
        assert (off.final_state, off.match_count) == (want.final_state, want.match_count)
    # carry-in start states through the renumbered variant
    cut = 1_234_567
    whole = oracle.scan(spec.table, spec.byte_to_symbol, spec.start, spec.accept, plain)
    _, va = device_text(torch, plain[:cut], 0)
    _, vb = device_text(torch, plain[cut:], 0)
    a = pm.parem_match(dfa, va, length=cut)
    b = pm.parem_match_ex(dfa, vb, None, pm.MatchOpts(start_state=a.final_state), length=plain.size - cut)
    assert (b.final_state, a.match_count + b.match_count) == (whole.final_state, whole.match_count)
    dfa.free()


def test_two_byte_stride_variant_declined_when_hot_states_do_not_cover(torch):
    # 200 short keywords: the most visited states that fit leave most 16-byte vectors to the byte
    # loop, so the learning step keeps layout 7 (and the results are the oracle's either way)
    spec = _pair_spec(200, 9, 3, 10)
    dfa = pm.parem_load_dfa(spec.table, spec.byte_to_symbol, spec.start, spec.accept)
    text = wl.zipf_words_text(6 << 20, seed_words=3, seed_plants=4, plant_rate=1e-4, keywords=spec.meta["keywords"])
    _, view = device_text(torch, text, 0)
    want = oracle.scan(spec.table, spec.byte_to_symbol, spec.start, spec.accept, text, want_positions=False)
    for _ in range(2):
        got = pm.parem_match_ex(dfa, view, None, pm.MatchOpts(pair_mode=pm.PAREM_PAIR_LEARN), length=text.size)
        assert (got.final_state, got.match_count) == (want.final_state, want.match_count)
        assert pm.parem_last_stats()["layout"] == 7
    assert pm.parem_dfa_get_info(dfa).pair_hot_states == 0
    dfa.free()
