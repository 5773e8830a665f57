"""Batched matching (parem_batch_*): every item's result equals parem_match on that item
(bit-exact final state, acceptance, count and positions), for mixed DFAs, text lengths
(empty, shorter than a row, many chunks), alignments, with and without positions, when the
captured graph is replayed, without the graph, and with the autotuner choosing the segment
sizes."""
import numpy as np
import pytest

import paper_1412_1741_gb300 as pm
from oracle import oracle
from paper_1412_1741_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t

    from paper_1412_1741_gb300 import build

    build.build()
    pm.load_library()
    assert _t.cuda.is_available()
    return _t


def _make(torch, n_items=40, seed=0, max_len=1 << 20):
    specs = wl.batch_dfas(12, seed=seed + 7, max_states=1500) + [wl.gattaca_dfa(), wl.keywords_ac_dfa()]
    dfas = [pm.parem_load_dfa(s.table, s.byte_to_symbol, s.start, s.accept) for s in specs]
    rng = np.random.default_rng(seed)
    lens = [0, 1, 17, 63, 64, 65, 80, 200, 4096, 4097] + list(
        np.exp(rng.uniform(np.log(300), np.log(max_len), size=n_items - 10)).astype(int))
    texts, items, want = [], [], []
    for i, L in enumerate(lens):
        k = i % len(specs)
        spec = specs[k]
        if spec.byte_to_symbol is not None:
            kws = spec.meta.get("keywords")
            text = wl.zipf_words_text(int(L), plant_rate=1e-3, keywords=kws if isinstance(kws, list) else None)
        else:
            text = rng.integers(0, spec.n_symbols, size=int(L), dtype=np.uint8)
        off = int(rng.integers(0, 16))
        buf = torch.zeros(int(L) + off + 16, dtype=torch.uint8, device="cuda")
        view = buf[off:off + int(L)]
        if L:
            view.copy_(torch.from_numpy(np.array(text)))
        ref = pm.parem_match(dfas[k], view, length=int(L))
        cap = max(1, ref.match_count)
        pos = torch.full((cap,), -1, dtype=torch.int64, device="cuda") if i % 3 != 1 else None
        ref_pos = None
        if pos is not None:
            ref_pos = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
            ref = pm.parem_match(dfas[k], view, ref_pos, length=int(L))
        texts.append((buf, view, text))
        items.append((dfas[k], view, pos))
        want.append((ref, ref_pos, spec, text))
    return dfas, texts, items, want


def _check(batch, items, want):
    res = batch.results()
    for (dfa, view, pos), r, (ref, ref_pos, spec, text) in zip(items, res, want):
        assert (r.final_state, r.accepted, r.match_count) == (ref.final_state, ref.accepted, ref.match_count)
        if pos is not None:
            assert r.n_written == ref.n_written
            assert bool((pos[: r.n_written] == ref_pos[: r.n_written]).all())
        else:
            assert r.n_written == 0


@pytest.mark.parametrize("use_graph", [1, 0])
def test_batch_matches_per_item_scans(torch, use_graph):
    dfas, texts, items, want = _make(torch)
    batch = pm.parem_batch_create(items, pm.BatchOpts(use_graph=use_graph))
    for _ in range(2):  # replaying the graph must give the same results
        for _, _, pos in items:
            if pos is not None:
                pos.fill_(-1)
        batch.run()
        _check(batch, items, want)
    batch.free()


def test_batch_against_the_oracle(torch):
    dfas, texts, items, want = _make(torch, n_items=16, seed=3, max_len=200_000)
    batch = pm.parem_batch_create(items)
    batch.run()
    for (dfa, view, pos), r, (ref, ref_pos, spec, text) in zip(items, batch.results(), want):
        o = oracle.scan(spec.table, spec.byte_to_symbol, spec.start, spec.accept, text)
        assert (r.final_state, r.match_count) == (o.final_state, o.match_count)
        if pos is not None:
            assert np.array_equal(pos[: r.n_written].cpu().numpy().astype(np.uint64), o.positions)
    batch.free()


def test_batch_autotuner_and_forced_segments(torch):
    dfas, texts, items, want = _make(torch, n_items=30, seed=5, max_len=4 << 20)
    batch = pm.parem_batch_create(items, pm.BatchOpts(autotune=1))
    batch.run()
    _check(batch, items, want)
    segs = batch.segments()
    assert all(s % 64 == 0 for s in segs)
    batch.free()
    batch = pm.parem_batch_create(items, pm.BatchOpts(segment_bytes=128))
    batch.run()
    _check(batch, items, want)
    batch.free()


def _expected_form(info, forced):
    """The speculation form a batch gives a DFA when `forced` is asked for: the forced form
    where it applies (grouped: candidate sets of at most 32 states; registers: at most 256;
    the state bitmap: DFAs of at most 16,384 states), else the default's."""
    m, n = info.max_candidates, info.compact_states
    if forced == pm.PAREM_BATCH_SPEC_GROUPED and m <= 32:
        return "grouped"
    if forced == pm.PAREM_BATCH_SPEC_WARP and m <= 256:
        return "warp"
    if forced == pm.PAREM_BATCH_SPEC_WARP_BITMAP and n <= 16384:
        return "warp_bitmap"
    return None


@pytest.mark.parametrize("warps", [16, 24])
@pytest.mark.parametrize("form", [pm.PAREM_BATCH_SPEC_GROUPED, pm.PAREM_BATCH_SPEC_WARP,
                                  pm.PAREM_BATCH_SPEC_WARP_BITMAP])
def test_batch_speculation_forms_and_block_shapes_against_the_oracle(torch, form, warps):
    """Each speculation form and block shape, forced on every DFA where it applies, gives
    every item the oracle's final state, count and positions; the batch reports the form,
    shape and segment size it used."""
    dfas, texts, items, want = _make(torch, n_items=16, seed=11, max_len=300_000)
    batch = pm.parem_batch_create(items, pm.BatchOpts(spec=form, warps_per_block=warps))
    batch.run()
    cfgs = batch.configs()
    segs = batch.segments()
    for (dfa, view, pos), r, (ref, ref_pos, spec, text), c, s in zip(items, batch.results(), want, cfgs, segs):
        o = oracle.scan(spec.table, spec.byte_to_symbol, spec.start, spec.accept, text)
        assert (r.final_state, r.match_count) == (o.final_state, o.match_count)
        if pos is not None:
            assert np.array_equal(pos[: r.n_written].cpu().numpy().astype(np.uint64), o.positions)
        assert c["warps_per_block"] == warps and c["segment_bytes"] == s
        exp = _expected_form(pm.parem_dfa_get_info(dfa), form)
        if exp is not None:
            assert c["spec"] == exp
        else:
            assert c["spec"] in ("grouped", "warp", "warp_bitmap")
    batch.free()


def test_batch_autotuner_reports_one_form_per_dfa(torch):
    """The autotuner's choice: one speculation form per DFA, one block shape for the batch,
    and results equal to the per-item scans."""
    dfas, texts, items, want = _make(torch, n_items=30, seed=9, max_len=4 << 20)
    batch = pm.parem_batch_create(items, pm.BatchOpts(autotune=1))
    batch.run()
    _check(batch, items, want)
    cfgs = batch.configs()
    assert len({c["warps_per_block"] for c in cfgs}) == 1 and cfgs[0]["warps_per_block"] in (16, 24)
    form_of = {}
    for (dfa, _, _), c in zip(items, cfgs):
        if c["segment_bytes"]:
            assert form_of.setdefault(id(dfa), c["spec"]) == c["spec"]
    batch.free()


def test_batch_autotuner_keeps_a_form_the_caller_fixed(torch):
    """With the form fixed by the caller, the autotuner only tunes row lengths and the block
    shape: every DFA where the form applies keeps it, and results equal the per-item scans."""
    dfas, texts, items, want = _make(torch, n_items=24, seed=13, max_len=4 << 20)
    batch = pm.parem_batch_create(items, pm.BatchOpts(autotune=1, spec=pm.PAREM_BATCH_SPEC_WARP_BITMAP))
    batch.run()
    _check(batch, items, want)
    for (dfa, _, _), c in zip(items, batch.configs()):
        if c["segment_bytes"] and _expected_form(pm.parem_dfa_get_info(dfa), pm.PAREM_BATCH_SPEC_WARP_BITMAP):
            assert c["spec"] == "warp_bitmap"
    batch.free()
