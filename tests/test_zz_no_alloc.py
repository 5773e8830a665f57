"""parem_match_noalloc: the scan for callers that cannot allocate device memory.

Some callers cannot let a library call cudaMalloc: their device memory is handed to their
own pool allocator at start-up, or allocation (and the synchronisation it may imply) is not
allowed on their path.  parem_match_noalloc runs the same kernels as parem_match with all
scratch in a fixed device array inside the library.  These checks compare it with
parem_match through the C ABI and with the CPU oracle, bit for bit, on two calls in a row
(the array keeps the last call's contents, so the second call checks that what must start at
zero is cleared) -- including automata whose rows resolve through slot maps and a dense DFA
whose positions go through the streaming emit pass -- and check the clear error for a request
that needs more scratch than the array holds.

The file is named so that pytest collects it last.
"""
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


def _cases():
    g = wl.gattaca_dfa()
    a = wl.keywords_ac_dfa()
    # permutation automata: their candidates never merge, so every row goes through a slot map
    parity = wl.DfaSpec(np.array([[1, 0], [0, 1]], np.uint32), 0, np.array([1, 0], np.uint8), None, "parity")
    mod3 = wl.DfaSpec(np.array([[(2 * q + b) % 3 for b in range(2)] for q in range(3)], np.uint32), 0,
                      np.array([1, 0, 0], np.uint8), None, "mod3")
    dense = wl.dense_dfa()  # 10 % of the bytes end a match: the streaming emit pass once learned
    return [
        (g, wl.uniform_text(1 << 20, 4, seed=0), 0),
        (g, wl.uniform_text(300_001, 5, seed=1), 3),  # bytes outside the alphabet, unaligned
        (a, wl.zipf_words_text(8 << 20, plant_rate=1e-4, keywords=a.meta["keywords"]), 7),
        (parity, wl.uniform_text((1 << 20) + 5, 2, seed=2), 1),
        (mod3, wl.uniform_text(600_007, 2, seed=3), 9),
        (dense, wl.uniform_text((4 << 20) + 3, 256, seed=5), 5),
    ]


def test_noalloc_matches_parem_match_and_the_oracle_on_two_calls_in_a_row(torch):
    for spec, text, offset in _cases():
        want = oracle.scan(spec.table, spec.byte_to_symbol, spec.start, spec.accept, text)
        dfa = pm.parem_load_dfa(spec.table, spec.byte_to_symbol, spec.start, spec.accept)
        buf = torch.zeros(text.size + offset + 16, dtype=torch.uint8, device="cuda")
        view = buf[offset:offset + text.size]
        view.copy_(torch.from_numpy(np.array(text)))
        # a count-only scan first: the DFA learns its match density, so that a dense DFA's
        # scans with positions below take the streaming emit pass in both entry points
        assert pm.parem_match(dfa, view).match_count == want.match_count
        cap = max(1, want.match_count)
        ref_pos = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
        ref = pm.parem_match(dfa, view, ref_pos)
        assert (ref.final_state, ref.accepted, ref.match_count) == (want.final_state, want.accepted, want.match_count)
        for _ in range(2):
            pos = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
            got = pm.parem_match_noalloc(dfa, view, pos)
            torch.cuda.synchronize()
            assert (got.final_state, got.accepted, got.match_count, got.n_written) == \
                   (ref.final_state, ref.accepted, ref.match_count, ref.n_written), spec.name
            assert torch.equal(pos, ref_pos), spec.name
            assert np.array_equal(pos[:want.match_count].cpu().numpy().view(np.uint64), want.positions), spec.name
            cnt = pm.parem_match_noalloc(dfa, view)  # count only
            assert (cnt.final_state, cnt.match_count) == (want.final_state, want.match_count), spec.name
        dfa.free()


def test_noalloc_rejects_requests_beyond_the_fixed_area(torch):
    # with positions requested, every row of the scan keeps a record and recorded positions
    # (112 bytes): a 256 MiB text has ~300k rows of under 1 KiB for the 8-state GATTACA DFA,
    # far more than the 16 MiB area holds
    spec = wl.gattaca_dfa()
    dfa = pm.parem_load_dfa(spec.table, spec.byte_to_symbol, spec.start, spec.accept)
    text = torch.zeros(256 << 20, dtype=torch.uint8, device="cuda")
    pos = torch.full((16,), -1, dtype=torch.int64, device="cuda")
    with pytest.raises(pm.ParemError) as e:
        pm.parem_match_noalloc(dfa, text, pos)
    assert e.value.status == pm.PAREM_ERR_TOO_LARGE
    assert "fixed area" in pm.parem_strerror(pm.PAREM_ERR_TOO_LARGE)
    assert bool((pos == -1).all())  # nothing written
    # the same text without positions fits
    got = pm.parem_match_noalloc(dfa, text)
    assert (got.final_state, got.match_count) == (0, 0)
    dfa.free()
