"""Request server (parem_server_*): every response equals parem_match on that request alone
(bit-exact final state, acceptance, count and positions), whether the request shares a batch
with others or not, in continuous-batching and FIFO modes, through submit/poll and through an
open-loop trace replay; memory admission splits batches that do not fit an arena and answers
TOO_LARGE for a request that cannot fit alone."""
import time

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


@pytest.fixture(scope="module")
def setup(torch):
    specs = wl.serve_dfas(16, seed=11, max_states=3000) + [wl.gattaca_dfa(), wl.keywords_ac_dfa()]
    specs[-2].meta.update(family="random", alphabet=4)
    specs[-1].meta.update(family="keywords", alphabet=27)
    dfas = [pm.parem_load_dfa(s.table, s.byte_to_symbol, s.start, s.accept) for s in specs]
    pools = wl.serve_pools_device(torch.device("cuda"), pool_bytes=8 << 20, seed=11)
    yield specs, dfas, pools
    for d in dfas:
        d.free()


def _requests(torch, specs, pools, n, seed, max_len=2 << 20, positions_every=2):
    rng = np.random.default_rng(seed)
    dfa = rng.integers(0, len(specs), size=n).astype(np.uint32)
    length = np.exp(rng.uniform(np.log(64), np.log(max_len), size=n)).astype(np.int64)
    length[:6] = [0, 1, 15, 63, 64, 65]
    addr = wl.serve_slices(specs, pools, dfa, length, seed=seed)
    req = pm.make_requests(dfa, addr, length)
    bufs = []
    for i in range(n):
        if i % positions_every == 0 and length[i] > 0:
            cap = int(length[i]) // 4 + 8
            b = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
            req["positions"][i] = b.data_ptr()
            req["capacity"][i] = cap
            bufs.append(b)
        else:
            bufs.append(None)
    return req, bufs


def _view(pools, specs, r, torch):
    """The request's text as a tensor view of its pool."""
    spec = specs[int(r["dfa_index"])]
    pool = pools[(spec.meta["family"], spec.meta["alphabet"])]
    off = int(r["text"]) - pool.data_ptr()
    return pool[off: off + int(r["len"])]


def _check(torch, specs, dfas, pools, req, bufs, resp):
    assert len(resp) == len(req)
    by_tag = {int(x["tag"]): x for x in resp}
    for i, r in enumerate(req):
        x = by_tag[int(r["tag"])]
        view = _view(pools, specs, r, torch)
        pos = None if bufs[i] is None else torch.full_like(bufs[i], -1)
        ref = pm.parem_match(dfas[int(r["dfa_index"])], view, pos, length=int(r["len"]))
        assert int(x["status"]) in (0, pm.PAREM_ERR_CAPACITY)
        assert (int(x["final_state"]), bool(x["accepted"]), int(x["match_count"])) == \
            (ref.final_state, ref.accepted, ref.match_count), i
        if bufs[i] is not None:
            assert int(x["n_written"]) == ref.n_written
            k = ref.n_written
            assert bool((bufs[i][:k] == pos[:k]).all()), i
        else:
            assert int(x["n_written"]) == 0
        assert x["done_ns"] >= x["launch_ns"] >= x["arrival_ns"] > 0


@pytest.mark.parametrize("mode", [pm.PAREM_SERVE_BATCH, pm.PAREM_SERVE_FIFO])
def test_submit_and_poll_equal_per_request_scans(torch, setup, mode):
    specs, dfas, pools = setup
    req, bufs = _requests(torch, specs, pools, 120, seed=1)
    srv = pm.parem_server_create(dfas, pm.ServerOpts(mode=mode))
    srv.submit(req[:60])
    srv.submit(req[60:])
    got, n, deadline = [], 0, time.time() + 300
    while n < len(req):
        assert time.time() < deadline, "server did not answer every request"
        g = srv.poll(4096, wait_s=1.0)
        got.append(g)
        n += len(g)
    resp = np.concatenate(got)
    st = srv.stats()
    assert st["submitted"] == st["answered"] == len(req)
    if mode == pm.PAREM_SERVE_BATCH:
        assert st["batches"] < len(req)  # requests shared launches
    srv.free()
    _check(torch, specs, dfas, pools, req, bufs, resp)


def test_replay_of_a_poisson_trace(torch, setup):
    specs, dfas, pools = setup
    arrival, dfa, length = wl.serve_trace(len(specs), rate_per_s=20000, duration_s=0.02, lo=64, hi=1 << 20, seed=3)
    addr = wl.serve_slices(specs, pools, dfa, length, seed=3)
    req = pm.make_requests(dfa, addr, length, arrival_ns=arrival)
    srv = pm.parem_server_create(dfas)
    resp = srv.replay(req)
    srv.free()
    assert np.array_equal(resp["tag"], np.arange(len(req)))
    lat = resp["done_ns"] - resp["arrival_ns"]
    assert (lat > 0).all()
    # arrival stamps are the trace's times from one origin
    assert np.array_equal(resp["arrival_ns"] - resp["arrival_ns"][0], arrival - arrival[0])
    _check(torch, specs, dfas, pools, req, [None] * len(req), resp)


def test_requests_against_the_oracle(torch, setup):
    specs, dfas, pools = setup
    req, bufs = _requests(torch, specs, pools, 24, seed=5, max_len=100_000, positions_every=1)
    srv = pm.parem_server_create(dfas)
    resp = srv.replay(req)  # arrival offsets 0: all at once
    srv.free()
    for i, r in enumerate(req):
        spec = specs[int(r["dfa_index"])]
        text = _view(pools, specs, r, torch).cpu().numpy()
        o = oracle.scan(spec.table, spec.byte_to_symbol, spec.start, spec.accept, text)
        assert (int(resp[i]["final_state"]), int(resp[i]["match_count"])) == (o.final_state, o.match_count)
        if bufs[i] is not None:
            k = int(resp[i]["n_written"])
            assert np.array_equal(bufs[i][:k].cpu().numpy().astype(np.uint64), o.positions[:k])


def test_memory_admission_splits_batches_and_rejects_oversized_requests(torch, setup):
    specs, dfas, pools = setup
    req, bufs = _requests(torch, specs, pools, 40, seed=7, max_len=64 << 10, positions_every=1)
    # 16 KiB arenas: with positions every row keeps a 112-byte record, so the 40 requests
    # (a few hundred rows) cannot share one launch
    srv = pm.parem_server_create(dfas, pm.ServerOpts(arena_scratch_bytes=16 << 10, max_items=64))
    resp = srv.replay(req)
    st = srv.stats()
    srv.free()
    assert st["batches"] > 1
    ok = resp["status"] != pm.PAREM_ERR_TOO_LARGE
    assert ok[:6].all()
    for i in np.nonzero(ok)[0]:
        r = req[i]
        view = _view(pools, specs, r, torch)
        pos = None if bufs[i] is None else torch.full_like(bufs[i], -1)
        ref = pm.parem_match(dfas[int(r["dfa_index"])], view, pos, length=int(r["len"]))
        assert (int(resp[i]["final_state"]), int(resp[i]["match_count"])) == (ref.final_state, ref.match_count)
    # a request that cannot fit an empty arena is answered, not dropped
    big = pm.make_requests(np.array([len(specs) - 1], np.uint32), np.array([pools[("keywords", 27)].data_ptr()], np.uint64),
                           np.array([8 << 20]))
    cap = 1 << 20
    b = torch.empty(cap, dtype=torch.int64, device="cuda")
    big["positions"] = b.data_ptr()
    big["capacity"] = cap
    srv = pm.parem_server_create(dfas, pm.ServerOpts(arena_scratch_bytes=64 << 10))
    out = srv.replay(big)
    srv.free()
    assert int(out[0]["status"]) == pm.PAREM_ERR_TOO_LARGE


def test_invalid_requests_are_rejected(torch, setup):
    specs, dfas, pools = setup
    srv = pm.parem_server_create(dfas)
    bad = pm.make_requests(np.array([len(dfas)], np.uint32), np.array([pools[("random", 4)].data_ptr()], np.uint64),
                           np.array([100]))
    with pytest.raises(pm.ParemError):
        srv.submit(bad)
    null_text = pm.make_requests(np.array([0], np.uint32), np.array([0], np.uint64), np.array([100]))
    with pytest.raises(pm.ParemError):
        srv.submit(null_text)
    assert srv.stats()["submitted"] == 0
    srv.free()


def test_batches_overlap_on_the_device_and_each_result_equals_the_oracle(torch, setup):
    # Continuous batching: a long request on the slowest random DFA occupies one arena; the
    # short requests that arrive while it runs are admitted into later batches on other arenas
    # and launched before the long one is done (their work overlaps on the device).  Every
    # result, in the mix, equals the oracle's run of that request alone.
    specs, dfas, pools = setup
    slow = max((i for i, s in enumerate(specs) if s.meta["family"] == "random"), key=lambda i: specs[i].n_states)
    big = wl.uniform_text_device(1 << 30, specs[slow].meta["alphabet"], torch.device("cuda"), seed=21)
    n_small = 48
    arrival = np.concatenate([[0], 2_000_000 + 250_000 * np.arange(n_small)]).astype(np.int64)
    rng = np.random.default_rng(9)
    dfa = np.concatenate([[slow], rng.integers(0, len(specs), size=n_small)]).astype(np.uint32)
    length = np.concatenate([[big.numel()], rng.integers(1 << 10, 1 << 20, size=n_small)]).astype(np.int64)
    addr = np.concatenate([[big.data_ptr()], wl.serve_slices(specs, pools, dfa[1:], length[1:], seed=9)])
    addr = addr.astype(np.uint64)
    req = pm.make_requests(dfa, addr, length, arrival_ns=arrival)
    srv = pm.parem_server_create(dfas)
    resp = srv.replay(req)
    st = srv.stats()
    srv.free()
    assert st["batches"] >= 2
    launch0, done0 = int(resp["launch_ns"][0]), int(resp["done_ns"][0])
    later = resp["launch_ns"][1:]
    overlapped = np.nonzero((later > launch0) & (later < done0))[0] + 1
    assert overlapped.size > 0, "no batch was launched while the long request's batch was running"
    assert (resp["status"] == 0).all()
    for i in range(len(req)):
        spec = specs[int(dfa[i])]
        text = big.cpu().numpy() if i == 0 else _view(pools, specs, req[i], torch).cpu().numpy()
        o = oracle.scan(spec.table, spec.byte_to_symbol, spec.start, spec.accept, text, want_positions=False)
        assert (int(resp["final_state"][i]), bool(resp["accepted"][i]), int(resp["match_count"][i])) == \
            (o.final_state, o.accepted, o.match_count), i
