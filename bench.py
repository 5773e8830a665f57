#!/usr/bin/env python
"""Benchmark of the chunked speculative DFA scan on GB300 (one JSON line on rank 0).

Default workload (the sparse-DFA configuration): the Aho-Corasick DFA of 64 random
lowercase keywords (lengths 8-24, ~1,000 states, 27 symbols a-z + space) over a 4 GiB text
of Zipf(1.1)-distributed words with keywords planted at rate 1e-5.  One step = one
parem_match over the whole device-resident text: speculation, main run, look-back and the
emission of every match position (two kernels).  value = text bytes / time (GB/s, 1e9).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--config d2|d1|d3|d4|d5|d6]

Under torchrun every rank scans its own text (independent problems, weak scaling, no
data-path collective); the timed region is bracketed by barriers and the max over ranks is
taken.  The reference arm (--impl reference) times the CPU oracle, as it stands, on a
bounded sample of the same workload on this host.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "scanned GB/s on 1 GB300 (fraction of HBM peak); batched vs plain; p99 ms"
# the device code of the plain scan: DRAM counters taken on it stay valid while these are unchanged
KERNEL_SOURCES = ["paper_1412_1741_gb300/csrc/parem_scan.cuh", "paper_1412_1741_gb300/csrc/parem_internal.h",
                  "paper_1412_1741_gb300/csrc/parem_k_byte.cu", "paper_1412_1741_gb300/csrc/parem_k_class.cu",
                  "paper_1412_1741_gb300/csrc/parem_k_global.cu", "paper_1412_1741_gb300/csrc/parem_k_win.cu",
                  "paper_1412_1741_gb300/csrc/parem_k_pair.cu"]

CONFIGS = {
    "d2": dict(workload="sparse DFA: Aho-Corasick of 64 random keywords (len 8-24) over a-z+space, "
                        "4 GiB Zipf(1.1) words, keywords planted at 1e-5", n=4 << 30),
    "d1": dict(workload="smallest: KMP automaton of Sigma*GATTACA (8 states), 1 MiB uniform ACGT (seed 0)",
               n=1 << 20),
    "d3": dict(workload="dense DFA: random complete 256 states x 256 bytes, 10% accepting, 8 GiB uniform bytes",
               n=8 << 30),
    "d6": dict(workload="paper-shaped: automaton of Table I ('parallel', 9 states, 5 symbols), "
                        "2^30 uniform symbols", n=1 << 30),
    "d4": dict(workload="batched: 4,096 texts, lengths log-uniform 1 KiB-16 MiB (7.27 GB), each with one of "
                        "32 DFAs (states log-uniform 4-4096, alphabets 4/27/256, half keyword unions, half "
                        "random); one persistent launch in a CUDA graph, autotuned segment size per DFA; "
                        "counts and final states", n=0),
    "d5": dict(workload="serving: 128 DFAs (states log-uniform 4-8192, alphabets 4/27/256, half keyword unions, "
                        "half random), Poisson arrivals at 20,000 requests/s for 10 s, lengths log-uniform "
                        "256 B-64 MiB, each request a slice of a 9 GiB device text arena; continuous batching "
                        "server; counts and final states", n=0),
}


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def host_cpu() -> dict:
    """The host's CPU model and logical core count (for the CPU baselines)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        import platform

        model = platform.processor() or platform.machine()
    return {"model": model, "nproc": os.cpu_count()}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profiled_traffic(config, n, plan):
    """DRAM bytes (read + write) per launch of the pass-1 kernel, from the committed ncu
    summary of the same kernel sources and the same launch shape (warps per block, blocks),
    scaled from the captured text size to n bytes (a streaming kernel: the text is read once
    and the per-row records grow with it, so traffic grows in proportion to the text; the
    capture may use a smaller text with proportionally shorter rows).  None when the sources
    or the launch shape differ."""
    p = os.path.join(ROOT, "profiles", f"traffic_{config}.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("kernel_hash") != kernel_hash():
        return None
    if any(d.get(k) != plan.get(k) for k in ("warps_per_block", "blocks")) or not d.get("text_bytes"):
        return None
    return int(round(d["dram_bytes_per_launch"] * n / d["text_bytes"]))


# ---------------------------------------------------------------------------------------
# multi-rank timing: every rank scans its own data (weak scaling); the job's time is the
# slowest rank's, and the job's throughput counts the bytes of all ranks
# ---------------------------------------------------------------------------------------
def max_over_ranks(ms: float, dist, device) -> float:
    """The largest of the ranks' times (ms); the value itself on one rank (dist None)."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gbs(bytes_per_rank_step: int, world: int, steps: int, max_ms: float) -> float:
    """Whole-job throughput: the bytes every rank scanned in every step over the slowest
    rank's time (GB/s, 1e9)."""
    return bytes_per_rank_step * world * steps / (max_ms / 1e3) / 1e9


# ---------------------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------------------
def make_workload(config, device, seed_shift=0):
    import torch

    from paper_1412_1741_gb300 import workloads as wl

    n = CONFIGS[config]["n"]
    if config == "d2":
        spec = wl.keywords_ac_dfa()
        text = wl.zipf_words_text_device(n, device, seed=2 + seed_shift, keywords=spec.meta["keywords"])
    elif config == "d1":
        spec = wl.gattaca_dfa()
        text = torch.from_numpy(wl.uniform_text(n, 4, 0 + seed_shift)).to(device)
    elif config == "d3":
        spec = wl.dense_dfa()
        text = wl.uniform_text_device(n, 256, device, seed=5 + seed_shift)
    elif config == "d6":
        spec = wl.parallel_dfa()
        text = wl.uniform_text_device(n, 5, device, seed=11 + seed_shift)
    else:
        raise ValueError(config)
    return spec, text


def host_sample(config, nbytes):
    """Host text of the same workload for the CPU reference arm (numpy generators)."""
    from paper_1412_1741_gb300 import workloads as wl

    if config == "d2":
        spec = wl.keywords_ac_dfa()
        return spec, wl.zipf_words_text(nbytes, keywords=spec.meta["keywords"])
    if config == "d1":
        return wl.gattaca_dfa(), wl.uniform_text(nbytes, 4, 0)
    if config == "d3":
        return wl.dense_dfa(), wl.uniform_text(nbytes, 256, 5)
    return wl.parallel_dfa(), wl.uniform_text(nbytes, 5, 11)


# ---------------------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = sorted(sm)[len(sm) // 2:] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------------------
def run_reference(args, rank):
    """CPU oracle, as it stands, on a bounded sample of the workload (rank 0 only)."""
    if rank != 0:
        return
    from oracle import oracle

    oracle.build()
    sample = min(CONFIGS[args.config]["n"], args.ref_sample_mb << 20)
    spec, text = host_sample(args.config, sample)
    for _ in range(args.warmup):
        oracle.scan(spec.table, spec.byte_to_symbol, spec.start, spec.accept, text[: 1 << 20], want_positions=False)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.scan(spec.table, spec.byte_to_symbol, spec.start, spec.accept, text, want_positions=True)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = sample * args.steps / tot / 1e9
    desc = f"first {sample >> 20} MiB of the {args.config} workload per step, single-threaded C oracle"
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(tot / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": CONFIGS[args.config]["workload"], "sample_bytes": sample, "matches_in_sample": r.match_count},
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": desc,
                         "host": host_cpu()},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_and_parity(spec, text_dev, got, pos_dev):
    """The oracle over the WHOLE text (copied to the host): the time of its pass that writes
    the positions is the CPU baseline (one thread: the sequential run does not split), and
    its result is compared with the GPU's last timed call -- final state, acceptance, match
    count and every position written.  Returns (cpu_baseline, parity)."""
    import numpy as np

    from oracle import oracle

    oracle.build()
    n = int(text_dev.numel())
    host = np.ascontiguousarray(text_dev.cpu().numpy())
    times = []
    want = oracle.scan(spec.table, spec.byte_to_symbol, spec.start, spec.accept, host,
                       want_positions=pos_dev is not None, times=times)
    dt = times[-1]
    checks = {"final_state": int(got.final_state) == int(want.final_state),
              "accepted": bool(got.accepted) == bool(want.accepted),
              "match_count": int(got.match_count) == int(want.match_count)}
    if pos_dev is not None:
        k = int(got.n_written)
        g = pos_dev[:k].cpu().numpy().view(np.uint64)
        checks["positions"] = bool(k == min(int(pos_dev.numel()), want.match_count) and
                                   np.array_equal(g, want.positions[:k]))
    ok = all(checks.values())
    parity = {"ok": ok, "checked": "whole text" + (", every position" if pos_dev is not None else ", count only"),
              "text_bytes": n, "oracle_matches": int(want.match_count), "gpu_matches": int(got.match_count),
              "oracle_final_state": int(want.final_state), "gpu_final_state": int(got.final_state), **checks}
    cpu = {"value": round(n / dt / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
           "sample": f"the whole {n / (1 << 30):.2f} GiB text, one single-threaded pass of the C oracle writing "
                     f"its {want.match_count} positions ({dt:.1f} s; a counting pass before it sizes the buffer)"}
    return cpu, parity


def oracle_all_cores(jobs):
    """Run independent oracle scans on all host cores (ctypes releases the GIL, so threads run
    the C loops in parallel).  jobs: list of (spec, host_text, start).  Returns (results,
    seconds, threads)."""
    import concurrent.futures as cf

    from oracle import oracle

    oracle.build()
    if jobs:  # load the library once before the threads start
        oracle.scan(jobs[0][0].table, jobs[0][0].byte_to_symbol, jobs[0][2], jobs[0][0].accept, jobs[0][1][:1],
                    want_positions=False)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(lambda j: oracle.scan(j[0].table, j[0].byte_to_symbol, j[2], j[0].accept, j[1],
                                                want_positions=False), jobs))
    return res, time.perf_counter() - t0, threads


def host_link_gbs(host_pinned, dev_buf, piece=512 << 20):
    """Host-to-device copy rate of a pinned buffer (GB/s, 1e9), copied as the host-buffer
    entry point copies it: pieces of 512 MiB alternating over two streams.  This is what
    bounds the end-to-end path with host buffers."""
    import torch

    n = host_pinned.numel()
    cur = torch.cuda.current_stream()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]

    def once():
        for st in streams:
            st.wait_stream(cur)
        for k, off in enumerate(range(0, n, piece)):
            with torch.cuda.stream(streams[k & 1]):
                dev_buf[off:off + piece].copy_(host_pinned[off:off + piece], non_blocking=True)
        for st in streams:
            cur.wait_stream(st)

    once()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(cur)
    for _ in range(3):
        once()
    b.record(cur)
    torch.cuda.synchronize()
    return 3 * n / (a.elapsed_time(b) / 1e3) / 1e9


def setup_rank(local_rank, world):
    import torch

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    return dev, dist


def batch_measure(args, rank, world, dev, dist):
    """Batched configuration: one graph launch per step over all texts (count only) vs a loop
    of plain calls on the same texts; every item's result is compared with the oracle, run
    over all texts on all host cores (its time is the CPU baseline).  Returns the line."""
    import numpy as np
    import torch

    import paper_1412_1741_gb300 as pm
    from paper_1412_1741_gb300 import workloads as wl

    n_texts = args.batch_texts
    specs = wl.batch_dfas(32, seed=6)
    lengths = wl.batch_lengths(n_texts, seed=6 + rank)
    dfas = [pm.parem_load_dfa(s.table, s.byte_to_symbol, s.start, s.accept) for s in specs]
    # the texts in the batch: all, or (--batch-dfa) those of one DFA alone, generated alone
    keep = [i for i in range(n_texts) if args.batch_dfa < 0 or i % len(dfas) == args.batch_dfa]
    if args.batch_dfa >= 0:
        arena, offs = wl.batch_texts_device([specs[args.batch_dfa]], lengths[keep], dev, seed=6 + rank)
    else:
        arena, offs = wl.batch_texts_device(specs, lengths, dev, seed=6 + rank)
    ptr = arena.data_ptr()
    at = {i: int(offs[k if args.batch_dfa >= 0 else i]) for k, i in enumerate(keep)}  # text i's arena offset
    items = [(dfas[i % len(dfas)], ptr + at[i], int(lengths[i]), None, 0) for i in keep]
    total = int(sum(int(lengths[i]) for i in keep))
    t0 = time.perf_counter()
    batch = pm.parem_batch_create(items, pm.BatchOpts(autotune=0 if args.batch_no_autotune else 1))
    plan_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        batch.run()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for a, b in evs:
        a.record(stream)
        batch.run()
        b.record(stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
    step_ms = sorted(a.elapsed_time(b) for a, b in evs)
    res = batch.results()
    segs = batch.segments()
    cfgs = batch.configs()
    # what the autotuner chose for each DFA (its longest rows; shorter texts get one row)
    per_dfa = []
    for d in range(len(dfas)):
        mine = [c for k, c in enumerate(cfgs) if keep[k] % len(dfas) == d and c["segment_bytes"]]
        if not mine:
            continue
        info = pm.parem_dfa_get_info(dfas[d])
        per_dfa.append({"dfa": d, "states": info.compact_states, "max_candidates": info.max_candidates,
                        "segment_bytes": max(c["segment_bytes"] for c in mine), "spec": mine[0]["spec"],
                        "table": "smem" if mine[0]["smem_table"] else "l2"})
    tuned = {"warps_per_block": cfgs[0]["warps_per_block"], "per_dfa": per_dfa}
    # plain: one parem_match per text on the same stream (same texts)
    for i in range(min(64, len(items))):
        pm.parem_match(items[i][0], items[i][1], length=items[i][2])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = [pm.parem_match(it[0], it[1], length=it[2]) for it in items]
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    agree = all((a.final_state, a.match_count) == (b.final_state, b.match_count) for a, b in zip(res, plain))
    batch.free()
    line = None
    if rank == 0:
        # the oracle on every text, all host cores; parity of every item
        host = arena.cpu().numpy()
        jobs = [(specs[i % len(specs)], host[at[i]:at[i] + int(lengths[i])], specs[i % len(specs)].start)
                for i in keep]
        want, cpu_s, threads = oracle_all_cores(jobs)
        bad = [i for i, (g, w) in enumerate(zip(res, want))
               if (int(g.final_state), int(g.match_count)) != (int(w.final_state), int(w.match_count))]
        del host
        value = job_gbs(total, world, args.steps, total_ms)
        plain_gbs = total / plain_s / 1e9
        peak, peak_kind = measured_peaks()
        achieved = total / (step_ms[len(step_ms) // 2] / 1e3) / 1e9
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": CONFIGS["d4"]["workload"], "texts": len(keep), "only_dfa": args.batch_dfa if args.batch_dfa >= 0 else None,
                       "autotuned": not args.batch_no_autotune, "text_bytes": total, "dfas": len(dfas),
                       "positions": "count only", "plan_seconds_with_autotune": round(plan_s, 3),
                       "segment_bytes_median": int(np.median([x for x in segs if x] or [0])),
                       "l2": "inputs larger than L2 (7.27 GB)", "parallelism": f"replicas x{world}"},
            "p50_ms": round(step_ms[len(step_ms) // 2], 4),
            "p99_ms": round(step_ms[min(len(step_ms) - 1, int(0.99 * len(step_ms)))], 4),
            "batched_vs_plain": {"batched_gbs": round(value / world, 2), "plain_gbs": round(plain_gbs, 2),
                                 "speedup": round(value / world / plain_gbs, 2), "plain_calls": len(keep),
                                 "results_agree": agree},
            "autotuned": tuned,
            "parity": {"ok": not bad, "checked": f"all {len(keep)} items: final state and match count vs the oracle",
                       "mismatched_items": bad[:8]},
            "cpu_baseline": {"value": round(total / cpu_s / 1e9, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
                             "host": host_cpu(),
                             "sample": f"all {len(keep)} texts ({total / 1e9:.2f} GB), independent oracle scans on "
                                       f"{threads} host threads ({cpu_s:.1f} s)"},
            "roofline": {"bound": "hbm", "kernel": "whole batch graph (k_batch_scan + tiny kernel + copies)",
                         "achieved": round(achieved, 1), "peak": peak,
                         "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)", "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": None},
            "gpu_launches": args.steps * 2,
            "clocks": clk,
        }
    for d in dfas:
        d.free()
    del arena
    torch.cuda.empty_cache()
    return line


def serve_measure(args, rank, world, dev):
    """Serving configuration: open-loop replay of a Poisson trace through the request server
    (continuous batching), the same trace's head through the FIFO plain server, a saturation
    sweep over arrival rates, and the oracle (all host cores) on a bounded sample of the
    trace's requests, whose responses it checks.  Returns the line."""
    import numpy as np
    import torch

    import paper_1412_1741_gb300 as pm
    from paper_1412_1741_gb300 import workloads as wl

    specs = wl.serve_dfas(128, seed=7)
    dfas = [pm.parem_load_dfa(s.table, s.byte_to_symbol, s.start, s.accept) for s in specs]
    pools = wl.serve_pools_device(dev, pool_bytes=1536 << 20, seed=7 + rank)
    torch.cuda.synchronize()

    def trace(rate, dur, seed):
        arr, d, length = wl.serve_trace(len(specs), rate, dur, seed=seed)
        return pm.make_requests(d, wl.serve_slices(specs, pools, d, length, seed=seed), length, arrival_ns=arr)

    def summary(req, resp):
        lat = (resp["done_ns"] - resp["arrival_ns"]) / 1e6
        span = (resp["done_ns"].max() - resp["arrival_ns"].min()) / 1e9
        queue = (resp["launch_ns"] - resp["arrival_ns"]) / 1e6  # waiting for a batch and an arena
        run = (resp["done_ns"] - resp["launch_ns"]) / 1e6      # launch of its batch to its answer
        return {"requests": int(len(req)), "bytes": int(req["len"].sum()),
                "gbs": round(float(req["len"].sum()) / span / 1e9, 2), "span_s": round(span, 3),
                "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
                "p50_queue_ms": round(float(np.percentile(queue, 50)), 3),
                "p50_run_ms": round(float(np.percentile(run, 50)), 3),
                "errors": int((resp["status"] != 0).sum())}

    srv = pm.parem_server_create(dfas, pm.ServerOpts(arenas=args.arenas, arena_scratch_bytes=args.arena_mb << 20))
    for w in range(args.warmup):
        srv.replay(trace(20000, 0.2, 100 + w))
    k0 = srv.stats()["kernels"]
    clocks = ClockSampler(dev.index)
    clocks.start()
    duration = float(args.serve_seconds)
    req = trace(20000, duration, 7 + rank)
    resp = srv.replay(req)
    clk = clocks.stop()
    main = summary(req, resp)
    kernels = srv.stats()["kernels"] - k0
    st = srv.stats()
    # saturation sweep: achieved throughput and p99 as the offered load grows
    sweep = []
    for rate in (20000, 40000, 80000, 160000):
        r = trace(rate, 1.0, 500 + rate // 1000)
        x = summary(r, srv.replay(r))
        x["rate_per_s"] = rate
        x["offered_gbs"] = round(float(r["len"].sum()) / 1.0 / 1e9, 2)
        sweep.append(x)
    srv.free()
    # FIFO plain server on the head of the same trace (bounded: its backlog grows without limit
    # once the offered load exceeds what one request at a time can serve)
    head = req[req["arrival_ns"] < int(args.fifo_seconds * 1e9)]
    fifo = pm.parem_server_create(dfas, pm.ServerOpts(mode=pm.PAREM_SERVE_FIFO))
    fresp = fifo.replay(head)
    fifo.free()
    fsum = summary(head, fresp)
    agree = bool(np.array_equal(fresp["final_state"], resp["final_state"][: len(head)]) and
                 np.array_equal(fresp["match_count"], resp["match_count"][: len(head)]))
    best = max(sweep, key=lambda x: x["gbs"])
    line = None
    if rank == 0:
        # the oracle on the first requests of the trace, all host cores, against the responses
        keys = [(sp.meta["family"], sp.meta["alphabet"]) for sp in specs]
        host = {k: v.cpu().numpy() for k, v in pools.items()}
        base = {k: v.data_ptr() for k, v in pools.items()}
        budget, jobs = args.serve_oracle_gb * 1e9, []
        for i in range(len(req)):
            k = keys[int(req["dfa_index"][i])]
            o = int(req["text"][i]) - base[k]
            jobs.append((specs[int(req["dfa_index"][i])], host[k][o:o + int(req["len"][i])],
                         specs[int(req["dfa_index"][i])].start))
            budget -= int(req["len"][i])
            if budget <= 0:
                break
        want, cpu_s, threads = oracle_all_cores(jobs)
        nb = sum(int(j[1].size) for j in jobs)
        bad = [i for i, w in enumerate(want)
               if (int(resp["final_state"][i]), int(resp["match_count"][i]), int(resp["status"][i])) !=
               (int(w.final_state), int(w.match_count), 0)]
        del host
        line = {
            "metric": METRIC, "value": main["gbs"], "unit": "GB/s", "n_gpus": world, "steps": 1,
            "warmup": args.warmup, "ms_per_step": round(main["span_s"] * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": CONFIGS["d5"]["workload"], "dfas": len(dfas), "trace_seconds": duration,
                       "requests": main["requests"], "text_bytes": main["bytes"], "positions": "count only",
                       "l2": "inputs larger than L2 (9 GiB arena)", "parallelism": f"replicas x{world}",
                       "step": "one replay of the whole trace"},
            "p50_ms": main["p50_ms"], "p99_ms": main["p99_ms"],
            "serving": {"batched": main, "batches": st["batches"], "max_batch": st["max_batch"],
                        "arenas": args.arenas, "arena_scratch_mib": args.arena_mb or None,
                        "fifo_plain": dict(fsum, trace_seconds=args.fifo_seconds), "fifo_results_agree": agree,
                        "saturation_sweep": sweep, "max_sustained_gbs": best["gbs"]},
            "parity": {"ok": not bad, "checked": f"the first {len(jobs)} requests of the trace ({nb / 1e9:.1f} GB): "
                                                 f"final state, match count and status vs the oracle",
                       "mismatched_requests": bad[:8]},
            "cpu_baseline": {"value": round(nb / cpu_s / 1e9, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
                             "host": host_cpu(),
                             "sample": f"the first {len(jobs)} requests of the trace ({nb / 1e9:.1f} GB), independent "
                                       f"oracle scans on {threads} host threads ({cpu_s:.1f} s)"},
            "e2e": {"value": main["gbs"], "unit": "GB/s", "h2d_bytes_per_step": int(len(req)) * 56,
                    "d2h_bytes_per_step": int(len(req)) * 64,
                    "note": "texts live in the device arena by design; each request's descriptor goes to the "
                            "device and its result to the host; latency is arrival to result on the host"},
            "roofline": {"bound": "hbm", "kernel": "k_batch_scan (continuous batches)", "achieved": main["gbs"],
                         "peak": measured_peaks()[0], "unit": "GB/s",
                         "frac": round(main["gbs"] / measured_peaks()[0], 4), "traffic": None},
            "gpu_launches": int(kernels),
            "clocks": clk,
        }
    for d in dfas:
        d.free()
    del pools
    torch.cuda.empty_cache()
    return line


def run_batch(args, rank, world, local_rank):
    import __graft_entry__ as ge

    ge.build()
    dev, dist = setup_rank(local_rank, world)
    line = batch_measure(args, rank, world, dev, dist)
    if line is not None:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_serve(args, rank, world, local_rank):
    import __graft_entry__ as ge

    ge.build()
    dev, dist = setup_rank(local_rank, world)
    line = serve_measure(args, rank, world, dev)
    if line is not None:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_ours(args, rank, world, local_rank):
    import __graft_entry__ as ge

    ge.build()
    dev, dist = setup_rank(local_rank, world)
    line = scan_line(args, rank, world, dev, dist)
    # the other two parts of the metric on the same GPU: batched vs plain, and serving; then
    # the dense and the paper-shaped single-text configurations, so that one run measures and
    # checks them all
    if world == 1 and args.config == "d2" and not args.no_extras and not args.size_mb:
        b = batch_measure(args, rank, world, dev, None)
        line["batched_vs_plain"] = dict(b["batched_vs_plain"], texts=b["config"]["texts"],
                                        text_bytes=b["config"]["text_bytes"], dfas=b["config"]["dfas"],
                                        p50_ms=b["p50_ms"], plan_seconds_with_autotune=b["config"]["plan_seconds_with_autotune"],
                                        parity=b["parity"], cpu_baseline=b["cpu_baseline"], clocks=b["clocks"],
                                        gpu_launches=b["gpu_launches"], roofline_frac=b["roofline"]["frac"],
                                        autotuned=b["autotuned"])
        line["gpu_launches"] += b["gpu_launches"]
        v = serve_measure(args, rank, world, dev)
        line["serving"] = dict(v["serving"], p50_ms=v["p50_ms"], p99_ms=v["p99_ms"], gbs=v["value"],
                               parity=v["parity"], cpu_baseline=v["cpu_baseline"], clocks=v["clocks"],
                               gpu_launches=v["gpu_launches"])
        line["gpu_launches"] += v["gpu_launches"]
        line["other_configs"] = {}
        for cfg in ("d3", "d6"):
            sub = argparse.Namespace(**vars(args))
            sub.config = cfg
            sub.steps = min(args.steps, 10)
            sub.no_e2e = cfg == "d3"  # 8 GiB of pinned host text and 7 GB of positions: device leg only
            o = scan_line(sub, rank, world, dev, dist)
            line["other_configs"][cfg] = {
                "workload": o["config"]["workload"], "value": o["value"], "unit": o["unit"],
                "ms_per_step": o["ms_per_step"], "steps": o["steps"], "matches": o["config"]["matches"],
                "roofline": {k: o["roofline"][k] for k in ("achieved", "frac", "scan_ms_avg", "emit_ms_avg", "traffic")},
                "step_frac_text_plus_positions": round(
                    (o["config"]["text_bytes"] + 8 * o["config"]["matches"]) / (o["ms_per_step"] / 1e3) / 1e9
                    / o["roofline"]["peak"], 4),
                "parity": o.get("parity"), "cpu_baseline": o.get("cpu_baseline"), "e2e": o.get("e2e"),
                "clocks": o["clocks"], "gpu_launches": o["gpu_launches"]}
            line["gpu_launches"] += o["gpu_launches"]
    if rank == 0:
        print(json.dumps(line), flush=True)
        bad = [k for k in ("parity",) if k in line and not line[k]["ok"]]
        bad += [k for k in ("batched_vs_plain", "serving") if k in line and not line[k]["parity"]["ok"]]
        bad += [k for k, o in line.get("other_configs", {}).items() if o["parity"] and not o["parity"]["ok"]]
        if bad:
            print(f"PARITY FAILURE against the oracle in: {', '.join(bad)}", file=sys.stderr, flush=True)
            sys.exit(3)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def scan_line(args, rank, world, dev, dist):
    """One single-text configuration (args.config): the timed device-resident steps, the
    library's per-pass kernel times for the roofline, the host-buffer leg and the whole-text
    oracle check.  Returns the JSON line (rank 0; None elsewhere)."""
    import torch

    import paper_1412_1741_gb300 as pm

    spec, text = make_workload(args.config, dev, seed_shift=rank)
    n = int(text.numel())
    dfa = pm.parem_load_dfa(spec.table, spec.byte_to_symbol, spec.start, spec.accept)
    stream = torch.cuda.current_stream()
    # size the position buffer from a first scan
    first = pm.parem_match(dfa, text)
    cap = max(1, first.match_count) if not args.count_only else 0
    pos = torch.empty(cap, dtype=torch.int64, device=dev) if cap else None
    opts = pm.MatchOpts(segment_bytes=args.segment_bytes, enumerate_all=1 if args.enumerate else 0)
    for _ in range(args.warmup):
        pm.parem_match_ex(dfa, text, pos, opts)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    ev0.record(stream)
    for i in range(args.steps):
        step_ev[i][0].record(stream)
        r = pm.parem_match_ex(dfa, text, pos, opts)
        step_ev[i][1].record(stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    kernels = args.steps * pm.parem_last_stats()["kernels"]
    # the kernel breakdown for the roofline: the same calls again with the library's own
    # CUDA events around pass 1 and the emit pass (outside the timed region above)
    opts_timed = pm.MatchOpts(record_kernel_times=1, segment_bytes=args.segment_bytes,
                              enumerate_all=1 if args.enumerate else 0)
    scan_ms, emit_ms = [], []
    for _ in range(min(args.steps, 10)):
        pm.parem_match_ex(dfa, text, pos, opts_timed)
        st = pm.parem_last_stats()
        scan_ms.append(st["scan_ms"])
        emit_ms.append(st["emit_ms"])
    total_ms = ev0.elapsed_time(ev1)
    total_ms = max_over_ranks(total_ms, dist, dev)
    step_ms = sorted(a.elapsed_time(b) for a, b in step_ev)
    value = job_gbs(n, world, args.steps, total_ms)
    line = None
    if rank == 0:
        peak, peak_kind = measured_peaks()
        scan_avg = sum(scan_ms) / len(scan_ms)
        achieved = n / (scan_avg / 1e3) / 1e9
        st = pm.parem_last_stats()
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {
                "workload": CONFIGS[args.config]["workload"], "text_bytes": n, "dfa_states": spec.n_states,
                "matches": r.match_count, "positions": "all emitted" if cap else "count only",
                "candidates": "all live states (enumeration)" if args.enumerate else "img(class of the previous byte)",
                "l2": "inputs larger than L2 (text >> 126 MB), no flush needed" if n > (256 << 20) else
                      "input smaller than L2: resident between steps",
                "segment_bytes": st["segment_bytes"], "chunks": st["chunks"], "blocks": st["blocks"],
                "warps_per_block": st["warps_per_block"], "parallelism": f"replicas x{world}",
            },
            "p50_ms": round(step_ms[len(step_ms) // 2], 4),
            "p99_ms": round(step_ms[min(len(step_ms) - 1, int(0.99 * len(step_ms)))], 4),
            "roofline": {
                "bound": "hbm", "kernel": "k_spec_scan (pass 1)", "achieved": round(achieved, 1), "peak": peak,
                "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)", "unit": "GB/s",
                "frac": round(achieved / peak, 4), "frac_of_nominal_8000": round(achieved / 8000.0, 4),
                "algorithmic_bytes_per_launch": n, "scan_ms_avg": round(scan_avg, 4),
                "emit_ms_avg": round(sum(emit_ms) / len(emit_ms), 4),
                "traffic": profiled_traffic(args.config, n, st),
            },
            "speculation": {"lookups_per_byte": round(st["spec_lookups"] / max(n, 1), 6),
                            "spec_lookups": st["spec_lookups"], "main_run_bytes": n,
                            "note": "table lookups of candidate runs before they merged (device counter), per "
                                    "text byte; the resolved run adds one lookup per byte"},
            "gpu_launches": kernels,
            "clocks": clk,
        }
    # end to end through the public API with host buffers (pinned)
    if not args.no_e2e:
        host_text = torch.empty(n, dtype=torch.uint8, pin_memory=True)
        host_text.copy_(text)
        host_pos = torch.empty(max(cap, 1), dtype=torch.int64, pin_memory=True) if cap else None
        # warm-up (as many calls as the device leg): staging buffers, copy streams and events are
        # created once, and the plans settle while the DFA's hints (longest merge, match density)
        # are learned from the pieces' scans (a plan that grows its scratch allocates once)
        for _ in range(max(3, args.warmup)):
            pm.parem_match_host(dfa, host_text, host_pos)
        # as many steps as the device leg: single slow steps (the host link of a shared machine
        # varies; one step of 20 took 98 ms where the others took 20.6) weigh in the mean
        e2e_steps = max(3, args.steps)
        torch.cuda.synchronize()
        step_s = []
        for _ in range(e2e_steps):
            t0 = time.perf_counter()
            re2e = pm.parem_match_host(dfa, host_text, host_pos)
            step_s.append(time.perf_counter() - t0)
        link = host_link_gbs(host_text, text) if n >= (64 << 20) else None
        # the same number of plain pinned host-to-device copies of the text, each timed alone:
        # what the host path would take if scanning were free (its slow steps are the link's)
        copy_s = []
        for _ in range(e2e_steps):
            t0 = time.perf_counter()
            text.copy_(host_text, non_blocking=True)
            torch.cuda.synchronize()
            copy_s.append(time.perf_counter() - t0)
        if rank == 0:
            # the mean over the steps is the headline; the median and the measured host link
            # (pinned host-to-device copy of the same buffer) are reported beside it
            line["e2e"] = {"value": round(n * e2e_steps / sum(step_s) / 1e9, 2), "unit": "GB/s",
                           "h2d_bytes_per_step": n, "d2h_bytes_per_step": re2e.n_written * 8 + 24,
                           "steps": e2e_steps, "statistic": "mean over steps",
                           "median_value": round(n / sorted(step_s)[len(step_s) // 2] / 1e9, 2),
                           "step_ms": [round(x * 1e3, 2) for x in step_s],
                           "host_link_gbs": round(link, 2) if link else None,
                           "plain_copy_mean_gbs": round(n * e2e_steps / sum(copy_s) / 1e9, 2),
                           "plain_copy_step_ms": [round(x * 1e3, 2) for x in copy_s]}
        del host_text, host_pos
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"], line["parity"] = cpu_baseline_and_parity(spec, text, r, pos)
    del text, pos
    dfa.free()
    torch.cuda.empty_cache()
    return line


def run_enum_compare(args, rank, world, local_rank):
    """PaREM against the general enumeration approach (every live state a candidate of every
    chunk) on the paper's own automaton (Table I, 'parallel', 9 states) over uniform texts of
    2^26 .. 2^30 symbols, the lengths of the paper's experiments (Section IV, Fig. 6).  Both
    arms run the same kernels; one JSON line per length with both arms' times, speculation
    lookups per byte, the candidate-run counts of the worked example's argument (Section II-C)
    and parity of both arms with the oracle.  Rank 0 only."""
    import numpy as np
    import torch

    import __graft_entry__ as ge
    import paper_1412_1741_gb300 as pm
    from oracle import oracle
    from paper_1412_1741_gb300 import workloads as wl

    if rank != 0:
        return
    ge.build()
    oracle.build()
    dev, _ = setup_rank(local_rank, 1)
    spec = wl.parallel_dfa()
    info = pm.parem_prepare_info(spec.table, spec.byte_to_symbol, spec.start, spec.accept)
    # candidate runs per row start over the text's symbols: |img(a)| = distinct states reached
    # on a from any state (Algorithm 1's L; S is every state for this complete DFA)
    tab = np.asarray(spec.table)
    img = [len(set(int(x) for x in tab[:, a])) for a in range(tab.shape[1])]
    peak, peak_kind = measured_peaks()
    for k in range(args.enum_min_log2, args.enum_max_log2 + 1):
        n = 1 << k
        text = wl.uniform_text_device(n, 5, dev, seed=11)
        host = text.cpu().numpy()
        want = oracle.scan(spec.table, spec.byte_to_symbol, spec.start, spec.accept, host)
        arms = {}
        for name, enum in (("parem", 0), ("enumeration", 1)):
            dfa = pm.parem_load_dfa(spec.table, spec.byte_to_symbol, spec.start, spec.accept)
            pos = torch.full((max(1, want.match_count),), -1, dtype=torch.int64, device=dev)
            opts = pm.MatchOpts(enumerate_all=enum)
            timed = pm.MatchOpts(enumerate_all=enum, record_kernel_times=1)
            for _ in range(args.warmup):
                pm.parem_match_ex(dfa, text, pos, opts)
            torch.cuda.synchronize()
            stream = torch.cuda.current_stream()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(args.steps):
                r = pm.parem_match_ex(dfa, text, pos, opts)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / args.steps
            scan = []
            for _ in range(5):
                pm.parem_match_ex(dfa, text, pos, timed)
                scan.append(pm.parem_last_stats()["scan_ms"])
            st = pm.parem_last_stats()
            ok = (r.final_state, r.accepted, r.match_count) == (want.final_state, want.accepted, want.match_count) and \
                np.array_equal(pos[:want.match_count].cpu().numpy().view(np.uint64), want.positions)
            arms[name] = {"ms_per_step": round(ms, 4), "gbs": round(n / (ms / 1e3) / 1e9, 2),
                          "scan_ms": round(float(np.median(scan)), 4),
                          "spec_lookups_per_byte": round(st["spec_lookups"] / n, 6),
                          "rows": st["rows"], "chunks": st["chunks"], "segment_bytes": st["segment_bytes"],
                          "parity": bool(ok)}
            dfa.free()
        line = {
            "metric": "PaREM vs general enumeration: time ratio (enumeration / PaREM) on 1 GB300",
            "value": round(arms["enumeration"]["ms_per_step"] / arms["parem"]["ms_per_step"], 3), "unit": "x",
            "higher_is_better": True, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "dtype": "u8", "data": "synthetic",
            "config": {"workload": "Table I automaton ('parallel', 9 states, 5 symbols), uniform i.i.d. text over "
                                   "{p,a,r,e,l} (the paper's experiment lengths)", "text_bytes": n, "log2_n": k,
                       "matches": want.match_count},
            "parem": arms["parem"], "enumeration": arms["enumeration"],
            "candidate_runs_per_row": {"parem_mean": round(float(np.mean(img)), 3), "parem_max": int(max(img)),
                                       "parem_per_symbol": dict(zip("parel", img)),
                                       "enumeration": int(tab.shape[0]),
                                       "note": "candidates per row start over the text's symbols: |img(a)| for "
                                               "PaREM (Algorithm 1's R = S n L), every state for enumeration; "
                                               "a row that meets a one-candidate symbol early needs no speculation"},
            "parity": arms["parem"]["parity"] and arms["enumeration"]["parity"],
            "paper_context": "the paper reports 2.3x at 48 threads on 1.07e9 symbols and 1.04x at 6 threads on 6.69e7 "
                             "(Section IV-A); other hardware, context only",
            "peak_gbs": peak,
        }
        print(json.dumps(line), flush=True)
        del text, host


# ---------------------------------------------------------------------------------------
# ncu summaries for profiles/ (read back from reports; no GPU needed)
# ---------------------------------------------------------------------------------------
NCU_METRICS = [
    ("gpu__time_duration.sum", "duration"), ("dram__bytes_read.sum", "DRAM read"),
    ("dram__bytes_write.sum", "DRAM write"), ("gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed", "DRAM throughput %"),
    ("sm__warps_active.avg.pct_of_peak_sustained_active", "warps active %"),
    ("smsp__issue_active.avg.pct_of_peak_sustained_active", "issue active %"),
    ("l1tex__throughput.avg.pct_of_peak_sustained_active", "L1/shared throughput %"),
    ("l1tex__data_pipe_lsu_wavefronts_mem_shared_op_ld.sum", "shared-load wavefronts"),
    ("l1tex__data_bank_conflicts_pipe_lsu_mem_shared_op_ld.sum", "shared-load bank conflicts"),
    ("smsp__sass_inst_executed_op_shared_ld.sum", "shared-load instructions"),
    ("sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_active", "tensor pipe %"),
    ("launch__registers_per_thread", "registers/thread"), ("launch__grid_size", "grid"),
    ("launch__block_size", "block"), ("launch__shared_mem_per_block_dynamic", "dynamic smem/block"),
]


def _ncu_raw(rep):
    import csv
    import io
    import subprocess

    out = subprocess.run(["ncu", "-i", rep, "--page", "raw", "--csv"], capture_output=True, text=True, check=True).stdout
    rows = list(csv.reader(io.StringIO(out)))
    return rows[0], rows[1], rows[2:]


def summarize_ncu(args):
    """Write profiles/<kernel>_<config>.md from a --set full report and, for the pass-1 kernel,
    profiles/traffic_<config>.json (DRAM bytes of the captured launch, its text size and plan)."""
    hdr, units, rows = _ncu_raw(args.ncu_report)
    col = {h: i for i, h in enumerate(hdr)}
    name = rows[0][col["Kernel Name"]]
    base = name.split("<")[0].split("(")[0].split("::")[-1].split()[-1]
    lines = [f"# {base} on {args.config} ({args.ncu_note})", "", "Command:", "", "```", args.ncu_command, "```", "",
             f"Kernel: `{name[:160]}`", "", "| metric | value | unit |", "|---|---|---|"]
    v = rows[0]
    for m, label in NCU_METRICS:
        if m in col:
            lines.append(f"| {label} (`{m}`) | {v[col[m]]} | {units[col[m]]} |")
    stalls = [(h[len("smsp__pcsamp_warps_issue_stalled_"):], float(v[i] or 0)) for h, i in col.items()
              if h.startswith("smsp__pcsamp_warps_issue_stalled_") and not h.endswith("not_issued")]
    tot = sum(x for _, x in stalls) or 1.0
    top = sorted(stalls, key=lambda x: -x[1])[:6]
    lines += ["", "Warp stall samples (top): " + ", ".join(f"{k} {100 * x / tot:.1f}%" for k, x in top)]
    os.makedirs(os.path.join(ROOT, "profiles"), exist_ok=True)
    path = os.path.join(ROOT, "profiles", f"{base}_{args.config}.md")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", path)
    if base == "k_spec_scan":
        def num(m):
            scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}.get(units[col[m]], 1)
            return float(v[col[m]].replace(",", "")) * scale
        d = {"kernel_hash": kernel_hash(), "config": args.config, "text_bytes": (args.size_mb << 20) if args.size_mb else CONFIGS[args.config]["n"],
             "segment_bytes": args.segment_bytes, "warps_per_block": int(num("launch__block_size")) // 32,
             "blocks": int(num("launch__grid_size")),
             "dram_bytes_per_launch": int(num("dram__bytes_read.sum") + num("dram__bytes_write.sum")),
             "source": os.path.basename(path)}
        tp = os.path.join(ROOT, "profiles", f"traffic_{args.config}.json")
        with open(tp, "w") as f:
            json.dump(d, f, indent=1)
        print("wrote", tp)


def summarize_launches(args):
    """Write profiles/launches_<config>.md from an ncu --csv launch list (gpu__time_duration.sum)."""
    import csv

    with open(args.ncu_launches) as f:
        text = [ln for ln in f if not ln.startswith("==")]
    rows = list(csv.DictReader(text))
    per = {}
    for r in rows:
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        full = r["Kernel Name"]
        if "parem::" in full:
            k = full.split("parem::", 1)[1].split("(")[0]
        else:
            k = "(input generation and other PyTorch kernels)"
        scale = {"ns": 1e-6, "us": 1e-3, "usecond": 1e-3, "nsecond": 1e-6, "ms": 1.0, "msecond": 1.0}[r["Metric Unit"]]
        t = float(r["Metric Value"].replace(",", "")) * scale
        n, tot = per.get(k, (0, 0.0))
        per[k] = (n + 1, tot + t)
    total = sum(t for _, t in per.values()) or 1.0
    ours = sum(t for k, (_, t) in per.items() if not k.startswith("(")) or 1.0
    lines = [f"# Launch list, {args.config} ({args.ncu_note})", "", "Command:", "", "```", args.ncu_command, "```", "",
             "Per-launch times are cold-cache and serialised (ncu); the shares are what compare with the bench.",
             "Share: of all captured kernel time; share of ours: of the library's kernels only.", "",
             "| kernel | launches | total ms | share | share of ours |", "|---|---|---|---|---|"]
    for k, (n, t) in sorted(per.items(), key=lambda x: -x[1][1]):
        mine = "" if k.startswith("(") else f"{100 * t / ours:.1f}%"
        lines.append(f"| {k} | {n} | {t:.3f} | {100 * t / total:.1f}% | {mine} |")
    path = os.path.join(ROOT, "profiles", f"launches_{args.config}.md")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", path)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="d2", choices=sorted(CONFIGS))
    ap.add_argument("--count-only", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ref-sample-mb", type=int, default=256)
    ap.add_argument("--size-mb", type=int, default=0, help="override the text size (profiling captures)")
    ap.add_argument("--segment-bytes", type=int, default=0,
                    help="fix the row length (profiling captures of a smaller text with the full-size plan)")
    ap.add_argument("--batch-texts", type=int, default=4096, help="texts of the batched configuration")
    ap.add_argument("--batch-dfa", type=int, default=-1,
                    help="batched configuration: only the texts of this DFA (0-31), alone in the batch")
    ap.add_argument("--batch-no-autotune", action="store_true",
                    help="batched configuration: the planner's default plan instead of the autotuner's")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="trace length of the serving configuration")
    ap.add_argument("--fifo-seconds", type=float, default=0.25, help="trace head replayed through the FIFO server")
    ap.add_argument("--arenas", type=int, default=256, help="batches in flight in the serving configuration")
    ap.add_argument("--arena-mb", type=int, default=0, help="device scratch per server arena in MiB (0: the library's)")
    ap.add_argument("--serve-oracle-gb", type=float, default=20.0,
                    help="bytes of the serving trace's first requests the oracle checks (GB)")
    ap.add_argument("--enumerate", action="store_true",
                    help="candidate set = every live state (the General Enumeration baseline)")
    ap.add_argument("--no-extras", action="store_true",
                    help="default line without its batched and serving parts")
    ap.add_argument("--enum-compare", action="store_true",
                    help="PaREM against general enumeration on the Table I automaton, one line per length")
    ap.add_argument("--enum-min-log2", type=int, default=26)
    ap.add_argument("--enum-max-log2", type=int, default=30)
    ap.add_argument("--ncu-report", default="", help="summarise this --set full report into profiles/")
    ap.add_argument("--ncu-launches", default="", help="summarise this ncu --csv launch list into profiles/")
    ap.add_argument("--ncu-command", default="", help="the command that made the report (recorded)")
    ap.add_argument("--ncu-note", default="", help="what the capture covers (recorded)")
    args = ap.parse_args()
    if args.ncu_report:
        summarize_ncu(args)
        return
    if args.ncu_launches:
        summarize_launches(args)
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.warmup < 3:
        args.warmup = 3
    if args.size_mb:
        CONFIGS[args.config]["n"] = args.size_mb << 20
        CONFIGS[args.config]["workload"] += f" (resized to {args.size_mb} MiB)"
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.enum_compare:
        run_enum_compare(args, rank, world, local_rank)
        return
    if args.config == "d4":
        run_batch(args, rank, world, local_rank)
        return
    if args.config == "d5":
        run_serve(args, rank, world, local_rank)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
