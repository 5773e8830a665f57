"""Python binding of libparem (include/parem.h): argument marshalling only.

Every step of the scan runs in the CUDA library; there is no Python or CPU implementation
of the matcher in this package, and every call raises if libparem.so cannot be loaded.

    import torch, paper_1412_1741_gb300 as pm
    dfa = pm.parem_load_dfa(table, byte_to_symbol, start, accept)   # numpy inputs
    text = torch.tensor(..., dtype=torch.uint8, device="cuda")
    pos = torch.empty(cap, dtype=torch.int64, device="cuda")
    r = pm.parem_match(dfa, text, pos)        # r.final_state, r.match_count, r.n_written

Functions keep the C names.  Text and position buffers are PyTorch CUDA tensors (or raw
device pointers given as ints with an explicit length); the stream defaults to PyTorch's
current stream.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

__all__ = [
    "PAREM_NONE", "PAREM_NONE16", "ParemError", "MatchResult", "DfaInfo", "Dfa", "MatchOpts",
    "load_library", "parem_load_dfa", "parem_prepare_info", "parem_dfa_get_info", "parem_free_dfa", "parem_pair_preview",
    "parem_match", "parem_match_ex", "parem_match_host", "parem_release_scratch", "parem_strerror",
    "parem_version", "parem_last_stats", "parem_match_noalloc", "Stats", "EXPORTED_SYMBOLS",
    "PAREM_ERR_TOO_LARGE", "PAREM_NOALLOC_SCRATCH_BYTES", "parem_batch_create", "Batch", "BatchOpts",
    "parem_server_create", "Server", "ServerOpts", "make_requests", "parem_clock_ns", "REQUEST_DTYPE",
    "RESPONSE_DTYPE", "PAREM_SERVE_BATCH", "PAREM_SERVE_FIFO", "PAREM_REGEX_ANCHORED", "RegexDfa",
    "parem_regex_compile", "parem_load_regex",
]

PAREM_NONE = 0xFFFFFFFF
PAREM_NONE16 = 0xFFFF
PAREM_PAIR_AUTO, PAREM_PAIR_LEARN, PAREM_PAIR_OFF = 0, 1, 2
PAREM_OK = 0
PAREM_ERR_CAPACITY = -3
PAREM_ERR_TOO_LARGE = -8
PAREM_NOALLOC_SCRATCH_BYTES = 16 << 20

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

# Every symbol declared in include/parem.h.
EXPORTED_SYMBOLS = [
    "parem_load_dfa", "parem_prepare_info", "parem_dfa_get_info", "parem_free_dfa", "parem_pair_preview", "parem_match",
    "parem_match_ex", "parem_match_host", "parem_release_scratch", "parem_strerror", "parem_version",
    "parem_last_stats", "parem_match_noalloc", "parem_batch_create", "parem_batch_run", "parem_batch_results",
    "parem_batch_item_segment", "parem_batch_item_config", "parem_batch_stats", "parem_batch_free", "parem_server_create", "parem_server_submit",
    "parem_server_poll", "parem_server_drain", "parem_server_replay", "parem_server_get_stats",
    "parem_server_free", "parem_clock_ns", "parem_regex_compile", "parem_regex_info", "parem_regex_export",
    "parem_regex_load", "parem_regex_free",
]


class ParemError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        super().__init__(f"{where}: {parem_strerror(status)} ({status})")


class _Result(ctypes.Structure):
    _fields_ = [("final_state", ctypes.c_uint32), ("accepted", ctypes.c_uint8),
                ("reserved", ctypes.c_uint8 * 3), ("match_count", ctypes.c_uint64),
                ("n_written", ctypes.c_uint64)]


class _Info(ctypes.Structure):
    _fields_ = [("n_states", ctypes.c_uint32), ("n_symbols", ctypes.c_uint32),
                ("compact_states", ctypes.c_uint32), ("n_classes", ctypes.c_uint32),
                ("has_dead", ctypes.c_uint32), ("entry_bytes", ctypes.c_uint32),
                ("layout", ctypes.c_uint32), ("table_bytes", ctypes.c_uint32),
                ("max_candidates", ctypes.c_uint32), ("sync_estimate", ctypes.c_uint32),
                ("mean_candidates", ctypes.c_double), ("pair_hot_states", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class MatchOpts(ctypes.Structure):
    _fields_ = [("start_state", ctypes.c_uint32), ("enumerate_all", ctypes.c_uint32),
                ("segment_bytes", ctypes.c_uint64), ("warps_per_block", ctypes.c_uint32),
                ("spec_cap_bytes", ctypes.c_uint32), ("wait_budget_cycles", ctypes.c_uint64),
                ("debug_skip_publish_chunk", ctypes.c_int64), ("record_kernel_times", ctypes.c_uint32),
                ("use_start_state", ctypes.c_uint32), ("pair_mode", ctypes.c_uint32)]

    def __init__(self, start_state=PAREM_NONE, enumerate_all=0, segment_bytes=0, warps_per_block=0,
                 spec_cap_bytes=0, wait_budget_cycles=0, debug_skip_publish_chunk=0, record_kernel_times=0,
                 pair_mode=0):
        # start_state PAREM_NONE: start at the DFA's q0
        use = 0 if start_state == PAREM_NONE else 1
        super().__init__(0 if not use else start_state, enumerate_all, segment_bytes, warps_per_block,
                         spec_cap_bytes, wait_budget_cycles, debug_skip_publish_chunk, record_kernel_times, use,
                         pair_mode)


class Stats(ctypes.Structure):
    _fields_ = [("scan_ms", ctypes.c_float), ("emit_ms", ctypes.c_float), ("segment_bytes", ctypes.c_uint64),
                ("rows", ctypes.c_uint64), ("chunks", ctypes.c_uint64), ("blocks", ctypes.c_uint32),
                ("warps_per_block", ctypes.c_uint32), ("candidate_regs", ctypes.c_uint32),
                ("spec_cap_bytes", ctypes.c_uint32), ("kernels", ctypes.c_uint32),
                ("emit_replays", ctypes.c_uint32), ("emit_max_window", ctypes.c_uint32),
                ("nonconv_rows", ctypes.c_uint32), ("conv_max", ctypes.c_uint32),
                ("cycles_spec", ctypes.c_uint64), ("cycles_main", ctypes.c_uint64),
                ("cycles_resolve", ctypes.c_uint64), ("cycles_bitmap", ctypes.c_uint64),
                ("cycles_lane", ctypes.c_uint64), ("spec_lookups", ctypes.c_uint64),
                ("layout", ctypes.c_uint32), ("pair_hot_states", ctypes.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


@dataclass
class MatchResult:
    final_state: int
    accepted: bool
    match_count: int
    n_written: int
    status: int = 0


@dataclass
class DfaInfo:
    n_states: int
    n_symbols: int
    compact_states: int
    n_classes: int
    has_dead: bool
    entry_bytes: int
    layout: int
    table_bytes: int
    max_candidates: int
    mean_candidates: float
    sync_estimate: int = 0
    pair_hot_states: int = 0


def library_path() -> str:
    return os.path.join(_HERE, "_build", "libparem.so")


def load_library(build_if_missing: bool = False):
    """Load libparem.so; raises (no fallback) when it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            from . import build as _b
            _b.build()
        else:
            raise ImportError(f"libparem.so not built ({path}); run paper_1412_1741_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    lib.parem_load_dfa.argtypes = [vp, u32, u32, vp, u32, vp, ctypes.POINTER(vp)]
    lib.parem_prepare_info.argtypes = [vp, u32, u32, vp, u32, vp, ctypes.POINTER(_Info)]
    lib.parem_dfa_get_info.argtypes = [vp, ctypes.POINTER(_Info)]
    lib.parem_free_dfa.argtypes = [vp]
    lib.parem_free_dfa.restype = None
    lib.parem_match.argtypes = [vp, vp, u64, vp, u64, vp, ctypes.POINTER(_Result)]
    lib.parem_match_ex.argtypes = [vp, vp, u64, vp, u64, ctypes.POINTER(MatchOpts), vp, ctypes.POINTER(_Result)]
    lib.parem_match_host.argtypes = [vp, vp, u64, vp, u64, vp, ctypes.POINTER(_Result)]
    lib.parem_match_noalloc.argtypes = [vp, vp, u64, vp, u64, vp, ctypes.POINTER(_Result)]
    lib.parem_release_scratch.argtypes = [vp]
    lib.parem_last_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.parem_strerror.argtypes = [ctypes.c_int]
    lib.parem_strerror.restype = ctypes.c_char_p
    lib.parem_version.restype = ctypes.c_char_p
    lib.parem_regex_compile.argtypes = [ctypes.c_char_p, u64, u32, u32, ctypes.POINTER(vp)]
    lib.parem_regex_info.argtypes = [vp, ctypes.POINTER(u32), ctypes.POINTER(u32)]
    lib.parem_regex_export.argtypes = [vp, vp, vp, vp, ctypes.POINTER(u32)]
    lib.parem_regex_load.argtypes = [vp, ctypes.POINTER(vp)]
    lib.parem_regex_free.argtypes = [vp]
    lib.parem_regex_free.restype = None
    for f in ("parem_load_dfa", "parem_prepare_info", "parem_dfa_get_info", "parem_match", "parem_match_ex",
              "parem_match_host", "parem_release_scratch", "parem_last_stats", "parem_match_noalloc",
              "parem_regex_compile", "parem_regex_info", "parem_regex_export", "parem_regex_load"):
        getattr(lib, f).restype = ctypes.c_int
    _LIB = lib
    return lib


def parem_strerror(status: int) -> str:
    return load_library().parem_strerror(int(status)).decode()


def parem_version() -> str:
    return load_library().parem_version().decode()


def _dfa_arrays(table, byte_to_symbol, accept):
    table = np.ascontiguousarray(table, dtype=np.uint32)
    if table.ndim != 2:
        raise ValueError("table must be 2-D [n_states, n_symbols]")
    accept = np.ascontiguousarray(accept, dtype=np.uint8)
    b2s = None if byte_to_symbol is None else np.ascontiguousarray(byte_to_symbol, dtype=np.uint16)
    return table, b2s, accept


class Dfa:
    """Handle of a DFA loaded on the current CUDA device (parem_dfa*)."""

    def __init__(self, handle, info: DfaInfo):
        self._h = handle
        self.info = info

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("DFA has been freed")
        return self._h

    def free(self):
        if self._h is not None:
            load_library().parem_free_dfa(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _info(i: _Info) -> DfaInfo:
    return DfaInfo(i.n_states, i.n_symbols, i.compact_states, i.n_classes, bool(i.has_dead), i.entry_bytes,
                   i.layout, i.table_bytes, i.max_candidates, i.mean_candidates, i.sync_estimate,
                   i.pair_hot_states)


class _PairInfo(ctypes.Structure):
    _fields_ = [("layout", ctypes.c_uint32), ("hot_states", ctypes.c_uint32), ("accepted", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("warp_slow_share", ctypes.c_double),
                ("pair_table_bytes", ctypes.c_uint64)]


@dataclass
class PairPreview:
    layout: int
    hot_states: int
    accepted: bool
    warp_slow_share: float
    hot_orig: np.ndarray      # original id of each hot state (row order)
    pair_table: np.ndarray    # (hot_states + 1) x 729 uint8


def parem_pair_preview(table, byte_to_symbol, start, accept, sample) -> PairPreview:
    """Host-only plan of the two-byte stride variant for this DFA and text sample (no GPU)."""
    lib = load_library()
    table, b2s, accept = _dfa_arrays(table, byte_to_symbol, accept)
    sample = np.ascontiguousarray(sample, dtype=np.uint8)
    info = _PairInfo()
    vp = ctypes.c_void_p
    lib.parem_pair_preview.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32, vp, ctypes.c_uint32, vp, vp,
                                       ctypes.c_uint64, ctypes.POINTER(_PairInfo), vp, vp, ctypes.c_uint64]
    lib.parem_pair_preview.restype = ctypes.c_int
    args = (table.ctypes.data, table.shape[0], table.shape[1], None if b2s is None else b2s.ctypes.data,
            int(start), accept.ctypes.data, sample.ctypes.data, int(sample.size))
    rc = lib.parem_pair_preview(*args, ctypes.byref(info), None, None, ctypes.c_uint64(0))
    if rc != PAREM_OK:
        raise ParemError(rc, "parem_pair_preview")
    hot = np.zeros(max(info.hot_states, 1), np.uint32)
    t2 = np.zeros(max(int(info.pair_table_bytes), 1), np.uint8)
    if info.hot_states:
        rc = lib.parem_pair_preview(*args, ctypes.byref(info), hot.ctypes.data, t2.ctypes.data,
                                    ctypes.c_uint64(t2.size))
        if rc != PAREM_OK:
            raise ParemError(rc, "parem_pair_preview")
    return PairPreview(info.layout, info.hot_states, bool(info.accepted), info.warp_slow_share,
                       hot[:info.hot_states], t2[:int(info.pair_table_bytes)].reshape(-1, 729) if info.hot_states
                       else np.zeros((0, 729), np.uint8))


def parem_prepare_info(table, byte_to_symbol, start, accept) -> DfaInfo:
    lib = load_library()
    table, b2s, accept = _dfa_arrays(table, byte_to_symbol, accept)
    info = _Info()
    rc = lib.parem_prepare_info(table.ctypes.data, table.shape[0], table.shape[1],
                                None if b2s is None else b2s.ctypes.data, int(start), accept.ctypes.data,
                                ctypes.byref(info))
    if rc != PAREM_OK:
        raise ParemError(rc, "parem_prepare_info")
    return _info(info)


def parem_load_dfa(table, byte_to_symbol, start, accept) -> Dfa:
    lib = load_library()
    table, b2s, accept = _dfa_arrays(table, byte_to_symbol, accept)
    h = ctypes.c_void_p()
    rc = lib.parem_load_dfa(table.ctypes.data, table.shape[0], table.shape[1],
                            None if b2s is None else b2s.ctypes.data, int(start), accept.ctypes.data,
                            ctypes.byref(h))
    if rc != PAREM_OK:
        raise ParemError(rc, "parem_load_dfa")
    info = _Info()
    lib.parem_dfa_get_info(h, ctypes.byref(info))
    return Dfa(h, _info(info))


PAREM_REGEX_ANCHORED = 1


@dataclass
class RegexDfa:
    """A compiled regular expression: the DFA in parem_load_dfa's form (host arrays)."""
    table: np.ndarray           # (n_states, n_symbols) uint32, PAREM_NONE where no match continues
    byte_to_symbol: np.ndarray  # (256,) uint16
    accept: np.ndarray          # (n_states,) uint8
    start: int


def parem_regex_compile(pattern, flags: int = 0, max_states: int = 0) -> RegexDfa:
    """Compile a regular expression (bytes or str) with the operators of Table III into a
    DFA (host only).  flags 0: search (accept after every position where a match ends);
    PAREM_REGEX_ANCHORED: prefixes."""
    lib = load_library()
    pat = pattern.encode() if isinstance(pattern, str) else bytes(pattern)
    h = ctypes.c_void_p()
    rc = lib.parem_regex_compile(pat, len(pat), int(flags), int(max_states), ctypes.byref(h))
    if rc != PAREM_OK:
        raise ParemError(rc, "parem_regex_compile")
    try:
        ns, nsym = ctypes.c_uint32(), ctypes.c_uint32()
        rc = lib.parem_regex_info(h, ctypes.byref(ns), ctypes.byref(nsym))
        if rc != PAREM_OK:
            raise ParemError(rc, "parem_regex_info")
        table = np.empty((ns.value, nsym.value), np.uint32)
        b2s = np.empty(256, np.uint16)
        acc = np.empty(ns.value, np.uint8)
        start = ctypes.c_uint32()
        rc = lib.parem_regex_export(h, table.ctypes.data, b2s.ctypes.data, acc.ctypes.data, ctypes.byref(start))
        if rc != PAREM_OK:
            raise ParemError(rc, "parem_regex_export")
    finally:
        lib.parem_regex_free(h)
    return RegexDfa(table, b2s, acc, int(start.value))


def parem_load_regex(pattern, flags: int = 0, max_states: int = 0) -> Dfa:
    """Compile a regular expression and load its DFA on the current device."""
    r = parem_regex_compile(pattern, flags, max_states)
    return parem_load_dfa(r.table, r.byte_to_symbol, r.start, r.accept)


def parem_dfa_get_info(dfa: Dfa) -> DfaInfo:
    """The DFA's description as the library reports it now (the two-byte stride variant's hot
    states appear once a scan has learned them)."""
    info = _Info()
    rc = load_library().parem_dfa_get_info(dfa.handle, ctypes.byref(info))
    if rc != PAREM_OK:
        raise ParemError(rc, "parem_dfa_get_info")
    return _info(info)


def parem_free_dfa(dfa: Dfa) -> None:
    dfa.free()


def _ptr_len(buf, length=None):
    """(pointer, length) of a CUDA tensor / numpy array / raw pointer int."""
    if buf is None:
        return None, 0
    if isinstance(buf, int):
        if length is None:
            raise ValueError("a raw pointer needs an explicit length")
        return buf, int(length)
    if hasattr(buf, "data_ptr"):
        return buf.data_ptr(), int(buf.numel() * buf.element_size()) if length is None else int(length)
    if isinstance(buf, np.ndarray):
        return buf.ctypes.data, int(buf.nbytes) if length is None else int(length)
    raise TypeError(f"unsupported buffer type {type(buf)}")


def _stream(stream):
    if stream is None:
        import torch
        raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)
        if raw is not None:  # the current stream's handle without building a Stream object
            return ctypes.c_void_p(raw(torch._C._cuda_getDevice()))
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _finish(rc, res: _Result, where):
    if rc not in (PAREM_OK, PAREM_ERR_CAPACITY):
        raise ParemError(rc, where)
    return MatchResult(res.final_state, bool(res.accepted), res.match_count, res.n_written, rc)


def parem_match_ex(dfa: Dfa, text, positions=None, opts: MatchOpts | None = None, stream=None,
                   length=None, capacity=None) -> MatchResult:
    lib = load_library()
    tp, n = _ptr_len(text, length)
    pp, pbytes = _ptr_len(positions)
    cap = (pbytes // 8 if capacity is None else int(capacity)) if pp else 0
    res = _Result()
    rc = lib.parem_match_ex(dfa.handle, tp, n, pp, cap, None if opts is None else ctypes.byref(opts),
                            _stream(stream), ctypes.byref(res))
    return _finish(rc, res, "parem_match_ex")


def parem_match(dfa: Dfa, text, positions=None, stream=None, length=None, capacity=None) -> MatchResult:
    lib = load_library()
    tp, n = _ptr_len(text, length)
    pp, pbytes = _ptr_len(positions)
    cap = (pbytes // 8 if capacity is None else int(capacity)) if pp else 0
    res = _Result()
    rc = lib.parem_match(dfa.handle, tp, n, pp, cap, _stream(stream), ctypes.byref(res))
    return _finish(rc, res, "parem_match")


def parem_match_host(dfa: Dfa, text, positions=None, stream=None) -> MatchResult:
    """Text and positions in host memory (numpy arrays, pinned torch tensors)."""
    lib = load_library()
    tp, n = _ptr_len(text)
    pp, pbytes = _ptr_len(positions)
    cap = pbytes // 8 if pp else 0
    res = _Result()
    rc = lib.parem_match_host(dfa.handle, tp, n, pp, cap, _stream(stream), ctypes.byref(res))
    return _finish(rc, res, "parem_match_host")


def parem_release_scratch(stream=None) -> None:
    rc = load_library().parem_release_scratch(_stream(stream))
    if rc != PAREM_OK:
        raise ParemError(rc, "parem_release_scratch")


def parem_last_stats(stream=None) -> dict:
    """Plan and (when record_kernel_times was set) kernel times of the last scan on a stream."""
    st = Stats()
    rc = load_library().parem_last_stats(_stream(stream), ctypes.byref(st))
    if rc != PAREM_OK:
        raise ParemError(rc, "parem_last_stats")
    return st.as_dict()


def parem_match_noalloc(dfa: Dfa, text, positions=None, stream=None, length=None, capacity=None) -> MatchResult:
    """parem_match with all scratch in the library's fixed device array (no allocation).

    For callers that cannot let the library allocate device memory.  Raises ParemError with
    status PAREM_ERR_TOO_LARGE when the text needs more scratch than the fixed area holds.
    Calls share the area, so calls that overlap on the GPU must be serialised by the caller.
    """
    lib = load_library()
    tp, n = _ptr_len(text, length)
    pp, pbytes = _ptr_len(positions)
    cap = (pbytes // 8 if capacity is None else int(capacity)) if pp else 0
    res = _Result()
    rc = lib.parem_match_noalloc(dfa.handle, tp, n, pp, cap, _stream(stream), ctypes.byref(res))
    return _finish(rc, res, "parem_match_noalloc")


# ---------------------------------------------------------------------------------------
# batched matching
# ---------------------------------------------------------------------------------------
class _BatchItem(ctypes.Structure):
    _fields_ = [("dfa", ctypes.c_void_p), ("text", ctypes.c_void_p), ("len", ctypes.c_uint64),
                ("positions", ctypes.c_void_p), ("capacity", ctypes.c_uint64)]


# speculation forms of a batch DFA (parem_batch_opts.spec, parem_batch_config.spec)
PAREM_BATCH_SPEC_AUTO = 0
PAREM_BATCH_SPEC_GROUPED = 1
PAREM_BATCH_SPEC_WARP = 2
PAREM_BATCH_SPEC_WARP_BITMAP = 3
BATCH_SPEC_NAMES = {1: "grouped", 2: "warp", 3: "warp_bitmap"}


class BatchOpts(ctypes.Structure):
    _fields_ = [("autotune", ctypes.c_uint32), ("warps_per_block", ctypes.c_uint32),
                ("segment_bytes", ctypes.c_uint64), ("use_graph", ctypes.c_uint32), ("spec", ctypes.c_uint32)]

    def __init__(self, autotune=0, warps_per_block=0, segment_bytes=0, use_graph=1, spec=PAREM_BATCH_SPEC_AUTO):
        super().__init__(autotune, warps_per_block, segment_bytes, use_graph, spec)


class _BatchConfig(ctypes.Structure):
    _fields_ = [("segment_bytes", ctypes.c_uint64), ("spec", ctypes.c_uint32), ("warps_per_block", ctypes.c_uint32),
                ("smem_table", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


def _bind_batch(lib):
    if getattr(lib, "_batch_bound", False):
        return
    vp = ctypes.c_void_p
    lib.parem_batch_create.argtypes = [ctypes.POINTER(_BatchItem), ctypes.c_uint32, ctypes.POINTER(BatchOpts),
                                       ctypes.POINTER(vp)]
    lib.parem_batch_create.restype = ctypes.c_int
    lib.parem_batch_run.argtypes = [vp, vp]
    lib.parem_batch_run.restype = ctypes.c_int
    lib.parem_batch_results.argtypes = [vp, ctypes.POINTER(_Result)]
    lib.parem_batch_results.restype = ctypes.c_int
    lib.parem_batch_item_segment.argtypes = [vp, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64)]
    lib.parem_batch_item_segment.restype = ctypes.c_int
    lib.parem_batch_item_config.argtypes = [vp, ctypes.c_uint32, ctypes.POINTER(_BatchConfig)]
    lib.parem_batch_item_config.restype = ctypes.c_int
    lib.parem_batch_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.parem_batch_stats.restype = ctypes.c_int
    lib.parem_batch_free.argtypes = [vp]
    lib.parem_batch_free.restype = None
    lib._batch_bound = True


class Batch:
    """A planned batch (parem_batch*): run() replays it; results() in the order given."""

    def __init__(self, handle, n, keep):
        self._h = handle
        self.n = n
        self._keep = keep  # the tensors whose memory the batch refers to

    def run(self, stream=None) -> int:
        lib = load_library()
        rc = lib.parem_batch_run(self._h, _stream(stream))
        if rc not in (PAREM_OK, PAREM_ERR_CAPACITY):
            raise ParemError(rc, "parem_batch_run")
        return rc

    def results(self):
        lib = load_library()
        arr = (_Result * self.n)()
        rc = lib.parem_batch_results(self._h, arr)
        if rc != PAREM_OK:
            raise ParemError(rc, "parem_batch_results")
        return [MatchResult(r.final_state, bool(r.accepted), r.match_count, r.n_written) for r in arr]

    def segments(self):
        lib = load_library()
        out = []
        v = ctypes.c_uint64()
        for i in range(self.n):
            lib.parem_batch_item_segment(self._h, i, ctypes.byref(v))
            out.append(v.value)
        return out

    def configs(self):
        """Per item (given order): the segment size, speculation form, block shape and table
        tier the batch chose."""
        lib = load_library()
        out = []
        c = _BatchConfig()
        for i in range(self.n):
            rc = lib.parem_batch_item_config(self._h, i, ctypes.byref(c))
            if rc != PAREM_OK:
                raise ParemError(rc, "parem_batch_item_config")
            out.append({"segment_bytes": c.segment_bytes, "spec": BATCH_SPEC_NAMES.get(c.spec, str(c.spec)),
                        "warps_per_block": c.warps_per_block, "smem_table": bool(c.smem_table)})
        return out

    def stats(self) -> dict:
        st = Stats()
        rc = load_library().parem_batch_stats(self._h, ctypes.byref(st))
        if rc != PAREM_OK:
            raise ParemError(rc, "parem_batch_stats")
        return st.as_dict()

    def free(self):
        if self._h is not None:
            load_library().parem_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def parem_batch_create(items, opts: BatchOpts | None = None) -> Batch:
    """items: sequence of (dfa, text, positions_or_None) with CUDA tensors (or
    (dfa, text_ptr, length, positions_ptr, capacity) tuples of raw device pointers)."""
    lib = load_library()
    _bind_batch(lib)
    arr = (_BatchItem * len(items))()
    keep = []
    for i, it in enumerate(items):
        if len(it) == 5:
            dfa, tp, n, pp, cap = it
        else:
            dfa, text, pos = it
            tp, n = _ptr_len(text)
            pp, pb = _ptr_len(pos)
            cap = pb // 8 if pp else 0
            keep.append((text, pos))
        arr[i] = _BatchItem(dfa.handle, tp, n, pp, cap)
    h = ctypes.c_void_p()
    rc = lib.parem_batch_create(arr, len(items), None if opts is None else ctypes.byref(opts), ctypes.byref(h))
    if rc != PAREM_OK:
        raise ParemError(rc, "parem_batch_create")
    return Batch(h, len(items), keep)


# ---------------------------------------------------------------------------------------
# request server (continuous batching)
# ---------------------------------------------------------------------------------------
PAREM_SERVE_BATCH = 0
PAREM_SERVE_FIFO = 1

# parem_request and parem_response as numpy records (the C layouts, 56 and 64 bytes)
REQUEST_DTYPE = np.dtype({
    "names": ["dfa_index", "text", "len", "positions", "capacity", "tag", "arrival_ns"],
    "formats": [np.uint32, np.uint64, np.uint64, np.uint64, np.uint64, np.uint64, np.int64],
    "offsets": [0, 8, 16, 24, 32, 40, 48], "itemsize": 56})
RESPONSE_DTYPE = np.dtype({
    "names": ["tag", "status", "batch_size", "final_state", "accepted", "match_count", "n_written",
              "arrival_ns", "launch_ns", "done_ns"],
    "formats": [np.uint64, np.int32, np.uint32, np.uint32, np.uint8, np.uint64, np.uint64,
                np.int64, np.int64, np.int64],
    "offsets": [0, 8, 12, 16, 20, 24, 32, 40, 48, 56], "itemsize": 64})


class ServerOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_uint32), ("arenas", ctypes.c_uint32), ("max_items", ctypes.c_uint32),
                ("reserved0", ctypes.c_uint32), ("max_batch_bytes", ctypes.c_uint64),
                ("arena_scratch_bytes", ctypes.c_uint64), ("reserved", ctypes.c_uint64 * 4)]

    def __init__(self, mode=PAREM_SERVE_BATCH, arenas=0, max_items=0, max_batch_bytes=0, arena_scratch_bytes=0):
        super().__init__(mode, arenas, max_items, 0, max_batch_bytes, arena_scratch_bytes)


class _ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("answered", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("bytes", ctypes.c_uint64), ("max_batch", ctypes.c_uint64), ("kernels", ctypes.c_uint64),
                ("reserved", ctypes.c_uint64 * 2)]


def _bind_server(lib):
    if getattr(lib, "_server_bound", False):
        return
    vp, u32 = ctypes.c_void_p, ctypes.c_uint32
    lib.parem_server_create.argtypes = [ctypes.POINTER(vp), u32, ctypes.POINTER(ServerOpts), ctypes.POINTER(vp)]
    lib.parem_server_submit.argtypes = [vp, vp, u32]
    lib.parem_server_poll.argtypes = [vp, vp, u32, ctypes.POINTER(u32), ctypes.c_int64]
    lib.parem_server_drain.argtypes = [vp]
    lib.parem_server_replay.argtypes = [vp, vp, u32, vp]
    lib.parem_server_get_stats.argtypes = [vp, ctypes.POINTER(_ServerStats)]
    for f in ("parem_server_create", "parem_server_submit", "parem_server_poll", "parem_server_drain",
              "parem_server_replay", "parem_server_get_stats"):
        getattr(lib, f).restype = ctypes.c_int
    lib.parem_server_free.argtypes = [vp]
    lib.parem_server_free.restype = None
    lib.parem_clock_ns.argtypes = []
    lib.parem_clock_ns.restype = ctypes.c_int64
    lib._server_bound = True


def make_requests(dfa_index, text_ptr, length, positions_ptr=0, capacity=0, tag=None, arrival_ns=0):
    """Vectorised construction of a parem_request array (device addresses as integers)."""
    n = len(np.atleast_1d(length))
    r = np.zeros(n, dtype=REQUEST_DTYPE)
    r["dfa_index"] = dfa_index
    r["text"] = text_ptr
    r["len"] = length
    r["positions"] = positions_ptr
    r["capacity"] = capacity
    r["tag"] = np.arange(n, dtype=np.uint64) if tag is None else tag
    r["arrival_ns"] = arrival_ns
    return r


class Server:
    """A request server (parem_server*): submit()/poll() or an open-loop replay() of a trace."""

    def __init__(self, handle, dfas):
        self._h = handle
        self._dfas = list(dfas)  # the DFAs must outlive the server

    def submit(self, requests) -> None:
        req = np.ascontiguousarray(requests, dtype=REQUEST_DTYPE)
        rc = load_library().parem_server_submit(self._h, req.ctypes.data, len(req))
        if rc != PAREM_OK:
            raise ParemError(rc, "parem_server_submit")

    def poll(self, max_n=4096, wait_s=0.0):
        out = np.zeros(max_n, dtype=RESPONSE_DTYPE)
        got = ctypes.c_uint32()
        rc = load_library().parem_server_poll(self._h, out.ctypes.data, max_n, ctypes.byref(got), int(wait_s * 1e9))
        if rc != PAREM_OK:
            raise ParemError(rc, "parem_server_poll")
        return out[: got.value]

    def drain(self) -> None:
        load_library().parem_server_drain(self._h)

    def replay(self, requests):
        """Submit requests[i] at (call time + requests[i]['arrival_ns']); returns the responses in
        request order."""
        req = np.ascontiguousarray(requests, dtype=REQUEST_DTYPE)
        out = np.zeros(len(req), dtype=RESPONSE_DTYPE)
        rc = load_library().parem_server_replay(self._h, req.ctypes.data, len(req), out.ctypes.data)
        if rc != PAREM_OK:
            raise ParemError(rc, "parem_server_replay")
        return out

    def stats(self) -> dict:
        st = _ServerStats()
        load_library().parem_server_get_stats(self._h, ctypes.byref(st))
        return {k: getattr(st, k) for k in ("submitted", "answered", "batches", "bytes", "max_batch", "kernels")}

    def free(self):
        if self._h is not None:
            load_library().parem_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def parem_server_create(dfas, opts: ServerOpts | None = None) -> Server:
    lib = load_library()
    _bind_server(lib)
    arr = (ctypes.c_void_p * len(dfas))(*[d.handle for d in dfas])
    h = ctypes.c_void_p()
    rc = lib.parem_server_create(arr, len(dfas), None if opts is None else ctypes.byref(opts), ctypes.byref(h))
    if rc != PAREM_OK:
        raise ParemError(rc, "parem_server_create")
    return Server(h, dfas)


def parem_clock_ns() -> int:
    lib = load_library()
    _bind_server(lib)
    return lib.parem_clock_ns()
