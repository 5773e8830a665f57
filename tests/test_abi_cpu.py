"""CPU-only checks of the C ABI: the library loads, exports every symbol the header declares,
and the host-side preparation (parem_prepare_info) validates inputs and plans as documented.
No GPU compute is called here."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1412_1741_gb300 as pm
from paper_1412_1741_gb300 import build as pbuild
from paper_1412_1741_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return pm.load_library()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(parem_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "parem_load_dfa" in names and "parem_match" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(pm.EXPORTED_SYMBOLS)


def test_strerror_and_version(lib):
    assert pm.parem_strerror(0) == "ok"
    assert "wait" in pm.parem_strerror(-4)
    assert re.match(r"^\d+\.\d+\.\d+$", pm.parem_version())


def test_prepare_info_of_the_workload_dfas(lib):
    g = wl.gattaca_dfa()
    i = pm.parem_prepare_info(g.table, g.byte_to_symbol, g.start, g.accept)
    # bytes >= 4 are outside {A,C,G,T}: a dead state is added; a tiny table is byte-indexed,
    # and with bytes 0..3 its own classes and all others one class it gets the 4-byte stride
    # table: 9 states x 5^4 one-byte entries after the 9 x 256 byte table
    assert i.has_dead and i.compact_states == 9 and i.layout == 6 and i.entry_bytes == 1
    assert i.n_classes == 5 and 9 * 256 + 9 * 625 <= i.table_bytes <= 9 * 260 + 9 * 625 + 32
    # img of each symbol of the KMP automaton of GATTACA: A->{0,2,5,7}, C->{0,6}, G->{1}, T->{0,3,4}
    assert i.max_candidates == 4
    d = wl.dense_dfa()
    i = pm.parem_prepare_info(d.table, d.byte_to_symbol, d.start, d.accept)
    assert not i.has_dead and i.compact_states == 256 and i.layout == 0 and i.entry_bytes == 1
    assert 140 <= i.max_candidates <= 200
    a = wl.keywords_ac_dfa()
    i = pm.parem_prepare_info(a.table, a.byte_to_symbol, a.start, a.accept)
    # 26 letters + space + the class of bytes outside the alphabet; too big to be byte-indexed;
    # every byte but a-z and space shares one class, so the columns are computed (layout 7)
    assert i.n_classes == 28 and i.layout == 7 and i.entry_bytes == 2 and i.has_dead
    assert 900 <= i.n_states <= 1100


def test_candidate_set_sizes_match_the_paper_example(lib):
    p = wl.parallel_dfa()
    # a complete DFA over its 5 symbols; identity byte map leaves bytes >= 5 outside
    i = pm.parem_prepare_info(p.table, None, 0, p.accept)
    assert i.layout == 6 and i.n_classes == 6
    # img(l) = {0,5,6,8} is the largest image (Section II-C)
    assert i.max_candidates == 4


def test_identical_columns_merge_into_one_class(lib):
    t = np.array([[1, 1, 0], [0, 0, 1]], dtype=np.uint32)  # symbols 0 and 1 act the same
    b2s = np.full(256, pm.PAREM_NONE16, np.uint16)
    b2s[ord("a")], b2s[ord("b")], b2s[ord("c")] = 0, 1, 2
    i = pm.parem_prepare_info(t, b2s, 0, np.array([0, 1], np.uint8))
    assert i.n_classes == 3  # {a,b}, {c}, outside


@pytest.mark.parametrize("case", ["entry", "start", "nstates", "b2s", "nsym"])
def test_invalid_inputs_are_rejected(lib, case):
    t = np.zeros((3, 2), np.uint32)
    acc = np.zeros(3, np.uint8)
    b2s = None
    start = 0
    if case == "entry":
        t[1, 1] = 3
    elif case == "start":
        start = 3
    elif case == "nstates":
        t = np.zeros((65536, 1), np.uint32)
        acc = np.zeros(65536, np.uint8)
    elif case == "b2s":
        b2s = np.zeros(256, np.uint16)
        b2s[7] = 2
    elif case == "nsym":
        t = np.zeros((1, 257), np.uint32)
        acc = np.zeros(1, np.uint8)
    with pytest.raises(pm.ParemError) as e:
        pm.parem_prepare_info(t, b2s, start, acc)
    assert e.value.status == -1


def test_null_pointers_are_rejected(lib):
    res = ctypes.c_void_p()
    assert lib.parem_load_dfa(None, 1, 1, None, 0, None, ctypes.byref(res)) == -1
    assert lib.parem_match(None, None, 0, None, 0, None, None) == -1
    assert lib.parem_dfa_get_info(None, None) == -1


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct the binding marshals has the C layout of include/parem.h: a C program
    compiled against the header prints each struct's size and each field's offset, which must
    equal the ctypes mirrors' (and the numpy records' for requests and responses)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = [("parem_result", pm._Result), ("parem_dfa_info", pm._Info), ("parem_match_opts", pm.MatchOpts),
               ("parem_stats", pm.Stats), ("parem_pair_info", pm._PairInfo), ("parem_batch_item", pm._BatchItem),
               ("parem_batch_opts", pm.BatchOpts), ("parem_batch_config", pm._BatchConfig),
               ("parem_server_opts", pm.ServerOpts), ("parem_server_stats", pm._ServerStats)]
    records = [("parem_request", pm.REQUEST_DTYPE), ("parem_response", pm.RESPONSE_DTYPE)]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "parem.h"', "int main(void) {"]
    want = {}
    for cname, cls in mirrors:
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        want[cname] = ctypes.sizeof(cls)
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
            want[f"{cname}.{fname}"] = getattr(cls, fname).offset
    nested = {"final_state", "accepted", "match_count", "n_written"}  # the response's parem_result
    for cname, dt in records:
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        want[cname] = dt.itemsize
        for fname in dt.names:
            member = f"result.{fname}" if cname == "parem_response" and fname in nested else fname
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {member}));')
            want[f"{cname}.{fname}"] = dt.fields[fname][1]
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(ln.rsplit(" ", 1) for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                           check=True).stdout.splitlines())
    assert {k: int(v) for k, v in got.items()} == want
