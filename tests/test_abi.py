"""The C ABI library builds and exports every entry point include/*.h declares (no GPU
needed: nothing here launches a kernel)."""
import ctypes
import glob
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(pastis_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2009_14467_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert {"pastis_encode", "pastis_build_kmers", "pastis_overlap_spgemm", "pastis_align_pairs",
            "pastis_filter_edges", "pastis_substitute_kmers"} <= declared
    for name in sorted(declared):
        assert hasattr(lib, name), f"{name} declared but not exported"


def test_host_only_entry_points():
    from paper_2009_14467_gb300 import pastis as P
    L = P.lib()
    assert L.pastis_status_string(3) == b"output buffer too small"
    cap, cpl = ctypes.c_int64(), ctypes.c_int64()
    assert L.pastis_kmat_sizes(10, 1000, 6, ctypes.byref(cap), ctypes.byref(cpl)) == 0
    assert cap.value == 1000 and cpl.value == 24 ** 6 + 1
    assert L.pastis_kmat_sizes(10, 1000, 7, ctypes.byref(cap), ctypes.byref(cpl)) == 1


def test_record_layouts_match_header():
    from paper_2009_14467_gb300 import pastis as P
    assert P.CAND_DTYPE.itemsize == P.ALN_DTYPE.itemsize == P.EDGE_DTYPE.itemsize == 20
    assert ctypes.sizeof(P.c_params) == 9 * 4 + 576
    assert ctypes.sizeof(P.c_kmat) == 4 + 4 + 8 + 8 + 6 * 8
    p = P.Params(matrix=np.zeros((24, 24), np.int8), k=5, m_subs=7).c()
    assert p.k == 5 and p.m_subs == 7 and p.gap_open == 11
