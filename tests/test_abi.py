"""The C-ABI library loads on a machine without a GPU and exports every function that
include/sgraph.h declares (no compute calls here)."""
import os
import re

import paper_2010_10055_gb300 as sg

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def declared():
    names = set()
    for f in os.listdir(HDR):
        if f.endswith(".h"):
            txt = open(os.path.join(HDR, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            txt = re.sub(r"typedef\s+sg_status\s*\(\*[^;]*;", "", txt)  # callback types, not functions
            names |= set(re.findall(r"\b(sg_[a-z0-9_]+)\s*\(", txt))
    return names


def test_header_declares_the_three_operations():
    d = declared()
    assert {"sg_build_kmer_matrix", "sg_overlap_spgemm", "sg_transitive_reduce"} <= d


def test_library_exports_every_declared_symbol():
    from paper_2010_10055_gb300 import build_lib
    build_lib.build()
    L = sg.lib()
    missing = [n for n in declared() if not hasattr(L, n)]
    assert not missing, missing
    assert set(sg.EXPORTS) <= declared()


def test_host_only_calls_work_without_gpu():
    L = sg.lib()
    assert isinstance(sg.launch_count(), int)
    sg.prof_enable(False)
    sg.prof_reset()
    assert sg.prof_collect() == {}
    assert L.sg_last_error() is not None
