"""Concurrent host callers: several threads calling the library at once, on one shared stream or on
a stream each, get exactly the results each call gives alone (the oracle's). A kernel that writes
past its own buffers corrupts a neighbouring allocation that, with interleaved callers, belongs to
another call; these tests catch that. The checked build (kernels verify their computed indices
and record the first violation instead of touching memory) runs the same workload and must record
none."""
import os
import subprocess
import sys
import threading

import numpy as np
import pytest

import oracle
import paper_2010_10055_gb300 as sg
from tests.gpu_util import assert_graph_equal, assert_kmer_equal, assert_overlap_equal, dev
from tests.test_gpu_serve import _jobs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cases():
    jobs = _jobs(21, 8)
    out = []
    for j in jobs:
        km = oracle.build_kmer_matrix(j["seq"], j["offsets"], 17, j["lo"], j["hi"])
        C = oracle.overlap_spgemm(km["A"], km["At"], 2, 2)
        S, it = oracle.transitive_reduce(j["R"], 300)
        out.append(dict(job=j, km=km, C=C, S=S, it=it))
    return out


def _full_path(case, stream):
    j = case["job"]
    km = sg.build_kmer_matrix(dev(j["seq"], np.uint8), dev(j["offsets"], np.int64), 17, j["lo"], j["hi"],
                              stream=stream)
    C = sg.overlap_spgemm(km, 2, 2, stream=stream)
    S, it = sg.transitive_reduce(sg.DeviceGraph.from_numpy(j["R"]), 300, stream=stream)
    return km.to_numpy(), C.to_numpy(), S.to_numpy(), it


def _run_threads(cases, nthreads, shared_stream, reps):
    import torch
    failures = []
    for _ in range(reps):
        streams = [torch.cuda.Stream() for _ in range(nthreads)]
        if shared_stream:
            streams = [streams[0]] * nthreads
        results = [[] for _ in range(nthreads)]

        def work(t):
            try:
                with torch.cuda.stream(streams[t]):
                    for q in range(t, len(cases), nthreads):
                        results[t].append((q, _full_path(cases[q], streams[t])))
            except Exception as e:  # reported below, not swallowed
                failures.append(repr(e))

        th = [threading.Thread(target=work, args=(t,)) for t in range(nthreads)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        torch.cuda.synchronize()
        assert failures == []
        for t in range(nthreads):
            for q, (km, C, S, it) in results[t]:
                assert_kmer_equal(km, cases[q]["km"])
                assert_overlap_equal(C, cases[q]["C"])
                assert_graph_equal(S, cases[q]["S"])
                assert it == cases[q]["it"]


def test_two_threads_one_shared_stream(cases):
    _run_threads(cases, 2, True, 4)


def test_three_threads_own_streams(cases):
    _run_threads(cases, 3, False, 4)


def test_concurrent_batches_match_their_items_alone(cases):
    import torch
    groups = [[0, 1, 2], [3, 4], [5, 6, 7]]
    out, failures = {}, []

    def work(g):
        st = torch.cuda.Stream()
        try:
            with torch.cuda.stream(st):
                items = [dict(seq=dev(cases[q]["job"]["seq"], np.uint8), offsets=dev(cases[q]["job"]["offsets"], np.int64),
                              lo=cases[q]["job"]["lo"], hi=cases[q]["job"]["hi"]) for q in g]
                r = sg.run_batch(items, k=17, stream=st)
                for b, q in enumerate(g):
                    out[q] = r.item(b)
        except Exception as e:
            failures.append(repr(e))

    th = [threading.Thread(target=work, args=(g,)) for g in groups]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert failures == []
    for q in range(8):
        assert_kmer_equal(out[q], cases[q]["km"])
        assert_overlap_equal(out[q]["C"], cases[q]["C"])


_CHECKED_SCRIPT = r"""
import sys, threading
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import paper_2010_10055_gb300 as sg
sg.use_checked_build()
from tests.gpu_util import dev
from tests.test_gpu_serve import _jobs
jobs = _jobs(22, 6)
def work(t):
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        for j in jobs[t::2]:
            km = sg.build_kmer_matrix(dev(j["seq"], np.uint8), dev(j["offsets"], np.int64), 17, j["lo"], j["hi"], stream=st)
            C = sg.overlap_spgemm(km, 2, 2, stream=st)
            S, it = sg.transitive_reduce(sg.DeviceGraph.from_numpy(j["R"]), 300, stream=st)
            S.to_numpy(); C.to_numpy()
th = [threading.Thread(target=work, args=(t,)) for t in range(2)]
[x.start() for x in th]; [x.join() for x in th]
torch.cuda.synchronize()
print("CHECK", sg.debug_check())
"""


def test_checked_build_records_no_violation():
    from paper_2010_10055_gb300 import build_lib
    build_lib.build(checked=True)
    p = subprocess.run([sys.executable, "-c", _CHECKED_SCRIPT, ROOT], capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    assert "CHECK None" in p.stdout, p.stdout[-2000:]
