"""The allocation-free min-plus product (sg_minplus_square_noalloc).

Callers that cannot allocate device memory when they need N = R^2 -- a process held under a hard
GPU memory cap, code running while a memory pool is exhausted or being torn down, a host thread
that must not take the allocator's locks -- use this entry point; its workspace is a fixed device
array that the library reserves at load time. This file runs last so that a failure here comes
after every other test. It calls the C ABI directly and checks the result against
sg_minplus_square, bit for bit, on consecutive calls that reuse the shared workspace."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import paper_2010_10055_gb300 as sg
import synth

pytestmark = pytest.mark.gpu

ARGS = [ctypes.POINTER(sg.GraphCsr), ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def hub_graph(n, hubs, hub_deg, deg, seed):
    """Random graph whose first `hubs` rows have `hub_deg` entries each (rows above 1,024 entries
    take the global-memory path and are listed after the shared-memory rows), the others 1 to
    2 deg - 1; sorted distinct columns, no diagonal."""
    rng = np.random.default_rng(seed)
    cols, rp = [], [0]
    for i in range(n):
        d = hub_deg if i < hubs else int(rng.integers(1, 2 * deg))
        c = rng.choice(n - 1, size=min(d, n - 1), replace=False)
        c = np.sort(c + (c >= i)).astype(np.int32)
        cols.append(c)
        rp.append(rp[-1] + c.size)
    col = np.concatenate(cols)
    return dict(n=n, row_ptr=np.array(rp, np.int64), col=col,
                suffix=rng.integers(0, 5000, col.size).astype(np.uint32),
                dir=rng.integers(0, 4, col.size).astype(np.uint8))


def _entry(name):
    from paper_2010_10055_gb300 import build_lib
    build_lib.build()
    fn = getattr(sg.lib(), name)
    fn.restype = ctypes.c_int
    fn.argtypes = ARGS
    return fn


def _run(fn, R, mode):
    import torch
    D = sg.DeviceGraph.from_numpy(R)
    N = torch.full((max(D.nnz, 1),), 7, dtype=torch.int32, device="cuda")
    Nd = torch.full((max(D.nnz, 1),), 9, dtype=torch.uint8, device="cuda")
    rc = fn(ctypes.byref(D.s), mode, ctypes.c_void_p(N.data_ptr()), ctypes.c_void_p(Nd.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, N[:D.nnz].cpu().numpy().view(np.uint32), Nd[:D.nnz].cpu().numpy()


def test_noalloc_matches_minplus_square_on_consecutive_calls():
    noalloc, plain = _entry("sg_minplus_square_noalloc"), _entry("sg_minplus_square")
    big = synth.random_graph(3000, 80.0, hub_frac=0.02, max_suffix=5000, seed=21)  # hub rows > 1024 entries
    assert np.diff(big["row_ptr"]).max() > 1024
    small = synth.random_graph(500, 6.0, max_suffix=300, seed=22)
    for R, mode in ((big, 0), (small, 1), (big, 1), (small, 0)):
        rc, N, Nd = _run(noalloc, R, mode)
        assert rc == sg.SG_OK, sg.lib().sg_last_error()
        rc2, N2, Nd2 = _run(plain, R, mode)
        assert rc2 == sg.SG_OK
        assert np.array_equal(N, N2)
        assert np.array_equal(Nd, Nd2)


def test_noalloc_rejects_graphs_beyond_its_workspace():
    noalloc = _entry("sg_minplus_square_noalloc")
    R = synth.random_graph(200000, 6.0, max_suffix=100, seed=23)  # ~22 MB of workspace > 16 MiB
    rc, _, _ = _run(noalloc, R, 0)
    assert rc == sg.SG_ERR_BUDGET
    assert b"scratch array" in sg.lib().sg_last_error()


def test_noalloc_hub_rows_first_match_plain_and_oracle():
    """Rows 0..19 above 1,024 entries: their per-entry minima start at the first bytes of the
    minima region, right after the row lists that name them."""
    noalloc, plain = _entry("sg_minplus_square_noalloc"), _entry("sg_minplus_square")
    R = hub_graph(1500, 20, 1100, 4, seed=31)
    for mode in (0, 1, 1, 0):
        rc, N, Nd = _run(noalloc, R, mode)
        assert rc == sg.SG_OK, sg.lib().sg_last_error()
        rc2, N2, Nd2 = _run(plain, R, mode)
        assert rc2 == sg.SG_OK
        assert np.array_equal(N, N2) and np.array_equal(Nd, Nd2)
        eN, eNd = oracle.minplus(R, mode)
        assert np.array_equal(N, eN) and np.array_equal(Nd, eNd)


_CHECKED_SCRIPT = r"""
import ctypes, sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import paper_2010_10055_gb300 as sg
sg.use_checked_build()
from tests.test_zz_no_alloc import hub_graph, ARGS
L = sg.lib()
out = []
for name in ("sg_minplus_square_noalloc", "sg_minplus_square"):
    fn = getattr(L, name); fn.restype = ctypes.c_int; fn.argtypes = ARGS
R = hub_graph(2000, 400, 1100, 4, seed=32)
D = sg.DeviceGraph.from_numpy(R)
res = {}
for mode in (0, 1):
    for name in ("sg_minplus_square_noalloc", "sg_minplus_square", "sg_minplus_square_noalloc"):
        N = torch.full((D.nnz,), 7, dtype=torch.int32, device="cuda")
        Nd = torch.full((D.nnz,), 9, dtype=torch.uint8, device="cuda")
        rc = getattr(L, name)(ctypes.byref(D.s), mode, ctypes.c_void_p(N.data_ptr()), ctypes.c_void_p(Nd.data_ptr()),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, L.sg_last_error()
        res.setdefault(mode, []).append((N.cpu().numpy(), Nd.cpu().numpy()))
torch.cuda.synchronize()
for mode, rs in res.items():
    for N, Nd in rs[1:]:
        assert np.array_equal(N, rs[0][0]) and np.array_equal(Nd, rs[0][1]), mode
print("ROWS", int((np.diff(R["row_ptr"]) > 1024).sum()), "SMS", torch.cuda.get_device_properties(0).multi_processor_count)
print("CHECK", sg.debug_check())
"""


def test_noalloc_many_hub_rows_checked_build():
    """400 rows above 1,024 entries from row 0 on -- more than the global-memory pass's 2 blocks
    per multiprocessor, so blocks take several of them in turn -- in the checked build, where
    every computed index is verified and a violation is recorded instead of touched: noalloc
    twice and the allocating form agree bit for bit, and nothing is out of bounds."""
    from paper_2010_10055_gb300 import build_lib
    build_lib.build(checked=True)
    p = subprocess.run([sys.executable, "-c", _CHECKED_SCRIPT, ROOT], capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    rows = [ln.split() for ln in p.stdout.splitlines() if ln.startswith("ROWS")][0]
    assert int(rows[1]) > 2 * int(rows[3])
    assert "CHECK None" in p.stdout, p.stdout[-2000:]
