"""The allocation-free min-plus product (sg_minplus_square_noalloc).

Callers that cannot allocate device memory when they need N = R^2 -- a process held under a hard
GPU memory cap, code running while a memory pool is exhausted or being torn down, a host thread
that must not take the allocator's locks -- use this entry point; its workspace is a fixed device
array that the library reserves at load time. This file runs last so that a failure here comes
after every other test. It calls the C ABI directly and checks the result against
sg_minplus_square, bit for bit, on consecutive calls that reuse the shared workspace."""
import ctypes

import numpy as np
import pytest

import paper_2010_10055_gb300 as sg
import synth

pytestmark = pytest.mark.gpu

ARGS = [ctypes.POINTER(sg.GraphCsr), ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]


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
