"""Helpers for the GPU parity tests: upload inputs, run the CUDA path, compare with the oracle."""
import numpy as np

import oracle
import paper_2010_10055_gb300 as sg


def dev(arr, dtype=None):
    import torch
    a = np.ascontiguousarray(arr if dtype is None else np.asarray(arr, dtype))
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def gpu_kmer(seq, offsets, k, lo, hi):
    km = sg.build_kmer_matrix(dev(seq, np.uint8), dev(offsets, np.int64), k=k, lo=lo, hi=hi)
    return km, km.to_numpy()


def assert_csr_equal(got, exp, what):
    assert got["n_rows"] == exp["n_rows"] and got["n_cols"] == exp["n_cols"], what
    for key in ("row_ptr", "col", "val"):
        assert np.array_equal(got[key], exp[key]), f"{what}.{key}"


def assert_kmer_equal(got, exp):
    assert np.array_equal(got["codes"], exp["codes"]), "codes"
    assert_csr_equal(got["A"], exp["A"], "A")
    assert_csr_equal(got["At"], exp["At"], "At")


def assert_overlap_equal(got, exp):
    for key in ("row_ptr", "col", "count", "seed_i", "seed_k"):
        assert np.array_equal(got[key], exp[key]), key


def assert_graph_equal(got, exp):
    for key in ("row_ptr", "col", "suffix", "dir"):
        assert np.array_equal(got[key], exp[key]), key


def first_mismatch(a, b):
    idx = np.nonzero(a != b)[0]
    return None if idx.size == 0 else (int(idx[0]), a[idx[0]], b[idx[0]])
