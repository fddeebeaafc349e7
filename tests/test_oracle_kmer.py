"""Pins of the oracle's k-mer matrix A (Sec. II canonical form, Sec. IV-C reliable range,
Sec. IV-D A_ij = position of k-mer j in read i) against the paper's printed example and a
pure-Python string brute force."""
import os

import numpy as np
import pytest

import oracle
import synth
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#") or not line.strip():
            continue
        key, val = line.split()
        out[key] = val
    return out


def _arr(s):
    return np.frombuffer(s.encode(), np.uint8).copy()


def test_canonical_example_sec2():
    g = _golden("canonical_sec2.txt")
    assert brute.revcomp(g["v"]) == g["revcomp"]
    # one read holding v, one holding its reverse complement: both windows map to the canonical
    # k-mer, on strand 0 and strand 1 respectively
    seq = _arr(g["v"] + g["revcomp"])
    out = oracle.build_kmer_matrix(seq, np.array([0, 5, 10]), k=5, lo=1, hi=100)
    assert out["codes"].tolist() == [brute.encode(g["canonical"])]
    assert out["A"]["row_ptr"].tolist() == [0, 1, 2]
    assert out["A"]["val"].tolist() == [0, 1 << 31]
    assert out["At"]["col"].tolist() == [0, 1]


def _check_against_brute(seq, offsets, k, lo, hi):
    out = oracle.build_kmer_matrix(seq, offsets, k=k, lo=lo, hi=hi)
    reads = brute.reads_to_strings(seq, offsets)
    reliable, per_read = brute.kmer_matrix(reads, k, lo, hi)
    assert out["codes"].tolist() == [brute.encode(c) for c in reliable]
    col_of = {c: j for j, c in enumerate(reliable)}
    A = out["A"]
    n = len(reads)
    assert A["n_rows"] == n and A["n_cols"] == len(reliable)
    for i in range(n):
        got = [(int(A["col"][e]), int(A["val"][e])) for e in range(A["row_ptr"][i], A["row_ptr"][i + 1])]
        exp = sorted((col_of[c], p | (s << 31)) for c, (p, s) in per_read[i].items())
        assert got == exp, f"row {i}"
    At = out["At"]
    for j in range(len(reliable)):
        got = [(int(At["col"][e]), int(At["val"][e])) for e in range(At["row_ptr"][j], At["row_ptr"][j + 1])]
        exp = [(i, per_read[i][reliable[j]][0] | (per_read[i][reliable[j]][1] << 31))
               for i in range(n) if reliable[j] in per_read[i]]
        assert got == exp, f"col {j}"
    return out


@pytest.mark.parametrize("k,lo,hi,seed", [(5, 2, 6, 1), (7, 1, 3, 2), (9, 2, 100, 3), (3, 1, 1000, 4)])
def test_kmer_matrix_brute_force(k, lo, hi, seed):
    rng = np.random.default_rng(seed)
    g = synth.genome(400, seed)
    rd = synth.reads(g, 6.0, 60.0, 20.0, 1, 0.05, 0.05, 0.05, seed)
    seq = rd["seq"].copy()
    # sprinkle non-ACGT characters: windows holding them are skipped
    for p in rng.integers(0, seq.size, size=max(1, seq.size // 200)):
        seq[p] = ord("N")
    _check_against_brute(seq, rd["offsets"], k, lo, hi)


def test_kmer_matrix_repeats_within_read():
    # a k-mer occurring twice in one read: A keeps the lowest position, freq counts both
    seq = _arr("ACGTTACGTT" + "GGGGG")
    out = _check_against_brute(seq, np.array([0, 10, 15]), 5, 2, 10)
    assert out["A"]["row_ptr"][-1] >= 1


def test_kmer_matrix_edge_cases():
    # empty input, reads shorter than k, a read of only N
    out = oracle.build_kmer_matrix(np.zeros(0, np.uint8), np.array([0]), k=17)
    assert out["codes"].size == 0 and out["A"]["row_ptr"].tolist() == [0]
    seq = _arr("ACG" + "NNNNNNNNNNNNNNNNNNNN" + "ACGTACGTACGTACGTACGTA")
    _check_against_brute(seq, np.array([0, 3, 23, 44]), 17, 1, 10)
    with pytest.raises(ValueError):
        oracle.build_kmer_matrix(seq, np.array([0, 3, 23, 44]), k=16)
    with pytest.raises(ValueError):
        oracle.build_kmer_matrix(seq, np.array([0, 3, 23, 44]), k=17, lo=5, hi=4)
