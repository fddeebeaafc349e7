"""Pins of the oracle's overlap product C = A A^T (Sec. IV-D): brute-force pairwise k-mer-set
intersection, the closed form for error-free reads of a repeat-free genome, and invariants."""
import numpy as np
import pytest

import oracle
import synth
from tests import brute


def _pairs(C):
    out = {}
    S = C["seed_i"].shape[0]
    for i in range(C["n"]):
        for e in range(C["row_ptr"][i], C["row_ptr"][i + 1]):
            seeds = [(int(C["seed_i"][s, e]), int(C["seed_k"][s, e])) for s in range(S)]
            out[(i, int(C["col"][e]))] = (int(C["count"][e]), seeds)
    return out


@pytest.mark.parametrize("k,lo,hi,t,S,seed", [(5, 2, 8, 2, 2, 1), (7, 1, 5, 1, 3, 2), (9, 2, 50, 3, 1, 3),
                                              (5, 2, 8, 2, 0, 4), (5, 1, 1000, 2, 8, 5)])
def test_overlap_brute_force(k, lo, hi, t, S, seed):
    g = synth.genome(500, seed)
    rd = synth.reads(g, 5.0, 80.0, 25.0, 1, 0.04, 0.03, 0.03, seed + 10)
    km = oracle.build_kmer_matrix(rd["seq"], rd["offsets"], k=k, lo=lo, hi=hi)
    C = oracle.overlap_spgemm(km["A"], km["At"], min_shared=t, max_seeds=S)
    reads = brute.reads_to_strings(rd["seq"], rd["offsets"])
    _, per_read = brute.kmer_matrix(reads, k, lo, hi)
    exp = brute.overlap_pairs(per_read, t, S)
    got = _pairs(C)
    assert set(got) == set(exp)
    for key, (cnt, seeds) in exp.items():
        gc, gs = got[key]
        assert gc == cnt, key
        assert gs[:len(seeds)] == seeds, key
        assert all(x == (oracle.INF, oracle.INF) for x in gs[len(seeds):]), key
    # rows list columns in ascending order
    for i in range(C["n"]):
        row = C["col"][C["row_ptr"][i]:C["row_ptr"][i + 1]]
        assert np.all(np.diff(row) > 0)


def _repeat_free_genome(G, k, seed):
    while True:
        g = synth.genome(G, seed)
        s = bytes(g).decode()
        seen = set()
        ok = True
        for p in range(G - k + 1):
            c, _ = brute.canonical(s[p:p + k])
            if c in seen:
                ok = False
                break
            seen.add(c)
        if ok:
            return g, s
        seed += 1000


def test_overlap_closed_form_error_free():
    """Error-free reads of a genome with no repeated canonical k-mer: C_ik exists iff the true
    intervals overlap by >= k + t - 1 bp, count = overlap - k + 1, and each seed is the same genome
    position seen from both reads, at the smallest canonical code of the shared region."""
    k, t, S = 11, 2, 2
    G = 3000
    g, gs = _repeat_free_genome(G, k, 77)
    rd = synth.reads(g, 8.0, 300.0, 80.0, 50, 0.0, 0.0, 0.0, 78)
    seq, off = rd["seq"], rd["offsets"]
    km = oracle.build_kmer_matrix(seq, off, k=k, lo=1, hi=1 << 30)
    C = _pairs(oracle.overlap_spgemm(km["A"], km["At"], min_shared=t, max_seeds=S))
    st, en, sd = rd["start"], rd["end"], rd["strand"]
    n = st.size

    def gpos(i, p):  # genome start of the k-mer at read position p
        return int(st[i] + p) if sd[i] == 0 else int(en[i] - p - k)

    expected = set()
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            ov = min(en[i], en[j]) - max(st[i], st[j])
            if ov - k + 1 >= t:
                expected.add((i, j))
                cnt, seeds = C[(i, j)]
                assert cnt == ov - k + 1
                lo_g = max(st[i], st[j])
                codes = sorted((brute.canonical(gs[q:q + k])[0], q) for q in range(lo_g, lo_g + ov - k + 1))
                for s in range(min(S, cnt)):
                    pi, pk = seeds[s]
                    rc = pk >> 31
                    assert gpos(i, pi) == gpos(j, pk & 0x7FFFFFFF) == codes[s][1]
                    assert rc == (sd[i] ^ sd[j])
    assert set(C) == expected


def test_overlap_symmetric_no_diagonal():
    w = synth.TINY
    d = synth.make(w, with_graph=False)
    km = oracle.build_kmer_matrix(d["seq"], d["offsets"], k=w.k, lo=w.lo, hi=w.hi)
    C = oracle.overlap_spgemm(km["A"], km["At"], min_shared=w.min_shared, max_seeds=w.max_seeds)
    P = _pairs(C)
    assert len(P) > 1000
    for (i, k), (cnt, seeds) in P.items():
        assert i != k and cnt >= w.min_shared
        cnt2, seeds2 = P[(k, i)]
        assert cnt2 == cnt
        for (a, b), (a2, b2) in zip(seeds, seeds2):
            if a == oracle.INF:
                assert (a2, b2) == (oracle.INF, oracle.INF)
            else:
                assert a2 == (b & 0x7FFFFFFF) and b2 == (a | (b & 0x80000000))


def test_overlap_invalid_args():
    km = oracle.build_kmer_matrix(np.frombuffer(b"ACGTACGTAC", np.uint8).copy(), np.array([0, 10]), k=3, lo=1)
    with pytest.raises(ValueError):
        oracle.overlap_spgemm(km["A"], km["At"], max_seeds=9)
    with pytest.raises(ValueError):
        oracle.overlap_spgemm(km["A"], km["At"], min_shared=0)
