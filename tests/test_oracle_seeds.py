"""Pins of the oracle's R from C's seeds (the overlap interval, containment, suffix and dir read
from C's first seed):

- closed form: for error-free reads of a genome with no repeated canonical k-mer, each seed is the
  same genome position seen from both reads, so the estimated intervals are the true ones and R
  must equal the graph built from the true coordinates (the generator's rule), entry for entry;
- the bidirected transpose rule holds for reads with errors: an edge and its mirror have
  d_ki = 2 (1 - in(d_ik)) + (1 - out(d_ik)), and R's pattern lies in C's.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.test_oracle_overlap import _repeat_free_genome


@pytest.mark.parametrize("k,G,mean,min_ov,seed", [(11, 3000, 300.0, 20, 77), (13, 6000, 700.0, 100, 91),
                                                  (17, 20000, 2000.0, 500, 105)])
def test_graph_from_seeds_closed_form_error_free(k, G, mean, min_ov, seed):
    g, _ = _repeat_free_genome(G, k, seed)
    rd = synth.reads(g, 10.0, mean, mean / 4, 2 * k, 0.0, 0.0, 0.0, seed + 1)
    km = oracle.build_kmer_matrix(rd["seq"], rd["offsets"], k=k, lo=1, hi=1 << 30)
    C = oracle.overlap_spgemm(km["A"], km["At"], min_shared=2, max_seeds=2)
    R = oracle.graph_from_seeds(C, rd["offsets"], k, min_ov)
    T = synth.overlap_graph(rd["start"], rd["end"], rd["strand"], max(min_ov, k + 1))
    assert R["col"].size > 50
    for key in ("row_ptr", "col", "suffix", "dir"):
        assert np.array_equal(R[key], T[key]), key


def test_graph_from_seeds_transpose_rule_with_errors():
    d = synth.make(synth.TINY)
    km = oracle.build_kmer_matrix(d["seq"], d["offsets"], 17, 2, 8)
    C = oracle.overlap_spgemm(km["A"], km["At"], 2, 2)
    R = oracle.graph_from_seeds(C, d["offsets"], 17, 200)
    n = R["n"]
    ent = {}
    for i in range(n):
        for x in range(R["row_ptr"][i], R["row_ptr"][i + 1]):
            ent[(i, int(R["col"][x]))] = (int(R["suffix"][x]), int(R["dir"][x]))
    cpat = {(i, int(C["col"][x])) for i in range(C["n"]) for x in range(C["row_ptr"][i], C["row_ptr"][i + 1])}
    assert len(ent) > 100 and set(ent) <= cpat
    mirrored = 0
    for (i, k), (s, dd) in ent.items():
        if (k, i) in ent:
            mirrored += 1
            assert ent[(k, i)][1] == 2 * (1 - (dd & 1)) + (1 - (dd >> 1)), (i, k)
    assert mirrored > 0.8 * len(ent)
