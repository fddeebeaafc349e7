"""Pins of the oracle's single-output functions (k-mer census, a read's windows, one row of C),
used by the full-size sampled parity checks: each is checked against pure-Python brute force
(strings) and against the whole-matrix oracle on small inputs."""
import numpy as np

import oracle
import synth
from tests import brute


def _small(seed=3):
    g = synth.genome(6000, seed)
    rd = synth.reads(g, 8.0, 600.0, 200.0, 1, 0.05, 0.04, 0.03, seed + 1)
    seq = rd["seq"].copy()
    rng = np.random.default_rng(seed)
    for p in rng.integers(0, seq.size, size=seq.size // 400):
        seq[p] = ord("N")
    return seq, rd["offsets"]


def test_census_frequencies_match_brute_force():
    seq, off = _small()
    reads = brute.reads_to_strings(seq, off)
    freq = {}
    for r in reads:
        for p in range(len(r) - 9 + 1):
            w = r[p:p + 9]
            if all(c in "ACGT" for c in w):
                c, _ = brute.canonical(w)
                freq[c] = freq.get(c, 0) + 1
    present = sorted(freq)
    rng = np.random.default_rng(1)
    pick = [present[i] for i in rng.choice(len(present), 300, replace=False)]
    absent = [brute.canonical("".join(rng.choice(list("ACGT"), 9)))[0] for _ in range(50)]
    query = [brute.encode(s) for s in pick + absent]
    c = oracle.kmer_census(seq, off, 9, query)
    got = {int(q): int(f) for q, f in zip(c["codes"], c["freq"])}
    for s in pick + absent:
        assert got[brute.encode(s)] == freq.get(s, 0), s


def test_census_occurrences_reproduce_at_rows():
    d = synth.make(synth.TINY)
    km = oracle.build_kmer_matrix(d["seq"], d["offsets"], 17, 2, 8)
    c = oracle.kmer_census(d["seq"], d["offsets"], 17, km["codes"])
    assert np.array_equal(c["codes"], km["codes"])
    assert ((c["freq"] >= 2) & (c["freq"] <= 8)).all()
    At = km["At"]
    # lowest position of each (k-mer, read): occurrences come in scan order
    first = {}
    for q, r, p, s in zip(c["occ_q"].tolist(), c["occ_read"].tolist(), c["occ_pos"].tolist(),
                          c["occ_strand"].tolist()):
        first.setdefault(q, {}).setdefault(r, p | (s << 31))
    for j in range(At["n_rows"]):
        rows = At["col"][At["row_ptr"][j]:At["row_ptr"][j + 1]]
        vals = At["val"][At["row_ptr"][j]:At["row_ptr"][j + 1]]
        exp = sorted(first.get(j, {}).items())
        assert list(zip(rows.tolist(), vals.tolist())) == exp, j


def test_read_windows_match_brute_force():
    seq, off = _small(5)
    reads = brute.reads_to_strings(seq, off)
    for i in (0, 3, len(reads) - 1):
        w = oracle.read_windows(seq, off, i, 11)
        exp = [(brute.encode(brute.canonical(reads[i][p:p + 11])[0]), p, brute.canonical(reads[i][p:p + 11])[1])
               for p in range(len(reads[i]) - 10) if all(ch in "ACGT" for ch in reads[i][p:p + 11])]
        assert list(zip(w["code"].tolist(), w["pos"].tolist(), w["strand"].tolist())) == exp


def test_overlap_row_matches_whole_product():
    d = synth.make(synth.TINY)
    km = oracle.build_kmer_matrix(d["seq"], d["offsets"], 17, 2, 8)
    for t, S in ((2, 2), (1, 3)):
        C = oracle.overlap_spgemm(km["A"], km["At"], t, S)
        for i in range(C["n"]):
            r = oracle.overlap_row(km["A"], km["At"], i, t, S)
            a, b = C["row_ptr"][i], C["row_ptr"][i + 1]
            assert np.array_equal(r["col"], C["col"][a:b]), i
            assert np.array_equal(r["count"], C["count"][a:b]), i
            assert np.array_equal(r["seed_i"], C["seed_i"][:, a:b]), i
            assert np.array_equal(r["seed_k"], C["seed_k"][:, a:b]), i
