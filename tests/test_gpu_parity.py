"""Parity of the CUDA path (through the C ABI) with the oracle, bit for bit, on seeded inputs
that span several thread blocks, ragged tails and the degenerate cases."""
import numpy as np
import pytest

import oracle
import paper_2010_10055_gb300 as sg
import synth
from tests.brute import dict_to_graph
from tests.gpu_util import (assert_graph_equal, assert_kmer_equal, assert_overlap_equal, dev, gpu_kmer)

pytestmark = pytest.mark.gpu


# ------------------------------------------------------------------------------ A, At
# k = 17 packs (code, window, strand) into the sort key (the top two code bits as buckets); k = 23
# on this input fits that only with a bucket bit; k = 31 is too wide for any packing and sorts
# (key, value) pairs. test_kmer_matrix_sort_forms covers the candidate-index packing.
@pytest.mark.parametrize("k,lo,hi,seed", [(17, 2, 8, 1), (5, 2, 6, 2), (7, 1, 3, 3), (31, 2, 50, 4),
                                          (1, 1, 1 << 30, 5), (9, 3, 3, 6), (23, 2, 9, 7)])
def test_kmer_matrix_random(k, lo, hi, seed):
    rng = np.random.default_rng(seed)
    g = synth.genome(20000, seed)
    rd = synth.reads(g, 8.0, 700.0, 300.0, 1, 0.05, 0.04, 0.03, seed)
    seq = rd["seq"].copy()
    for p in rng.integers(0, seq.size, size=seq.size // 500):
        seq[p] = rng.choice(np.frombuffer(b"NnX-", np.uint8))
    exp = oracle.build_kmer_matrix(seq, rd["offsets"], k, lo, hi)
    _, got = gpu_kmer(seq, rd["offsets"], k, lo, hi)
    assert_kmer_equal(got, exp)


# (k, bucket bits allowed, genome): 10x reads of G bases hold 2^18 (20 kbp), 2^19 (40 kbp) or
# 2^20 (60 kbp) positions, so k = 23 needs 1, 2 or 3 bucket bits for (code, position, strand) to
# fit 64 bits; with none allowed it packs (code, candidate index); k = 31 sorts pairs.
@pytest.mark.parametrize("k,buckets,G", [(23, 3, 20000), (23, 3, 40000), (23, 3, 60000), (23, 0, 40000),
                                         (17, 3, 40000), (31, 3, 40000)])
def test_kmer_matrix_sort_forms(k, buckets, G):
    """Each packing of the candidate records, on a read set with ragged reads and N's."""
    g = synth.genome(G, 11)
    rd = synth.reads(g, 10.0, 900.0, 400.0, 1, 0.05, 0.04, 0.03, 12)
    seq = rd["seq"].copy()
    seq[::997] = ord("N")
    exp = oracle.build_kmer_matrix(seq, rd["offsets"], k, 2, 12)
    saved = sg.tunables()
    try:
        sg.tune("kmer_sort_buckets", buckets)
        for direct in (1, 0):  # segments from the sorted packed keys, or from unpacked arrays
            sg.tune("kmer_direct_seg", direct)
            _, got = gpu_kmer(seq, rd["offsets"], k, 2, 12)
            assert_kmer_equal(got, exp)
    finally:
        for name in ("kmer_sort_buckets", "kmer_direct_seg"):
            sg.tune(name, saved[name])


def test_kmer_matrix_edge_cases():
    # empty input
    _, got = gpu_kmer(np.zeros(0, np.uint8), np.array([0]), 17, 2, 8)
    assert got["codes"].size == 0 and got["A"]["row_ptr"].tolist() == [0]
    # empty reads, reads shorter than k, all-N read, one long read
    parts = [b"", b"ACG", b"N" * 40, b"", b"ACGT" * 3000, b"TTTTTTTTTTTTTTTTTTTTT", b""]
    seq = np.frombuffer(b"".join(parts), np.uint8).copy()
    off = np.cumsum([0] + [len(p) for p in parts])
    for k, lo, hi in ((17, 1, 100000), (3, 2, 5), (21, 2, 1 << 20)):
        exp = oracle.build_kmer_matrix(seq, off, k, lo, hi)
        _, got = gpu_kmer(seq, off, k, lo, hi)
        assert_kmer_equal(got, exp)


@pytest.mark.parametrize("shift", [1, 2, 3])
def test_kmer_matrix_unaligned_sequence(shift):
    """A sequence that starts off a 4-byte boundary (a view into a larger buffer) is staged byte
    by byte; the result is the same."""
    import torch
    g = synth.genome(30000, 40 + shift)
    rd = synth.reads(g, 6.0, 900.0, 300.0, 1, 0.04, 0.03, 0.02, 41 + shift)
    buf = torch.zeros(rd["seq"].size + 8, dtype=torch.uint8, device="cuda")
    buf[shift:shift + rd["seq"].size] = dev(rd["seq"], np.uint8)
    seq = buf[shift:shift + rd["seq"].size]
    assert seq.data_ptr() % 4 == shift
    got = sg.build_kmer_matrix(seq, dev(rd["offsets"], np.int64), k=17, lo=2, hi=8).to_numpy()
    assert_kmer_equal(got, oracle.build_kmer_matrix(rd["seq"], rd["offsets"], 17, 2, 8))


def test_kmer_matrix_invalid():
    seq = dev(np.frombuffer(b"ACGTACGTAC", np.uint8).copy())
    for off, k, lo, hi in (([0, 5, 10], 4, 1, 2), ([0, 5, 10], 3, 3, 2), ([0, 7, 5], 3, 1, 2),
                           ([1, 5, 10], 3, 1, 2), ([0, 5, 9], 3, 1, 2)):
        with pytest.raises(sg.SgError) as e:
            sg.build_kmer_matrix(seq, dev(off, np.int64), k=k, lo=lo, hi=hi)
        assert e.value.status == sg.SG_ERR_INVALID


def test_kmer_matrix_tiny_workload():
    w = synth.TINY
    d = synth.make(w, with_graph=False)
    exp = oracle.build_kmer_matrix(d["seq"], d["offsets"], w.k, w.lo, w.hi)
    _, got = gpu_kmer(d["seq"], d["offsets"], w.k, w.lo, w.hi)
    assert_kmer_equal(got, exp)


# ------------------------------------------------------------------------------ C
@pytest.mark.parametrize("t,S", [(2, 2), (1, 0), (3, 1), (1, 8), (2, 5)])
def test_overlap_tiny_workload(t, S):
    w = synth.TINY
    d = synth.make(w, with_graph=False)
    km, got_km = gpu_kmer(d["seq"], d["offsets"], w.k, w.lo, w.hi)
    exp_km = oracle.build_kmer_matrix(d["seq"], d["offsets"], w.k, w.lo, w.hi)
    assert_kmer_equal(got_km, exp_km)
    exp = oracle.overlap_spgemm(exp_km["A"], exp_km["At"], t, S)
    got = sg.overlap_spgemm(km, min_shared=t, max_seeds=S).to_numpy()
    assert_overlap_equal(got, exp)


def test_overlap_wide_rows_use_every_bin():
    # a repeat-rich genome with a high frequency ceiling makes rows of very different work,
    # including rows whose hash tables spill to the global-memory pool
    g = synth.genome(60000, 9, n_families=6, copies=(20.0, 60.0), fam_len=(300, 2000), divergence=(0.0, 0.01))
    rd = synth.reads(g, 25.0, 1500.0, 900.0, 1, 0.02, 0.02, 0.01, 10)
    k, lo, hi = 15, 2, 100000
    exp_km = oracle.build_kmer_matrix(rd["seq"], rd["offsets"], k, lo, hi)
    km, got_km = gpu_kmer(rd["seq"], rd["offsets"], k, lo, hi)
    assert_kmer_equal(got_km, exp_km)
    At = exp_km["At"]
    a = np.diff(At["row_ptr"])
    assert a.max() > 100
    for t, S in ((2, 2), (1, 3)):
        exp = oracle.overlap_spgemm(exp_km["A"], exp_km["At"], t, S)
        got = sg.overlap_spgemm(km, min_shared=t, max_seeds=S).to_numpy()
        assert_overlap_equal(got, exp)


def test_overlap_degenerate():
    # no reliable k-mer at all -> empty A, empty C
    seq = np.frombuffer(b"ACGTTGCAAC" * 3, np.uint8).copy()
    off = np.array([0, 10, 20, 30])
    km, _ = gpu_kmer(seq, off, 9, 100, 200)
    C = sg.overlap_spgemm(km).to_numpy()
    assert C["row_ptr"].tolist() == [0, 0, 0, 0] and C["col"].size == 0
    with pytest.raises(sg.SgError):
        sg.overlap_spgemm(km, max_seeds=9)


# ------------------------------------------------------------------------------ TR
def _tr_check(R, fuzz, mode=oracle.DIRMATCH):
    D = sg.DeviceGraph.from_numpy(R)
    N, Nd = sg.minplus_square(D, mode & 1)  # the product does not depend on the row-max form
    eN, eNd = oracle.minplus(R, mode & 1)
    assert np.array_equal(N.cpu().numpy().view(np.uint32), eN)
    assert np.array_equal(Nd.cpu().numpy(), eNd)
    S, it = sg.transitive_reduce(D, fuzz=fuzz, mode=mode)
    eS, eit = oracle.transitive_reduce(R, fuzz, mode)
    assert_graph_equal(S.to_numpy(), eS)
    assert it == eit


def test_tr_worked_example():
    R = dict_to_graph(4, {(1, 0): (30, 0), (2, 0): (80, 0), (2, 1): (30, 0), (3, 1): (80, 0), (3, 2): (30, 0)})
    _tr_check(R, 10)


@pytest.mark.parametrize("seed,n,deg,hub,fuzz,mode", [(1, 500, 6.0, 0.05, 100, 0), (2, 3000, 12.0, 0.02, 0, 0),
                                                      (3, 2000, 10.0, 0.1, 500, 1), (4, 800, 40.0, 0.0, 50, 1),
                                                      (5, 4000, 3.0, 0.0, 1000, 0), (6, 2000, 10.0, 0.05, 300, 2),
                                                      (7, 1500, 20.0, 0.02, 100, 3)])
def test_tr_random_graphs(seed, n, deg, hub, fuzz, mode):
    _tr_check(synth.random_graph(n, deg, hub_frac=hub, max_suffix=2000, seed=seed), fuzz, mode)


def test_tr_high_degree_rows_global_path():
    # hub rows with more entries than the shared-memory staging limit
    R = synth.random_graph(3000, 300.0, hub_frac=0.02, max_suffix=5000, seed=7)
    assert np.diff(R["row_ptr"]).max() > 1024
    _tr_check(R, 200, 0)
    _tr_check(R, 200, 1)
    _tr_check(R, 200, sg.DIRMATCH | sg.PER_END)


def test_tr_tiny_workload_and_layouts():
    d = synth.make(synth.TINY)
    _tr_check(d["R"], synth.TINY.fuzz)
    rd = synth.reads(synth.genome(100000, 3), 15.0, 3000.0, 1000.0, 500, 0, 0, 0, 4)
    R = synth.overlap_graph(rd["start"], rd["end"], rd["strand"], 1, jitter=40, seed=5)
    _tr_check(R, 30)
    _tr_check(R, 30, 1)


@pytest.mark.parametrize("graph,fuzz,mode", [("tiny", 0, 0), ("random", 500, 1), ("random", 100, 0)])
def test_tr_checkpoint_resume(graph, fuzz, mode):
    """Algorithm 1's loop state is R itself: stopping after r rounds and resuming from the
    intermediate graph gives the oracle's S, and the rounds of the pieces add up."""
    R = synth.make(synth.TINY)["R"] if graph == "tiny" else synth.random_graph(2000, 12.0, hub_frac=0.05,
                                                                                   max_suffix=2000, seed=9)
    eS, eit = oracle.transitive_reduce(R, fuzz, mode)
    assert eit >= 2
    for r in range(1, eit + 1):
        S1, r1, conv = sg.transitive_reduce_rounds(sg.DeviceGraph.from_numpy(R), fuzz, r, mode)
        assert r1 == min(r, eit)
        if conv:
            assert r1 == eit
            assert_graph_equal(S1.to_numpy(), eS)
            continue
        S2, it2 = sg.transitive_reduce(S1, fuzz, mode)
        assert_graph_equal(S2.to_numpy(), eS)
        assert r1 + it2 == eit


def test_tr_edge_cases():
    empty = dict(n=0, row_ptr=np.zeros(1, np.int64), col=np.zeros(0, np.int32), suffix=np.zeros(0, np.uint32),
                 dir=np.zeros(0, np.uint8))
    _tr_check(empty, 0)
    no_edges = dict(n=5, row_ptr=np.zeros(6, np.int64), col=np.zeros(0, np.int32), suffix=np.zeros(0, np.uint32),
                    dir=np.zeros(0, np.uint8))
    _tr_check(no_edges, 0)
    bad = dict_to_graph(3, {(0, 0): (5, 0)})
    with pytest.raises(sg.SgError) as e:
        sg.transitive_reduce(sg.DeviceGraph.from_numpy(bad))
    assert e.value.status == sg.SG_ERR_INVALID
    unsorted = dict(n=3, row_ptr=np.array([0, 2, 2, 2]), col=np.array([2, 1], np.int32),
                    suffix=np.array([1, 2], np.uint32), dir=np.array([0, 0], np.uint8))
    with pytest.raises(sg.SgError):
        sg.transitive_reduce(sg.DeviceGraph.from_numpy(unsorted))
    with pytest.raises(sg.SgError):
        sg.transitive_reduce(sg.DeviceGraph.from_numpy(dict_to_graph(3, {(0, 1): (5, 0)})), fuzz=1 << 30)


def test_injected_allocation_failure_is_reported_and_leaves_nothing():
    d = synth.make(synth.TINY, with_graph=False)
    seq, off = dev(d["seq"], np.uint8), dev(d["offsets"], np.int64)
    for nth in (1, 5, 12):
        sg.debug_fail_alloc_after(nth)
        try:
            with pytest.raises(sg.SgError) as e:
                sg.build_kmer_matrix(seq, off, 17, 2, 8)
            assert e.value.status == sg.SG_ERR_OOM
        finally:
            sg.debug_fail_alloc_after(0)
    km = sg.build_kmer_matrix(seq, off, 17, 2, 8)  # still works afterwards
    assert km.A.nnz > 0


# ------------------------------------------------------------------ host-buffer pipeline
def test_host_pipeline_matches_oracle():
    w = synth.TINY
    d = synth.make(w)
    ekm = oracle.build_kmer_matrix(d["seq"], d["offsets"], w.k, w.lo, w.hi)
    eC = oracle.overlap_spgemm(ekm["A"], ekm["At"], w.min_shared, w.max_seeds)
    eS, eit = oracle.transitive_reduce(d["R"], w.fuzz)
    a = np.diff(ekm["At"]["row_ptr"]).astype(np.int64)
    hp = sg.HostPipeline()
    for _ in range(2):  # the second call reuses the arena
        out = hp.run(d["seq"], d["offsets"], w, d["R"])
        assert_overlap_equal(out["C"], eC)
        assert_graph_equal(out["S"], eS)
        assert out["iterations"] == eit
        assert out["products"] == int((a * a).sum())
        assert out["m"] == ekm["codes"].size and out["nnz_a"] == ekm["A"]["col"].size
    # without R: only C comes back
    out = hp.run(d["seq"], d["offsets"], w)
    assert_overlap_equal(out["C"], eC) and "S" not in out
    hp.close()


# --------------------------------------------------------------------- R from C's seeds
@pytest.mark.parametrize("workload,scale,min_ov", [("tiny", 1.0, 200), ("bacterial", 0.02, 1000)])
def test_graph_from_seeds_matches_oracle_and_reduces(workload, scale, min_ov):
    w = synth.TINY if workload == "tiny" else synth.BACTERIAL.scaled(scale)
    d = synth.make(w, with_graph=False)
    ekm = oracle.build_kmer_matrix(d["seq"], d["offsets"], w.k, w.lo, w.hi)
    eC = oracle.overlap_spgemm(ekm["A"], ekm["At"], w.min_shared, w.max_seeds)
    eR = oracle.graph_from_seeds(eC, d["offsets"], w.k, min_ov)
    off = dev(d["offsets"], np.int64)
    km = sg.build_kmer_matrix(dev(d["seq"], np.uint8), off, w.k, w.lo, w.hi)
    C = sg.overlap_spgemm(km, w.min_shared, w.max_seeds)
    R = sg.overlap_graph_from_seeds(C, off, w.k, min_ov)
    assert_graph_equal(R.to_numpy(), eR)
    # reads -> A -> C -> R -> S without true coordinates
    S, it = sg.transitive_reduce(R, fuzz=w.fuzz)
    eS, eit = oracle.transitive_reduce(eR, w.fuzz)
    assert_graph_equal(S.to_numpy(), eS)
    assert it == eit


def test_graph_from_seeds_closed_form_error_free():
    from tests.test_oracle_overlap import _repeat_free_genome
    g, _ = _repeat_free_genome(20000, 17, 105)
    rd = synth.reads(g, 10.0, 2000.0, 500.0, 34, 0.0, 0.0, 0.0, 106)
    off = dev(rd["offsets"], np.int64)
    km = sg.build_kmer_matrix(dev(rd["seq"], np.uint8), off, 17, 1, 1 << 30)
    C = sg.overlap_spgemm(km, 2, 1)
    R = sg.overlap_graph_from_seeds(C, off, 17, 500).to_numpy()
    T = synth.overlap_graph(rd["start"], rd["end"], rd["strand"], 500)
    assert R["col"].size > 50
    assert_graph_equal(R, T)


def test_graph_from_seeds_invalid():
    d = synth.make(synth.TINY, with_graph=False)
    off = dev(d["offsets"], np.int64)
    km = sg.build_kmer_matrix(dev(d["seq"], np.uint8), off, 17, 2, 8)
    C0 = sg.overlap_spgemm(km, 2, 0)  # no seeds kept
    with pytest.raises(sg.SgError) as e:
        sg.overlap_graph_from_seeds(C0, off, 17, 100)
    assert e.value.status == sg.SG_ERR_INVALID
    C = sg.overlap_spgemm(km, 2, 2)
    with pytest.raises(sg.SgError):
        sg.overlap_graph_from_seeds(C, off, 16, 100)  # even k
