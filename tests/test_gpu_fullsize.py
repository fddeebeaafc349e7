"""Parity at the benchmark's full size (the bacterial workload, default launch configuration, the
calls bench.py times), where the whole-matrix oracle is too slow for the k-mer stage and C:

- the transitive reduction is compared with the oracle element by element (it finishes in about
  a second at this size);
- sampled columns of At: the oracle's census of each column's code over all 153.5 M windows gives
  its frequency (must be in [lo, hi]) and its occurrences, whose lowest position per read must be
  At's row exactly;
- sampled rows of A: the read's own windows (oracle) and their census give the read's reliable
  k-mers, which must be A's row (columns by code rank, lowest position, strand) exactly;
- sampled rows of C: the oracle's single-row product on the same A and At;
- properties that hold at any size: codes strictly ascending, A and At transposes, C symmetric
  with no diagonal and counts >= t, S a subgraph of R.
"""
import numpy as np
import pytest

import oracle
import paper_2010_10055_gb300 as sg
import synth
from tests.gpu_util import assert_graph_equal, dev

pytestmark = pytest.mark.gpu

W = synth.BACTERIAL


@pytest.fixture(scope="module")
def full():
    d = synth.make(W)
    km = sg.build_kmer_matrix(dev(d["seq"], np.uint8), dev(d["offsets"], np.int64), W.k, W.lo, W.hi)
    C = sg.overlap_spgemm(km, W.min_shared, W.max_seeds)
    S, it = sg.transitive_reduce(sg.DeviceGraph.from_numpy(d["R"]), W.fuzz)
    return d, km.to_numpy(), C.to_numpy(), S.to_numpy(), it


@pytest.fixture(scope="module")
def census(full):
    """One census over all windows for the sampled columns' codes and the sampled reads' codes."""
    d, km, _, _, _ = full
    rng = np.random.default_rng(2011)
    m = km["At"]["n_rows"]
    cols = np.unique(np.concatenate([rng.choice(m, 3000, replace=False), [0, m - 1]]))
    n = km["A"]["n_rows"]
    reads = np.unique(np.concatenate([rng.choice(n, 60, replace=False), [0, n - 1]]))
    windows = {int(i): oracle.read_windows(d["seq"], d["offsets"], int(i), W.k) for i in reads}
    query = np.concatenate([km["codes"][cols]] + [w["code"] for w in windows.values()])
    c = oracle.kmer_census(d["seq"], d["offsets"], W.k, query, occ_cap=1 << 24)
    return cols, windows, c


def test_fullsize_transitive_reduction(full):
    d, _, _, S, it = full
    eS, eit = oracle.transitive_reduce(d["R"], W.fuzz)
    assert_graph_equal(S, eS)
    assert it == eit


def test_fullsize_sampled_at_rows(full, census):
    _, km, _, _, _ = full
    cols, _, c = census
    At = km["At"]
    q_of = np.searchsorted(c["codes"], km["codes"][cols])
    assert np.array_equal(c["codes"][q_of], km["codes"][cols])
    f = c["freq"][q_of]
    assert ((f >= W.lo) & (f <= W.hi)).all()
    want = set(q_of.tolist())
    first = {}
    for q, r, p, s in zip(c["occ_q"].tolist(), c["occ_read"].tolist(), c["occ_pos"].tolist(),
                          c["occ_strand"].tolist()):
        if q in want:
            first.setdefault(q, {}).setdefault(r, p | (s << 31))
    for j, q in zip(cols.tolist(), q_of.tolist()):
        a, b = At["row_ptr"][j], At["row_ptr"][j + 1]
        got = list(zip(At["col"][a:b].tolist(), At["val"][a:b].tolist()))
        assert got == sorted(first.get(q, {}).items()), j


def test_fullsize_sampled_a_rows(full, census):
    _, km, _, _, _ = full
    _, windows, c = census
    A = km["A"]
    for i, w in windows.items():
        qi = np.searchsorted(c["codes"], w["code"])
        f = c["freq"][qi]
        rel = (f >= W.lo) & (f <= W.hi)
        exp = {}
        for code, p, s in zip(w["code"][rel].tolist(), w["pos"][rel].tolist(), w["strand"][rel].tolist()):
            exp.setdefault(code, p | (s << 31))  # lowest position first
        a, b = A["row_ptr"][i], A["row_ptr"][i + 1]
        cols = A["col"][a:b]
        got = dict(zip(km["codes"][cols].tolist(), A["val"][a:b].tolist()))
        assert got == exp, i
        assert (np.diff(cols) > 0).all()


def test_fullsize_sampled_c_rows(full):
    _, km, C, _, _ = full
    rng = np.random.default_rng(2012)
    n = C["n"]
    for i in np.unique(np.concatenate([rng.choice(n, 200, replace=False), [0, n - 1]])).tolist():
        r = oracle.overlap_row(km["A"], km["At"], i, W.min_shared, W.max_seeds)
        a, b = C["row_ptr"][i], C["row_ptr"][i + 1]
        assert np.array_equal(C["col"][a:b], r["col"]), i
        assert np.array_equal(C["count"][a:b], r["count"]), i
        assert np.array_equal(C["seed_i"][:, a:b], r["seed_i"]), i
        assert np.array_equal(C["seed_k"][:, a:b], r["seed_k"]), i


def _entries(M, rows):
    r = np.repeat(np.arange(rows, dtype=np.int64), np.diff(M["row_ptr"]))
    return r, M["col"].astype(np.int64)


def test_fullsize_properties(full):
    d, km, C, S, _ = full
    assert (np.diff(km["codes"].astype(np.uint64)) > 0).all()
    A, At = km["A"], km["At"]
    ar, ac = _entries(A, A["n_rows"])
    tr, tc = _entries(At, At["n_rows"])
    o = np.lexsort((ar, ac))  # A's entries ordered by (col, row) = At's order
    assert np.array_equal(ac[o], tr) and np.array_equal(ar[o], tc) and np.array_equal(A["val"][o], At["val"])
    cr, cc = _entries(C, C["n"])
    assert (cr != cc).all() and (C["count"] >= W.min_shared).all()
    o = np.lexsort((cr, cc))  # the transpose's entries in row-major order
    assert np.array_equal(cc[o], cr) and np.array_equal(cr[o], cc) and np.array_equal(C["count"][o], C["count"])
    R = d["R"]
    rr, rc = _entries(R, R["n"])
    sr, sc = _entries(S, S["n"])
    key = lambda r, c: r * (R["n"] + 1) + c
    assert np.isin(key(sr, sc), key(rr, rc)).all()
