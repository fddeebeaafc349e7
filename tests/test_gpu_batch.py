"""The batched form: every set's slice of one sg_run_batch call equals the oracle run on that set
alone (A, At, codes, C, S and the number of reduction rounds), bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import paper_2010_10055_gb300 as sg
import synth
from tests.gpu_util import assert_csr_equal, assert_graph_equal, assert_overlap_equal

pytestmark = pytest.mark.gpu


def _sets(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        G = int(rng.integers(8000, 60000))
        g = synth.genome(G, seed * 100 + b)
        rd = synth.reads(g, float(rng.uniform(6, 20)), float(rng.uniform(600, 2500)), 300.0, 100,
                         0.05, 0.04, 0.02, seed * 100 + b + 7)
        R = synth.overlap_graph(rd["start"], rd["end"], rd["strand"], int(rng.integers(1, 400)))
        hi = int(max(4, round(0.75 * rng.uniform(6, 20))))
        out.append(dict(seq=rd["seq"], offsets=rd["offsets"], lo=2, hi=hi, R=R))
    return out


def _device(sets, with_r):
    items = []
    for b, x in enumerate(sets):
        it = dict(seq=torch.from_numpy(x["seq"]).cuda(), offsets=torch.from_numpy(x["offsets"]).cuda(),
                  lo=x["lo"], hi=x["hi"])
        if with_r[b]:
            it["R"] = sg.DeviceGraph.from_numpy(x["R"])
        items.append(it)
    return items


@pytest.mark.parametrize("seed,count,fuzz,S", [(1, 7, 200, 2), (2, 12, 0, 3)])
def test_batch_slices_match_oracle(seed, count, fuzz, S):
    sets = _sets(seed, count)
    # an empty set and a set without R in the mix
    sets.insert(2, dict(seq=np.zeros(0, np.uint8), offsets=np.zeros(1, np.int64), lo=2, hi=8,
                        R=dict(n=0, row_ptr=np.zeros(1, np.int64), col=np.zeros(0, np.int32),
                               suffix=np.zeros(0, np.uint32), dir=np.zeros(0, np.uint8))))
    with_r = [b != 4 for b in range(len(sets))]
    res = sg.run_batch(_device(sets, with_r), k=17, min_shared=2, max_seeds=S, fuzz=fuzz)
    for b, x in enumerate(sets):
        got = res.item(b)
        km = oracle.build_kmer_matrix(x["seq"], x["offsets"], 17, x["lo"], x["hi"])
        assert np.array_equal(got["codes"], km["codes"]), b
        assert_csr_equal(got["A"], km["A"], f"A[{b}]")
        assert_csr_equal(got["At"], km["At"], f"At[{b}]")
        assert_overlap_equal(got["C"], oracle.overlap_spgemm(km["A"], km["At"], 2, S))
        if with_r[b]:
            eS, eit = oracle.transitive_reduce(x["R"], fuzz)
            assert_graph_equal(got["S"], eS)
            assert got["iterations"] == eit, b
        else:
            assert got["S"]["col"].size == 0 and got["iterations"] == 0


def test_batch_rejects_out_of_set_columns():
    sets = _sets(3, 2)
    bad = dict(sets[1]["R"])
    bad["col"] = bad["col"].copy()
    bad["col"][0] = bad["n"] + 5  # points into another set of the union
    sets[1]["R"] = bad
    with pytest.raises(sg.SgError) as e:
        sg.run_batch(_device(sets, [True, True]), k=17)
    assert e.value.status == sg.SG_ERR_INVALID


@pytest.mark.parametrize("cfg", [{"batch_group_kb": 1200, "batch_alone_kb": 700},
                                 {"batch_group_kb": 1200, "batch_alone_kb": 0},
                                 {"batch_group_kb": 100000, "batch_alone_kb": 500}],
                         ids=["groups+alone", "groups", "alone"])
def test_batch_in_groups_matches_oracle(cfg):
    """The batch split into several unions (and items that run on their own), their results moved
    into one batch result: every slice still equals the oracle on its set alone. The first two
    sets have no R, so a group without any R sits beside groups with one."""
    sets = _sets(4, 10)
    with_r = [b >= 2 for b in range(len(sets))]
    saved = sg.tunables()
    try:
        for k, v in cfg.items():
            sg.tune(k, v)
        res = sg.run_batch(_device(sets, with_r), k=17, min_shared=2, max_seeds=2, fuzz=150)
    finally:
        for k, v in saved.items():
            sg.tune(k, v)
    for b, x in enumerate(sets):
        got = res.item(b)
        km = oracle.build_kmer_matrix(x["seq"], x["offsets"], 17, x["lo"], x["hi"])
        assert np.array_equal(got["codes"], km["codes"]), b
        assert_csr_equal(got["A"], km["A"], f"A[{b}]")
        assert_csr_equal(got["At"], km["At"], f"At[{b}]")
        assert_overlap_equal(got["C"], oracle.overlap_spgemm(km["A"], km["At"], 2, 2))
        if with_r[b]:
            eS, eit = oracle.transitive_reduce(x["R"], 150)
            assert_graph_equal(got["S"], eS)
            assert got["iterations"] == eit, b
        else:
            assert got["S"]["col"].size == 0 and got["iterations"] == 0


def test_batch_at_stated_sizes_equals_each_set_alone():
    """Sets drawn from the batched workload's own distribution (genomes log-uniform 20 kbp - 2 Mbp,
    coverage 10-40x), the largest of them included, under the default planner: every slice of the
    batch equals the three calls on that set alone on the GPU, bit for bit (the plain calls are
    the ones the oracle pins elsewhere), and the smallest sets also equal the oracle."""
    sets = synth.batched_sets(512, 20e3, 2e6)
    order = np.argsort([x["seq"].size for x in sets])
    pick = sorted(set(order[:8].tolist()) | set(order[-4:].tolist()) | set(order[250:262].tolist()))
    sub = [sets[b] for b in pick]
    items = _device(sub, [True] * len(sub))
    res = sg.run_batch(items, k=17, min_shared=2, max_seeds=2, fuzz=1000)
    for b, (x, it) in enumerate(zip(sub, items)):
        got = res.item(b)
        km = sg.build_kmer_matrix(it["seq"], it["offsets"], 17, x["lo"], x["hi"])
        kmn = km.to_numpy()
        assert np.array_equal(got["codes"], kmn["codes"]), b
        assert_csr_equal(got["A"], kmn["A"], f"A[{b}]")
        assert_csr_equal(got["At"], kmn["At"], f"At[{b}]")
        assert_overlap_equal(got["C"], sg.overlap_spgemm(km, 2, 2).to_numpy())
        S, it_ = sg.transitive_reduce(it["R"], 1000)
        assert_graph_equal(got["S"], S.to_numpy())
        assert got["iterations"] == it_, b
        if x["seq"].size < 400_000:
            ekm = oracle.build_kmer_matrix(x["seq"], x["offsets"], 17, x["lo"], x["hi"])
            assert_overlap_equal(got["C"], oracle.overlap_spgemm(ekm["A"], ekm["At"], 2, 2))
