"""The input generator: determinism, shapes, error model."""
import numpy as np

import synth


def test_deterministic():
    a = synth.make(synth.TINY)
    b = synth.make(synth.TINY)
    for key in ("genome", "seq", "offsets", "start", "end", "strand"):
        assert np.array_equal(a[key], b[key])
    for key in ("row_ptr", "col", "suffix", "dir"):
        assert np.array_equal(a["R"][key], b["R"][key])


def test_tiny_shape():
    d = synth.make(synth.TINY)
    n = d["offsets"].size - 1
    assert 200 < n < 320
    L = d["end"] - d["start"]
    assert abs(L.sum() / synth.TINY.G - 10.0) < 0.5
    assert set(np.unique(d["seq"]).tolist()) <= set(b"ACGT")
    # 6% insertions, 4% deletions: reads are ~2% longer than their templates
    assert 1.0 < np.diff(d["offsets"]).sum() / L.sum() < 1.04


def test_error_free_reads_match_genome():
    g = synth.genome(5000, 1)
    rd = synth.reads(g, 3.0, 300.0, 50.0, 20, 0.0, 0.0, 0.0, 2)
    comp = bytes.maketrans(b"ACGT", b"TGCA")
    for i in range(rd["start"].size):
        r = bytes(rd["seq"][rd["offsets"][i]:rd["offsets"][i + 1]])
        t = bytes(g[rd["start"][i]:rd["end"][i]])
        assert r == (t if rd["strand"][i] == 0 else t.translate(comp)[::-1])


def test_overlap_graph_rule():
    # contained pairs are not edges; R_ab, R_ba follow the coordinate rule
    R = synth.overlap_graph(np.array([0, 10, 20]), np.array([100, 50, 130]), np.array([0, 1, 0], np.uint8))
    ent = {}
    for i in range(3):
        for e in range(R["row_ptr"][i], R["row_ptr"][i + 1]):
            ent[(i, int(R["col"][e]))] = (int(R["suffix"][e]), int(R["dir"][e]))
    assert (0, 1) not in ent and (1, 0) not in ent          # [10,50) inside [0,100)
    assert ent[(0, 2)] == (30, 0) and ent[(2, 0)] == (20, 3)
    assert ent[(1, 2)] == (80, 2) and ent[(2, 1)] == (10, 2)
