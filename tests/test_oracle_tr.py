"""Pins of the oracle's transitive reduction (Algorithm 1 with the MinPlus semiring of
Algorithm 3, Sec. IV-E): the paper's worked example, the overhang example of Sec. II, layouts
drawn from a genome (which must reduce to a path), single-bit orientation corruptions (which
must not reduce), a dense all-intermediates brute force, and invariants."""
import itertools
import os

import numpy as np
import pytest

import oracle
import synth
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_worked_example():
    blocks, cur, scalars = {}, None, {}
    for line in open(os.path.join(GOLDEN, "tr_worked_example.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        if len(parts) == 2 and parts[0] in ("fuzz", "iterations"):
            scalars[parts[0]] = int(parts[1])
        elif len(parts) == 1:
            cur = parts[0]
            blocks[cur] = []
        else:
            blocks[cur].append([oracle.INF if x == "inf" else int(x) for x in parts])
    return blocks, scalars


def _dense_to_graph(M):
    n = len(M)
    ent = {(i, k): (M[i][k], 0) for i in range(n) for k in range(n) if M[i][k] != 0}
    return brute.dict_to_graph(n, ent)


def _graph_to_dense(G):
    M = [[0] * G["n"] for _ in range(G["n"])]
    for (i, k), (s, _) in brute.graph_to_dict(G).items():
        M[i][k] = s
    return M


def test_worked_example_sec4e():
    b, sc = _read_worked_example()
    R = _dense_to_graph(b["R"])
    N, Nd = oracle.minplus(R)
    for (i, k), e in zip(sorted(brute.graph_to_dict(R)), range(len(N))):
        assert N[e] == b["N_on_pattern_of_R"][i][k], (i, k)
    S, it = oracle.transitive_reduce(R, fuzz=sc["fuzz"])
    assert _graph_to_dense(S) == b["S"]
    assert it == sc["iterations"]
    # the v + x vector: row maxima of R plus fuzz
    rowmax = [max(r) for r in b["R"]]
    assert rowmax == b["rowmax"][0]
    assert [x + sc["fuzz"] if x else 0 for x in rowmax] == b["rowmax_plus_fuzz"][0]


def test_overhang_example_sec2():
    g = {}
    for line in open(os.path.join(GOLDEN, "overhang_sec2.txt")):
        if line.strip() and not line.startswith("#"):
            kk, v = line.split()
            g[kk] = v
    # v1 occupies genome [0, 5), v2 occupies [1, 7): check the layout, then the suffix rule
    genome = "TACGACC"
    assert genome[0:5] == g["v1"] and genome[1:7] == g["v2"]
    R = synth.overlap_graph(np.array([0, 1]), np.array([5, 7]), np.array([0, 0], np.uint8))
    assert brute.graph_to_dict(R)[(0, 1)] == (int(g["suffix_12"]), 0)


def _layout(starts, lens, strands):
    s = np.array(starts, np.int64)
    e = s + np.array(lens, np.int64)
    return synth.overlap_graph(s, e, np.array(strands, np.uint8))


@pytest.mark.parametrize("strands", list(itertools.product([0, 1], repeat=3)))
def test_three_read_layout_all_orientations(strands):
    """Reads a < b < c staggered on a genome, any strands: the edges a<->c are transitive."""
    R = _layout([0, 40, 80], [100, 100, 100], strands)
    ent = brute.graph_to_dict(R)
    assert len(ent) == 6
    S, it = oracle.transitive_reduce(R, fuzz=0)
    assert set(brute.graph_to_dict(S)) == {(0, 1), (1, 0), (1, 2), (2, 1)}
    assert it == 2


@pytest.mark.parametrize("edge,bit", list(itertools.product([(0, 1), (1, 2), (0, 2)], [0, 1])))
def test_corrupted_orientation_keeps_edge(edge, bit):
    """Flipping one orientation bit on the walk a->b->c or on a->c breaks either the walk's
    validity (heads at b) or an endpoint rule, so a->c must survive."""
    for strands in itertools.product([0, 1], repeat=3):
        R = _layout([0, 40, 80], [100, 100, 100], strands)
        ent = brute.graph_to_dict(R)
        s, d = ent[edge]
        ent[edge] = (s, d ^ (1 << bit))
        S, _ = oracle.transitive_reduce(brute.dict_to_graph(3, ent), fuzz=1000)
        assert (0, 2) in brute.graph_to_dict(S)


@pytest.mark.parametrize("seed,n,deg,fuzz", [(1, 12, 3.0, 0), (2, 20, 4.0, 50), (3, 30, 2.5, 200),
                                             (4, 25, 6.0, 10), (5, 16, 8.0, 1000)])
def test_dense_brute_force(seed, n, deg, fuzz):
    R = synth.random_graph(n, deg, hub_frac=0.1, max_suffix=300, seed=seed)
    ent = brute.graph_to_dict(R)
    surv, rounds, N1, _ = brute.dense_tr(n, ent, fuzz)
    N, _ = oracle.minplus(R)
    for e, (i, k) in enumerate(sorted(ent)):
        assert N[e] == N1[i, k]
    S, it = oracle.transitive_reduce(R, fuzz=fuzz)
    assert brute.graph_to_dict(S) == surv
    assert it == rounds


def test_jittered_layout_brute_force():
    w = synth.genome(3000, 5)
    rd = synth.reads(w, 6.0, 400.0, 150.0, 50, 0, 0, 0, 6)
    R = synth.overlap_graph(rd["start"], rd["end"], rd["strand"], 1, jitter=30, seed=7)
    ent = brute.graph_to_dict(R)
    surv, rounds, _, _ = brute.dense_tr(R["n"], ent, 20)
    S, it = oracle.transitive_reduce(R, fuzz=20)
    assert brute.graph_to_dict(S) == surv and it == rounds


def test_path_closed_form():
    """Equal-length reads (so no read contains another) from true coordinates: the string graph
    is exactly the edges between reads adjacent in start order, both directions, per connected
    stretch; one effective round and one no-change round."""
    rng = np.random.default_rng(3)
    n, L = 200, 1000
    starts = np.sort(rng.choice(np.arange(0, 60000), size=n, replace=False))
    strands = rng.integers(0, 2, n).astype(np.uint8)
    perm = rng.permutation(n)  # read ids not in genome order
    st = np.empty(n, np.int64); st[perm] = starts
    sd = np.empty(n, np.uint8); sd[perm] = strands
    R = synth.overlap_graph(st, st + L, sd)
    for fuzz in (0, 1000):
        S, it = oracle.transitive_reduce(R, fuzz=fuzz)
        got = set(brute.graph_to_dict(S))
        exp = set()
        for a in range(n - 1):
            if starts[a + 1] < starts[a] + L:
                exp |= {(int(perm[a]), int(perm[a + 1])), (int(perm[a + 1]), int(perm[a]))}
        assert got == exp
        assert it == (2 if len(brute.graph_to_dict(R)) > len(exp) else 1)


def test_subgraph_and_idempotent():
    R = synth.random_graph(300, 6.0, hub_frac=0.05, max_suffix=2000, seed=9)
    ent = brute.graph_to_dict(R)
    for mode in (oracle.DIRMATCH, oracle.LITERAL):
        S, it = oracle.transitive_reduce(R, fuzz=100, mode=mode)
        sent = brute.graph_to_dict(S)
        assert all(ent[key] == v for key, v in sent.items())
        S2, it2 = oracle.transitive_reduce(S, fuzz=100, mode=mode)
        assert brute.graph_to_dict(S2) == sent and it2 == 1


def test_literal_mode_removes_subset_of_dirmatch():
    # LITERAL looks at one minimising walk per entry, DIRMATCH at every walk with matching
    # endpoints, so on one round LITERAL can only remove entries DIRMATCH also removes.
    R = synth.random_graph(200, 8.0, max_suffix=500, seed=11)
    N0, _ = oracle.minplus(R, oracle.DIRMATCH)
    N1, D1 = oracle.minplus(R, oracle.LITERAL)
    lit = (N1 != oracle.INF) & (D1 == R["dir"])
    assert np.all(N0[lit] <= N1[lit])


def test_edge_cases_and_validation():
    empty = dict(n=0, row_ptr=np.zeros(1, np.int64), col=np.zeros(0, np.int32),
                 suffix=np.zeros(0, np.uint32), dir=np.zeros(0, np.uint8))
    S, it = oracle.transitive_reduce(empty)
    assert S["n"] == 0 and it == 1
    bad = brute.dict_to_graph(3, {(0, 0): (5, 0)})
    assert not oracle.validate_graph(bad)
    with pytest.raises(ValueError):
        oracle.transitive_reduce(bad)
    big = brute.dict_to_graph(3, {(0, 1): (1 << 30, 0)})
    with pytest.raises(ValueError):
        oracle.transitive_reduce(big)
    with pytest.raises(ValueError):
        oracle.transitive_reduce(brute.dict_to_graph(3, {(0, 1): (5, 0)}), fuzz=1 << 30)


# ---------------------------------------------------------------- per-end row maxima (mode bit 1)
@pytest.mark.parametrize("seed,n,deg,fuzz", [(1, 12, 3.0, 0), (2, 20, 4.0, 50), (3, 30, 2.5, 200),
                                             (4, 25, 6.0, 10), (5, 16, 8.0, 1000)])
def test_per_end_dense_brute_force(seed, n, deg, fuzz):
    R = synth.random_graph(n, deg, hub_frac=0.1, max_suffix=300, seed=seed)
    surv, rounds, _, _ = brute.dense_tr(n, brute.graph_to_dict(R), fuzz, per_end=True)
    S, it = oracle.transitive_reduce(R, fuzz=fuzz, mode=oracle.DIRMATCH | oracle.PER_END)
    assert brute.graph_to_dict(S) == surv
    assert it == rounds


def test_per_end_jittered_layout_brute_force():
    w = synth.genome(3000, 5)
    rd = synth.reads(w, 6.0, 400.0, 150.0, 50, 0, 0, 0, 6)
    R = synth.overlap_graph(rd["start"], rd["end"], rd["strand"], 1, jitter=30, seed=7)
    surv, rounds, _, _ = brute.dense_tr(R["n"], brute.graph_to_dict(R), 20, per_end=True)
    S, it = oracle.transitive_reduce(R, fuzz=20, mode=oracle.PER_END)
    assert brute.graph_to_dict(S) == surv and it == rounds


@pytest.mark.parametrize("strands", list(itertools.product([0, 1], repeat=3)))
def test_per_end_three_read_layout_all_orientations(strands):
    """A transitive edge uses the same end of its read as the walk's first edge, so the per-end
    bound still removes a <-> c in every orientation."""
    R = _layout([0, 40, 80], [100, 100, 100], strands)
    S, it = oracle.transitive_reduce(R, fuzz=0, mode=oracle.PER_END)
    assert set(brute.graph_to_dict(S)) == {(0, 1), (1, 0), (1, 2), (2, 1)}
    assert it == 2


def test_per_end_bound_is_the_end_max():
    """Read 0 has a long edge on one end (0 -> 3, suffix 5000) and a transitive triple on its
    other end (0 -> 1 -> 2 with suffixes 30 + 40 against 0 -> 2 with 50): the whole-row bound
    (5000) removes 0 -> 2; the per-end bound (max 50 on that end, fuzz 10 -> 60 < 70) keeps it."""
    ent = {(0, 1): (30, 0), (1, 2): (40, 0), (0, 2): (50, 0), (0, 3): (5000, 3)}
    R = brute.dict_to_graph(4, ent)
    whole, _ = oracle.transitive_reduce(R, fuzz=10)
    per, _ = oracle.transitive_reduce(R, fuzz=10, mode=oracle.PER_END)
    assert (0, 2) not in brute.graph_to_dict(whole)
    assert (0, 2) in brute.graph_to_dict(per)
    per20, _ = oracle.transitive_reduce(R, fuzz=20, mode=oracle.PER_END)  # 50 + 20 >= 70
    assert (0, 2) not in brute.graph_to_dict(per20)


def test_per_end_first_round_removes_subset_of_whole_row():
    """Each end's max is at most the row's max, so in the first round the per-end form removes a
    subset of what the whole-row form removes (graphs with no second round: every transitive
    entry goes in round one)."""
    for strands in itertools.product([0, 1], repeat=4):
        R = _layout([0, 30, 60, 90], [100, 100, 100, 100], strands)
        whole, itw = oracle.transitive_reduce(R, fuzz=0)
        per, itp = oracle.transitive_reduce(R, fuzz=0, mode=oracle.PER_END)
        assert set(brute.graph_to_dict(whole)) <= set(brute.graph_to_dict(per))
        assert itw == 2 and itp == 2
    R = synth.random_graph(300, 8.0, hub_frac=0.05, max_suffix=2000, seed=21)
    ent = set(brute.graph_to_dict(R))
    for sem in (oracle.DIRMATCH, oracle.LITERAL):
        per, _ = oracle.transitive_reduce(R, fuzz=100, mode=sem | oracle.PER_END)
        assert set(brute.graph_to_dict(per)) <= ent


# ------------------------------------------------------- LITERAL semiring reading (mode bit 0)
RANDOM_GRAPHS = [(1, 12, 3.0, 0), (2, 20, 4.0, 50), (3, 30, 2.5, 200), (4, 25, 6.0, 10), (5, 16, 8.0, 1000)]


@pytest.mark.parametrize("per_end", [False, True])
@pytest.mark.parametrize("seed,n,deg,fuzz", RANDOM_GRAPHS)
def test_literal_dense_brute_force(seed, n, deg, fuzz, per_end):
    """LITERAL (Algorithm 3 carrying one (sum, composite) minimum per entry, endpoint rule after)
    against the dense brute force that compares every valid walk as a tuple: N, its composite,
    S and the round count, with and without per-end bounds."""
    R = synth.random_graph(n, deg, hub_frac=0.1, max_suffix=300, seed=seed)
    ent = brute.graph_to_dict(R)
    surv, rounds, N1, D1 = brute.dense_tr(n, ent, fuzz, per_end=per_end, literal=True)
    N, Nd = oracle.minplus(R, oracle.LITERAL)
    for e, (i, k) in enumerate(sorted(ent)):
        assert N[e] == N1[i, k], (i, k)
        assert Nd[e] == D1[i, k], (i, k)
    mode = oracle.LITERAL | (oracle.PER_END if per_end else 0)
    S, it = oracle.transitive_reduce(R, fuzz=fuzz, mode=mode)
    assert brute.graph_to_dict(S) == surv
    assert it == rounds


@pytest.mark.parametrize("per_end", [False, True])
def test_literal_jittered_layout_brute_force(per_end):
    w = synth.genome(3000, 5)
    rd = synth.reads(w, 6.0, 400.0, 150.0, 50, 0, 0, 0, 6)
    R = synth.overlap_graph(rd["start"], rd["end"], rd["strand"], 1, jitter=30, seed=7)
    surv, rounds, _, _ = brute.dense_tr(R["n"], brute.graph_to_dict(R), 20, per_end=per_end, literal=True)
    mode = oracle.LITERAL | (oracle.PER_END if per_end else 0)
    S, it = oracle.transitive_reduce(R, fuzz=20, mode=mode)
    assert brute.graph_to_dict(S) == surv and it == rounds


def test_literal_keeps_edge_whose_min_walk_has_other_ends():
    """Two walks 0 -> 1 -> 3 (suffixes 10 + 20, ends forward/forward: composite 0) and
    0 -> 2 -> 3 (15 + 15, composite 3) tie at 30 under the entry 0 -> 3 (suffix 25, dir 3).
    LITERAL keeps the walk with the smaller composite (0), which differs from d_03, so 0 -> 3
    stays; DIRMATCH lets only the composite-3 walk compete and removes 0 -> 3 (25 + 10 >= 30)."""
    ent = {(0, 1): (10, 0), (1, 3): (20, 0), (0, 2): (15, 2), (2, 3): (15, 1), (0, 3): (25, 3)}
    R = brute.dict_to_graph(4, ent)
    e03 = sorted(ent).index((0, 3))
    N0, D0 = oracle.minplus(R, oracle.DIRMATCH)
    N1, D1 = oracle.minplus(R, oracle.LITERAL)
    assert (N0[e03], D0[e03]) == (30, 3)
    assert (N1[e03], D1[e03]) == (30, 0)
    dm, _ = oracle.transitive_reduce(R, fuzz=10)
    lit, _ = oracle.transitive_reduce(R, fuzz=10, mode=oracle.LITERAL)
    assert (0, 3) not in brute.graph_to_dict(dm)
    assert (0, 3) in brute.graph_to_dict(lit)
    # a strictly shorter walk with the right ends wins in both readings
    ent2 = dict(ent)
    ent2[(2, 3)] = (14, 1)
    lit2, _ = oracle.transitive_reduce(brute.dict_to_graph(4, ent2), fuzz=10, mode=oracle.LITERAL)
    assert (0, 3) not in brute.graph_to_dict(lit2)
