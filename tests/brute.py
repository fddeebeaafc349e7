"""Brute-force checkers written independently of the oracle (pure Python, strings and dense
arrays). They follow the paper's definitions in a different representation so that a slip in
the oracle's index arithmetic shows up as a mismatch."""
from __future__ import annotations

import numpy as np

COMP = {"A": "T", "C": "G", "G": "C", "T": "A"}
INF = 0xFFFFFFFF


def revcomp(s: str) -> str:
    return "".join(COMP[c] for c in reversed(s))


def canonical(s: str):
    """(canonical string, strand): the lexicographically smaller of s and its reverse complement
    (Sec. II); strand 1 when the reverse complement is the smaller one."""
    r = revcomp(s)
    return (r, 1) if r < s else (s, 0)


def reads_to_strings(seq: np.ndarray, offsets: np.ndarray) -> list:
    b = bytes(np.asarray(seq, np.uint8))
    return [b[offsets[i]:offsets[i + 1]].decode("ascii") for i in range(len(offsets) - 1)]


def kmer_matrix(reads: list, k: int, lo: int, hi: int):
    """Returns (sorted reliable k-mer strings, per read dict kmer -> (lowest pos, strand))."""
    freq = {}
    per_read = []
    for r in reads:
        d = {}
        for p in range(len(r) - k + 1):
            w = r[p:p + k]
            if any(c not in "ACGT" for c in w):
                continue
            c, s = canonical(w)
            freq[c] = freq.get(c, 0) + 1
            if c not in d:
                d[c] = (p, s)
        per_read.append(d)
    reliable = sorted(c for c, f in freq.items() if lo <= f <= hi)
    rel = set(reliable)
    per_read = [{c: v for c, v in d.items() if c in rel} for d in per_read]
    return reliable, per_read


def encode(s: str) -> int:
    v = 0
    for c in s:
        v = v * 4 + "ACGT".index(c)
    return v


def overlap_pairs(per_read: list, min_shared: int, max_seeds: int) -> dict:
    """Pairwise set intersection: {(i, k): (count, [(seed_i, seed_k_with_rc_bit)...])}."""
    out = {}
    sets = [set(d) for d in per_read]
    for i in range(len(per_read)):
        for k in range(len(per_read)):
            if i == k:
                continue
            shared = sets[i] & sets[k]
            if len(shared) < min_shared:
                continue
            seeds = []
            for c in sorted(shared)[:max_seeds]:
                pi, si = per_read[i][c]
                pk, sk = per_read[k][c]
                seeds.append((pi, pk | ((si ^ sk) << 31)))
            out[(i, k)] = (len(shared), seeds)
    return out


def dense_tr(n: int, entries: dict, fuzz: int, per_end: bool = False, literal: bool = False):
    """Algorithm 1 on dense n x n arrays, every intermediate j tried for every pair (i, k).
    entries: {(i, k): (suffix, dir)}. per_end: an entry is bounded by the max over the entries of
    its row that use the same end of read i (dir >> 1) instead of the whole row's max.
    literal: the MinPlus entry is the smallest (sum, composite dir) pair over every valid walk,
    compared as a Python tuple, and the endpoint rule is applied to that one walk afterwards;
    otherwise only walks whose ends already agree with d_ik compete. Returns (surviving entries,
    rounds, N of the first reduction round, composite dir of that N's walk or d_ik)."""
    W = np.full((n, n), -1, np.int64)
    D = np.zeros((n, n), np.int64)
    for (i, k), (s, d) in entries.items():
        W[i, k] = s
        D[i, k] = d
    rounds = 0
    first_N = first_D = None
    while True:
        rounds += 1
        prev = int((W >= 0).sum())
        N = np.full((n, n), INF, np.int64)
        ND = D.copy()
        for i in range(n):
            for k in range(n):
                if W[i, k] < 0:
                    continue
                best = None
                for j in range(n):
                    if W[i, j] < 0 or W[j, k] < 0:
                        continue
                    # heads at j must point opposite ways: orientation of j seen from (i, j)
                    # equals orientation of j seen from (j, k)
                    if (D[i, j] & 1) != (D[j, k] >> 1):
                        continue
                    # the walk's end orientations: read i as in (i, j), read k as in (j, k)
                    ends = (int(D[i, j] >> 1), int(D[j, k] & 1))
                    if not literal and ends != (int(D[i, k] >> 1), int(D[i, k] & 1)):
                        continue
                    cand = (int(W[i, j] + W[j, k]), 2 * ends[0] + ends[1])
                    if best is None or cand < best:
                        best = cand
                if best is not None:
                    N[i, k] = best[0]
                    ND[i, k] = best[1]
        if first_N is None:
            first_N, first_D = N.copy(), ND.copy()
        if per_end:
            ends = D >> 1
            bound = np.zeros((n, n), np.int64)
            for e in (0, 1):
                m = np.where((W >= 0) & (ends == e), W, 0).max(axis=1) if n else np.zeros(0, np.int64)
                bound = np.where(ends == e, m[:, None], bound)
        else:
            rowmax = np.where(W >= 0, W, 0).max(axis=1) if n else np.zeros(0, np.int64)
            bound = rowmax[:, None]
        drop = (W >= 0) & (N != INF) & (ND == D) & ((bound + fuzz) >= N)
        W[drop] = -1
        if int((W >= 0).sum()) == prev:
            break
    surv = {(int(i), int(k)): (int(W[i, k]), int(D[i, k])) for i, k in zip(*np.nonzero(W >= 0))}
    return surv, rounds, first_N, first_D


def graph_to_dict(R: dict) -> dict:
    out = {}
    for i in range(R["n"]):
        for e in range(R["row_ptr"][i], R["row_ptr"][i + 1]):
            out[(i, int(R["col"][e]))] = (int(R["suffix"][e]), int(R["dir"][e]))
    return out


def dict_to_graph(n: int, entries: dict) -> dict:
    keys = sorted(entries)
    row_ptr = np.zeros(n + 1, np.int64)
    for i, _ in keys:
        row_ptr[i + 1] += 1
    row_ptr = np.cumsum(row_ptr)
    return dict(n=n, row_ptr=row_ptr.astype(np.int64),
                col=np.array([k for _, k in keys], np.int32),
                suffix=np.array([entries[x][0] for x in keys], np.uint32),
                dir=np.array([entries[x][1] for x in keys], np.uint8))
