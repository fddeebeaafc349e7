"""Seeded synthetic inputs (genomes, long reads, overlap graphs) for tests and the benchmark.

This package holds none of the method's arithmetic; both the CUDA path and the oracle read
what it draws.  ``build()`` compiles ``synth.c`` with gcc into ``libsynth.so`` beside it.

The five workload shapes stand in for the paper's PacBio CLR data sets (C. elegans 40x,
11 kbp mean, 13-15% error, 100 Mb; Table IV), which are not available here.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", _SO, src, "-lm"])
    return _SO


class _Reads(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("total", ctypes.c_int64),
                ("seq", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("start", ctypes.c_void_p), ("end", ctypes.c_void_p), ("strand", ctypes.c_void_p)]


class _Graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("suffix", ctypes.c_void_p), ("dir", ctypes.c_void_p)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        i64, u64, f64, i32, u32, vp = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_double,
                                        ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p)
        lib.synth_genome.restype = i64
        lib.synth_genome.argtypes = [vp, i64, u64, i32, f64, f64, f64, i64, i64, f64, f64]
        lib.synth_reads.restype = ctypes.c_int
        lib.synth_reads.argtypes = [vp, i64, f64, f64, f64, i64, f64, f64, f64, u64, i64,
                                    ctypes.POINTER(_Reads)]
        lib.synth_overlap_graph.restype = ctypes.c_int
        lib.synth_overlap_graph.argtypes = [vp, vp, vp, i64, i64, u32, u64, ctypes.POINTER(_Graph)]
        lib.synth_random_graph.restype = ctypes.c_int
        lib.synth_random_graph.argtypes = [i64, f64, f64, u32, u64, ctypes.POINTER(_Graph)]
        lib.synth_free.argtypes = [vp]
        _lib = lib
    return _lib


def _take(lib, ptr, n, dtype):
    """Copy a malloc'd C array into numpy and free it."""
    dtype = np.dtype(dtype)
    if n > 0 and ptr:
        out = np.frombuffer((ctypes.c_char * (n * dtype.itemsize)).from_address(ptr), dtype=dtype).copy()
    else:
        out = np.zeros(0, dtype=dtype)
    if ptr:
        lib.synth_free(ptr)
    return out


def genome(G: int, seed: int, n_families: int = 0, repeat_fraction: float = 0.0,
           copies=(1.0, 1.0), fam_len=(1, 1), divergence=(0.0, 0.0)) -> np.ndarray:
    """Uniform ACGT genome (ASCII uint8) with optional repeat families pasted in."""
    lib = _load()
    out = np.empty(int(G), dtype=np.uint8)
    rc = lib.synth_genome(out.ctypes.data, int(G), int(seed) & (2**64 - 1), int(n_families),
                          float(repeat_fraction), float(copies[0]), float(copies[1]),
                          int(fam_len[0]), int(fam_len[1]), float(divergence[0]), float(divergence[1]))
    if rc < 0:
        raise MemoryError("synth_genome: out of host memory")
    return out


def reads(genome_seq: np.ndarray, coverage: float, len_mean: float, len_sd: float, len_min: int,
          p_ins: float, p_del: float, p_sub: float, seed: int, max_reads: int = 0) -> dict:
    """Reads sampled from ``genome_seq``: dict(seq, offsets, start, end, strand)."""
    lib = _load()
    g = np.ascontiguousarray(genome_seq, dtype=np.uint8)
    r = _Reads()
    rc = lib.synth_reads(g.ctypes.data, int(g.size), float(coverage), float(len_mean), float(len_sd),
                         int(len_min), float(p_ins), float(p_del), float(p_sub),
                         int(seed) & (2**64 - 1), int(max_reads), ctypes.byref(r))
    if rc != 0:
        raise MemoryError("synth_reads: out of host memory")
    n = r.n
    return dict(seq=_take(lib, r.seq, r.total, np.uint8), offsets=_take(lib, r.offsets, n + 1, np.int64),
                start=_take(lib, r.start, n, np.int64), end=_take(lib, r.end, n, np.int64),
                strand=_take(lib, r.strand, n, np.uint8))


def _graph_out(lib, g: _Graph) -> dict:
    return dict(n=int(g.n), row_ptr=_take(lib, g.row_ptr, g.n + 1, np.int64),
                col=_take(lib, g.col, g.nnz, np.int32), suffix=_take(lib, g.suffix, g.nnz, np.uint32),
                dir=_take(lib, g.dir, g.nnz, np.uint8))


def overlap_graph(start, end, strand, min_overlap: int = 1, jitter: int = 0, seed: int = 0) -> dict:
    """Bidirected overlap graph R (CSR) from true read coordinates; see synth.c for the rule."""
    lib = _load()
    s = np.ascontiguousarray(start, dtype=np.int64)
    e = np.ascontiguousarray(end, dtype=np.int64)
    d = np.ascontiguousarray(strand, dtype=np.uint8)
    g = _Graph()
    if lib.synth_overlap_graph(s.ctypes.data, e.ctypes.data, d.ctypes.data, int(s.size),
                               int(min_overlap), int(jitter), int(seed), ctypes.byref(g)) != 0:
        raise MemoryError("synth_overlap_graph: out of host memory")
    return _graph_out(lib, g)


def random_graph(n: int, avg_deg: float, hub_frac: float = 0.0, max_suffix: int = 1000,
                 seed: int = 0) -> dict:
    """Random graph with random suffixes and dirs (CSR, cols ascending, no diagonal)."""
    lib = _load()
    g = _Graph()
    if lib.synth_random_graph(int(n), float(avg_deg), float(hub_frac), int(max_suffix), int(seed),
                              ctypes.byref(g)) != 0:
        raise MemoryError("synth_random_graph: out of host memory")
    return _graph_out(lib, g)


# ----------------------------------------------------------------------------- workloads
@dataclasses.dataclass
class Workload:
    """One synthetic read set and the parameters the three operations take."""
    name: str
    G: int
    coverage: float
    len_mean: float
    len_sd: float
    p_ins: float
    p_del: float
    p_sub: float
    k: int = 17
    lo: int = 2
    hi: int = 8
    min_shared: int = 2
    max_seeds: int = 2
    fuzz: int = 0
    min_overlap: int = 1
    n_families: int = 0
    repeat_fraction: float = 0.0
    copies: tuple = (1.0, 1.0)
    fam_len: tuple = (1, 1)
    divergence: tuple = (0.0, 0.0)
    seed: int = 2010

    def scaled(self, f: float) -> "Workload":
        """Same shape on a genome f times as long (repeat copies keep their density)."""
        w = dataclasses.replace(self, G=max(int(self.G * f), 20000))
        if self.n_families > 0:
            w.n_families = max(1, int(round(self.n_families * f)))
        return w


# Plain method, tiny: 50 kbp, 10x, mean 2 kbp / sd 0.5 kbp, 12% errors (6 ins / 4 del / 2 sub),
# k=17, reliable range [2, 8], >= 2 shared k-mers, TR on all true overlaps with fuzz 0.
TINY = Workload("tiny-50kbp-10x", G=50_000, coverage=10.0, len_mean=2000.0, len_sd=500.0,
                p_ins=0.06, p_del=0.04, p_sub=0.02, lo=2, hi=8, fuzz=0, min_overlap=1, seed=2010)
# Bacterial-scale: 5 Mbp with 10 repeat families x 5 copies (5-8 kbp, 1% divergence), 30x,
# mean 10 kbp / sd 4 kbp, 15% errors (3:2:1 ins:del:sub), range [2, 20], fuzz 1000.
BACTERIAL = Workload("bacterial-5Mbp-30x", G=5_000_000, coverage=30.0, len_mean=10000.0, len_sd=4000.0,
                     p_ins=0.075, p_del=0.05, p_sub=0.025, lo=2, hi=20, fuzz=1000, min_overlap=1000,
                     n_families=10, copies=(5.0, 5.0), fam_len=(5000, 8000), divergence=(0.01, 0.01),
                     seed=2011)
# C. elegans-shaped: 100 Mbp, 2% repeats (copy number 2-200 log-uniform, 1-10 kbp, 0.5-3%
# divergence), 40x, mean 10 kbp / sd 4 kbp, 15% errors, range [2, 30], fuzz 1000.
ELEGANS = Workload("elegans-100Mbp-40x", G=100_000_000, coverage=40.0, len_mean=10000.0, len_sd=4000.0,
                   p_ins=0.075, p_del=0.05, p_sub=0.025, lo=2, hi=30, fuzz=1000, min_overlap=1000,
                   repeat_fraction=0.02, copies=(2.0, 200.0), fam_len=(1000, 10000),
                   divergence=(0.005, 0.03), seed=2012)

WORKLOADS = {w.name: w for w in (TINY, BACTERIAL, ELEGANS)}


def make(w: Workload, with_graph: bool = True) -> dict:
    """Draw the genome, reads and (optionally) the overlap graph R of a workload."""
    g = genome(w.G, w.seed, w.n_families, w.repeat_fraction, w.copies, w.fam_len, w.divergence)
    r = reads(g, w.coverage, w.len_mean, w.len_sd, max(w.k + 1, 500), w.p_ins, w.p_del, w.p_sub,
              w.seed + 1)
    out = dict(workload=w, genome=g, **r)
    if with_graph:
        out["R"] = overlap_graph(r["start"], r["end"], r["strand"], w.min_overlap, 0, w.seed + 2)
    return out


# ------------------------------------------------------------------ batched / served job mixes
def _parallel(fn, args, workers: int):
    """fn over args in order; the generator's C calls release the GIL, so threads run in parallel."""
    if workers <= 1 or len(args) <= 1:
        return [fn(*a) for a in args]
    import concurrent.futures
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        return list(ex.map(lambda a: fn(*a), args))


def _default_workers() -> int:
    try:
        return max(1, min(16, len(os.sched_getaffinity(0))))
    except (AttributeError, OSError):
        return 1


def batched_sets(count: int = 512, g_lo: float = 20e3, g_hi: float = 2e6, seed: int = 2013,
                 workers: int | None = None) -> list:
    """Independent read sets of the batched workload: genome log-uniform in [g_lo, g_hi], coverage
    U[10, 40], mean read length U[2, 10] kbp (sd 0.4 x mean), errors U[12, 15] % split 3:2:1
    (ins:del:sub), k = 17, reliable range [2, max(8, round(0.75 x coverage))], R from true
    coordinates (overlaps >= 500 bp). Set b is seeded from (seed, b); the sets are drawn on
    `workers` host threads with the same result."""
    rng = np.random.default_rng(seed)
    params = []
    for b in range(count):
        G = int(np.exp(rng.uniform(np.log(g_lo), np.log(g_hi))))
        cov = float(rng.uniform(10, 40))
        mean = float(rng.uniform(2000, 10000))
        err = float(rng.uniform(0.12, 0.15))
        params.append((b, G, cov, mean, err))

    def one(b, G, cov, mean, err):
        g = genome(G, seed * 100003 + b)
        rd = reads(g, cov, mean, 0.4 * mean, 500, err / 2, err / 3, err / 6, seed * 100003 + b + 1)
        R = overlap_graph(rd["start"], rd["end"], rd["strand"], 500)
        return dict(seq=rd["seq"], offsets=rd["offsets"], lo=2, hi=max(8, int(round(0.75 * cov))), R=R, genome=G)

    return _parallel(one, params, _default_workers() if workers is None else workers)


def served_jobs(count: int = 500, rate: float = 200.0, g_min: float = 20e3, g_max: float = 20e6,
                alpha: float = 1.5, seed: int = 2014, workers: int | None = None) -> list:
    """Jobs of the served workload: Poisson arrivals at `rate` per second; genome size Pareto(alpha)
    from g_min, truncated at g_max; 30x, mean read length 10 kbp (sd 4 kbp), 15 % errors (3:2:1),
    range [2, 20], R from true coordinates (overlaps >= 500 bp). Each job has an arrival time.
    Drawn on `workers` host threads with the same result."""
    rng = np.random.default_rng(seed)
    t = 0.0
    params = []
    for b in range(count):
        t += float(rng.exponential(1.0 / rate))
        G = int(min(g_max, g_min * (1.0 - rng.uniform()) ** (-1.0 / alpha)))
        params.append((b, G, t))

    def one(b, G, t):
        g = genome(G, seed * 100003 + b)
        rd = reads(g, 30.0, 10000.0, 4000.0, 500, 0.075, 0.05, 0.025, seed * 100003 + b + 1)
        R = overlap_graph(rd["start"], rd["end"], rd["strand"], 500)
        return dict(seq=rd["seq"], offsets=rd["offsets"], lo=2, hi=20, R=R, genome=G, arrival=t)

    return _parallel(one, params, _default_workers() if workers is None else workers)
