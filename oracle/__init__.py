"""ORACLE -- test infrastructure, not part of the product.

Plain CPU definitions (``sgo.c``) of the three operations of the overlap-and-layout hot path of
diBELLA 2D (arXiv 2010.10055): the reads-by-k-mers matrix A (Sec. II, IV-C, IV-D), the overlap
product C = A A^T (Sec. IV-D) and the transitive reduction (Algorithms 1 and 3, Sec. IV-E).
Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline / reference leg
may import this package. It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsgo.so")
_lib = None

OK, INVALID, OOM = 0, 1, 2
INF = 0xFFFFFFFF
DIRMATCH, LITERAL = 0, 1
PER_END = 2  # mode flag: per-read-end row maxima in the reduction (or-ed with the semiring)


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "sgo.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", _SO, src])
    return _SO


class _Csr(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class _Overlap(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("max_seeds", ctypes.c_int32),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("count", ctypes.c_void_p),
                ("seed_i", ctypes.c_void_p), ("seed_k", ctypes.c_void_p)]


class _Graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("suffix", ctypes.c_void_p), ("dir", ctypes.c_void_p)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        vp, i64, i32, u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
        lib.sgo_build_kmer_matrix.restype = ctypes.c_int
        lib.sgo_build_kmer_matrix.argtypes = [vp, vp, i64, i32, u32, u32, ctypes.POINTER(_Csr),
                                              ctypes.POINTER(_Csr), ctypes.POINTER(vp),
                                              ctypes.POINTER(i64)]
        lib.sgo_overlap_spgemm.restype = ctypes.c_int
        lib.sgo_overlap_spgemm.argtypes = [ctypes.POINTER(_Csr), ctypes.POINTER(_Csr), u32, i32,
                                           ctypes.POINTER(_Overlap)]
        lib.sgo_minplus.restype = ctypes.c_int
        lib.sgo_minplus.argtypes = [ctypes.POINTER(_Graph), i32, vp, vp]
        lib.sgo_validate_graph.restype = ctypes.c_int
        lib.sgo_validate_graph.argtypes = [ctypes.POINTER(_Graph)]
        lib.sgo_transitive_reduce.restype = ctypes.c_int
        lib.sgo_transitive_reduce.argtypes = [ctypes.POINTER(_Graph), u32, i32, ctypes.POINTER(_Graph),
                                              ctypes.POINTER(i32)]
        lib.sgo_kmer_census.restype = ctypes.c_int
        lib.sgo_kmer_census.argtypes = [vp, vp, i64, i32, vp, i64, vp, i64, vp, vp, vp, vp, ctypes.POINTER(i64)]
        lib.sgo_read_windows.restype = ctypes.c_int
        lib.sgo_read_windows.argtypes = [vp, vp, i64, i32, i64, vp, vp, vp, ctypes.POINTER(i64)]
        lib.sgo_overlap_row.restype = ctypes.c_int
        lib.sgo_overlap_row.argtypes = [ctypes.POINTER(_Csr), ctypes.POINTER(_Csr), i64, u32, i32, vp, vp, vp, vp,
                                        ctypes.POINTER(i64)]
        lib.sgo_graph_from_seeds.restype = ctypes.c_int
        lib.sgo_graph_from_seeds.argtypes = [ctypes.POINTER(_Overlap), vp, i32, i64, ctypes.POINTER(_Graph)]
        lib.sgo_free.argtypes = [vp]
        _lib = lib
    return _lib


def _take(lib, ptr, n, dtype):
    dtype = np.dtype(dtype)
    if n > 0 and ptr:
        out = np.frombuffer((ctypes.c_char * (n * dtype.itemsize)).from_address(ptr), dtype=dtype).copy()
    else:
        out = np.zeros(0, dtype=dtype)
    if ptr:
        lib.sgo_free(ptr)
    return out


def _check(rc, what):
    if rc == INVALID:
        raise ValueError(f"oracle {what}: invalid argument")
    if rc != OK:
        raise OracleError(f"oracle {what}: status {rc}")


def _csr_in(d) -> tuple:
    arrs = (np.ascontiguousarray(d["row_ptr"], np.int64), np.ascontiguousarray(d["col"], np.int32),
            np.ascontiguousarray(d["val"], np.uint32))
    c = _Csr(int(d["n_rows"]), int(d["n_cols"]), int(arrs[1].size), arrs[0].ctypes.data,
             arrs[1].ctypes.data, arrs[2].ctypes.data)
    return c, arrs


def _graph_in(R) -> tuple:
    arrs = (np.ascontiguousarray(R["row_ptr"], np.int64), np.ascontiguousarray(R["col"], np.int32),
            np.ascontiguousarray(R["suffix"], np.uint32), np.ascontiguousarray(R["dir"], np.uint8))
    g = _Graph(int(R["n"]), int(arrs[1].size), arrs[0].ctypes.data, arrs[1].ctypes.data,
               arrs[2].ctypes.data, arrs[3].ctypes.data)
    return g, arrs


def build_kmer_matrix(seq, offsets, k: int = 17, lo: int = 2, hi: int = 8) -> dict:
    """A, At (CSR dicts: n_rows, n_cols, row_ptr, col, val) and the column codes."""
    lib = _load()
    s = np.ascontiguousarray(seq, np.uint8)
    o = np.ascontiguousarray(offsets, np.int64)
    A, At, codes, m = _Csr(), _Csr(), ctypes.c_void_p(), ctypes.c_int64()
    _check(lib.sgo_build_kmer_matrix(s.ctypes.data if s.size else None, o.ctypes.data, int(o.size - 1),
                                     int(k), int(lo), int(hi), ctypes.byref(A), ctypes.byref(At),
                                     ctypes.byref(codes), ctypes.byref(m)), "build_kmer_matrix")

    def out(c):
        return dict(n_rows=int(c.n_rows), n_cols=int(c.n_cols),
                    row_ptr=_take(lib, c.row_ptr, c.n_rows + 1, np.int64),
                    col=_take(lib, c.col, c.nnz, np.int32), val=_take(lib, c.val, c.nnz, np.uint32))
    return dict(A=out(A), At=out(At), codes=_take(lib, codes.value, m.value, np.uint64))


def overlap_spgemm(A: dict, At: dict, min_shared: int = 2, max_seeds: int = 2) -> dict:
    """C = A At over the overlap semiring: dict(n, row_ptr, col, count, seed_i, seed_k [S, nnz])."""
    lib = _load()
    a, keep_a = _csr_in(A)
    t, keep_t = _csr_in(At)
    C = _Overlap()
    _check(lib.sgo_overlap_spgemm(ctypes.byref(a), ctypes.byref(t), int(min_shared), int(max_seeds),
                                  ctypes.byref(C)), "overlap_spgemm")
    nnz, S = int(C.nnz), int(C.max_seeds)
    return dict(n=int(C.n), row_ptr=_take(lib, C.row_ptr, C.n + 1, np.int64),
                col=_take(lib, C.col, nnz, np.int32), count=_take(lib, C.count, nnz, np.uint32),
                seed_i=_take(lib, C.seed_i, nnz * S, np.uint32).reshape(S, nnz),
                seed_k=_take(lib, C.seed_k, nnz * S, np.uint32).reshape(S, nnz))


def validate_graph(R: dict) -> bool:
    lib = _load()
    g, keep = _graph_in(R)
    return lib.sgo_validate_graph(ctypes.byref(g)) == OK


def minplus(R: dict, mode: int = DIRMATCH) -> tuple:
    """N = R^2 (Algorithm 3) on the pattern of R: (N uint32 with INF = 0xFFFFFFFF, Ndir uint8)."""
    lib = _load()
    g, keep = _graph_in(R)
    nnz = int(g.nnz)
    N = np.empty(max(nnz, 1), np.uint32)
    Nd = np.empty(max(nnz, 1), np.uint8)
    _check(lib.sgo_minplus(ctypes.byref(g), int(mode), N.ctypes.data, Nd.ctypes.data), "minplus")
    return N[:nnz].copy(), Nd[:nnz].copy()


def transitive_reduce(R: dict, fuzz: int = 0, mode: int = DIRMATCH) -> tuple:
    """Algorithm 1: (S as a graph dict, number of rounds including the final no-change round)."""
    lib = _load()
    g, keep = _graph_in(R)
    S, it = _Graph(), ctypes.c_int32()
    _check(lib.sgo_transitive_reduce(ctypes.byref(g), int(fuzz), int(mode), ctypes.byref(S),
                                     ctypes.byref(it)), "transitive_reduce")
    nnz = int(S.nnz)
    return (dict(n=int(S.n), row_ptr=_take(lib, S.row_ptr, S.n + 1, np.int64),
                 col=_take(lib, S.col, nnz, np.int32), suffix=_take(lib, S.suffix, nnz, np.uint32),
                 dir=_take(lib, S.dir, nnz, np.uint8)), int(it.value))


def kmer_census(seq, offsets, k: int, codes, occ_cap: int = 1 << 22) -> dict:
    """Frequency of each canonical code in `codes` over all windows of all reads, and up to occ_cap
    occurrences (q = index into the sorted unique codes, read, pos, strand) in scan order.
    Returns dict(codes=sorted unique codes, freq, occ_q, occ_read, occ_pos, occ_strand)."""
    lib = _load()
    s = np.ascontiguousarray(seq, np.uint8)
    o = np.ascontiguousarray(offsets, np.int64)
    q = np.unique(np.asarray(codes, np.uint64))
    freq = np.zeros(max(q.size, 1), np.uint64)
    oq = np.zeros(occ_cap, np.int64)
    orr = np.zeros(occ_cap, np.int32)
    op = np.zeros(occ_cap, np.uint32)
    ost = np.zeros(occ_cap, np.uint32)
    nocc = ctypes.c_int64()
    _check(lib.sgo_kmer_census(s.ctypes.data, o.ctypes.data, o.size - 1, int(k), q.ctypes.data, q.size,
                               freq.ctypes.data, occ_cap, oq.ctypes.data, orr.ctypes.data, op.ctypes.data,
                               ost.ctypes.data, ctypes.byref(nocc)), "kmer_census")
    c = int(nocc.value)
    return dict(codes=q, freq=freq[:q.size], occ_q=oq[:c], occ_read=orr[:c], occ_pos=op[:c], occ_strand=ost[:c])


def read_windows(seq, offsets, i: int, k: int) -> dict:
    """Every valid window of read i: dict(code, pos, strand) by position."""
    lib = _load()
    s = np.ascontiguousarray(seq, np.uint8)
    o = np.ascontiguousarray(offsets, np.int64)
    cap = max(int(o[i + 1] - o[i]), 1)
    code = np.zeros(cap, np.uint64)
    pos = np.zeros(cap, np.uint32)
    st = np.zeros(cap, np.uint32)
    cnt = ctypes.c_int64()
    _check(lib.sgo_read_windows(s.ctypes.data, o.ctypes.data, int(i), int(k), cap, code.ctypes.data,
                                pos.ctypes.data, st.ctypes.data, ctypes.byref(cnt)), "read_windows")
    c = int(cnt.value)
    return dict(code=code[:c], pos=pos[:c], strand=st[:c])


def overlap_row(A: dict, At: dict, i: int, min_shared: int = 2, max_seeds: int = 2) -> dict:
    """Row i of C = A At over the overlap semiring: dict(col, count, seed_i [S, e], seed_k [S, e])."""
    lib = _load()
    a, keep_a = _csr_in(A)
    t, keep_t = _csr_in(At)
    n = int(A["n_rows"])
    S = int(max_seeds)
    col = np.zeros(max(n, 1), np.int32)
    cnt = np.zeros(max(n, 1), np.uint32)
    si = np.zeros(max(n, 1) * max(S, 1), np.uint32)
    sk = np.zeros(max(n, 1) * max(S, 1), np.uint32)
    e = ctypes.c_int64()
    _check(lib.sgo_overlap_row(ctypes.byref(a), ctypes.byref(t), int(i), int(min_shared), S, col.ctypes.data,
                               cnt.ctypes.data, si.ctypes.data, sk.ctypes.data, ctypes.byref(e)), "overlap_row")
    m = int(e.value)
    return dict(col=col[:m], count=cnt[:m], seed_i=si[:m * S].reshape(m, S).T.copy(),
                seed_k=sk[:m * S].reshape(m, S).T.copy())


def graph_from_seeds(C: dict, offsets, k: int, min_overlap: int) -> dict:
    """R estimated from C's first seeds (see sgo_graph_from_seeds): dict(n, row_ptr, col, suffix, dir)."""
    lib = _load()
    o = np.ascontiguousarray(offsets, np.int64)
    nnz = int(C["col"].size)
    arrs = (np.ascontiguousarray(C["row_ptr"], np.int64), np.ascontiguousarray(C["col"], np.int32),
            np.ascontiguousarray(C["count"], np.uint32),
            np.ascontiguousarray(np.asarray(C["seed_i"], np.uint32).reshape(-1)),
            np.ascontiguousarray(np.asarray(C["seed_k"], np.uint32).reshape(-1)))
    S = np.asarray(C["seed_i"]).shape[0]  # seeds are [S, nnz], slot-major
    c = _Overlap(int(C["n"]), nnz, int(S), arrs[0].ctypes.data, arrs[1].ctypes.data, arrs[2].ctypes.data,
                 arrs[3].ctypes.data, arrs[4].ctypes.data)
    R = _Graph()
    _check(lib.sgo_graph_from_seeds(ctypes.byref(c), o.ctypes.data, int(k), int(min_overlap), ctypes.byref(R)),
           "graph_from_seeds")
    e = int(R.nnz)
    return dict(n=int(R.n), row_ptr=_take(lib, R.row_ptr, R.n + 1, np.int64), col=_take(lib, R.col, e, np.int32),
                suffix=_take(lib, R.suffix, e, np.uint32), dir=_take(lib, R.dir, e, np.uint8))
