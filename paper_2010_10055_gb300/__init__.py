"""sgraph -- GB300 (sm_103a) library for the overlap-and-layout hot path of diBELLA 2D
(arXiv 2010.10055): the reads x k-mers matrix A, C = A A^T over the overlap semiring, and the
transitive reduction of the bidirected overlap graph (Algorithms 1 and 3).

This module is the thin Python binding of the C ABI in ``include/sgraph.h``: it marshals torch
tensors (device memory, current stream) into the C calls and exposes the library-allocated
outputs as zero-copy torch tensors. Every step of the computation runs in the library's CUDA
kernels; there is no CPU path. If ``libsgraph.so`` is missing, calls raise ``RuntimeError``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsgraph.so")
LIB_PATH_CHECKED = os.path.join(_HERE, "libsgraph_checked.so")

(SG_OK, SG_ERR_INVALID, SG_ERR_OOM, SG_ERR_CUDA, SG_ERR_TIMEOUT, SG_ERR_BUDGET, SG_ERR_OVERFLOW,
 SG_ERR_CANCELLED) = range(8)
DIRMATCH, LITERAL = 0, 1
PER_END = 2  # mode flag: per-read-end row maxima in the reduction (or-ed with the semiring)
INF = 0xFFFFFFFF

EXPORTS = ("sg_build_kmer_matrix", "sg_overlap_spgemm", "sg_overlap_spgemm_tiled", "sg_minplus_square", "sg_transitive_reduce",
           "sg_transitive_reduce_rounds", "sg_overlap_graph_from_seeds",
           "sg_pipeline_host", "sg_host_arena_create", "sg_host_arena_destroy", "sg_run_batch", "sg_free_batch",
           "sg_server_create", "sg_server_submit", "sg_server_poll", "sg_server_wait", "sg_job_result_free",
           "sg_server_destroy", "sg_server_cancel",
           "sg_free_csr_u32", "sg_free_overlap", "sg_free_graph", "sg_free", "sg_last_error",
           "sg_set_allocator", "sg_debug_fail_alloc_after", "sg_debug_stall_lookback", "sg_debug_check",
           "sg_debug_record_classes", "sg_debug_spgemm_classes", "sg_last_kmer_stats", "sg_launch_count", "sg_memory_stats", "sg_memory_reset_peak", "sg_prof_enable", "sg_prof_select", "sg_tune_set", "sg_tune_get", "sg_tune_name",
           "sg_prof_reset", "sg_prof_collect", "sg_prof_entry")


class SgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"sgraph status {status}: {msg}")
        self.status = status


class CsrU32(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class OverlapCsr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("max_seeds", ctypes.c_int32),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("count", ctypes.c_void_p),
                ("seed_i", ctypes.c_void_p), ("seed_k", ctypes.c_void_p)]


class GraphCsr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("suffix", ctypes.c_void_p), ("dir", ctypes.c_void_p)]


class PipelineJob(ctypes.Structure):
    _fields_ = [("seq", ctypes.c_void_p), ("offsets", ctypes.c_void_p), ("n_reads", ctypes.c_int64),
                ("total_len", ctypes.c_int64), ("k", ctypes.c_int32), ("lo", ctypes.c_uint32), ("hi", ctypes.c_uint32),
                ("min_shared", ctypes.c_uint32), ("max_seeds", ctypes.c_int32), ("r_row_ptr", ctypes.c_void_p),
                ("r_col", ctypes.c_void_p), ("r_suffix", ctypes.c_void_p), ("r_dir", ctypes.c_void_p),
                ("r_nnz", ctypes.c_int64), ("fuzz", ctypes.c_uint32), ("tr_mode", ctypes.c_int32)]

    @staticmethod
    def make(seq, offsets, n, total, w, r_row_ptr=None, r_col=None, r_suffix=None, r_dir=None, r_nnz=0,
             tr_mode=0):
        """Job from host addresses and a parameter set with k, lo, hi, min_shared, max_seeds, fuzz."""
        return PipelineJob(seq, offsets, int(n), int(total), int(w.k), int(w.lo), int(w.hi), int(w.min_shared),
                           int(w.max_seeds), r_row_ptr, r_col, r_suffix, r_dir, int(r_nnz), int(w.fuzz),
                           int(tr_mode))


class PipelineResult(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("nnz_a", ctypes.c_int64), ("nnz_c", ctypes.c_int64),
                ("nnz_s", ctypes.c_int64), ("iterations", ctypes.c_int32), ("max_seeds", ctypes.c_int32),
                ("products", ctypes.c_uint64), ("c_row_ptr", ctypes.c_void_p), ("c_col", ctypes.c_void_p),
                ("c_count", ctypes.c_void_p), ("c_seed_i", ctypes.c_void_p), ("c_seed_k", ctypes.c_void_p),
                ("s_row_ptr", ctypes.c_void_p), ("s_col", ctypes.c_void_p), ("s_suffix", ctypes.c_void_p),
                ("s_dir", ctypes.c_void_p), ("error", ctypes.c_char * 192)]


class BatchItem(ctypes.Structure):
    _fields_ = [("d_seq", ctypes.c_void_p), ("d_offsets", ctypes.c_void_p), ("n_reads", ctypes.c_int64),
                ("total_len", ctypes.c_int64), ("lo", ctypes.c_uint32), ("hi", ctypes.c_uint32),
                ("R", ctypes.POINTER(GraphCsr))]


class BatchParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("min_shared", ctypes.c_uint32), ("max_seeds", ctypes.c_int32),
                ("fuzz", ctypes.c_uint32), ("tr_mode", ctypes.c_int32)]


class BatchResultC(ctypes.Structure):
    _fields_ = [("n_items", ctypes.c_int32), ("read_off", ctypes.c_void_p), ("col_off", ctypes.c_void_p),
                ("iterations", ctypes.c_void_p), ("iterations_all", ctypes.c_int32), ("A", CsrU32), ("At", CsrU32),
                ("d_kmer_codes", ctypes.c_void_p), ("C", OverlapCsr), ("S", GraphCsr)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_batch", ctypes.c_int32), ("workers", ctypes.c_int32),
                ("device", ctypes.c_int32), ("params", BatchParams)]


class Job(ctypes.Structure):
    _fields_ = [("seq", ctypes.c_void_p), ("offsets", ctypes.c_void_p), ("n_reads", ctypes.c_int64),
                ("total_len", ctypes.c_int64), ("lo", ctypes.c_uint32), ("hi", ctypes.c_uint32),
                ("r_row_ptr", ctypes.c_void_p), ("r_col", ctypes.c_void_p), ("r_suffix", ctypes.c_void_p),
                ("r_dir", ctypes.c_void_p), ("r_nnz", ctypes.c_int64)]


class KmerStats(ctypes.Structure):
    _fields_ = [("windows", ctypes.c_int64), ("candidates", ctypes.c_int64), ("m", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("sort_key_bytes", ctypes.c_int32), ("sort_val_bytes", ctypes.c_int32),
                ("sort_passes", ctypes.c_int32), ("a_sort_passes", ctypes.c_int32), ("bloom_bins", ctypes.c_int64),
                ("bloom_b2_bytes", ctypes.c_int64)]


class JobResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("n", ctypes.c_int64), ("m", ctypes.c_int64), ("nnz_c", ctypes.c_int64),
                ("nnz_s", ctypes.c_int64), ("iterations", ctypes.c_int32), ("max_seeds", ctypes.c_int32),
                ("batch_size", ctypes.c_int32), ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double), ("c_row_ptr", ctypes.c_void_p), ("c_col", ctypes.c_void_p),
                ("c_count", ctypes.c_void_p), ("c_seed_i", ctypes.c_void_p), ("c_seed_k", ctypes.c_void_p),
                ("s_row_ptr", ctypes.c_void_p), ("s_col", ctypes.c_void_p), ("s_suffix", ctypes.c_void_p),
                ("s_dir", ctypes.c_void_p), ("error", ctypes.c_char * 192)]


_lib = None


def use_checked_build():
    """Loads the checked build (kernels verify computed indices; see debug_check) instead of the
    normal one. Must be called before any other call of this module."""
    global LIB_PATH
    if _lib is not None:
        raise RuntimeError("the library is already loaded")
    LIB_PATH = LIB_PATH_CHECKED


def lib():
    """The loaded C library (loads it on first use; raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2010_10055_gb300.build_lib`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
        L.sg_build_kmer_matrix.restype = ctypes.c_int
        L.sg_build_kmer_matrix.argtypes = [vp, vp, i64, i64, i32, u32, u32, ctypes.POINTER(CsrU32),
                                           ctypes.POINTER(CsrU32), ctypes.POINTER(vp), vp]
        L.sg_overlap_spgemm.restype = ctypes.c_int
        L.sg_overlap_spgemm.argtypes = [ctypes.POINTER(CsrU32), ctypes.POINTER(CsrU32), u32, i32,
                                        ctypes.POINTER(OverlapCsr), vp]
        L.sg_overlap_spgemm_tiled.restype = ctypes.c_int
        L.sg_overlap_spgemm_tiled.argtypes = [ctypes.POINTER(CsrU32), ctypes.POINTER(CsrU32), u32, i32,
                                              ctypes.c_size_t, TILE_FN, vp, ctypes.POINTER(i64), vp]
        L.sg_minplus_square.restype = ctypes.c_int
        L.sg_minplus_square.argtypes = [ctypes.POINTER(GraphCsr), i32, vp, vp, vp]
        L.sg_transitive_reduce.restype = ctypes.c_int
        L.sg_transitive_reduce.argtypes = [ctypes.POINTER(GraphCsr), u32, i32, ctypes.POINTER(GraphCsr),
                                           ctypes.POINTER(i32), vp]
        L.sg_overlap_graph_from_seeds.restype = ctypes.c_int
        L.sg_overlap_graph_from_seeds.argtypes = [ctypes.POINTER(OverlapCsr), vp, i32, u32,
                                                  ctypes.POINTER(GraphCsr), vp]
        L.sg_transitive_reduce_rounds.restype = ctypes.c_int
        L.sg_transitive_reduce_rounds.argtypes = [ctypes.POINTER(GraphCsr), u32, i32, i32, ctypes.POINTER(GraphCsr),
                                                  ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), vp]
        L.sg_server_cancel.restype = ctypes.c_int
        L.sg_server_cancel.argtypes = [vp, ctypes.c_uint64]
        L.sg_free_csr_u32.argtypes = [ctypes.POINTER(CsrU32), vp]
        L.sg_free_overlap.argtypes = [ctypes.POINTER(OverlapCsr), vp]
        L.sg_free_graph.argtypes = [ctypes.POINTER(GraphCsr), vp]
        L.sg_free.argtypes = [vp, vp]
        L.sg_last_error.restype = ctypes.c_char_p
        L.sg_debug_fail_alloc_after.argtypes = [i64]
        L.sg_debug_stall_lookback.argtypes = [ctypes.c_int]
        L.sg_launch_count.restype = ctypes.c_uint64
        L.sg_memory_stats.argtypes = [ctypes.POINTER(ctypes.c_uint64)] * 3
        L.sg_debug_check.restype = ctypes.c_uint64
        L.sg_prof_enable.argtypes = [ctypes.c_int]
        L.sg_prof_select.argtypes = [ctypes.c_char_p]
        L.sg_prof_collect.restype = ctypes.c_int
        L.sg_prof_entry.restype = ctypes.c_int
        L.sg_prof_entry.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(i64),
                                    ctypes.POINTER(ctypes.c_double)]
        L.sg_host_arena_create.restype = ctypes.c_int
        L.sg_host_arena_create.argtypes = [ctypes.POINTER(vp)]
        L.sg_host_arena_destroy.argtypes = [vp]
        L.sg_tune_set.restype = ctypes.c_int
        L.sg_tune_set.argtypes = [ctypes.c_char_p, i64]
        L.sg_tune_get.restype = i64
        L.sg_tune_get.argtypes = [ctypes.c_char_p]
        L.sg_tune_name.restype = ctypes.c_char_p
        L.sg_tune_name.argtypes = [ctypes.c_int]
        L.sg_server_create.restype = ctypes.c_int
        L.sg_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
        L.sg_server_submit.restype = ctypes.c_int
        L.sg_server_submit.argtypes = [vp, ctypes.POINTER(Job), ctypes.POINTER(ctypes.c_uint64)]
        L.sg_server_poll.restype = ctypes.c_int
        L.sg_server_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(JobResult)]
        L.sg_server_wait.restype = ctypes.c_int
        L.sg_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(JobResult)]
        L.sg_job_result_free.argtypes = [ctypes.POINTER(JobResult)]
        L.sg_server_destroy.argtypes = [vp]
        L.sg_run_batch.restype = ctypes.c_int
        L.sg_run_batch.argtypes = [ctypes.POINTER(BatchItem), ctypes.c_int32, ctypes.POINTER(BatchParams),
                                   ctypes.POINTER(BatchResultC), vp]
        L.sg_free_batch.argtypes = [ctypes.POINTER(BatchResultC), vp]
        L.sg_pipeline_host.restype = ctypes.c_int
        L.sg_pipeline_host.argtypes = [ctypes.POINTER(PipelineJob), vp, ctypes.POINTER(PipelineResult), vp]
        _lib = L
    return _lib


def _check(status: int, what: str):
    if status != SG_OK:
        raise SgError(status, f"{what}: {lib().sg_last_error().decode(errors='replace')}")


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


class _DevView:
    """A library-owned device array, viewable as a torch tensor without copying."""

    def __init__(self, ptr, n, typestr, owner):
        self.__cuda_array_interface__ = dict(shape=(int(n),), typestr=typestr, data=(int(ptr or 0), False),
                                             version=3, strides=None, stream=None)
        self.owner = owner


# unsigned 32/64-bit arrays are exposed with the signed torch dtype of the same width
_TS = {"i8": "<i8", "i4": "<i4", "u4": "<i4", "u1": "|u1", "u8": "<i8"}
_NP = {"i8": np.int64, "i4": np.int32, "u4": np.uint32, "u1": np.uint8, "u8": np.uint64}


def _view(ptr, n, kind, owner):
    import torch
    if n == 0:
        dt = {"i8": torch.int64, "i4": torch.int32, "u4": torch.int32, "u1": torch.uint8, "u8": torch.int64}[kind]
        return torch.empty(0, dtype=dt, device="cuda")
    return torch.as_tensor(_DevView(ptr, n, _TS[kind], owner), device="cuda")


def _host(t, kind):
    return t.cpu().numpy().view(_NP[kind])


class _Owned:
    """Owns one output struct; frees it (stream-ordered) when released or collected."""
    _free_name = ""

    def __init__(self, struct, stream):
        self.s = struct
        self._stream = stream
        self._alive = True

    def free(self):
        if self._alive and _lib is not None:
            getattr(_lib, self._free_name)(ctypes.byref(self.s), self._stream)
        self._alive = False

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class CsrMatrix(_Owned):
    """A or At (CSR, 32-bit values pos | strand << 31)."""
    _free_name = "sg_free_csr_u32"

    @property
    def shape(self):
        return (int(self.s.n_rows), int(self.s.n_cols))

    @property
    def nnz(self):
        return int(self.s.nnz)

    KINDS = dict(row_ptr="i8", col="i4", val="u4")

    def tensors(self):
        return dict(row_ptr=_view(self.s.row_ptr, self.s.n_rows + 1, "i8", self),
                    col=_view(self.s.col, self.s.nnz, "i4", self),
                    val=_view(self.s.val, self.s.nnz, "u4", self))

    def to_numpy(self):
        d = {k: _host(v, self.KINDS[k]) for k, v in self.tensors().items()}
        d["n_rows"], d["n_cols"] = self.shape
        return d


class KmerMatrix:
    """Result of build_kmer_matrix: A, At and the canonical code of every column."""

    def __init__(self, A: CsrMatrix, At: CsrMatrix, codes_ptr, m, stream):
        self.A, self.At = A, At
        self._codes = codes_ptr
        self.m = m
        self._stream = stream

    def codes(self):
        """Column codes (uint64 bit patterns in an int64 tensor)."""
        return _view(self._codes, self.m, "u8", self)

    def free(self):
        self.A.free()
        self.At.free()
        if self._codes and _lib is not None:
            _lib.sg_free(self._codes, self._stream)
        self._codes = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def to_numpy(self):
        return dict(A=self.A.to_numpy(), At=self.At.to_numpy(), codes=_host(self.codes(), "u8"))


class Overlap(_Owned):
    """C = A At over the overlap semiring."""
    _free_name = "sg_free_overlap"

    @property
    def nnz(self):
        return int(self.s.nnz)

    KINDS = dict(row_ptr="i8", col="i4", count="u4", seed_i="u4", seed_k="u4")

    def tensors(self):
        S, nnz = int(self.s.max_seeds), int(self.s.nnz)
        return dict(row_ptr=_view(self.s.row_ptr, self.s.n + 1, "i8", self),
                    col=_view(self.s.col, nnz, "i4", self),
                    count=_view(self.s.count, nnz, "u4", self),
                    seed_i=_view(self.s.seed_i, S * nnz, "u4", self).view(S, nnz),
                    seed_k=_view(self.s.seed_k, S * nnz, "u4", self).view(S, nnz))

    def to_numpy(self):
        d = {k: _host(v, self.KINDS[k]) for k, v in self.tensors().items()}
        d["n"] = int(self.s.n)
        return d


class Graph(_Owned):
    """A bidirected overlap / string graph in CSR (suffix uint32, dir uint8)."""
    _free_name = "sg_free_graph"

    @property
    def nnz(self):
        return int(self.s.nnz)

    KINDS = dict(row_ptr="i8", col="i4", suffix="u4", dir="u1")

    def tensors(self):
        nnz = int(self.s.nnz)
        return dict(row_ptr=_view(self.s.row_ptr, self.s.n + 1, "i8", self),
                    col=_view(self.s.col, nnz, "i4", self),
                    suffix=_view(self.s.suffix, nnz, "u4", self),
                    dir=_view(self.s.dir, nnz, "u1", self))

    def to_numpy(self):
        d = {k: _host(v, self.KINDS[k]) for k, v in self.tensors().items()}
        d["n"] = int(self.s.n)
        return d


# ------------------------------------------------------------------------------- calls
def build_kmer_matrix(seq, offsets, k: int = 17, lo: int = 2, hi: int = 8, stream=None) -> KmerMatrix:
    """Reads -> A, At (see sg_build_kmer_matrix). seq: uint8 CUDA tensor of ASCII bases;
    offsets: int64 CUDA tensor [n+1]."""
    L = lib()
    st = _stream(stream)
    A, At, codes = CsrU32(), CsrU32(), ctypes.c_void_p()
    n = int(offsets.numel()) - 1
    rc = L.sg_build_kmer_matrix(_ptr(seq), _ptr(offsets), n, int(seq.numel()), int(k), int(lo), int(hi),
                                ctypes.byref(A), ctypes.byref(At), ctypes.byref(codes), st)
    _check(rc, "build_kmer_matrix")
    a, at = CsrMatrix(A, st), CsrMatrix(At, st)
    return KmerMatrix(a, at, codes.value, int(A.n_cols), st)


TILE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(OverlapCsr), ctypes.c_int64, ctypes.c_void_p)


def overlap_spgemm_tiled(km: KmerMatrix, budget_bytes: int, min_shared: int = 2, max_seeds: int = 2,
                         stream=None, on_tile=None):
    """C = A At formed in row tiles under a device-memory budget (see sg_overlap_spgemm_tiled).
    Each tile is copied to the host as it arrives; on_tile(row_begin, tile_dict) is called with it
    if given. Returns (C on the host, as Overlap.to_numpy() gives it, and the number of tiles)."""
    L = lib()
    st = _stream(stream)
    parts = []
    failure = []

    def cb(tile_p, row_begin, _user):
        try:
            t = tile_p.contents
            S, nnz = int(t.max_seeds), int(t.nnz)
            d = dict(row_ptr=_host(_view(t.row_ptr, t.n + 1, "i8", None), "i8"),
                     col=_host(_view(t.col, nnz, "i4", None), "i4"),
                     count=_host(_view(t.count, nnz, "u4", None), "u4"),
                     seed_i=_host(_view(t.seed_i, S * nnz, "u4", None), "u4").reshape(S, nnz),
                     seed_k=_host(_view(t.seed_k, S * nnz, "u4", None), "u4").reshape(S, nnz))
            parts.append((int(row_begin), d))
            if on_tile is not None:
                on_tile(int(row_begin), d)
            return SG_OK
        except Exception as ex:  # reported after the call; the library stops at a non-OK status
            failure.append(ex)
            return SG_ERR_INVALID

    fn = TILE_FN(cb)
    nt = ctypes.c_int64(0)
    rc = L.sg_overlap_spgemm_tiled(ctypes.byref(km.A.s), ctypes.byref(km.At.s), int(min_shared), int(max_seeds),
                                   int(budget_bytes), fn, None, ctypes.byref(nt), st)
    if failure:
        raise failure[0]
    _check(rc, "overlap_spgemm_tiled")
    n = km.A.shape[0]
    S = int(max_seeds)
    rp = [np.zeros(1, np.int64)]
    off = 0
    for _, d in parts:
        rp.append(d["row_ptr"][1:] + off)
        off += int(d["row_ptr"][-1])
    out = dict(n=n, row_ptr=np.concatenate(rp) if parts else np.zeros(n + 1, np.int64),
               col=np.concatenate([d["col"] for _, d in parts]) if parts else np.zeros(0, np.int32),
               count=np.concatenate([d["count"] for _, d in parts]) if parts else np.zeros(0, np.uint32),
               seed_i=np.concatenate([d["seed_i"] for _, d in parts], axis=1) if parts else np.zeros((S, 0), np.uint32),
               seed_k=np.concatenate([d["seed_k"] for _, d in parts], axis=1) if parts else np.zeros((S, 0), np.uint32))
    return out, int(nt.value)


def overlap_spgemm(km: KmerMatrix, min_shared: int = 2, max_seeds: int = 2, stream=None) -> Overlap:
    """C = A At over the overlap semiring (see sg_overlap_spgemm)."""
    L = lib()
    st = _stream(stream)
    C = OverlapCsr()
    _check(L.sg_overlap_spgemm(ctypes.byref(km.A.s), ctypes.byref(km.At.s), int(min_shared), int(max_seeds),
                               ctypes.byref(C), st), "overlap_spgemm")
    return Overlap(C, st)


class DeviceGraph:
    """A caller-owned graph (torch tensors) to pass as R."""

    def __init__(self, n, row_ptr, col, suffix, dir):
        self.n, self.row_ptr, self.col, self.suffix, self.dir = int(n), row_ptr, col, suffix, dir
        self.s = GraphCsr(self.n, int(col.numel()), row_ptr.data_ptr(), col.data_ptr() if col.numel() else 0,
                          suffix.data_ptr() if suffix.numel() else 0, dir.data_ptr() if dir.numel() else 0)

    @property
    def nnz(self):
        return int(self.col.numel())

    @staticmethod
    def from_numpy(R: dict, device="cuda") -> "DeviceGraph":
        import torch
        return DeviceGraph(R["n"], torch.from_numpy(np.ascontiguousarray(R["row_ptr"], np.int64)).to(device),
                           torch.from_numpy(np.ascontiguousarray(R["col"], np.int32)).to(device),
                           torch.from_numpy(np.ascontiguousarray(R["suffix"], np.uint32).view(np.int32)).to(device),
                           torch.from_numpy(np.ascontiguousarray(R["dir"], np.uint8)).to(device))


def _graph_struct(R):
    if isinstance(R, (DeviceGraph, Graph)):
        return R.s
    raise TypeError("R must be a DeviceGraph or a Graph returned by this library")


def transitive_reduce(R, fuzz: int = 0, mode: int = DIRMATCH, stream=None):
    """Algorithm 1: returns (S as Graph, iterations)."""
    L = lib()
    st = _stream(stream)
    S, it = GraphCsr(), ctypes.c_int32()
    _check(L.sg_transitive_reduce(ctypes.byref(_graph_struct(R)), int(fuzz), int(mode), ctypes.byref(S),
                                  ctypes.byref(it), st), "transitive_reduce")
    return Graph(S, st), int(it.value)


def overlap_graph_from_seeds(C: "Overlap", offsets, k: int = 17, min_overlap: int = 1000, stream=None) -> "Graph":
    """R estimated from C's first seeds (see sg_overlap_graph_from_seeds). offsets: int64 CUDA
    tensor [n+1] of the reads C was built from."""
    L = lib()
    st = _stream(stream)
    R = GraphCsr()
    _check(L.sg_overlap_graph_from_seeds(ctypes.byref(C.s), _ptr(offsets), int(k), int(min_overlap), ctypes.byref(R),
                                         st), "overlap_graph_from_seeds")
    return Graph(R, st)


def transitive_reduce_rounds(R, fuzz: int = 0, max_rounds: int = 1, mode: int = DIRMATCH, stream=None):
    """Algorithm 1 for at most max_rounds rounds: returns (S as Graph, rounds, converged). Pass S
    back as R to resume."""
    L = lib()
    st = _stream(stream)
    S, it, conv = GraphCsr(), ctypes.c_int32(), ctypes.c_int32()
    _check(L.sg_transitive_reduce_rounds(ctypes.byref(_graph_struct(R)), int(fuzz), int(mode), int(max_rounds),
                                         ctypes.byref(S), ctypes.byref(it), ctypes.byref(conv), st),
           "transitive_reduce_rounds")
    return Graph(S, st), int(it.value), bool(conv.value)


def minplus_square(R, mode: int = DIRMATCH, stream=None):
    """N = R^2 over Algorithm 3's semiring on the pattern of R: (N, Ndir) CUDA tensors; N holds
    uint32 bit patterns in an int32 tensor (0xFFFFFFFF = no qualifying walk)."""
    import torch
    L = lib()
    st = _stream(stream)
    s = _graph_struct(R)
    N = torch.empty(max(int(s.nnz), 1), dtype=torch.int32, device="cuda")  # uint32 bit patterns
    D = torch.empty(max(int(s.nnz), 1), dtype=torch.uint8, device="cuda")
    _check(L.sg_minplus_square(ctypes.byref(s), int(mode), _ptr(N), _ptr(D), st), "minplus_square")
    return N[: int(s.nnz)], D[: int(s.nnz)]


# ----------------------------------------------------------------------------- tooling
def last_kmer_stats() -> dict:
    """Sizes of this thread's last k-mer matrix build (see sg_last_kmer_stats)."""
    st = KmerStats()
    lib().sg_last_kmer_stats(ctypes.byref(st))
    return {f: int(getattr(st, f)) for f, _ in KmerStats._fields_}


def memory_stats() -> tuple:
    """(reserved, in_use, in_use_peak) bytes of the library's device memory pool (see
    sg_memory_stats)."""
    r, u, h = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().sg_memory_stats(ctypes.byref(r), ctypes.byref(u), ctypes.byref(h)), "memory_stats")
    return int(r.value), int(u.value), int(h.value)


def memory_reset_peak():
    lib().sg_memory_reset_peak()


def launch_count() -> int:
    return int(lib().sg_launch_count())


def prof_enable(on: bool = True):
    lib().sg_prof_enable(1 if on else 0)


def prof_select(prefix: str | None = None):
    """Time only kernels whose name starts with `prefix` (None = all)."""
    lib().sg_prof_select(prefix.encode() if prefix else None)


def prof_reset():
    lib().sg_prof_reset()


def prof_collect() -> dict:
    """{kernel name: (launches, total ms)} for the launches recorded since the last reset."""
    L = lib()
    n = L.sg_prof_collect()
    out = {}
    for i in range(n):
        name, cnt, ms = ctypes.c_char_p(), ctypes.c_int64(), ctypes.c_double()
        if L.sg_prof_entry(i, ctypes.byref(name), ctypes.byref(cnt), ctypes.byref(ms)):
            out[name.value.decode()] = (int(cnt.value), float(ms.value))
    return out


def tunables() -> dict:
    """{name: current value} of the library's launch parameters."""
    L, out, i = lib(), {}, 0
    while True:
        nm = L.sg_tune_name(i)
        if not nm:
            return out
        out[nm.decode()] = int(L.sg_tune_get(nm))
        i += 1


def tune(name: str, value: int):
    if not lib().sg_tune_set(name.encode(), int(value)):
        raise ValueError(f"unknown tunable or value out of range: {name}={value}")


def debug_check():
    """Checked build: (site, index) of the first out-of-bounds index a kernel detected and skipped
    since the last call, or None."""
    v = int(lib().sg_debug_check())
    return None if v == 0 else (v >> 40, v & ((1 << 40) - 1))


def debug_record_classes(on: bool):
    """Test hook: record which numeric launch handles each row of C (see sg_debug_record_classes)."""
    lib().sg_debug_record_classes(1 if on else 0)


def debug_spgemm_classes(n: int):
    """Per-row launch codes of the last fused overlap product on this thread, or None."""
    L = lib()
    L.sg_debug_spgemm_classes.restype = ctypes.c_int64
    L.sg_debug_spgemm_classes.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    out = np.zeros(max(int(n), 1), np.int32)
    got = int(L.sg_debug_spgemm_classes(out.ctypes.data, int(n)))
    return None if got < 0 else out[:min(got, int(n))]


def debug_stall_lookback(on: bool):
    """Test hook: multi-tile scans withhold their first tile's prefix, so calls fail with
    SG_ERR_TIMEOUT after their bounded waits run out (see sg_debug_stall_lookback)."""
    lib().sg_debug_stall_lookback(1 if on else 0)


def debug_fail_alloc_after(n: int):
    lib().sg_debug_fail_alloc_after(int(n))


# ------------------------------------------------------------------ host-buffer pipeline
class HostPipeline:
    """The whole path on host (numpy) buffers through sg_pipeline_host, with its own arena."""

    def __init__(self):
        self.arena = ctypes.c_void_p()
        _check(lib().sg_host_arena_create(ctypes.byref(self.arena)), "host_arena_create")

    def close(self):
        if self.arena and _lib is not None:
            _lib.sg_host_arena_destroy(self.arena)
        self.arena = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, seq, offsets, params, R=None, tr_mode=DIRMATCH, stream=None) -> dict:
        """Returns numpy copies of C, S and the sizes. `params` has k, lo, hi, min_shared,
        max_seeds and fuzz attributes."""
        seq = np.ascontiguousarray(seq, np.uint8)
        offsets = np.ascontiguousarray(offsets, np.int64)
        keep = [seq, offsets]
        rargs = (None, None, None, None, 0)
        if R is not None:
            rr = (np.ascontiguousarray(R["row_ptr"], np.int64), np.ascontiguousarray(R["col"], np.int32),
                  np.ascontiguousarray(R["suffix"], np.uint32), np.ascontiguousarray(R["dir"], np.uint8))
            keep += list(rr)
            rargs = tuple(a.ctypes.data for a in rr) + (int(rr[1].size),)
        job = PipelineJob.make(seq.ctypes.data if seq.size else None, offsets.ctypes.data, offsets.size - 1,
                               seq.size, params, *rargs, tr_mode=tr_mode)
        res = PipelineResult()
        _check(lib().sg_pipeline_host(ctypes.byref(job), self.arena, ctypes.byref(res), _stream(stream)),
               "pipeline_host")
        n = offsets.size - 1

        def arr(ptr, count, dtype):
            if count == 0 or not ptr:
                return np.zeros(0, dtype)
            return np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(np.ctypeslib.as_ctypes_type(dtype))),
                                         shape=(count,)).copy()

        S_ = int(res.max_seeds)
        out = dict(m=int(res.m), nnz_a=int(res.nnz_a), products=int(res.products), iterations=int(res.iterations),
                   C=dict(n=n, row_ptr=arr(res.c_row_ptr, n + 1, np.int64), col=arr(res.c_col, res.nnz_c, np.int32),
                          count=arr(res.c_count, res.nnz_c, np.uint32),
                          seed_i=arr(res.c_seed_i, res.nnz_c * S_, np.uint32).reshape(S_, -1),
                          seed_k=arr(res.c_seed_k, res.nnz_c * S_, np.uint32).reshape(S_, -1)))
        if R is not None:
            out["S"] = dict(n=n, row_ptr=arr(res.s_row_ptr, n + 1, np.int64), col=arr(res.s_col, res.nnz_s, np.int32),
                            suffix=arr(res.s_suffix, res.nnz_s, np.uint32), dir=arr(res.s_dir, res.nnz_s, np.uint8))
        return out


# --------------------------------------------------------------------------------- batches
class BatchResult:
    """Result of run_batch: the union outputs on the device plus per-set offsets; item(b) gives set
    b's slice with local indices (numpy), identical to running the three calls on set b alone."""

    def __init__(self, r: BatchResultC, stream, keep):
        self.r = r
        self._stream = stream
        self._keep = keep  # the items' device buffers must outlive the call only; kept for safety
        n = int(r.n_items)
        self.n_items = n
        self.read_off = np.ctypeslib.as_array(ctypes.cast(r.read_off, ctypes.POINTER(ctypes.c_int64)), (n + 1,)).copy()
        self.col_off = np.ctypeslib.as_array(ctypes.cast(r.col_off, ctypes.POINTER(ctypes.c_int64)), (n + 1,)).copy()
        self.iterations = np.ctypeslib.as_array(ctypes.cast(r.iterations, ctypes.POINTER(ctypes.c_int32)), (n,)).copy()
        self.iterations_all = int(r.iterations_all)
        self._host = None

    def free(self):
        if self.r is not None and _lib is not None:
            _lib.sg_free_batch(ctypes.byref(self.r), self._stream)
        self.r = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def to_numpy(self):
        """The union outputs on the host (downloaded once)."""
        if self._host is None:
            r = self.r
            A = CsrMatrix.__new__(CsrMatrix); A.s = r.A
            At = CsrMatrix.__new__(CsrMatrix); At.s = r.At
            C = Overlap.__new__(Overlap); C.s = r.C
            out = dict(A=A.to_numpy(), At=At.to_numpy(), C=C.to_numpy(),
                       codes=_host(_view(r.d_kmer_codes, int(r.A.n_cols), "u8", self), "u8"))
            if r.S.row_ptr:
                S = Graph.__new__(Graph); S.s = r.S
                out["S"] = S.to_numpy()
            self._host = out
        return self._host

    def item(self, b: int) -> dict:
        h = self.to_numpy()
        r0, r1 = int(self.read_off[b]), int(self.read_off[b + 1])
        c0, c1 = int(self.col_off[b]), int(self.col_off[b + 1])

        def rows(M, lo, hi):
            rp = M["row_ptr"][lo:hi + 1]
            return rp - rp[0], slice(int(rp[0]), int(rp[-1]))

        rp, sl = rows(h["A"], r0, r1)
        A = dict(n_rows=r1 - r0, n_cols=c1 - c0, row_ptr=rp, col=h["A"]["col"][sl] - c0, val=h["A"]["val"][sl])
        rp, sl = rows(h["At"], c0, c1)
        At = dict(n_rows=c1 - c0, n_cols=r1 - r0, row_ptr=rp, col=h["At"]["col"][sl] - r0, val=h["At"]["val"][sl])
        rp, sl = rows(h["C"], r0, r1)
        C = dict(n=r1 - r0, row_ptr=rp, col=h["C"]["col"][sl] - r0, count=h["C"]["count"][sl],
                 seed_i=h["C"]["seed_i"][:, sl], seed_k=h["C"]["seed_k"][:, sl])
        out = dict(A=A, At=At, codes=h["codes"][c0:c1], C=C, iterations=int(self.iterations[b]))
        if "S" in h:
            rp, sl = rows(h["S"], r0, r1)
            out["S"] = dict(n=r1 - r0, row_ptr=rp, col=h["S"]["col"][sl] - r0, suffix=h["S"]["suffix"][sl],
                            dir=h["S"]["dir"][sl])
        return out


def run_batch(items: list, k: int = 17, min_shared: int = 2, max_seeds: int = 2, fuzz: int = 0,
              tr_mode: int = DIRMATCH, stream=None) -> BatchResult:
    """items: dicts with seq (uint8 CUDA tensor), offsets (int64 CUDA tensor), lo, hi and optionally
    R (DeviceGraph over the set's reads)."""
    L = lib()
    st = _stream(stream)
    arr = (BatchItem * len(items))()
    keep = []
    for b, it in enumerate(items):
        R = it.get("R")
        rs = ctypes.pointer(R.s) if R is not None else None
        keep.append((it, rs))
        arr[b] = BatchItem(it["seq"].data_ptr() if it["seq"].numel() else None, it["offsets"].data_ptr(),
                           int(it["offsets"].numel()) - 1, int(it["seq"].numel()), int(it["lo"]), int(it["hi"]), rs)
    params = BatchParams(int(k), int(min_shared), int(max_seeds), int(fuzz), int(tr_mode))
    out = BatchResultC()
    _check(L.sg_run_batch(arr, len(items), ctypes.byref(params), ctypes.byref(out), st), "run_batch")
    return BatchResult(out, st, keep)


# --------------------------------------------------------------------------------- serving
def _arr(ptr, count, dtype):
    if count <= 0 or not ptr:
        return np.zeros(0, dtype)
    return np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(np.ctypeslib.as_ctypes_type(dtype))),
                                 shape=(int(count),)).copy()


class Server:
    """Continuous-batching server (sg_server_*): submit host read sets, wait for C and S."""

    def __init__(self, hbm_budget: int, max_batch: int = 64, workers: int = 2, device: int = 0, k: int = 17,
                 min_shared: int = 2, max_seeds: int = 2, fuzz: int = 0, tr_mode: int = DIRMATCH):
        cfg = ServerConfig(int(hbm_budget), int(max_batch), int(workers), int(device),
                           BatchParams(int(k), int(min_shared), int(max_seeds), int(fuzz), int(tr_mode)))
        self.h = ctypes.c_void_p()
        _check(lib().sg_server_create(ctypes.byref(cfg), ctypes.byref(self.h)), "server_create")

    def submit(self, seq, offsets, lo: int, hi: int, R: dict | None = None) -> int:
        seq = np.ascontiguousarray(seq, np.uint8)
        off = np.ascontiguousarray(offsets, np.int64)
        keep = [seq, off]
        rr = (None, None, None, None, 0)
        if R is not None:
            a = (np.ascontiguousarray(R["row_ptr"], np.int64), np.ascontiguousarray(R["col"], np.int32),
                 np.ascontiguousarray(R["suffix"], np.uint32), np.ascontiguousarray(R["dir"], np.uint8))
            keep += list(a)
            rr = tuple(x.ctypes.data for x in a) + (int(a[1].size),)
        job = Job(seq.ctypes.data if seq.size else None, off.ctypes.data, off.size - 1, seq.size, int(lo), int(hi),
                  *rr)
        t = ctypes.c_uint64()
        _check(lib().sg_server_submit(self.h, ctypes.byref(job), ctypes.byref(t)), "server_submit")
        return int(t.value)

    @staticmethod
    def _convert(r: JobResult) -> dict:
        n, cn, sn, S = int(r.n), int(r.nnz_c), int(r.nnz_s), int(r.max_seeds)
        out = dict(status=int(r.status), n=n, m=int(r.m), iterations=int(r.iterations), batch_size=int(r.batch_size),
                   t_submit=r.t_submit, t_start=r.t_start, t_done=r.t_done,
                   error=r.error.decode(errors="replace"))
        if r.status == SG_OK:
            out["C"] = dict(n=n, row_ptr=_arr(r.c_row_ptr, n + 1, np.int64), col=_arr(r.c_col, cn, np.int32),
                            count=_arr(r.c_count, cn, np.uint32),
                            seed_i=_arr(r.c_seed_i, cn * S, np.uint32).reshape(S, cn),
                            seed_k=_arr(r.c_seed_k, cn * S, np.uint32).reshape(S, cn))
            if r.s_row_ptr:
                out["S"] = dict(n=n, row_ptr=_arr(r.s_row_ptr, n + 1, np.int64), col=_arr(r.s_col, sn, np.int32),
                                suffix=_arr(r.s_suffix, sn, np.uint32), dir=_arr(r.s_dir, sn, np.uint8))
        lib().sg_job_result_free(ctypes.byref(r))
        return out

    def poll(self, ticket: int):
        r = JobResult()
        rc = lib().sg_server_poll(self.h, int(ticket), ctypes.byref(r))
        if rc == SG_ERR_TIMEOUT:
            return None
        _check(rc, "server_poll")
        return self._convert(r)

    def wait(self, ticket: int, timeout: float = 120.0) -> dict:
        r = JobResult()
        _check(lib().sg_server_wait(self.h, int(ticket), float(timeout), ctypes.byref(r)), "server_wait")
        return self._convert(r)

    def cancel(self, ticket: int) -> bool:
        """Cancels a job still in the queue (True); False if it already started, finished or is unknown."""
        return lib().sg_server_cancel(self.h, ctypes.c_uint64(int(ticket))) == SG_OK

    def close(self):
        if self.h and _lib is not None:
            _lib.sg_server_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
