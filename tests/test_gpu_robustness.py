"""Failure detection and order independence on the GPU, without faulting it.

- Bounded waits: the scan's tiles wait on earlier tiles' published prefixes. With the test hook
  on, the first tile withholds its prefix (a flag nothing sets); the later tiles' waits run out,
  the call returns SG_ERR_TIMEOUT, and the context stays usable.
- Launch parameters (tunables) change grids, slice counts, table sizes and which rows take the
  global-memory path, never the results: every accumulation is commutative (the seeds keep the
  smallest column indices, counts are sums, the min-plus is a min), so each configuration must
  reproduce the oracle bit for bit.
"""
import numpy as np
import pytest

import oracle
import paper_2010_10055_gb300 as sg
import synth
from tests.gpu_util import assert_graph_equal, assert_kmer_equal, assert_overlap_equal, dev, gpu_kmer

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_reports_timeout():
    R = synth.random_graph(6000, 8.0, hub_frac=0.02, max_suffix=2000, seed=11)  # kept[] scan: 2 tiles
    D = sg.DeviceGraph.from_numpy(R)
    sg.debug_stall_lookback(True)
    try:
        with pytest.raises(sg.SgError) as e:
            sg.transitive_reduce(D, fuzz=100)
        assert e.value.status == sg.SG_ERR_TIMEOUT
        assert "bounded wait" in str(e.value)
    finally:
        sg.debug_stall_lookback(False)
    # the same call now completes and is exact
    S, it = sg.transitive_reduce(D, fuzz=100)
    eS, eit = oracle.transitive_reduce(R, 100)
    assert_graph_equal(S.to_numpy(), eS)
    assert it == eit


CONFIGS = [
    {},
    {"bloom_binned": 0, "bloom_bits": 4, "bloom_slice_mb": 1},       # many small Bloom slices
    {"bloom_binned": 0, "bloom_bits": 12, "bloom_unroll": 8},
    {"bloom_bin_kb": 16, "bloom_bits": 32},                          # many shared-memory bins
    {"bloom_bin_room_pct": 50},                                      # bins overflow: sliced redo
    {"bloom_bin_kb": 64, "bloom_scatter_cfg": 1},                    # smaller bins, 256 x 16 tiles
    {"bloom_scatter_levels": 2, "bloom_bin_kb": 16},                 # two grouping passes
    {"bloom_scatter_levels": 2, "bloom_bin_room_pct": 50},           # superbins overflow: sliced redo
    {"bloom_scatter_cfg": 2, "kmer_sort_buckets": 0},                # 256 x 32 tiles, one bucket
    {"kmer_direct_seg": 0},                                          # unpacked keys, then segments
    {"kmer_direct_seg": 0, "kmer_sort_buckets": 0},
    {"spgemm_fused": 0, "sym_guess_shift": 8},                      # two passes, tiny symbolic guesses
    {"spgemm_fused": 0, "sym_guess_shift": 0, "spgemm_blocks_per_sm": 1, "tr_blocks_per_sm": 1},
    {"spgemm_guess_pct": 25},                                        # fused, most rows overflow
    {"spgemm_guess_pct": 10000},                                     # fused, guesses past shared memory
    {"spgemm_guess_pct": 100, "spgemm_big_threads": 512},            # 4 K+ tables, 512 threads
    {"spgemm_fused_max_mb": 0},                                      # fused path over budget: fallback
    {"spgemm_filter_work": 0},                                       # no seen-twice filter
    {"spgemm_filter_mode": 2, "spgemm_filter_work": 1},              # every row filtered first
    {"spgemm_filter_mode": 2, "spgemm_filter_work": 1, "spgemm_guess_pct": 5},  # filtered rows overflow
    {"spgemm_sample_rows": 0},                                       # no sample: a partner per A entry
    {"spgemm_sample_rows": 1, "spgemm_guess_pct": 25},               # one sampled row, tables too small
    {"spgemm_tmp_pct": 1},                                           # temporary region full: retries
    {"spgemm_tmp_pct": 1, "spgemm_upper": 0},                        # ... for whole rows
    {"spgemm_tab_warps": 0},                                         # fixed threads per table size
    {"spgemm_tab_warps": 8, "spgemm_blocks_per_sm": 1},              # few warps, small grid
    {"spgemm_upper": 0},                                             # whole rows, no mirror
    {"spgemm_upper": 0, "spgemm_guess_pct": 25},                     # whole rows, most rows overflow
    {"spgemm_upper": 0, "spgemm_filter_mode": 2, "spgemm_filter_work": 1},  # whole rows, filtered
    {"spgemm_mirror_sort": 0, "spgemm_lower_smem": 16, "spgemm_guess_pct": 25},  # mixed row sorts
    {"spgemm_blocks_per_sm": 1, "spgemm_big_threads": 512, "spgemm_lower_smem": 64},
    {"tr_warp_rows": 0},                                             # min-plus over flattened products
    {"spgemm_at_records": 0},                                        # At rows gathered, no records
    {"spgemm_at_records": 0, "spgemm_upper": 0},
    {"spgemm_filter_mode": 1},                                       # filter where the sample says
    {"spgemm_mirror_sort": 0},                                       # mirror by atomics + row sorts
    {"spgemm_mirror_rec": 0},                                        # mirror gathers C's arrays
    {"spgemm_mirror_sort": 0, "spgemm_lower_smem": 1},               # ... all in global memory
]


@pytest.fixture(scope="module")
def medium():
    w = synth.BACTERIAL.scaled(0.02)  # 100 kbp genome, two repeat families
    d = synth.make(w)
    km = oracle.build_kmer_matrix(d["seq"], d["offsets"], w.k, w.lo, w.hi)
    C = oracle.overlap_spgemm(km["A"], km["At"], w.min_shared, w.max_seeds)
    S, it = oracle.transitive_reduce(d["R"], w.fuzz)
    return w, d, km, C, S, it


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: ",".join(f"{k}={v}" for k, v in c.items()) or "defaults")
def test_tunables_never_change_results(medium, cfg):
    w, d, ekm, eC, eS, eit = medium
    saved = sg.tunables()
    try:
        for k, v in cfg.items():
            sg.tune(k, v)
        km, got = gpu_kmer(d["seq"], d["offsets"], w.k, w.lo, w.hi)
        assert_kmer_equal(got, ekm)
        C = sg.overlap_spgemm(km, w.min_shared, w.max_seeds)
        assert_overlap_equal(C.to_numpy(), eC)
        S, it = sg.transitive_reduce(sg.DeviceGraph.from_numpy(d["R"]), w.fuzz)
        assert_graph_equal(S.to_numpy(), eS)
        assert it == eit
    finally:
        for k, v in saved.items():
            sg.tune(k, v)


@pytest.mark.parametrize("cfg", [{"spgemm_filter_mode": 2, "spgemm_filter_work": 1, "spgemm_filter_log2": 10},
                                 {"spgemm_filter_mode": 2, "spgemm_filter_work": 1, "spgemm_filter_log2": 10,
                                  "spgemm_guess_pct": 10}],
                         ids=["hashed-filter", "hashed-filter-small-tables"])
def test_hashed_seen_twice_filter(cfg):
    """More reads (about 1500) than filter bits (2^10): partners share filter bits, count-1
    partners reach the table, and C must still be exact."""
    w = synth.BACTERIAL.scaled(0.1)
    d = synth.make(w)
    km = oracle.build_kmer_matrix(d["seq"], d["offsets"], w.k, w.lo, w.hi)
    assert km["A"]["n_rows"] > 1024
    eC = oracle.overlap_spgemm(km["A"], km["At"], w.min_shared, w.max_seeds)
    saved = sg.tunables()
    try:
        for k, v in cfg.items():
            sg.tune(k, v)
        gkm, got = gpu_kmer(d["seq"], d["offsets"], w.k, w.lo, w.hi)
        assert_kmer_equal(got, km)
        assert_overlap_equal(sg.overlap_spgemm(gkm, w.min_shared, w.max_seeds).to_numpy(), eC)
    finally:
        for k, v in saved.items():
            sg.tune(k, v)


def _every_entry_point(w, d):
    """One pass through every device entry point on the workload, all outputs released."""
    seq, off = dev(d["seq"], np.uint8), dev(d["offsets"], np.int64)
    km = sg.build_kmer_matrix(seq, off, w.k, w.lo, w.hi)
    C = sg.overlap_spgemm(km, w.min_shared, w.max_seeds)
    G = sg.overlap_graph_from_seeds(C, off, w.k, w.min_overlap)
    R = sg.DeviceGraph.from_numpy(d["R"])
    S, _ = sg.transitive_reduce(R, w.fuzz)
    S1, _, _ = sg.transitive_reduce_rounds(R, w.fuzz, max_rounds=1)
    N = sg.minplus_square(R)  # torch outputs; its work memory is the library's
    hp = sg.HostPipeline()
    hp.run(d["seq"], d["offsets"], w, d["R"])
    hp.close()
    b = sg.run_batch([dict(seq=seq, offsets=off, lo=w.lo, hi=w.hi, R=R)] * 2, k=w.k, fuzz=w.fuzz)
    b.free()
    for x in (km, C, G, S, S1):
        x.free()
    del N


def test_every_call_returns_its_memory(medium):
    """After the outputs are freed, the library pool's in-use bytes return to where they were, for
    every entry point and for calls that fail part way (allocation failures injected at each
    successive allocation of the k-mer, SpGEMM and reduction calls)."""
    import gc

    import torch
    w, d = medium[0], medium[1]
    _every_entry_point(w, d)
    torch.cuda.synchronize()
    gc.collect()
    base = sg.memory_stats()[1]
    _every_entry_point(w, d)
    torch.cuda.synchronize()
    gc.collect()
    assert sg.memory_stats()[1] == base
    seq, off = dev(d["seq"], np.uint8), dev(d["offsets"], np.int64)
    km = sg.build_kmer_matrix(seq, off, w.k, w.lo, w.hi)
    R = sg.DeviceGraph.from_numpy(d["R"])
    torch.cuda.synchronize()
    held = sg.memory_stats()[1]
    calls = [lambda: sg.build_kmer_matrix(seq, off, w.k, w.lo, w.hi),
             lambda: sg.overlap_spgemm(km, w.min_shared, w.max_seeds),
             lambda: sg.transitive_reduce(R, w.fuzz)[0]]
    for call in calls:
        for nth in range(1, 80):
            sg.debug_fail_alloc_after(nth)
            try:
                out = call()
            except sg.SgError as e:
                assert e.status == sg.SG_ERR_OOM
                out = None
            finally:
                sg.debug_fail_alloc_after(0)
            if out is None:
                torch.cuda.synchronize()
                gc.collect()
                assert sg.memory_stats()[1] == held, nth
            else:  # fewer allocations than nth: the call completed
                out.free()
                break
    km.free()
