"""Memory-bounded formation of C in row tiles (sg_overlap_spgemm_tiled; the paper's closing
remark, Sec. VIII, on forming C partially under a memory bound). The concatenated tiles must equal
the oracle's C element by element (and the untiled call's), the call must hold at most its budget
of device memory on top of its inputs (the library pool's high-water mark), a budget below one row
must fail with SG_ERR_BUDGET before any tile, and a callback error must stop the call."""
import numpy as np
import pytest

import oracle
import paper_2010_10055_gb300 as sg
import synth
from tests.gpu_util import assert_overlap_equal, gpu_kmer

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def medium():
    w = synth.BACTERIAL.scaled(0.02)
    d = synth.make(w, with_graph=False)
    km, got = gpu_kmer(d["seq"], d["offsets"], w.k, w.lo, w.hi)
    eC = oracle.overlap_spgemm(got["A"], got["At"], w.min_shared, w.max_seeds)
    return w, km, eC


@pytest.mark.parametrize("budget_mb", [5, 6, 12, 4096])
def test_tiles_equal_oracle_and_stay_within_budget(medium, budget_mb):
    w, km, eC = medium
    base = sg.memory_stats()[1]
    sg.memory_reset_peak()
    C, tiles = sg.overlap_spgemm_tiled(km, budget_mb << 20, w.min_shared, w.max_seeds)
    peak = sg.memory_stats()[2]
    assert_overlap_equal(C, eC)
    assert tiles >= 1
    if budget_mb <= 6:
        assert tiles > 1
    assert peak - base <= budget_mb << 20, (peak - base, budget_mb)


@pytest.mark.parametrize("max_seeds,min_shared", [(0, 1), (1, 2), (3, 3), (8, 2)])
def test_tiles_every_seed_form(medium, max_seeds, min_shared):
    w, km, _ = medium
    C, tiles = sg.overlap_spgemm_tiled(km, 5 << 20, min_shared, max_seeds)
    ref = sg.overlap_spgemm(km, min_shared, max_seeds).to_numpy()
    assert tiles > 1
    assert_overlap_equal(C, ref)


def test_budget_below_one_row_fails_before_any_tile(medium):
    w, km, _ = medium
    seen = []
    with pytest.raises(sg.SgError) as e:
        sg.overlap_spgemm_tiled(km, 1 << 16, w.min_shared, w.max_seeds, on_tile=lambda r, d: seen.append(r))
    assert e.value.status == sg.SG_ERR_BUDGET and not seen


def test_callback_error_stops_the_call(medium):
    w, km, _ = medium
    seen = []

    def stop_after_two(r, d):
        seen.append(r)
        if len(seen) == 2:
            raise KeyError("stop")

    with pytest.raises(KeyError):
        sg.overlap_spgemm_tiled(km, 6 << 20, w.min_shared, w.max_seeds, on_tile=stop_after_two)
    assert len(seen) == 2
    # the library is still usable and leaks nothing
    before = sg.memory_stats()[1]
    C, _ = sg.overlap_spgemm_tiled(km, 6 << 20, w.min_shared, w.max_seeds)
    assert sg.memory_stats()[1] == before
