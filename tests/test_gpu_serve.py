"""The served form: every job's result equals the oracle on that job alone, whatever it was batched
with (tolerance 0), and jobs larger than the budget are refused."""
import time

import numpy as np
import pytest

import oracle
import paper_2010_10055_gb300 as sg
import synth
from tests.gpu_util import assert_graph_equal, assert_overlap_equal

pytestmark = pytest.mark.gpu


def _jobs(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        G = int(rng.integers(10000, 80000))
        g = synth.genome(G, seed * 1000 + b)
        rd = synth.reads(g, 12.0, float(rng.uniform(800, 3000)), 500.0, 200, 0.06, 0.04, 0.02, seed * 1000 + b + 1)
        R = synth.overlap_graph(rd["start"], rd["end"], rd["strand"], 100)
        out.append(dict(seq=rd["seq"], offsets=rd["offsets"], lo=2, hi=int(rng.integers(6, 12)), R=R))
    return out


def _check(res, job, fuzz):
    assert res["status"] == sg.SG_OK
    km = oracle.build_kmer_matrix(job["seq"], job["offsets"], 17, job["lo"], job["hi"])
    assert_overlap_equal(res["C"], oracle.overlap_spgemm(km["A"], km["At"], 2, 2))
    eS, eit = oracle.transitive_reduce(job["R"], fuzz)
    assert_graph_equal(res["S"], eS)
    assert res["iterations"] == eit


def test_server_results_match_oracle_alone_and_mixed():
    jobs = _jobs(5, 14)
    srv = sg.Server(hbm_budget=1 << 30, max_batch=5, workers=2, fuzz=300)
    try:
        # arrivals in a burst and then staggered: jobs are admitted while other batches run
        tickets = []
        for b, j in enumerate(jobs):
            tickets.append(srv.submit(j["seq"], j["offsets"], j["lo"], j["hi"], j["R"]))
            if b >= 7:
                time.sleep(0.002)
        mixed = [srv.wait(t) for t in tickets]
        for r, j in zip(mixed, jobs):
            _check(r, j, 300)
        # the same job alone
        alone = srv.wait(srv.submit(jobs[3]["seq"], jobs[3]["offsets"], jobs[3]["lo"], jobs[3]["hi"], jobs[3]["R"]))
        assert alone["batch_size"] == 1
        for key in ("row_ptr", "col", "count", "seed_i", "seed_k"):
            assert np.array_equal(alone["C"][key], mixed[3]["C"][key])
        for key in ("row_ptr", "col", "suffix", "dir"):
            assert np.array_equal(alone["S"][key], mixed[3]["S"][key])
    finally:
        srv.close()


def test_server_refuses_jobs_over_budget_and_keeps_going():
    jobs = _jobs(6, 2)
    srv = sg.Server(hbm_budget=4 << 20, max_batch=4, workers=1)  # smaller than any job's estimate
    try:
        r = srv.wait(srv.submit(jobs[0]["seq"], jobs[0]["offsets"], 2, 8, jobs[0]["R"]))
        assert r["status"] == sg.SG_ERR_BUDGET
        assert srv.poll(12345) is None  # unknown / not ready
    finally:
        srv.close()
    srv = sg.Server(hbm_budget=1 << 30, max_batch=4, workers=1)
    try:
        r = srv.wait(srv.submit(jobs[1]["seq"], jobs[1]["offsets"], jobs[1]["lo"], jobs[1]["hi"], jobs[1]["R"]))
        _check(r, jobs[1], 0)
    finally:
        srv.close()


def test_server_batches_jobs_that_queue_up():
    """One worker, a burst of submissions: jobs that queue while a batch runs share the next one."""
    jobs = _jobs(7, 6) * 5
    srv = sg.Server(hbm_budget=1 << 30, max_batch=64, workers=1)
    try:
        tickets = [srv.submit(j["seq"], j["offsets"], j["lo"], j["hi"], j["R"]) for j in jobs]
        res = [srv.wait(t) for t in tickets]
        assert [(r["status"], r["error"]) for r in res if r["status"] != sg.SG_OK] == []
        assert max(r["batch_size"] for r in res) > 1
        # identical inputs give identical outputs wherever they were batched
        for b in range(6, len(jobs)):
            for key in ("row_ptr", "col", "count", "seed_i", "seed_k"):
                assert np.array_equal(res[b]["C"][key], res[b % 6]["C"][key])
            for key in ("row_ptr", "col", "suffix", "dir"):
                assert np.array_equal(res[b]["S"][key], res[b % 6]["S"][key])
        for r in res:  # latencies are ordered: submitted <= started <= done
            assert r["t_submit"] <= r["t_start"] <= r["t_done"]
    finally:
        srv.close()


def test_server_cancel_queued_job():
    """A queued job can be cancelled: it never runs and reports SG_ERR_CANCELLED; the others are
    unaffected; running, finished and unknown tickets cannot be cancelled."""
    big = synth.genome(1_500_000, 31)
    rd = synth.reads(big, 30.0, 10000.0, 4000.0, 500, 0.075, 0.05, 0.025, 32)
    jobs = _jobs(8, 3)
    srv = sg.Server(hbm_budget=8 << 30, max_batch=1, workers=1, fuzz=300)
    try:
        t0 = srv.submit(rd["seq"], rd["offsets"], 2, 20)  # keeps the single worker busy
        ts = [srv.submit(j["seq"], j["offsets"], j["lo"], j["hi"], j["R"]) for j in jobs]
        assert srv.cancel(ts[1])
        assert not srv.cancel(ts[1])  # already cancelled
        assert not srv.cancel(987654321)
        r0 = srv.wait(t0)
        assert r0["status"] == sg.SG_OK
        assert not srv.cancel(t0)  # finished
        res = [srv.wait(t) for t in ts]
        assert res[1]["status"] == sg.SG_ERR_CANCELLED and "cancel" in res[1]["error"]
        _check(res[0], jobs[0], 300)
        _check(res[2], jobs[2], 300)
    finally:
        srv.close()


def test_server_admits_job_over_budget_with_c_in_tiles():
    """A job whose one-piece estimate exceeds the budget, but whose resident part (inputs, A, At,
    R) plus a tile budget fits, runs alone with C formed in row tiles: its result equals the
    oracle's, and a small job queued behind it still completes."""
    g = synth.genome(100_000, 41)
    rd = synth.reads(g, 60.0, 10000.0, 3000.0, 500, 0.075, 0.05, 0.025, 42)
    R = synth.overlap_graph(rd["start"], rd["end"], rd["strand"], 500)
    job = dict(seq=rd["seq"], offsets=rd["offsets"], lo=2, hi=40, R=R)
    L, n1, rn = rd["seq"].size, rd["offsets"].size, R["col"].size
    est = 64 * L + 48 * rn + 64 * n1 + (1 << 20)
    est_tiled = max(40 * L + 64 * n1 + (1 << 20), 24 * L + 48 * rn + 64 * n1 + (1 << 20) + (64 << 20))
    budget = est_tiled + (1 << 20)
    assert est > budget
    small = _jobs(9, 1)[0]
    srv = sg.Server(hbm_budget=budget, max_batch=4, workers=2, fuzz=300)
    try:
        t_big = srv.submit(job["seq"], job["offsets"], job["lo"], job["hi"], job["R"])
        t_small = srv.submit(small["seq"], small["offsets"], small["lo"], small["hi"], small["R"])
        r = srv.wait(t_big)
        assert r["status"] == sg.SG_OK, r["error"]
        assert r["batch_size"] == 1
        _check(r, job, 300)
        _check(srv.wait(t_small), small, 300)
    finally:
        srv.close()


def test_served_jobs_at_stated_sizes_equal_plain_calls():
    """Jobs drawn from the served workload's own distribution (Pareto genome sizes from 20 kbp,
    30x), submitted as a burst so that they share batches: each result equals the plain three
    calls on that job alone, bit for bit."""
    jobs = synth.served_jobs(60, 200.0)
    srv = sg.Server(hbm_budget=150 << 30, max_batch=16, workers=2, fuzz=1000)
    try:
        res = [srv.wait(srv.submit(j["seq"], j["offsets"], j["lo"], j["hi"], j["R"])) for j in jobs[:4]]
        tickets = [srv.submit(j["seq"], j["offsets"], j["lo"], j["hi"], j["R"]) for j in jobs[4:]]
        res += [srv.wait(t) for t in tickets]
    finally:
        srv.close()
    assert max(r["batch_size"] for r in res) > 1
    import torch
    for r, j in zip(res, jobs):
        assert r["status"] == sg.SG_OK, r["error"]
        km = sg.build_kmer_matrix(torch.from_numpy(j["seq"]).cuda(), torch.from_numpy(j["offsets"]).cuda(), 17,
                                  j["lo"], j["hi"])
        assert_overlap_equal(r["C"], sg.overlap_spgemm(km, 2, 2).to_numpy())
        S, it = sg.transitive_reduce(sg.DeviceGraph.from_numpy(j["R"]), 1000)
        assert_graph_equal(r["S"], S.to_numpy())
        assert r["iterations"] == it
