"""Autotuner for the library's launch parameters.

Coordinate descent: each tunable in turn is set to every candidate value while the others stay
fixed, one timed call of `step` (after a warm-up call) is taken per candidate and repetition, and
the fastest median wins. The parameters (Bloom slice size, symbolic table guess, grid sizes) only
change speed, never results. The chosen values can be cached per GPU and workload signature.
"""
from __future__ import annotations

import json
import os
import statistics

import paper_2010_10055_gb300 as sg

SPACE = {
    "bloom_binned": [0, 1],
    "bloom_bin_kb": [64, 128],
    "bloom_scatter_cfg": [0, 1, 2],
    "kmer_sort_buckets": [0, 2, 3],
    "bloom_bits": [6, 8, 10, 12],
    "radix_lookback": [4, 8],
    "spgemm_upper": [0, 1],
    "spgemm_guess_pct": [150, 200, 250, 300],
    "spgemm_escalate": [0, 1],
    "spgemm_filter_mode": [0, 1],
    "spgemm_tab_warps": [32, 48, 64],
    "spgemm_tab_warps_big": [16, 32, 64],
    "spgemm_mirror_rec": [0, 1],
    "kmer_direct_seg": [0, 1],
    "spgemm_tmp_pct": [110, 125, 200],
    "spgemm_blocks_per_sm": [4, 8, 16],
    "tr_blocks_per_sm": [8, 16, 32],
    "tr_warp_rows": [0, 1],
}
# the batched form adds the planner's thresholds
BATCH_SPACE = {"batch_alone_kb": [32000, 64000, 128000], "batch_group_kb": [100000, 250000, 500000, 1000000]}


def _time_ms(step, reps: int) -> float:
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step()  # warm-up with the new setting
    ts = []
    for _ in range(reps):
        e0.record()
        out = step()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
        del out
    return statistics.median(ts)


def autotune(step, space: dict | None = None, reps: int = 3, rounds: int = 1, log=None, timer=None) -> dict:
    """Tunes in place and returns {"params": chosen values, "ms": best step time, "trials": n}.
    timer(step, reps) -> ms times one setting (default: CUDA events around `step`, median of reps
    after a warm-up call)."""
    space = space or SPACE
    _time = timer or _time_ms
    best = _time(step, reps)
    trials = 1
    for _ in range(rounds):
        for name, cands in space.items():
            cur = sg.tunables()[name]
            choice, choice_ms = cur, best
            for v in cands:
                if v == cur:
                    continue
                sg.tune(name, v)
                ms = _time(step, reps)
                trials += 1
                if log:
                    log(f"{name}={v}: {ms:.3f} ms")
                if ms < choice_ms:
                    choice, choice_ms = v, ms
            sg.tune(name, choice)
            best = choice_ms
    return {"params": sg.tunables(), "ms": best, "trials": trials}


DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json")


def device_id() -> str:
    """GPU name and multiprocessor count of the current device (part of every cache key)."""
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|{p.multi_processor_count}"


def cache_key(signature: str, device: str | None = None) -> str:
    return f"{device or device_id()}|{signature}"


def load(path: str, signature: str, device: str | None = None) -> bool:
    """Applies cached values for this GPU and workload signature; returns whether any were found.
    Values of tunables this library does not know, or out of their range, are skipped."""
    try:
        entry = json.load(open(path)).get(cache_key(signature, device))
    except (OSError, ValueError):
        return False
    if not entry:
        return False
    known = sg.tunables()
    applied = False
    for k, v in entry["params"].items():
        if k in known:
            try:
                sg.tune(k, v)
                applied = True
            except ValueError:
                pass
    return applied


def store(path: str, signature: str, result: dict, device: str | None = None) -> None:
    try:
        data = json.load(open(path))
    except (OSError, ValueError):
        data = {}
    data[cache_key(signature, device)] = result
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "w") as f:
        json.dump(data, f, indent=1)


def _main():
    """Tunes on a synthetic workload: the full step (k-mer matrix, overlap product, reduction) of a
    named workload, or with --batched one sg_run_batch over `--sets` read sets of the batched
    shape. Prints every trial and the choice; --cache stores it for this GPU and workload."""
    import argparse

    import torch

    import synth

    p = argparse.ArgumentParser(description=_main.__doc__)
    p.add_argument("--workload", default="bacterial-5Mbp-30x")
    p.add_argument("--batched", action="store_true")
    p.add_argument("--sets", type=int, default=128)
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--cache", default=None)
    a = p.parse_args()
    if a.batched:
        sets = synth.batched_sets(a.sets, 20e3, 2e6)
        items = [dict(seq=torch.from_numpy(x["seq"]).cuda(), offsets=torch.from_numpy(x["offsets"]).cuda(),
                      lo=x["lo"], hi=x["hi"], R=sg.DeviceGraph.from_numpy(x["R"])) for x in sets]
        signature = f"batched-{a.sets}"  # the bench's batched measurement loads this key

        def step():
            sg.run_batch(items, k=17, min_shared=2, max_seeds=2, fuzz=1000)
    else:
        w = synth.WORKLOADS[a.workload]
        d = synth.make(w)
        seq, off = torch.from_numpy(d["seq"]).cuda(), torch.from_numpy(d["offsets"]).cuda()
        R = sg.DeviceGraph.from_numpy(d["R"])
        signature = w.name

        def step():
            km = sg.build_kmer_matrix(seq, off, w.k, w.lo, w.hi)
            sg.overlap_spgemm(km, w.min_shared, w.max_seeds)
            sg.transitive_reduce(R, w.fuzz)
    before = sg.tunables()
    space = {**SPACE, **BATCH_SPACE} if a.batched else SPACE
    res = autotune(step, space=space, reps=a.reps, log=lambda s: print(s, flush=True))
    changed = {k: (before[k], v) for k, v in res["params"].items() if before.get(k) != v}
    print(json.dumps({"signature": signature, "ms": res["ms"], "trials": res["trials"], "changed": changed,
                      "params": res["params"]}), flush=True)
    if a.cache:
        store(a.cache, signature, res)


if __name__ == "__main__":
    _main()
