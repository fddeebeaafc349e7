"""Benchmark of the overlap-and-layout hot path on one GB300 (or N independent replicas).

One step = the whole path over one seeded synthetic read set: build A and At from the reads
(canonical k-mers, Bloom pass, exact count, reliable filter), C = A At over the overlap semiring,
and the transitive reduction of the overlap graph R (Algorithm 1). The workload is the
C. elegans-shaped read set (100 Mbp genome with 2% of it in repeat families, 40x, 10 kbp mean,
15% errors, k = 17, reliable range [2, 30], >= 2 shared k-mers, fuzz 1000); the bacterial-scale
set (5 Mbp, 30x) is timed beside it under "bacterial".

value  = A A^T semiring products (sum_j nnz(At_j)^2) per second over whole steps, inputs resident
         in HBM, L2 flushed (256 MB write) between steps.
e2e    = the same through sg_pipeline_host: reads and R copied from pinned host memory, C and S
         copied back, every step.
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "A·Aᵀ semiring products/s & TR edges/s (bit-exact); batched vs plain; p99"
UNIT = "products/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--workload", default="elegans-100Mbp-40x")
    p.add_argument("--scale", type=float, default=1.0,
                   help="genome length factor: a smaller case of the same workload, for profiling captures")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-forms", action="store_true", help="skip the batched and served measurements")
    return p.parse_args()


def combine_ranks(total_ms: float, products: int, tr_ms: float, edges: int, world: int, device: str = "cuda"):
    """Whole-job figures of a replica run: the slowest rank's step and TR times (MAX over ranks)
    and the work of all ranks (SUM), as (total_ms, products, tr_ms, edges)."""
    if world <= 1:
        return float(total_ms), float(products), float(tr_ms), float(edges)
    import torch
    import torch.distributed as dist
    times = torch.tensor([float(total_ms), float(tr_ms)], dtype=torch.float64, device=device)
    work = torch.tensor([float(products), float(edges)], dtype=torch.float64, device=device)
    dist.all_reduce(times, op=dist.ReduceOp.MAX)
    dist.all_reduce(work, op=dist.ReduceOp.SUM)
    return float(times[0]), float(work[0]), float(times[1]), float(work[1])


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- roofline
def algorithmic_bytes(kernel: str, sz: dict) -> float | None:
    """Bytes the method must move per step in `kernel` (inputs read once, outputs written once),
    from the per-unit figures: a 4-byte filter hash and 2 bits of packed base per position,
    4-byte filter words (a touch is a read and a write), 8-byte keys, 24-byte C entries."""
    if kernel == "pack":
        return 1.0 * sz["total"] + 4.25 * sz["total"]          # bases in; hash + packed base out
    k = sz.get("kstats") or {}
    if kernel == "bloom_insert" and k.get("bloom_bins"):      # shared-memory bins: binned hashes in, B2 out
        return 4.0 * sz["windows"] + k["bloom_b2_bytes"]
    if kernel == "bloom_bin_scatter":                         # hashes in, binned hashes out
        return 4.0 * sz["total"] + 4.0 * sz["windows"]
    if kernel == "bloom_insert":
        return 4.0 * sz["total"] + 8.0 * sz["windows"]         # hashes in + filter word read and write
    if kernel == "cand_count":
        return 4.0 * sz["total"] + 4.0 * sz["windows"]         # hashes in + second-filter word probe
    if kernel == "cand_emit" and k:                           # candidate masks and packed bases in, keys out
        return 0.125 * sz["windows"] + 0.25 * sz["total"] + 8.0 * k["candidates"]
    if kernel == "seg_mark" and k and sz.get("direct_seg"):  # sorted keys in, two flag bits out
        return 8.25 * k["candidates"]
    if kernel == "emit_at" and k and sz.get("direct_seg"):   # sorted keys and flags in; At, A pairs, codes out
        return 8.25 * k["candidates"] + 20.0 * k["nnz"] + 16.0 * k["m"]
    if kernel == "radix_onesweep" and sz.get("kstats"):
        k = sz["kstats"]  # every pass reads and writes each record once (the histogram is its own kernel)
        return (2.0 * k["sort_passes"] * k["candidates"] * (k["sort_key_bytes"] + k["sort_val_bytes"])
                + 2.0 * k["a_sort_passes"] * k["nnz"] * (4 + 8))
    if kernel == "spgemm_numeric":
        if sz.get("upper"):  # partners k > i only: half the off-diagonal products, half of C
            return (8.0 * sz["nnzA"] + 8.0 * sz["products_half"] + (8.0 + 8.0 * sz["S"]) * sz["nnzC"] / 2
                    + 8.0 * (sz["n"] + 1))
        return 8.0 * sz["nnzA"] + 8.0 * sz["products"] + (8.0 + 8.0 * sz["S"]) * sz["nnzC"] + 8.0 * (sz["n"] + 1)
    if kernel == "spgemm_symbolic":
        return 4.0 * sz["nnzA"] + 4.0 * sz["products"] + 8.0 * (sz["n"] + 1)
    if kernel == "tr_minplus_mark":
        return (9.0 * sz["nnzR"] + 9.0 * sz["tr_products"] + 1.0 * sz["nnzR"] + 8.0 * sz["n"]) * sz["rounds"]
    return None


def family(name: str) -> str:
    """Kernel family of a launch name: the SpGEMM passes launch one class per table size
    (spgemm_numeric_t1k, ..., and _f1k, ... for filtered rows), which are one kernel."""
    return re.sub(r"_[tf]\d+k?$", "", name)


def by_family(prof: dict) -> dict:
    out = {}
    for k, (c, ms) in prof.items():
        f = out.setdefault(family(k), [0, 0.0])
        f[0] += c
        f[1] += ms
    return {k: tuple(v) for k, v in out.items()}


def measured_traffic(kernel: str, workload: str, launch_bytes: float | None = None):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if that summary was taken
    on the current source of the kernel and on `workload` (else None: the counters are stale or
    belong to another read set). A summary taken on a smaller case of the same workload states
    its algorithmic bytes per launch; its traffic is then scaled by the ratio of this launch's
    algorithmic bytes to those (traffic grows with the work done)."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
        src = open(os.path.join(ROOT, "paper_2010_10055_gb300", "csrc", t["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != t["source_sha256_16"]:
            return None
        if t.get("workload") == workload:
            return float(t["dram_bytes_per_launch"])
        if t.get("small_case_of") == workload and launch_bytes and t.get("algorithmic_bytes_per_launch"):
            return float(t["dram_bytes_per_launch"]) * launch_bytes / float(t["algorithmic_bytes_per_launch"])
        return None
    except Exception:
        return None


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    import numpy as np
    import torch

    import paper_2010_10055_gb300 as sg
    import synth

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = synth.WORKLOADS[args.workload]
    if args.scale != 1.0:
        w = w.scaled(args.scale)
        w.name = f"{w.name}@{args.scale:g}"
    w = synth.Workload(**{**w.__dict__, "seed": w.seed + 1000 * rank})  # independent replica per rank
    from paper_2010_10055_gb300 import autotune
    defaults = sg.tunables()
    tuned = autotune.load(autotune.DEFAULT_CACHE, w.name.split("@")[0])  # this GPU's cached choice, if any
    tuned_params = {k: v for k, v in sg.tunables().items() if defaults.get(k) != v}
    d = synth.make(w)
    n = int(d["offsets"].size - 1)
    total = int(d["seq"].size)
    seq = torch.from_numpy(d["seq"]).cuda()
    off = torch.from_numpy(d["offsets"]).cuda()
    R = sg.DeviceGraph.from_numpy(d["R"])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        km = sg.build_kmer_matrix(seq, off, w.k, w.lo, w.hi)
        C = sg.overlap_spgemm(km, w.min_shared, w.max_seeds)
        S, it = sg.transitive_reduce(R, w.fuzz)
        return km, C, S, it

    for _ in range(args.warmup):
        out = step()
        del out
    torch.cuda.synchronize()
    # sizes for the units and the roofline, and the per-kernel breakdown: one untimed step with
    # every launch bracketed by events
    sg.prof_reset()
    sg.prof_select(None)
    sg.prof_enable(True)
    km, C, S, it = step()
    torch.cuda.synchronize()
    sg.prof_enable(False)
    collected = sg.prof_collect()
    stages = {k[len("stage/"):]: {"count": c, "ms": ms} for k, (c, ms) in collected.items() if k.startswith("stage/")}
    breakdown = {k: v for k, v in collected.items() if not k.startswith("stage/")}
    at_rp = km.At.to_numpy()["row_ptr"]
    a = np.diff(at_rp).astype(np.int64)
    products = int((a * a).sum())
    deg = np.diff(d["R"]["row_ptr"]).astype(np.int64)
    tr_products = int(deg[d["R"]["col"]].sum()) if d["R"]["col"].size else 0
    sz = dict(n=n, total=total, windows=max(total - (w.k - 1) * n, 0), nnzA=km.A.nnz, products=products,
              products_half=int((a * (a - 1) // 2).sum()), upper=bool(sg.tunables().get("spgemm_upper", 0)),
              nnzC=C.nnz, S=w.max_seeds, nnzR=R.nnz, tr_products=tr_products, nnzS=S.nnz, rounds=it, m=km.m,
              kstats=sg.last_kmer_stats(), direct_seg=bool(sg.tunables().get("kmer_direct_seg", 0)))
    del km, C, S

    # ---- timed region: K steps, per-step events, L2 flushed in between; only the dominant
    # kernel of the breakdown is bracketed by events (the roofline's launch time)
    fam_breakdown = by_family(breakdown)
    dom_name = max(fam_breakdown.items(), key=lambda kv: kv[1][1])[0] if fam_breakdown else None
    clocks = ClockSampler(local)
    sg.prof_reset()
    sg.prof_select(dom_name)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = sg.launch_count()
    sg.memory_reset_peak()
    sg.prof_enable(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    tr_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        km = sg.build_kmer_matrix(seq, off, w.k, w.lo, w.hi)
        C = sg.overlap_spgemm(km, w.min_shared, w.max_seeds)
        tr_ev[i][0].record(stream)
        S, it = sg.transitive_reduce(R, w.fuzz)
        tr_ev[i][1].record(stream)
        ev[i][1].record(stream)
        del km, C, S
    torch.cuda.synchronize()
    sg.prof_enable(False)
    launches = sg.launch_count() - launches0
    mem_peak = sg.memory_stats()[2]
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = [a0.elapsed_time(a1) for a0, a1 in ev]
    tr_ms = [a0.elapsed_time(a1) for a0, a1 in tr_ev]
    total_ms = sum(step_ms)
    prof = by_family(sg.prof_collect())
    total_ms_all, products_all, tr_ms_max, edges_all = combine_ranks(total_ms, products, sum(tr_ms), R.nnz, world)
    value = products_all * args.steps / (total_ms_all / 1e3)

    # ---- roofline of the dominant kernel
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak_src = "measured"
    except Exception:
        peak_src = "fallback"
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    ktot = sum(v[1] for v in breakdown.values()) or 1.0
    roof = None
    if dom_name and dom_name in prof:
        cnt, ms = prof[dom_name]  # over the K timed steps
        ab = algorithmic_bytes(dom_name, sz)  # per step
        ms_step = ms / args.steps
        ach = (ab / (ms_step / 1e3) / 1e9) if ab else None
        abl = (ab * args.steps / cnt) if ab else None
        roof = {"kernel": dom_name, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": (ach / hbm) if ach else None, "traffic": measured_traffic(dom_name, w.name, abl),
                "peak_source": peak_src, "algorithmic_bytes_per_launch": (ab * args.steps / cnt) if ab else None,
                "launch_ms": ms / max(cnt, 1), "launches_per_step": cnt / args.steps,
                "share": fam_breakdown[dom_name][1] / ktot}
    # per-kernel shares from the untimed, fully event-bracketed step
    kernels = {k: {"launches": c, "ms": ms, "share": ms / ktot}
               for k, (c, ms) in sorted(breakdown.items(), key=lambda kv: -kv[1][1])}
    # the same roofline for every kernel family with a byte model, from the breakdown step's
    # event times (the dominant kernel's line above is timed inside the timed region instead)
    rooflines = []
    for f, (c, ms) in sorted(fam_breakdown.items(), key=lambda kv: -kv[1][1]):
        ab = algorithmic_bytes(f, sz)
        if ab and ms > 0:
            ach = ab / (ms / 1e3) / 1e9
            rooflines.append({"kernel": f, "achieved": ach, "frac": ach / hbm, "unit": "GB/s", "ms": ms,
                              "share": ms / ktot})

    # ---- the chain without true coordinates: C -> R from C's seeds -> S (one untimed pass)
    from_seeds = measure_from_seeds(sg, seq, off, w)

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        try:
            e2e = measure_e2e(sg, d, w, args)
        except sg.SgError as ex:  # reported in the line, with the device's memory state
            free_b, total_b = torch.cuda.mem_get_info()
            e2e = {"value": None, "unit": UNIT, "error": str(ex)[:300], "device_free_gb": free_b / 1e9,
                   "device_total_gb": total_b / 1e9, "torch_reserved_gb": torch.cuda.memory_reserved() / 1e9}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": w.name, "reads": n, "bases": total, "k": w.k, "reliable": [w.lo, w.hi],
                       "min_shared": w.min_shared, "max_seeds": w.max_seeds, "fuzz": w.fuzz,
                       "m": sz["m"], "nnz_A": sz["nnzA"], "products": products, "nnz_C": sz["nnzC"],
                       "products_half": sz["products_half"], "spgemm_form": "upper" if sz["upper"] else "rows",
                       "nnz_R": sz["nnzR"], "nnz_S": sz["nnzS"], "tr_rounds": sz["rounds"],
                       "candidates": sz["kstats"]["candidates"],
                       "candidate_sort_bytes": sz["kstats"]["sort_key_bytes"] + sz["kstats"]["sort_val_bytes"],
                       "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"},
            "tr_edges_per_s": edges_all * args.steps / (tr_ms_max / 1e3) if tr_ms_max else None,
            "step_ms_p50": statistics.median(step_ms), "step_ms_max": max(step_ms),
            "e2e": e2e, "roofline": roof, "rooflines": rooflines, "kernels": kernels, "stages": stages,
            "clocks": clk,
            "gpu_launches": launches, "device_memory_peak_gb": mem_peak / 1e9, "from_seeds": from_seeds,
            "tunables_from_cache": tuned_params if tuned else None}
    if w.name != "bacterial-5Mbp-30x" and args.scale == 1.0 and not args.no_forms:
        try:
            line["bacterial"] = measure_extra(sg, "bacterial-5Mbp-30x", args.steps, args.warmup, 1000 * rank)
        except Exception as ex:
            line["bacterial"] = {"error": str(ex)[:300]}
    if not args.no_forms:
        for key, fn in (("batched", lambda: measure_batched(sg, 512, 2e6)),
                        ("served", lambda: measure_served(sg, 10000, 200.0, warmup=1000))):
            try:
                line[key] = fn()
            except Exception as ex:  # reported in the line; the headline stands
                line[key] = {"error": str(ex)[:300]}
    if rank == 0 and not args.no_cpu:
        # a bounded sample: about 15 Mbp of reads (0.1 of the bacterial genome), ~5-10 s of oracle
        # time on one thread; beside it the same oracle on every host core at once
        cscale = min(1.0, 1.5e7 / (w.G * w.coverage))
        line["cpu_baseline"] = cpu_baseline(w, scale=cscale)
        try:
            line["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores(w, scale=cscale)
        except Exception as ex:  # reported, not fatal: the one-thread figure stands
            line["cpu_baseline"]["all_cores"] = {"error": str(ex)[:200]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def measure_extra(sg, name: str, steps: int, warmup: int, seed_off: int = 0) -> dict:
    """Another plain workload timed the same way as the headline (inputs resident, L2 flushed,
    CUDA events per step): products/s, ms per step and TR edges/s."""
    import numpy as np
    import torch

    import synth

    w = synth.WORKLOADS[name]
    w = synth.Workload(**{**w.__dict__, "seed": w.seed + seed_off})
    d = synth.make(w)
    seq = torch.from_numpy(d["seq"]).cuda()
    off = torch.from_numpy(d["offsets"]).cuda()
    R = sg.DeviceGraph.from_numpy(d["R"])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        km = sg.build_kmer_matrix(seq, off, w.k, w.lo, w.hi)
        sg.overlap_spgemm(km, w.min_shared, w.max_seeds)
        sg.transitive_reduce(R, w.fuzz)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    products = nnz_c = 0
    for i in range(steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        km = sg.build_kmer_matrix(seq, off, w.k, w.lo, w.hi)
        C = sg.overlap_spgemm(km, w.min_shared, w.max_seeds)
        ev[i][1].record(stream)
        S, it = sg.transitive_reduce(R, w.fuzz)
        ev[i][2].record(stream)
        if i == 0:
            a = np.diff(km.At.to_numpy()["row_ptr"]).astype(np.int64)
            products, nnz_c = int((a * a).sum()), C.nnz
        del km, C, S
    torch.cuda.synchronize()
    step = [e[0].elapsed_time(e[2]) for e in ev]
    tr = [e[1].elapsed_time(e[2]) for e in ev]
    return {"workload": w.name, "steps": steps, "warmup": warmup, "ms_per_step": sum(step) / steps,
            "value": products * steps / (sum(step) / 1e3), "unit": UNIT, "products": products, "nnz_C": nnz_c,
            "nnz_R": R.nnz, "tr_edges_per_s": R.nnz * steps / (sum(tr) / 1e3),
            "l2": "flushed between steps (256 MB write)"}


def measure_e2e(sg, d, w, args):
    """Products/s through sg_pipeline_host: pinned host inputs in, C and S out, every step."""
    import ctypes

    import numpy as np
    import torch

    L = sg.lib()
    pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in
           dict(seq=d["seq"], off=d["offsets"], rp=d["R"]["row_ptr"], col=d["R"]["col"],
                suf=d["R"]["suffix"].view(np.int32), dir=d["R"]["dir"]).items()}
    job = sg.PipelineJob.make(pin["seq"].data_ptr(), pin["off"].data_ptr(), int(d["offsets"].size - 1),
                              int(d["seq"].size), w, pin["rp"].data_ptr(), pin["col"].data_ptr(),
                              pin["suf"].data_ptr(), pin["dir"].data_ptr(), int(d["R"]["col"].size))
    arena = ctypes.c_void_p()
    sg._check(L.sg_host_arena_create(ctypes.byref(arena)), "host_arena_create")
    res = sg.PipelineResult()
    stream = torch.cuda.current_stream()
    st = ctypes.c_void_p(stream.cuda_stream)
    try:
        for _ in range(max(args.warmup, 1)):
            sg._check(L.sg_pipeline_host(ctypes.byref(job), arena, ctypes.byref(res), st), "pipeline_host")
        times = []
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sg._check(L.sg_pipeline_host(ctypes.byref(job), arena, ctypes.byref(res), st), "pipeline_host")
            times.append(time.perf_counter() - t0)
        h2d = sum(int(t.numel() * t.element_size()) for t in pin.values())
        nrow = int(d["offsets"].size)  # n + 1 row pointers for C and for S
        d2h = 8 * nrow * 2 + res.nnz_c * (8 + 8 * res.max_seeds) + res.nnz_s * 9 + 8
        return {"value": float(res.products) * args.steps / sum(times), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * sum(times) / args.steps,
                "step_ms_min": 1e3 * min(times), "step_ms_max": 1e3 * max(times),
                "nnz_C": int(res.nnz_c), "nnz_S": int(res.nnz_s)}
    finally:
        L.sg_host_arena_destroy(arena)


def measure_batched(sg, count: int, g_hi: float, reps: int = 3) -> dict:
    """The batched workload's sets run as one sg_run_batch vs one plain call sequence per set, on
    the same GPU (device-resident inputs, CUDA events around each variant)."""
    import numpy as np
    import torch

    import synth

    t_gen = time.perf_counter()
    sets = synth.batched_sets(count, 20e3, g_hi)
    t_gen = time.perf_counter() - t_gen
    sg.memory_reset_peak()
    items = [dict(seq=torch.from_numpy(x["seq"]).cuda(), offsets=torch.from_numpy(x["offsets"]).cuda(),
                  lo=x["lo"], hi=x["hi"], R=sg.DeviceGraph.from_numpy(x["R"])) for x in sets]

    def plain():
        for it in items:
            km = sg.build_kmer_matrix(it["seq"], it["offsets"], 17, it["lo"], it["hi"])
            sg.overlap_spgemm(km, 2, 2)
            sg.transitive_reduce(it["R"], 1000)

    from paper_2010_10055_gb300 import autotune
    saved = sg.tunables()

    def batched():
        return sg.run_batch(items, k=17, min_shared=2, max_seeds=2, fuzz=1000)

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(f):
        f()  # warm-up
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            e0.record()
            out = f()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
            del out
        return statistics.median(ts)

    plain_ms = timed(plain)
    tuned = autotune.load(autotune.DEFAULT_CACHE, f"batched-{count}")  # this GPU's cached choice, if any
    try:
        batched_ms = timed(batched)
        res = batched()
    finally:
        for k, v in saved.items():
            sg.tune(k, v)
    a = np.diff(res.to_numpy()["At"]["row_ptr"]).astype(np.int64)
    prod = int((a * a).sum())
    return {"sets": count, "genome_bp": [20000, int(g_hi)], "bases": int(sum(x["seq"].size for x in sets)),
            "generation_s": t_gen, "device_memory_peak_gb": sg.memory_stats()[2] / 1e9,
            "tunables_from_cache": bool(tuned),
            "products": prod, "plain_ms": plain_ms, "batched_ms": batched_ms, "speedup": plain_ms / batched_ms,
            "products_per_s_batched": prod / (batched_ms / 1e3), "products_per_s_plain": prod / (plain_ms / 1e3)}


def measure_served(sg, n_jobs: int, rate: float, warmup: int = 0) -> dict:
    """The served workload: a Poisson stream of warmup + n_jobs requests into the continuous-
    batching server; p50 / p99 of submit -> result-on-host latency and jobs/s over the n_jobs after
    the warm-up ones, beside one-at-a-time plain calls through sg_pipeline_host (host buffers in
    and out) and the server fed the same n_jobs all at once."""
    import numpy as np

    import synth

    t_gen = time.perf_counter()
    stream = synth.served_jobs(warmup + n_jobs, rate)
    t_gen = time.perf_counter() - t_gen
    jobs = stream[warmup:]
    srv = sg.Server(hbm_budget=150 << 30, max_batch=64, workers=2, fuzz=1000)
    try:
        for j in stream[:min(16, len(stream))]:  # first kernels, pools and streams of the server
            srv.wait(srv.submit(j["seq"], j["offsets"], j["lo"], j["hi"], j["R"]))

        def run(js, arrivals, measured_from):
            t0 = time.perf_counter()
            tickets = []
            for j, at in zip(js, arrivals):
                d = t0 + at - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                tickets.append(srv.submit(j["seq"], j["offsets"], j["lo"], j["hi"], j["R"]))
            res = [srv.wait(t) for t in tickets]
            bad = [r["error"] for r in res if r["status"] != sg.SG_OK]
            assert not bad, bad[:3]
            res = res[measured_from:]
            lat = np.array([r["t_done"] - r["t_submit"] for r in res]) * 1e3
            span = max(r["t_done"] for r in res) - min(r["t_submit"] for r in res)
            return lat, span, float(np.mean([r["batch_size"] for r in res]))

        lat, span, mb = run(stream, [j["arrival"] for j in stream], warmup)
        lat_b, span_b, mb_b = run(jobs, [0.0] * len(jobs), 0)
    finally:
        srv.close()
    hp = sg.HostPipeline()
    t0 = time.perf_counter()
    for j in jobs:
        hp.run(j["seq"], j["offsets"], synth.Workload("job", 0, 0, 0, 0, 0, 0, 0, lo=2, hi=20, fuzz=1000), j["R"])
    plain_s = time.perf_counter() - t0
    hp.close()
    bases = np.array([j["seq"].size for j in jobs], np.float64)
    return {"jobs": n_jobs, "warmup_jobs": warmup, "rate_per_s": rate,
            "genome": "Pareto(1.5) from 20 kbp, max 20 Mbp, 30x", "mean_bases": float(bases.mean()),
            "max_bases": float(bases.max()), "generation_s": t_gen,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "jobs_per_s": n_jobs / span, "mean_batch": mb,
            "saturated": {"jobs_per_s": n_jobs / span_b, "p50_ms": float(np.percentile(lat_b, 50)),
                          "p99_ms": float(np.percentile(lat_b, 99)), "mean_batch": mb_b},
            "plain_one_at_a_time_jobs_per_s": n_jobs / plain_s}


def measure_from_seeds(sg, seq, off, w) -> dict:
    """reads -> A -> C -> R estimated from C's seeds -> S: the overlap graph comes from the seeds
    instead of true coordinates (min_overlap as the coordinate-built R). CUDA-event times of the
    graph estimate and of the reduction on it, after one warm-up (none where C holds more than
    5e7 entries: there the estimate keeps hundreds of millions of edges and one reduction takes
    seconds)."""
    import torch

    km = sg.build_kmer_matrix(seq, off, w.k, w.lo, w.hi)
    C = sg.overlap_spgemm(km, w.min_shared, w.max_seeds)
    del km
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for rep in range(2 if C.nnz <= 5e7 else 1):
        ev[0].record()
        R = sg.overlap_graph_from_seeds(C, off, w.k, w.min_overlap)
        ev[1].record()
        S, it = sg.transitive_reduce(R, w.fuzz)
        ev[2].record()
        torch.cuda.synchronize()
    return {"min_overlap": w.min_overlap, "nnz_R": R.nnz, "nnz_S": S.nnz, "tr_rounds": it,
            "graph_ms": ev[0].elapsed_time(ev[1]), "tr_ms": ev[1].elapsed_time(ev[2])}


def _oracle_worker(wdict, scale, seed_off, barrier, out):
    """One host process of the all-cores oracle timing: draws its own sample of the workload
    (seed offset per process), waits for the others, then times the three oracle operations."""
    import numpy as np

    import oracle
    import synth

    w = synth.Workload(**{**wdict, "seed": wdict["seed"] + 7919 * seed_off})
    ws = w.scaled(scale)
    d = synth.make(ws)
    oracle.build()
    barrier.wait()
    t0 = time.perf_counter()
    km = oracle.build_kmer_matrix(d["seq"], d["offsets"], ws.k, ws.lo, ws.hi)
    oracle.overlap_spgemm(km["A"], km["At"], ws.min_shared, ws.max_seeds)
    oracle.transitive_reduce(d["R"], ws.fuzz)
    t1 = time.perf_counter()
    a = np.diff(km["At"]["row_ptr"]).astype(np.int64)
    out.put((int((a * a).sum()), t0, t1))


def cpu_baseline_all_cores(w, scale: float, procs: int | None = None) -> dict:
    """The oracle as it stands, one independent sample per host core, all running at once
    (spawned processes, so no GPU state is inherited): products of all samples / the wall time
    from the common start to the last finish."""
    import multiprocessing as mp

    procs = procs or len(os.sched_getaffinity(0))
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(procs), ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(dict(w.__dict__), scale, r, barrier, out)) for r in range(procs)]
    for p in ps:
        p.start()
    res = [out.get(timeout=900) for _ in ps]
    for p in ps:
        p.join()
    prod = sum(r[0] for r in res)
    wall = max(r[2] for r in res) - min(r[1] for r in res)
    return {"value": prod / wall, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{procs} independent samples of {w.name} at {scale:.3g} of the genome, one process per "
                      f"core, {wall:.1f} s wall for build_kmer_matrix + overlap_spgemm + transitive_reduce"}


def cpu_baseline(w, scale: float):
    """The oracle, as it stands (single host thread), on the same workload shape at `scale` of
    the genome: products/s over the three operations."""
    import numpy as np

    import oracle
    import synth

    ws = w.scaled(scale)
    d = synth.make(ws)
    t0 = time.perf_counter()
    km = oracle.build_kmer_matrix(d["seq"], d["offsets"], ws.k, ws.lo, ws.hi)
    oracle.overlap_spgemm(km["A"], km["At"], ws.min_shared, ws.max_seeds)
    oracle.transitive_reduce(d["R"], ws.fuzz)
    dt = time.perf_counter() - t0
    a = np.diff(km["At"]["row_ptr"]).astype(np.int64)
    prod = int((a * a).sum())
    return {"value": prod / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{w.name} at {scale:.3g} of the genome ({ws.G} bp, {d['offsets'].size - 1} reads), "
                      f"{dt:.1f} s for build_kmer_matrix + overlap_spgemm + transitive_reduce"}


def reference_arm(args, rank, world):
    """The oracle timed on the host cores as the reference arm (rank 0 only)."""
    if rank != 0:
        return
    import numpy as np

    import oracle
    import synth

    w = synth.WORKLOADS[args.workload]
    scale = min(0.04, 6e6 / (w.G * w.coverage))  # about 6 Mbp of reads per step
    ws = w.scaled(scale)
    d = synth.make(ws)

    def one():
        km = oracle.build_kmer_matrix(d["seq"], d["offsets"], ws.k, ws.lo, ws.hi)
        oracle.overlap_spgemm(km["A"], km["At"], ws.min_shared, ws.max_seeds)
        oracle.transitive_reduce(d["R"], ws.fuzz)
        return km

    for _ in range(args.warmup):
        one()
    times = []
    km = None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        km = one()
        times.append(time.perf_counter() - t0)
    a = np.diff(km["At"]["row_ptr"]).astype(np.int64)
    prod = int((a * a).sum())
    value = prod * args.steps / sum(times)
    sample = f"{w.name} at {scale:.3g} of the genome ({ws.G} bp, {d['offsets'].size - 1} reads) per step"
    print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                      "data": "synthetic", "impl": "reference",
                      "config": {"workload": w.name, "parallelism": "host, 1 thread"},
                      "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
                      "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)


if __name__ == "__main__":
    main()
